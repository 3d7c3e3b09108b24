"""Slab decomposition with one halo exchange per pass (the multi-device split the paper names
as future work, arXiv 1802.00438 Sec. 1 and 8), on the CPU: the exchange schedule and the pass
loop of paper_1802_00438_gb300.slab, with the oracle advancing each rank's extended slab (as the
engine's plans do on a device, clamped at the slab's own edges).  The owned rows must equal the
oracle's whole-grid run bit for bit: every cell a rank owns is computed from exact neighbours.
Two processes over gloo run the torch.distributed exchange; one process runs the in-process
copies between slabs."""
import os
import socket
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _slab_mod():
    # slab.py is pure host logic; load it without loading the CUDA library
    import importlib.util
    if "stencil_slab" in sys.modules:
        return sys.modules["stencil_slab"]
    spec = importlib.util.spec_from_file_location(
        "stencil_slab", os.path.join(ROOT, "paper_1802_00438_gb300", "slab.py"))
    m = importlib.util.module_from_spec(spec)
    sys.modules["stencil_slab"] = m
    spec.loader.exec_module(m)
    return m


def _oracle_advance(orc, w, sl):
    p = None if w.power is None else np.ascontiguousarray(w.power[sl.ext_lo:sl.ext_hi])

    def advance(grid, ts):
        grid[...] = orc.run(w.kind, np.asarray(grid), w.coef, ts, p)
    return advance


def test_partition_and_halos():
    S = _slab_mod()
    assert S.partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    sl = S.slabs(100, 4, 8)
    assert [(s.ext_lo, s.ext_hi) for s in sl] == [(0, 33), (17, 58), (42, 83), (67, 100)]
    for a, b in zip(sl, sl[1:]):
        # a's bottom halo is b's first owned rows, b's top halo a's last ones (same sizes)
        assert a.bottom_halo()[1] - a.bottom_halo()[0] == b.send_up()[1] - b.send_up()[0] == 8
        assert b.top_halo()[1] - b.top_halo()[0] == a.send_down()[1] - a.send_down()[0] == 8
        assert a.ext_lo + a.bottom_halo()[0] == b.lo and b.ext_lo + b.send_up()[0] == b.lo
    assert S.passes(19, 8) == [8, 8, 3]
    with pytest.raises(ValueError):
        S.slabs(20, 4, 8)            # 5-row slabs cannot feed an 8-row halo


@pytest.mark.parametrize("kind,ndim,shape,steps,T,parts", [
    (0, 2, (37, 29), 19, 4, 3), (1, 2, (41, 23), 13, 5, 2), (0, 3, (9, 7, 26), 7, 2, 3),
    (1, 3, (8, 6, 21), 6, 3, 2), (1, 2, (40, 17), 0, 4, 2)])
def test_local_slabs_match_oracle(orc, kind, ndim, shape, steps, T, parts):
    S = _slab_mod()
    w = synth.make(kind, ndim, *shape, steps=steps, seed=4100 + 7 * kind + ndim)
    n = w.u0.shape[0]
    sls = S.slabs(n, parts, T)
    grids = [np.ascontiguousarray(w.u0[s.ext_lo:s.ext_hi]).copy() for s in sls]
    adv = [_oracle_advance(orc, w, s) for s in sls]
    S.run_local(sls, grids, steps, T, lambda r, g, ts: adv[r](g, ts))
    got = np.concatenate([g[s.own()[0]:s.own()[1]] for s, g in zip(sls, grids)])
    assert np.array_equal(got, orc.run(kind, w.u0, w.coef, steps, w.power))


def test_without_exchange_the_cut_is_wrong(orc):
    """The exchange matters: skipping it leaves the owned rows next to the cut wrong."""
    S = _slab_mod()
    w = synth.make(0, 2, 31, 30, steps=8, seed=4200)
    sls = S.slabs(30, 2, 4)
    grids = [np.ascontiguousarray(w.u0[s.ext_lo:s.ext_hi]).copy() for s in sls]
    adv = [_oracle_advance(orc, w, s) for s in sls]
    for _ in S.passes(8, 4):
        for r in range(2):
            adv[r](grids[r], 4)
    got = np.concatenate([g[s.own()[0]:s.own()[1]] for s, g in zip(sls, grids)])
    assert not np.array_equal(got, orc.run(0, w.u0, w.coef, 8))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, case):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    S = _slab_mod()
    kind, ndim, shape, steps, T = case
    w = synth.make(kind, ndim, *shape, steps=steps, seed=4300 + kind + ndim)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sl = S.slabs(w.u0.shape[0], world, T)[rank]
    grid = torch.from_numpy(np.ascontiguousarray(w.u0[sl.ext_lo:sl.ext_hi]).copy())
    adv = _oracle_advance(oracle, w, sl)
    S.run_slab(sl, grid, steps, T, lambda g, ts: adv(g.numpy(), ts), S.DistExchange(sl, dist))
    a, b = sl.own()
    np.save(os.path.join(out_dir, f"own{rank}.npy"), grid[a:b].numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", [(1, 2, (45, 31), 21, 8), (0, 3, (7, 6, 20), 9, 4)])
def test_two_ranks_gloo_match_oracle(orc, tmp_path, case):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), case),
                       nprocs=world, join=True, start_method="spawn")
    kind, ndim, shape, steps, T = case
    w = synth.make(kind, ndim, *shape, steps=steps, seed=4300 + kind + ndim)
    got = np.concatenate([np.load(tmp_path / f"own{r}.npy") for r in range(world)])
    assert np.array_equal(got, orc.run(kind, w.u0, w.coef, steps, w.power))
