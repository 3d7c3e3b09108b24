"""The performance model against the paper's own printed estimates (Table 4, Sec. 4 Eqs. 3-9),
and the GPU restatement's basic properties.  Host only."""
import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table4_model.json")


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__._engine_build_module().build()
    import paper_1802_00438_gb300 as st
    return st


def _fpga(st, row, th_max):
    kernel, ndim, nread, dev, bsize, vec, ptime, dim, est, fmax = row
    return st.stencil_model_fpga(ndim=ndim, dim_x=dim, dim_y=dim, dim_z=dim, bsize_x=bsize,
                                 bsize_y=bsize, rad=1, par_vec=vec, par_time=ptime, size_cell=4,
                                 num_read=nread, num_write=1, iter=1000, fmax_hz=fmax * 1e6,
                                 th_max_gbs=th_max[dev])


def test_table4_estimates(st):
    g = json.load(open(GOLDEN))
    exact = capped = 0
    for row in g["rows"]:
        r = _fpga(st, row, g["th_max"])
        est = row[8]
        rel = abs(r["throughput_gbs"] - est) / est
        if r["th_mem_gbs"] < g["th_max"][row[3]]:
            # memory throughput below the cap: Eqs. 3-9 reproduce the printed value
            assert rel < 5e-4, (row, r["throughput_gbs"])
            exact += 1
        else:
            # capped rows: the paper's cap is slightly above the nominal Table 3 figure
            assert rel < 2e-3, (row, r["throughput_gbs"])
            capped += 1
    assert exact >= 12 and exact + capped == len(g["rows"])


def test_worked_example_diffusion2d_a10(st):
    # Table 4, Diffusion 2D, Arria 10, bsize 4096, par_vec 8, par_time 36, dim 16096
    r = st.stencil_model_fpga(ndim=2, dim_x=16096, dim_y=16096, dim_z=1, bsize_x=4096, bsize_y=0,
                              rad=1, par_vec=8, par_time=36, size_cell=4, num_read=1,
                              num_write=1, iter=1000, fmax_hz=343.76e6, th_max_gbs=34.1)
    assert r["csize_x"] == 4096 - 72 and r["bnum_x"] == 4
    assert r["th_mem_gbs"] == pytest.approx(343.76e6 * 8 * 4 * 2 / 1e9)
    assert r["throughput_gbs"] == pytest.approx(780.500, abs=5e-3)


def test_model_invalid(st):
    with pytest.raises(st.StencilError):
        st.stencil_model_fpga(ndim=2, dim_x=100, dim_y=100, dim_z=1, bsize_x=8, bsize_y=0, rad=1,
                              par_vec=1, par_time=4, size_cell=4, num_read=1, num_write=1,
                              iter=10, fmax_hz=1e8, th_max_gbs=10)   # block no wider than halos


def _gpu(st, **kw):
    base = dict(ndim=2, nx=16384, ny=16384, nz=1, steps=1000, T=8, bx=128, by=0, halo_x=8,
                halo_y=0, sms=152, sm_hz=2.07e9, hbm_gbs=6789.6, bytes_per_cell=12,
                ops_per_cell=12.5, issue_eff=0.8, hbm_eff=0.9, stream_overhead=0.05,
                launch_s=3e-6)
    base.update(kw)
    return st.stencil_model_gpu(**base)


def test_gpu_model_properties(st):
    r = _gpu(st)
    assert r["passes"] == 125
    assert r["bytes_per_pass"] == 12 * 16384 * 16384
    # HBM time of a pass does not depend on T; issue time grows with it
    r16 = _gpu(st, T=16, halo_x=16)
    assert r16["t_hbm_s"] == pytest.approx(r["t_hbm_s"])
    assert r16["t_alu_s"] > 1.9 * r["t_alu_s"]
    # with free compute the run is HBM-bound: gcells = BW * eff * T / bytes
    rf = _gpu(st, ops_per_cell=1e-9, launch_s=0.0)
    assert rf["gcells"] == pytest.approx(6789.6 * 0.9 * 8 / 12, rel=1e-9)
    # wider halos waste more compute
    assert _gpu(st, halo_x=12)["t_alu_s"] > r["t_alu_s"]
