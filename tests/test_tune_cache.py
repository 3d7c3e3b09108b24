"""Host-side checks of the tuning cache (Sec. 5.3's measured choice among the model's
candidates, remembered per problem): file round trip, rejection of malformed files without
side effects, and argument checks of stencil_tune that return before any device work."""
import ctypes

import pytest


@pytest.fixture()
def st():
    import paper_1802_00438_gb300 as st
    st.stencil_tune_cache_clear()
    yield st
    st.stencil_tune_cache_clear()


# kind ndim nx ny nz storage exact rad | T bx by vec partial_rows resident | GCell/s
ENTRIES = ["1 2 16384 16384 1 0 0 0 8 0 0 8 1 -1 2465.2",
           "0 3 512 512 512 0 0 0 3 64 64 8 0 0 921",
           "0 2 1000 700 1 0 1 0 4 512 0 4 0 -1 310.5",
           "0 2 4096 4096 1 0 0 2 4 0 0 0 0 -1 958",
           "0 2 1024 1024 1 0 0 0 8 0 0 4 0 1 1500"]


def test_round_trip(st, tmp_path):
    src = tmp_path / "a.txt"
    src.write_text("\n".join(ENTRIES) + "\n\n")
    st.stencil_tune_cache_load(str(src))
    assert st.stencil_tune_cache_size() == len(ENTRIES)
    out = tmp_path / "b.txt"
    st.stencil_tune_cache_save(str(out))
    assert sorted(out.read_text().split("\n")[:-1]) == sorted(ENTRIES)
    # loading again replaces equal keys instead of adding entries
    st.stencil_tune_cache_load(str(out))
    assert st.stencil_tune_cache_size() == len(ENTRIES)
    st.stencil_tune_cache_clear()
    assert st.stencil_tune_cache_size() == 0


@pytest.mark.parametrize("bad", ["1 2 16384 16384 1 0 0 0 8 0 0 8 1 -1",          # a field short
                                 "1 2 16384 16384 1 0 0 0 8 0 0 8 1 -1 2465 7",    # a field more
                                 "1 2 16384 16384 1 0 0 0 8 0 1 8 2465.2",         # old format
                                 "5 2 64 64 1 0 0 0 4 0 0 4 0 0 1.0",              # bad kind
                                 "0 2 64 64 3 0 0 0 4 0 0 4 0 0 1.0",              # 2D with nz > 1
                                 "0 2 64 64 1 0 0 0 0 0 0 4 0 0 1.0",              # T = 0
                                 "0 2 64 64 1 9 0 0 4 0 0 4 0 0 1.0",              # bad storage
                                 "0 2 64 64 1 0 0 0 4 0 0 4 3 0 1.0",              # bad rows
                                 "0 2 64 64 1 0 0 0 4 0 0 4 0 2 1.0",              # bad resident
                                 "x"])
def test_malformed_file_changes_nothing(st, tmp_path, bad):
    good = tmp_path / "g.txt"
    good.write_text(ENTRIES[0] + "\n")
    st.stencil_tune_cache_load(str(good))
    f = tmp_path / "bad.txt"
    f.write_text(ENTRIES[1] + "\n" + bad + "\n")
    with pytest.raises(st.StencilError) as e:
        st.stencil_tune_cache_load(str(f))
    assert e.value.code == st.ST_ERR_INVALID_ARG
    assert st.stencil_tune_cache_size() == 1


def test_missing_file(st, tmp_path):
    with pytest.raises(st.StencilError):
        st.stencil_tune_cache_load(str(tmp_path / "none.txt"))
    assert st.lib.stencil_tune_cache_save(None) == st.ST_ERR_INVALID_ARG


def test_tune_argument_checks(st):
    d = st.stencil_desc(1, 2, 64, 64, 1, 0, 0, 0, 0, 0, 0, 0, None, 0, 0, 0)
    r = st.stencil_tune_result()
    k = (ctypes.c_float * 5)(0.5, 0.1, 0.1, 0.001, 80.0)
    fake = 1 << 40   # never dereferenced: every case below fails its checks first
    call = lambda dd, steps=10, top_k=3, res=ctypes.byref(r): st.lib.stencil_tune(
        ctypes.byref(dd), fake, fake + 4096, fake + 8192, k, steps, top_k, res)
    assert call(d, steps=0) == st.ST_ERR_INVALID_ARG
    assert call(d, top_k=-1) == st.ST_ERR_INVALID_ARG
    assert call(d, res=None) == st.ST_ERR_INVALID_ARG
    forced = st.stencil_desc(1, 2, 64, 64, 1, 0, 8, 0, 0, 0, 0, 0, None, 0)
    assert call(forced) == st.ST_ERR_INVALID_ARG
    for rows, res in ((1, 0), (0, 1), (0, -1)):   # the two named choices are the tuner's too
        named = st.stencil_desc(1, 2, 64, 64, 1, 0, 0, 0, 0, 0, 0, 0, None, 0, rows, res)
        assert call(named) == st.ST_ERR_INVALID_ARG
    assert st.lib.stencil_tune(ctypes.byref(d), fake, fake, None, k, 10, 3, ctypes.byref(r)) == \
        st.ST_ERR_INVALID_ARG   # in place: the timed runs would overwrite the input
    assert st.lib.stencil_tune(None, fake, fake, None, k, 10, 3, ctypes.byref(r)) == st.ST_ERR_INVALID_ARG
    assert st.lib.stencil_plan_tuned(None) == 0
    assert st.stencil_tune_cache_size() == 0
