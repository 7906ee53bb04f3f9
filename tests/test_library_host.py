"""Host-side checks of libgbpf that need no GPU: the library loads and exports
every entry point of include/gbpf.h, input validation, and the symbolic
analysis (ordering, fill, elimination tree, levels) bit-exact against the
oracle's independent implementation."""
import ctypes as C

import numpy as np
import pytest

from paper_1811_02512_gb300 import gbpf, gridgen


@pytest.fixture(scope="module")
def lib():
    from paper_1811_02512_gb300 import build
    build.build()
    return gbpf.load()


def test_exports_every_header_symbol(lib):
    names = gbpf.header_functions()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(lib, nm), nm
        assert C.cast(getattr(lib, nm), C.c_void_p).value


def _tables(case):
    return case.bus_table(), case.branch_table()


def test_create_rejects_bad_tables(lib):
    case = gridgen.config_raw(0)
    bus, br = _tables(case)
    bad = br.copy(); bad["to"][3] = case.n + 5
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(bus, bad)
    assert e.value.status == gbpf.PF_ERR_ARG
    bad = br.copy(); bad["x"][0] = np.nan
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(bus, bad)
    assert e.value.status == gbpf.PF_ERR_ARG
    b2 = bus.copy(); b2["type"][5] = gridgen.SLACK
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(b2, br)
    assert e.value.status == gbpf.PF_ERR_ARG
    # island: take every branch of one leaf bus out of service
    deg = np.bincount(np.concatenate([case.f, case.t]), minlength=case.n)
    leaf = int(np.nonzero(deg == 1)[0][0])
    bad = br.copy(); bad["status"][(case.f == leaf) | (case.t == leaf)] = 0
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(bus, bad)
    assert e.value.status == gbpf.PF_ERR_ISLAND


@pytest.mark.parametrize("cfg", [0, 1, 3])
def test_symbolic_bit_exact_vs_oracle(lib, oracle, cfg):
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        ref = oracle.analyze(case, name)
        got = g.symbolic(which)
        assert g.info.n[which] == ref["buses"].shape[0]
        assert np.array_equal(got["perm"], ref["perm"])
        assert np.array_equal(got["Lp"], ref["Lp"])
        assert np.array_equal(got["Li"], ref["Li"])
        assert np.array_equal(got["parent"], ref["parent"])
        assert np.array_equal(got["level"], ref["level"])
        assert g.info.nlevels[which] == ref["nlevels"]
    g.close()


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_small_random_grids(lib, oracle, seed):
    case = gridgen.small_raw(8 + 7 * seed, 300 + seed)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        ref = oracle.analyze(case, name, literal=True)
        got = g.symbolic(which)
        for k in ("perm", "Lp", "Li", "parent", "level"):
            assert np.array_equal(got[k], ref[k]), k
    g.close()


def test_outage_keeps_pattern(lib):
    case = gridgen.config_raw(0)
    c2 = case.copy()
    c2.status[7] = 0
    a, b = gbpf.Grid(case), gbpf.Grid(c2)
    for w in (0, 1):
        sa, sb = a.symbolic(w), b.symbolic(w)
        assert np.array_equal(sa["Li"], sb["Li"]) and np.array_equal(sa["perm"], sb["perm"])
    a.close(); b.close()


def test_device_calls_fail_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = gbpf.Grid(gridgen.config_raw(0))
    with pytest.raises(gbpf.PFError) as e:
        g.set_cases(1)
    assert e.value.status in (gbpf.PF_ERR_CUDA, gbpf.PF_ERR_OOM)
    g.close()


def test_tuning_fields_validated(lib):
    case = gridgen.config_raw(0)
    ctx = gbpf.pf_create(*_tables(case))
    gbpf.pf_analyze(ctx)
    assert gbpf.pf_get_tuning(ctx) == {"engine": 0, "cluster": 0, "factor": 0, "tail": 0, "outage": 0,
                                       "ms": 0.0}
    gbpf.pf_set_tuning(ctx, engine=gbpf.PF_ENGINE_LANES, cluster=8, factor=1, tail=2, outage=2)
    t = gbpf.pf_get_tuning(ctx)
    assert (t["engine"], t["cluster"], t["factor"], t["tail"], t["outage"]) == (gbpf.PF_ENGINE_LANES, 8, 1, 2, 2)
    for bad in ({"cluster": 3}, {"factor": 3}, {"tail": -1}, {"engine": 7}, {"outage": 3}):
        with pytest.raises(gbpf.PFError) as e:
            gbpf.pf_set_tuning(ctx, **bad)
        assert e.value.status == gbpf.PF_ERR_ARG
    gbpf.pf_destroy(ctx)


def test_pack_create_validates(lib):
    case = gridgen.config_raw(0)
    ctx = gbpf.pf_create(*_tables(case))
    arr = (C.c_void_p * 2)(ctx, ctx)
    h = C.c_void_p()
    assert lib.pf_pack_create(arr, 2, C.byref(h)) == gbpf.PF_ERR_STATE  # not analysed
    gbpf.pf_analyze(ctx)
    assert lib.pf_pack_create(arr, 2, C.byref(h)) == gbpf.PF_ERR_ARG  # repeated
    assert lib.pf_pack_create(arr, 0, C.byref(h)) == gbpf.PF_ERR_ARG
    assert lib.pf_pack_create(arr, 1, C.byref(h)) == gbpf.PF_OK
    lib.pf_pack_destroy(h)
    gbpf.pf_destroy(ctx)
