"""CUDA-graph replay of repeated pf_run_to_tol calls (pf_set_graphs).

The second identical call captures the run's device work into a graph and
later calls launch it.  Every kernel is deterministic (fixed orders of
operations), so replayed runs must give bit-identical results to direct
ones; the factor's dependency flags use a reserved epoch inside the graph,
so direct factorisations and solves between replays must stay correct."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1811_02512_gb300 import gbpf, gridgen  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02512_gb300 import build
    build.build()
    gbpf.load()


def _launches(g):
    return sum(gbpf.pf_get_profile(g.ctx, k)[0] for k in range(len(gbpf.KERNEL_KINDS)))


@pytest.mark.parametrize("engine,ncase,prec", [(gbpf.PF_ENGINE_BLOCK, 6, gbpf.PF_FP32),
                                               (gbpf.PF_ENGINE_BLOCK, 6, gbpf.PF_FP64),
                                               (gbpf.PF_ENGINE_CLUSTER, 1, gbpf.PF_FP64)])
def test_graph_replays_match_direct_runs(oracle, engine, ncase, prec):
    base = gridgen.config(1)
    g = gbpf.Grid(base)
    if ncase > 1:
        sc = gridgen.scenarios(base, n_load=3, n_outage=3, seed=77)
        g.set_cases(sc.ncase, sc.load_scale, sc.outage)
        gbpf.pf_set_tuning(g.ctx, engine=engine, cluster=1, factor=1, tail=1, outage=2)
    else:
        g.set_cases(1)
        gbpf.pf_set_tuning(g.ctx, engine=engine, factor=1, tail=1)
    vm = torch.zeros((ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=1e-10, max_iter=300)
    gbpf.pf_set_graphs(g.ctx, False)
    st, res0 = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    ref = (vm.clone(), va.clone())
    gbpf.pf_set_graphs(g.ctx, True)
    counts = []
    for k in range(4):  # direct, capture + launch, replay, replay
        vm.zero_()
        va.zero_()
        before = _launches(g)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
        assert st == gbpf.PF_OK, (k, gbpf.pf_last_error(g.ctx))
        counts.append(_launches(g) - before)
        assert torch.equal(vm, ref[0]) and torch.equal(va, ref[1]), k
        assert np.array_equal(res["iters"], res0["iters"])
    assert counts[0] > 0 and counts[1] == counts[2] == counts[3] == counts[0]
    # a direct factorisation and solve between replays (the flags' epochs)
    name = "bp"
    an, Lx0, d0, _ = oracle.factor_bmatrix(base, name)
    n = an["buses"].shape[0]
    gbpf.pf_factor(g.ctx, gbpf.PF_MAT_BP, gbpf.PF_FP64)
    rhs = torch.ones((1, n), dtype=torch.float64, device=DEV)
    gbpf.pf_solve(g.ctx, gbpf.PF_MAT_BP, gbpf.PF_FP64, rhs, 1)
    torch.cuda.synchronize()
    xs = oracle.lu_solve(n, an["Lp"], an["Li"], Lx0, Lx0 * d0[np.repeat(np.arange(n), np.diff(an["Lp"]))],
                         d0, np.ones(n))
    x_ref = np.empty(n)
    x_ref[an["perm"]] = xs
    assert np.max(np.abs(rhs.cpu().numpy()[0] - x_ref)) <= 1e-11 * np.max(np.abs(x_ref))
    vm.zero_()
    va.zero_()
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)  # a replay again
    assert st == gbpf.PF_OK
    assert torch.equal(vm, ref[0]) and torch.equal(va, ref[1])
    g.close()


def test_new_loads_on_the_same_cases_reuse_the_batch(oracle):
    """pf_set_cases with the same cases (same count, same outages) and new
    load scales keeps the batch's arrays, factors and CUDA graph and only
    forms the specified injections again: the replayed run solves the new
    loads (against the oracle), and going back to the first loads gives the
    first results bit for bit."""
    base = gridgen.config(0)
    sc = gridgen.scenarios(base, n_load=2, n_outage=2, seed=5)
    loads_b = sc.load_scale * 1.3
    g = gbpf.Grid(base)
    g.set_cases(sc.ncase, sc.load_scale, sc.outage)
    gbpf.pf_set_graphs(g.ctx, True)
    vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-11, max_iter=300)
    for _ in range(3):  # direct, capture + launch, replay
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
        assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    first = (vm.clone(), va.clone())
    g.set_cases(sc.ncase, loads_b, sc.outage)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    v, a = vm.cpu().numpy(), va.cpu().numpy()
    for c in range(sc.ncase):
        cc = base.copy()
        cc.pd = cc.pd * loads_b[c]
        cc.qd = cc.qd * loads_b[c]
        if sc.outage[c] >= 0:
            cc.status = cc.status.copy()
            cc.status[sc.outage[c]] = 0
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        assert np.max(np.abs(v[c] - vm0)) <= 1e-8 and np.max(np.abs(a[c] - va0)) <= 1e-8, c
    g.set_cases(sc.ncase, sc.load_scale, sc.outage)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
    assert st == gbpf.PF_OK
    assert torch.equal(vm, first[0]) and torch.equal(va, first[1])
    # non-finite new scales of the same cases are refused on the device and
    # leave the injections as they were
    bad = sc.load_scale.copy()
    bad[sc.ncase - 1, base.n // 2] = np.inf
    with pytest.raises(gbpf.PFError) as e:
        g.set_cases(sc.ncase, bad, sc.outage)
    assert e.value.status == gbpf.PF_ERR_ARG
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
    assert st == gbpf.PF_OK
    assert torch.equal(vm, first[0]) and torch.equal(va, first[1])
    g.close()


def test_new_scales_of_a_large_batch_are_checked_on_the_device():
    """New load scales for the same cases of a batch with more than 2^20 of
    them (128 cases of the 10k grid) are checked by a device kernel: a NaN is
    refused with PF_ERR_ARG and leaves the injections (and so the solution)
    as they were; finite scales are taken."""
    base = gridgen.config(1)
    ncase = 128
    rng = np.random.default_rng(8)
    loads = 1.0 + 0.05 * rng.standard_normal((ncase, base.n))
    g = gbpf.Grid(base)
    g.set_cases(ncase, loads)
    vm = torch.zeros((ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-9, max_iter=300)
    for _ in range(2):
        st, _ = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
        assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    first = (vm.clone(), va.clone())
    g.set_cases(ncase, loads * 1.01)
    st, _ = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
    assert st == gbpf.PF_OK
    assert not torch.equal(va, first[1])
    bad = loads.copy()
    bad[ncase // 2, 7] = np.nan
    with pytest.raises(gbpf.PFError) as e:
        g.set_cases(ncase, bad)
    assert e.value.status == gbpf.PF_ERR_ARG
    g.set_cases(ncase, loads)
    st, _ = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
    assert st == gbpf.PF_OK
    assert torch.equal(vm, first[0]) and torch.equal(va, first[1])
    g.close()
