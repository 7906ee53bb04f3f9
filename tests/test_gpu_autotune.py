"""Project autotuner (pf_autotune) and explicit kernel mappings (pf_set_tuning).

Every mapping the tuner may choose -- cluster size of a single case, the
dependency-driven or block-per-instance factor, the scatter, level-by-level
or partitioned-inverse narrow top, the block or lane engine of a batch, the
block size -- must reach the oracle's
solution (1e-8 p.u./rad, both sides run tight); the tuner must return one of
them with a positive time, and leave it set on the context.
"""
import itertools

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


def test_every_single_case_mapping_matches_oracle(oracle):
    case = gridgen.config(1)
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    g = gbpf.Grid(case)
    g.set_cases(1)
    vm = torch.zeros((1, case.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    for prec, cl, fac, tail in itertools.product([gbpf.PF_FP64, gbpf.PF_FP32], [1, 8, 16], [1, 2], [1, 2, 3]):
        gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_BLOCK, cluster=cl, factor=fac, tail=tail)
        opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=1e-11, max_iter=300)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 1)
        assert st == gbpf.PF_OK, (prec, cl, fac, tail, gbpf.pf_last_error(g.ctx))
        assert np.max(np.abs(vm.cpu().numpy()[0] - vm0)) <= 1e-8, (prec, cl, fac, tail)
        assert np.max(np.abs(va.cpu().numpy()[0] - va0)) <= 1e-8, (prec, cl, fac, tail)
    g.close()


def test_autotune_single_and_batch(oracle):
    base = gridgen.config(1)
    g = gbpf.Grid(base)
    g.set_cases(1)
    vm = torch.zeros((1, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-8, max_iter=200)
    t = gbpf.pf_autotune(g.ctx, opts, vm, va, reps=2)
    assert t["ms"] > 0 and t["factor"] in (1, 2) and t["tail"] in (1, 2, 3)
    # the cluster engine's field is its subtree levels per step
    assert t["cluster"] in ((1, 2, 3, 4) if t["engine"] == gbpf.PF_ENGINE_CLUSTER else (1, 8, 16))
    assert t["threads"] == 0  # block sizes are a batch choice
    assert gbpf.pf_get_tuning(g.ctx) == t
    g.close()
    sc = gridgen.scenarios(base, n_load=32, n_outage=32, seed=5)
    g = gbpf.Grid(base)
    g.set_cases(sc.ncase, sc.load_scale, sc.outage)
    vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP32, tol=1e-11, max_iter=300)
    t = gbpf.pf_autotune(g.ctx, opts, vm, va, reps=1)
    assert t["ms"] > 0 and t["engine"] in (gbpf.PF_ENGINE_BLOCK, gbpf.PF_ENGINE_LANES)
    assert t["threads"] in (128, 256, 512) if t["engine"] == gbpf.PF_ENGINE_BLOCK else t["threads"] == 0
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
    assert st == gbpf.PF_OK
    v, a = vm.cpu().numpy(), va.cpu().numpy()
    for c in (0, 31, 32, 63):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        assert np.max(np.abs(v[c] - vm0)) <= 1e-8 and np.max(np.abs(a[c] - va0)) <= 1e-8
    g.close()


@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
def test_low_rank_outages_match_oracle(oracle, precision):
    """Outage cases solved with the base factors and the low-rank (Woodbury)
    correction of every solve reach the oracle's solution of each outaged
    grid, as the per-case factors do."""
    base = gridgen.config(1)
    sc = gridgen.scenarios(base, n_load=2, n_outage=14, seed=9)
    g = gbpf.Grid(base)
    g.set_cases(sc.ncase, sc.load_scale, sc.outage)
    vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, precision, tol=1e-11, max_iter=300)
    out = {}
    # (outage form, tail form): per-case factors; low-rank with the scatter
    # top; low-rank with the top's partitioned inverse (tail form 3); and
    # form 3 asked for with per-case factors, which runs the scatter top
    for outage, tail in ((1, 1), (2, 1), (2, 3), (1, 3)):
        gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_BLOCK, outage=outage, tail=tail)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
        assert st == gbpf.PF_OK, (outage, tail, gbpf.pf_last_error(g.ctx))
        out[outage, tail] = (vm.cpu().numpy().copy(), va.cpu().numpy().copy())
    for c in (0, 2, 7, 15):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        for key in out:
            assert np.max(np.abs(out[key][0][c] - vm0)) <= 1e-8, (key, c)
            assert np.max(np.abs(out[key][1][c] - va0)) <= 1e-8, (key, c)
    g.close()


@pytest.mark.parametrize("cfg,group", [(0, 0), (1, 0), (1, 1), (1, 2), (1, 4)])
def test_cluster_engine_matches_oracle(oracle, cfg, group):
    """The single-case cluster engine (substitutions shared by a 16-block
    cluster, the narrow top of the elimination tree through its explicit
    inverse, the subtree levels `group` at a time through their blocks'
    inverses; 0 = the default): voltages against the oracle's run to a tight
    mismatch, every factor form, twice in a row on the same context (the
    programs stay resident, the inverses are formed again from each
    factorisation)."""
    case = gridgen.config(cfg)
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    g = gbpf.Grid(case)
    g.set_cases(1)
    vm = torch.zeros((1, case.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    for fac, tail in itertools.product([1, 2], [1, 2]):
        gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_CLUSTER, cluster=group, factor=fac, tail=tail)
        for _ in range(2):
            vm.zero_()
            va.zero_()
            opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-11, max_iter=300)
            st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 1)
            assert st == gbpf.PF_OK, (fac, tail, gbpf.pf_last_error(g.ctx))
            assert np.max(np.abs(vm.cpu().numpy()[0] - vm0)) <= 1e-8, (fac, tail)
            assert np.max(np.abs(va.cpu().numpy()[0] - va0)) <= 1e-8, (fac, tail)
    g.close()


@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
@pytest.mark.parametrize("threads", [256, 128])
def test_smaller_case_blocks_match_oracle(oracle, precision, threads):
    """One block per case with 256 or 128 threads (more cases per SM, the
    solve vector in global memory): a batch of load and outage cases of the
    10k grid, both outage forms, against the oracle's solution of each
    sampled case; the run reports the same iteration counts as 512-thread
    blocks give."""
    base = gridgen.config(1)
    sc = gridgen.scenarios(base, n_load=6, n_outage=6, seed=21)
    g = gbpf.Grid(base)
    g.set_cases(sc.ncase, sc.load_scale, sc.outage)
    vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, precision, tol=1e-11, max_iter=300)
    refs = {}
    for c in (0, 5, 6, 11):
        rc, vm0, va0, _, _ = oracle.power_flow(gridgen.apply_scenario(base, sc, c), oracle.NR, tol=1e-12,
                                               max_iter=30)
        assert rc == oracle.OK
        refs[c] = (vm0, va0)
    for outage in (1, 2):
        its = {}
        for th in (512, threads):
            gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_BLOCK, cluster=1, factor=1, tail=1, outage=outage,
                               threads=th)
            vm.zero_()
            va.zero_()
            st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
            assert st == gbpf.PF_OK, (th, outage, gbpf.pf_last_error(g.ctx))
            its[th] = res["iters"].copy()
            v, a = vm.cpu().numpy(), va.cpu().numpy()
            for c, (vm0, va0) in refs.items():
                assert np.max(np.abs(v[c] - vm0)) <= 1e-8, (th, outage, c)
                assert np.max(np.abs(a[c] - va0)) <= 1e-8, (th, outage, c)
        assert np.max(np.abs(its[512] - its[threads])) <= 1
    g.close()
