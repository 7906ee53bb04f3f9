"""Parity at the benchmark's full sizes, in the launch configurations that
bench.py times: the 1,024-case batch of the 10,000-bus grid (512 load
scenarios and 512 single-branch outages, the same seeded set as the bench)
with one block per case, low-rank outages and the FP32 solves refined in
FP64 to the bench's forcing term, and the single 10,000-bus case on the
cluster engine.  Sampled cases against the oracle's Newton-Raphson solution
run to 1e-12 p.u.

Bounds: a run stopped at the bench's 1e-8 p.u. mismatch defines the state
only to about |J^-1| 1e-8 (measured: at most 5e-9 over all 1,024 cases), so
those runs are held to 1e-7; runs to 1e-11 are held to the suite's 1e-8."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1811_02512_gb300 import gbpf, gridgen  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SAMPLE = (0, 1, 255, 511, 512, 700, 1022, 1023)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02512_gb300 import build
    build.build()
    gbpf.load()


@pytest.fixture(scope="module")
def batch(oracle):
    base = gridgen.config(1)
    sc = gridgen.scenarios(base, n_load=512, n_outage=512)
    refs = {}
    for c in SAMPLE:
        rc, vm0, va0, _, _ = oracle.power_flow(gridgen.apply_scenario(base, sc, c), oracle.NR, tol=1e-12,
                                               max_iter=30)
        assert rc == oracle.OK
        refs[c] = (vm0, va0)
    return base, sc, refs


@pytest.mark.parametrize("precision,threads,tail", [(gbpf.PF_FP32, 512, 1), (gbpf.PF_FP32, 256, 1),
                                                   (gbpf.PF_FP64, 512, 1), (gbpf.PF_FP32, 512, 3),
                                                   (gbpf.PF_FP32, 256, 3), (gbpf.PF_FP64, 512, 3)])
def test_batch10k_full_size_sampled(batch, precision, threads, tail):
    base, sc, refs = batch
    g = gbpf.Grid(base)
    g.set_cases(sc.ncase, sc.load_scale, sc.outage)
    gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_BLOCK, cluster=1, factor=1, tail=tail, outage=2,
                       threads=threads)
    vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    for tol, bound in ((1e-8, 1e-7), (1e-11, 1e-8)):
        vm.zero_()
        va.zero_()
        opts = gbpf.run_opts(gbpf.PF_FDPF, precision, tol=tol, max_iter=300, ir_tol=1e-3)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
        assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
        assert np.all(res["status"] == gbpf.PF_OK) and np.all(res["max_mismatch"] <= tol)
        assert np.all(res["method"] == gbpf.PF_FDPF)
        v, a = vm.cpu().numpy(), va.cpu().numpy()
        for c, (vm0, va0) in refs.items():
            assert np.max(np.abs(v[c] - vm0)) <= bound, (tol, c)
            assert np.max(np.abs(a[c] - va0)) <= bound, (tol, c)
    g.close()


def test_plain10k_full_size_every_bus(oracle):
    base = gridgen.config(1)
    rc, vm0, va0, _, _ = oracle.power_flow(base, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    g = gbpf.Grid(base)
    g.set_cases(1)
    gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_CLUSTER, cluster=0, factor=1, tail=1, outage=1)
    vm = torch.zeros((1, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-8, max_iter=200)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 1)
    assert st == gbpf.PF_OK and res[0]["max_mismatch"] <= 1e-8
    assert np.max(np.abs(vm.cpu().numpy()[0] - vm0)) <= 1e-7
    assert np.max(np.abs(va.cpu().numpy()[0] - va0)) <= 1e-7
    g.close()
