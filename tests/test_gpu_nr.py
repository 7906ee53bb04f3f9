"""Newton-Raphson, objective and adjoint of libgbpf against the CPU oracle.

Voltages within 1e-8 p.u./rad of the oracle (both run tight); objective
value to 1e-10 relative; objective gradient against central differences of
the oracle's objective; adjoint against the oracle's FP64 adjoint (fresh
factor at the state) to 1e-8 relative, and against central differences
(h = 1e-6 p.u.) of the objective at re-solved power flows, normwise:
max |g_adj - g_fd| <= 1e-6 ||g_fd||inf.  (Componentwise 1e-6 is below the
resolution of FP64 central differences at h = 1e-6 here: the perturbed
solutions sit at the FP64 mismatch floor, so the differences carry about
1e-6 absolute noise whatever the adjoint -- the oracle's own exact adjoint
shows the same spread.)
"""
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


def _grid(case, ncase=1, load_scale=None, outage=None):
    g = gbpf.Grid(case)
    g.set_cases(ncase, load_scale, outage)
    return g


def _nr(g, ncase, precision=gbpf.PF_FP64, tol=1e-11, max_iter=30):
    vm = torch.zeros((ncase, g.nbus), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    st, res = gbpf.pf_run_to_tol(g.ctx, gbpf.run_opts(gbpf.PF_NR, precision, tol=tol,
                                                      max_iter=max_iter), vm, va, ncase)
    return st, res, vm, va


@pytest.mark.parametrize("cfg", [0, 1])
@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
def test_nr_voltages_vs_oracle(oracle, cfg, precision):
    case = gridgen.config(cfg)
    g = _grid(case)
    st, res, vm, va = _nr(g, 1, precision)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    assert res[0]["iters"] <= 10
    rc, vm0, va0, it0, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    assert np.max(np.abs(vm.cpu().numpy()[0] - vm0)) <= 1e-8
    assert np.max(np.abs(va.cpu().numpy()[0] - va0)) <= 1e-8
    g.close()


def test_nr_batched_load_and_outage(oracle):
    base = gridgen.config(0)
    sc = gridgen.scenarios(base, n_load=3, n_outage=3, seed=31)
    g = _grid(base, sc.ncase, sc.load_scale, sc.outage)
    st, res, vm, va = _nr(g, sc.ncase)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    vm, va = vm.cpu().numpy(), va.cpu().numpy()
    for c in range(sc.ncase):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        assert np.max(np.abs(vm[c] - vm0)) <= 1e-8 and np.max(np.abs(va[c] - va0)) <= 1e-8
    g.close()


def test_objective_value_and_gradient(oracle):
    case = gridgen.config(0)
    rng = np.random.default_rng(2)
    vm = rng.uniform(0.95, 1.05, case.n)
    va = rng.uniform(-0.2, 0.2, case.n)
    g = _grid(case)
    vm_d = torch.tensor(vm[None], device=DEV)
    va_d = torch.tensor(va[None], device=DEV)
    J = torch.zeros(1, dtype=torch.float64, device=DEV)
    gva = torch.zeros_like(vm_d)
    gvm = torch.zeros_like(vm_d)
    gbpf.pf_objective(g.ctx, vm_d, va_d, J, gva, gvm)
    torch.cuda.synchronize()
    J0 = oracle.objective(case, vm, va)
    assert abs(J.item() - J0) <= 1e-10 * max(1.0, abs(J0))
    h = 1e-6
    gva, gvm = gva.cpu().numpy()[0], gvm.cpu().numpy()[0]
    for k in range(case.n):
        a1, a2 = va.copy(), va.copy()
        a1[k] += h; a2[k] -= h
        fd = (oracle.objective(case, vm, a1) - oracle.objective(case, vm, a2)) / (2 * h)
        assert abs(gva[k] - fd) <= 1e-6 * max(1.0, abs(fd))
        v1, v2 = vm.copy(), vm.copy()
        v1[k] += h; v2[k] -= h
        fd = (oracle.objective(case, v1, va) - oracle.objective(case, v2, va)) / (2 * h)
        assert abs(gvm[k] - fd) <= 1e-6 * max(1.0, abs(fd))
    g.close()


def _adjoint_at(g, case, vm0, va0, precision):
    vm_d = torch.tensor(vm0[None], device=DEV)
    va_d = torch.tensor(va0[None], device=DEV)
    J = torch.zeros(1, dtype=torch.float64, device=DEV)
    gva = torch.zeros_like(vm_d)
    gvm = torch.zeros_like(vm_d)
    gbpf.pf_objective(g.ctx, vm_d, va_d, J, gva, gvm)
    dP = torch.zeros_like(vm_d)
    dQ = torch.zeros_like(vm_d)
    gbpf.pf_adjoint(g.ctx, precision, vm_d, va_d, gva, gvm, dP, dQ, 1)
    return dP.cpu().numpy()[0], dQ.cpu().numpy()[0], J.item()


@pytest.mark.parametrize("cfg", [0, 3])
@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
def test_adjoint_vs_oracle_adjoint(oracle, cfg, precision):
    """The forward factors come from the last Newton step (an earlier state);
    the refined transposed solve reaches the oracle's exact FP64 adjoint."""
    case = gridgen.config(cfg)
    g = _grid(case)
    st, res, vm, va = _nr(g, 1, precision, tol=1e-11)
    assert st == gbpf.PF_OK
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    dP0, dQ0, J0 = oracle.adjoint(case, vm0, va0)
    dP, dQ, J = _adjoint_at(g, case, vm0, va0, precision)
    scale = max(np.max(np.abs(dP0)), np.max(np.abs(dQ0)))
    assert abs(J - J0) <= 1e-10 * max(1.0, abs(J0))
    assert np.max(np.abs(dP - dP0)) <= 1e-8 * scale
    assert np.max(np.abs(dQ - dQ0)) <= 1e-8 * scale
    pv = case.btype == gridgen.PV
    assert np.all(dQ[pv] == 0.0) and dP[0] == 0.0 and dQ[0] == 0.0
    g.close()


def test_adjoint_vs_central_differences_20k(oracle):
    """64 seeded coordinates of the 20,000-bus grid, h = 1e-6 p.u., each side
    re-solved by the oracle's Newton-Raphson to 1e-13 p.u."""
    case = gridgen.config(3)
    g = _grid(case)
    st, res, vm, va = _nr(g, 1, gbpf.PF_FP32, tol=1e-11)
    assert st == gbpf.PF_OK
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-13, max_iter=30)
    assert rc == oracle.OK
    dP, dQ, _ = _adjoint_at(g, case, vm0, va0, gbpf.PF_FP32)
    rng = np.random.default_rng(1811)
    nons = np.nonzero(case.btype != gridgen.SLACK)[0]
    pq = np.nonzero(case.btype == gridgen.PQ)[0]
    picks = [("P", int(i)) for i in rng.choice(nons, 32, replace=False)] + \
            [("Q", int(i)) for i in rng.choice(pq, 32, replace=False)]
    h = 1e-6
    fds, ads = [], []
    for kind, i in picks:
        vals = []
        for sgn in (1, -1):
            c = case.copy()
            if kind == "P":
                c.pd[i] -= sgn * h
            else:
                c.qd[i] -= sgn * h
            rc2, vm2, va2, _, _ = oracle.power_flow(c, oracle.NR, tol=1e-13, max_iter=30,
                                                    vm0=vm0, va0=va0)
            assert rc2 == oracle.OK
            vals.append(oracle.objective(c, vm2, va2))
        fds.append((vals[0] - vals[1]) / (2 * h))
        ads.append(dP[i] if kind == "P" else dQ[i])
    fds, ads = np.array(fds), np.array(ads)
    err = np.max(np.abs(ads - fds)) / np.max(np.abs(fds))
    assert err <= 1e-6, float(err)
    g.close()


def test_autograd_chain(oracle):
    """loss = Objective(PowerFlow(Psp, Qsp)); loss.backward() gives dJ/dPsp,
    dJ/dQsp equal to the oracle's adjoint."""
    case = gridgen.config(0)
    g = _grid(case)
    psp = torch.tensor((case.pg - case.pd)[None], device=DEV, requires_grad=True)
    qsp = torch.tensor((-case.qd)[None], device=DEV, requires_grad=True)
    vm, va = gbpf.PowerFlowFn.apply(g, psp, qsp, gbpf.PF_FP64, 1e-11)
    loss = gbpf.ObjectiveFn.apply(g, vm, va).sum()
    loss.backward()
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12)
    dP0, dQ0, J0 = oracle.adjoint(case, vm0, va0)
    scale = max(np.max(np.abs(dP0)), np.max(np.abs(dQ0)))
    assert abs(loss.item() - J0) <= 1e-9 * max(1.0, abs(J0))
    assert np.max(np.abs(psp.grad.cpu().numpy()[0] - dP0)) <= 1e-7 * scale
    assert np.max(np.abs(qsp.grad.cpu().numpy()[0] - dQ0)) <= 1e-7 * scale
    g.close()
