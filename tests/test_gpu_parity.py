"""GPU parity of libgbpf against the CPU oracle, through the C ABI.

Tolerances:
  * admittance matrix, mismatch: FP64, different summation order only ->
    1e-12 relative to the row scale;
  * FP64 factor and solve: 1e-11 relative (left-looking vs the oracle's
    dense-work-column LU: same operations, different rounding order);
  * FP32 factor: the componentwise backward-error bound of LDL^T without
    pivoting, |P A P^T - L D L^T| <= gamma_{c+1} |L||D||L^T|, u = 2^-24;
  * voltages: |dV| <= 1e-8 p.u., |dtheta| <= 1e-8 rad with both sides run to
    a tight mismatch (the power-flow solution is only defined to
    ||J^-1|| * tol by a tolerance-based stop).
"""
import ctypes as C

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


CASES = {0: lambda: gridgen.config(0), 1: lambda: gridgen.config(1)}


@pytest.mark.parametrize("cfg", [0, 1])
def test_ybus_parity(oracle, cfg):
    case = CASES[cfg]()
    case.gs = np.linspace(0, 0.01, case.n)
    case.bs = np.linspace(-0.02, 0.02, case.n)
    g = _grid(case)
    rp, col, G, B = gbpf.pf_get_ybus(g.ctx, case.n, g.info.nnz_ybus)
    rp0, col0, G0, B0 = oracle.ybus(case)
    assert np.array_equal(rp, rp0) and np.array_equal(col, col0)
    scale = np.repeat(np.maximum(np.abs(G0[rp0[1:] - rp0[1:] + rp0[:-1]]), 1.0), np.diff(rp0))
    assert np.max(np.abs(G - G0)) < 1e-12 * np.max(np.abs(G0))
    assert np.max(np.abs(B - B0)) < 1e-12 * np.max(np.abs(B0))
    g.close()


@pytest.mark.parametrize("cfg", [0, 1])
@pytest.mark.parametrize("which,name", [(gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")])
def test_factor_parity_fp64_fp32(oracle, cfg, which, name):
    case = CASES[cfg]()
    g = _grid(case)
    an, Lx0, d0, _ = oracle.factor_bmatrix(case, name)
    gbpf.pf_factor(g.ctx, which, gbpf.PF_FP64)
    D, Lx, st = gbpf.pf_get_factor(g.ctx, which, gbpf.PF_FP64, 0, g.info)
    assert st == gbpf.PF_OK
    assert np.max(np.abs(D - d0) / np.abs(d0)) < 1e-11
    assert np.max(np.abs(Lx - Lx0)) < 1e-11 * max(1.0, np.max(np.abs(Lx0)))
    gbpf.pf_factor(g.ctx, which, gbpf.PF_FP32)
    D, Lx, st = gbpf.pf_get_factor(g.ctx, which, gbpf.PF_FP32, 0, g.info)
    assert st == gbpf.PF_OK
    # FP32 LDL^T without pivoting is backward stable (componentwise):
    # |P A P^T - L D L^T| <= gamma_{c+1} |L| |D| |L^T|, gamma_k = k u / (1 - k u),
    # u = 2^-24, c = largest column count.  Checked on the sparse product.
    _check_backward_error(an, Lx, D, g.info.max_col[which], *_)
    g.close()


def _check_backward_error(an, Lx, D, max_col, Ap, Ai, Ax):
    import scipy.sparse as sp
    n = an["buses"].shape[0]
    Lp, Li = an["Lp"], an["Li"]
    cols = np.repeat(np.arange(n), np.diff(Lp))
    L = sp.csc_matrix((np.concatenate([np.ones(n), Lx]),
                       (np.concatenate([np.arange(n), Li]), np.concatenate([np.arange(n), cols]))),
                      shape=(n, n))
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    Dm = sp.diags(D)
    R = (A - L @ Dm @ L.T).tocoo()
    M = (abs(L) @ abs(Dm) @ abs(L).T).tocsr()
    u = 2.0 ** -24
    k = max_col + 1
    gamma = k * u / (1 - k * u)
    bound = np.asarray(M[R.row, R.col]).ravel() * gamma
    assert np.all(np.abs(R.data) <= bound + 1e-300), float(np.max(np.abs(R.data) / (bound + 1e-300)))


@pytest.mark.parametrize("cfg", [0, 1])
@pytest.mark.parametrize("which,name", [(gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")])
def test_solve_parity(oracle, cfg, which, name):
    case = CASES[cfg]()
    g = _grid(case, ncase=3)
    an, Lx0, d0, (Ap, Ai, Ax) = oracle.factor_bmatrix(case, name)
    n = an["buses"].shape[0]
    rng = np.random.default_rng(cfg * 10 + which)
    rhs = rng.standard_normal((3, n))
    iperm = np.empty(n, np.int64)
    iperm[an["perm"]] = np.arange(n)
    gbpf.pf_factor(g.ctx, which, gbpf.PF_FP64)
    x_dev = torch.tensor(rhs, dtype=torch.float64, device=DEV)
    gbpf.pf_solve(g.ctx, which, gbpf.PF_FP64, x_dev, 3)
    torch.cuda.synchronize()
    x = x_dev.cpu().numpy()
    for c in range(3):
        # oracle works in step order: x_step = solve(P A P^T, rhs_step)
        xs = oracle.lu_solve(n, an["Lp"], an["Li"], Lx0, Lx0 * d0[np.repeat(np.arange(n), np.diff(an["Lp"]))],
                             d0, rhs[c][an["perm"]])
        ref = np.empty(n)
        ref[an["perm"]] = xs
        assert np.max(np.abs(x[c] - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))
    g.close()


@pytest.mark.parametrize("cfg", [0, 1])
def test_mismatch_parity(oracle, cfg):
    case = CASES[cfg]()
    rng = np.random.default_rng(7)
    g = _grid(case, ncase=2)
    vm = rng.uniform(0.95, 1.05, (2, case.n))
    va = rng.uniform(-0.2, 0.2, (2, case.n))
    vm_d = torch.tensor(vm, device=DEV)
    va_d = torch.tensor(va, device=DEV)
    dp = torch.zeros_like(vm_d)
    dq = torch.zeros_like(vm_d)
    mx = torch.zeros(2, dtype=torch.float64, device=DEV)
    gbpf.pf_mismatch(g.ctx, vm_d, va_d, dp, dq, mx, 2)
    torch.cuda.synchronize()
    rp, col, G, B = oracle.ybus(case)
    for c in range(2):
        dP0, dQ0, m0 = oracle.mismatch(case, rp, col, G, B, vm[c], va[c])
        scale = max(1.0, np.max(np.abs(B)))
        assert np.max(np.abs(dp[c].cpu().numpy() - dP0)) < 1e-12 * scale
        assert np.max(np.abs(dq[c].cpu().numpy() - dQ0)) < 1e-12 * scale
        assert abs(mx[c].item() - m0) < 1e-12 * scale
    g.close()


def _run(g, ncase, precision=gbpf.PF_FP64, tol=1e-8, max_iter=200):
    vm = torch.zeros((ncase, g.nbus), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, precision, tol=tol, max_iter=max_iter)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
    return st, res, vm.cpu().numpy(), va.cpu().numpy()


@pytest.mark.parametrize("cfg", [0, 1])
def test_fdpf_voltages_vs_oracle(oracle, cfg):
    case = CASES[cfg]()
    g = _grid(case)
    st, res, vm, va = _run(g, 1, tol=1e-11, max_iter=300)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    rc, vm0, va0, it0, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    assert np.max(np.abs(vm[0] - vm0)) <= 1e-8
    assert np.max(np.abs(va[0] - va0)) <= 1e-8
    # at the production tolerance the iteration count matches the oracle's FDPF
    st, res, vm, va = _run(g, 1, tol=1e-8)
    rc, _, _, it1, _ = oracle.power_flow(case, oracle.FDPF, tol=1e-8)
    assert st == gbpf.PF_OK and rc == oracle.OK
    assert abs(int(res[0]["iters"]) - it1) <= 1
    assert res[0]["max_mismatch"] <= 1e-8
    g.close()


def test_batched_load_and_outage_cases(oracle):
    base = gridgen.config(0)
    sc = gridgen.scenarios(base, n_load=5, n_outage=5, seed=11)
    g = _grid(base, sc.ncase, sc.load_scale, sc.outage)
    st, res, vm, va = _run(g, sc.ncase, tol=1e-11, max_iter=400)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    for c in range(sc.ncase):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        assert np.max(np.abs(vm[c] - vm0)) <= 1e-8, c
        assert np.max(np.abs(va[c] - va0)) <= 1e-8, c
    g.close()


def test_singular_bpp_reported_not_trapped():
    """A PQ bus whose B'' diagonal is exactly zero (charging cancels the series
    susceptance) gives PF_ERR_SINGULAR from the pivot check."""
    r, x = 0.01, 0.1
    b = 2 * x / (r * r + x * x)
    case = gridgen.Case(name="sing", btype=np.array([3, 1], np.int32), pd=np.array([0, 0.1]),
                        qd=np.array([0, 0.05]), gs=np.zeros(2), bs=np.zeros(2), pg=np.zeros(2),
                        vset=np.ones(2), va=np.zeros(2), f=np.array([0], np.int32),
                        t=np.array([1], np.int32), r=np.array([r]), x=np.array([x]),
                        b=np.array([b]), tap=np.ones(1), status=np.ones(1, np.int32))
    g = _grid(case)
    gbpf.pf_factor(g.ctx, gbpf.PF_MAT_BPP, gbpf.PF_FP64)
    _, _, st = gbpf.pf_get_factor(g.ctx, gbpf.PF_MAT_BPP, gbpf.PF_FP64, 0, g.info)
    assert st == gbpf.PF_ERR_SINGULAR
    st, res, _, _ = _run(g, 1)
    assert st == gbpf.PF_ERR_SINGULAR and res[0]["status"] == gbpf.PF_ERR_SINGULAR
    g.close()


def test_iteration_limit_reported():
    g = _grid(gridgen.config(0))
    st, res, _, _ = _run(g, 1, max_iter=1)
    assert st == gbpf.PF_ERR_NOT_CONVERGED
    assert res[0]["status"] == gbpf.PF_ERR_NOT_CONVERGED and res[0]["iters"] == 2
    g.close()


def _pieces(g, which, lst):
    L = gbpf.load()
    f = L.gbpf_debug_pieces
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]
    cnt = C.c_int(0)
    assert f(g.ctx, which, lst, C.byref(cnt), None, 0) == 0
    out = np.zeros(max(1, 8 * cnt.value), np.int32)
    assert f(g.ctx, which, lst, C.byref(cnt), out.ctypes.data, out.shape[0]) == 0
    return out[:8 * cnt.value].reshape(-1, 8)


def _selftest_sweep(g, which, prec, stall, hold, spin, x_dev):
    L = gbpf.load()
    f = L.gbpf_selftest_sweep
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_void_p, C.c_void_p]
    st = C.c_int(-1)
    rc = f(g.ctx, which, prec, stall, hold, spin, x_dev.data_ptr(), C.byref(st))
    assert rc == 0
    return st.value


@pytest.mark.parametrize("which,name", [(gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")])
def test_sweep_gives_up_together_and_context_survives(oracle, which, name):
    """The substitution sweeps' give-up path, made to happen for certain with
    the ring's self-test hooks: the producer stops issuing at a chosen piece
    (its copies never come, so the consumers' bounded waits run out), or the
    consumers keep one stage (so the producer's bounded wait runs out).  The
    stop points cover the first piece, block-wide pieces, the first piece of
    a single-warp run (the scatter tail) and the backward sweep.  Every such
    solve returns PF_ERR_TIMEOUT instead of hanging; afterwards an ordinary
    solve matches the oracle and a full power flow converges."""
    case = gridgen.config(1)
    g = _grid(case)
    gbpf.pf_factor(g.ctx, which, gbpf.PF_FP64)
    fwd, bwd = _pieces(g, which, 2), _pieces(g, which, 3)
    if fwd.shape[0] == 0:
        fwd, bwd = _pieces(g, which, 0), _pieces(g, which, 1)
    nf, nb = fwd.shape[0], bwd.shape[0]
    run_f = [j for j in range(nf) if 2 <= fwd[j, 4] <= 4]
    run_b = [j for j in range(nb) if 2 <= bwd[j, 4] <= 4]
    assert run_f and run_b and nf > 8 and nb > 8
    stalls = sorted({0, nf // 2, run_f[0], run_f[-1], nf - 1, nf, nf + run_b[0], nf + nb - 1})
    holds = sorted(h for h in {0, run_f[0], nf // 3, nf, nf + run_b[0]} if h + 4 < nf + nb)
    n = g.info.n[which]
    rhs = torch.ones(n, dtype=torch.float64, device=DEV)
    for stall in stalls:
        x = rhs.clone()
        assert _selftest_sweep(g, which, gbpf.PF_FP64, stall, -1, 20000, x) == gbpf.PF_ERR_TIMEOUT, stall
    for hold in holds:
        x = rhs.clone()
        assert _selftest_sweep(g, which, gbpf.PF_FP64, -1, hold, 20000, x) == gbpf.PF_ERR_TIMEOUT, hold
    # the hooks off: the same self-test solve completes and is correct
    x = rhs.clone()
    assert _selftest_sweep(g, which, gbpf.PF_FP64, -1, -1, 1 << 22, x) == gbpf.PF_OK
    an, Lx0, d0, _ = oracle.factor_bmatrix(case, name)
    xs = oracle.lu_solve(n, an["Lp"], an["Li"], Lx0, Lx0 * d0[np.repeat(np.arange(n), np.diff(an["Lp"]))],
                         d0, np.ones(n))
    x_ref = np.empty(n)
    x_ref[an["perm"]] = xs
    assert np.max(np.abs(x.cpu().numpy() - x_ref)) <= 1e-11 * np.max(np.abs(x_ref))
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-11, max_iter=300)
    vm = torch.zeros((1, case.n), dtype=torch.float64, device=DEV)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, torch.zeros_like(vm), 1)
    assert st == gbpf.PF_OK
    g.close()


def test_waits_that_never_complete_give_up():
    """The bounded-wait primitives of the sweeps (mbarrier) and of the
    dependency-driven factor (done flag) on a barrier nothing arrives on and
    a flag nothing sets: both give up after their limit and say so."""
    L = gbpf.load()
    out = (C.c_longlong * 4)()
    assert L.gbpf_selftest_waits(C.c_uint(20000), out) == 0
    assert out[0] == 1 and out[1] == 1
    assert 0 < out[2] < 2_000_000_000 and 0 < out[3] < 2_000_000_000


def test_no_pq_bus_empty_bpp(oracle):
    """Degenerate grid: every non-slack bus is PV, so B'' is empty."""
    case = gridgen.config(0)
    case.btype = np.where(case.btype == gridgen.SLACK, gridgen.SLACK, gridgen.PV).astype(np.int32)
    case.vset = np.where(case.vset == 1.0, 1.01, case.vset)
    case.pg = case.pg - case.pd
    case.pd = np.zeros(case.n)
    case.qd = np.zeros(case.n)
    g = _grid(case)
    assert g.info.n[1] == 0
    st, res, vm, va = _run(g, 1, tol=1e-11, max_iter=300)
    assert st == gbpf.PF_OK
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12)
    assert rc == oracle.OK
    assert np.max(np.abs(va[0] - va0)) <= 1e-8
    g.close()


@pytest.mark.parametrize("cfg", [0, 1])
def test_fp32_factor_with_fp64_refinement(oracle, cfg):
    """FP32 factor and substitution, FP64 mismatch and FP64 refinement of every
    linear solve: voltages reach the FP64 oracle's within 1e-8."""
    case = CASES[cfg]()
    g = _grid(case)
    vm = torch.zeros((1, case.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP32, tol=1e-11, max_iter=300, ir_max=5,
                         ir_tol=1e-10)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 1)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    assert res[0]["ir_steps"] > 0
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert np.max(np.abs(vm.cpu().numpy()[0] - vm0)) <= 1e-8
    assert np.max(np.abs(va.cpu().numpy()[0] - va0)) <= 1e-8
    g.close()


def test_fp32_batched_cases_refined(oracle):
    base = gridgen.config(0)
    sc = gridgen.scenarios(base, n_load=4, n_outage=4, seed=21)
    g = _grid(base, sc.ncase, sc.load_scale, sc.outage)
    st, res, vm, va = _run(g, sc.ncase, precision=gbpf.PF_FP32, tol=1e-11, max_iter=400)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    for c in range(sc.ncase):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert np.max(np.abs(vm[c] - vm0)) <= 1e-8, c
        assert np.max(np.abs(va[c] - va0)) <= 1e-8, c
    g.close()


def test_small_angle_rotation_series_vs_cuda_sincos():
    """The Maclaurin sin/cos used to rotate cached cos/sin by a step agree with
    the CUDA math library's sincos to within 2 ulp on |x| <= 0.2, both in
    full and in the short form that warps of small steps take (|x| <= 1e-3,
    down to 1e-12, both signs), and across the boundary of the two."""
    import ctypes as C
    L = gbpf.load()
    rng = np.random.default_rng(11)
    tiny = 10.0 ** rng.uniform(-12, -3, 65536) * rng.choice([-1.0, 1.0], 65536)
    x = torch.cat([torch.linspace(-0.2, 0.2, 200001, dtype=torch.float64),
                   torch.linspace(-1e-3, 1e-3, 65537, dtype=torch.float64),
                   torch.linspace(0.9e-3, 1.1e-3, 4097, dtype=torch.float64),
                   torch.from_numpy(tiny)]).to(DEV)
    s, c, sr, cr = (torch.empty_like(x) for _ in range(4))
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    assert L.gbpf_selftest_small_sincos(p(x), p(s), p(c), p(sr), p(cr), C.c_int(x.numel())) == 0
    ulp_s = torch.abs(s - sr) / torch.clamp(torch.abs(sr), min=1e-300) / 2.0 ** -52
    ulp_c = torch.abs(c - cr) / torch.abs(cr) / 2.0 ** -52
    nz = torch.abs(x) > 1e-300
    assert ulp_s[nz].max().item() <= 2.0
    assert ulp_c.max().item() <= 2.0


def test_pivot_reciprocal_vs_cuda_division():
    """The factorisations' pivot reciprocal (Newton's iteration from the FP32
    reciprocal) agrees with CUDA's FP64 division 1 / v to within 2 ulp over
    pivots spanning the magnitudes of the admittance matrices and beyond,
    both signs, and falls back to the division outside the FP32 range."""
    import ctypes as C
    L = gbpf.load()
    rng = np.random.default_rng(3)
    mags = 10.0 ** rng.uniform(-40, 40, 400000)
    v_np = np.concatenate([mags, -mags, [1.0, -1.0, 3.0, 1e-30, 1e30, 2e-30, 5e29]])
    v = torch.from_numpy(v_np).to(DEV)
    r, ref = torch.empty_like(v), torch.empty_like(v)
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    assert L.gbpf_selftest_pivot_recip(p(v), p(r), p(ref), C.c_int(v.numel())) == 0
    rel = torch.abs(r - ref) / torch.abs(ref)
    assert rel.max().item() <= 2.0 * 2.0 ** -52
    out = (torch.abs(v) < 1e-30) | (torch.abs(v) > 1e30)
    assert torch.equal(r[out], ref[out])


@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
def test_lane_engine_batched_vs_oracle(oracle, precision):
    """Lockstep lane engine (groups of 32 cases, graph-replayed half-iterations):
    load and outage cases, partly filled groups, voltages against the oracle."""
    base = gridgen.config(0)
    sc = gridgen.scenarios(base, n_load=7, n_outage=6, seed=41)
    g = _grid(base, sc.ncase, sc.load_scale, sc.outage)
    vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, precision, tol=1e-11, max_iter=300,
                         engine=gbpf.PF_ENGINE_LANES)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    vm, va = vm.cpu().numpy(), va.cpu().numpy()
    for c in range(sc.ncase):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        assert np.max(np.abs(vm[c] - vm0)) <= 1e-8, c
        assert np.max(np.abs(va[c] - va0)) <= 1e-8, c
    g.close()


def test_lane_engine_10k_batch_sampled(oracle):
    """64 cases of the 10,000-bus grid (32 load, 32 outage) in FP32 with FP64
    mismatch and refinement; 6 sampled cases against the oracle, and the same
    batch on the block-per-case engine."""
    base = gridgen.config(1)
    sc = gridgen.scenarios(base, n_load=32, n_outage=32, seed=43)
    g = _grid(base, sc.ncase, sc.load_scale, sc.outage)
    out = {}
    for eng in (gbpf.PF_ENGINE_LANES, gbpf.PF_ENGINE_BLOCK):
        vm = torch.zeros((sc.ncase, base.n), dtype=torch.float64, device=DEV)
        va = torch.zeros_like(vm)
        opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP32, tol=1e-11, max_iter=300, engine=eng)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, sc.ncase)
        assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
        out[eng] = (vm.cpu().numpy(), va.cpu().numpy())
    a, b = out[gbpf.PF_ENGINE_LANES], out[gbpf.PF_ENGINE_BLOCK]
    assert np.max(np.abs(a[0] - b[0])) <= 1e-8 and np.max(np.abs(a[1] - b[1])) <= 1e-8
    for c in (0, 5, 31, 32, 40, 63):
        cc = gridgen.apply_scenario(base, sc, c)
        rc, vm0, va0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        assert np.max(np.abs(a[0][c] - vm0)) <= 1e-8, c
        assert np.max(np.abs(a[1][c] - va0)) <= 1e-8, c
    g.close()


@pytest.mark.parametrize("cfg", [0, 1])
def test_branch_flows_vs_oracle(oracle, cfg):
    """Branch flows and total losses of solved cases (one load scenario, one
    single-branch outage) against the oracle's definition at the same
    voltages, element by element."""
    base = CASES[cfg]()
    sc = gridgen.scenarios(base, n_load=1, n_outage=1, seed=3)
    g = _grid(base, sc.ncase, sc.load_scale, sc.outage)
    st, res, vm, va = _run(g, sc.ncase, tol=1e-10, max_iter=300)
    assert st == gbpf.PF_OK
    vm_d = torch.tensor(vm, device=DEV)
    va_d = torch.tensor(va, device=DEV)
    flows = torch.zeros((sc.ncase, base.m, 4), dtype=torch.float64, device=DEV)
    loss = torch.zeros(sc.ncase, dtype=torch.float64, device=DEV)
    gbpf.pf_branch_flows(g.ctx, vm_d, va_d, sc.ncase, flows, loss)
    torch.cuda.synchronize()
    fl, ls = flows.cpu().numpy(), loss.cpu().numpy()
    for c in range(sc.ncase):
        cc = gridgen.apply_scenario(base, sc, c)
        Pf, Qf, Pt, Qt, l0 = oracle.branch_flows(cc, vm[c], va[c])
        ref = np.stack([Pf, Qf, Pt, Qt], axis=1)
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(fl[c] - ref)) <= 1e-12 * scale
        assert abs(ls[c] - l0) <= 1e-11 * max(1.0, abs(l0))
        if sc.outage[c] >= 0:
            assert np.all(fl[c, sc.outage[c]] == 0.0)
    g.close()


def _high_rx(base, seed=0):
    """The 120-bus grid with r/x about 2: the XB fast decoupled iteration
    stalls there while Newton-Raphson converges (checked on the oracle)."""
    rng = np.random.default_rng(seed)
    c = base.copy()
    c.x = c.r * rng.uniform(0.5, 1.5, c.m) * 0.5
    return c


def test_fdpf_nr_fallback(oracle):
    """Without the fallback the stalled case reports PF_ERR_NOT_CONVERGED; with
    it the case is re-run by Newton-Raphson and matches the oracle's NR; a
    grid FDPF solves keeps its FDPF result."""
    case = _high_rx(gridgen.config(0))
    rf, *_ = oracle.power_flow(case, oracle.FDPF, tol=1e-8, max_iter=60)
    rn, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert rf == oracle.ERR_NOT_CONVERGED and rn == oracle.OK
    g = _grid(case, 2)
    vm = torch.zeros((2, case.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-11, max_iter=60)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 2)
    assert st == gbpf.PF_ERR_NOT_CONVERGED and res[0]["method"] == gbpf.PF_FDPF
    for prec in (gbpf.PF_FP64, gbpf.PF_FP32):
        opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=1e-11, max_iter=60, fallback=1)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 2)
        assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
        assert all(res["method"] == gbpf.PF_NR) and all(res["status"] == gbpf.PF_OK)
        for c in range(2):
            assert np.max(np.abs(vm.cpu().numpy()[c] - vm0)) <= 1e-8
            assert np.max(np.abs(va.cpu().numpy()[c] - va0)) <= 1e-8
    g.close()
    g = _grid(gridgen.config(0), 1)
    st, res, _, _ = _run(g, 1)
    opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-8, max_iter=200, fallback=1)
    vm = torch.zeros((1, g.nbus), dtype=torch.float64, device=DEV)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, torch.zeros_like(vm), 1)
    assert st == gbpf.PF_OK and res[0]["method"] == gbpf.PF_FDPF
    g.close()


# Load levels of the 120-bus grid: at 1.0 and 2.0 times the nominal loads the
# fast decoupled iteration reaches 1e-10 in 18 and 40 half-iterations, at 2.4
# it is still at 2e-5 after 60 while Newton-Raphson converges in 7 steps
# (checked on the oracle).
MIXED_LOADS = (1.0, 2.4, 2.0, 2.4)


def _mixed_batch(base):
    return np.stack([np.full(base.n, s) for s in MIXED_LOADS])


def _run_launches(g):
    return gbpf.pf_get_profile(g.ctx, gbpf.PF_K_RUN)[0]


@pytest.mark.parametrize("prec", [gbpf.PF_FP64, gbpf.PF_FP32])
@pytest.mark.parametrize("cluster", [1, 16])
def test_fdpf_nr_fallback_in_launch(oracle, prec, cluster):
    """FDPF -> NR inside the iteration launch (Section III): in a batch whose
    heavy-load cases the fast decoupled iteration leaves unconverged, those
    cases (and only those) switch to Newton-Raphson from a flat start within
    the same launch -- one iteration launch per run, no second one -- and
    report method PF_NR; the others keep their FDPF results.  Every case
    matches the oracle's Newton-Raphson solution of its own loading.  Direct
    runs, a capture and graph replays give bit-identical results."""
    base = gridgen.config(0)
    ls = _mixed_batch(base)
    ncase = ls.shape[0]
    refs = []
    for c in range(ncase):
        cc = base.copy()
        cc.pd = cc.pd * ls[c]
        cc.qd = cc.qd * ls[c]
        rc, v0, a0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        refs.append((v0, a0))
    g = _grid(base, ncase, ls)
    gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_BLOCK, cluster=cluster, factor=1, tail=1, outage=1)
    vm = torch.zeros((ncase, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=1e-10, max_iter=30)
    st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
    assert st == gbpf.PF_ERR_NOT_CONVERGED
    assert list(res["status"]) == [0 if s < 2.2 else gbpf.PF_ERR_NOT_CONVERGED for s in MIXED_LOADS]
    opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=1e-10, max_iter=30, fallback=1)
    first = None
    for k in range(4):  # direct (graphs off), capture + launch, replay, replay
        gbpf.pf_set_graphs(g.ctx, k > 0)
        vm.zero_()
        va.zero_()
        before = _run_launches(g)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase)
        assert st == gbpf.PF_OK, (k, gbpf.pf_last_error(g.ctx))
        assert _run_launches(g) - before == 1, k
        assert list(res["method"]) == [gbpf.PF_FDPF if s < 2.2 else gbpf.PF_NR for s in MIXED_LOADS]
        assert all(res["status"] == gbpf.PF_OK) and all(res["max_mismatch"] <= 1e-10)
        for c in range(ncase):
            assert np.max(np.abs(vm.cpu().numpy()[c] - refs[c][0])) <= 1e-8, (k, c)
            assert np.max(np.abs(va.cpu().numpy()[c] - refs[c][1])) <= 1e-8, (k, c)
        if first is None:
            first = (vm.clone(), va.clone(), res.copy())
        else:
            assert torch.equal(vm, first[0]) and torch.equal(va, first[1]), k
            assert np.array_equal(res["iters"], first[2]["iters"]), k
    g.close()


def test_fdpf_nr_fallback_cluster_engine(oracle):
    """The same switch on the single-case cluster engine: the case's cluster
    of 16 CTAs drops its resident substitution programs and runs
    Newton-Raphson in the same launch."""
    base = gridgen.config(0)
    cc = base.copy()
    cc.pd = cc.pd * 2.4
    cc.qd = cc.qd * 2.4
    rc, v0, a0, _, _ = oracle.power_flow(cc, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    g = _grid(base, 1, np.full((1, base.n), 2.4))
    gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_CLUSTER, cluster=0, factor=1, tail=1)
    vm = torch.zeros((1, base.n), dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    for fb in (0, 1):
        opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=1e-10, max_iter=30, fallback=fb)
        before = _run_launches(g)
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 1)
        assert _run_launches(g) - before == 1
        if not fb:
            assert st == gbpf.PF_ERR_NOT_CONVERGED and res[0]["method"] == gbpf.PF_FDPF
            continue
        assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
        assert res[0]["method"] == gbpf.PF_NR and res[0]["max_mismatch"] <= 1e-10
        assert np.max(np.abs(vm.cpu().numpy()[0] - v0)) <= 1e-8
        assert np.max(np.abs(va.cpu().numpy()[0] - a0)) <= 1e-8
    g.close()


@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
def test_largest_grid_single_case(oracle, precision):
    """The largest grid of the uneven multi-grid set (79,035 buses: its FP64
    solve vector does not fit shared memory, its factor columns are the
    longest) as a single case, against the oracle's Newton-Raphson."""
    sizes = gridgen.config4_sizes()
    g_ = int(np.argmax([n for n, _ in sizes]))
    n, seed = sizes[g_]
    case = gridgen.with_loading_factor(gridgen.delaunay_raw(n, seed, name=f"multigrid{g_}"))
    rc, vm0, va0, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    assert rc == oracle.OK
    g = _grid(case)
    st, res, vm, va = _run(g, 1, precision=precision, tol=1e-11, max_iter=300)
    assert st == gbpf.PF_OK, gbpf.pf_last_error(g.ctx)
    assert np.max(np.abs(vm[0] - vm0)) <= 1e-8 and np.max(np.abs(va[0] - va0)) <= 1e-8
    g.close()
