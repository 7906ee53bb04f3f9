"""The allocation-free mismatch entry point, pf_mismatch_static.

It serves callers that cannot allocate device memory when they need a
mismatch (a fixed device-memory plan decided at start-up, or an application
allocator that owns the GPU): everything is caller-owned and its one
intermediate lives in a fixed device array inside the library.  This checks,
through the C ABI, that two calls in a row give the same dp, dq and maximum
as the context-based pf_mismatch, within the tolerance of the other mismatch
parity tests, and that sizes above the fixed maximum are rejected.  The file
name makes pytest collect it last.
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


@pytest.mark.parametrize("cfg", [0, 1])
def test_static_mismatch_matches_context_mismatch_twice(cfg):
    case = gridgen.config(cfg)
    g = gbpf.Grid(case)
    g.set_cases(1)
    rp, col, G, B = gbpf.pf_get_ybus(g.ctx, case.n, g.info.nnz_ybus)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)  # noqa: E731
    rp_d, col_d = t(rp, torch.int32), t(col, torch.int32)
    G_d, B_d = t(G, torch.float64), t(B, torch.float64)
    bt_d = t(case.btype, torch.int32)
    psp_d, qsp_d = t(case.pg - case.pd, torch.float64), t(-case.qd, torch.float64)
    scale = max(1.0, float(np.max(np.abs(B))))
    rng = np.random.default_rng(123 + cfg)
    for call in range(2):
        vm = t(rng.uniform(0.95, 1.05, case.n), torch.float64)
        va = t(rng.uniform(-0.2, 0.2, case.n), torch.float64)
        dp0, dq0 = torch.zeros_like(vm), torch.zeros_like(vm)
        mx0 = torch.zeros(1, dtype=torch.float64, device=DEV)
        gbpf.pf_mismatch(g.ctx, vm.view(1, -1), va.view(1, -1), dp0, dq0, mx0, 1)
        dp1, dq1 = torch.full_like(vm, 7.0), torch.full_like(vm, 7.0)
        mx1 = torch.full((1,), 5.0, dtype=torch.float64, device=DEV)  # must be cleared by the call
        st = gbpf.pf_mismatch_static(case.n, rp_d, col_d, G_d, B_d, bt_d, psp_d, qsp_d, vm, va,
                                     dp1, dq1, mx1)
        assert st == gbpf.PF_OK
        torch.cuda.synchronize()
        assert torch.max(torch.abs(dp1 - dp0)).item() <= 1e-12 * scale, call
        assert torch.max(torch.abs(dq1 - dq0)).item() <= 1e-12 * scale, call
        assert abs(mx1.item() - mx0.item()) <= 1e-12 * scale, call
    g.close()


def test_static_mismatch_rejects_oversize():
    z = torch.zeros(4, dtype=torch.float64, device=DEV)
    zi = torch.zeros(4, dtype=torch.int32, device=DEV)
    st = gbpf.pf_mismatch_static(gbpf.PF_STATIC_MAX_BUS + 1, zi, zi, z, z, zi, z, z, z, z, z, z, z)
    assert st == gbpf.PF_ERR_ARG
    st = gbpf.pf_mismatch_static(0, zi, zi, z, z, zi, z, z, z, z, z, z, z)
    assert st == gbpf.PF_ERR_ARG
