"""Uneven multi-grid batch (pf_pack_*) of libgbpf against the CPU oracle.

Grids of the uneven-batch family (their loading factors written by
oracle/find_loading_factors.py) of different sizes, one of them too large
for its FP64 solve vector to fit in shared memory, are packed into one
launch and run to 1e-11 p.u. in FP64 and in FP32 with FP64 refinement; every
grid's voltages must be within 1e-8 p.u./rad of the oracle's Newton-Raphson
run to 1e-12 p.u.  A second pack run reuses the pack (its scratch and the
grids' factors are rebuilt) and must give identical results.
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


def _pick():
    """Indices of the uneven-batch grids used here: the one nearest 26,000
    buses (its FP64 vector exceeds shared memory) and the three smallest."""
    sizes = [n for n, _ in gridgen.config4_sizes()]
    big = int(np.argmin([abs(n - 26000) for n in sizes]))
    small = [int(i) for i in np.argsort(sizes)[:3]]
    return [small[0], big, small[1], small[2]]


@pytest.fixture(scope="module")
def grids():
    sizes = gridgen.config4_sizes()
    table = gridgen.load_loading_factors()
    out = []
    for g in _pick():
        n, seed = sizes[g]
        raw = gridgen.delaunay_raw(n, seed, name=f"multigrid{g}")
        out.append(gridgen.with_loading_factor(raw, table))
    return out


@pytest.mark.parametrize("precision", [gbpf.PF_FP64, gbpf.PF_FP32])
def test_pack_vs_oracle(oracle, grids, precision):
    gs = [gbpf.Grid(c) for c in grids]
    for g in gs:
        g.set_cases(1)
    pk = gbpf.Pack(gs)
    tot = int(pk.offset[-1])
    vm = torch.zeros(tot, dtype=torch.float64, device=DEV)
    va = torch.zeros_like(vm)
    opts = gbpf.run_opts(gbpf.PF_FDPF, precision, tol=1e-11, max_iter=300)
    st, res = pk.run(opts, vm, va)
    assert st == gbpf.PF_OK, pk.last_error()
    v1, a1 = vm.cpu().numpy().copy(), va.cpu().numpy().copy()
    st2, res2 = pk.run(opts, vm, va)
    assert st2 == gbpf.PF_OK
    assert np.array_equal(vm.cpu().numpy(), v1) and np.array_equal(va.cpu().numpy(), a1)
    for k, c in enumerate(grids):
        rc, vm0, va0, _, _ = oracle.power_flow(c, oracle.NR, tol=1e-12, max_iter=30)
        assert rc == oracle.OK
        lo, hi = pk.offset[k], pk.offset[k + 1]
        assert np.max(np.abs(v1[lo:hi] - vm0)) <= 1e-8, (k, c.n)
        assert np.max(np.abs(a1[lo:hi] - va0)) <= 1e-8, (k, c.n)
        assert res[k]["status"] == gbpf.PF_OK and res[k]["max_mismatch"] <= 1e-11
    pk.close()
    for g in gs:
        g.close()


def test_pack_rejects_bad_arguments(grids):
    g = gbpf.Grid(grids[0])
    with pytest.raises(gbpf.PFError):
        gbpf.Pack([g, g])
    pk = gbpf.Pack([g])
    vm = torch.zeros(g.nbus, dtype=torch.float64, device=DEV)
    opts = gbpf.run_opts(gbpf.PF_NR, gbpf.PF_FP64, tol=1e-8, max_iter=20)
    with pytest.raises(gbpf.PFError):
        pk.run(opts, vm, vm.clone())
    pk.close()
    g.close()
