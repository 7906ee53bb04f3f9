"""Elimination tree and level sets computed on the GPU (pf_etree_levels_device)
from the filled pattern, bit-identical to the host analysis (itself bit-exact
against the oracle in test_library_host.py), on the named grids and on small
random grids whose B'' is a forest."""
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


def _check(case):
    g = gbpf.Grid(case)
    for which in (gbpf.PF_MAT_BP, gbpf.PF_MAT_BPP):
        sym = g.symbolic(which)
        n = int(g.info.n[which])
        if n == 0:
            continue
        Lp = torch.tensor(sym["Lp"], device=DEV)
        Li = torch.tensor(sym["Li"] if len(sym["Li"]) else np.zeros(1, np.int32), device=DEV)
        parent = torch.full((n,), -7, dtype=torch.int32, device=DEV)
        level = torch.zeros(n, dtype=torch.int32, device=DEV)
        nlev = torch.zeros(1, dtype=torch.int32, device=DEV)
        scratch = torch.zeros(3 * n, dtype=torch.int32, device=DEV)
        gbpf.pf_etree_levels_device(n, Lp, Li, parent, level, nlev, scratch)
        torch.cuda.synchronize()
        assert np.array_equal(parent.cpu().numpy(), sym["parent"])
        assert np.array_equal(level.cpu().numpy(), sym["level"])
        assert int(nlev.item()) == int(g.info.nlevels[which])
    g.close()


@pytest.mark.parametrize("cfg", [0, 1, 3])
def test_device_etree_levels_named_grids(cfg):
    _check(gridgen.config(cfg))


@pytest.mark.parametrize("seed", range(6))
def test_device_etree_levels_small_grids(seed):
    _check(gridgen.small_raw(12 + 5 * seed, 100 + seed))
