"""The allocation-free deflation entry point (smpm_apply_deflation_noalloc):
for callers that cannot allocate device memory when they call (a framework's
caching allocator owns the free memory, or cudaMalloc's implicit device
synchronisation is not allowed).  Its output must match smpm_apply_deflation
on two calls in a row, which share the one static scratch array.  This file
sorts last so that a failure here stops a -x run only after every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid
from paper_1601_03432_gb300 import _binding as B


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("opts", [{}, {"precision": 1}, {"precond": 1}, {"precond": 0}],
                         ids=["fp64", "mixed", "block-jacobi", "no-precond"])
@pytest.mark.parametrize("shape", [(4, 3, 6), (16, 16, 8), (9, 7, 5)])
def test_matches_allocating_entry_point(built, shape, opts):
    g = Grid(*shape)
    g.factor(**opts)
    rng = np.random.default_rng(31)
    for call in range(2):
        v = torch.as_tensor(rng.standard_normal(g.kp), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(v)
        out = torch.full_like(v, float("nan"))
        g.apply_deflation(v, ref)
        g.apply_deflation_noalloc(v, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o)), call
        assert np.linalg.norm(o - r) <= 1e-12 * max(np.linalg.norm(r), 1e-300), call


def test_rejects_grids_beyond_the_scratch(built):
    g = Grid(129, 129, 2)               # 33,024 interfaces > 32,768
    v = torch.zeros(g.kp, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SmpmError) as ei:
        g.apply_deflation_noalloc(v, torch.empty_like(v))
    assert ei.value.status == B.SMPM_EINVAL
    assert "32768" in str(ei.value)


def test_rejects_an_unfactored_handle(built):
    g = Grid(4, 3, 6)
    v = torch.zeros(g.kp, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SmpmError) as ei:
        g.apply_deflation_noalloc(v, torch.empty_like(v))
    assert ei.value.status == B.SMPM_ESTATE
