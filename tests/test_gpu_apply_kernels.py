"""Every kernel of y = S v selectable on a handle (smpm_set_apply_kernel:
one warp per element, 2 and 4 warps per element, the shared-memory stream,
the element-class-shared product) against the oracle's S, FP64 to 1e-12 and
FP32 to 1e-5 relative, and the autotuner (smpm_autotune_apply) choosing one
of the available kernels from its timings."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, inputs
from paper_1601_03432_gb300 import _binding as B
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem

KINDS = [B.APPLY_AUTO, B.APPLY_WARP, B.APPLY_WARP2, B.APPLY_WARP4, B.APPLY_STREAM, B.APPLY_CLASS]


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("spec", [(8, 7, 8, {}), (5, 4, 26, {}),
                                  (4, 3, 6, {"xs": [0.0, 0.2, 0.5, 1.0, 1.3], "ys": [0.0, 0.35, 0.5, 1.1]})],
                         ids=["8x7n8", "5x4n26", "graded4x3n6"])
def test_every_apply_kernel_matches_oracle(built, spec):
    mx, my, n, kw = spec
    og = SMPMGrid(mx, my, n, **kw)
    osys = SchurSystem(og)
    lg = Grid(mx, my, n, **kw)
    lg.factor(precision=1)
    v = np.random.default_rng(71).standard_normal(og.k)
    ref = osys.apply_S(v)
    vp = torch.as_tensor(og.to_padded(v), device="cuda")
    avail = []
    for kind in KINDS:
        try:
            lg.set_apply_kernel(kind)
        except B.SmpmError as e:
            assert e.status == B.SMPM_EINVAL
            assert kind in (B.APPLY_WARP, B.APPLY_WARP2, B.APPLY_WARP4) and 4 * n > 96, kind
            continue
        avail.append(kind)
        out = torch.zeros(og.kp, dtype=torch.float64, device="cuda")
        lg.apply_schur(vp, out)
        torch.cuda.synchronize()
        assert rel(og.from_padded(out.cpu().numpy()), ref) < 1e-12, kind
        out32 = torch.zeros(og.kp, dtype=torch.float32, device="cuda")
        lg.apply_schur32(vp.float(), out32)
        torch.cuda.synchronize()
        assert rel(og.from_padded(out32.double().cpu().numpy()), ref) < 1e-5, kind
    assert B.APPLY_STREAM in avail
    for precision in (0, 1):
        chosen, ms = lg.autotune_apply(precision=precision, reps=3, flush=precision == 0)
        assert chosen in avail and chosen in ms and all(t > 0 for t in ms.values())
        assert set(ms) == set(k for k in avail if k != B.APPLY_AUTO)
        out = torch.zeros(og.kp, dtype=torch.float64, device="cuda")
        lg.apply_schur(vp, out)
        torch.cuda.synchronize()
        assert rel(og.from_padded(out.cpu().numpy()), ref) < 1e-12
