"""The contraction-stage probe (tdks_contraction_probe) against an FP64 reference.

One 1-D contraction stage of the element kernels (Sec. VI.A sum factorization)
applied `reps` times to many lines, in FP32 and double-float on the CUDA cores and
with BF16 or three-TF32 products on the tensor cores.  The reference M^reps x is a
plain FP64 matrix power; the errors must sit where each arithmetic puts them, which
also checks the tensor-core fragment layouts (a wrong layout gives O(1) errors).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_13130_gb300.build import build
    build()


@pytest.mark.parametrize("P1", [4, 7, 8])
def test_contraction_stage_errors(P1):
    from paper_1810_13130_gb300 import tdks
    rng = np.random.default_rng(100 + P1)
    op, _ = np.linalg.qr(rng.standard_normal((P1, P1)))        # orthogonal: powers stay O(1)
    n, reps = 512 * 40, 8
    x = rng.standard_normal((n, P1))
    ref = x @ np.linalg.matrix_power(op, reps).T
    xd = torch.from_numpy(x).cuda()
    bounds = {0: (0.0, 1e-5), 1: (0.0, 1e-12), 2: (1e-4, 0.2), 3: (0.0, 1e-5)}
    for variant, (lo, hi) in bounds.items():
        y, ms = tdks.contraction_probe(variant, op, xd, reps)
        err = float(np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max())
        assert lo <= err <= hi, (variant, err)
        assert ms > 0
    with pytest.raises(tdks.TDKSError):
        tdks.contraction_probe(0, op, xd[:100], reps)
