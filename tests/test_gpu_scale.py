"""Scale covariance on the GPU: with positions and box scaled by s, the potential scales by 1/s
and the field by 1/s^2 (phi(s x; s d) = phi(x; d) / s: the kernel is 1/r and the method's
steps -- R0, check points, the fit, the box integrals -- scale with the box).  Any constant of
the device path in absolute units (a distance threshold, a padding position, a near-unit
reach) would break it at one end of the range.  With s = 2^-10 and 2^10 every operation of
every path scales exactly (measured: bitwise equal results in all three precisions, also at
2^-20 and 2^20), so the comparison is held to 1e-14 (float64 rounding of the rescaling), not
to the paths' tolerances; s = 1e-3 and 1e3 give independent float32 roundings (FP32C 7e-7)."""
import numpy as np
import pytest

from parity_check import assert_close
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXACT = 1e-14


def _eval(x, q, d, precision, pairs):
    pc = B.PeriodicCoulomb(d, 8, 200, precision=precision, pairs=pairs)
    try:
        phi, g = pc(torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda"))
        return phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()


@pytest.mark.parametrize("pairs", ["one-sided", "symmetric"])
@pytest.mark.parametrize("precision", ["fp64", "fp32c", "ff"])
@pytest.mark.parametrize("scale", [2.0 ** -10, 2.0 ** 10])
def test_potential_and_field_scale_with_the_box(scale, precision, pairs):
    s = W.uniform_gauss(N=3000, d=(1.0, 1.5, 2.0), p=8, M=200, seed=12)
    phi1, g1 = _eval(s.x, s.q, s.d, precision, pairs)
    phis, gs = _eval(s.x * scale, s.q, tuple(scale * v for v in s.d), precision, pairs)
    assert np.all(np.isfinite(phis)) and np.all(np.isfinite(gs))
    assert_close(phis * scale, phi1, EXACT, f"phi at scale {scale}")
    assert_close(gs * scale * scale, g1, EXACT, f"grad at scale {scale}")
