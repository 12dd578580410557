"""The step kernels' float32 arccos(x)/3 (the polynomial form of Abramowitz &
Stegun 4.4.46 with the library's own degree-7 coefficients) against the exact
value and against CUDA's acosf, on every float32 near the ends of [-1, 1] and
a dense grid between: within 2.5e-7 absolute of arccos(x)/3 in float64 (float32
evaluation of the fitted form: 1.1e-7 in an emulation with unfused operations)
and within 3e-7 of acosf(x)/3."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_polynomial_arccos_third(gpu):
    torch = pytest.importorskip("torch")
    grid = np.linspace(-1.0, 1.0, 4_000_001).astype(np.float32)
    near = np.arange(1, 4096, dtype=np.float32) * np.float32(2.0 ** -24)
    xs = np.concatenate([grid, np.float32(1) - near, np.float32(-1) + near,
                         np.float32([-1.0, 1.0, 0.0, -0.0, 1e-30, -1e-30, 0.5, -0.5])])
    x = torch.from_numpy(xs).cuda()
    poly = gpu.adot_math_probe(0, x).cpu().numpy().astype(np.float64)
    lib = gpu.adot_math_probe(1, x).cpu().numpy().astype(np.float64)
    ref = np.arccos(xs.astype(np.float64)) / 3.0
    assert np.isfinite(poly).all()
    assert np.abs(poly - ref).max() <= 2.5e-7, np.abs(poly - ref).max()
    assert np.abs(poly - lib).max() <= 3e-7, np.abs(poly - lib).max()
    # the ends are exact to float32 rounding: arccos(1) = 0, arccos(-1)/3 = pi/3
    assert poly[np.flatnonzero(xs == 1.0)[0]] == 0.0
    assert abs(poly[np.flatnonzero(xs == -1.0)[0]] - np.pi / 3) <= 1e-7
