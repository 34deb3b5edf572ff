"""Host-side pins of bench.py's FP32-RHS acceptance analysis (no GPU):
the midpoint interpolation that carries a cell-centred solution to the
centres of the cells twice as wide is exact on polynomials of degree 5 per
axis and not on degree 6, and the Richardson estimate recovers a planted
error C h^p and its order p from three resolutions."""
import numpy as np
import pytest

import bench


def _centres(N, half):
    h = 2.0 * half / N
    x = -half + h * (np.arange(N) + 0.5)
    return x[None, None, :], x[None, :, None], x[:, None, None]


@pytest.mark.parametrize("deg,exact", [(5, True), (6, False)])
def test_midpoint_interpolation_degree(deg, exact):
    N, half = 16, 2.0
    f = lambda X, Y, Z: X ** deg + 0.5 * Y ** (deg - 2) * Z ** 2 - 0.25 * X * Y * Z ** (deg - 3) + 1.5
    G = f(*_centres(N, half))[None]
    C = bench.to_coarse(G)[0]
    ref = f(*_centres(N // 2, half))
    inner = (slice(1, N // 2 - 1),) * 3
    assert not np.isnan(C[inner]).any() and np.isnan(C[0]).all()
    err = np.abs(C[inner] - ref[inner]).max()
    assert (err < 1e-12) == exact, err


@pytest.mark.parametrize("p", [4.0, 6.0])
def test_richardson_recovers_planted_error(p):
    """u_h = u + C(x) h^p at three spacings; the FP32 stand-in adds 1% of the
    error at h: the estimate must be C h^p, the ratio 0.01, the order p."""
    half, N = 4.0, 32
    u = lambda X, Y, Z: np.sin(0.3 * X) * np.cos(0.2 * Y) + 0.1 * Z
    C = lambda X, Y, Z: 1.0 + 0.2 * X * Y - 0.05 * Z ** 2

    def state(n):
        X, Y, Z = _centres(n, half)
        h = 2.0 * half / n
        v = u(X, Y, Z) + C(X, Y, Z) * h ** p
        return np.broadcast_to(v, (22,) + v.shape).copy()

    fine, coarse, finer = state(N), state(N // 2), state(2 * N)
    X, Y, Z = _centres(N, half)
    h = 2.0 * half / N
    f32 = fine + 0.01 * C(X, Y, Z) * h ** p
    res = bench.fp32_acceptance(fine, f32, coarse, half, finer64=finer, r_min=0.5)
    assert abs(res["order_p"] - p) < 0.05, res["order_p"]
    assert np.allclose(res["ratio"], 0.01, rtol=0.05), res["ratio"]
