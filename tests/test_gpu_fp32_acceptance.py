"""FP32-RHS acceptance against the FP64 discretisation error (Sec. 4.1:
accuracy is judged by convergence under resolution).

The single-puncture problem of the benchmark (order 6, KO 0.5, 1+log,
Gamma-driver, Sommerfeld, Schwarzschild M = 1) on [-8, 8]^3 at the
benchmark's spacing h = 1/4 (64^3 cells), evolved 50 RK4 steps (t = 3.125,
the step count of the FP32-RHS configuration), and in FP64 also at 2h and
h/2 to the same time.  Away from the puncture (r > 1), per field, the RMS
difference FP32-RHS minus FP64 at h must stay below 1/10 of the Richardson
estimate of the FP64 truncation error at h, |u(2h) - u(h)| / (2^p - 1),
with the order p measured from the three FP64 runs.  The puncture lapse
(min alpha) and the Hamiltonian-constraint norm are held to the same bar
(the truncation error of ||H||_2 is ||H||_2 itself: H vanishes in the
continuum)."""
import numpy as np
import pytest

import bench

pytestmark = pytest.mark.gpu


def test_fp32_rhs_below_truncation_error():
    from paper_2409_10383_gb300 import z4c
    res = bench.fp32_truncation_check(z4c, N=64, nb=2, half=8.0, steps=50, finer=True)
    ratio = np.array(res["ratio"])
    info = {k: res[k] for k in ("order_p", "orders_per_field", "ratio", "puncture_lapse", "hamiltonian_l2")}
    assert res["order_p"] > 2.0, info
    assert ratio.max() <= 0.1, info
    assert res["puncture_lapse"]["ratio"] <= 0.1, info
    assert res["hamiltonian_l2"]["ratio_to_own"] <= 0.1, info
