"""GPU parity of the diagnostics beside the step (paper Sec. 3.2 refinement
indicators, Sec. 3.3 puncture tracker) against the oracle, evaluated on the
same state: the GPU's state after RK4 steps, copied to the oracle.
min chi is a selection of stored values (bit-exact); max |grad chi| and the
interpolated shift agree to rounding."""
import numpy as np
import pytest

import helpers as H
from paper_2409_10383_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _check(oracle, w, punctures, steps):
    from paper_2409_10383_gb300.z4c import Z4c
    m = H.oracle_mesh(oracle, w)
    g = Z4c.from_workload(w)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    dt = w.get("dt", 0.25 * float(np.min(w["h"])))
    g.z4c_rk4_step(dt, steps)
    cmin, gmax = g.z4c_block_indicators()
    x_gpu, b_gpu = g.z4c_track_punctures(punctures, dt)
    u = g.z4c_get_state()
    m.fill_ghosts(u)
    cmin_o, gmax_o = m.block_indicators(u)
    x_o, b_o = m.track_punctures(u, punctures, dt)
    assert np.array_equal(cmin, cmin_o)
    assert np.abs(gmax - gmax_o).max() <= 1e-13 * np.abs(gmax_o).max()
    assert np.abs(b_gpu - b_o).max() <= 1e-14 + 1e-13 * np.abs(b_o).max()
    assert np.abs(x_gpu - x_o).max() <= 1e-14
    g.close()
    return cmin, gmax, b_gpu


def test_diagnostics_two_level_puncture(oracle):
    nn, lo, h, lev = inputs.octree_mesh((4, 4, 4), 8, (-8.0,) * 3, (8.0,) * 3, [(0.1, 0.2, 0.3)], [0.5], 1)
    w = dict(n=nn, lo=lo, h=h, level=lev, ghosts=4, order=6, periodic=False, dom_lo=(-8.0,) * 3,
             dom_hi=(8.0,) * 3, lapse=1, shift=1, ko_sigma=0.5, kappa1=0.02, kappa2=0.0, eta=2.0, chi_floor=1e-6,
             cfl=0.25, id_kind=inputs.ID_SCHWARZSCHILD, id_par=[1.0, 0.0], precision=64)
    pts = np.array([[0.05, 0.07, -0.02], [1.3, -2.2, 0.4], [0.0, 0.0, 0.0]])
    cmin, gmax, beta = _check(oracle, w, pts, 3)
    # the smallest chi and the steepest chi sit in the refined blocks around
    # the puncture at the origin; the shift there is non-zero after 3 steps
    fine = np.where(lev == 1)[0]
    assert np.argmin(cmin) in fine and np.argmax(gmax) in fine
    assert np.abs(beta).max() > 0


def test_diagnostics_bl_binary_full_mesh(oracle):
    """The refined two-puncture mesh (680 blocks): indicators and one
    tracker step of both punctures after 2 RK4 steps."""
    w = inputs.workload("bl_binary_smr")
    cmin, gmax, beta = _check(oracle, w, np.array([[3.0, 0.0, 0.0], [-3.0, 0.0, 0.0]]), 2)
    finest = np.where(w["level"] == w["level"].max())[0]
    assert np.argmin(cmin) in finest
    # mirror symmetry x -> -x: the punctures' shifts are mirror images (the
    # shift at a puncture is ~1e-11 after 2 steps; rounding ~1e-12 of it)
    assert abs(beta[0, 0] + beta[1, 0]) <= 1e-10 * abs(beta[0, 0])
    assert abs(beta[0, 1] - beta[1, 1]) <= 1e-10 * max(abs(beta[0, 1]), abs(beta[0, 0]))


def test_tracker_rejects_outside_and_batches(oracle):
    from paper_2409_10383_gb300 import z4c
    from paper_2409_10383_gb300.z4c import Z4c
    w = H.small_workload("puncture", 6, (1, 1, 1), 16)
    g = Z4c.from_workload(w)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    with pytest.raises(z4c.Z4cError, match="status -1"):
        g.z4c_track_punctures([[1e3, 0.0, 0.0]], 0.1)
    g.close()
    ws = inputs.uneven_batch_small()[:2]
    b = Z4c.batch(ws)
    with pytest.raises(z4c.Z4cError, match="status -3"):
        b.z4c_track_punctures([[0.0, 0.0, 0.0]], 0.1)
    b.close()
