"""GPU parity of the Weyl scalar Psi4 on the grid (paper Sec. 3.3; the
coordinate tetrad of reading R20) against the oracle, evaluated on the same
state: a closed-form linear wave at orders 2, 4, 6, the GPU's own puncture
state after RK4 steps (uniform and two-level meshes), and every instance of
a batch.  Interior cells agree to rounding: within 8x the oracle's own
change under one-ulp perturbations of its input (two seeded draws), plus
1e-12 of the largest |Psi4| (Psi4 comes out of cancelling O(1) curvature
terms: where it is near zero, e.g. a puncture at t = 0, a bound relative to
Psi4 alone would ask for more than rounding allows).  Every other cell is
exactly 0 on both sides."""
import numpy as np
import pytest

import analytic as an
import helpers as H
from paper_2409_10383_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _split(m, flat):
    out, off = [], 0
    for b in range(m.nblocks):
        ex, ey, ez = m.ext(b)
        S = ex * ey * ez
        out.append((flat[off:off + S] + 1j * flat[off + S:off + 2 * S]).reshape(ez, ey, ex))
        off += 2 * S
    return out


def _compare(m, u, got_flat):
    """u: the state the GPU saw (ghosts filled the same way on both sides)."""
    ref = m.psi4(u)
    got = _split(m, got_flat)
    scale = max(np.abs(r).max() for r in ref)
    assert scale > 0
    floor = [np.zeros(r.shape) for r in ref]
    for seed in (0, 1):
        v = u * (1.0 + 2.0 ** -52 * np.random.default_rng(seed).uniform(-1.0, 1.0, u.shape))
        for b, p in enumerate(m.psi4(v)):
            floor[b] = np.maximum(floor[b], np.abs(p - ref[b]))
    for b in range(m.nblocks):
        mk = m.interior_mask(b)
        assert np.all(got[b][~mk] == 0)
        err = np.abs(got[b][mk] - ref[b][mk])
        bar = 8 * floor[b][mk].max() + 1e-12 * scale
        assert err.max() <= bar, (b, err.max(), bar, scale)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_psi4_linear_wave(oracle, order):
    from paper_2409_10383_gb300.z4c import Z4c
    n = 12
    w = dict(n=np.array([[n, n, n]] * 2), lo=np.array([[0.3, 0.2, 0.25], [0.3 + n * 0.025, 0.2, 0.25]]),
             h=np.full(2, 0.025), ghosts=order // 2 + 1, order=order, periodic=False,
             dom_lo=(0.3, 0.2, 0.25), dom_hi=(0.3 + 2 * n * 0.025, 0.2 + n * 0.025, 0.25 + n * 0.025),
             lapse=1, shift=1, ko_sigma=0.0, kappa1=0.0, kappa2=0.0, eta=2.0, chi_floor=1e-6, cfl=0.25,
             id_kind=inputs.ID_LINEAR_WAVE, id_par=[0.05, 1.0, 0.0], precision=64)
    m = H.oracle_mesh(oracle, w)
    u = an.state_on_mesh(m, "linear_wave", (0.05, 1.0), time=0.13)
    m.fill_ghosts(u)
    g = Z4c.from_workload(w)
    g.z4c_set_state(u)
    _compare(m, u, g.z4c_psi4().cpu().numpy())
    g.close()


@pytest.mark.parametrize("order", [6, 2])
def test_psi4_puncture_after_steps(oracle, order):
    from paper_2409_10383_gb300.z4c import Z4c
    w = H.small_workload("puncture", order, (2, 2, 2), 12)
    m = H.oracle_mesh(oracle, w)
    g = Z4c.from_workload(w)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    g.z4c_rk4_step(0.25 * float(w["h"][0]), 3)
    got = g.z4c_psi4().cpu().numpy()
    u = g.z4c_get_state()
    m.fill_ghosts(u)
    _compare(m, u, got)
    g.close()


def test_psi4_two_level_mesh(oracle):
    """A refined puncture mesh (the fill's restriction and prolongation feed
    the stencils next to level boundaries)."""
    from paper_2409_10383_gb300.z4c import Z4c
    nn, lo, h, lev = inputs.octree_mesh((4, 4, 4), 8, (-8.0,) * 3, (8.0,) * 3, [(0.1, 0.2, 0.3)], [0.5], 1)
    w = dict(n=nn, lo=lo, h=h, level=lev, ghosts=4, order=6, periodic=False, dom_lo=(-8.0,) * 3,
             dom_hi=(8.0,) * 3, lapse=1, shift=1, ko_sigma=0.5, kappa1=0.02, kappa2=0.0, eta=2.0, chi_floor=1e-6,
             cfl=0.25, id_kind=inputs.ID_SCHWARZSCHILD, id_par=[1.0, 0.0], precision=64)
    m = H.oracle_mesh(oracle, w)
    g = Z4c.from_workload(w)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    g.z4c_rk4_step(0.25 * float(np.min(h)), 2)
    got = g.z4c_psi4().cpu().numpy()
    u = g.z4c_get_state()
    m.fill_ghosts(u)
    _compare(m, u, got)
    g.close()


def test_psi4_batch(oracle):
    """Every instance of a batch (punctures and gauge waves, orders 4/6) in
    one call, each against the oracle on its own mesh."""
    from paper_2409_10383_gb300.z4c import Z4c
    ws = inputs.uneven_batch_small()
    g = Z4c.batch(ws)
    for i, w in enumerate(ws):
        g.z4c_set_initial_data_instance(i, w["id_kind"], w["id_par"])
    got = g.z4c_psi4().cpu().numpy()
    state = g.z4c_get_state()
    off = 0
    for i, w in enumerate(ws):
        m = H.oracle_mesh(oracle, w)
        u = state[g.instance_slice(i)].copy()
        m.fill_ghosts(u)
        n2 = 2 * m.size() // 22
        if np.abs(np.concatenate([p.ravel() for p in m.psi4(u)])).max() > 0:
            _compare(m, u, got[off:off + n2])
        off += n2
    assert off == got.size
    g.close()


def test_psi4_fp32_only_context(oracle):
    """A context with FP32-RHS blocks only has no FP64 pre-pass store: Psi4
    then keeps the y/z derivatives in the accumulator register, and the
    state register is left as it was (interior cells; the call fills the
    ghosts)."""
    from paper_2409_10383_gb300.z4c import Z4c
    w = H.small_workload("puncture", 6, (2, 1, 1), 12)
    m = H.oracle_mesh(oracle, w)
    g = Z4c.from_workload(w, precision=32)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    g.z4c_rk4_step(0.25 * float(w["h"][0]), 2)
    before = g.z4c_get_state()
    got = g.z4c_psi4().cpu().numpy()
    u = g.z4c_get_state()
    for b in range(m.nblocks):
        mk = m.interior_mask(b)
        assert np.array_equal(m.blocks(u)[b][:, mk], m.blocks(before)[b][:, mk])
    m.fill_ghosts(u)
    _compare(m, u, got)
    g.close()
