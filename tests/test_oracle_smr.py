"""Pins for the oracle's static-mesh-refinement ghost fill (paper Sec. 3.1).

Restriction and prolongation are 5-point Lagrange interpolation per axis
(n = N_g + 1 points with 4 ghosts, 3D tensor product).  So every ghost value
must be exact on tensor polynomials of degree <= 4 per axis, inexact one
degree above, and converge at 5th order on smooth data (Sec. 3.1.1: error
O(h^5) for 4 ghosts).  On a linear wave with a refined region the solution
error keeps converging (Sec. 4.1, refined-quadrant run).
"""
import numpy as np
import pytest

from paper_2409_10383_gb300 import inputs


def two_level(oracle, n=8, nb=4, half=8.0, order=6, periodic=False, centre=(0.1, 0.2, 0.3), radius=0.5,
              **kw):
    nn, lo, h, lev = inputs.octree_mesh((nb,) * 3, n, (-half,) * 3, (half,) * 3, [centre], [radius], 1)
    m = oracle.Mesh(n=nn, lo=lo, h=h, level=lev, ghosts=order // 2 + 1, order=order,
                    dom_lo=(-half,) * 3, dom_hi=(half,) * 3, periodic=periodic, **kw)
    return m


def fill_with(m, fn):
    u = m.zeros()
    for b, blk in enumerate(m.blocks(u)):
        v = fn(*m.centres(b))
        blk[:] = v[None] * (1 + 0.1 * np.arange(22))[:, None, None, None]
    return u


def ghost_masks(m):
    """per block: ghost cells that are filled (not interior, inside the domain)"""
    return [~m.interior_mask(b) & ~m.sommerfeld_mask(b) for b in range(m.nblocks)]


def test_mesh_has_two_levels(oracle):
    m = two_level(oracle)
    assert set(m.level.tolist()) == {0, 1} and (m.level == 1).sum() == 64


@pytest.mark.parametrize("deg", [(4, 4, 4), (3, 2, 4), (0, 4, 1)])
def test_transfer_exact_on_degree4_polynomials(oracle, deg):
    m = two_level(oracle)
    p = lambda X, Y, Z: (0.3 + X) ** deg[0] * (0.2 - Y) ** deg[1] * (0.1 + Z) ** deg[2]
    u = fill_with(m, p)
    ref = u.copy()
    for b, blk in enumerate(m.blocks(u)):   # poison ghosts that the fill must overwrite
        blk[:, ghost_masks(m)[b]] = np.nan
    m.fill_ghosts(u)
    err, scale = 0.0, 0.0
    for b in range(m.nblocks):
        g = ghost_masks(m)[b]
        got, want = m.blocks(u)[b][:, g], m.blocks(ref)[b][:, g]
        assert np.all(np.isfinite(got))
        err = max(err, np.abs(got - want).max())
        scale = max(scale, np.abs(want).max())
    assert err <= 1e-11 * scale, (err, scale)


def boundary_two_level(oracle, n=8):
    """Refined blocks on the x = +8 face next to coarse blocks on the same
    face: prolongation stencils there need the shift into the domain."""
    return two_level(oracle, n=n, centre=(7.9, 0.1, 0.2), radius=0.5)


def test_boundary_mesh_needs_shifted_stencils(oracle):
    m = boundary_two_level(oracle)
    fine = np.where(m.level == 1)[0]
    assert len(fine) > 0 and np.all(np.isclose(m.lo[fine, 0] + m.n[fine, 0] * m.h[fine], 8.0) |
                                    (m.lo[fine, 0] + m.n[fine, 0] * m.h[fine] < 8.0))
    assert np.any(np.isclose(m.lo[fine, 0] + m.n[fine, 0] * m.h[fine], 8.0))
    assert np.any((m.level == 0) & np.isclose(m.lo[:, 0] + m.n[:, 0] * m.h, 8.0))


@pytest.mark.parametrize("deg", [(4, 4, 4), (4, 0, 2)])
def test_transfer_exact_near_outer_boundary(oracle, deg):
    """Reading R13: near a non-periodic face the 5 coarse cells of a
    prolongation stencil are shifted into the domain; Lagrange interpolation
    on any 5 nodes stays exact for degree <= 4."""
    m = boundary_two_level(oracle)
    p = lambda X, Y, Z: (0.3 + X) ** deg[0] * (0.2 - Y) ** deg[1] * (0.1 + Z) ** deg[2]
    u = fill_with(m, p)
    ref = u.copy()
    for b, blk in enumerate(m.blocks(u)):
        blk[:, ghost_masks(m)[b]] = np.nan
    m.fill_ghosts(u)
    err, scale = 0.0, 0.0
    for b in range(m.nblocks):
        g = ghost_masks(m)[b]
        got, want = m.blocks(u)[b][:, g], m.blocks(ref)[b][:, g]
        assert np.all(np.isfinite(got))
        err = max(err, np.abs(got - want).max())
        scale = max(scale, np.abs(want).max())
    assert err <= 1e-11 * scale, (err, scale)


def test_boundary_transfer_converges_at_fifth_order(oracle):
    """The shifted stencils keep the 5th-order interpolation error."""
    errs = []
    for n in (8, 16):
        m = two_level(oracle, n=n, centre=(7.9, 0.1, 0.2), radius=0.5 * 8 / n)
        fn = lambda X, Y, Z: np.sin(0.6 * X + 0.3) * np.cos(0.5 * Y - 0.2) * np.sin(0.4 * Z + 0.7)
        u = fill_with(m, fn)
        ref = u.copy()
        m.fill_ghosts(u)
        errs.append(max(np.abs(m.blocks(u)[b] - m.blocks(ref)[b])[:, ghost_masks(m)[b]].max()
                        for b in range(m.nblocks) if m.level[b] == 1))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 4.5, (errs, rate)


def test_transfer_not_exact_on_degree5(oracle):
    m = two_level(oracle)
    u = fill_with(m, lambda X, Y, Z: (0.3 + X) ** 5)
    ref = u.copy()
    m.fill_ghosts(u)
    errs = [np.abs(m.blocks(u)[b] - m.blocks(ref)[b])[:, ghost_masks(m)[b]].max() for b in range(m.nblocks)]
    assert max(errs) > 1e-6


def test_transfer_converges_at_fifth_order(oracle):
    errs = []
    for n in (8, 16):
        m = two_level(oracle, n=n, radius=0.5 * 8 / n)
        fn = lambda X, Y, Z: np.sin(0.6 * X + 0.3) * np.cos(0.5 * Y - 0.2) * np.sin(0.4 * Z + 0.7)
        u = fill_with(m, fn)
        ref = u.copy()
        m.fill_ghosts(u)
        errs.append(max(np.abs(m.blocks(u)[b] - m.blocks(ref)[b])[:, ghost_masks(m)[b]].max()
                        for b in range(m.nblocks) if m.level[b] == 1))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 4.5, (errs, rate)


def test_linear_wave_with_refined_region(oracle):
    """Sec. 4.1: periodic linear wave with a refined region, 6th order + RK4:
    the L1_RMS error of g_ab (the paper's metric) keeps converging at >= 4th
    order with the refinement interface (5th-order transfer feeding the
    second-derivative stencils)."""
    def run(n):
        half = 0.5
        nn, lo, h, lev = inputs.octree_mesh((2, 2, 2), n, (-half,) * 3, (half,) * 3, [(0.25, 0.25, 0.25)],
                                            [0.15], 1)
        m = oracle.Mesh(n=nn, lo=lo, h=h, level=lev, ghosts=4, order=6, dom_lo=(-half,) * 3,
                        dom_hi=(half,) * 3, periodic=True, lapse=1, shift=1, eta=2.0, ko_sigma=0.02)
        u = m.initial_data(inputs.ID_LINEAR_WAVE, [1e-6, 1.0, 0.0])
        dt = 0.25 * h.min()
        nsteps = int(round(0.125 / dt))
        m.rk4(u, dt, nsteps)
        ua = m.initial_data(inputs.ID_LINEAR_WAVE, [1e-6, 1.0, dt * nsteps])
        vol = sum(h[b] ** 3 * np.prod(nn[b]) for b in range(len(h)))
        tot = 0.0
        for a in range(3):
            for c in range(3):
                q = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)].index((min(a, c), max(a, c)))
                acc = 0.0
                for b in range(m.nblocks):
                    mk, B, A = m.interior_mask(b), m.blocks(u)[b], m.blocks(ua)[b]
                    acc += np.abs(B[1 + q][mk] / B[0][mk] - A[1 + q][mk] / A[0][mk]).sum() * h[b] ** 3
                tot += (acc / vol) ** 2
        return np.sqrt(tot), (lev == 1).sum()
    e8, nref = run(8)
    e12, _ = run(12)
    assert nref == 8
    assert np.log(e8 / e12) / np.log(1.5) > 3.5, (e8, e12)


def test_bl_binary_mesh_fills_exactly_on_quartics(oracle):
    """The refined two-puncture mesh (2x2x2 roots of 16^3 at h = 2 over
    [-32,32]^3, levels 0..6): 680 blocks, symmetric under x -> -x, 2:1
    balanced; the oracle fills every ghost cell of it (no stencil reaches two
    levels apart or leaves the domain, reading R13 at the outer faces) and
    the fill is exact on a tensor quartic."""
    w = inputs.workload("bl_binary_smr")
    assert len(w["h"]) == 680 and w["level"].max() == 6
    assert np.isclose(w["h"].min(), 1.0 / 32) and np.isclose(w["h"].max(), 1.0)
    pairs = inputs.mirror_blocks(w["n"], w["lo"], w["h"])
    assert np.all(pairs[pairs] == np.arange(len(pairs)))
    m = oracle.Mesh(n=w["n"], lo=w["lo"], h=w["h"], level=w["level"], ghosts=4, order=6, dom_lo=w["dom_lo"],
                    dom_hi=w["dom_hi"], periodic=False)
    p = lambda X, Y, Z: 1.0 + 1e-6 * (X + 1.0) ** 4 * (2.0 - Y) ** 3 * (Z + 0.5) ** 2
    u = fill_with(m, p)
    ref = u.copy()
    masks = ghost_masks(m)
    for b, blk in enumerate(m.blocks(u)):
        blk[:, masks[b]] = np.nan
    m.fill_ghosts(u)
    assert np.all(np.isfinite(u))
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()


# --- 2 ghosts (2nd-order differencing): 3-point transfer, reading R19 ---
# n = N_g + 1 = 3 Lagrange points per axis (Sec. 3.1.1): exact for degree <= 2
# per axis, not for 3, error O(h^3).

def _max_ghost_error(m, fn, fine_only=False):
    u = fill_with(m, fn)
    ref = u.copy()
    for b, blk in enumerate(m.blocks(u)):
        blk[:, ghost_masks(m)[b]] = np.nan
    m.fill_ghosts(u)
    err, scale = 0.0, 0.0
    for b in range(m.nblocks):
        if fine_only and m.level[b] != 1:
            continue
        g = ghost_masks(m)[b]
        got, want = m.blocks(u)[b][:, g], m.blocks(ref)[b][:, g]
        assert np.all(np.isfinite(got))
        err = max(err, np.abs(got - want).max())
        scale = max(scale, np.abs(want).max())
    return err, scale


@pytest.mark.parametrize("centre", [(0.1, 0.2, 0.3), (7.9, 0.1, 0.2)])
@pytest.mark.parametrize("deg", [(2, 2, 2), (1, 0, 2), (0, 2, 1)])
def test_two_ghost_transfer_exact_on_quadratics(oracle, centre, deg):
    """Interior refined region and one touching the x = +8 face (the
    3-point prolongation stencil shifted by one into the domain)."""
    m = two_level(oracle, order=2, centre=centre)
    assert m.ghosts == 2
    p = lambda X, Y, Z: (0.3 + X) ** deg[0] * (0.2 - Y) ** deg[1] * (0.1 + Z) ** deg[2]
    err, scale = _max_ghost_error(m, p)
    assert err <= 1e-12 * scale, (err, scale)


def test_two_ghost_transfer_not_exact_on_cubics(oracle):
    m = two_level(oracle, order=2)
    err, _ = _max_ghost_error(m, lambda X, Y, Z: (0.3 + X) ** 3)
    assert err > 1e-6


@pytest.mark.parametrize("centre", [(0.1, 0.2, 0.3), (7.9, 0.1, 0.2)])
def test_two_ghost_transfer_converges_at_third_order(oracle, centre):
    fn = lambda X, Y, Z: np.sin(0.6 * X + 0.3) * np.cos(0.5 * Y - 0.2) * np.sin(0.4 * Z + 0.7)
    errs = [_max_ghost_error(two_level(oracle, n=n, order=2, centre=centre, radius=0.5 * 8 / n), fn,
                             fine_only=True)[0] for n in (8, 16)]
    rate = np.log2(errs[0] / errs[1])
    assert 2.5 < rate < 4.0, (errs, rate)
