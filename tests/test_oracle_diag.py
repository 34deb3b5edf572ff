"""Pins for the oracle's diagnostics beside the step: the refinement
indicators of Sec. 3.2 (per block min chi, max |grad chi|) and the puncture
tracker of Sec. 3.3 (dx/dt = -beta(x), 4-point Lagrange interpolation of
beta).  Checked against closed forms: fields whose gradient the centred
stencils take exactly, shift fields the cubic interpolation reproduces
exactly, and one degree above, where it does not."""
import numpy as np
import pytest

from paper_2409_10383_gb300 import inputs

NF = 22


def mesh(oracle, order=6, nb=(2, 2, 1), n=8, periodic=False, level=False):
    if level:
        nn, lo, h, lev = inputs.octree_mesh((2, 2, 2), n, (-1.0,) * 3, (1.0,) * 3, [(0.3, 0.2, 0.1)], [0.05], 1)
        return oracle.Mesh(n=nn, lo=lo, h=h, level=lev, ghosts=order // 2 + 1, order=order, dom_lo=(-1.0,) * 3,
                           dom_hi=(1.0,) * 3, periodic=periodic)
    return oracle.uniform_mesh(nb, n, order=order, dom_lo=(-1.0,) * 3, dom_hi=(1.0, 1.0, 0.0 if nb[2] == 1 else 1.0),
                               periodic=periodic)


def fill(m, fchi=None, fbeta=None):
    """State with chi and beta from closed forms at the cell centres (ghosts
    included, so no ghost fill is needed)."""
    u = m.zeros()
    for b, blk in enumerate(m.blocks(u)):
        X, Y, Z = m.centres(b)
        blk[0] = fchi(X, Y, Z) if fchi else 1.0
        if fbeta:
            for c in range(3):
                blk[19 + c] = fbeta(c, X, Y, Z)
    return u


@pytest.mark.parametrize("order", [2, 4, 6])
def test_indicators_linear_chi(oracle, order):
    """chi = 1 + a.x: every centred stencil gives grad chi = a exactly, and
    the minimum sits at the corner cell nearest -a."""
    m = mesh(oracle, order)
    a = np.array([0.3, -0.2, 0.15])
    u = fill(m, lambda X, Y, Z: 1.0 + a[0] * X + a[1] * Y + a[2] * Z)
    cmin, gmax = m.block_indicators(u)
    assert np.allclose(gmax, np.linalg.norm(a), rtol=1e-12, atol=0)
    for b in range(m.nblocks):
        mk = m.interior_mask(b)
        X, Y, Z = m.centres(b)
        want = (1.0 + a[0] * X + a[1] * Y + a[2] * Z)[mk].min()
        assert abs(cmin[b] - want) <= 1e-15


def test_indicators_quadratic_chi(oracle):
    """chi = 1 - r^2/2 (degree 2, so the 4th- and 6th-order stencils are
    exact): |grad chi| = r at each cell centre; the block maximum is the
    largest r of its interior cells."""
    for order in (4, 6):
        m = mesh(oracle, order)
        u = fill(m, lambda X, Y, Z: 1.0 - 0.5 * (X * X + Y * Y + Z * Z))
        cmin, gmax = m.block_indicators(u)
        for b in range(m.nblocks):
            mk = m.interior_mask(b)
            X, Y, Z = m.centres(b)
            r = np.sqrt(X * X + Y * Y + Z * Z)[mk]
            assert abs(gmax[b] - r.max()) <= 1e-12
            assert abs(cmin[b] - (1.0 - 0.5 * r.max() ** 2)) <= 1e-14


def test_indicators_see_the_gradient_not_one_degree_above(oracle):
    """A degree-7 chi along x defeats the 6th-order first derivative: the
    indicator then differs from the exact gradient (so it is not computed
    from anything but the stencil)."""
    m = mesh(oracle, 6)
    u = fill(m, lambda X, Y, Z: 1.0 + 0.01 * X ** 7)
    _, gmax = m.block_indicators(u)
    exact = []
    for b in range(m.nblocks):
        X, _, _ = m.centres(b)
        exact.append((0.07 * X ** 6)[m.interior_mask(b)].max())
    assert np.max(np.abs(gmax - np.array(exact))) > 1e-9


@pytest.mark.parametrize("level", [False, True])
def test_tracker_exact_on_cubic_shift(oracle, level):
    """beta = cubic polynomial per component: the 4-point Lagrange
    interpolation is exact, so one step moves the puncture by exactly
    -dt beta(x), on a uniform mesh and inside a refined block."""
    m = mesh(oracle, 6, nb=(2, 2, 2), level=level)
    coef = [(0.1, -0.2, 0.05), (0.03, 0.2, -0.1), (-0.07, 0.01, 0.3)]

    def beta(c, X, Y, Z):
        a, b2, c3 = coef[c]
        return a * X ** 3 + b2 * X * Y * Z + c3 * Z ** 2 * Y + 0.02 * c

    u = fill(m, fbeta=beta)
    pts = np.array([[0.31, 0.22, 0.11], [-0.52, 0.13, -0.77], [0.0101, -0.0203, 0.4]])
    dt = 0.05
    new, got = m.track_punctures(u, pts, dt)
    want = np.array([[beta(c, *p) for c in range(3)] for p in pts])
    assert np.allclose(got, want, rtol=0, atol=1e-14)
    assert np.allclose(new, pts - dt * want, rtol=0, atol=1e-15)


def test_tracker_not_exact_on_quartic_shift(oracle):
    m = mesh(oracle, 6, nb=(2, 2, 2))
    u = fill(m, fbeta=lambda c, X, Y, Z: X ** 4 if c == 0 else 0.0 * X)
    _, got = m.track_punctures(u, [[0.33, 0.1, 0.2]], 0.1)
    assert abs(got[0, 0] - 0.33 ** 4) > 1e-9


def test_tracker_constant_shift_and_outside(oracle):
    """A constant shift advects the puncture by -dt beta exactly over many
    steps; a puncture outside every block is an error."""
    m = mesh(oracle, 4, nb=(2, 2, 2))
    u = fill(m, fbeta=lambda c, X, Y, Z: 0.0 * X + (0.25, -0.5, 0.125)[c])
    x = np.array([[0.1, 0.2, -0.3]])
    for _ in range(10):
        x, _ = m.track_punctures(u, x, 0.1)
    assert np.allclose(x, [[0.1 - 0.25, 0.2 + 0.5, -0.3 - 0.125]], atol=1e-15)
    with pytest.raises(ValueError):
        m.track_punctures(u, [[3.0, 0.0, 0.0]], 0.1)
