"""Pins for the oracle's Weyl scalar Psi4 on the grid (Sec. 3.3: the
outgoing Weyl scalar computed with a coordinate tetrad; reading R20).

  - Against sympy: for the linear TT wave (non-zero E, B and K_ij
    derivatives) the electric and magnetic parts E_ij, B_ij are derived
    symbolically from the ADM variables (tests/analytic.py, no conformal
    variables, no code shared with the oracle); the tetrad and the
    contraction are redone here in numpy.  The oracle converges to that at
    the differencing order.
  - Physics that fixes the conventions: a wave travelling along +x has
    Psi4 = d_t^2 (h_yy - i h_yz) on the +x axis, one travelling along -x
    has none (a sign error in B or in the tetrad swaps the two).
  - Spherical symmetry: Schwarzschild in isotropic (time-symmetric) and in
    Kerr-Schild form (K_ij != 0, shift) has Psi4 = 0 in a radial tetrad; the
    oracle converges to 0.
  - Flat spacetime in wavy coordinates (the gauge wave): the Weyl tensor
    vanishes, so R_ij must cancel against K K_ij - K_ik K^k_j; Psi4 -> 0.
"""
import numpy as np
import pytest

import analytic as an
from paper_2409_10383_gb300 import inputs


def order_of(e):
    e = np.asarray(e, dtype=float)
    return np.log2(e[:-1] / e[1:])


def psi4_closed_form(kind, params, X, Y, Z, time=0.0):
    """(E - i B)(mb, mb) from the sympy E, B and gamma, with the tetrad of
    reading R20 built here: Gram-Schmidt in gamma on x^i, (-y, x, 0),
    (x z, y z, -(x^2 + y^2)); mb = (e_th - i e_ph) / sqrt(2)."""
    E, B, g = an.weyl(kind, params, X, Y, Z, time)
    u = [np.stack([X, Y, Z]), np.stack([-Y, X, 0 * X]), np.stack([X * Z, Y * Z, -(X * X + Y * Y)])]
    dot = lambda a, b: np.einsum("i...,ij...,j...->...", a, g, b)
    e = []
    for v in u:
        v = v.copy()
        for w in e:
            v = v - dot(w, v) * w
        e.append(v / np.sqrt(dot(v, v)))
    ph, th = e[1], e[2]
    mb = (th - 1j * ph) / np.sqrt(2.0)
    return np.einsum("i...,ij...,j...->...", mb, E - 1j * B, mb)


def interior_psi4(m, u):
    out = m.psi4(u)
    return [out[b][m.interior_mask(b)] for b in range(m.nblocks)]


def box_mesh(oracle, n, order, lo, hi, **kw):
    return oracle.uniform_mesh(n=n, order=order, periodic=False, dom_lo=lo, dom_hi=hi, **kw)


@pytest.mark.parametrize("order,ns", [(2, (8, 16, 32)), (4, (8, 16, 32)), (6, (6, 12, 24))])
def test_psi4_linear_wave_matches_sympy(oracle, order, ns):
    """A = 0.05, so that the terms quadratic in the wave (the K K parts of
    E_ij among them) are a few per cent of Psi4."""
    A, d, T = 0.05, 1.0, 0.13
    lo, hi = (0.3, 0.2, 0.25), (0.7, 0.6, 0.65)
    errs = []
    for n in ns:
        m = box_mesh(oracle, n, order, lo, hi)
        u = an.state_on_mesh(m, "linear_wave", (A, d), time=T)
        got = interior_psi4(m, u)[0]
        X, Y, Z = (c[m.interior_mask(0)] for c in m.centres(0))
        want = psi4_closed_form("linear_wave", (A, d), X, Y, Z, T)
        errs.append(np.abs(got - want).max() / np.abs(want).max())
    assert np.all(order_of(errs) > order - 0.5), errs
    assert errs[-1] < {2: 1e-2, 4: 1e-4, 6: 1e-6}[order], errs


def test_psi4_sees_the_outgoing_wave_only(oracle):
    """Near the +x axis (|y|, |z| <= 0.05 at x in [2, 3]) the outgoing wave
    gives Psi4 = d_t^2 h_yy = -(2 pi / d)^2 A sin(2 pi (x - t) / d) (real; the
    tetrad turns by at most 0.025 rad there), the ingoing one almost none."""
    A, d, T = 1e-4, 1.0, 0.2
    m = box_mesh(oracle, (40, 4, 4), 6, (2.0, -0.05, -0.05), (3.0, 0.05, 0.05))
    X, Y, Z = (c[m.interior_mask(0)] for c in m.centres(0))
    out = interior_psi4(m, an.state_on_mesh(m, "linear_wave", (A, d), time=T))[0]
    inn = interior_psi4(m, an.state_on_mesh(m, "linear_wave_in", (A, d), time=T))[0]
    hdd = -(2 * np.pi / d) ** 2 * A * np.sin(2 * np.pi * (X - T) / d)
    scale = np.abs(hdd).max()
    assert np.abs(out.real - hdd).max() <= 0.01 * scale
    assert np.abs(out.imag).max() <= 0.06 * scale
    assert np.abs(inn).max() <= 1e-3 * scale


@pytest.mark.parametrize("order", [4, 6])
def test_psi4_vanishes_for_schwarzschild(oracle, order):
    """Isotropic Schwarzschild (K_ij = 0) and Kerr-Schild (K_ij != 0, shift):
    Psi4 -> 0 at the differencing order, in a box off the axes."""
    lo, hi = (1.5, 1.2, 1.3), (2.5, 2.2, 2.3)
    ns = (8, 16, 32) if order == 4 else (6, 12, 24)
    iso, ks = [], []
    for n in ns:
        m = box_mesh(oracle, n, order, lo, hi)
        u = m.initial_data(inputs.ID_SCHWARZSCHILD, [1.0, 1])
        iso.append(np.abs(interior_psi4(m, u)[0]).max())
        u = an.state_on_mesh(m, "kerr_schild", (1.0,))
        ks.append(np.abs(interior_psi4(m, u)[0]).max())
    assert np.all(order_of(iso) > order - 0.6), iso
    assert np.all(order_of(ks) > order - 0.6), ks


@pytest.mark.parametrize("order", [2, 4, 6])
def test_psi4_vanishes_for_the_gauge_wave(oracle, order):
    A, d, T = 0.1, 1.0, 0.07
    lo, hi = (0.3, 0.2, 0.25), (0.7, 0.6, 0.65)
    ns = (6, 12, 24) if order == 6 else (8, 16, 32)
    errs, scale = [], []
    for n in ns:
        m = box_mesh(oracle, n, order, lo, hi)
        u = an.state_on_mesh(m, "gauge_wave", (A, d), time=T)
        errs.append(np.abs(interior_psi4(m, u)[0]).max())
    # d_t^2 of the metric is (2 pi / d)^2 A ~ 4: Psi4 is truncation error only
    assert np.all(order_of(errs) > order - 0.6), errs
    assert errs[-1] < {2: 2e-2, 4: 1e-4, 6: 1e-6}[order], errs


def test_psi4_is_zero_outside_the_interior(oracle):
    m = box_mesh(oracle, 8, 4, (0.3, 0.2, 0.25), (0.7, 0.6, 0.65))
    u = an.state_on_mesh(m, "linear_wave", (1e-3, 1.0), time=0.1)
    out = m.psi4(u)[0]
    assert np.all(out[~m.interior_mask(0)] == 0) and np.all(out[m.interior_mask(0)] != 0)
