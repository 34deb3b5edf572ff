"""Closed-form spacetimes, conformally decomposed with sympy (test-only).

Given a lapse alpha, shift beta^i and spatial metric gamma_ij as explicit
functions of (t, x, y, z), this derives the 22 Z4c variables and their exact
time derivatives, independently of the oracle's code:
  K_ij   = -(d_t gamma_ij - D_i beta_j - D_j beta_i) / (2 alpha)
  chi    = det(gamma)^(-1/3),  gt_ij = chi gamma_ij,  K = gamma^ij K_ij
  At_ij  = chi (K_ij - gamma_ij K / 3),  Khat = K,  Theta = 0
  Gam^i  = -d_j gt^ij
These are the standard conformal decomposition used by the Z4c system
(Sec. 2 of the paper defers the details to the GR-Athena++ paper).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import sympy as sp

NF = 22
x, y, z, t = sp.symbols("x y z t", real=True)
XS = (x, y, z)
SYM = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def _decompose(alpha, beta_u, gamma):
    g = sp.Matrix(3, 3, lambda i, j: gamma[i][j])
    detg = g.det()
    adj = g.adjugate()
    gi = adj / detg
    # Christoffel symbols of gamma
    dg = [[[sp.diff(g[i, j], XS[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    Gam = [[[sum(gi[k, l] * (dg[l][i][j] + dg[l][j][i] - dg[i][j][l]) for l in range(3)) / 2
             for j in range(3)] for i in range(3)] for k in range(3)]
    beta_d = [sum(g[i, j] * beta_u[j] for j in range(3)) for i in range(3)]
    Db = [[sp.diff(beta_d[j], XS[i]) - sum(Gam[k][i][j] * beta_d[k] for k in range(3))
           for j in range(3)] for i in range(3)]
    K = [[-(sp.diff(g[i, j], t) - Db[i][j] - Db[j][i]) / (2 * alpha) for j in range(3)]
         for i in range(3)]
    trK = sum(gi[i, j] * K[i][j] for i in range(3) for j in range(3))
    chi = detg ** sp.Rational(-1, 3)
    gt = [[chi * g[i, j] for j in range(3)] for i in range(3)]
    At = [[chi * (K[i][j] - g[i, j] * trK / 3) for j in range(3)] for i in range(3)]
    gti = [[gi[i, j] / chi for j in range(3)] for i in range(3)]
    Gamt = [-sum(sp.diff(gti[i][j], XS[j]) for j in range(3)) for i in range(3)]
    fields = [chi] + [gt[i][j] for i, j in SYM] + [trK] + [At[i][j] for i, j in SYM] + \
        Gamt + [sp.Integer(0), alpha] + list(beta_u)
    return fields


def _spacetime(kind: str, params: tuple):
    """(alpha, beta^i, gamma_ij) of a named closed-form spacetime."""
    if kind == "gauge_wave":
        A, d = params
        H = 1 - A * sp.sin(2 * sp.pi * (x - t) / d)
        return sp.sqrt(H), [0, 0, 0], [[H, 0, 0], [0, 1, 0], [0, 0, 1]]
    if kind in ("linear_wave", "linear_wave_in"):
        # TT wave along +x (linear_wave) or -x (linear_wave_in)
        A, d = params
        a = A * sp.sin(2 * sp.pi * (x - t if kind == "linear_wave" else x + t) / d)
        return sp.Integer(1), [0, 0, 0], [[1, 0, 0], [0, 1 + a, 0], [0, 0, 1 - a]]
    if kind == "kerr_schild":
        (M,) = params
        r = sp.sqrt(x * x + y * y + z * z)
        Hs = M / r
        l = [x / r, y / r, z / r]
        gamma = [[sp.KroneckerDelta(i, j) + 2 * Hs * l[i] * l[j] for j in range(3)] for i in range(3)]
        return 1 / sp.sqrt(1 + 2 * Hs), [2 * Hs / (1 + 2 * Hs) * l[i] for i in range(3)], gamma
    raise KeyError(kind)


def _weyl_parts(alpha, beta_u, gamma):
    """Electric and magnetic parts of the Weyl tensor of a vacuum 3+1 slice,
    from the ADM variables directly (no conformal decomposition):
      E_ij = R_ij + K K_ij - K_ik gamma^kl K_lj,
      B_ij = sym(gamma_im eps^mkl D_k K_lj),  eps^mkl = [mkl] / sqrt(det gamma),
    with K_ij = -(d_t gamma_ij - D_i beta_j - D_j beta_i) / (2 alpha)."""
    g = sp.Matrix(3, 3, lambda i, j: gamma[i][j])
    detg = g.det()
    gi = g.adjugate() / detg
    dg = [[[sp.diff(g[i, j], XS[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    Gam = [[[sum(gi[k, l] * (dg[l][i][j] + dg[l][j][i] - dg[i][j][l]) for l in range(3)) / 2
             for j in range(3)] for i in range(3)] for k in range(3)]
    beta_d = [sum(g[i, j] * beta_u[j] for j in range(3)) for i in range(3)]
    Db = [[sp.diff(beta_d[j], XS[i]) - sum(Gam[k][i][j] * beta_d[k] for k in range(3))
           for j in range(3)] for i in range(3)]
    K = [[-(sp.diff(g[i, j], t) - Db[i][j] - Db[j][i]) / (2 * alpha) for j in range(3)]
         for i in range(3)]
    trK = sum(gi[i, j] * K[i][j] for i in range(3) for j in range(3))
    Ric = [[sum(sp.diff(Gam[k][i][j], XS[k]) - sp.diff(Gam[k][i][k], XS[j]) +
                sum(Gam[k][k][l] * Gam[l][i][j] - Gam[k][j][l] * Gam[l][i][k] for l in range(3))
                for k in range(3)) for j in range(3)] for i in range(3)]
    E = [[Ric[i][j] + trK * K[i][j] - sum(K[i][k] * gi[k, l] * K[l][j] for k in range(3) for l in range(3))
          for j in range(3)] for i in range(3)]
    DK = [[[sp.diff(K[l][j], XS[k]) - sum(Gam[m][k][l] * K[m][j] + Gam[m][k][j] * K[l][m] for m in range(3))
            for j in range(3)] for l in range(3)] for k in range(3)]
    sq = sp.sqrt(detg)
    Bt = [[sum(g[i, m] * sp.LeviCivita(m, k, l) / sq * DK[k][l][j]
               for m in range(3) for k in range(3) for l in range(3)) for j in range(3)] for i in range(3)]
    B = [[(Bt[i][j] + Bt[j][i]) / 2 for j in range(3)] for i in range(3)]
    return [E[i][j] for i, j in SYM] + [B[i][j] for i, j in SYM] + [g[i, j] for i, j in SYM]


@lru_cache(maxsize=None)
def _compiled_weyl(kind: str, params: tuple):
    return sp.lambdify((t, x, y, z), _weyl_parts(*_spacetime(kind, params)), modules="numpy", cse=True)


def weyl(kind: str, params: tuple, X, Y, Z, time: float = 0.0):
    """(E, B, gamma) at the points: three (3, 3) + X.shape arrays."""
    vals = _compiled_weyl(kind, tuple(params))(time, X, Y, Z)
    v = [np.broadcast_to(np.asarray(q, dtype=float), X.shape) for q in vals]
    out = []
    for base in (0, 6, 12):
        T = np.zeros((3, 3) + X.shape)
        for q, (i, j) in enumerate(SYM):
            T[i, j] = T[j, i] = v[base + q]
        out.append(T)
    return out


@lru_cache(maxsize=None)
def _compiled(kind: str, params: tuple):
    fields = _decompose(*_spacetime(kind, params))
    dfields = [sp.diff(f, t) for f in fields]
    fn = sp.lambdify((t, x, y, z), fields, modules="numpy", cse=True)
    dfn = sp.lambdify((t, x, y, z), dfields, modules="numpy", cse=True)
    return fn, dfn


def evaluate(kind: str, params: tuple, X, Y, Z, time: float = 0.0, dt: bool = False) -> np.ndarray:
    """(22,) + X.shape array of the fields (or of their time derivatives)."""
    fn, dfn = _compiled(kind, tuple(params))
    vals = (dfn if dt else fn)(time, X, Y, Z)
    return np.stack([np.broadcast_to(np.asarray(v, dtype=float), X.shape) for v in vals])


def state_on_mesh(mesh, kind, params, time=0.0, dt=False) -> np.ndarray:
    """Flat state array in the oracle's layout, every storage cell filled."""
    u = mesh.zeros()
    for b, blk in enumerate(mesh.blocks(u)):
        X, Y, Z = mesh.centres(b)
        blk[...] = evaluate(kind, params, X, Y, Z, time, dt)
    return u


# ---------------------------------------------------------------------------
# A spatially constant Z4c state with linear Khat and Theta along x, and the
# closed form of its right-hand side (the standard Z4c equations reduced to
# algebra: every other derivative vanishes; see test_oracle_rhs.py)
# ---------------------------------------------------------------------------
CONST_STATE = dict(kh=0.31, th=-0.12, gam=(0.05, -0.02, 0.03), beta=(0.2, -0.1, 0.05),
                   At=((0.04, 0.015, -0.01), (0.015, -0.025, 0.02), (-0.01, 0.02, -0.015)))


def constant_z4c_state(mesh, a=0.0, c=0.0, alpha0=1.0, chi0=1.0):
    """Every storage cell of every block: gt = delta, chi = chi0, alpha =
    alpha0, constant Gam, beta and trace-free At, Khat = kh + a x,
    Theta = th + c x."""
    P = CONST_STATE
    At = np.array(P["At"])
    u = mesh.zeros()
    for b, B in enumerate(mesh.blocks(u)):
        X = mesh.centres(b)[0]
        B[0] = chi0
        for q, (i, j) in enumerate(SYM):
            B[1 + q] = 1.0 if i == j else 0.0
            B[8 + q] = At[i, j]
        B[7], B[17], B[18] = P["kh"] + a * X, P["th"] + c * X, alpha0
        for i in range(3):
            B[14 + i], B[19 + i] = P["gam"][i], P["beta"][i]
    return u


def constant_z4c_rhs(x, a, c, kappa1, kappa2, eta, lapse, alpha0=1.0, chi0=1.0):
    """(22, len(x)) right-hand side of constant_z4c_state at cells with
    coordinate x (K = Khat + 2 Theta at the cell, indices moved with delta).
    Every derivative of chi, alpha, gt, Gam and beta vanishes, so R_ij = 0,
    D_i D_j alpha = 0 and Gam_d = 0; the lapse alpha0 multiplies every term
    the Z4c equations (Sec. 2) carry it on, and chi0 enters only d_t chi."""
    P = CONST_STATE
    At, gam, beta = np.array(P["At"]), np.array(P["gam"]), np.array(P["beta"])
    al = alpha0
    kh, th = P["kh"] + a * x, P["th"] + c * x
    K = kh + 2 * th
    AA, A2 = float(np.sum(At * At)), At @ At
    w = np.zeros((22, np.size(x)))
    w[0] = 2.0 / 3.0 * chi0 * al * K
    for q, (i, j) in enumerate(SYM):
        w[1 + q] = -2.0 * al * At[i, j]
        w[8 + q] = al * (K * At[i, j] - 2.0 * A2[i, j])
    w[7] = al * (AA + K * K / 3.0) + kappa1 * (1.0 - kappa2) * al * th + beta[0] * a
    w[17] = 0.5 * al * (2.0 / 3.0 * K * K - AA) - al * kappa1 * (2.0 + kappa2) * th + beta[0] * c
    for i in range(3):
        w[14 + i] = -2.0 * al * kappa1 * gam[i] - (2.0 / 3.0 * al * (2 * a + c) if i == 0 else 0.0)
        w[19 + i] = gam[i] - eta * beta[i]
    w[18] = -2.0 * al * kh if lapse == 1 else -al * al * kh
    return w
