"""Pins for the oracle's finite-difference operators (Sec. 3, Sec. 4.3).

Each stencil must be exact on polynomials up to its design degree and must
NOT be exact one degree higher (so a wrong coefficient or offset fails), and
must converge at its order on sinusoids.  KO dissipation must annihilate
polynomials of degree < 2N and damp the grid Nyquist mode at rate sigma/h.
Orders 2, 4 and 6 (2nd order: the paper's default with 2 ghosts).
"""
import math

import numpy as np
import pytest

H = 0.37
NPT = 13
C = NPT // 2


def grid():
    a = (np.arange(NPT) - C) * H + 0.11
    Z, Y, X = np.meshgrid(a, a, a, indexing="ij")
    return X, Y, Z


def mono(e):
    X, Y, Z = grid()
    return X ** e[0] * Y ** e[1] * Z ** e[2]


def dmono(e, dirs):
    """exact derivative of x^a y^b z^c at the centre point"""
    e = list(e)
    coef = 1.0
    for d in dirs:
        if e[d] == 0:
            return 0.0
        coef *= e[d]
        e[d] -= 1
    x0 = np.array([0.11, 0.11, 0.11])
    return coef * np.prod(x0 ** np.array(e))


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_first_derivative_exactness(oracle, order, d):
    for deg in range(order + 2):
        e = [0, 0, 0]
        e[d] = deg
        got = oracle.fd(0, order, mono(e), C, C, C, d, h=H)
        ref = dmono(e, [d])
        if deg <= order:
            assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (deg, got, ref)
        else:
            assert abs(got - ref) > 1e-8, "stencil exact beyond its order"


@pytest.mark.parametrize("order", [2, 4, 6])
def test_second_derivative_exactness(oracle, order):
    for d in range(3):
        for deg in range(order + 3):
            e = [0, 0, 0]
            e[d] = deg
            got = oracle.fd(1, order, mono(e), C, C, C, d, h=H)
            ref = dmono(e, [d, d])
            if deg <= order + 1:
                assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (d, deg, got, ref)
            else:
                assert abs(got - ref) > 1e-8


@pytest.mark.parametrize("order", [2, 4, 6])
def test_mixed_derivative_exactness(oracle, order):
    for (a, b) in [(0, 1), (0, 2), (1, 2), (1, 0)]:
        for da in range(order + 1):
            for db in range(order + 1):
                e = [0, 0, 0]
                e[a], e[b] = da, db
                got = oracle.fd(2, order, mono(e), C, C, C, a, b, h=H)
                ref = dmono(e, [a, b])
                assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (a, b, da, db)
        e = [0, 0, 0]
        e[a], e[b] = order + 1, 1
        got = oracle.fd(2, order, mono(e), C, C, C, a, b, h=H)
        assert abs(got - dmono(e, [a, b])) > 1e-8


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_lopsided_exactness(oracle, order, sign):
    for d in range(3):
        for deg in range(order + 2):
            e = [0, 0, 0]
            e[d] = deg
            got = oracle.fd(3, order, mono(e), C, C, C, d, h=H, arg=sign)
            ref = dmono(e, [d])
            if deg <= order:
                assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (d, deg)
            else:
                assert abs(got - ref) > 1e-8


@pytest.mark.parametrize("order", [2, 4, 6])
def test_lopsided_leans_upwind(oracle, order):
    """A spike just on the + side changes the beta>0 derivative, a spike the
    same distance on the - side beyond the stencil's short arm does not."""
    N = order // 2 + 1
    f = np.zeros((NPT, NPT, NPT))
    f[C, C, C + N] = 1.0      # farthest + point of the beta>0 stencil
    assert oracle.fd(3, order, f, C, C, C, 0, h=1.0, arg=1.0) != 0.0
    assert oracle.fd(3, order, f, C, C, C, 0, h=1.0, arg=-1.0) == 0.0
    g = np.zeros((NPT, NPT, NPT))
    g[C, C, C - N] = 1.0
    assert oracle.fd(3, order, g, C, C, C, 0, h=1.0, arg=-1.0) != 0.0
    assert oracle.fd(3, order, g, C, C, C, 0, h=1.0, arg=1.0) == 0.0


@pytest.mark.parametrize("order", [2, 4, 6])
def test_kreiss_oliger(oracle, order):
    N = order // 2 + 1
    sigma = 0.7
    for d in range(3):
        for deg in range(2 * N + 1):
            e = [0, 0, 0]
            e[d] = deg
            got = oracle.fd(4, order, mono(e), C, C, C, d, h=H, arg=sigma)
            if deg < 2 * N:
                assert abs(got) <= 1e-9 * max(1.0, np.abs(mono(e)).max()), (d, deg, got)
            else:
                assert abs(got) > 1e-6
        # Nyquist mode (-1)^i is damped at rate sigma / h
        idx = np.indices((NPT, NPT, NPT))[2 - d]
        f = (-1.0) ** idx
        got = oracle.fd(4, order, f, C, C, C, d, h=H, arg=sigma)
        assert got == pytest.approx(-sigma / H * f[C, C, C], rel=1e-13)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_convergence_on_sinusoids(oracle, order):
    """sin(k x + l y + m z): errors of every operator fall like h^order."""
    kv = np.array([1.1, -0.7, 0.9])
    x0 = np.array([0.3, -0.2, 0.1])
    errs = {}
    hs = (0.3, 0.15, 0.075) if order == 6 else (0.1, 0.05, 0.025)
    for h in hs:
        a = (np.arange(NPT) - C) * h
        Z, Y, X = np.meshgrid(a + x0[2], a + x0[1], a + x0[0], indexing="ij")
        f = np.sin(kv[0] * X + kv[1] * Y + kv[2] * Z)
        ph = kv @ x0
        res = []
        for d in range(3):
            res.append(oracle.fd(0, order, f, C, C, C, d, h=h) - kv[d] * math.cos(ph))
            res.append(oracle.fd(1, order, f, C, C, C, d, h=h) + kv[d] ** 2 * math.sin(ph))
            res.append(oracle.fd(3, order, f, C, C, C, d, h=h, arg=1.0) - kv[d] * math.cos(ph))
            res.append(oracle.fd(3, order, f, C, C, C, d, h=h, arg=-1.0) - kv[d] * math.cos(ph))
            b = (d + 1) % 3
            res.append(oracle.fd(2, order, f, C, C, C, d, b, h=h) + kv[d] * kv[b] * math.sin(ph))
        errs[h] = np.abs(res)
    r1 = np.log2(errs[hs[0]] / errs[hs[1]])
    r2 = np.log2(errs[hs[1]] / errs[hs[2]])
    assert np.all(r2 > order - 0.3), (r1, r2)
    assert np.all(r2 < order + 1.3), (r1, r2)
