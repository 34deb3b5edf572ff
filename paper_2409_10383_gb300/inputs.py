"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the method: only mesh shapes (block
lists), parameter sets and seeded random perturbations.  Both sides build
their own meshes from these descriptions; random numbers are drawn here and
passed to both sides as plain arrays.

Workloads (shapes and values follow the paper's test problems, Secs. 4-5):
  gauge_wave_32     one 32^3 block, 3 ghosts, periodic [-1/2,1/2]^3, order 4,
                    KO 0.02, harmonic lapse, frozen zero shift, A = 0.01
  single_puncture   128^3 as 2x2x2 blocks of 64^3, 4 ghosts, [-16,16]^3,
                    Sommerfeld outer boundary, order 6, KO 0.5, 1+log,
                    Gamma-driver eta = 2, kappa1 = 0.02, Schwarzschild M = 1
                    with pre-collapsed lapse
  uneven_batch      seeded instances of mixed sizes (see uneven_batch())
"""
from __future__ import annotations

import numpy as np

NF = 22
SEED = 20240916

# initial-data kinds understood by both sides
ID_FLAT, ID_GAUGE_WAVE, ID_LINEAR_WAVE, ID_SCHWARZSCHILD, ID_BRILL_LINDQUIST = 0, 1, 2, 3, 4


def uniform_blocks(nb=(1, 1, 1), n=32, dom_lo=(-0.5,) * 3, dom_hi=(0.5,) * 3):
    """nb[0] x nb[1] x nb[2] equal blocks covering the box; returns (n, lo, h) arrays."""
    n3 = np.array((n, n, n) if np.isscalar(n) else n, dtype=np.int64)
    L = np.array(dom_hi, float) - np.array(dom_lo, float)
    hs = L / (np.array(nb) * n3)
    if not np.allclose(hs, hs[0]):
        raise ValueError("blocks must have cubic cells")
    h = float(hs[0])
    ns, los = [], []
    for kb in range(nb[2]):
        for jb in range(nb[1]):
            for ib in range(nb[0]):
                ns.append(n3.copy())
                los.append([dom_lo[0] + ib * n3[0] * h, dom_lo[1] + jb * n3[1] * h,
                            dom_lo[2] + kb * n3[2] * h])
    return np.array(ns, np.int64), np.array(los, float), np.full(len(ns), h)


def workload(name: str) -> dict:
    """Named workload: mesh + parameters + initial data (no arithmetic of the method)."""
    if name == "gauge_wave_32":
        n, lo, h = uniform_blocks((1, 1, 1), 32)
        return dict(name=name, n=n, lo=lo, h=h, ghosts=3, order=4, periodic=True,
                    dom_lo=(-0.5,) * 3, dom_hi=(0.5,) * 3, lapse=0, shift=0, ko_sigma=0.02,
                    kappa1=0.0, kappa2=0.0, eta=0.0, chi_floor=1e-6, cfl=0.25, steps=10,
                    id_kind=ID_GAUGE_WAVE, id_par=[0.01, 1.0, 0.0])
    if name == "single_puncture_128":
        n, lo, h = uniform_blocks((2, 2, 2), 64, (-16.0,) * 3, (16.0,) * 3)
        return dict(name=name, n=n, lo=lo, h=h, ghosts=4, order=6, periodic=False,
                    dom_lo=(-16.0,) * 3, dom_hi=(16.0,) * 3, lapse=1, shift=1, ko_sigma=0.5,
                    kappa1=0.02, kappa2=0.0, eta=2.0, chi_floor=1e-6, cfl=0.25, steps=100,
                    id_kind=ID_SCHWARZSCHILD, id_par=[1.0, 0.0])
    if name.startswith("single_puncture_"):
        # same physics at a smaller size: single_puncture_<N>_<nb>
        _, _, N, nb = name.split("_")
        N, nb = int(N), int(nb)
        n, lo, h = uniform_blocks((nb, nb, nb), N // nb, (-16.0,) * 3, (16.0,) * 3)
        return dict(name=name, n=n, lo=lo, h=h, ghosts=4, order=6, periodic=False,
                    dom_lo=(-16.0,) * 3, dom_hi=(16.0,) * 3, lapse=1, shift=1, ko_sigma=0.5,
                    kappa1=0.02, kappa2=0.0, eta=2.0, chi_floor=1e-6, cfl=0.25, steps=100,
                    id_kind=ID_SCHWARZSCHILD, id_par=[1.0, 0.0])
    raise KeyError(name)


def noise(size: int, seed: int, amp: float = 1.0) -> np.ndarray:
    """Uniform noise in [-amp, amp], seeded."""
    return np.random.default_rng(seed).uniform(-amp, amp, size)


def perturbation(shape_per_block, seed: int, amp: float) -> list:
    """Seeded random perturbation per block: a list of (22, ez, ey, ex) arrays
    of uniform noise in [-amp, amp].  Adding it to a state keeps gt SPD and
    chi, alpha positive as long as amp << 1."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(-amp, amp, (NF,) + tuple(s)) for s in shape_per_block]


def _instance(kind, n, order, precision, value):
    """One single-block problem: a puncture of mass `value` on [-16,16]^3 with
    the Sommerfeld boundary, or a gauge wave of amplitude `value` on the
    periodic [-1/2,1/2]^3; 4 or 6th order, FP64 or FP32-RHS."""
    if kind == "puncture":
        L, per, ko = 16.0, False, 0.5
        idk, idp = ID_SCHWARZSCHILD, [value, 0.0]
        lapse, shift, eta, k1 = 1, 1, 2.0, 0.02
    else:
        L, per, ko = 0.5, True, 0.02
        idk, idp = ID_GAUGE_WAVE, [value, 1.0, 0.0]
        lapse, shift, eta, k1 = 0, 0, 0.0, 0.0
    nn, lo, h = uniform_blocks((1, 1, 1), n, (-L,) * 3, (L,) * 3)
    return dict(name=f"{kind}_{n}", n=nn, lo=lo, h=h, ghosts=order // 2 + 1, order=order, periodic=per,
                dom_lo=(-L,) * 3, dom_hi=(L,) * 3, lapse=lapse, shift=shift, ko_sigma=ko, kappa1=k1,
                kappa2=0.0, eta=eta, chi_floor=1e-6, cfl=0.25, id_kind=idk, id_par=idp,
                precision=precision)


def uneven_batch(seed: int = SEED, sizes=(24, 48, 64, 96), n_puncture=64, n_wave=16):
    """The uneven batch: 64 single-puncture instances with seeded masses in
    [0.5, 2] and seeded sizes from {24, 48, 64, 96}^3, plus 16 gauge-wave
    instances with seeded amplitudes in [0.001, 0.1]; the instance index
    alternates the order (even: 6, odd: 4) and, in pairs, the precision
    (FP64, FP64, FP32, FP32, ...).  Draws in the order instance -> size ->
    mass/amplitude.  Returns a list of single-instance workloads."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_puncture + n_wave):
        n = int(sizes[rng.integers(0, len(sizes))])
        kind = "puncture" if i < n_puncture else "gauge_wave"
        value = float(rng.uniform(0.5, 2.0)) if kind == "puncture" else float(rng.uniform(0.001, 0.1))
        out.append(_instance(kind, n, 6 if i % 2 == 0 else 4, 64 if (i // 2) % 2 == 0 else 32, value))
    return out


def uneven_batch_small(seed: int = SEED):
    """The same mix at test size: 6 punctures and 2 gauge waves of 8..20^3."""
    return uneven_batch(seed, sizes=(8, 12, 16, 20), n_puncture=6, n_wave=2)


# ---------------------------------------------------------------------------
# static mesh refinement: oct-tree of equal MeshBlocks (paper Sec. 3, 2:1)
# ---------------------------------------------------------------------------
def _touch(a_lo, a_hi, b_lo, b_hi, tol):
    """Boxes touch or overlap (faces, edges, corners count)."""
    return all(a_lo[d] <= b_hi[d] + tol and b_lo[d] <= a_hi[d] + tol for d in range(3))


def octree_mesh(root_nb, n, dom_lo, dom_hi, centres, radii, max_level, reach=None):
    """Leaves of an oct-tree of n^3-cell blocks over the box.  A leaf at level
    L < max_level is refined while its box lies within radii[L] of one of the
    centres; then 2:1 balance is enforced (a leaf touching a leaf two levels
    finer, across a face, edge or corner, is refined), and every coarse leaf
    that the prolongation stencil of a finer neighbour would need two levels
    apart (within `reach` coarse cells of the fine block, default n/4 + 2) is
    refined too.  Returns (n, lo, h, level) arrays for the leaves, sorted by
    level then position."""
    dom_lo = np.asarray(dom_lo, float)
    dom_hi = np.asarray(dom_hi, float)
    h0 = (dom_hi[0] - dom_lo[0]) / (root_nb[0] * n)
    reach = n // 4 + 2 if reach is None else reach
    leaves = set()
    for k in range(root_nb[2]):
        for j in range(root_nb[1]):
            for i in range(root_nb[0]):
                leaves.add((0, i, j, k))

    def box(leaf):
        L, i, j, k = leaf
        w = n * h0 / 2 ** L
        lo = dom_lo + np.array([i, j, k]) * w
        return lo, lo + w

    def dist(leaf, c):
        lo, hi = box(leaf)
        d = np.maximum(0.0, np.maximum(lo - c, c - hi))
        return float(np.sqrt((d * d).sum()))

    def refine(leaf):
        L, i, j, k = leaf
        leaves.discard(leaf)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    leaves.add((L + 1, 2 * i + di, 2 * j + dj, 2 * k + dk))

    for L in range(max_level):
        for leaf in [f for f in leaves if f[0] == L]:
            if any(dist(leaf, np.asarray(c, float)) < radii[L] for c in centres):
                refine(leaf)
    changed = True
    while changed:
        changed = False
        ls = sorted(leaves)
        boxes = {f: box(f) for f in ls}
        for a in ls:
            if a not in leaves:
                continue
            alo, ahi = boxes[a]
            for b in ls:
                if b not in leaves or b[0] <= a[0]:
                    continue
                blo, bhi = boxes[b]
                wb = n * h0 / 2 ** b[0]
                if b[0] >= a[0] + 2 and _touch(alo, ahi, blo, bhi, 1e-9 * wb):
                    refine(a)
                    changed = True
                    break
                if b[0] == a[0] + 1:
                    # b's prolongation reads a's cells within `reach` coarse cells;
                    # those must not be two levels finer than a: any leaf of
                    # level >= b+1 there forces a refinement of a
                    hc = 2 * wb / n
                    grow = reach * hc
                    if _touch(alo, ahi, blo - grow, bhi + grow, 1e-9 * wb):
                        for c in ls:
                            if c in leaves and c[0] >= b[0] + 1:
                                clo, chi = boxes[c]
                                if _touch(clo, chi, blo - grow, bhi + grow, 1e-9 * wb) and \
                                        _touch(clo, chi, alo, ahi, 1e-9 * wb):
                                    refine(a)
                                    changed = True
                                    break
                        if changed:
                            break
            if changed:
                break
    ls = sorted(leaves)
    ns, los, hs, lev = [], [], [], []
    for f in ls:
        lo, _ = box(f)
        ns.append([n, n, n])
        los.append(lo)
        hs.append(h0 / 2 ** f[0])
        lev.append(f[0])
    return (np.array(ns, np.int64), np.array(los, float), np.array(hs, float), np.array(lev, np.int64))
