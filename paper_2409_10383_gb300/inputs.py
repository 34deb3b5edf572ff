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
  bl_binary_smr     two Brill-Lindquist punctures (m = 1/2 at x = +-3) on an
                    oct-tree of 16^3 blocks, 2x2x2 roots at h = 2 over
                    [-32,32]^3, 6 refinement levels down to h = 1/32, 4
                    ghosts, order 6, puncture gauge, Sommerfeld boundary,
                    dt = 1/128 for every block (680 blocks; see octree_mesh)
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
    """Named workload: mesh + parameters + initial data (no arithmetic of the method).
    A name ending in "_o2" is the same problem with 2nd-order differencing
    and 2 ghosts (the paper's default with 2 ghost cells)."""
    if name.endswith("_o2"):
        w = workload(name[:-3])
        w.update(name=name, order=2, ghosts=2)
        return w
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
    if name == "linear_wave_256":
        # The throughput workload of the paper's Table 1: the linear
        # gravitational wave (amplitude 1e-8, periodic) on 64^3 MeshBlocks,
        # 6th-order differencing and RK4; here 4 x 4 x 4 blocks (16.8 M
        # cells, well past what saturates the GPU) with the puncture gauge.
        # The paper's wave runs along the diagonal, this one along x: the
        # cost per cell is the same.
        n, lo, h = uniform_blocks((4, 4, 4), 64)
        return dict(name=name, n=n, lo=lo, h=h, ghosts=4, order=6, periodic=True,
                    dom_lo=(-0.5,) * 3, dom_hi=(0.5,) * 3, lapse=1, shift=1, ko_sigma=0.5,
                    kappa1=0.02, kappa2=0.0, eta=2.0, chi_floor=1e-6, cfl=0.25, steps=10,
                    id_kind=ID_LINEAR_WAVE, id_par=[1e-8, 1.0, 0.0])
    if name.startswith("bl_binary_smr"):
        # bl_binary_smr[_<max_level>]: levels 0..max_level (default 6)
        parts = name.split("_")
        max_level = int(parts[3]) if len(parts) > 3 else 6
        n, lo, h, level = octree_mesh((2, 2, 2), 16, (-32.0,) * 3, (32.0,) * 3, BL_BINARY_CENTRES,
                                      BL_BINARY_RADII, max_level)
        return dict(name=name, n=n, lo=lo, h=h, level=level, ghosts=4, order=6, periodic=False,
                    dom_lo=(-32.0,) * 3, dom_hi=(32.0,) * 3, lapse=1, shift=1, ko_sigma=0.5,
                    kappa1=0.02, kappa2=0.0, eta=2.0, chi_floor=1e-6, cfl=0.25, steps=50,
                    dt=0.25 * float(h.min()), id_kind=ID_BRILL_LINDQUIST,
                    id_par=[2.0, 0.5, 3.0, 0.0, 0.0, 0.5, -3.0, 0.0, 0.0])
    raise KeyError(name)


def mirror_blocks(n, lo, h):
    """For each block, the index of the block that is its image under
    x -> -x (KeyError if the mesh is not symmetric)."""
    key = {(round(lo[b, 0] / h[b]), round(lo[b, 1] / h[b]), round(lo[b, 2] / h[b]), round(np.log2(h[b]))): b
           for b in range(len(h))}
    out = []
    for b in range(len(h)):
        xm = -(lo[b, 0] + n[b, 0] * h[b])
        out.append(key[(round(xm / h[b]), round(lo[b, 1] / h[b]), round(lo[b, 2] / h[b]), round(np.log2(h[b])))])
    return np.array(out)


# Two punctures at x = +-3; a level-L block is refined when it comes within
# half its own width (16 / 2^L) of one.  Both punctures lie on block faces at
# every level, so any radius below the block width gives the same 680-block
# tree: the smallest 2:1-balanced tree that keeps each puncture inside the
# finest level on all sides.
BL_BINARY_CENTRES = [(3.0, 0.0, 0.0), (-3.0, 0.0, 0.0)]
BL_BINARY_RADII = [16.0 / 2 ** L for L in range(6)]


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


def mixed_order_batch_small(seed: int = SEED):
    """uneven_batch_small plus two 2nd-order (2 ghosts) instances: an FP64
    puncture of 12^3 and an FP32-RHS gauge wave of 16^3, so that all three
    differencing orders share one batch."""
    return uneven_batch_small(seed) + [_instance("puncture", 12, 2, 64, 1.0),
                                       _instance("gauge_wave", 16, 2, 32, 0.05)]


# ---------------------------------------------------------------------------
# static mesh refinement: oct-tree of equal MeshBlocks (paper Sec. 3, 2:1)
# ---------------------------------------------------------------------------
def octree_mesh(root_nb, n, dom_lo, dom_hi, centres, radii, max_level):
    """Leaves of an oct-tree of n^3-cell blocks over the box (Sec. 3.1).

    A leaf at level L < max_level is refined while its box comes within
    radii[L] of one of the centres; then, until nothing changes, a leaf is
    refined if it touches (face, edge or corner) a leaf two levels finer
    (2:1 balance).  For n >= 8 and ghost depth <= 4 this balance also keeps
    every prolongation stencil (ghost depth / 2 + 2 coarse cells beyond a
    fine block) inside leaves at most one level finer than the coarse
    neighbour, so no extra rule is needed.  Returns (n, lo, h, level) arrays
    for the leaves, sorted by level then position."""
    dom_lo = np.asarray(dom_lo, float)
    dom_hi = np.asarray(dom_hi, float)
    h0 = (dom_hi[0] - dom_lo[0]) / (root_nb[0] * n)
    leaves = {(0, i, j, k) for k in range(root_nb[2]) for j in range(root_nb[1]) for i in range(root_nb[0])}

    def boxes(ls):
        a = np.array(ls, dtype=np.int64).reshape(-1, 4)
        w = n * h0 / 2.0 ** a[:, 0]
        lo = dom_lo + a[:, [1, 2, 3]] * w[:, None]
        return a[:, 0], lo, lo + w[:, None], w

    def refine(leaf):
        L, i, j, k = leaf
        leaves.discard(leaf)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    leaves.add((L + 1, 2 * i + di, 2 * j + dj, 2 * k + dk))

    cs = np.asarray(centres, float).reshape(-1, 3)
    for L in range(max_level):
        ls = [f for f in leaves if f[0] == L]
        if not ls:
            continue
        _, lo, hi, _ = boxes(ls)
        d = np.maximum(0.0, np.maximum(lo[:, None, :] - cs[None], cs[None] - hi[:, None, :]))
        near = (np.sqrt((d * d).sum(-1)) < radii[L]).any(axis=1)
        for f, r in zip(ls, near):
            if r:
                refine(f)
    while True:
        ls = sorted(leaves)
        lev, lo, hi, w = boxes(ls)
        tol = 1e-9 * w.min()
        touch = np.all((lo[:, None, :] <= hi[None, :, :] + tol) & (lo[None, :, :] <= hi[:, None, :] + tol), axis=-1)
        bad = (touch & (lev[None, :] >= lev[:, None] + 2)).any(axis=1)
        if not bad.any():
            break
        for ia in np.where(bad)[0]:
            refine(ls[ia])
    ls = sorted(leaves)
    lev, lo, _, _ = boxes(ls)
    h = h0 / 2.0 ** lev
    return (np.tile(np.array([n, n, n], np.int64), (len(ls), 1)), lo, h, lev.astype(np.int64))
