"""ctypes wrapper around the plain FP64 CPU oracle (oracle/z4c_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path never imports
it.  It shares no code with the CUDA path; both sides only share the seeded
input generators in ``paper_2409_10383_gb300/inputs.py``.

Layout of a state array: for each block (in order) and each of the 22 fields,
an (n_z+2g, n_y+2g, n_x+2g) array, i fastest, blocks concatenated.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

NF = 22
FIELDS = ("chi", "gxx", "gxy", "gxz", "gyy", "gyz", "gzz", "Khat",
          "Axx", "Axy", "Axz", "Ayy", "Ayz", "Azz", "Gamx", "Gamy", "Gamz",
          "Theta", "alpha", "betax", "betay", "betaz")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "z4c_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int32), ("ghosts", ctypes.c_int32), ("order", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("lapse", ctypes.c_int32), ("shift", ctypes.c_int32),
                ("dom_lo", ctypes.c_double * 3), ("dom_hi", ctypes.c_double * 3),
                ("ko_sigma", ctypes.c_double), ("kappa1", ctypes.c_double),
                ("kappa2", ctypes.c_double), ("eta", ctypes.c_double),
                ("chi_floor", ctypes.c_double),
                ("n", ctypes.POINTER(ctypes.c_int32)), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(ctypes.c_double)),
                ("level", ctypes.POINTER(ctypes.c_int32))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        mp = ctypes.POINTER(_Mesh)
        sig = {
            "orc_state_size": (L, [mp]),
            "orc_fd": (D, [I, I, P, I, I, I, I, I, I, I, I, D, D]),
            "orc_rhs": (None, [mp, P, P]),
            "orc_rhs_cells": (None, [mp, P, P, L, P]),
            "orc_fill_ghosts": (I, [mp, P]),
            "orc_enforce": (None, [mp, P]),
            "orc_rk4_step": (I, [mp, P, D, I]),
            "orc_constraints": (None, [mp, P, D, P, P]),
            "orc_initial_data": (None, [mp, P, I, P]),
            "orc_set_threads": (I, [I]),
            "orc_block_indicators": (None, [mp, P, P, P]),
            "orc_track_punctures": (I, [mp, P, I, P, D, P]),
            "orc_psi4": (None, [mp, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Mesh:
    """A pack of uniform-spacing MeshBlocks on one Mesh (Sec. 3)."""
    n: np.ndarray            # (nb, 3) interior cells
    lo: np.ndarray           # (nb, 3) lower corner of active region
    h: np.ndarray            # (nb,)
    ghosts: int
    order: int
    dom_lo: tuple
    dom_hi: tuple
    periodic: bool
    lapse: int = 1           # 0 harmonic, 1 one-plus-log
    shift: int = 1           # 0 frozen, 1 Gamma-driver
    ko_sigma: float = 0.0
    kappa1: float = 0.0
    kappa2: float = 0.0
    eta: float = 2.0
    chi_floor: float = 1e-6
    level: np.ndarray = None  # (nb,) refinement level per block, or None (all 0)
    _c: _Mesh = field(default=None, repr=False)

    def __post_init__(self):
        self.n = np.ascontiguousarray(self.n, dtype=np.int32).reshape(-1, 3)
        self.lo = np.ascontiguousarray(self.lo, dtype=np.float64).reshape(-1, 3)
        self.h = np.ascontiguousarray(self.h, dtype=np.float64).reshape(-1)
        c = _Mesh()
        c.nblocks = len(self.h)
        c.ghosts, c.order = self.ghosts, self.order
        c.periodic, c.lapse, c.shift = int(self.periodic), self.lapse, self.shift
        c.dom_lo[:] = list(self.dom_lo)
        c.dom_hi[:] = list(self.dom_hi)
        c.ko_sigma, c.kappa1, c.kappa2 = self.ko_sigma, self.kappa1, self.kappa2
        c.eta, c.chi_floor = self.eta, self.chi_floor
        c.n = self.n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c.lo = self.lo.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.h = self.h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if self.level is not None:
            self.level = np.ascontiguousarray(self.level, dtype=np.int32).reshape(-1)
            c.level = self.level.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        self._c = c

    @property
    def nblocks(self):
        return len(self.h)

    def ext(self, b):
        return tuple(int(v) + 2 * self.ghosts for v in self.n[b])

    def size(self) -> int:
        return int(lib().orc_state_size(ctypes.byref(self._c)))

    def zeros(self) -> np.ndarray:
        return np.zeros(self.size(), dtype=np.float64)

    def blocks(self, u: np.ndarray):
        """Views (22, nz+2g, ny+2g, nx+2g) of each block of a flat state."""
        out, off = [], 0
        for b in range(self.nblocks):
            ex, ey, ez = self.ext(b)
            cnt = NF * ex * ey * ez
            out.append(u[off:off + cnt].reshape(NF, ez, ey, ex))
            off += cnt
        return out

    def centres(self, b):
        """Cell-centre coordinates (x, y, z) of block b, each (nz', ny', nx')."""
        g = self.ghosts
        ax = [self.lo[b, d] + (np.arange(self.ext(b)[d]) - g + 0.5) * self.h[b] for d in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return x, y, z

    def interior_mask(self, b):
        g = self.ghosts
        ex, ey, ez = self.ext(b)
        m = np.zeros((ez, ey, ex), dtype=bool)
        nx, ny, nz = self.n[b]
        m[g:g + nz, g:g + ny, g:g + nx] = True
        return m

    def sommerfeld_mask(self, b):
        if self.periodic:
            return np.zeros_like(self.interior_mask(b))
        x, y, z = self.centres(b)
        out = np.zeros(x.shape, dtype=bool)
        for d, c in enumerate((x, y, z)):
            out |= (c < self.dom_lo[d]) | (c > self.dom_hi[d])
        return out & ~self.interior_mask(b)

    def evolved_mask(self, b):
        return self.interior_mask(b) | self.sommerfeld_mask(b)

    # ---- oracle calls ----
    def initial_data(self, kind: int, par) -> np.ndarray:
        u = self.zeros()
        p = np.ascontiguousarray(np.asarray(par, dtype=np.float64).reshape(-1))
        if p.size == 0:
            p = np.zeros(1)
        lib().orc_initial_data(ctypes.byref(self._c), _ptr(u), int(kind), _ptr(p))
        return u

    def fill_ghosts(self, u: np.ndarray) -> np.ndarray:
        rc = lib().orc_fill_ghosts(ctypes.byref(self._c), _ptr(u))
        if rc == -3:
            raise MemoryError("oracle coarse-buffer allocation failed")
        if rc != 0:
            raise ValueError("ghost fill needs data two refinement levels apart")
        return u

    def rhs(self, u: np.ndarray) -> np.ndarray:
        out = self.zeros()
        lib().orc_rhs(ctypes.byref(self._c), _ptr(u), _ptr(out))
        return out

    def rhs_cells(self, u: np.ndarray, cells: np.ndarray) -> np.ndarray:
        cells = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 4)
        out = np.zeros((len(cells), NF))
        lib().orc_rhs_cells(ctypes.byref(self._c), _ptr(u), _ptr(cells), len(cells), _ptr(out))
        return out

    def enforce(self, u: np.ndarray) -> np.ndarray:
        lib().orc_enforce(ctypes.byref(self._c), _ptr(u))
        return u

    def rk4(self, u: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
        rc = lib().orc_rk4_step(ctypes.byref(self._c), _ptr(u), float(dt), int(nsteps))
        if rc == -2:
            raise ValueError("ghost fill needs data two refinement levels apart")
        if rc != 0:
            raise MemoryError("oracle rk4 allocation failed")
        return u

    def constraints(self, u: np.ndarray, r_mask: float = 0.0, per_cell: bool = False):
        norms = np.zeros(6)
        pc = None
        if per_cell:
            pc = np.zeros(4 * self.size() // NF)
        lib().orc_constraints(ctypes.byref(self._c), _ptr(u), float(r_mask),
                              _ptr(pc) if pc is not None else None, _ptr(norms))
        return norms, pc

    def block_indicators(self, u: np.ndarray):
        """Per block (min chi, max |grad chi|) over interior cells; the
        ghosts of u must be filled."""
        cmin, gmax = np.zeros(self.nblocks), np.zeros(self.nblocks)
        lib().orc_block_indicators(ctypes.byref(self._c), _ptr(u), _ptr(cmin), _ptr(gmax))
        return cmin, gmax

    def psi4(self, u: np.ndarray):
        """Weyl scalar Psi4 (reading R20) at every interior cell: per block a
        complex (nz+2g, ny+2g, nx+2g) array, zero outside the interior; the
        ghosts of u must be filled."""
        out = np.zeros(2 * self.size() // NF)
        lib().orc_psi4(ctypes.byref(self._c), _ptr(u), _ptr(out))
        res, off = [], 0
        for b in range(self.nblocks):
            ex, ey, ez = self.ext(b)
            S = ex * ey * ez
            res.append((out[off:off + S] + 1j * out[off + S:off + 2 * S]).reshape(ez, ey, ex))
            off += 2 * S
        return res

    def track_punctures(self, u: np.ndarray, xyz, dt: float):
        """One tracker step of each puncture: (new positions, beta at the old
        ones); the ghosts of u must be filled."""
        x = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3)).copy()
        beta = np.zeros_like(x)
        if lib().orc_track_punctures(ctypes.byref(self._c), _ptr(u), len(x), _ptr(x), float(dt),
                                     _ptr(beta)) != 0:
            raise ValueError("a puncture lies outside every block")
        return x, beta


def fd(kind: int, order: int, f: np.ndarray, i: int, j: int, k: int, dir1: int, dir2: int = 0,
       h: float = 1.0, arg: float = 0.0) -> float:
    """One finite-difference operator of the oracle at cell (i, j, k) of a (nz, ny, nx) array."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    return lib().orc_fd(kind, order, _ptr(f), nx, ny, nz, i, j, k, dir1, dir2, float(h), float(arg))


def uniform_mesh(nb=(1, 1, 1), n=32, ghosts=None, order=4, dom_lo=(-0.5,) * 3, dom_hi=(0.5,) * 3,
                 periodic=True, **params) -> Mesh:
    """nb[0] x nb[1] x nb[2] equal blocks covering [dom_lo, dom_hi]; n is the
    interior size per block (int or 3-tuple)."""
    if ghosts is None:
        ghosts = order // 2 + 1
    n3 = np.array((n, n, n) if np.isscalar(n) else n, dtype=np.int64)
    L = np.array(dom_hi, dtype=float) - np.array(dom_lo, dtype=float)
    hs = L / (np.array(nb) * n3)
    assert np.allclose(hs, hs[0]), "blocks must have cubic cells"
    h = hs[0]
    ns, los, hh = [], [], []
    for kb in range(nb[2]):
        for jb in range(nb[1]):
            for ib in range(nb[0]):
                ns.append(n3)
                los.append([dom_lo[0] + ib * n3[0] * h, dom_lo[1] + jb * n3[1] * h,
                            dom_lo[2] + kb * n3[2] * h])
                hh.append(h)
    return Mesh(n=np.array(ns), lo=np.array(los), h=np.array(hh), ghosts=ghosts, order=order,
                dom_lo=tuple(dom_lo), dom_hi=tuple(dom_hi), periodic=periodic, **params)
