"""Thin ctypes binding of the C ABI in include/z4c.h (same names).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  If the library is missing this module raises on import of the
library (no fallback of any kind).  ``Z4c`` allocates the caller-owned
device buffers with PyTorch and binds them with a dedicated CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

NF = 22
HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libz4c_gb300.so")

Z4C_OK, Z4C_ERR_BAD_ARG, Z4C_ERR_BAD_MESH, Z4C_ERR_UNSUPPORTED = 0, -1, -2, -3
Z4C_ERR_CUDA, Z4C_ERR_TIMEOUT, Z4C_ERR_NAN, Z4C_ERR_NOT_BOUND = -4, -5, -6, -7
REG_U0, REG_STAGE_A, REG_STAGE_B, REG_ACC = 0, 1, 2, 3

# every entry point declared in include/z4c.h
EXPORTS = ("z4c_create", "z4c_create_batch", "z4c_set_initial_data_instance", "z4c_rk4_step_batch",
           "z4c_constraints_instance", "z4c_state_bytes", "z4c_scratch_bytes", "z4c_bind",
           "z4c_set_initial_data", "z4c_fill_ghosts", "z4c_rhs", "z4c_rk4_step",
           "z4c_constraints", "z4c_get_state", "z4c_set_state", "z4c_evolve_host",
           "z4c_sync", "z4c_profile_steps", "z4c_set_variant", "z4c_autotune", "z4c_peak_fma", "z4c_constraints_static",
           "z4c_launches_per_step", "z4c_last_error", "z4c_destroy", "z4c_block_indicators",
           "z4c_track_punctures", "z4c_psi4", "z4c_peak_convert", "z4c_test_wait_timeout",
           "z4c_set_epilogue", "z4c_tile_shape", "z4c_set_prepass", "z4c_prepass_tma_blocks",
           "z4c_test_prepass_timeout")
Z4C_MAX_PUNCTURES = 64


class z4c_mesh(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int32), ("outer_bc", ctypes.c_int32)]


class z4c_block(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("lo", ctypes.c_double * 3),
                ("h", ctypes.c_double), ("instance", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class z4c_params(ctypes.Structure):
    _fields_ = [("ko_sigma", ctypes.c_double), ("kappa1", ctypes.c_double),
                ("kappa2", ctypes.c_double), ("eta", ctypes.c_double),
                ("chi_floor", ctypes.c_double), ("cfl", ctypes.c_double),
                ("lapse", ctypes.c_int32), ("shift", ctypes.c_int32),
                ("rhs_precision", ctypes.c_int32), ("schedule", ctypes.c_int32)]


class z4c_instance(ctypes.Structure):
    _fields_ = [("mesh", z4c_mesh), ("params", z4c_params), ("ghosts", ctypes.c_int32),
                ("fd_order", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                               "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        sig = {
            "z4c_create": (I, [ctypes.POINTER(z4c_mesh), ctypes.POINTER(z4c_block), I, I, I,
                               ctypes.POINTER(z4c_params), ctypes.POINTER(P)]),
            "z4c_create_batch": (I, [ctypes.POINTER(z4c_instance), I, ctypes.POINTER(z4c_block), I,
                                     ctypes.POINTER(P)]),
            "z4c_set_initial_data_instance": (I, [P, I, I, P, I]),
            "z4c_rk4_step_batch": (I, [P, P, I]),
            "z4c_constraints_instance": (I, [P, I, D, P, P]),
            "z4c_state_bytes": (I, [P, ctypes.POINTER(S)]),
            "z4c_scratch_bytes": (I, [P, ctypes.POINTER(S)]),
            "z4c_bind": (I, [P, P, P, P, P, P, P]),
            "z4c_set_initial_data": (I, [P, I, P, I]),
            "z4c_fill_ghosts": (I, [P, I]),
            "z4c_rhs": (I, [P, I, P]),
            "z4c_rk4_step": (I, [P, D, I]),
            "z4c_constraints": (I, [P, D, P, P]),
            "z4c_get_state": (I, [P, I, P, S]),
            "z4c_set_state": (I, [P, I, P, S]),
            "z4c_evolve_host": (I, [P, P, P, S, D, I]),
            "z4c_sync": (I, [P]),
            "z4c_test_wait_timeout": (I, [P, I]),
            "z4c_set_epilogue": (I, [P, I]),
            "z4c_set_prepass": (I, [P, I]),
            "z4c_prepass_tma_blocks": (I, [P]),
            "z4c_test_prepass_timeout": (I, [P]),
            "z4c_tile_shape": (I, [P, I, P, P, P]),
            "z4c_profile_steps": (I, [P, D, I, P]),
            "z4c_set_variant": (I, [P, I, I]),
            "z4c_autotune": (I, [P, I, P, P]),
            "z4c_peak_fma": (I, [I, P, P]),
            "z4c_constraints_static": (I, [P, P, I, I, P, D, D, D, P, P]),
            "z4c_block_indicators": (I, [P, I, P, P]),
            "z4c_track_punctures": (I, [P, I, I, P, D, P]),
            "z4c_psi4": (I, [P, I, P]),
            "z4c_peak_convert": (I, [I, P, P]),
            "z4c_launches_per_step": (I, [P]),
            "z4c_last_error": (ctypes.c_char_p, [P]),
            "z4c_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _lib = L
    return _lib


class Z4cError(RuntimeError):
    pass


def _check(rc, ctx=None, what=""):
    if rc != Z4C_OK:
        msg = lib().z4c_last_error(ctx).decode() if ctx else ""
        raise Z4cError(f"{what} failed with status {rc}: {msg}")


def z4c_create(mesh: z4c_mesh, blocks, ghosts: int, fd_order: int, params: z4c_params):
    arr = (z4c_block * len(blocks))(*blocks)
    out = ctypes.c_void_p()
    rc = lib().z4c_create(ctypes.byref(mesh), arr, len(blocks), ghosts, fd_order,
                          ctypes.byref(params), ctypes.byref(out))
    return rc, out


class Z4c:
    """One context plus its caller-owned device buffers (torch tensors).

    ``Z4c(**workload)`` makes a single-problem context; ``Z4c.batch([w0, w1,
    ...])`` a batch of independent problems (z4c_create_batch).  A workload
    is a dict with n, lo, h (per block), ghosts, order, dom_lo, dom_hi,
    periodic and the physics parameters."""

    def __init__(self, n=None, lo=None, h=None, ghosts=None, order=None, dom_lo=None, dom_hi=None,
                 periodic=None, ko_sigma=0.0, kappa1=0.0, kappa2=0.0, eta=2.0, chi_floor=1e-6, lapse=1,
                 shift=1, precision=64, schedule=0, device="cuda", stream=None, instances=None, level=None,
                 **_):
        import torch
        self.torch = torch
        if instances is None:
            instances = [dict(n=n, lo=lo, h=h, ghosts=ghosts, order=order, dom_lo=dom_lo, dom_hi=dom_hi,
                              periodic=periodic, ko_sigma=ko_sigma, kappa1=kappa1, kappa2=kappa2, eta=eta,
                              chi_floor=chi_floor, lapse=lapse, shift=shift, precision=precision,
                              schedule=schedule, level=level)]
        self.instances = instances
        insts = (z4c_instance * len(instances))()
        self.blocks = []
        self.block_elems = []
        for i, w in enumerate(instances):
            I = insts[i]
            I.mesh.lo[:] = [float(v) for v in w["dom_lo"]]
            I.mesh.hi[:] = [float(v) for v in w["dom_hi"]]
            I.mesh.periodic = int(bool(w["periodic"]))
            I.mesh.outer_bc = 0 if w["periodic"] else 1
            I.params = z4c_params(w.get("ko_sigma", 0.0), w.get("kappa1", 0.0), w.get("kappa2", 0.0),
                                  w.get("eta", 2.0), w.get("chi_floor", 1e-6), 0.25, w.get("lapse", 1),
                                  w.get("shift", 1), w.get("precision", 64), w.get("schedule", 0))
            I.ghosts, I.fd_order = int(w["ghosts"]), int(w["order"])
            nn = np.asarray(w["n"]).reshape(-1, 3)
            ll = np.asarray(w["lo"], float).reshape(-1, 3)
            hh = np.broadcast_to(np.asarray(w["h"], float), (len(nn),))
            lev = np.zeros(len(nn), int) if w.get("level") is None else np.asarray(w["level"]).reshape(-1)
            for b in range(len(nn)):
                B = z4c_block()
                B.level, B.instance = int(lev[b]), i
                B.n[:] = [int(v) for v in nn[b]]
                B.lo[:] = [float(v) for v in ll[b]]
                B.h = float(hh[b])
                self.blocks.append(B)
                self.block_elems.append(NF * int(np.prod(nn[b] + 2 * int(w["ghosts"]))))
        w0 = instances[0]
        self.n, self.ghosts, self.order = np.asarray(w0["n"]).reshape(-1, 3), w0["ghosts"], w0["order"]
        self.params = insts[0].params
        arr = (z4c_block * len(self.blocks))(*self.blocks)
        out = ctypes.c_void_p()
        rc = lib().z4c_create_batch(insts, len(instances), arr, len(self.blocks), ctypes.byref(out))
        _check(rc, None, "z4c_create_batch")
        self.ctx = out
        sb, sc = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().z4c_state_bytes(self.ctx, ctypes.byref(sb)), self.ctx, "z4c_state_bytes")
        _check(lib().z4c_scratch_bytes(self.ctx, ctypes.byref(sc)), self.ctx, "z4c_scratch_bytes")
        self.state_bytes, self.scratch_bytes = sb.value, sc.value
        self.nelem = self.state_bytes // 8
        dev = torch.device(device)
        self.regs = [torch.empty(self.nelem, dtype=torch.float64, device=dev) for _ in range(4)]
        self.scratch = torch.empty(max(256, self.scratch_bytes), dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        _check(lib().z4c_bind(self.ctx, *[r.data_ptr() for r in self.regs], self.scratch.data_ptr(),
                              self.stream.cuda_stream), self.ctx, "z4c_bind")

    @classmethod
    def from_workload(cls, w: dict, **kw):
        args = dict(w)
        args.update(kw)
        args.setdefault("precision", 64)
        return cls(**args)

    @classmethod
    def batch(cls, workloads, device="cuda", stream=None):
        return cls(instances=list(workloads), device=device, stream=stream)

    def instance_slice(self, i: int) -> slice:
        """Elements of instance i's blocks in a register."""
        first = sum(1 for B in self.blocks if B.instance < i)
        last = first + sum(1 for B in self.blocks if B.instance == i)
        start = sum(self.block_elems[:first])
        return slice(start, start + sum(self.block_elems[first:last]))

    # --- stream ordering between torch's current stream and the context's ---
    def _enter(self):
        """Work queued by torch on its current stream (e.g. writes into an
        output tensor) must finish before the context's kernels read it."""
        if self.regs[0].is_cuda:
            self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self, *tensors):
        """Results written on the context's stream become visible to torch's
        current stream (e.g. a following .cpu())."""
        if self.regs[0].is_cuda:
            self.torch.cuda.current_stream().wait_stream(self.stream)
            for t in tensors:
                if t is not None:
                    t.record_stream(self.stream)

    # --- C ABI calls (same names) ---
    def z4c_set_initial_data(self, kind, par):
        p = np.ascontiguousarray(np.asarray(par, dtype=np.float64).reshape(-1))
        _check(lib().z4c_set_initial_data(self.ctx, int(kind), p.ctypes.data if p.size else None,
                                          int(p.size)), self.ctx, "z4c_set_initial_data")

    def z4c_set_initial_data_instance(self, instance, kind, par):
        p = np.ascontiguousarray(np.asarray(par, dtype=np.float64).reshape(-1))
        _check(lib().z4c_set_initial_data_instance(self.ctx, int(instance), int(kind),
                                                   p.ctypes.data if p.size else None, int(p.size)),
               self.ctx, "z4c_set_initial_data_instance")

    def z4c_rk4_step_batch(self, dts, nsteps=1):
        d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64).reshape(-1))
        assert d.size == len(self.instances)
        _check(lib().z4c_rk4_step_batch(self.ctx, d.ctypes.data, int(nsteps)), self.ctx, "z4c_rk4_step_batch")
        self._leave()

    def z4c_constraints_instance(self, instance, r_mask=0.0):
        norms = np.zeros(6)
        self._enter()
        rc = lib().z4c_constraints_instance(self.ctx, int(instance), float(r_mask), norms.ctypes.data, None)
        self._leave()
        if rc not in (Z4C_OK, Z4C_ERR_NAN):
            _check(rc, self.ctx, "z4c_constraints_instance")
        return norms, rc

    def z4c_fill_ghosts(self, reg=REG_U0):
        self._enter()
        _check(lib().z4c_fill_ghosts(self.ctx, int(reg)), self.ctx, "z4c_fill_ghosts")
        self._leave()

    def z4c_rhs(self, reg=REG_U0, out=None):
        if out is None:
            out = self.torch.empty(self.nelem, dtype=self.torch.float64, device=self.regs[0].device)
        self._enter()
        _check(lib().z4c_rhs(self.ctx, int(reg), out.data_ptr()), self.ctx, "z4c_rhs")
        self._leave(out)
        return out

    def z4c_rk4_step(self, dt, nsteps=1):
        _check(lib().z4c_rk4_step(self.ctx, float(dt), int(nsteps)), self.ctx, "z4c_rk4_step")
        self._leave()

    def z4c_constraints(self, r_mask=0.0, per_cell=False):
        norms = np.zeros(6)
        pc = None
        if per_cell:
            pc = self.torch.empty(self.nelem // NF * 4, dtype=self.torch.float64,
                                  device=self.regs[0].device)
        self._enter()
        rc = lib().z4c_constraints(self.ctx, float(r_mask), norms.ctypes.data,
                                   pc.data_ptr() if pc is not None else None)
        self._leave(pc)
        if rc not in (Z4C_OK, Z4C_ERR_NAN):
            _check(rc, self.ctx, "z4c_constraints")
        return norms, pc, rc

    def z4c_get_state(self, reg=REG_U0, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.nelem, dtype=np.float64)
        _check(lib().z4c_get_state(self.ctx, int(reg), out.ctypes.data, self.state_bytes),
               self.ctx, "z4c_get_state")
        return out

    def z4c_set_state(self, host: np.ndarray, reg=REG_U0):
        host = np.ascontiguousarray(host, dtype=np.float64)
        _check(lib().z4c_set_state(self.ctx, int(reg), host.ctypes.data, self.state_bytes),
               self.ctx, "z4c_set_state")

    def z4c_evolve_host(self, host_in, host_out, dt, nsteps):
        """host_in/host_out: numpy arrays or pinned CPU torch tensors."""
        pin = host_in.ctypes.data if isinstance(host_in, np.ndarray) else host_in.data_ptr()
        pout = host_out.ctypes.data if isinstance(host_out, np.ndarray) else host_out.data_ptr()
        _check(lib().z4c_evolve_host(self.ctx, pin, pout, self.state_bytes, float(dt), int(nsteps)),
               self.ctx, "z4c_evolve_host")

    def z4c_sync(self):
        _check(lib().z4c_sync(self.ctx), self.ctx, "z4c_sync")

    def z4c_test_wait_timeout(self, rounds=64):
        """Failure-detection aid: a kernel whose bounded mbarrier wait runs
        out.  Returns (status, z4c_last_error text)."""
        rc = lib().z4c_test_wait_timeout(self.ctx, int(rounds))
        return rc, lib().z4c_last_error(self.ctx).decode()

    def z4c_test_prepass_timeout(self):
        """Failure-detection aid: the TMA-fed pre-pass with a zero wait
        limit.  Returns (status, z4c_last_error text)."""
        self._enter()
        rc = lib().z4c_test_prepass_timeout(self.ctx)
        return rc, lib().z4c_last_error(self.ctx).decode()

    def z4c_block_indicators(self, reg=REG_U0):
        """Per block (min chi, max |grad chi|) over its interior cells
        (paper Sec. 3.2 refinement criteria); fills reg's ghosts first."""
        nb = len(self.blocks)
        cmin, gmax = np.zeros(nb), np.zeros(nb)
        self._enter()
        _check(lib().z4c_block_indicators(self.ctx, int(reg), cmin.ctypes.data, gmax.ctypes.data), self.ctx,
               "z4c_block_indicators")
        return cmin, gmax

    def z4c_track_punctures(self, xyz, dt, reg=REG_U0):
        """One tracker step x <- x - dt beta(x) of each puncture (paper Sec.
        3.3): returns (new positions, beta at the old ones)."""
        x = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3)).copy()
        beta = np.zeros_like(x)
        self._enter()
        _check(lib().z4c_track_punctures(self.ctx, int(reg), len(x), x.ctypes.data, float(dt), beta.ctypes.data),
               self.ctx, "z4c_track_punctures")
        return x, beta

    def z4c_psi4(self, reg=REG_U0, out=None):
        """Weyl scalar Psi4 (paper Sec. 3.3, coordinate tetrad) at every
        interior cell: a device tensor of 2 * (register elements / 22)
        doubles, per block the real part then the imaginary part over its
        storage cells; fills reg's ghosts first."""
        n = 2 * (self.nelem // 22)
        if out is None:
            out = self.torch.empty(n, dtype=self.torch.float64, device=self.regs[0].device)
        self._enter()
        _check(lib().z4c_psi4(self.ctx, int(reg), out.data_ptr()), self.ctx, "z4c_psi4")
        self._leave(out)
        return out

    def z4c_profile_steps(self, dt, nsteps):
        ms = np.zeros(4)
        _check(lib().z4c_profile_steps(self.ctx, float(dt), int(nsteps), ms.ctypes.data), self.ctx,
               "z4c_profile_steps")
        return ms

    def z4c_set_variant(self, schedule, occupancy=1):
        _check(lib().z4c_set_variant(self.ctx, int(schedule), int(occupancy)), self.ctx, "z4c_set_variant")

    def z4c_tile_shape(self, block=0):
        """(tx, ty, cells per thread) of the block's interior tiles under the
        current kernel variant."""
        tx, ty, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().z4c_tile_shape(self.ctx, int(block), ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(c)),
               self.ctx, "z4c_tile_shape")
        return tx.value, ty.value, c.value

    def z4c_set_epilogue(self, kind):
        """FP32-RHS split schedules: 1 bulk-copy stage-update kernel, 0 plain."""
        _check(lib().z4c_set_epilogue(self.ctx, int(kind)), self.ctx, "z4c_set_epilogue")

    def z4c_set_prepass(self, kind):
        """FP32-RHS y/z pre-pass: 1 the z-walking kernel fed by TMA where the
        blocks allow it (default), 0 the plane-tiled kernel."""
        _check(lib().z4c_set_prepass(self.ctx, int(kind)), self.ctx, "z4c_set_prepass")

    def z4c_prepass_tma_blocks(self) -> int:
        """Blocks whose y/z pre-pass runs the TMA-fed kernel."""
        n = lib().z4c_prepass_tma_blocks(self.ctx)
        if n < 0:
            _check(n, self.ctx, "z4c_prepass_tma_blocks")
        return n

    def z4c_autotune(self, reps=3):
        sch, occ = ctypes.c_int(), ctypes.c_int()
        self._enter()
        _check(lib().z4c_autotune(self.ctx, int(reps), ctypes.byref(sch), ctypes.byref(occ)), self.ctx,
               "z4c_autotune")
        return sch.value, occ.value

    def z4c_launches_per_step(self) -> int:
        return int(lib().z4c_launches_per_step(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            lib().z4c_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def z4c_peak_fma(fp64: bool, stream=None) -> float:
    """FP64/FP32 FMA throughput of the current GPU in FLOP/s."""
    out = ctypes.c_double()
    st = stream.cuda_stream if stream is not None else None
    _check(lib().z4c_peak_fma(int(bool(fp64)), st, ctypes.byref(out)), None, "z4c_peak_fma")
    return out.value


def z4c_peak_convert(mode: int, stream=None) -> float:
    """float <-> double conversions per second of the current GPU: mode 0/1
    float -> double by the hardware / on the integer pipe, 2/3 double ->
    float likewise."""
    out = ctypes.c_double()
    st = stream.cuda_stream if stream is not None else None
    _check(lib().z4c_peak_convert(int(mode), st, ctypes.byref(out)), None, "z4c_peak_convert")
    return out.value


def z4c_constraints_static(u_device_ptr: int, n, ghosts: int, fd_order: int, lo, h: float,
                           chi_floor: float, r_mask: float, stream=None):
    """Constraint norms of one block in device memory, allocating nothing
    (see include/z4c.h).  Returns (status, norms)."""
    n_arr = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    lo_arr = (ctypes.c_double * 3)(*[float(v) for v in lo])
    norms = np.zeros(6)
    st = stream.cuda_stream if stream is not None else None
    rc = lib().z4c_constraints_static(u_device_ptr, n_arr, int(ghosts), int(fd_order), lo_arr,
                                      float(h), float(chi_floor), float(r_mask), norms.ctypes.data, st)
    return rc, norms
