"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point declared in include/z4c.h, and rejects bad arguments with
the documented status codes without touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2409_10383_gb300 import z4c

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2409_10383_gb300 import build
    build.build()
    return z4c.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "z4c.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(z4c_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(z4c.EXPORTS)


def _mesh(per=1):
    m = z4c.z4c_mesh()
    m.lo[:] = [-0.5] * 3
    m.hi[:] = [0.5] * 3
    m.periodic = per
    return m


def _block(n=32, lo=(-0.5, -0.5, -0.5), h=1 / 32):
    b = z4c.z4c_block()
    b.n[:] = [n] * 3
    b.lo[:] = list(lo)
    b.h = h
    return b


def _params(prec=64, schedule=0):
    return z4c.z4c_params(0.02, 0, 0, 0, 1e-6, 0.25, 0, 0, prec, schedule)


def test_create_validates_arguments(L):
    ok, ctx = z4c.z4c_create(_mesh(), [_block()], 3, 4, _params())
    assert ok == 0 and ctx.value
    L.z4c_destroy(ctx)
    assert z4c.z4c_create(_mesh(), [_block()], 3, 5, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    assert z4c.z4c_create(_mesh(), [_block()], 2, 4, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    assert z4c.z4c_create(_mesh(), [_block()], 3, 6, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    assert z4c.z4c_create(_mesh(), [_block()], 4, 4, _params(16))[0] == z4c.Z4C_ERR_UNSUPPORTED
    # 2nd-order differencing needs 2 ghosts; orders other than 2, 4, 6 are refused
    ok, ctx = z4c.z4c_create(_mesh(), [_block()], 2, 2, _params())
    assert ok == 0 and ctx.value
    L.z4c_destroy(ctx)
    assert z4c.z4c_create(_mesh(), [_block()], 1, 2, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    assert z4c.z4c_create(_mesh(), [_block()], 3, 3, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    assert z4c.z4c_create(_mesh(), [_block()], 5, 8, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    # block does not tile the mesh
    assert z4c.z4c_create(_mesh(), [_block(n=16)], 3, 4, _params())[0] == z4c.Z4C_ERR_BAD_MESH
    # overlapping blocks
    b = _block(n=16, h=1 / 32)
    assert z4c.z4c_create(_mesh(), [b] * 8, 3, 4, _params())[0] == z4c.Z4C_ERR_BAD_MESH
    # off-lattice block
    assert z4c.z4c_create(_mesh(), [_block(lo=(-0.49, -0.5, -0.5))], 3, 4,
                          _params())[0] == z4c.Z4C_ERR_BAD_MESH
    # a block thinner than the ghost width (a ghost region would span two
    # neighbours) is refused; one exactly as wide is accepted
    assert z4c.z4c_create(_mesh(), [_block(n=2, h=0.5)], 3, 4, _params())[0] == z4c.Z4C_ERR_UNSUPPORTED
    ok, ctx = z4c.z4c_create(_mesh(), [_block(n=3, h=1 / 3)], 3, 4, _params())
    assert ok == 0 and ctx.value
    L.z4c_destroy(ctx)
    # no blocks
    assert z4c.z4c_create(_mesh(), [], 3, 4, _params())[0] != 0


def test_sizes_and_unbound_calls(L):
    rc, ctx = z4c.z4c_create(_mesh(), [_block()], 3, 4, _params(32))
    sb, sc = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.z4c_state_bytes(ctx, ctypes.byref(sb)) == 0
    assert sb.value == 22 * 38 ** 3 * 8
    assert L.z4c_scratch_bytes(ctx, ctypes.byref(sc)) == 0
    assert sc.value >= 2 * 22 * 38 ** 3 * 4  # two FP32 shadows
    assert L.z4c_rk4_step(ctx, 0.01, 1) == z4c.Z4C_ERR_NOT_BOUND
    assert b"z4c_bind" in L.z4c_last_error(ctx)
    # periodic FP32-RHS, default split schedule: ghost fill + pre-pass + RHS
    # kernel + stage-update kernel per stage
    assert L.z4c_launches_per_step(ctx) == 16
    L.z4c_destroy(ctx)
    # a single block with the Sommerfeld boundary on every face: no ghost
    # copies; pre-pass + RHS + stage update, and the FP32 Sommerfeld cells'
    # RHS and stage-update kernels, per stage (FP64 cells: one kernel)
    rc, ctx = z4c.z4c_create(_mesh(per=0), [_block()], 3, 4, _params(32))
    assert rc == 0 and L.z4c_launches_per_step(ctx) == 4 * 5
    L.z4c_destroy(ctx)
    rc, ctx = z4c.z4c_create(_mesh(per=0), [_block()], 3, 4, _params(64))
    assert rc == 0 and L.z4c_launches_per_step(ctx) == 4 * (1 + 1 + 1)  # pre-pass, fused, Sommerfeld
    L.z4c_destroy(ctx)
    rc, ctx = z4c.z4c_create(_mesh(), [_block()], 3, 4, _params(64, schedule=1))
    assert rc == 0 and L.z4c_launches_per_step(ctx) == 8  # single fused kernel
    L.z4c_destroy(ctx)
    assert z4c.z4c_create(_mesh(), [_block()], 3, 4, _params(64, schedule=7))[0] == z4c.Z4C_ERR_BAD_ARG
    rc, ctx = z4c.z4c_create(_mesh(), [_block()], 3, 4, _params(64))
    assert L.z4c_set_variant(ctx, 2, 4) == z4c.Z4C_ERR_UNSUPPORTED  # FP64 has one occupancy
    assert L.z4c_set_variant(ctx, 3, 1) == z4c.Z4C_ERR_UNSUPPORTED  # schedule 3 is FP32-RHS only
    assert L.z4c_set_variant(ctx, 1, 1) == 0 and L.z4c_launches_per_step(ctx) == 8
    L.z4c_destroy(ctx)
    rc, ctx = z4c.z4c_create(_mesh(), [_block()], 3, 4, _params(32))
    assert L.z4c_set_variant(ctx, 2, 2) == 0 and L.z4c_set_variant(ctx, 1, 4) == z4c.Z4C_ERR_UNSUPPORTED
    assert L.z4c_set_variant(ctx, 3, 4) == 0
    assert L.z4c_set_variant(ctx, 4, 4) == 0 and L.z4c_set_variant(ctx, 4, 1) == z4c.Z4C_ERR_UNSUPPORTED
    L.z4c_destroy(ctx)


def test_diagnostic_calls_check_arguments(L):
    """Argument checks that come before any CUDA call."""
    out = ctypes.c_double()
    assert L.z4c_peak_convert(4, None, ctypes.byref(out)) == z4c.Z4C_ERR_BAD_ARG
    assert L.z4c_peak_convert(-1, None, ctypes.byref(out)) == z4c.Z4C_ERR_BAD_ARG
    assert L.z4c_peak_convert(0, None, None) == z4c.Z4C_ERR_BAD_ARG
    rc, ctx = z4c.z4c_create(_mesh(), [_block()], 3, 4, _params())
    assert L.z4c_psi4(ctx, 0, None) == z4c.Z4C_ERR_NOT_BOUND  # not bound yet
    L.z4c_destroy(ctx)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built CUDA library every call raises: there is no CPU or
    other fallback path behind the binding."""
    monkeypatch.setattr(z4c, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(z4c, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        z4c.lib()
    with pytest.raises(RuntimeError, match="no fallback"):
        z4c.z4c_create(_mesh(), [_block()], 3, 4, _params())


def test_tile_shape_reports_the_variant(L):
    """z4c_tile_shape (no CUDA call): FP32-RHS blocks of 64^3 take 64 x 2
    tiles under schedules 5 and 6 (two cells per thread under 6), 32^3
    blocks 32 x 4, 16^3 blocks stay on 16 x 8; schedule 4 and FP64 blocks
    use 16 x 8 with one cell per thread."""
    def ctx(n, prec):
        ok, c = z4c.z4c_create(_mesh(), [_block(n=n, h=1.0 / n)], 4, 6, _params(prec))
        assert ok == 0
        return c

    def shape(c):
        tx, ty, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        assert L.z4c_tile_shape(c, 0, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(k)) == 0
        return tx.value, ty.value, k.value

    for n, wide in ((64, (64, 2)), (32, (32, 4)), (16, (16, 8))):
        c = ctx(n, 32)
        assert shape(c) == (16, 8, 1)  # default schedule 4
        assert L.z4c_set_variant(c, 5, 4) == 0
        assert shape(c) == wide + (1,)
        assert L.z4c_set_variant(c, 6, 4) == 0
        assert shape(c) == wide + (2 if wide != (16, 8) else 1,)
        tx = ctypes.c_int()
        assert L.z4c_tile_shape(c, 1, ctypes.byref(tx), ctypes.byref(tx), ctypes.byref(tx)) == z4c.Z4C_ERR_BAD_ARG
        L.z4c_destroy(c)
    c = ctx(64, 64)
    assert shape(c) == (16, 8, 1)
    L.z4c_destroy(c)


def test_prepass_kind_and_qualifying_blocks(L):
    """z4c_set_prepass / z4c_prepass_tma_blocks (no CUDA call): FP32-RHS
    blocks of order 4 or 6 whose rows, fields and offsets are multiples of
    4 floats take the TMA-fed pre-pass by default, kind 0 switches it off,
    FP64 blocks and a 26-cell storage row never take it."""
    def ctx(n, g, order, prec):
        ok, c = z4c.z4c_create(_mesh(), [_block(n=n, h=1.0 / n)], g, order, _params(prec))
        assert ok == 0, ok
        return c

    c = ctx(32, 4, 6, 32)  # storage 40^3
    assert L.z4c_prepass_tma_blocks(c) == 1
    assert L.z4c_set_prepass(c, 0) == 0 and L.z4c_prepass_tma_blocks(c) == 0
    assert L.z4c_set_prepass(c, 1) == 0 and L.z4c_prepass_tma_blocks(c) == 1
    assert L.z4c_set_prepass(c, 2) == z4c.Z4C_ERR_BAD_ARG
    L.z4c_destroy(c)
    c = ctx(26, 3, 4, 32)  # storage 32^3, order 4
    assert L.z4c_prepass_tma_blocks(c) == 1
    L.z4c_destroy(c)
    c = ctx(20, 3, 4, 32)  # storage rows of 26 floats
    assert L.z4c_prepass_tma_blocks(c) == 0
    L.z4c_destroy(c)
    c = ctx(32, 4, 6, 64)  # FP64
    assert L.z4c_prepass_tma_blocks(c) == 0
    L.z4c_destroy(c)
    assert L.z4c_prepass_tma_blocks(None) == z4c.Z4C_ERR_BAD_ARG
