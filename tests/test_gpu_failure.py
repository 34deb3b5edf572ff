"""Failure detection without a GPU fault.

- A bounded device-side wait that runs out: z4c_test_wait_timeout launches
  one kernel whose mbarrier waits for bulk-copy bytes that no copy will
  deliver (none is issued); mbar_wait gives up after a few rounds, the
  kernel sets the status word and returns, and the host reports
  Z4C_ERR_TIMEOUT with its text.  The context stays usable: an RK4 step
  afterwards still matches the oracle.
- The same for the y/z pre-pass fed by TMA: z4c_test_prepass_timeout runs
  it with a zero wait limit, so every CTA gives up at its first wait on
  copies it has issued, waits a bounded time for them to land, sets the
  status word and returns; Z4C_ERR_TIMEOUT is reported and RK4 steps
  afterwards are bit-identical to those of a fresh context.
- A NaN planted on the host (z4c_set_state) in one interior cell: the
  constraint norms come out NaN and both constraint calls, the context's
  and the allocation-free one, return Z4C_ERR_NAN; evolving through it
  raises no CUDA error.
"""
import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(oracle):
    from paper_2409_10383_gb300 import z4c
    w = H.small_workload("puncture", 6, (2, 1, 1), 12)
    m = H.oracle_mesh(oracle, w)
    g = H.gpu_ctx(w)
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    rc, msg = g.z4c_test_wait_timeout(64)
    assert rc == z4c.Z4C_ERR_TIMEOUT, (rc, msg)
    assert "gave up" in msg, msg
    # reported once: the status word is cleared
    g.z4c_sync()
    u = m.initial_data(w["id_kind"], w["id_par"])
    dt = 0.25 * float(w["h"][0])
    g.z4c_rk4_step(dt, 2)
    g.z4c_sync()
    m.rk4(u, dt, 2)
    rel, absd = H.field_errors(m, u, g.z4c_get_state())
    assert rel.max() <= 1e-10, (rel, absd)
    # out-of-range limits are rejected before any launch
    rc, _ = g.z4c_test_wait_timeout(0)
    assert rc == z4c.Z4C_ERR_BAD_ARG
    g.close()


def test_tma_prepass_wait_gives_up_and_context_survives():
    from paper_2409_10383_gb300 import z4c
    w = H.small_workload("puncture", 6, (2, 1, 1), 32)
    dt = 0.25 * float(w["h"][0])
    ref = H.gpu_ctx(w, precision=32)
    ref.z4c_set_initial_data(w["id_kind"], w["id_par"])
    ref.z4c_rk4_step(dt, 2)
    want = ref.z4c_get_state()
    ref.close()
    g = H.gpu_ctx(w, precision=32)
    assert g.z4c_prepass_tma_blocks() == 2
    g.z4c_set_initial_data(w["id_kind"], w["id_par"])
    rc, msg = g.z4c_test_prepass_timeout()
    assert rc == z4c.Z4C_ERR_TIMEOUT, (rc, msg)
    assert "gave up" in msg, msg
    g.z4c_sync()  # reported once: the status word is cleared
    g.z4c_rk4_step(dt, 2)
    assert np.array_equal(g.z4c_get_state(), want)
    g.close()
    # no block on that kernel: refused before any launch
    f = H.gpu_ctx(w, precision=64)
    rc, _ = f.z4c_test_prepass_timeout()
    assert rc == z4c.Z4C_ERR_UNSUPPORTED
    f.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_host_planted_nan_is_reported(oracle, precision):
    from paper_2409_10383_gb300 import z4c
    w = H.small_workload("puncture", 6, (1, 1, 1), 16)
    m = H.oracle_mesh(oracle, w)
    u = m.initial_data(w["id_kind"], w["id_par"])
    m.fill_ghosts(u)
    g = H.gpu_ctx(w, precision=precision)
    g.z4c_set_state(u)
    norms, _, rc = g.z4c_constraints(r_mask=1.0)
    assert rc == z4c.Z4C_OK and np.all(np.isfinite(norms))
    # one interior cell of Khat (field 7), block 0
    v = u.copy()
    blk = m.blocks(v)[0]
    gw = w["ghosts"]
    blk[7, gw + 5, gw + 6, gw + 7] = np.nan
    g.z4c_set_state(v)
    norms, _, rc = g.z4c_constraints(r_mask=1.0)
    assert rc == z4c.Z4C_ERR_NAN and np.isnan(norms[0]), (rc, norms)
    g.z4c_sync()
    rc, norms = z4c.z4c_constraints_static(g.regs[0].data_ptr(), w["n"][0], gw, 6, w["lo"][0],
                                           float(w["h"][0]), w["chi_floor"], 1.0, g.stream)
    assert rc == z4c.Z4C_ERR_NAN and np.isnan(norms[0]), (rc, norms)
    # evolving through the NaN is no CUDA error; the norms stay NaN
    g.z4c_rk4_step(0.25 * float(w["h"][0]), 1)
    g.z4c_sync()
    norms, _, rc = g.z4c_constraints(r_mask=1.0)
    assert rc == z4c.Z4C_ERR_NAN
    g.close()
