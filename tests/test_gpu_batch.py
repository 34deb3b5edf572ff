"""Batched evolution of independent problems (one graph launch per RK4 step).

A batch mixes block sizes, orders 2/4/6, FP64 and FP32-RHS, punctures and
gauge waves, each instance with its own dt.  Packing must not change any
instance's arithmetic: every instance's state is bit-identical to the same
instance evolved alone, FP64 instances match the oracle (1e-10), and the
per-instance constraint norms match the single-instance ones.
"""
import numpy as np
import pytest

import helpers as H
from paper_2409_10383_gb300 import inputs

pytestmark = pytest.mark.gpu

STEPS = 3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _dt(w):
    return w["cfl"] * float(w["h"][0])


def _pair_mix():
    """FP32-RHS instances of 32^3 (32 x 4 tiles), 64^3 (64 x 2) and 16^3
    (16 x 8 tiles) in one wide-tile list, beside FP64 instances."""
    I = inputs._instance
    return [I("puncture", 32, 6, 32, 1.0), I("puncture", 16, 6, 32, 1.5), I("gauge_wave", 32, 6, 32, 0.01),
            I("puncture", 16, 6, 64, 1.2), I("puncture", 64, 6, 32, 0.8), I("puncture", 16, 4, 32, 0.9)]


@pytest.mark.parametrize("mix,schedule", [("uneven_batch_small", 0), ("mixed_order_batch_small", 0),
                                          ("pair_mix", 5), ("pair_mix", 6)])
def test_batch_equals_single_instances(oracle, mix, schedule):
    """mixed_order_batch_small adds 2nd-order instances (FP64 and FP32-RHS);
    schedules 5 and 6 run the FP32-RHS instances whose blocks allow it on
    wide tiles (6: two cells per thread), alone and in the batch alike."""
    from paper_2409_10383_gb300.z4c import Z4c
    ws = _pair_mix() if mix == "pair_mix" else getattr(inputs, mix)()
    g = Z4c.batch(ws)
    if schedule:
        g.z4c_set_variant(schedule, 4)
    for i, w in enumerate(ws):
        g.z4c_set_initial_data_instance(i, w["id_kind"], w["id_par"])
    g.z4c_rk4_step_batch([_dt(w) for w in ws], STEPS)
    got = g.z4c_get_state()
    for i, w in enumerate(ws):
        s = Z4c.from_workload(w, precision=w["precision"])
        if schedule and w["precision"] == 32:
            s.z4c_set_variant(schedule, 4)
        s.z4c_set_initial_data(w["id_kind"], w["id_par"])
        s.z4c_rk4_step(_dt(w), STEPS)
        ref = s.z4c_get_state()
        assert np.array_equal(got[g.instance_slice(i)], ref), (i, w["name"], w["order"], w["precision"])
        if w["precision"] == 64:
            m = H.oracle_mesh(oracle, w)
            u = m.initial_data(w["id_kind"], w["id_par"])
            m.rk4(u, _dt(w), STEPS)
            rel, _ = H.field_errors(m, u, ref)
            assert rel.max() <= 1e-10, (i, rel.max())
        n_b, rc = g.z4c_constraints_instance(i, r_mask=1.0)
        n_s, _, rc2 = s.z4c_constraints(r_mask=1.0)
        assert rc == 0 and rc2 == 0
        assert np.allclose(n_b, n_s, rtol=1e-12, atol=0), (i, n_b, n_s)
        s.close()


def test_batch_rejects_bad_layouts():
    from paper_2409_10383_gb300 import z4c
    from paper_2409_10383_gb300.z4c import Z4c
    ws = inputs.uneven_batch_small()[:2]
    g = Z4c.batch(ws)
    assert g.z4c_launches_per_step() > 0
    # blocks out of instance order are refused
    blocks = list(reversed(g.blocks))
    import ctypes
    insts = (z4c.z4c_instance * 2)()
    arr = (z4c.z4c_block * len(blocks))(*blocks)
    out = ctypes.c_void_p()
    assert z4c.lib().z4c_create_batch(insts, 2, arr, len(blocks), ctypes.byref(out)) == z4c.Z4C_ERR_BAD_ARG
