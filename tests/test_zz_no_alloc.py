"""The allocation-free constraint entry point against the regular one and
against the oracle.

z4c_constraints_static() serves callers that cannot allocate device memory
(e.g. a diagnostic hook inside a host code that owns the device memory
pool): its reduction records live in a fixed device array inside the
library.  Here it must reproduce z4c_constraints() of a context holding the
same block, and the oracle's constraint norms of the same state, within the
constraint-norm tolerance of the parity tests (relative 1e-10), on two
calls in a row (the second sees the array the first one left behind), and
again on a smaller block after a larger one (fewer records than the array
holds from the previous call).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu


def _case(oracle, order, n, seed):
    w = H.small_workload("puncture", order, (1, 1, 1), n)
    m = H.oracle_mesh(oracle, w)
    u = m.initial_data(w["id_kind"], w["id_par"])
    H.perturb(m, u, seed, 1e-3)
    m.fill_ghosts(u)
    g = H.gpu_ctx(w)
    g.z4c_set_state(u)
    ref, _, rc = g.z4c_constraints(r_mask=1.0)  # also fills U0's ghosts
    assert rc == 0
    g.z4c_sync()
    want, _ = m.constraints(u, r_mask=1.0)
    return w, g, ref, want


def _static(z4c, w, g, order):
    return z4c.z4c_constraints_static(g.regs[0].data_ptr(), w["n"][0], w["ghosts"], order, w["lo"][0],
                                      float(w["h"][0]), w["chi_floor"], 1.0, g.stream)


@pytest.mark.parametrize("order,n", [(6, 32), (4, (24, 20, 18)), (2, (22, 14, 10))])
def test_static_constraints_match_context(oracle, order, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2409_10383_gb300 import z4c
    w, g, ref, want = _case(oracle, order, n, 31 + order)
    assert np.allclose(ref, want, rtol=1e-10, atol=0), (ref, want)
    for _ in range(2):
        rc, norms = _static(z4c, w, g, order)
        assert rc == 0
        assert np.allclose(norms, ref, rtol=1e-10, atol=0), (norms, ref)
        assert np.allclose(norms, want, rtol=1e-10, atol=0), (norms, want)
    # a block beyond the fixed array is rejected, nothing launched
    rc, _ = z4c.z4c_constraints_static(g.regs[0].data_ptr(), (256, 256, 256), w["ghosts"], order,
                                       w["lo"][0], float(w["h"][0]), w["chi_floor"], 1.0, g.stream)
    assert rc == z4c.Z4C_ERR_UNSUPPORTED
    g.close()


def test_static_constraints_smaller_block_after_larger(oracle):
    """The array keeps the records of the last call: a 40^3 block (5 x 3 x
    40 tiles) followed by a 12^3 block (1 x 2 x 12 tiles) must read only the
    records the second call wrote."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2409_10383_gb300 import z4c
    big = _case(oracle, 6, 40, 5)
    small = _case(oracle, 6, 12, 6)
    for w, g, ref, want in (big, small, big, small):
        rc, norms = _static(z4c, w, g, 6)
        assert rc == 0
        assert np.allclose(norms, ref, rtol=1e-10, atol=0), (norms, ref)
        assert np.allclose(norms, want, rtol=1e-10, atol=0), (norms, want)
    big[1].close()
    small[1].close()
