"""The allocation-free constraint entry point against the regular one.

z4c_constraints_static() serves callers that cannot allocate device memory
(e.g. a diagnostic hook inside a host code that owns the device memory
pool): its reduction records live in a fixed device array inside the
library.  Here it must reproduce z4c_constraints() of a context holding the
same block, within the constraint-norm tolerance of the parity tests
(relative 1e-10), on two calls in a row (the second sees the array the
first one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import helpers as H
from paper_2409_10383_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order,n", [(6, 32), (4, (24, 20, 18))])
def test_static_constraints_match_context(oracle, order, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2409_10383_gb300 import z4c
    w = H.small_workload("puncture", order, (1, 1, 1), n)
    m = H.oracle_mesh(oracle, w)
    u = m.initial_data(w["id_kind"], w["id_par"])
    H.perturb(m, u, 31 + order, 1e-3)
    g = H.gpu_ctx(w)
    g.z4c_set_state(u)
    ref, _, rc = g.z4c_constraints(r_mask=1.0)  # also fills U0's ghosts
    assert rc == 0
    g.z4c_sync()
    for _ in range(2):
        rc, norms = z4c.z4c_constraints_static(g.regs[0].data_ptr(), w["n"][0], w["ghosts"], order,
                                               w["lo"][0], float(w["h"][0]), w["chi_floor"], 1.0,
                                               g.stream)
        assert rc == 0
        assert np.allclose(norms, ref, rtol=1e-10, atol=0), (norms, ref)
    # a block beyond the fixed array is rejected, nothing launched
    rc, _ = z4c.z4c_constraints_static(g.regs[0].data_ptr(), (256, 256, 256), w["ghosts"], order,
                                       w["lo"][0], float(w["h"][0]), w["chi_floor"], 1.0, g.stream)
    assert rc == z4c.Z4C_ERR_UNSUPPORTED
