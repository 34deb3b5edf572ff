"""The algorithmic flop count of the oracle's RK4 step (oracle/flopcount.py,
the oracle's C source on a counting scalar type): it runs, the step succeeds,
the count grows with the stencil width (orders 2 < 4 < 6), and the one power
per cell and stage is the enforcement's det^(-1/3) at every order."""
import pytest

from oracle import flopcount


@pytest.fixture(scope="module")
def counts():
    return {o: flopcount.count(o) for o in (2, 4, 6)}


def test_flop_count_runs_and_orders(counts):
    for o, c in counts.items():
        assert c["rc"] == 0 and c["order"] == o
        assert c["add"] > 1000 and c["mul"] > 1000
    f = [counts[o]["flops_per_cell_stage"] for o in (2, 4, 6)]
    assert f[0] < f[1] < f[2]
    # the enforcement's det^(-1/3) is the only power: once per cell and stage
    assert all(abs(counts[o]["pow"] - 1.0) < 1e-12 for o in (2, 4, 6))
    assert all(counts[o]["sqrt"] == 0 for o in (2, 4, 6))
