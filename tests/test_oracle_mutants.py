"""Each planted mistake in the oracle (oracle.c, PLANT=n) must be caught by
at least two independent pins: this shows the pins are sharp enough to notice a dropped
term, a wrong comparison, a missing root or an invalid selection."""
import pytest

import oracle
import pins

PLANTS = {
    1: "BZ moves a neighbour with equal degree",
    2: "CSD counts SD >= k instead of SD > k",
    3: "K-SuperiorInsert keeps removed vertices in V_k",
    4: "DeleteRemove cascades at cd <= k instead of cd < k",
    5: "equal-core deletion roots only one endpoint",
    6: "selection ignores the second constrained endpoint",
}


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=lambda p: f"plant{p}")
def test_planted_mistake_is_caught(plant):
    oracle.build(plant)
    caught = []
    for check in pins.ALL:
        try:
            check(plant)
        except AssertionError:
            caught.append(check.__name__)
        except (ValueError, oracle.OracleError):
            caught.append(check.__name__)
    assert len(caught) >= 2, f"fewer than two pins catch: {PLANTS[plant]} (caught by {caught})"
