"""The CPU oracle against closed forms, brute force, golden fixtures and the
invariants of Section IV (see tests/pins.py for what pins what)."""
import pytest

import pins


@pytest.mark.parametrize("check", pins.ALL, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(0)
