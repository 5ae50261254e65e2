"""The oracle against facts fixed outside it (brute force, closed forms,
invariants).  CPU only."""
import pytest

import oracle.conker_oracle as O
from tests import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(check):
    assert check(O)
