"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import pytest

import pins


@pytest.mark.parametrize("check", pins._all_checks(), ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check()
