"""The CPU oracle against facts fixed outside it (see tests/oracle_pins.py)."""
import pytest

import oracle
import oracle_pins as P

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def lib_path():
    return oracle.ensure_built()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(lib_path, pin):
    pin(lib_path)
