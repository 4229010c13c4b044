"""Each planted mistake in the oracle (a wrong sign, a dropped term, a wrong
index, a transposed operand, a wrong monomial order) must make at least one
pin fail.  The mistakes are compiled into throw-away copies of oracle.c on
the CPU; the real oracle is built without them."""

import os

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins


def _pins_pass():
    checks = [
        lambda: pins.test_bruteforce_m61(3, 4, 20, 25, 3),
        lambda: pins.test_bruteforce_i64(11),
        lambda: pins.test_power_of_linear_form(3, 4, 5),
        lambda: pins.test_evaluation_at_points("m61", 1),
        lambda: pins.test_commutative_and_identity_and_shift(),
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5])
def test_planted_mistake_is_caught(plant, tmp_path):
    path = oracle.build_variant(plant, str(tmp_path / f"liboracle_plant{plant}.so"))
    saved = oracle._lib
    oracle._lib = oracle._load(path)
    try:
        assert not _pins_pass(), f"planted mistake {plant} passed every pin"
    finally:
        oracle._lib = saved


def test_unplanted_build_passes():
    assert _pins_pass()
