"""Planted mistakes in a private copy of the oracle (CPU only).

Each mutant is the oracle's own C source compiled with one ``-D`` flag that
plants a plausible error (a transposed block, a flipped sign on one block, an
off-by-one X row, a dropped output row; for the sampled product, a block
stored transposed and a lost term of the sum over n).  At least one pin must fail for
every mutant; otherwise the pins could not tell that mistake from the
definition.
"""
import os

import pytest

import oracle
from oracle import build as obuild
from test_oracle_pins import ALL_CHECKS, SDDMM_CHECKS

MUTANTS = ["ORACLE_MUTANT_TRANSPOSE", "ORACLE_MUTANT_SIGN",
           "ORACLE_MUTANT_COLSHIFT", "ORACLE_MUTANT_DROP_LAST"]


@pytest.mark.parametrize("flag", MUTANTS)
def test_pins_catch_planted_mistake(flag, tmp_path):
    path = obuild.build_variant(os.path.join(str(tmp_path), flag + ".so"), [flag])
    lib = oracle.load_variant(path)
    failed = []
    for check in ALL_CHECKS:
        try:
            check(lib)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, "no pin detects " + flag


@pytest.mark.parametrize("flag", ["ORACLE_MUTANT_SDDMM_TRANSPOSE", "ORACLE_MUTANT_SDDMM_DROP_TERM"])
def test_sddmm_pins_catch_planted_mistake(flag, tmp_path):
    path = obuild.build_variant(os.path.join(str(tmp_path), flag + ".so"), [flag])
    lib = oracle.load_variant(path)
    failed = []
    for check in SDDMM_CHECKS:
        try:
            check(lib)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, "no pin detects " + flag
