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
import numpy as np

from test_oracle_pins import ALL_CHECKS, E4M3_CHECKS, SDDMM_CHECKS

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


# Planted mistakes in the E4M3 block-value helper: the scale broadcast along
# a block's rows or columns instead of over the whole block, scales taken in
# the block-CSR order of the pins' pattern (rows 1, 0) instead of the
# pattern's order, and the sign bit dropped.
def _mut_scale_rows(codes, scales):
    return oracle.e4m3_to_f64(codes) * np.asarray(scales, np.float64).reshape(1, -1, 1)


def _mut_scale_cols(codes, scales):
    return oracle.e4m3_to_f64(codes) * np.asarray(scales, np.float64).reshape(1, 1, -1)


def _mut_csr_order(codes, scales):
    s = np.asarray(scales, np.float64)[np.argsort([1, 0], kind="stable")]
    return oracle.e4m3_to_f64(codes) * s[:, None, None]


def _mut_unsigned(codes, scales):
    return np.abs(oracle.e4m3_to_f64(codes)) * np.asarray(scales, np.float64)[:, None, None]


@pytest.mark.parametrize("fn", [_mut_scale_rows, _mut_scale_cols, _mut_csr_order, _mut_unsigned],
                         ids=lambda f: f.__name__)
def test_e4m3_pins_catch_planted_mistake(fn):
    failed = []
    for check in E4M3_CHECKS:
        try:
            check(fn)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, "no pin detects " + fn.__name__
