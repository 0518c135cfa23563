"""Appendix A.2's closed forms (equal partition, bucket size) from the text
fixture tests/golden/appendix_a2_closed_forms.txt, evaluated by hand from the
formulas: the oracle and the C ABI must both reproduce every line."""
import os
from fractions import Fraction

import pytest

from oracle import plan as P
from paper_2303_16999_gb300 import spmm as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_a2_closed_forms.txt")


def _cases(kind):
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split(":")
        f = lhs.split()
        if f[0] == kind:
            out.append(([int(v) for v in f[1:]], [int(v) for v in rhs.split()]))
    return out


@pytest.fixture(scope="module")
def native():
    from paper_2303_16999_gb300 import build
    build.build()
    return S.lib()


def test_fixture_is_populated():
    assert len(_cases("partition")) >= 5 and len(_cases("bucket")) >= 4


@pytest.mark.parametrize("args,want", _cases("partition"))
def test_equal_partition(args, want, native):
    m, q = args
    assert P.equal_partition(m, q) == want
    assert S.spmm_equal_partition(m, q) == want
    assert sum(want) == m


@pytest.mark.parametrize("args,want", _cases("bucket"))
def test_bucket_size(args, want, native):
    m, k, num, den, qm, qk = args
    assert P.bucket_size(m, k, Fraction(num, den), qm, qk) == want[0]
    assert S.spmm_bucket_size(m, k, num, den, qm, qk) == want[0]
