"""The literal constants of the double-float assembly (k_solve.cu) against their
definitions, computed here in 60-digit decimal arithmetic: each hi/lo pair is the FP32
value nearest to the constant followed by the FP32 value nearest to the rest, so the
pair carries the constant to about 2^-48 relative.  A mistyped digit in a table entry
fails here, on the CPU."""
import os
import re
from decimal import Decimal, getcontext

import numpy as np
import pytest

getcontext().prec = 60
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1708_02207_gb300", "csrc", "k_solve.cu")


def _source():
    with open(SRC) as fh:
        return fh.read()


def _floats(text):
    return [float(x) for x in re.findall(r"(-?\d+\.\d+(?:e[-+]?\d+)?)f", text)]


def _array(name):
    m = re.search(name + r"\[[^\]]*\](?:\[2\])?\s*=\s*\{(.*?)\};", _source(), re.S)
    assert m, name
    v = _floats(m.group(1))
    return list(zip(v[0::2], v[1::2]))


def _scalar(name):
    m = re.search(name + r"\s*=\s*(-?\d+\.\d+(?:e[-+]?\d+)?)f", _source())
    assert m, name
    return float(m.group(1))


def _pair_ok(pair, exact):
    hi, lo = (np.float32(x) for x in pair)
    assert float(hi) == pair[0] and float(lo) == pair[1]   # the literals are FP32 values
    assert hi == np.float32(float(exact))                  # hi: the FP32 value nearest to it
    rest = exact - Decimal(float(hi))
    assert lo == np.float32(float(rest))                   # lo: the FP32 value nearest to the rest
    err = abs(exact - Decimal(float(hi)) - Decimal(float(lo))) / abs(exact)
    assert err <= Decimal(2) ** -48


def test_table_of_2_to_the_j_over_16():
    table = _array("kExp2J16")
    assert len(table) == 16
    for j, pair in enumerate(table):
        _pair_ok(pair, Decimal(2) ** (Decimal(j) / 16))


def test_reciprocal_factorials():
    pairs = _array("kInvFact")
    assert len(pairs) == 5
    fact = 1
    for n, pair in enumerate(pairs):
        fact *= max(n, 1)
        if n <= 2:
            assert pair == (1.0 / fact, 0.0)
        else:
            _pair_ok(pair, Decimal(1) / fact)
    assert np.float32(_scalar("kInv120")) == np.float32(1.0 / 120)
    assert np.float32(_scalar("kInv720")) == np.float32(1.0 / 720)


def test_ln2_split_and_reduction_factor():
    ln2 = Decimal(2).ln()
    _pair_ok((_scalar("kLn2Hi"), _scalar("kLn2Lo")), ln2)
    assert np.float32(_scalar("kSixteenOverLn2")) == np.float32(float(16 / ln2))
    # ln2/16 is formed by scaling the pair by 1/16, which is exact in binary
    assert float(np.float32(_scalar("kLn2Hi")) * np.float32(0.0625)) == _scalar("kLn2Hi") / 16
