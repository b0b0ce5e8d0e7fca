"""The constants of the table-driven exponential of the Boltzmann factors (Tang's method, ACM TOMS
15 (1989)): every table entry is 2^(j/64) correctly rounded to FP64, and ln2/64 is split into a
leading part and a remainder whose sum is ln2/64 to far beyond FP64 precision.  Checked in
60-digit decimal arithmetic against the literals in the CUDA source (no GPU needed)."""
import os
import re
from decimal import Decimal, getcontext

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2609_17273_b300", "csrc", "kernels_lines.cu")


def _source():
    with open(SRC) as f:
        return f.read()


def test_table_entries_are_correctly_rounded():
    getcontext().prec = 60
    s = _source()
    body = s[s.index("kExp2J64[64] = {"):]
    body = body[:body.index("};")]
    vals = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == 64
    for j, v in enumerate(vals):
        exact = Decimal(2) ** (Decimal(j) / 64)
        assert v == float(exact), j
        ulp = Decimal(float.fromhex("0x1p-52")) * (1 if v < 2 else 2)
        assert abs(Decimal(v) - exact) <= ulp / 2


def test_ln2_split_and_reciprocal():
    getcontext().prec = 60
    s = _source()
    hi = float.fromhex(re.search(r"0x1\.62e42fefa39efp-7", s).group(0))
    lo = float.fromhex(re.search(r"0x1\.abc9e3b39803fp-62", s).group(0))
    ln2_64 = Decimal(2).ln() / 64
    assert abs(Decimal(hi) + Decimal(lo) - ln2_64) < Decimal(10) ** -35
    assert "92.332482616893657" in s
    assert abs(Decimal("92.332482616893657") - 64 / Decimal(2).ln()) < Decimal(10) ** -14
