"""CPU checks of the arithmetic the kernels rely on, restated step by step in exact rational
arithmetic (fractions) with IEEE rounding applied where the device rounds.  They pin the error
bounds the device code's comments state; the GPU parity tests check the kernels themselves.

* Tang's table-driven exponential of the Boltzmann factors (ACM TOMS 15, 1989): within 2 ulp of
  exp over the range it serves.
* The window quotients ceil((nu - cut - nu_min)/dnu) and floor((nu + cut - nu_min)/dnu): the
  reciprocal-multiply shortcut gives the same integers as the rounded division whenever it is
  taken (near-integer quotients fall back to the division).
* The 12-bit state codes: FP32 scaling of the FP64 difference E - Emin stays within one code of
  the exact floor, the slack the prefilter's bounds allow.
"""
import math
import os
import re
from fractions import Fraction

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2609_17273_b300", "csrc", "kernels_lines.cu")


def _rn(q: Fraction) -> float:
    """Round a rational to the nearest double (ties to even)."""
    return float(q)


def _fma(a: float, b: float, c: float) -> float:
    return _rn(Fraction(a) * Fraction(b) + Fraction(c))


def _table():
    s = open(SRC).read()
    body = s[s.index("kExp2J64[64] = {"):]
    body = body[:body.index("};")]
    return [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]


def _exp_tang(x: float, tab) -> float:
    # the device steps: n by the 1.5 2^52 shift, r = x - n ln2/64 in two parts, e^r - 1 by a
    # degree-5 Taylor polynomial, 2^(j/64) from the table, the power of two into the exponent
    tn = _fma(x, 92.332482616893657, float.fromhex("0x1.8p52"))
    n = tn - float.fromhex("0x1.8p52")
    ni = int(n)
    r = _fma(-n, float.fromhex("0x1.abc9e3b39803fp-62"), _fma(-n, float.fromhex("0x1.62e42fefa39efp-7"), x))
    p = _fma(_fma(_fma(_fma(r, 1.0 / 120.0, 1.0 / 24.0), r, 1.0 / 6.0), r, 0.5), r, 1.0)
    q = r * p
    t = tab[ni & 63]
    v = _fma(t, q, t)
    return math.ldexp(v, ni >> 6)


def test_tang_exponential_within_two_ulp():
    tab = _table()
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(-699.0, 699.0, 1500), rng.uniform(-1.0, 1.0, 300),
                         np.array([0.0, -0.0, 1e-300, -1e-20, 0.5 * math.log(2) / 64, -699.9, 699.9])])
    worst = 0.0
    for x in xs:
        got = _exp_tang(float(x), tab)
        ref = math.exp(float(x))
        err = abs(got - ref) / math.ulp(ref)
        worst = max(worst, err)
    assert worst <= 2.0, worst


def _quotient_clear(q: float) -> bool:
    return abs(q - round(q)) > 2.0 ** -51 * abs(q)


def test_window_quotient_shortcut_matches_the_division():
    rng = np.random.default_rng(3)
    cases = []
    random_taken = random_n = 0
    for den in (0.01, 0.001, 0.1, 0.002, 1.0 / 3.0, 0.3, 7.25e-4, 1e-5):
        inv = 1.0 / den
        uniform = rng.uniform(-50.0, 50000.0, 400)
        random_n += uniform.size
        random_taken += sum(_quotient_clear(float(n) * inv) for n in uniform)
        nums = list(uniform)
        # near-integer and exactly integer quotients
        ks = rng.integers(-1000, 3_000_000, 200)
        nums += [float(k) * den for k in ks]
        nums += [math.nextafter(float(k) * den, math.inf) for k in ks[:50]]
        nums += [math.nextafter(float(k) * den, -math.inf) for k in ks[:50]]
        nums += [0.0, -0.0, 5e-324, -5e-324]
        cases += [(n, den, inv) for n in nums]
    taken = 0
    for num, den, inv in cases:
        q = num * inv
        exact = Fraction(num) / Fraction(den)
        div = num / den  # the rounded division (what __ddiv_rn returns)
        if _quotient_clear(q):
            taken += 1
            assert math.ceil(q) == math.ceil(div) == math.ceil(exact), (num, den)
            assert math.floor(q) == math.floor(div) == math.floor(exact), (num, den)
    assert taken > 0.5 * len(cases)
    assert random_taken >= 0.99 * random_n  # the division is the rare path for arbitrary windows


def test_state_codes_within_one_code():
    rng = np.random.default_rng(5)
    for emin, span in ((0.0, 1.6e5), (1e6, 1.0), (-3000.0, 5e4), (2.5e4, 1e11), (0.0, 3e30)):
        E = emin + rng.uniform(0.0, span, 4000)
        E = np.concatenate([E, [emin, emin + span]])
        inv_res = (4094 - 2) / span
        inv_f = np.float32(inv_res)
        d = (E - emin).astype(np.float64)                 # FP64 difference
        x32 = np.floor(d.astype(np.float32) * inv_f)      # FP32 scaling
        exact = np.array([math.floor((Fraction(float(e)) - Fraction(emin)) * Fraction(inv_res)) for e in E])
        assert np.all(np.abs(x32.astype(np.float64) - exact) <= 1), (emin, span)
