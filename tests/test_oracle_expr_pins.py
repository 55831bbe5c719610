"""Pins of the scalar-expression oracle against exact rational arithmetic.

On integer-valued inputs every + - * stays exact in float64 (|values| < 2^53),
so the oracle must equal the exact Fraction result; a single division or
square root must equal the correctly rounded exact value; min, max, abs and
neg are exact.  IEEE special values follow the fmin/fmax and division rules.
"""

import math
import random
from fractions import Fraction

import pytest

import oracle

OPS = ["add", "sub", "mul", "min", "max", "neg", "abs"]


def _exact(terms, vals):
    st = []
    for t in terms:
        if t[0] == "scalar":
            st.append(Fraction(vals[t[1]]))
        elif t[0] == "const":
            st.append(Fraction(t[1]))
        elif t[0] in ("add", "sub", "mul", "min", "max"):
            b, a = st.pop(), st.pop()
            st.append({"add": a + b, "sub": a - b, "mul": a * b, "min": min(a, b), "max": max(a, b)}[t[0]])
        else:
            a = st.pop()
            st.append(-a if t[0] == "neg" else abs(a))
    return st[0]


def _random_terms(rng, depth):
    if depth == 0 or rng.random() < 0.3:
        return [("scalar", rng.choice("xyzw"))] if rng.random() < 0.7 else [("const", rng.randint(-9, 9))]
    op = rng.choice(OPS)
    if op in ("neg", "abs"):
        return _random_terms(rng, depth - 1) + [(op,)]
    return _random_terms(rng, depth - 1) + _random_terms(rng, depth - 1) + [(op,)]


def test_exact_on_integers():
    rng = random.Random(5)
    for _ in range(300):
        terms = _random_terms(rng, 4)
        vals = {k: rng.randint(-50, 50) for k in "xyzw"}
        assert oracle.expr_eval(terms, vals) == float(_exact(terms, vals))


def test_single_rounding_of_division_and_sqrt():
    rng = random.Random(9)
    for _ in range(200):
        a, b = rng.randint(-10**6, 10**6), rng.randint(1, 10**6)
        assert oracle.expr_eval([("scalar", "a"), ("scalar", "b"), ("div",)], {"a": a, "b": b}) == float(Fraction(a, b))
        k = rng.randint(0, 10**7)
        assert oracle.expr_eval([("scalar", "k"), ("sqrt",)], {"k": k * k}) == float(k)
        assert oracle.expr_eval([("scalar", "k"), ("sqrt",)], {"k": k}) == math.sqrt(k)  # correctly rounded (IEEE)


def test_special_values():
    ev = oracle.expr_eval
    assert ev([("const", 1.0), ("const", 0.0), ("div",)], {}) == math.inf
    assert math.isnan(ev([("const", 0.0), ("const", 0.0), ("div",)], {}))
    assert ev([("scalar", "a"), ("scalar", "b"), ("min",)], {"a": math.nan, "b": 2.0}) == 2.0
    assert ev([("scalar", "a"), ("scalar", "b"), ("max",)], {"a": 3.0, "b": math.nan}) == 3.0
    assert math.copysign(1.0, ev([("const", -0.0), ("neg",)], {})) == 1.0
    assert ev([("const", 4.0), ("recip",)], {}) == 0.25


def test_malformed_terms():
    with pytest.raises(ValueError):
        oracle.expr_eval([("const", 1.0), ("const", 2.0)], {})
