"""Plain evaluator of scalar expressions (the oracle of the device Eval path).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may use it.

An expression is a postfix list of terms (Sec. 3.2.1 builds the same
expressions from overloaded operators): ("scalar", name) pushes the value of
a named scalar, ("const", c) pushes c, a binary operator pops b then a and
pushes a op b, a unary one pops a and pushes op(a).  Every operation is one
IEEE float64 operation in numpy (+ - * / and sqrt correctly rounded, min and
max as fmin/fmax: a NaN operand yields the other one); sin, cos, exp and log
come from the host's libm.  Nothing is simplified or folded.
"""

from __future__ import annotations

import numpy as np

BINARY = {"add", "sub", "mul", "div", "min", "max"}
UNARY = {"neg", "recip", "sqrt", "abs", "sin", "cos", "exp", "log"}


def expr_eval(terms, values: dict) -> float:
    st = []
    with np.errstate(all="ignore"):
        for t in terms:
            op = t[0]
            if op == "scalar":
                st.append(np.float64(values[t[1]]))
            elif op == "const":
                st.append(np.float64(t[1]))
            elif op in BINARY:
                b = st.pop()
                a = st.pop()
                st.append(
                    {
                        "add": lambda: a + b,
                        "sub": lambda: a - b,
                        "mul": lambda: a * b,
                        "div": lambda: a / b,
                        "min": lambda: np.fmin(a, b),
                        "max": lambda: np.fmax(a, b),
                    }[op]()
                )
            elif op in UNARY:
                a = st.pop()
                st.append(
                    {
                        "neg": lambda: -a,
                        "recip": lambda: np.float64(1.0) / a,
                        "sqrt": lambda: np.sqrt(a),
                        "abs": lambda: np.abs(a),
                        "sin": lambda: np.sin(a),
                        "cos": lambda: np.cos(a),
                        "exp": lambda: np.exp(a),
                        "log": lambda: np.log(a),
                    }[op]()
                )
            else:
                raise ValueError(f"unknown term {t!r}")
    if len(st) != 1:
        raise ValueError("the terms leave %d values" % len(st))
    return float(st[0])
