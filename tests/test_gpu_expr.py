"""Device scalar expressions (Eval, Sec. 3.2.1) against the oracle's evaluator.

* Random postfix expressions over four scalars with the IEEE operators
  (+ - * / sqrt neg recip abs min max): bit for bit equal to the oracle, with
  and without the freeze-time folding and rewrites taking effect.
* sin, cos, exp, log: within 4 ulp of the host's libm (CUDA documents at most
  2 ulp for these in double precision; the host's libm adds up to 1).
* Freezing: equal subexpressions become one instruction, constant subtrees
  fold, the value-keeping rewrites apply, the worked example of Sec. 3.2.1.
* Fusion: y += e x with e evaluated inside the AXPY equals executing e and
  then the AXPY; ordering across contexts follows the marking rules.
"""

import ctypes as C
import math
import random

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402

V = C.c_void_p
IEEE_BIN = ["add", "sub", "mul", "div", "min", "max"]
IEEE_UN = ["neg", "recip", "sqrt", "abs"]


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    apcg.load()
    ctx = apcg.ctx_create()
    sc = {k: apcg.scalar_create() for k in "xyzw"}
    out = apcg.scalar_create()
    yield ctx, sc, out
    for s in list(sc.values()) + [out]:
        apcg.call("apcg_scalar_destroy", V(s))
    apcg.call("apcg_ctx_destroy", V(ctx))


def _set(ctx, sc, vals):
    for k, v in vals.items():
        apcg.call("apcg_scalar_set_async", V(ctx), V(sc[k]), C.c_double(v))


def _run(ctx, sc, out, terms):
    e = apcg.expr_create(terms, sc)
    try:
        apcg.call("apcg_expr_execute_async", V(ctx), V(e), V(out))
        return apcg.scalar_get(out), apcg.expr_describe(e)
    finally:
        apcg.call("apcg_expr_destroy", V(e))


def _same(a, b):
    return (math.isnan(a) and math.isnan(b)) or (a == b and math.copysign(1, a) == math.copysign(1, b))


def _random_terms(rng, depth):
    if depth == 0 or rng.random() < 0.25:
        r = rng.random()
        if r < 0.7:
            return [("scalar", rng.choice("xyzw"))]
        return [("const", rng.choice([0.0, 1.0, -1.0, 2.0, 0.1, rng.uniform(-5, 5)]))]
    if rng.random() < 0.35:
        return _random_terms(rng, depth - 1) + [(rng.choice(IEEE_UN),)]
    return _random_terms(rng, depth - 1) + _random_terms(rng, depth - 1) + [(rng.choice(IEEE_BIN),)]


def test_random_ieee_expressions_bit_exact(env):
    ctx, sc, out = env
    rng = random.Random(11)
    for _ in range(150):
        terms = _random_terms(rng, 5)
        vals = {k: rng.choice([rng.uniform(-10, 10), rng.uniform(0, 1e-3), float(rng.randint(-4, 4))]) for k in "xyzw"}
        _set(ctx, sc, vals)
        got, _ = _run(ctx, sc, out, terms)
        ref = oracle.expr_eval(terms, vals)
        assert _same(got, ref), (terms, vals, got, ref)


@pytest.mark.parametrize("op", ["sin", "cos", "exp", "log"])
def test_transcendental_within_ulp(env, op):
    ctx, sc, out = env
    rng = random.Random(3)
    for _ in range(40):
        v = rng.uniform(0.01, 20.0) if op == "log" else rng.uniform(-20.0, 20.0)
        _set(ctx, sc, {"x": v})
        got, _ = _run(ctx, sc, out, [("scalar", "x"), (op,)])
        ref = oracle.expr_eval([("scalar", "x"), (op,)], {"x": v})
        assert abs(got - ref) <= 4 * math.ulp(ref), (op, v, got, ref)


def test_freezing(env):
    ctx, sc, out = env
    _set(ctx, sc, {"x": 1.5, "y": -0.25, "z": 3.0, "w": 2.0})
    # the worked example of Sec. 3.2.1: sin(((x + y) / z) * z) + 15, z loaded once
    terms = [("scalar", "x"), ("scalar", "y"), ("add",), ("scalar", "z"), ("div",), ("scalar", "z"), ("mul",),
             ("sin",), ("const", 15.0), ("add",)]
    got, d = _run(ctx, sc, out, terms)
    assert d["inputs"] == 3 and d["instructions"] == 9  # x y add z div mul sin 15 add
    assert abs(got - oracle.expr_eval(terms, {"x": 1.5, "y": -0.25, "z": 3.0})) <= 4 * math.ulp(got)
    # common subexpression: (x + y) * (x + y) computes the sum once
    _, d = _run(ctx, sc, out, [("scalar", "x"), ("scalar", "y"), ("add",), ("scalar", "x"), ("scalar", "y"), ("add",),
                               ("mul",)])
    assert d["instructions"] == 4
    # constant folding and value-keeping rewrites
    got, d = _run(ctx, sc, out, [("const", 2.0), ("const", 3.0), ("add",), ("scalar", "x"), ("mul",)])
    assert d["instructions"] == 3 and got == 7.5
    got, d = _run(ctx, sc, out, [("scalar", "x"), ("const", 1.0), ("mul",), ("const", 0.0), ("sub",), ("neg",), ("neg",)])
    assert d["instructions"] == 1 and got == 1.5
    # x + 0 is not rewritten (-0 + 0 = +0)
    _set(ctx, sc, {"x": -0.0})
    got, d = _run(ctx, sc, out, [("scalar", "x"), ("const", 0.0), ("add",)])
    assert d["instructions"] == 3 and math.copysign(1, got) == 1.0


def test_malformed_expressions(env):
    ctx, sc, out = env
    for terms in ([("add",)], [("scalar", "x"), ("scalar", "y")], [("const", 1.0), ("neg",), ("mul",)]):
        with pytest.raises(apcg.ApcgError):
            apcg.expr_create(terms, sc)


def test_fused_axpy_and_marking(env):
    ctx, sc, out = env
    n = 100_003
    dev = torch.device("cuda:0")
    x = torch.randn(n, dtype=torch.float64, device=dev)
    y1 = torch.randn(n, dtype=torch.float64, device=dev)
    y2 = y1.clone()
    vx, v1, v2 = apcg.vec_wrap(x), apcg.vec_wrap(y1), apcg.vec_wrap(y2)
    other = apcg.ctx_create()
    # the input scalar is produced on another context: the fused AXPY must wait for it
    apcg.call("apcg_scalar_set_async", V(other), V(sc["x"]), C.c_double(0.75))
    apcg.call("apcg_scalar_set_async", V(other), V(sc["y"]), C.c_double(4.0))
    terms = [("scalar", "x"), ("scalar", "y"), ("sqrt",), ("div",), ("neg",)]  # -(x / sqrt(y)) = -0.375
    e = apcg.expr_create(terms, sc)
    apcg.reset_counters()
    apcg.call("apcg_vec_axpy_expr_async", V(ctx), V(v1), V(e), V(vx))
    c = apcg.get_counters()
    assert c["kernel_launches"] == 1 and c["waits_inserted"] + c["waits_elided"] >= 1
    apcg.call("apcg_expr_execute_async", V(ctx), V(e), V(out))
    apcg.call("apcg_vec_axpy_async", V(ctx), V(v2), V(out), 0, V(vx))
    apcg.call("apcg_ctx_synchronize", V(ctx))
    assert apcg.scalar_get(out) == -0.375
    assert torch.equal(y1, y2)
    apcg.call("apcg_expr_destroy", V(e))
    for h in (vx, v1, v2):
        apcg.call("apcg_vec_destroy", V(h))
    apcg.call("apcg_ctx_destroy", V(other))
