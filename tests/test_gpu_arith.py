"""Device md arithmetic (mdls_vec_op) against the oracle's exact-then-rounded
operations, elementwise, for dd, qd and od, on random, mixed-magnitude and
cancelling operands."""
import numpy as np
import pytest

import oracle
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def operands(p, n, seed):
    rng = np.random.default_rng(seed)
    def draw(scale_exp):
        x = np.zeros((p, n))
        x[0] = rng.uniform(-1, 1, n) * 2.0 ** scale_exp
        for i in range(1, p):
            x[i] = x[i - 1] * 2.0 ** -54 * rng.uniform(-1, 1, n)
        return x
    a = draw(rng.integers(-20, 20, n))
    b = draw(rng.integers(-20, 20, n))
    k = n // 4
    b[:, :k] = -a[:, :k]                                # exact cancellation
    b[p - 1, :k] += a[p - 1, :k] * 2.0 ** -30           # leaves a tiny remainder
    b[:, k:2 * k] = draw(rng.integers(-200, -100, n))[:, :k]   # far smaller operand
    return a, b


def exact_ref(op, a, b, c=None):
    n = a.shape[1]
    out = np.zeros_like(a)
    for i in range(n):
        if op == "fma":
            out[:, i] = oracle.add(c[:, i], oracle.mul(a[:, i], b[:, i]))
        elif op == "sqrt":
            out[:, i] = oracle.sqrt(a[:, i])
        else:
            out[:, i] = getattr(oracle, op)(a[:, i], b[:, i])
    return out


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "fma", "sqrt"])
def test_vec_op_matches_oracle(p, op):
    import paper_2110_08375_gb300 as mdls
    n = 4096
    a, b = operands(p, n, 17 * p + len(op))
    if op == "sqrt":
        a = a * np.sign(a[0])[None, :]                     # nonnegative
    c0 = operands(p, n, 99 + p)[0] if op == "fma" else None
    cd = to_dev(c0) if c0 is not None else None
    got = to_host(mdls.mdls_vec_op(op, to_dev(a), to_dev(b), cd))
    ref = exact_ref(op, a, b, c0)
    d = np.abs(oracle.diff(got, ref))
    # error relative to the operands' scale (the bound md arithmetic promises)
    if op in ("add", "sub"):
        scale = np.abs(a[0]) + np.abs(b[0])
    elif op == "mul":
        scale = np.abs(a[0] * b[0])
    elif op == "fma":
        scale = np.abs(c0[0]) + np.abs(a[0] * b[0])
    elif op == "div":
        scale = np.abs(a[0] / b[0])
    else:
        scale = np.sqrt(np.abs(a[0]))
    bound = {2: 2.0 ** -100, 4: 2.0 ** -204, 8: 2.0 ** -410}[p]
    worst = np.max(d / np.where(scale > 0, scale, 1.0))
    assert worst <= bound, (op, p, worst)
    # outputs are normalised: each limb within 2 ulps of the one above
    for i in range(p - 1):
        hi = np.abs(got[i])
        ok = (np.abs(got[i + 1]) <= 2 * np.spacing(hi)) | (hi == 0)
        assert ok.all(), (op, p, i)
