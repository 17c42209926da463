"""The product's flop convention (paper_2110_08375_gb300.opcount) agrees with
the oracle's operation counters, and the Table 1 multipliers it uses are the
paper's (Section 1.1, Table 1)."""
import numpy as np
import pytest

import oracle
import synth
from paper_2110_08375_gb300 import opcount


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n", [(9, 5), (16, 11), (30, 30)])
def test_lstsq_counts_match_oracle_counters(p, m, n):
    A, b = synth.lstsq_problem(p, m, n, seed=2, tag="opc")
    oracle.reset_counts()
    oracle.lstsq(A, b)
    got = oracle.counts()
    exp = opcount.lstsq_counts(m, n)
    # opcount leaves out the extra division of the x0 > 0 reflector branch
    # and treats a square matrix's last column as the identity reflector
    if m == n and got["flip"]:
        L = 1
        exp["mul"] += 2 * L + 1
        exp["add"] += 2 * L
    assert got["add"] == exp["add"]
    assert got["mul"] == exp["mul"]
    assert got["sqrt"] == exp["sqrt"]
    assert got["div"] == exp["div"] + got["pos_branch"]


@pytest.mark.parametrize("p", [2, 4, 8])
def test_qr_counts_with_q_match_oracle(p):
    m, n = 14, 9
    A, _ = synth.lstsq_problem(p, m, n, seed=3, tag="opc")
    oracle.reset_counts()
    oracle.qr(A, want_q=True)
    got = oracle.counts()
    exp = opcount.qr_counts(m, n, want_q=True)
    assert (got["add"], got["mul"], got["sqrt"]) == (exp["add"], exp["mul"], exp["sqrt"])
    assert got["div"] == exp["div"] + got["pos_branch"]


def test_table1_multipliers_are_the_papers():
    for p in (2, 4, 8):
        for op in ("add", "mul", "div"):
            assert opcount.TABLE1_SIGMA[p][op] == oracle.TABLE1[p][op][4]


def test_leading_term():
    """Square n: about (2/3) n^3 md mul and add for QR of [A|b] + back
    substitution; the Table 1 flops at n=1024 follow."""
    n = 1024
    c = opcount.lstsq_counts(n, n)
    assert abs(c["mul"] / (2 * n ** 3 / 3) - 1) < 0.01
    assert abs(c["add"] / (2 * n ** 3 / 3) - 1) < 0.01


def test_device_fma_cost_structure():
    # dd: two_prod + two_sum (order 0), 2 FMAs + 2 adds (order 1), one two_sum
    # (renorm); a two_sum is one FP64 addition, its error formed on the
    # integer pipe
    assert opcount.fma_cost(2) == (2 + 1 + 2 + 2 + 1, 3 + 1 + 4 + 2 + 1)
    assert opcount.add_cost(2) == (1 + 2 + 1, 1 + 2 + 1)
    assert opcount.fma_cost(4)[0] < opcount.fma_cost(8)[0]


def test_gemm_loop_cost_defers_renormalisation():
    """The product loops renormalise once per 16 steps: per md FMA they issue
    the bins of md_fma plus a sixteenth of its renormalisation."""
    for p in (2, 4, 8):
        full, rn = opcount.fma_cost(p)[0], opcount.renorm_cost(p)[0]
        assert opcount.gemm_fma_cost(p) == full - rn + rn / 16
        assert opcount.gemm_fma_cost(p, renorm_every=1) == full


def test_two_sum_form_per_bin():
    """The device's two_sum form by bin (csrc/md.cuh two_sum_pd): one FP64
    addition (error on the integer pipe) for dd, qd and od's first five
    bins; Fast2Sum (three) in od's last bins and renormalisation."""
    for p in (2, 4):
        assert all(opcount.two_sum_cost(p, d) == opcount.TWO_SUM_INT for d in range(p + 1))
    assert [opcount.two_sum_cost(8, d)[0] for d in range(9)] == [1, 1, 1, 1, 1, 3, 3, 3, 3]
    # od md FMA in the product loops: bins 0..4 hold 1+4+9+16+25 two_sums at
    # one instruction, bins 5 and 6 36+49 at three; 28 two_prods; the last
    # bin's 8 FMAs + 7 low parts + 49 errors; 13 renormalisation two_sums
    # once per 16 steps
    expect = (55 * 1 + 85 * 3) + 28 * 2 + (8 + 7 + 49) + 13 * 3 / 16
    assert abs(opcount.gemm_fma_cost(8) - expect) < 1e-9


@pytest.mark.parametrize("m,n,t", [(10, 7, 3), (16, 16, 4), (9, 9, 9)])
def test_product_counts_by_enumeration(m, n, t):
    # one md FMA per (output, term) of X = W^T C, C += Y X, G = Y^T Y (upper
    # triangle) and W = -Y T (T upper triangular), enumerated term by term
    trail = wy = 0
    for j0 in range(0, n, t):
        w, r = min(t, n - j0), m - j0
        nc = n + 1 - (j0 + w)
        if nc <= 0:
            continue
        trail += sum(1 for _i in range(w) for _j in range(nc) for _k in range(r))
        trail += sum(1 for _i in range(r) for _j in range(nc) for _k in range(w))
        wy += sum(1 for i in range(w) for j in range(i, w) for _k in range(r))
        wy += sum(1 for _i in range(r) for j in range(w) for _k in range(j + 1))
    assert opcount.trailing_md_fmas(m, n, t, extra_cols=1) == trail
    assert opcount.wy_md_fmas(m, n, t, extra_cols=1) == wy
