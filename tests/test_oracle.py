"""Pins of the CPU oracle against facts fixed outside it: a hand-worked
example, dense brute force, a library routine, exact integer arithmetic and
the invariants of the partition (Sec. III-A, Fig. 3b)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import OraclePlan, csr_spmv, csr_absdot
from paper_2203_02530_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dense(n, rp, ci, va):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i, ci[k]] += va[k]
    return A


# ---------------------------------------------------------------- hand example
def test_hand_worked_4x4():
    g = json.load(open(os.path.join(GOLD, "hand_4x4.json")))
    n, P = g["n"], g["P"]
    rp, ci, va = g["row_ptr"], g["col_idx"], g["vals"]
    x = np.array(g["x"], dtype=float)
    y = csr_spmv(n, rp, ci, va, x)
    assert y.tolist() == g["y"]
    pl = OraclePlan(n, rp, ci, va, P)
    assert pl.export(oracle.BOUNDS).tolist() == g["bounds"]
    for p, r in enumerate(g["ranks"]):
        assert pl.export(oracle.L_PTR, p).tolist() == r["l_ptr"]
        assert pl.export(oracle.L_COL, p).tolist() == r["l_col"]
        assert pl.export(oracle.L_VAL, p).tolist() == r["l_val"]
        assert pl.export(oracle.HALO, p).tolist() == r["halo"]
        assert pl.export(oracle.R_PTR, p).tolist() == r["r_ptr"]
        assert pl.export(oracle.R_COL, p).tolist() == r["r_col"]
        assert pl.export(oracle.R_VAL, p).tolist() == r["r_val"]
    assert pl.export(oracle.SEND_IDX).tolist() == g["send_idx"]
    assert pl.export(oracle.HALO_OFF).tolist() == g["halo_off"]
    assert pl.export(oracle.SEG_OFF).tolist() == g["seg_off"]
    pl.pack(-1, x)
    assert pl.export(oracle.SENDBUF).tolist() == g["sendbuf_after_pack"]
    assert pl.spmv(x).tolist() == g["y"]


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("P", [1, 2, 3, 5])
@pytest.mark.parametrize("seed", range(6))
def test_dense_brute_force(P, seed):
    n = [1, 7, 16, 33, 64, 50][seed]
    n, rp, ci, va = W.random_csr(n, density=0.25, seed=seed, duplicates=seed % 2 == 1,
                                 shuffle_cols=seed % 3 == 2)
    x = W.uniform_x(n, seed=100 + seed)
    A = dense(n, rp, ci, va)
    want = A @ x
    scale = np.abs(A) @ np.abs(x)
    got = csr_spmv(n, rp, ci, va, x)
    assert np.all(np.abs(got - want) <= 1e-13 * scale + 1e-300)
    got_p = OraclePlan(n, rp, ci, va, P).spmv(x)
    assert np.all(np.abs(got_p - want) <= 1e-13 * scale + 1e-300)
    ab = csr_absdot(n, rp, ci, va, x)
    absA = dense(n, rp, ci, np.abs(va))
    assert np.allclose(ab, absA @ np.abs(x), rtol=1e-13, atol=0)


def test_scipy_csr_matvec():
    sp = pytest.importorskip("scipy.sparse")
    n, rp, ci, va = W.powerlaw(5000, seed=11, cap=300)
    x = W.uniform_x(n, seed=12)
    A = sp.csr_matrix((va, ci, rp), shape=(n, n))
    want = A @ x
    scale = abs(A) @ np.abs(x)
    got = csr_spmv(n, rp, ci, va, x)
    assert np.all(np.abs(got - want) <= 1e-12 * scale)
    got_p = OraclePlan(n, rp, ci, va, 4).spmv(x)
    assert np.all(np.abs(got_p - want) <= 1e-12 * scale)


def test_rows_parallel_product_equals_serial_bit_for_bit():
    """The timing-only parallel oracle sums every row as the serial one."""
    import oracle
    n, rp, ci, va = W.powerlaw(20000, seed=13, cap=500)
    x = W.uniform_x(n, seed=14)
    a = csr_spmv(n, rp, ci, va, x)
    for threads in (0, 1, 3):
        b = oracle.csr_spmv_rows_parallel(n, rp, ci, va, x, threads)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert oracle.max_threads() >= 1


def test_local_plus_remote_exact_on_integers():
    """A = A_L + A_R (Sec. III-A): with small integers every sum is exact, so
    the partitioned product equals the plain one bit for bit."""
    for seed, P in [(0, 2), (1, 3), (2, 7), (3, 1)]:
        n, rp, ci, va = W.random_csr(120, density=0.1, seed=seed, integer=True,
                                     duplicates=True)
        x = W.uniform_x(n, seed=seed, integer=True)
        y0 = csr_spmv(n, rp, ci, va, x)
        y1 = OraclePlan(n, rp, ci, va, P).spmv(x)
        assert np.array_equal(y0, y1)
        assert np.array_equal(y0, dense(n, rp, ci, va) @ x)


# ---------------------------------------------------------------- plan invariants
def check_plan(n, rp, ci, va, P):
    pl = OraclePlan(n, rp, ci, va, P)
    b = pl.export(oracle.BOUNDS)
    assert b.tolist() == [(p * n) // P for p in range(P + 1)]
    send = pl.export(oracle.SEND_IDX)
    hoff = pl.export(oracle.HALO_OFF)
    seg = pl.export(oracle.SEG_OFF)
    for p in range(P):
        lo, hi = b[p], b[p + 1]
        H = pl.export(oracle.HALO, p)
        assert np.all(np.diff(H) > 0), "H_p sorted and distinct"
        assert np.all((H < lo) | (H >= hi)), "H_p holds remote columns only"
        # destination p's slice of the send buffer is exactly H_p
        assert np.array_equal(send[hoff[p]:hoff[p + 1]], H)
        for q in range(P):
            s = send[seg[p * P + q]:seg[p * P + q + 1]]
            assert np.all((s >= b[q]) & (s < b[q + 1])), "segment owned by q"
            assert np.all(np.diff(s) > 0)
        assert seg[p * P] == hoff[p]
        lp, lc, lv = (pl.export(k, p) for k in (oracle.L_PTR, oracle.L_COL, oracle.L_VAL))
        rpp, rc, rv = (pl.export(k, p) for k in (oracle.R_PTR, oracle.R_COL, oracle.R_VAL))
        assert np.all((lc >= 0) & (lc < hi - lo))
        assert np.all((rc >= 0) & (rc < max(len(H), 1)))
        # every row of A is exactly its local plus its remote entries
        for i in range(hi - lo):
            orig = sorted(zip(ci[rp[lo + i]:rp[lo + i + 1]].tolist(),
                              va[rp[lo + i]:rp[lo + i + 1]].tolist()))
            loc = [(int(c) + lo, float(v)) for c, v in
                   zip(lc[lp[i]:lp[i + 1]], lv[lp[i]:lp[i + 1]])]
            rem = [(int(H[c]), float(v)) for c, v in
                   zip(rc[rpp[i]:rpp[i + 1]], rv[rpp[i]:rpp[i + 1]])]
            assert sorted(loc + rem) == orig
    assert hoff[-1] == len(send) == seg[-1]
    return pl


@pytest.mark.parametrize("case", range(8))
def test_plan_invariants(case):
    n = [0, 1, 5, 40, 64, 100, 3, 17][case]
    P = [1, 3, 2, 4, 5, 7, 8, 16][case]     # includes P > n
    n, rp, ci, va = W.random_csr(n, density=0.3, seed=case, duplicates=True,
                                 shuffle_cols=case % 2 == 0)
    check_plan(n, rp, ci, va, P)


def test_plan_invariants_stencil():
    n, rp, ci, va = W.stencil_27pt(12, seed=1)
    pl = check_plan(n, rp, ci, va, 4)
    # slab partition of a 27-point stencil: the outer ranks need one
    # neighbouring plane-band, the inner ranks two
    sizes = [len(pl.export(oracle.HALO, p)) for p in range(4)]
    assert sizes[0] == sizes[3] and sizes[1] == sizes[2] and sizes[1] > sizes[0]


def test_pack_and_copy_fill_x_of_halo():
    n, rp, ci, va = W.powerlaw(3000, seed=4, cap=200)
    x = W.uniform_x(n, seed=5)
    pl = OraclePlan(n, rp, ci, va, 5)
    pl.pack(-1, x)
    pl.copy(-1)
    rb = pl.export(oracle.RECVBUF)
    hoff = pl.export(oracle.HALO_OFF)
    for p in range(5):
        assert np.array_equal(rb[hoff[p]:hoff[p + 1]], x[pl.export(oracle.HALO, p)])


def test_invalid_csr_rejected():
    with pytest.raises(ValueError):
        OraclePlan(2, [0, 1, 2], [0, 5], [1.0, 1.0], 1)
    with pytest.raises(ValueError):
        OraclePlan(2, [0, 2, 1], [0, 1], [1.0, 1.0], 1)
    with pytest.raises(ValueError):
        OraclePlan(2, [0, 1, 2], [0, 1], [1.0, 1.0], 0)


# ---------------------------------------------------------------- mutation checks
def test_pins_catch_planted_mistakes():
    """Plausible mistakes, planted in copies of the oracle's outputs on the
    CPU, are caught by the pins above."""
    n, rp, ci, va = W.random_csr(40, density=0.3, seed=3)
    x = W.uniform_x(n, seed=4)
    A = dense(n, rp, ci, va)
    y = OraclePlan(n, rp, ci, va, 3).spmv(x)
    scale = np.abs(A) @ np.abs(x)
    ok = lambda v: np.all(np.abs(v - A @ x) <= 1e-13 * scale + 1e-300)
    assert ok(y)
    # a dropped remote term
    pl = OraclePlan(n, rp, ci, va, 3)
    yl = np.zeros(n)
    pl.local(-1, x, yl)
    assert not ok(yl)
    # a transposed operand
    assert not ok(A.T @ x) or np.allclose(A, A.T)
    # a wrong sign on the remote product
    pl.pack(-1, x)
    pl.copy(-1)
    yr = np.zeros(n)
    pl.remote(-1, yr)
    assert not ok(yl - yr)
    # a halo list off by one position
    H = pl.export(oracle.HALO, 1)
    if len(H) > 1:
        assert not np.all(np.diff(np.roll(H, 1)) > 0)


def test_plan_and_product_properties_on_random_matrices():
    """Property check over random small matrices (sizes 0-48, 1-9 ranks so
    P > n occurs, densities up to 0.6, duplicate and unsorted columns): the
    plan keeps every invariant above, the partitioned product equals the
    dense brute force within the dot-product error bound, and on integer
    data the partitioned and plain products are equal bit for bit."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    @settings(max_examples=80, deadline=None, derandomize=True)
    @given(n=st.integers(0, 48), P=st.integers(1, 9), density=st.floats(0.0, 0.6),
           seed=st.integers(0, 2**31 - 1), dup=st.booleans(), shuf=st.booleans())
    def prop(n, P, density, seed, dup, shuf):
        n, rp, ci, va = W.random_csr(n, density=density, seed=seed, duplicates=dup, shuffle_cols=shuf)
        pl = check_plan(n, rp, ci, va, P)
        x = W.uniform_x(n, seed=seed % 1000)
        y = pl.spmv(x)
        want = dense(n, rp, ci, va) @ x
        scale = csr_absdot(n, rp, ci, va, x)
        assert np.all(np.abs(y - want) <= 1e-12 * scale + 1e-300)
        n, rp, ci, va = W.random_csr(n, density=density, seed=seed, integer=True, duplicates=dup,
                                     shuffle_cols=shuf)
        xi = W.uniform_x(n, seed=seed % 1000, integer=True)
        assert np.array_equal(OraclePlan(n, rp, ci, va, P).spmv(xi), csr_spmv(n, rp, ci, va, xi))

    prop()
