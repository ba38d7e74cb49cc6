"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- published test vectors, closed forms, algebraic invariants of
the Householder reflection, exact brute force on tiny inputs, and
distributional properties of the label draws."""
import itertools
import math
import os
from fractions import Fraction

import mpmath
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2605_08048_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# --------------------------------------------------------------------------
# HB-LABEL-v1 label draws (sequential selection sampling)
# --------------------------------------------------------------------------
def _unpack(bits, N):
    b = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")
    return b[:, :N].astype(np.int64), b[:, N:]


@pytest.mark.parametrize("n,N", [(1, 2), (3, 7), (200, 500), (31, 32), (33, 65), (7, 14), (64, 64 + 1)])
def test_labels_exactly_n_ones(n, N):
    L, tail = _unpack(O.labels(7, 0, n, N, 0, 300), N)
    assert (L.sum(axis=1) == n).all()
    assert not tail.any()


def test_labels_uniform_over_subsets():
    n, N, B = 3, 6, 40000
    L, _ = _unpack(O.labels(11, 0, n, N, 0, B), N)
    keys = (L * (1 << np.arange(N))).sum(axis=1)
    subsets = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(N), n))
    counts = np.array([(keys == s).sum() for s in subsets])
    assert counts.sum() == B
    assert stats.chisquare(counts).pvalue > 1e-4


def test_labels_position_and_pair_marginals():
    n, N, B = 20, 50, 20000
    L, _ = _unpack(O.labels(3, 5, n, N, 0, B), N)
    p1 = n / N
    z = (L.mean(axis=0) - p1) / math.sqrt(p1 * (1 - p1) / B)
    assert np.abs(z).max() < 5.0
    p2 = n * (n - 1) / (N * (N - 1))
    for a, b in [(0, 1), (0, N - 1), (17, 18), (N - 2, N - 1)]:
        f = (L[:, a] & L[:, b]).mean()
        assert abs(f - p2) / math.sqrt(p2 * (1 - p2) / B) < 5.0


def test_labels_counter_addressing():
    full = O.labels(99, 2, 40, 130, 0, 20)
    part = O.labels(99, 2, 40, 130, 5, 7)
    assert (full[5:12] == part).all()
    assert not (O.labels(99, 3, 40, 130, 0, 20) == full).all()
    assert not (O.labels(98, 2, 40, 130, 0, 20) == full).all()


def test_labels_forced_tail():
    """Algorithm S: once the remaining positions equal the remaining ones,
    every remaining position is selected; once n ones are placed, none is."""
    n, N = 5, 40
    L, _ = _unpack(O.labels(1, 0, n, N, 0, 2000), N)
    for row in L:
        c = np.cumsum(row)
        for i in range(N):
            before = c[i - 1] if i else 0
            if before == n:
                assert row[i] == 0
            if n - before == N - i:
                assert row[i:].all()
                break


def test_exhaustive_is_colex():
    for n, N in [(1, 4), (2, 5), (3, 7), (7, 14), (5, 12)]:
        got = O.labels_exhaustive(n, N)[:, 0].astype(np.int64)
        want = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(N), n))
        assert got.tolist() == want


# --------------------------------------------------------------------------
# Householder alignment (Sec. 3.1, Eq. householder_fast, App. D)
# --------------------------------------------------------------------------
def _pair(seed=5, n=40, m=55, d=24, dtype="f32", angle=50.0):
    return synth.pair(seed, n, m, d, 0.35, 0.35, angle, dtype)


def _f64(a):
    return synth.bf16_bits_to_f32(a).astype(np.float64) if a.dtype == np.uint16 else a.astype(np.float64)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_reflection_geometry(dtype):
    X, Y = _pair(dtype=dtype)
    st, Z, u, zf, skipped = O.align(X, Y)
    assert st == O.OK and skipped == 0
    x, y = _f64(X), _f64(Y)
    mux = x.mean(0) / np.linalg.norm(x.mean(0))
    muy = y.mean(0) / np.linalg.norm(y.mean(0))
    v = (mux - muy) / np.linalg.norm(mux - muy)
    xr = zf[: len(x)]
    # x' - x is parallel to mu_x - mu_y; (x + x')/2 is orthogonal to it
    diff = xr - x
    par = diff @ v
    assert np.allclose(diff, np.outer(par, v), atol=1e-13)
    assert np.abs(((x + xr) / 2) @ v).max() < 1e-13
    # norms preserved (H orthogonal)
    assert np.allclose(np.linalg.norm(xr, axis=1), np.linalg.norm(x, axis=1), rtol=1e-13)
    # reflected mean direction equals the other cloud's (H mu_x = mu_y)
    mxr = xr.mean(0) / np.linalg.norm(xr.mean(0))
    assert np.abs(mxr - muy).max() < 1e-12
    # Y untouched
    assert (Z[len(x):] == Y).all()
    # axis = unit (mu_x - mu_y)
    assert np.abs(u - v).max() < 1e-12


def test_reflection_maximises_merged_mrl():
    """App. D: after alignment the merged-set MRL reaches its upper bound
    (n ||x_bar|| + m ||y_bar||)/(n + m); the unaligned merged set stays below."""
    X, Y = _pair(angle=70.0)
    st, Z, u, zf, _ = O.align(X, Y)
    x, y = _f64(X), _f64(Y)
    n, m = len(x), len(y)
    bound = (n * np.linalg.norm(x.mean(0)) + m * np.linalg.norm(y.mean(0))) / (n + m)
    assert abs(np.linalg.norm(zf.mean(0)) - bound) < 1e-12
    assert np.linalg.norm(np.vstack([x, y]).mean(0)) < bound - 1e-3


def test_reflect_side_y():
    X, Y = _pair()
    st, Z, u, zf, skipped = O.align(X, Y, reflect_side=1)
    assert st == O.OK and skipped == 0
    x, y = _f64(X), _f64(Y)
    mux = x.mean(0) / np.linalg.norm(x.mean(0))
    yr = zf[len(x):]
    assert np.abs(yr.mean(0) / np.linalg.norm(yr.mean(0)) - mux).max() < 1e-12
    assert (Z[: len(x)] == X).all()


def _nearest_bf16_ok(x: float, got_bits: int) -> bool:
    got = float(synth.bf16_bits_to_f32(np.array([got_bits], dtype=np.uint16))[0])
    fx = Fraction(x)
    a = abs(fx)
    if a == 0:
        return got == 0
    e = math.floor(math.log2(a))
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    q = Fraction(2) ** (max(e, -126) - 7)
    lo = (a // q) * q
    hi = lo + q
    dlo, dhi = a - lo, hi - a
    if dlo < dhi:
        want = lo
    elif dhi < dlo:
        want = hi
    else:
        want = lo if (lo / q) % 2 == 0 else hi
    want = want if fx > 0 else -want
    return Fraction(got) == want


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_storage_rounding_is_nearest_even(dtype):
    X, Y = _pair(dtype=dtype, n=20, m=10, d=32)
    st, Z, u, zf, _ = O.align(X, Y)
    xr = zf[:20].ravel()
    zs = Z[:20].ravel()
    if dtype == "f32":
        assert (xr.astype(np.float32) == zs).all()  # numpy casts with round-to-nearest-even
    else:
        for k in range(0, len(xr), 7):
            assert _nearest_bf16_ok(float(xr[k]), int(zs[k]))


def test_identical_clouds_skip_reflection():
    X, _ = _pair()
    st, Z, u, zf, skipped = O.align(X, X.copy())
    assert st == O.OK and skipped == 1
    assert (Z == np.vstack([X, X])).all() and not u.any()


def test_naive_mode_leaves_data():
    X, Y = _pair(dtype="bf16")
    st, Z, u, zf, skipped = O.align(X, Y, align=0)
    assert st == O.OK and skipped == 1
    assert (Z == np.vstack([X, Y])).all()


def test_degenerate_and_invalid_inputs():
    d = 8
    X = np.zeros((4, d), np.float32)
    X[0, 0], X[1, 0], X[2, 1], X[3, 1] = 1, -1, 1, -1
    _, Y = _pair(d=d, n=4, m=6)
    assert O.align(X, Y)[0] == O.ERR_DEGENERATE
    Xn = Y.copy()
    Xn[2, 3] = np.nan
    assert O.align(Xn, Y)[0] == O.ERR_INVALID_ARG
    r, _, _ = O.perm_test(Y[:1], Y, O.opts(B=9))
    assert r["status"] == O.ERR_DEGENERATE


# --------------------------------------------------------------------------
# Statistic closed forms (Eqs. r, v, tobs)
# --------------------------------------------------------------------------
def _basis(rows, d, start=0):
    A = np.zeros((rows, d), np.float32)
    for i in range(rows):
        A[i, start + i] = 1.0
    return A


def test_closed_forms_orthonormal_rows():
    n, m, d = 4, 9, 16
    X, Y = _basis(n, d), _basis(m, d, start=n)
    r1, _, _ = O.perm_test(X, Y, O.opts(B=5, stat=O.STAT_ONE_MINUS_R2, align=0))
    assert abs(r1["r_x"] - 1 / math.sqrt(n)) < 1e-15 and abs(r1["r_y"] - 1 / math.sqrt(m)) < 1e-15
    assert abs(r1["T_obs"] - ((1 - 1 / n) - (1 - 1 / m))) < 1e-15
    r2, _, _ = O.perm_test(X, Y, O.opts(B=5, stat=O.STAT_MEAN_COSDIST, align=0))
    assert abs(r2["T_obs"]) < 1e-15  # every pair orthogonal: mean cosine distance 1 in both
    r3, _, _ = O.perm_test(X, Y, O.opts(B=5, stat=O.STAT_LOGVOL_VMF, align=0))

    def g(r):
        return r * (d - r * r) / (1 - r * r)

    want = math.log(g(1 / math.sqrt(m))) - math.log(g(1 / math.sqrt(n)))
    assert abs(r3["T_obs"] - want) < 1e-13


def test_n2_m2_by_hand():
    """n = m = 2, d = 3: X = {e0, e1}, Y = {e0, e2}.  Splits of {e0, e1, e0', e2}:
    pairing the two copies of e0 gives r = 1 (all other pairs are orthogonal,
    r = 1/sqrt 2).  Under 1 - r^2 the observed T is 0; with all six splits
    enumerated every |T_b| >= 0, so p = 1; 'greater' counts T_b >= 0: the
    split {e0, e0'} vs {e1, e2} has T = -1/2, its complement +1/2, the other
    four 0 -> 5 of 6."""
    d = 3
    X = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
    Y = np.array([[1, 0, 0], [0, 0, 1]], np.float32)
    r, T, _ = O.perm_test(X, Y, O.opts(stat=O.STAT_ONE_MINUS_R2, align=0, exhaustive=1), want_T=True)
    assert r["B_eff"] == 6 and r["count"] == 6 and r["p"] == 1.0
    assert sorted(T.tolist()) == [-0.5, 0.0, 0.0, 0.0, 0.0, 0.5]
    r, _, _ = O.perm_test(X, Y, O.opts(stat=O.STAT_ONE_MINUS_R2, align=0, exhaustive=1, alt=O.ALT_GREATER))
    assert r["count"] == 5


# --------------------------------------------------------------------------
# Exact brute force on tiny inputs (independent: rational group sums,
# 60-digit logarithms)
# --------------------------------------------------------------------------
def _brute_p(Z, n, d, stat, alt):
    mpmath.mp.dps = 60
    rows = [[Fraction(float(v)) for v in r] for r in _f64(Z)]
    N = len(rows)
    m = N - n

    def val(idx, ng):
        s = [sum(rows[i][j] for i in idx) for j in range(d)]
        q = sum(v * v for v in s)
        if stat == O.STAT_ONE_MINUS_R2:
            return 1 - q / (ng * ng)
        if stat == O.STAT_MEAN_COSDIST:
            return (ng * ng - q) / (ng * (ng - 1))
        rr = mpmath.mpf(q.numerator) / q.denominator / (ng * ng)
        return mpmath.sqrt(rr) * (d - rr) / (1 - rr)

    def T(A1, A2):
        if stat == O.STAT_LOGVOL_VMF:
            return mpmath.log(A2) - mpmath.log(A1)
        return A1 - A2

    To = T(val(range(n), n), val(range(n, N), m))
    cnt = 0
    for c in itertools.combinations(range(N), n):
        rest = [i for i in range(N) if i not in c]
        Tb = T(val(c, n), val(rest, m))
        if alt == O.ALT_GREATER:
            diff = Tb - To
        elif alt == O.ALT_LESS:
            diff = To - Tb
        else:
            diff = abs(Tb) - abs(To)
        if isinstance(diff, Fraction):
            cnt += 1 if diff >= 0 else 0
        else:
            cnt += 1 if (diff >= 0 or abs(diff) < mpmath.mpf("1e-45")) else 0
    return cnt, math.comb(N, n)


@pytest.mark.parametrize("stat", [O.STAT_LOGVOL_VMF, O.STAT_ONE_MINUS_R2, O.STAT_MEAN_COSDIST])
@pytest.mark.parametrize("alt", [O.ALT_TWO_SIDED, O.ALT_GREATER, O.ALT_LESS])
@pytest.mark.parametrize("n,m,align,dtype", [(4, 6, 1, "f32"), (5, 5, 1, "bf16"), (3, 7, 0, "f32")])
def test_exhaustive_matches_exact_brute_force(stat, alt, n, m, align, dtype):
    X, Y = synth.pair(100 + n + 10 * m, n, m, 8, 0.5, 0.5, 60.0, dtype)
    r, _, _ = O.perm_test(X, Y, O.opts(stat=stat, alt=alt, align=align, exhaustive=1))
    assert r["status"] == O.OK
    _, Z, _, _, _ = O.align(X, Y, align=align)
    cnt, C = _brute_p(Z, n, 8, stat, alt)
    assert r["B_eff"] == C
    assert r["count"] == cnt
    assert r["p"] == cnt / C


def test_complement_split_is_an_exact_tie():
    """n = m: the complement of the observed split gives T = -T_obs exactly,
    and the two-sided rule counts it (ties count, Eq. pvalue uses >=)."""
    X, Y = synth.pair(8, 5, 5, 8, 0.4, 0.5, 40.0, "f32")
    labs = O.labels_exhaustive(5, 10)[:, 0]
    comp = int(np.nonzero(labs == 0b1111100000)[0][0])
    ident = int(np.nonzero(labs == 0b0000011111)[0][0])
    r, T, dec = O.perm_test(X, Y, O.opts(exhaustive=1), want_T=True)
    assert T[ident] == r["T_obs"] and T[comp] == -r["T_obs"]
    assert dec[ident] == 1 and dec[comp] == 1


# --------------------------------------------------------------------------
# Monte Carlo p against the exact permutation p; swap invariance; Alg. 1 = Alg. 2
# --------------------------------------------------------------------------
def test_monte_carlo_p_within_binomial_band():
    X, Y = synth.pair(21, 7, 7, 16, 0.35, 0.45, 30.0, "f32")
    ex, _, _ = O.perm_test(X, Y, O.opts(exhaustive=1))
    pe = ex["p"]
    B = 20000
    mc, _, _ = O.perm_test(X, Y, O.opts(B=B, seed=4))
    sd = math.sqrt(B * pe * (1 - pe))
    assert abs(mc["count"] - B * pe) <= 4.5 * sd + 1
    assert mc["p"] == (1 + mc["count"]) / (B + 1)


@pytest.mark.parametrize("stat", [O.STAT_LOGVOL_VMF, O.STAT_ONE_MINUS_R2])
def test_swap_invariance_of_two_sided_p(stat):
    X, Y = synth.pair(31, 5, 8, 8, 0.35, 0.45, 30.0, "f32")
    a, _, _ = O.perm_test(X, Y, O.opts(stat=stat, align=0, exhaustive=1))
    b, _, _ = O.perm_test(Y, X, O.opts(stat=stat, align=0, exhaustive=1))
    assert a["count"] == b["count"] and a["p"] == b["p"]
    c, _, _ = O.perm_test(X, Y, O.opts(stat=stat, align=1, exhaustive=1))
    e, _, _ = O.perm_test(Y, X, O.opts(stat=stat, align=1, exhaustive=1))
    assert abs(c["count"] - e["count"]) <= 2


def test_sign_matrix_formulation_agrees():
    """Algorithm 2 (U = S Z with +-1 signs, sigma = (t +- U)/2) gives the same
    T_b as the oracle's direct group sums (Algorithm 1)."""
    X, Y = synth.pair(41, 30, 45, 32, 0.35, 0.35, 80.0, "bf16")
    o = O.opts(B=200, seed=9)
    r, T, _ = O.perm_test(X, Y, o, want_T=True)
    _, Z, _, _, _ = O.align(X, Y)
    z = _f64(Z)
    n, m, N, d = 30, 45, 75, 32
    L, _ = _unpack(O.labels(9, 0, n, N, 0, 200), N)
    S = 2.0 * L - 1.0
    t = z.sum(0)
    U = S @ z
    s1, s2 = (t + U) / 2, (t - U) / 2
    r1 = np.linalg.norm(s1, axis=1) / n
    r2 = np.linalg.norm(s2, axis=1) / m

    def g(r):
        return r * (d - r * r) / (1 - r * r)

    T2 = np.log(g(r2)) - np.log(g(r1))
    assert np.allclose(T2, T, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("stat", [O.STAT_LOGVOL_VMF, O.STAT_ONE_MINUS_R2, O.STAT_MEAN_COSDIST])
def test_stats_for_sampled_b_match_full_run(stat):
    X, Y = synth.pair(51, 25, 35, 16, 0.35, 0.35, 45.0, "f32")
    o = O.opts(B=300, seed=3, stat=stat)
    r, T, dec = O.perm_test(X, Y, o, want_T=True)
    bl = [0, 5, 77, 299]
    r2, T2, dec2, q = O.perm_stats(X, Y, o, bl)
    assert (T2 == T[bl]).all() and (dec2 == dec[bl]).all()
    assert int(dec.sum()) == r["count"]


def test_null_p_values_are_uniform():
    """Equal dispersion and equal mean direction: p ~ U(0, 1)."""
    ps = []
    for k in range(200):
        X, Y = synth.pair(1000 + k, 14, 18, 8, 0.5, 0.5, 0.0, "f32")
        r, _, _ = O.perm_test(X, Y, O.opts(B=199, seed=k))
        ps.append(r["p"])
    assert stats.kstest(ps, "uniform").pvalue > 1e-3


def test_batched_equals_single():
    b = synth.batch(77, 5, d=16, dtype="bf16", sizes=([6, 9, 12, 5, 20], [7, 4, 15, 30, 8]))
    o = O.opts(B=120, seed=2)
    res = O.perm_test_batched(b.XY, b.n, b.m, o)
    for p in range(5):
        X, Y = b.pair(p)
        r, _, _ = O.perm_test(X, Y, o)
        assert r == res[p]
