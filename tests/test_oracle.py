"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these checks re-types the oracle's own formulas: they compare it with
hand-derived closed forms (tests/golden), library rounding (numpy float16 /
float32 casts), exact rational arithmetic (fractions), the paper's error
theorems, and special cases with a textbook answer.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads
from golden_cases import load_cases

CASES = load_cases()


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_closed_forms(orc, case):
    r = orc.qdot(case.x, case.y, eps=case.eps, block=case.block, split_budget=case.split,
                 mant_reading=case.mant, explain=True)
    assert r.status == 0
    np.testing.assert_array_equal(r.cls, case.classes)
    assert r.value == case.z


def test_quantizer_matches_library_casts(orc):
    rng = np.random.default_rng(1)
    # half normal range [2^-14, 65504) and single normal range, random signs
    vh = np.exp2(rng.uniform(-14, 15.9, 20000)) * rng.choice([-1.0, 1.0], 20000)
    vs = np.exp2(rng.uniform(-120, 120, 20000)) * rng.choice([-1.0, 1.0], 20000)
    # exact ties of the half / single grids (the round-to-even cases)
    ties_h = (1 + (2 * rng.integers(0, 1024, 2000) + 1) * 2.0**-11) * np.exp2(rng.integers(-10, 10, 2000))
    ties_s = (1 + (2 * rng.integers(0, 2**23, 2000) + 1) * 2.0**-24) * np.exp2(rng.integers(-50, 50, 2000))
    for v in np.concatenate([vh, ties_h]):
        assert orc.quantize(v, orc.HALF) == float(np.float16(v))
    for v in np.concatenate([vs, ties_s]):
        assert orc.quantize(v, orc.SINGLE) == float(np.float32(v))
    for v in vs[:100]:
        assert orc.quantize(v, orc.DOUBLE) == v
        assert orc.quantize(v, orc.PERF) == 0.0


def test_quantizer_hand_ties(orc):
    assert orc.quantize(1 + 2.0**-11, orc.HALF) == 1.0           # tie, even below
    assert orc.quantize(1 + 3 * 2.0**-11, orc.HALF) == 1 + 2.0**-9  # tie, even above
    assert orc.quantize(2 - 2.0**-12, orc.HALF) == 2.0           # carry into the exponent
    assert orc.quantize(1 + 2.0**-24, orc.SINGLE) == 1.0
    assert orc.quantize(-(1 + 3 * 2.0**-24), orc.SINGLE) == -(1 + 2.0**-22)


def test_quantizer_unbounded_exponent(orc):
    # far outside the half / single exponent ranges: only the significand rounds
    for e in (-1000, -300, 200, 1000):
        v = (1 + 2.0**-11 + 2.0**-30) * 2.0**e
        assert orc.quantize(v, orc.HALF) == (1 + 2.0**-10) * 2.0**e
        w = (1 + 2.0**-24 + 2.0**-40) * 2.0**e
        assert orc.quantize(w, orc.SINGLE) == (1 + 2.0**-23) * 2.0**e
    # subnormal: (2^11 + 1) * 2^-1074 has 12 significant bits -> tie -> even (2^11)
    assert orc.quantize((2**11 + 1) * 2.0**-1074, orc.HALF) == 2**11 * 2.0**-1074
    assert orc.quantize(3 * 2.0**-1074, orc.HALF) == 3 * 2.0**-1074


def _frac_sum(qx, qy, cls):
    return sum((Fraction(a) * Fraction(b) for a, b, c in zip(qx, qy, cls) if c in (1, 2, 3)), Fraction(0))


@pytest.mark.parametrize("block", [0, 1, 2, 3, 7, 32, 64])
@pytest.mark.parametrize("kind", ["a", "b", "c", "cfg0"])
def test_exact_sum_bruteforce(orc, block, kind):
    """For n <= 64 the oracle's z equals the exact rational sum of its own
    quantized products, rounded once (Fraction arithmetic, independent)."""
    for seed in range(3):
        x, y = workloads.pair(kind, 61, 100 + seed)
        for eps in (1e-16, 1e-8, 1e-3, 0.5):
            r = orc.qdot(x, y, eps=eps, block=block, explain=True)
            exact = _frac_sum(r.qx, r.qy, r.cls)
            assert r.value == float(exact)
            # class partial sums
            for c in (1, 2, 3):
                sc = sum((Fraction(a) * Fraction(b) for a, b, k in zip(r.qx, r.qy, r.cls) if k == c),
                         Fraction(0))
                assert r.class_sum[c] == float(sc)
            dropped = sum((Fraction(a) * Fraction(b) for a, b, k in zip(x, y, r.cls) if k == 0), Fraction(0))
            assert r.class_sum[0] == float(dropped)
            assert sum(r.count) == 61


@pytest.mark.parametrize("kind", ["a", "b", "c"])
def test_quantized_values_match_casts(orc, kind):
    """Per-component q values of the explain output equal numpy's casts of the
    component to half / single (scaled into the cast's normal range first)."""
    x, y = workloads.pair(kind, 4000, 7)
    r = orc.qdot(x, y, eps=1e-1, block=1, explain=True)
    for v, q, c in zip(np.concatenate([x, y]), np.concatenate([r.qx, r.qy]), np.concatenate([r.cls, r.cls])):
        if c in (0, 4):
            assert q == 0.0
            continue
        m, e = math.frexp(v)  # v = m 2^e, scale to [0.5, 1)
        if c == 1:
            ref = math.ldexp(float(np.float16(m)), e)
        elif c == 2:
            ref = math.ldexp(float(np.float32(m)), e)
        else:
            ref = v
        assert q == ref


def test_reduces_to_exact_dot(orc):
    """With a tolerance so small that every score exceeds m_single, every bin is
    double and z is the correctly rounded exact x.y (Fraction reference)."""
    for kind in ("a", "b", "c", "cfg0"):
        x, y = workloads.pair(kind, 300, 3)
        exact = sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0))
        for block in (0, 1, 32):
            r = orc.qdot(x, y, eps=1e-300, block=block)
            assert r.count[3] == 300
            assert r.value == float(exact)
        assert orc.dot_exact(x, y) == float(exact)


def test_theorem5_early_termination(orc):
    """Thm 5: e_max - e_min <= -floor(log2 eps) - m_single => every bin double."""
    rng = np.random.default_rng(5)
    hits = 0
    for t in range(200):
        n = int(rng.integers(1, 300))
        x = rng.uniform(0.5, 1.0, n) * np.exp2(rng.integers(0, 6, n))
        y = rng.uniform(0.5, 1.0, n) * np.exp2(rng.integers(0, 6, n))
        eps = float(np.exp2(rng.uniform(-60, -20)))
        for block in (0, 1, 16):
            r = orc.qdot(x, y, eps=eps, block=block)
            if r.e_max - r.e_min <= -r.f - 23:
                hits += 1
                assert r.count[3] == n
    assert hits > 50


def _exact_error(x, y, r):
    approx = _frac_sum(r.qx, r.qy, r.cls)
    exact = sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0))
    return abs(approx - exact), exact


@pytest.mark.parametrize("mant", [0, 1])
@pytest.mark.parametrize("split", [1, 0])
def test_error_bound_chain(orc, split, mant):
    """Thm 1 (per component), Thm 4 (per bin) and the eps budget: the exact error
    of the quantized sum is bounded by the element-wise bound, which is bounded
    by the bin-wise bound, which is bounded by N_bins 2^(e_max + f); with the
    eps / N_bins split that is at most eps 2^e_max."""
    rng = np.random.default_rng(11 + split + 2 * mant)
    for trial in range(40):
        kind = ["a", "b", "c", "cfg0"][trial % 4]
        n = int(rng.integers(1, 500))
        x, y = workloads.pair(kind, n, 1000 + trial)
        for block in (0, 1, 5, 32):
            for eps in (1e-12, 1e-6, 1e-2, 10.0):
                r = orc.qdot(x, y, eps=eps, block=block, split_budget=split, mant_reading=mant, explain=True)
                err, exact = _exact_error(x, y, r)
                assert err <= Fraction(r.bound_elem)
                assert Fraction(r.bound_elem) <= Fraction(r.bound_bins)
                assert Fraction(r.bound_bins) <= Fraction(r.bound_apriori)
                if split:
                    assert Fraction(r.bound_apriori) <= Fraction(eps) * Fraction(2) ** r.e_max
                else:
                    assert Fraction(r.bound_apriori) <= r.n_bins * Fraction(eps) * Fraction(2) ** r.e_max


def test_relative_bound_for_norms(orc):
    """Thm 4 hypothesis holds for x.x (Sec. 3.1): relative error <= eps."""
    for kind in ("a", "b", "c", "cfg0"):
        for seed in range(4):
            x, _ = workloads.pair(kind, 700, 50 + seed)
            for block in (0, 1, 32):
                for eps in (1e-10, 1e-5, 1e-2, 0.3):
                    r = orc.qdot(x, x, eps=eps, block=block, explain=True)
                    err, exact = _exact_error(x, x, r)
                    assert err <= Fraction(eps) * exact


def test_floor_log2_ratio_definition(orc):
    """f is the largest integer k with N 2^k <= eps (checked with Fractions)."""
    rng = np.random.default_rng(3)
    vals = [1e-16, 1e-15, 1e-8, 0.1, 1.0, 2.0, 3.0, 1e3, 2.0**-1074, 5e-324 * 7, 1.7e308]
    vals += list(np.exp2(rng.uniform(-60, 10, 50))) + [float(2.0**k) for k in range(-40, 40, 7)]
    for eps in vals:
        for N in (1, 2, 3, 7, 1000, 2**20, 2**28 + 5, 3 * 2**40):
            k = orc.floor_log2_ratio(eps, N)
            E = Fraction(eps)
            assert N * Fraction(2) ** k <= E
            assert N * Fraction(2) ** (k + 1) > E


def test_monotone_in_eps(orc):
    """Raising eps never raises a component's precision (the score decreases
    with floor(log2 eps_eff) and the precision function is monotone)."""
    for kind in ("a", "b", "c"):
        x, y = workloads.pair(kind, 2000, 9)
        for block in (0, 1, 32):
            prev = None
            for eps in (1e-16, 1e-12, 1e-8, 1e-4, 1e-1, 10.0, 1e4):
                cls = orc.qdot(x, y, eps=eps, block=block, explain=True).cls.astype(int)
                if prev is not None:
                    nz = prev != 4
                    assert np.all(cls[nz] <= prev[nz])
                prev = cls


def test_block_mode_special_cases(orc):
    """Blocks of 1 with pairwise-distinct keys coincide with exact binning, and
    one block covering a vector with a single key coincides with exact binning."""
    n = 200
    x = np.exp2(np.arange(n, dtype=np.float64) - 100) * 1.37
    y = np.full(n, -1.11)
    for eps in (1e-12, 1e-4, 1.0):
        a = orc.qdot(x, y, eps=eps, block=0, explain=True)
        b = orc.qdot(x, y, eps=eps, block=1, explain=True)
        np.testing.assert_array_equal(a.cls, b.cls)
        assert a.value == b.value
    x = np.random.default_rng(2).uniform(1.0, 2.0, 333)
    y = np.random.default_rng(3).uniform(-2.0, -1.0, 333)
    for eps in (1e-12, 1e-4, 1.0, 100.0):
        a = orc.qdot(x, y, eps=eps, block=0, explain=True)
        b = orc.qdot(x, y, eps=eps, block=333, explain=True)
        c = orc.qdot(x, y, eps=eps, block=100000, explain=True)
        np.testing.assert_array_equal(a.cls, b.cls)
        np.testing.assert_array_equal(a.cls, c.cls)
        assert a.value == b.value == c.value


def test_statistics(orc):
    x = np.array([2.0**-1074, 1.5, -3.0, 0.0, 1e300])
    y = np.array([1.0, 4.0, 0.25, 7.0, 1e-300])
    r = orc.qdot(x, y, eps=1e-16, block=0)
    keys = [-1074 + 0, 0 + 2, 1 - 2, 996 - 997]
    assert r.e_max == max(keys) and r.e_min == min(keys)
    assert r.n_bins == len(set(keys))
    assert r.count[4] == 1
    r = orc.qdot(x, y, eps=1e-16, block=2)
    assert r.n_bins == 3  # blocks {0,1}, {2,3}, {4}


def test_edge_cases(orc):
    r = orc.qdot(np.zeros(0), np.zeros(0), eps=1e-8)
    assert r.status == 0 and r.value == 0.0 and r.n_bins == 0 and sum(r.count) == 0
    r = orc.qdot(np.zeros(10), np.ones(10), eps=1e-8, block=3)
    assert r.value == 0.0 and r.count[4] == 10 and r.n_bins == 0
    r = orc.qdot(np.array([1.0, np.nan]), np.ones(2), eps=1e-8)
    assert r.status == 2
    r = orc.qdot(np.array([1.0, np.inf]), np.ones(2), eps=1e-8)
    assert r.status == 2
    r = orc.qdot(np.ones(2), np.ones(2), eps=0.0)
    assert r.status == 1
    r = orc.qdot(np.ones(2), np.ones(2), eps=-1.0)
    assert r.status == 1
    # single element, every class reachable
    for eps, cls in ((2.0**-22, 3), (2.0**-21, 2), (2.0**-9, 2), (2.0**-8, 1), (2.0, 1), (4.0, 0)):
        r = orc.qdot(np.array([3.0]), np.array([5.0]), eps=eps, block=1, explain=True)
        # key = 1 + 2 = 3 = e_max, M = 1, N_bins = 1: sigma = 1 - floor(log2 eps)
        assert int(r.cls[0]) == cls


def test_cg_oracle_solves_system(orc):
    rp, col, val = workloads.poisson3d(8, 7, 6)
    n = rp.shape[0] - 1
    b = workloads.rhs(n)
    import scipy.sparse as sp
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    x, it, rr, counts, st = orc.cg(rp, col, val, b, rel_tol=1e-10, max_it=5000, eps=1e-300)
    assert st == 0 and rr <= 1e-10
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-8
    # a textbook CG with numpy dots: on this ill-conditioned operator (cond ~ 3e5)
    # finite-precision CG needs many more steps than n, and the count depends
    # on rounding details, so only closeness is required
    xr = np.zeros(n); r = b.copy(); p = r.copy(); c = r @ r; k = 0
    while math.sqrt(c) / np.linalg.norm(b) > 1e-10:
        q = A @ p; a = c / (p @ q); xr += a * p; r -= a * q; cn = r @ r; p = r + (cn / c) * p; c = cn; k += 1
    assert abs(k - it) <= 0.02 * k
    # loose qdot tolerance still converges on this small well-posed system
    _, it2, rr2, counts2, _ = orc.cg(rp, col, val, b, rel_tol=1e-10, max_it=5000, eps=1e-3)
    assert rr2 <= 1e-10
    assert counts2[0] + counts2[1] + counts2[2] > 0  # some components were lowered


def test_spmv_oracle(orc):
    rp, col, val = workloads.poisson2d(9, 11)
    import scipy.sparse as sp
    n = rp.shape[0] - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    x = workloads.rhs(n, 3)
    np.testing.assert_allclose(orc.spmv(rp, col, val, x), A @ x, rtol=1e-13, atol=1e-12)


def test_power_oracle_dominant_eigenvalue(orc):
    rp, col, val = workloads.poisson2d(10, 9)
    import scipy.sparse as sp
    n = rp.shape[0] - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()
    lam_max = np.linalg.eigvalsh(A)[-1]
    lam, x, it, counts, st = orc.power(rp, col, val, workloads.unit_start(n), iters=3000, eps=1e-300)
    assert st == 0
    assert abs(lam - lam_max) <= 1e-6 * lam_max
    np.testing.assert_allclose(np.linalg.norm(x), 1.0, rtol=1e-12)


def test_backward_oracle(orc):
    x, y = workloads.pair("b", 3000, 21)
    r = orc.qdot(x, y, eps=1e-3, block=32, explain=True)
    g = -1.75
    gx, gy = orc.backward(x, y, r.cls, g)
    keep = (r.cls == 1) | (r.cls == 2) | (r.cls == 3)
    assert np.all(gx[~keep] == 0) and np.all(gy[~keep] == 0)
    # half / single components: gradient = g * library cast of the scaled significand
    for i in np.nonzero(keep)[0][:500]:
        m, e = math.frexp(y[i])
        ref = {1: lambda v: float(np.float16(v)), 2: lambda v: float(np.float32(v)), 3: lambda v: v}[int(r.cls[i])](m)
        assert gx[i] == g * math.ldexp(ref, e)
    # central finite differences of the class-frozen surrogate g * sum_keep x_i q(y_i)
    qy = r.qy
    h = 1e-7
    for i in np.nonzero(keep)[0][:50]:
        xp = x.copy(); xp[i] += h
        xm = x.copy(); xm[i] -= h
        fp = Fraction(g) * sum(Fraction(a) * Fraction(b) for a, b, k in zip(xp, qy, keep) if k)
        fm = Fraction(g) * sum(Fraction(a) * Fraction(b) for a, b, k in zip(xm, qy, keep) if k)
        fd = float((fp - fm) / (Fraction(xp[i]) - Fraction(xm[i])))
        assert fd == pytest.approx(gx[i], rel=1e-12, abs=0)


def _adversarial_pairs():
    """Small vectors with mixed signs, subnormals, huge and tiny magnitudes and
    exact cancellation: the cases a sloppy exact accumulator gets wrong."""
    rng = np.random.default_rng(77)
    cases = []
    tiny = [5e-324, 3 * 2.0**-1074, 2.0**-1022, 1e-310, -7e-320]
    huge = [1e150, -1e148, 2.0**490, -2.0**480, 3.0 * 2.0**450]  # products and sums stay finite
    for t in range(12):
        n = int(rng.integers(1, 65))
        x = rng.choice(tiny + huge + [1.0, -1.0, 0.0, 1e-300, 2.0**-60], n) * rng.uniform(0.5, 2.0, n)
        y = rng.choice(tiny + huge + [1.0, -3.0, 0.0, 1e-8], n) * rng.uniform(0.5, 2.0, n)
        cases.append((x, y))
    # exact cancellation: x.y = a - a + small
    a = 2.0**500
    cases.append((np.array([a, 1.0, -a, 2.0**-700]), np.array([a, 3.0, a, 1.0])))
    # random signs over a wide exponent range
    for t in range(6):
        n = int(rng.integers(1, 65))
        x = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-1000, 500, n))
        y = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-1000, 500, n))
        cases.append((x, y))
    return cases


def test_abs_dot_and_sum_exact_pinned(orc):
    """orc.abs_dot_exact (the scale of every GPU parity tolerance) and
    orc.sum_exact equal the correctly rounded exact rational results
    (Fraction sums of the same doubles), on adversarial inputs."""
    for x, y in _adversarial_pairs():
        ax = sum((abs(Fraction(a) * Fraction(b)) for a, b in zip(x, y)), Fraction(0))
        assert orc.abs_dot_exact(x, y) == float(ax)
        sx = sum((Fraction(v) for v in x), Fraction(0))
        assert orc.sum_exact(x) == float(sx)
        d = sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0))
        assert orc.dot_exact(x, y) == float(d)
    # a sum whose exact value is a tie between two doubles rounds to even
    v = np.array([1.0, 2.0**-53])
    assert orc.sum_exact(v) == 1.0
    v = np.array([1.0 + 2.0**-52, 2.0**-53])
    assert orc.sum_exact(v) == 1.0 + 2.0**-51


def test_value_ld_within_long_double_rounding(orc):
    """value_ld (the long-double accumulation of the quantized products) is
    within the rounding of a long-double sum of n products of the exact sum:
    |value_ld - z_exact| <= (n + 2) eps_ld sum|q(x) q(y)| + 2^-53 |z_exact|,
    eps_ld the long-double machine epsilon of this host (64-bit significand
    on x86-64, 113-bit on AArch64)."""
    eps_ld = Fraction(float(np.finfo(np.longdouble).eps))
    for kind in ("a", "b", "c", "cfg0"):
        for seed in range(3):
            x, y = workloads.pair(kind, 300, 500 + seed)
            for block in (0, 1, 32):
                for eps in (1e-16, 1e-6, 1e-2):
                    r = orc.qdot(x, y, eps=eps, block=block, explain=True)
                    exact = _frac_sum(r.qx, r.qy, r.cls)
                    sabs = sum((abs(Fraction(a) * Fraction(b)) for a, b, c in zip(r.qx, r.qy, r.cls)
                                if c in (1, 2, 3)), Fraction(0))
                    tol = (len(x) + 2) * eps_ld * sabs + Fraction(2) ** -53 * abs(exact)
                    assert abs(Fraction(r.value_ld) - exact) <= tol


@pytest.mark.parametrize("unit", [1, 7, 32, 256])
@pytest.mark.parametrize("block", [0, 1, 32])
def test_unit_sums_bruteforce(orc, unit, block):
    """Algorithm 1's partial sums over index ranges: each range's sum of
    q(x_i) q(y_i) and of |x_i y_i| equals the correctly rounded Fraction sum
    over the same range (classes and q values from the pinned explain
    output); together they add up to z."""
    for kind in ("a", "b", "c"):
        x, y = workloads.pair(kind, 300, 70 + unit + block)
        x[::17] = 0.0
        for eps in (1e-16, 1e-6, 0.5):
            r = orc.qdot(x, y, eps=eps, block=block, explain=True)
            sums, abss = orc.unit_sums(x, y, unit, eps=eps, block=block)
            assert len(sums) == (len(x) + unit - 1) // unit
            for k in range(len(sums)):
                sl = slice(k * unit, (k + 1) * unit)
                q = _frac_sum(r.qx[sl], r.qy[sl], r.cls[sl])
                a = sum((abs(Fraction(p) * Fraction(t)) for p, t in zip(x[sl], y[sl])), Fraction(0))
                assert sums[k] == float(q)
                assert abss[k] == float(a)
            tot = sum((Fraction(v) for v in sums), Fraction(0))
            assert abs(tot - _frac_sum(r.qx, r.qy, r.cls)) <= len(sums) * Fraction(2) ** -53 * sum(
                (abs(Fraction(v)) for v in sums), Fraction(0))


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_oracle_equals_serial(orc, threads):
    """The CPU-baseline helper that spreads the oracle over host threads gives
    exactly the serial oracle's value, counts and statistics (exact sums are
    order independent), zeros, subnormals and non-finite values included."""
    rng = np.random.default_rng(threads)
    for kind in ("a", "b", "c", "cfg0"):
        x, y = workloads.pair(kind, 20011, 40 + threads)
        x[rng.random(x.shape[0]) < 0.01] = 0.0
        y[::997] = 5e-324
        for block in (0, 1, 7, 32, 256):
            for eps in (1e-16, 1e-8, 1e-2):
                a = orc.qdot(x, y, eps=eps, block=block)
                b = orc.qdot_threads(x, y, eps=eps, block=block, threads=threads)
                assert b.status == 0
                assert np.float64(a.value).tobytes() == np.float64(b.value).tobytes()
                assert a.count == b.count
                assert (a.e_max, a.e_min, a.n_bins, a.f) == (b.e_max, b.e_min, b.n_bins, b.f)
    x = np.ones(100)
    x[50] = np.nan
    assert orc.qdot_threads(x, np.ones(100), eps=1e-8, threads=threads).status == 2


def test_cpu_fp64_dot_within_rounding(orc):
    """The host FP64 dot (one fused multiply-add chain per thread, partials
    added in order) is within the rounding bound of such a sum of the exact
    dot: |dot - x.y| <= (n / t + t + 1) 2^-53 sum |x_i y_i|."""
    for kind in ("a", "b", "c"):
        x, y = workloads.pair(kind, 100003, 9)
        ex = Fraction(orc.dot_exact(x, y))
        sabs = Fraction(orc.abs_dot_exact(x, y))
        for t in (1, 4, 8):
            d = orc.dot_fp64(x, y, t)
            assert abs(Fraction(d) - ex) <= Fraction(x.shape[0] // t + t + 2, 2**53) * sabs
