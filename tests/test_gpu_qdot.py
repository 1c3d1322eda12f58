"""GPU parity of qdot (C ABI through the Python binding) against the CPU oracle.

Bar: class map, quantized values, class counts, e_max,
e_min, N_bins and f bit-exact; z within 1e-13 * sum_i |x_i y_i| (the exact
sum of absolute products, from the oracle).
"""
import numpy as np
import pytest

import workloads
from golden_cases import load_cases

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_00115_gb300 import build as qbuild
    qbuild.build()
    import paper_2105_00115_gb300 as qq
    qq.load()
    return qq


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.int64), np.asarray(b).view(np.int64))


def _check(q, orc, x, y, eps, block, split=1, mant=0, explain=True, path="auto"):
    ref = orc.qdot(x, y, eps=eps, block=block, split_budget=split, mant_reading=mant, explain=explain)
    xd, yd = _dev(x), _dev(y)
    tol = TOL * orc.abs_dot_exact(x, y)
    if explain:
        r, cls, qx, qy = q.explain(xd, yd, eps=eps, block=block, split_budget=split, mant_reading=mant)
        np.testing.assert_array_equal(cls.cpu().numpy(), ref.cls)
        assert _same_bits(qx.cpu().numpy(), ref.qx)
        assert _same_bits(qy.cpu().numpy(), ref.qy)
    else:
        r = q.qdot(xd, yd, eps=eps, block=block, split_budget=split, mant_reading=mant, path=path)
    assert r.status == 0
    assert r.count == tuple(ref.count)
    assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
    assert abs(r.value - ref.value) <= tol, (r.value, ref.value, tol)
    assert r.bound == ref.bound_apriori
    return r, ref


CASES = load_cases()


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_closed_forms_gpu(q, orc, case):
    if case.block & (case.block - 1):
        pytest.skip("the GPU path takes block sizes that are powers of two")
    xd, yd = _dev(case.x), _dev(case.y)
    r, cls, qx, qy = q.explain(xd, yd, eps=case.eps, block=case.block, split_budget=case.split,
                               mant_reading=case.mant)
    np.testing.assert_array_equal(cls.cpu().numpy(), case.classes)
    assert r.value == case.z
    r2 = q.qdot(xd, yd, eps=case.eps, block=case.block, split_budget=case.split, mant_reading=case.mant)
    assert r2.value == case.z


@pytest.mark.parametrize("block", [0, 1, 2, 4, 16, 32, 64, 128, 256, 1024])
@pytest.mark.parametrize("kind", ["a", "b", "c", "cfg0"])
def test_parity_grid(q, orc, kind, block):
    # auto takes the fused launch for blocks of 32..256 (and the two-pass one
    # for blocks of 1) at these sizes; the one-pass path is checked explicitly
    paths = ("auto", "one_pass") if (32 <= block <= 256 or block == 1) else ("auto",)
    for n in (1, 63, 64, 65, 1000, 4097, 100003):
        x, y = workloads.pair(kind, n, 17 + n)
        for eps in (1e-16, 1e-8, 1e-3, 0.5):
            _check(q, orc, x, y, eps, block)
            for path in paths:
                _check(q, orc, x, y, eps, block, explain=False, path=path)


@pytest.mark.parametrize("block", [0, 1, 32, 256])
def test_split_and_mant_readings(q, orc, block):
    x, y = workloads.pair("b", 50000, 3)
    for split in (0, 1):
        for mant in (0, 1):
            for eps in (1e-12, 1e-6, 1e-2):
                _check(q, orc, x, y, eps, block, split=split, mant=mant)
                if block > 0:
                    _check(q, orc, x, y, eps, block, split=split, mant=mant, explain=False, path="one_pass")


@pytest.mark.parametrize("block", [0, 1, 8, 32, 64, 512])
def test_misaligned_inputs_use_scalar_loads(q, orc, block):
    import torch
    x, y = workloads.pair("b", 30001, 8)
    xd, yd = _dev(x), _dev(y)
    # 8-byte aligned views: forces the 64-bit load variant
    xs, ys = xd[1:], yd[1:]
    assert xs.data_ptr() % 16 == 8
    ref = orc.qdot(x[1:], y[1:], eps=1e-6, block=block, explain=True)
    r, cls, qx, qy = q.explain(xs, ys, eps=1e-6, block=block)
    np.testing.assert_array_equal(cls.cpu().numpy(), ref.cls)
    assert _same_bits(qx.cpu().numpy(), ref.qx)
    assert r.count == tuple(ref.count)
    assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x[1:], y[1:])
    r2 = q.qdot(xs, ys, eps=1e-6, block=block)
    assert r2.count == tuple(ref.count)
    del torch


def test_edge_cases(q, orc):
    import torch
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    for block in (0, 1, 32, 256):
        r = q.qdot(e, e, eps=1e-8, block=block)
        assert r.value == 0.0 and r.n_bins == 0 and sum(r.count) == 0
        z = torch.zeros(1000, dtype=torch.float64, device="cuda")
        o = torch.ones(1000, dtype=torch.float64, device="cuda")
        r = q.qdot(z, o, eps=1e-8, block=block)
        assert r.value == 0.0 and r.count[4] == 1000 and r.n_bins == 0
    # a single component, every class reachable (key 3 = e_max, M = 1)
    for eps, cls in ((2.0**-22, 3), (2.0**-21, 2), (2.0**-8, 1), (4.0, 0)):
        r, c, _, _ = q.explain(_dev(np.array([3.0])), _dev(np.array([5.0])), eps=eps, block=1)
        assert int(c.cpu()[0]) == cls
    # non-finite components are reported, not summed
    for bad in (np.nan, np.inf, -np.inf):
        x = np.ones(5000)
        x[4321] = bad
        with pytest.raises(q.QdotError):
            q.qdot(_dev(x), _dev(np.ones(5000)), eps=1e-8, block=32)
    # subnormal and huge components
    x = np.array([5e-324, 3 * 2.0**-1074, 1e-310, 1.5, 1e300, -1e308, 2.0**-1022])
    y = np.array([1e300, 2.0**1000, 3.0, -2.0, 1e-300, 1.0, 7.0])
    for block in (0, 1, 2, 8):
        for eps in (1e-16, 1e-3, 10.0):
            _check(q, orc, x, y, eps, block)
            if block == 1:
                _check(q, orc, x, y, eps, block, explain=False, path="one_pass")


def test_invalid_arguments_raise(q):
    import torch
    x = torch.ones(10, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QdotError):
        q.qdot(x, x, eps=0.0)
    with pytest.raises(q.QdotError):
        q.qdot(x, x, eps=1e-8, block=3)


def test_dot_fp64_comparator(q, orc):
    for kind in ("a", "b", "c"):
        for n in (1, 7, 1000, 1 << 20):
            x, y = workloads.pair(kind, n, 40 + n)
            v = q.dot_fp64(_dev(x), _dev(y))
            assert abs(v - orc.dot_exact(x, y)) <= TOL * orc.abs_dot_exact(x, y)


def test_from_host_end_to_end(q, orc):
    import torch
    x, y = workloads.pair("b", 200001, 77)
    ref = orc.qdot(x, y, eps=1e-8, block=32)
    # pinned host memory (read in place) and pageable host memory (copied)
    for xh, yh in ((torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()),
                   (torch.from_numpy(x.copy()), torch.from_numpy(y.copy()))):
        for block in (32, 1):
            r = q.from_host(xh, yh, eps=1e-8, block=block)
            ref_b = ref if block == 32 else orc.qdot(x, y, eps=1e-8, block=1)
            assert r.count == tuple(ref_b.count)
            assert abs(r.value - ref_b.value) <= TOL * orc.abs_dot_exact(x, y)


def _repairs(q, x, y, eps, block):
    """(result, blocks whose candidate the gather recomputed) of one-pass qdot."""
    import ctypes
    import torch
    sel = torch.zeros(ctypes.sizeof(q.Selection), dtype=torch.uint8, device="cuda")
    out = q.qdot_async(_dev(x), _dev(y), eps=eps, block=block, path="one_pass", selection=sel)
    r = q.decode_result(out.cpu().numpy())
    s = q.Selection.from_buffer_copy(bytes(sel.cpu().numpy()))
    return r, s.reserved[0]


@pytest.mark.parametrize("block", [32, 64, 256])
@pytest.mark.parametrize("eps", [1e-15, 1e-8, 1e-3, 10.0])
def test_one_pass_skipped_candidates_recomputed(q, orc, block, eps):
    """Inputs whose magnitudes grow along the vector: the streaming kernel's
    running bound of e_max lags, it skips candidates the final classes need,
    and the gather recomputes them.  Results must still match the oracle."""
    n = (1 << 20) + 77
    x, y = workloads.pair("a", n, 91)
    ramp = np.exp2(np.linspace(0.0, 60.0, n))
    x = x * ramp
    r, rep = _repairs(q, x, y, eps, block)
    ref = orc.qdot(x, y, eps=eps, block=block)
    assert r.count == tuple(ref.count)
    assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
    assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, y)
    # a shuffled copy of the same components needs (almost) no recomputation
    perm = np.random.default_rng(3).permutation(n)
    r2, rep2 = _repairs(q, x[perm], y[perm], eps, block)
    ref2 = orc.qdot(x[perm], y[perm], eps=eps, block=block)
    assert r2.count == tuple(ref2.count)
    assert abs(r2.value - ref2.value) <= TOL * orc.abs_dot_exact(x, y)
    assert rep2 <= rep


@pytest.mark.parametrize("block", [32, 64, 256])
def test_one_pass_recompute_path(q, orc, block):
    """A ramp 2^0 .. 2^40 whose last component is 2^60: until the end every
    block looks DOUBLE to the streaming kernel, but the final e_max makes the
    blocks with u_b in [12, 35) HALF or SINGLE, so the gather must recompute
    those candidates (n large enough that each warp runs many items)."""
    n = (1 << 24) + 77
    rng = np.random.default_rng(17)
    x = np.exp2(np.linspace(0.0, 40.0, n)) * rng.uniform(1.0, 2.0, n)
    x[-1] = 2.0**60
    y = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    r, rep = _repairs(q, x, y, 1e-8, block)
    ref = orc.qdot(x, y, eps=1e-8, block=block)
    assert rep > 0
    assert r.count[1] > 0 and r.count[2] > 0
    assert r.count == tuple(ref.count)
    assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
    assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, y)


@pytest.mark.parametrize("eps", [1e-15, 1e-8, 1e-3, 10.0])
def test_one_pass_components(q, orc, eps):
    """Blocks of one component in one pass.  An item of 256 components is
    accepted when the warp's bound of e_max was exact and f equals f_spec, and
    recomputed otherwise: a ramp (the bound lags), a ramp whose last component
    dwarfs the rest, and vectors where a third of the products are zero (so
    f > f_spec and every item is recomputed).  Results must match the oracle."""
    import ctypes
    lib = q.load()
    n = (1 << 21) + 77
    rng = np.random.default_rng(29)
    ramp = np.exp2(np.linspace(0.0, 60.0, n)) * rng.uniform(1.0, 2.0, n)
    spike = ramp.copy()
    spike[-1] = 2.0**80
    sparse, ys = workloads.pair("b", n, 41)
    sparse[rng.random(n) < 0.34] = 0.0
    y = rng.uniform(-2.0, 2.0, n)
    for x, yy, need_rep in ((ramp, y, False), (spike, y, True), (sparse, ys, True)):
        r, rep = _repairs(q, x, yy, eps, 1)
        ref = orc.qdot(x, yy, eps=eps, block=1)
        assert r.count == tuple(ref.count)
        assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
        assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, yy)
        if need_rep:
            assert rep > 0
    p = q.params(1e-8, 1, 1, 0, "auto")
    assert lib.qdot_select_path(1 << 24, ctypes.byref(p), 1) == 2  # QDOT_PATH_ONE_PASS
    assert lib.qdot_select_path((1 << 24) - 1, ctypes.byref(p), 1) == 1  # QDOT_PATH_TWO_PASS


@pytest.mark.parametrize("eps", [1e-8, 1e-3])
def test_one_pass_items_blocks_of_32(q, orc, eps):
    """Blocks of 32 with item records (when the library takes them, from
    n = 2^25): the classes per block, the item summed on its own grid and
    recomputed when the bound of e_max it used was not exact (every warp's
    first items at least).  Uniform+outliers with a ragged end, a ramp (the
    bound lags) and vectors with zeros (the general recompute) must match
    the oracle."""
    import ctypes
    lib = q.load()
    n = (1 << 25) + 333
    if lib.qdot_stream_kernel(n, ctypes.byref(q.params(eps, 32, 1, 0, "auto")), 1) != b"k_onepass_items":
        pytest.skip("this build keeps blocks of 32 on block records")
    rng = np.random.default_rng(31)
    x, y = workloads.pair("c", n, 77)
    ramp = x * np.exp2(np.linspace(0.0, 40.0, n))
    sparse = x.copy()
    sparse[rng.random(n) < 0.01] = 0.0
    for xx in (x, ramp, sparse):
        r, rep = _repairs(q, xx, y, eps, 32)
        ref = orc.qdot(xx, y, eps=eps, block=32)
        assert rep > 0
        assert r.count == tuple(ref.count)
        assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
        assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(xx, y)


@pytest.mark.parametrize("block", [32, 64, 128, 256])
def test_fused_path(q, orc, block):
    """One cooperative launch (the solvers' sizes): parity with the oracle and
    with the selection qdot() reports; the largest n it takes and one past."""
    import ctypes
    lib = q.load()
    p = q.params(1e-8, block, 1, 0, "fused")
    n_max = 0
    for n in (257, 1 << 20, 2097152 + 3, 3 * 10**6 + 1):
        x, y = workloads.pair("b", n, 7 + block)
        assert lib.qdot_select_path(n, ctypes.byref(p), 1) == 4  # QDOT_PATH_FUSED
        assert lib.qdot_kernel_launches(n, ctypes.byref(p), 1) == 1
        for eps in (1e-15, 1e-8, 0.1):
            _check(q, orc, x, y, eps, block, explain=False, path="fused")
    # beyond the fused capacity the call falls back to the one-pass path
    big = 1 << 25
    assert lib.qdot_select_path(big, ctypes.byref(p), 1) == 2


@pytest.mark.parametrize("block", [0, 1])
def test_fused_bins_path(q, orc, block):
    """Exact binning and blocks of one in one cooperative launch (selected with
    path="fused"): statistics and the bin counts M_k from one read, the sums
    from a second read out of L2.  Every distribution, the 65536-component
    configuration of +-10^U(-8,0) values, the solvers' sizes and the largest n
    the grid covers; past it the call takes two passes.  AUTO keeps two passes
    for these modes (faster at every size measured)."""
    import ctypes
    lib = q.load()
    p = q.params(1e-8, block, 1, 0, "fused")
    pa = q.params(1e-8, block, 1, 0, "auto")
    for n in (257, 65536, 1 << 20, 2097152 + 3, 3 * 10**6 + 1):
        assert lib.qdot_select_path(n, ctypes.byref(p), 1) == 4  # QDOT_PATH_FUSED
        assert lib.qdot_kernel_launches(n, ctypes.byref(p), 1) == 1
        assert lib.qdot_stream_kernel(n, ctypes.byref(p), 1) == b"k_qdot_fused_bins"
        assert lib.qdot_select_path(n, ctypes.byref(pa), 1) == 1  # AUTO: two passes
        for kind in ("a", "b", "c", "cfg0"):
            if n > 65536 and kind in ("a", "cfg0"):
                continue
            x, y = workloads.pair(kind, n, 70 + block + n % 97)
            for eps in (1e-16, 1e-8, 1e-3, 0.5):
                _check(q, orc, x, y, eps, block, explain=False, path="fused")
    assert lib.qdot_select_path(1 << 23, ctypes.byref(p), 1) == 1  # two passes


def test_fused_bins_edge_cases(q, orc):
    """Zeros, subnormal products, a single component, all components equal
    (one bin of M = n), and a bin count that is an exact power of two."""
    rng = np.random.default_rng(5)
    n = 100000
    x, y = workloads.pair("b", n, 71)
    z = x.copy()
    z[rng.random(n) < 0.05] = 0.0
    sub = x.copy()
    sub[:1000] = 1e-310 * rng.uniform(1.0, 2.0, 1000)
    ones = np.full(4096, 1.0 + 2.0**-20)
    pow2 = np.concatenate([np.full(1024, 3.0), np.full(3000, 2.0**-30)])
    cases = [(z, y), (sub, y), (x[:1], y[:1]), (ones, ones), (pow2, pow2[::-1].copy())]
    for xx, yy in cases:
        for block in (0, 1):
            for eps in (1e-16, 1e-8, 2.0**-8, 4.0, 0.5):
                _check(q, orc, xx, yy, eps, block, explain=False, path="fused")


def test_fused_bins_matches_item_path_bits(q, orc):
    """Blocks of one: the fused launch and the one-pass item path quantize and
    sum every item the same way, so they return the same bits."""
    n = (1 << 21) + 77
    for kind in ("b", "c"):
        x, y = workloads.pair(kind, n, 72)
        xd, yd = _dev(x), _dev(y)
        for eps in (1e-15, 1e-8, 1e-1):
            ra = q.qdot(xd, yd, eps=eps, block=1, path="fused")
            rb = q.qdot(xd, yd, eps=eps, block=1, path="one_pass")
            assert np.float64(ra.value).tobytes() == np.float64(rb.value).tobytes()
            assert ra.count == rb.count


def test_deterministic_repeat(q, orc):
    x, y = workloads.pair("c", 1 << 20, 5)
    xd, yd = _dev(x), _dev(y)
    vals = {q.qdot(xd, yd, eps=1e-3, block=b).value for b in (32,) for _ in range(5)}
    assert len(vals) == 1


@pytest.mark.parametrize("block", [1, 32, 256])
def test_full_size_lognormal(q, orc, block):
    """n = 2^28, lognormal sigma = 4, eps = 1e-8: the benchmark's launch shape,
    checked against a full oracle run."""
    n = 1 << 28
    x, y = workloads.pair("b", n, 2106)
    xd, yd = _dev(x), _dev(y)
    r = q.qdot(xd, yd, eps=1e-8, block=block)
    ref = orc.qdot(x, y, eps=1e-8, block=block)
    assert r.count == tuple(ref.count)
    assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
    assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, y)


@pytest.mark.parametrize("kind,ts", [("A", (10, 40, 100)), ("B", (2, 10, 30))])
def test_paper_distributions_within_bound(q, orc, kind, ts):
    """The paper's synthetic arrays (s 2^p, s ~ U[0.5, 1), p uniform or
    normal with parameter t): the GPU value's error against the exact dot stays
    within the a-priori bound N_bins 2^(e_max + f) (plus the GPU's summation
    tolerance), and the class counts match the oracle's."""
    for n in (100, 1000, 10**4, 10**5):
        for t in ts:
            xd = workloads.exponent_dist(kind, n, t, 900 + n + t)
            yd = workloads.exponent_dist(kind, n, t, 950 + n + t)
            x, y = xd.cpu().numpy(), yd.cpu().numpy()
            exact = orc.dot_exact(x, y)
            for eps in (1e-16, 1e-8, 1e-3):
                for block in (0, 1, 32):
                    r = q.qdot(xd, yd, eps=eps, block=block)
                    ref = orc.qdot(x, y, eps=eps, block=block)
                    assert r.count == tuple(ref.count)
                    assert abs(r.value - exact) <= r.bound + TOL * orc.abs_dot_exact(x, y)
                    assert r.bound <= eps * 2.0 ** r.e_max  # N_bins 2^f <= eps
