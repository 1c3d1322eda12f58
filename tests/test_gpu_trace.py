"""Element-wise parity of the timed kernels (fused, one-pass with block
records, one-pass with item records) against the CPU oracle, through
qdot_trace(): the same launches as qdot(), plus what they decided.

For every unit of work (a block of B components, or a warp item of 256):
- the class the selection gave it (expanded to components; on item paths the
  per-component class map the kernels summed with) equals the oracle's class
  map bit for bit;
- the value the final sum took from it, value * 2^grid, is within
  unit * 2^-52 * sum_unit |x_i y_i| of the oracle's exact sum of
  q(x_i) q(y_i) over the same components (the per-lane chain roundings and
  grid truncations of the kernels, derived in qdot_chunk.cuh, stay below
  that);
- a perforated or empty unit adds exactly 0.
A wrong candidate slot, a stale window or a wrong recomputation changes a
unit's value by far more than its tolerance, even when the total stays
within 1e-13 sum |x_i y_i|.

Every candidate has one definition whatever route computes it, so repeated
calls, and the fused and one-pass paths on the same data, agree bit for bit.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-13
SRC = {"none": 0, "slot0": 1, "slot1": 2, "slot3": 3, "recomputed": 4, "fused": 5, "item": 6, "item_recomputed": 7,
       "item_fixed": 8}


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


def _class_map(units, per, cls, x, y, block):
    """Per-component classes the kernels used: item paths report them per
    component; block paths per block (ZERO for the block's zero products)."""
    if cls is not None:
        return cls.cpu().numpy()
    n = x.shape[0]
    m = np.repeat(units["cls"], per)[:n].copy()
    m[(x == 0.0) | (y == 0.0)] = 4
    return m


def check_trace(q, orc, x, y, eps, block, path="auto", expect_kernel=None, xd=None, yd=None):
    """Run qdot_trace and compare it with the oracle unit by unit; returns
    (result, units) for further checks."""
    lib = q.load()
    if xd is None:
        xd, yd = _dev(x), _dev(y)
    if expect_kernel is not None:
        p = q.params(eps, block, 1, 0, path)
        assert lib.qdot_stream_kernel(x.shape[0], ctypes.byref(p), 1).decode() == expect_kernel
    r, units, per, cls = q.trace(xd, yd, eps=eps, block=block, path=path)
    ref = orc.qdot(x, y, eps=eps, block=block, explain=True)
    assert r.status == 0
    assert r.count == tuple(ref.count)
    assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
    assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, y)
    # the class map, bit for bit
    np.testing.assert_array_equal(_class_map(units, per, cls, x, y, block), ref.cls)
    # every unit's value against the oracle's exact partial sum
    sums, abss = orc.unit_sums(x, y, per, eps=eps, block=block)
    assert len(units) == len(sums)
    val = np.ldexp(units["value"].astype(np.float64), units["grid"])
    err = np.abs(val - sums)
    tol = per * 2.0**-52 * abss + 2.0**-1074
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, (f"{bad.size} units off, first {bad[:5]}: value {val[bad[:5]]} oracle {sums[bad[:5]]} "
                           f"sources {units['source'][bad[:5]]}")
    # perforated and empty units add exactly nothing
    if per == block:
        none = units["source"] == SRC["none"]
        assert np.all(np.isin(units["cls"][none], (0, 4)))
        assert np.all(units["value"][none] == 0)
    return r, units


@pytest.mark.parametrize("block", [32, 64, 256])
def test_trace_fused(q, orc, block):
    """The one-launch path at the solvers' sizes (Theorem 5 fast path included:
    eps = 1e-15 leaves every block DOUBLE on kind a)."""
    n = (1 << 21) + 77
    for kind in ("a", "b", "c"):
        x, y = workloads.pair(kind, n, 300 + block)
        xd, yd = _dev(x), _dev(y)
        for eps in (1e-15, 1e-8, 1e-1):
            _, units = check_trace(q, orc, x, y, eps, block, expect_kernel="k_qdot_fused", xd=xd, yd=yd)
            assert np.all(np.isin(units["source"], (SRC["none"], SRC["fused"])))


@pytest.mark.parametrize("block", [0, 1])
def test_trace_fused_bins(q, orc, block):
    """The one-launch path for exact binning and blocks of one: the class map
    it summed with and every item's value; zeros in one case."""
    n = (1 << 21) + 77
    rng = np.random.default_rng(9)
    for kind in ("b", "c", "cfg0"):
        x, y = workloads.pair(kind, n, 310 + block)
        if kind == "c":
            x[rng.random(n) < 0.01] = 0.0
        xd, yd = _dev(x), _dev(y)
        for eps in (1e-16, 1e-8, 1e-1):
            _, units = check_trace(q, orc, x, y, eps, block, path="fused", expect_kernel="k_qdot_fused_bins",
                                   xd=xd, yd=yd)
            assert np.all(np.isin(units["source"], (SRC["none"], SRC["fused"])))


@pytest.mark.parametrize("block", [32, 64, 256])
def test_trace_one_pass_blocks(q, orc, block):
    """k_onepass + k_op_gather at a size past the fused limit, a ragged end,
    every class reachable."""
    n = (1 << 24) + 333
    for kind, epss in (("b", (1e-15, 1e-8, 1e-1)), ("c", (1e-8,))):
        x, y = workloads.pair(kind, n, 400 + block)
        xd, yd = _dev(x), _dev(y)
        for eps in epss:
            _, units = check_trace(q, orc, x, y, eps, block, expect_kernel="k_onepass", xd=xd, yd=yd)
            used = set(np.unique(units["source"]).tolist())
            assert used <= {SRC["none"], SRC["slot0"], SRC["slot1"], SRC["slot3"], SRC["recomputed"]}


@pytest.mark.parametrize("block", [32, 64, 256])
def test_trace_one_pass_recomputed(q, orc, block):
    """A ramp whose last component dwarfs the rest: the streaming kernel keeps
    the wrong candidates for many blocks and the gather recomputes them; the
    recomputed values must be those of the oracle, block by block."""
    n = (1 << 24) + 77
    rng = np.random.default_rng(17)
    x = np.exp2(np.linspace(0.0, 40.0, n)) * rng.uniform(1.0, 2.0, n)
    x[-1] = 2.0**60
    y = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    x[rng.random(n) < 0.001] = 0.0  # blocks with zeros take the general route
    _, units = check_trace(q, orc, x, y, 1e-8, block, path="one_pass")
    assert np.count_nonzero(units["source"] == SRC["recomputed"]) > 0


@pytest.mark.parametrize("eps", [1e-15, 1e-8, 1e-1])
def test_trace_one_pass_components(q, orc, eps):
    """k_onepass_items + k_op_gather_items (blocks of one component): the
    per-component class map the kernels summed with, and every item's value;
    lognormal, uniform with outliers, zeros (statistics-only items), and a
    spike at the end (every item recomputed)."""
    n = (1 << 24) + 77
    rng = np.random.default_rng(23)
    xb, yb = workloads.pair("b", n, 61)
    xc, yc = workloads.pair("c", n, 62)
    sparse = xb.copy()
    sparse[rng.random(n) < 0.02] = 0.0
    spike = xc.copy()
    spike[-1] = 1e30
    for x, y, need_rec in ((xb, yb, False), (xc, yc, False), (sparse, yb, True), (spike, yc, True)):
        _, units = check_trace(q, orc, x, y, eps, 1, expect_kernel="k_onepass_items")
        assert set(np.unique(units["source"]).tolist()) <= {SRC["item"], SRC["item_recomputed"]}
        if need_rec:
            assert np.count_nonzero(units["source"] == SRC["item_recomputed"]) > 0


def _boundary_operands(n, seed):
    """float64 values whose significands sit on the rounding boundaries of
    both classes (exact HALF and SINGLE ties, one unit above and below them,
    all-ones fractions that carry into the exponent) or are random, with
    exponents spread over [-40, 40] so that every class occurs in every warp."""
    rng = np.random.default_rng(seed)
    kind = rng.integers(0, 8, n)
    r10 = rng.integers(0, 1 << 10, n, dtype=np.uint64)
    r23 = rng.integers(0, 1 << 23, n, dtype=np.uint64)
    one = np.uint64(1)
    frac = np.select(
        [kind == 0, kind == 1, kind == 2, kind == 3, kind == 4, kind == 5, kind == 6],
        [(r10 << np.uint64(42)) | (one << np.uint64(41)),                                  # HALF tie
         (r10 << np.uint64(42)) | (one << np.uint64(41)) | one,                             # just above
         (r10 << np.uint64(42)) | ((one << np.uint64(41)) - one),                           # just below
         (r23 << np.uint64(29)) | (one << np.uint64(28)),                                   # SINGLE tie
         (r23 << np.uint64(29)) | (one << np.uint64(28)) | one,
         (r23 << np.uint64(29)) | ((one << np.uint64(28)) - one),
         (one << np.uint64(52)) - one],                                                     # all ones: carry
        rng.integers(0, 1 << 52, n, dtype=np.uint64))
    expo = (rng.integers(-40, 41, n) + 1023).astype(np.uint64)
    sign = rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63)
    return (sign | (expo << np.uint64(52)) | frac).view(np.float64)


@pytest.mark.parametrize("eps", [1e-8, 1e-3])
def test_trace_components_rounding_boundaries(q, orc, eps):
    """Blocks of one on operands at the rounding boundaries: ties to even,
    one unit off a tie, and carries out of the significand, for HALF and
    SINGLE components mixed with PERF and DOUBLE ones in every warp (the
    streaming kernel's per-class rounding table), on the item path and on
    the one-launch path for blocks of one."""
    n = (1 << 24) + 77
    x, y = _boundary_operands(n, 71), _boundary_operands(n, 72)
    r, units = check_trace(q, orc, x, y, eps, 1, expect_kernel="k_onepass_items")
    assert all(c > 0 for c in r.count[:4])  # every class occurs
    m = (1 << 21) + 77
    r2, _ = check_trace(q, orc, x[:m], y[:m], eps, 1, path="fused")
    assert all(c > 0 for c in r2.count[:4])


def test_trace_one_pass_items_blocks_of_32(q, orc):
    """k_onepass_items + k_op_gather_items with blocks of 32 (n from 2^25):
    each block classed from its key log2 B + u_b, each item of 256 summed on
    its own grid or recomputed; the per-component class map and every item's
    value against the oracle.  Lognormal and uniform-with-outliers data with a
    ragged end, zeros (statistics-only items, general recompute) and a ramp
    whose bound of e_max lags (many items recomputed)."""
    n = (1 << 25) + 333
    rng = np.random.default_rng(41)
    for kind in ("b", "c"):
        x, y = workloads.pair(kind, n, 600)
        xd, yd = _dev(x), _dev(y)
        for eps in (1e-15, 1e-8, 1e-1):
            _, units = check_trace(q, orc, x, y, eps, 32, expect_kernel="k_onepass_items", xd=xd, yd=yd)
            assert set(np.unique(units["source"]).tolist()) <= {SRC["item"], SRC["item_recomputed"],
                                                                 SRC["item_fixed"]}
    x, y = workloads.pair("c", n, 601)
    sparse = x.copy()
    sparse[rng.random(n) < 0.01] = 0.0
    ramp = x * np.exp2(np.linspace(0.0, 40.0, n))
    for xx in (sparse, ramp):
        _, units = check_trace(q, orc, xx, y, 1e-8, 32, expect_kernel="k_onepass_items")
        assert np.count_nonzero(np.isin(units["source"], (SRC["item_recomputed"], SRC["item_fixed"]))) > 0


def test_trace_items_late_maximum(q, orc):
    """Blocks of 32 and of one on item records when the largest product sits in
    the last item: every earlier item was summed with a bound of e_max below
    the final one.  Blocks of one: those items are summed again.  Blocks of
    32: an item whose blocks all keep their class is taken as recorded; in the
    others only the changed blocks are summed again and swapped in
    (QDOT_TRACE_ITEM_FIXED), unless the item's grid is finer than the final
    sum's, where the item is summed again whole.  Every item's value and the class map must still be the
    oracle's."""
    n = (1 << 25) + 256 * 7
    x, y = workloads.pair("b", n, 602)
    for spike in (2.0**3, 2.0**10):  # the last item's product lies 6 or 20 binades above the rest
        xx, yy = x.copy(), y.copy()
        xx[-3] = np.abs(x).max() * spike
        yy[-3] = np.abs(y).max() * spike
        xd, yd = _dev(xx), _dev(yy)
        for block, eps in ((32, 1e-15), (32, 1e-8), (32, 1e-1), (1, 1e-8)):
            r, units = check_trace(q, orc, xx, yy, eps, block, expect_kernel="k_onepass_items", xd=xd, yd=yd)
            src = units["source"]
            if block == 1:
                assert np.count_nonzero(src == SRC["item_recomputed"]) > src.size // 2
            else:
                assert np.count_nonzero(src == SRC["item_fixed"]) > 0
                # only items whose grid 2^(u - 52) is finer than the sum's 2^(e_max - L) are summed again whole
                keys = (np.frexp(xx)[1] - 1) + (np.frexp(yy)[1] - 1)
                u = keys.reshape(-1, 256).max(axis=1)
                L = min(104, 124 - int(np.ceil(np.log2(n))))
                fine = np.count_nonzero(u - 52 < r.e_max - L)
                assert np.count_nonzero(src == SRC["item_recomputed"]) <= fine + 3 * 3648  # + every warp's first items


def test_trace_repeatable_bit_for_bit(q, orc):
    """The one-pass path's speculation depends on timing (a shared running
    bound of e_max), but every candidate has one definition: repeated calls
    return the same bits, unit by unit, for blocks of 32 and 256 and for
    single components."""
    n = (1 << 25) + 333
    x, y = workloads.pair("b", n, 2107)
    xd, yd = _dev(x), _dev(y)
    for block in (32, 256, 1):
        first = None
        for _ in range(4):
            r, units, per, _ = q.trace(xd, yd, eps=1e-8, block=block, path="one_pass", want_cls=False)
            key = (np.float64(r.value).tobytes(), units["value"].tobytes(), units["grid"].tobytes(),
                   units["cls"].tobytes())
            if first is None:
                first = key
            assert key == first
        for _ in range(3):
            r2 = q.qdot(xd, yd, eps=1e-8, block=block, path="one_pass")
            assert np.float64(r2.value).tobytes() == first[0]


def test_fused_and_one_pass_agree_bit_for_bit(q, orc):
    """The fused and one-pass paths form every candidate the same way, so on
    the same data they return the same bits (blocks of 32 .. 256)."""
    n = (1 << 21) + 77
    for kind in ("b", "c"):
        x, y = workloads.pair(kind, n, 500)
        xd, yd = _dev(x), _dev(y)
        for block in (32, 64, 128, 256):
            for eps in (1e-15, 1e-8, 1e-1):
                ra, ua, _, _ = q.trace(xd, yd, eps=eps, block=block, path="fused")
                rb, ub, _, _ = q.trace(xd, yd, eps=eps, block=block, path="one_pass")
                assert np.float64(ra.value).tobytes() == np.float64(rb.value).tobytes()
                assert ra.count == rb.count
                assert np.array_equal(ua["cls"], ub["cls"])
                kept = ua["cls"] != 0
                assert np.array_equal(ua["value"][kept], ub["value"][kept])
                assert np.array_equal(ua["grid"][kept], ub["grid"][kept])


def test_trace_full_size_benched_cell(q, orc):
    """The benchmark's own cell (n = 2^28, lognormal sigma = 4, blocks of 32,
    eps = 1e-8, the same seed and launch shape as bench.py), unit by unit."""
    n = 1 << 28
    x, y = workloads.pair("b", n, 2106)
    check_trace(q, orc, x, y, 1e-8, 32, expect_kernel="k_onepass_items")


def test_trace_rejects_two_pass(q):
    import torch
    x = torch.ones(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QdotError):
        q.trace(x, x, eps=1e-8, block=0)
    with pytest.raises(q.QdotError):
        q.trace(x, x, eps=1e-8, block=8)
