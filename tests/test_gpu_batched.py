"""GPU parity of the batched qdot against the oracle, problem by problem."""
import numpy as np
import pytest

import workloads

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


def _pack(arrays):
    """Copy host vectors into one device buffer at 16-byte aligned offsets."""
    import torch
    sizes = [a.shape[0] for a in arrays]
    offs = np.cumsum([0] + [s + (s & 1) for s in sizes])
    buf = torch.empty(int(offs[-1]) + 2, dtype=torch.float64, device="cuda")
    host = np.zeros(int(offs[-1]) + 2)
    for a, o in zip(arrays, offs):
        host[o:o + a.shape[0]] = a
    buf.copy_(torch.from_numpy(host))
    return buf, [buf[o:o + s] for o, s in zip(offs, sizes)]


@pytest.mark.parametrize("block", [32, 64, 256])
def test_batched_matches_oracle(q, orc, block):
    rng = np.random.default_rng(block)
    lengths = [0, 1, 2, 31, 32, 33, 255, 256, 257, 1000, 4097] + list(
        np.floor(np.exp2(rng.uniform(0, 17, 60))).astype(int))
    kinds = ["a", "b", "c", "cfg0"]
    xs, ys = [], []
    for i, n in enumerate(lengths):
        x, y = workloads.pair(kinds[i % 4], int(n), 3000 + i)
        if i % 7 == 3 and n > 3:
            x[1] = 0.0      # zero components inside a block
            y[n - 1] = 0.0
        xs.append(x)
        ys.append(y)
    bx, xd = _pack(xs)
    by, yd = _pack(ys)
    for eps in (1e-12, 1e-8, 1e-2):
        b = q.Batch(xd, yd, eps=eps, block=block)
        b.launch()
        res = b.results()
        for i, (x, y, r) in enumerate(zip(xs, ys, res)):
            ref = orc.qdot(x, y, eps=eps, block=block)
            assert r.status == 0, (i, r)
            assert r.count == tuple(ref.count), (i, r.count, ref.count)
            assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f), i
            assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, y), (i, r.value, ref.value)


def test_batched_graph_replay_and_bad_pair(q, orc):
    import torch
    lengths = [5000, 70000, 3, 123457, 0, 65536]
    xs = [workloads.pair("b", n, 77 + n)[0] for n in lengths]
    ys = [workloads.pair("b", n, 77 + n)[1] for n in lengths]
    bx, xd = _pack(xs)
    by, yd = _pack(ys)
    b = q.Batch(xd, yd, eps=1e-8, block=32)
    b.launch()
    torch.cuda.synchronize()
    first = b.results()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.launch(stream=s)  # warm the stream before capture
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        b.launch(stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    again = b.results()
    for r1, r2, x, y in zip(first, again, xs, ys):
        ref = orc.qdot(x, y, eps=1e-8, block=32)
        assert r1.value == r2.value and r1.count == r2.count == tuple(ref.count)
    # a misaligned problem is reported, the others are unaffected
    xm = [xd[0], xd[1][1:], xd[3]]
    ym = [yd[0], yd[1][1:], yd[3]]
    bm = q.Batch(xm, ym, eps=1e-8, block=32)
    bm.launch()
    rm = bm.results()
    assert rm[1].status == 1
    assert rm[0].count == first[0].count and rm[2].count == first[3].count


def test_batched_late_maximum_and_large_pairs(q, orc):
    """Blocks of 32 (item records per pair): pairs whose largest product sits
    in their last item, so that most of their items were summed with a stale
    bound and are taken with changed blocks swapped in or summed again; a pair
    of 2^20 components split over many warps; many one-item pairs."""
    import torch
    rng = np.random.default_rng(8)
    lengths = [1 << 20, 300000, 65536, 4096, 256, 257] + [int(v) for v in rng.integers(1, 600, 40)]
    xs, ys = [], []
    for i, n in enumerate(lengths):
        x, y = workloads.pair("b", n, 900 + i)
        if n > 1000 and i % 2 == 0:  # the largest product in the last item
            x[-2] = np.abs(x).max() * 8.0
            y[-2] = np.abs(y).max() * 8.0
        xs.append(x)
        ys.append(y)
    bx, xd = _pack(xs)
    by, yd = _pack(ys)
    for eps in (1e-15, 1e-8, 1e-1):
        b = q.Batch(xd, yd, eps=eps, block=32)
        b.launch()
        res = b.results()
        for i, (x, y, r) in enumerate(zip(xs, ys, res)):
            ref = orc.qdot(x, y, eps=eps, block=32)
            assert r.status == 0, (i, r)
            assert r.count == tuple(ref.count), (i, r.count, ref.count)
            assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f), i
            assert abs(r.value - ref.value) <= TOL * orc.abs_dot_exact(x, y), (i, r.value, ref.value)


@pytest.mark.parametrize("block", [32, 64])
def test_every_launch_shape_gives_the_same_results(q, orc, tmp_path, block):
    """Every launch shape the tuner tries gives the same values (blocks of 32:
    item records, whose speculation depends on the shape but whose values do
    not; blocks of 64: block records)."""
    import numpy as np
    import torch
    from paper_2105_00115_gb300 import _abi, tune
    lengths = [0, 1, 255, 256, 257, 4096, 70001, 33, 1 << 16]
    xs, ys, ref = [], [], []
    for i, n in enumerate(lengths):
        x, y = workloads.pair("b", n, 300 + i)
        xs.append(torch.from_numpy(x).cuda())
        ys.append(torch.from_numpy(y).cuda())
        ref.append(orc.qdot(x, y, eps=1e-8, block=block))
    batch = q.Batch(xs, ys, eps=1e-8, block=block)
    seen = set()
    for threads, ctas, staged in tune.CANDIDATES:
        batch.tuning = _abi.BatchedTuning(threads, ctas, 0, staged)
        batch.launch()
        res = batch.results()
        seen.add(tuple(r.value for r in res))
        for r, o, x in zip(res, ref, xs):
            assert r.count == tuple(o.count)
    assert len(seen) == 1  # identical values for every launch shape
    tuning, times = batch.autotune(reps=2, path=str(tmp_path / f"t{block}.json"))
    assert (tuning.threads_per_cta, tuning.ctas_per_sm, tuning.staged) in tune.CANDIDATES
    assert len(times) == len(tune.CANDIDATES)
    tuning2, _ = batch.autotune(reps=2, path=str(tmp_path / f"t{block}.json"))  # from the cache
    assert (tuning2.threads_per_cta, tuning2.ctas_per_sm, tuning2.staged) == \
        (tuning.threads_per_cta, tuning.ctas_per_sm, tuning.staged)
