"""GPU ACG (Algorithm 4) and APM (Algorithm 5) against the oracle's.

The GPU qdot meets the oracle's value within 1e-13 * sum |x_i y_i| (not bit
for bit), so iterates drift apart by rounding-sized amounts.  The bar:
  * first iteration: the class counts of qdot(p0, A p0) equal the oracle's
    (identical inputs), values within the qdot tolerance;
  * well-conditioned operator: identical iteration counts, solutions within
    1e-8 relative;
  * variable-coefficient (ill-conditioned) operator: both converge, iteration
    counts within 3%, the true residual small;
  * power method: eigenvalue within 1e-10 relative of the oracle's.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("block,eps", [(0, 1e-16), (1, 1e-3), (32, 1e-8), (256, 1e-2)])
def test_cg_first_iteration(q, orc, block, eps):
    rp, col, val = workloads.poisson3d(12, 10, 9)
    n = rp.shape[0] - 1
    b = workloads.rhs(n)
    x, info, hist = q.cg(q.Csr(rp, col, val), _dev(b), rel_tol=1e-10, max_it=1, eps=eps, block=block, history=True)
    xo, it, rr, counts, st = orc.cg(rp, col, val, b, rel_tol=1e-10, max_it=1, eps=eps, block=block)
    assert info["iters"] == it == 1 and info["status"] == q.QDOT_ERR_NOCONV
    # p0 = b and q0 = A b are bit-identical on both sides
    Ab = orc.spmv(rp, col, val, b)
    ref = orc.qdot(b, Ab, eps=eps, block=block)
    np.testing.assert_array_equal(hist[0, 0], ref.count)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-12 * np.linalg.norm(xo)
    assert abs(info["relres"] - rr) <= 1e-10 * rr


@pytest.mark.parametrize("block,eps", [(0, 1e-16), (1, 1e-6), (32, 1e-8), (256, 1e-4)])
def test_cg_well_conditioned(q, orc, block, eps):
    rp, col, val = workloads.laplace3d(14, 12, 10)
    n = rp.shape[0] - 1
    b = workloads.rhs(n)
    x, info, hist = q.cg(q.Csr(rp, col, val), _dev(b), rel_tol=1e-10, max_it=5000, eps=eps, block=block,
                        history=True)
    xo, it, rr, counts, st = orc.cg(rp, col, val, b, rel_tol=1e-10, max_it=5000, eps=eps, block=block)
    assert st == 0 and info["status"] == 0
    assert info["iters"] == it
    assert info["relres"] <= 1e-10 and rr <= 1e-10
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    assert hist.shape == (it, 2, 5) and int(hist.sum()) == sum(info["counts"]) - n  # minus the initial r.r
    assert info["true_relres"] <= 1e-9


@pytest.mark.parametrize("block,eps", [(0, 1e-16), (32, 1e-8)])
def test_cg_variable_coefficients(q, orc, block, eps):
    rp, col, val = workloads.poisson3d(12, 10, 9)
    n = rp.shape[0] - 1
    b = workloads.rhs(n)
    A = q.Csr(rp, col, val)
    x, info, _ = q.cg(A, _dev(b), rel_tol=1e-10, max_it=40000, eps=eps, block=block)
    xo, it, rr, counts, st = orc.cg(rp, col, val, b, rel_tol=1e-10, max_it=40000, eps=eps, block=block)
    assert st == 0 and info["status"] == 0 and info["relres"] <= 1e-10
    assert abs(info["iters"] - it) <= 0.03 * it, (info["iters"], it)
    # the comparator: the same GPU solver with plain FP64 dot products
    x64, i64, _ = q.cg(A, _dev(b), rel_tol=1e-10, max_it=40000, dot="fp64")
    assert i64["status"] == 0 and sum(i64["counts"]) == 0
    assert abs(info["iters"] - i64["iters"]) <= 0.03 * i64["iters"], (info["iters"], i64["iters"])


def test_cg_iteration_cap_and_fp64_mode(q, orc):
    rp, col, val = workloads.laplace3d(10, 10, 10)
    n = rp.shape[0] - 1
    b = workloads.rhs(n)
    A = q.Csr(rp, col, val)
    x, info, _ = q.cg(A, _dev(b), rel_tol=1e-14, max_it=7, eps=1e-16, block=0)
    assert info["iters"] == 7 and info["status"] == q.QDOT_ERR_NOCONV
    # plain-FP64 mode against a textbook CG in numpy (same recurrences, numpy dots)
    x64, i64, _ = q.cg(A, _dev(b), rel_tol=1e-10, max_it=5000, dot="fp64")
    import scipy.sparse as sp
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    xr = np.zeros(n); r = b.copy(); p = r.copy(); c = r @ r; k = 0
    while k < 5000 and np.sqrt(c) / np.linalg.norm(b) > 1e-10:
        qv = M @ p; a = c / (p @ qv); xr += a * p; r -= a * qv; cn = r @ r; p = r + (cn / c) * p; c = cn; k += 1
    assert i64["status"] == 0 and abs(i64["iters"] - k) <= 1
    assert np.linalg.norm(x64.cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)


@pytest.mark.parametrize("block,eps,tau", [(0, 1e-16, 0.0), (0, 1e-7, 0.0), (32, 1e-4, 0.0), (1, 1e-2, 0.0),
                                           (32, 1e-8, 1e-9)])
def test_power_matches_oracle(q, orc, block, eps, tau):
    rp, col, val = workloads.poisson2d(40, 33)
    n = rp.shape[0] - 1
    x0 = workloads.unit_start(n)
    lam, x, info, hist = q.power(q.Csr(rp, col, val), _dev(x0), iters=300, tau=tau, eps=eps, block=block,
                                 history=True)
    lo, xo, it, counts, st = orc.power(rp, col, val, x0, iters=300, tau=tau, eps=eps, block=block)
    assert st == 0 and info["status"] == 0
    if tau == 0.0:
        assert info["iters"] == it == 300
    else:
        assert abs(info["iters"] - it) <= 1
    assert abs(lam - lo) <= 1e-10 * abs(lo)
    assert hist.shape == (info["iters"], 2, 5)
    assert (hist.sum(axis=2) == n).all()
    # the first iteration's Rayleigh quotient sees identical inputs
    ref = orc.qdot(x0, orc.spmv(rp, col, val, x0), eps=eps, block=block)
    np.testing.assert_array_equal(hist[0, 0], ref.count)


def test_power_iters_zero(q):
    rp, col, val = workloads.poisson2d(8, 8)
    n = rp.shape[0] - 1
    x0 = workloads.unit_start(n)
    lam, x, info, _ = q.power(q.Csr(rp, col, val), _dev(x0), iters=0)
    assert info["iters"] == 0 and lam == 0.0
    np.testing.assert_array_equal(x.cpu().numpy(), x0)


def _systems(kind, edges, seed=500):
    blocks = []
    for i, e in enumerate(edges):
        if kind == "laplace":
            blocks.append(workloads.laplace3d(e, e + 1, e))
        else:
            blocks.append(workloads.poisson3d(e, e, e, seed=seed + i))
    return blocks


@pytest.mark.parametrize("block,eps", [(32, 1e-16), (32, 1e-6), (64, 1e-3), (256, 1e-8)])
def test_cg_batched_matches_single(q, orc, block, eps):
    """Each system of the batch follows the single-system solver exactly (the
    batched qdot and the single qdot compute the same values) and, on these
    well-conditioned operators, takes the oracle's iteration count."""
    blocks = _systems("laplace", [3, 6, 4, 9, 5, 7, 8])
    rp, col, val, off = workloads.block_diagonal(blocks)
    b = workloads.rhs(int(off[-1]), seed=77)
    x, infos = q.cg_batched(q.Csr(rp, col, val), off, _dev(b), rel_tol=1e-10, max_it=3000, eps=eps, block=block)
    xg = x.cpu().numpy()
    for s, (brp, bcol, bval) in enumerate(blocks):
        bs = b[off[s]:off[s + 1]]
        xs1, info1, _ = q.cg(q.Csr(brp, bcol, bval), _dev(bs), rel_tol=1e-10, max_it=3000, eps=eps, block=block)
        assert infos[s]["status"] == 0 and infos[s]["iters"] == info1["iters"], (s, infos[s], info1)
        np.testing.assert_allclose(xg[off[s]:off[s + 1]], xs1.cpu().numpy(), rtol=0, atol=1e-12 * np.abs(xg).max())
        xo, it, rr, counts, st = orc.cg(brp, bcol, bval, bs, rel_tol=1e-10, max_it=3000, eps=eps, block=block)
        assert it == infos[s]["iters"]
        assert infos[s]["relres"] <= 1e-10 and infos[s]["true_relres"] <= 1e-9


def test_cg_batched_variable_coefficients_and_fp64(q, orc):
    blocks = _systems("poisson", [4, 7, 5, 6])
    rp, col, val, off = workloads.block_diagonal(blocks)
    b = workloads.rhs(int(off[-1]), seed=78)
    A = q.Csr(rp, col, val)
    x, infos = q.cg_batched(A, off, _dev(b), rel_tol=1e-10, max_it=20000, eps=1e-8, block=32)
    x64, i64 = q.cg_batched(A, off, _dev(b), rel_tol=1e-10, max_it=20000, dot="fp64")
    for s, (brp, bcol, bval) in enumerate(blocks):
        bs = b[off[s]:off[s + 1]]
        xo, it, rr, counts, st = orc.cg(brp, bcol, bval, bs, rel_tol=1e-10, max_it=20000, eps=1e-8, block=32)
        assert infos[s]["status"] == 0 and infos[s]["relres"] <= 1e-10
        assert abs(infos[s]["iters"] - it) <= max(3, 0.03 * it)
        # plain FP64 dots: converges (on these tiny ill-conditioned systems the
        # count itself moves with the summation order of the dots)
        assert i64[s]["status"] == 0 and sum(i64[s]["counts"]) == 0 and i64[s]["relres"] <= 1e-10


def test_cg_batched_iteration_cap_and_bad_column(q):
    blocks = _systems("laplace", [5, 6])
    rp, col, val, off = workloads.block_diagonal(blocks)
    b = workloads.rhs(int(off[-1]), seed=79)
    x, infos = q.cg_batched(q.Csr(rp, col, val), off, _dev(b), rel_tol=1e-14, max_it=5, eps=1e-16, block=32)
    assert all(i["iters"] == 5 and i["status"] == q.QDOT_ERR_NOCONV for i in infos)
    # a column that reaches into the other system is refused (not read)
    col2 = col.copy()
    col2[3] = int(off[1]) + 2
    x, infos = q.cg_batched(q.Csr(rp, col2, val), off, _dev(b), rel_tol=1e-10, max_it=50, eps=1e-16, block=32)
    assert all(i["status"] == q.QDOT_ERR_ARG for i in infos)


# ---------------------------------------------------------------------------
# The paper's problem shapes (Sec. 4.2 and 4.3): the 27-point operator on a
# chimney-like box with b = A 1 and x0 = 0, stopped on an absolute residual
# tau = 1e-8; the power method on a random graph Laplacian with tau = 1e-6 and
# at most 300 iterations.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("block,eps", [(0, 1e-16), (0, 1.0), (0, 1e2), (32, 1e-8), (32, 1e2), (1, 1e-3)])
def test_cg_stencil27_matches_oracle(q, orc, block, eps):
    """27-point chimney-like box (30 x 30 x 3): the first iteration's class
    counts equal the oracle's (identical inputs), and the whole solve takes the
    oracle's iteration count (well-conditioned operator), to the same x."""
    rp, col, val = workloads.stencil27(30, 30, 3)
    n = rp.shape[0] - 1
    b = workloads.ones_rhs(rp, col, val)
    rel = 1e-8 / np.linalg.norm(b)  # Algorithm 4 stops on ||r|| <= tau = 1e-8
    A = q.Csr(rp, col, val)
    x, info, hist = q.cg(A, _dev(b), rel_tol=rel, max_it=2000, eps=eps, block=block, history=True)
    xo, it, rr, counts, st = orc.cg(rp, col, val, b, rel_tol=rel, max_it=2000, eps=eps, block=block)
    ref = orc.qdot(b, orc.spmv(rp, col, val, b), eps=eps, block=block)
    np.testing.assert_array_equal(hist[0, 0], ref.count)
    assert st == 0 and info["status"] == 0
    assert info["iters"] == it
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    assert np.linalg.norm(xg - 1.0) <= 1e-6 * np.sqrt(n)


def test_cg_stencil27_paper_protocol(q, orc):
    """The paper's ACG protocol on a small chimney box: eps swept x10 from
    1e-16 to 1e3 with exact binning; at every eps the GPU solver takes the
    oracle's iteration count, and the largest eps that keeps the FP64-dot
    count is the same on both sides."""
    rp, col, val = workloads.stencil27(40, 40, 1)
    b = workloads.ones_rhs(rp, col, val)
    rel = 1e-8 / np.linalg.norm(b)
    A = q.Csr(rp, col, val)
    bd = _dev(b)
    _, i64, _ = q.cg(A, bd, rel_tol=rel, max_it=5000, dot="fp64")
    best_gpu = best_orc = None
    for k in range(-16, 4):
        eps = 10.0 ** k
        _, info, _ = q.cg(A, bd, rel_tol=rel, max_it=5000, eps=eps, block=0)
        _, it, _, _, st = orc.cg(rp, col, val, b, rel_tol=rel, max_it=5000, eps=eps, block=0)
        assert info["iters"] == it, (eps, info["iters"], it)
        if info["status"] == 0 and info["iters"] == i64["iters"]:
            best_gpu = eps
        if st == 0 and it == i64["iters"]:
            best_orc = eps
    assert best_gpu is not None and best_gpu == best_orc


@pytest.mark.parametrize("block,eps", [(0, 1e-16), (0, 1e-7), (0, 1e-3), (32, 1e-7), (1, 1e-5)])
def test_power_graph_laplacian(q, orc, block, eps):
    """Random graph Laplacian (n = 3000): APM with tau = 1e-6 and at most 300
    iterations takes the oracle's iteration count and eigenvalue; the first
    Rayleigh quotient's class counts equal the oracle's."""
    rp, col, val = workloads.graph_laplacian(3000, 8)
    n = rp.shape[0] - 1
    x0 = workloads.unit_start(n)
    lam, x, info, hist = q.power(q.Csr(rp, col, val), _dev(x0), iters=300, tau=1e-6, eps=eps, block=block,
                                 history=True)
    lo, xo, it, counts, st = orc.power(rp, col, val, x0, iters=300, tau=1e-6, eps=eps, block=block)
    assert st == 0 and info["status"] == 0
    assert abs(info["iters"] - it) <= 1
    assert abs(lam - lo) <= 1e-9 * abs(lo)
    ref = orc.qdot(x0, orc.spmv(rp, col, val, x0), eps=eps, block=block)
    np.testing.assert_array_equal(hist[0, 0], ref.count)
