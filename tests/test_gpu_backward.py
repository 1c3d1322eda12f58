"""GPU backward of qdot (the class map held fixed) against the oracle gradient
and central finite differences.

Bar: gx = g * q_c(y), gy = g * q_c(x) bit for bit against the oracle's
backward with the oracle's class map (g taken from the GPU's upstream
gradient, so both sides multiply the same numbers); finite differences of the
GPU forward agree with the gradient on components whose class stays double.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_00115_gb300 import build as qbuild
    qbuild.build()
    import paper_2105_00115_gb300 as qq
    qq.load()
    from paper_2105_00115_gb300 import autograd
    return autograd


def _dev(a, grad=True):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().requires_grad_(grad)


def _bits(a):
    return np.asarray(a).view(np.int64)


@pytest.mark.parametrize("block,eps", [(0, 1e-16), (0, 1e-4), (1, 1e-3), (2, 1e-6), (8, 1e-2), (16, 1e-8),
                                       (32, 1e-8), (64, 1.0), (128, 1e-5), (256, 1e-3), (1024, 1e-6),
                                       (4096, 1e-2)])
def test_backward_matches_oracle(ag, orc, block, eps):
    import torch
    x, y = workloads.pair("b", 20011, 77)
    xt, yt = _dev(x), _dev(y)
    z = ag.qdot_fn(xt, yt, eps=eps, block=block)
    g = -1.75
    z.backward(torch.tensor(g, dtype=torch.float64, device="cuda"))
    ref = orc.qdot(x, y, eps=eps, block=block, explain=True)
    gx, gy = orc.backward(x, y, ref.cls, g)
    np.testing.assert_array_equal(_bits(xt.grad.cpu().numpy()), _bits(gx))
    np.testing.assert_array_equal(_bits(yt.grad.cpu().numpy()), _bits(gy))


@pytest.mark.parametrize("block", [0, 4, 32, 512])
def test_backward_unaligned_and_one_sided(ag, orc, block):
    import torch
    x, y = workloads.pair("c", 9001, 78)
    xs = torch.from_numpy(np.concatenate([[0.0], x])).cuda()[1:].requires_grad_(True)  # 8-byte aligned only
    yt = _dev(y, grad=False)
    z = ag.qdot_fn(xs, yt, eps=1e-6, block=block)
    z.backward(torch.tensor(3.0, dtype=torch.float64, device="cuda"))
    ref = orc.qdot(x, y, eps=1e-6, block=block, explain=True)
    gx, _ = orc.backward(x, y, ref.cls, 3.0)
    np.testing.assert_array_equal(_bits(xs.grad.cpu().numpy()), _bits(gx))
    assert yt.grad is None


def test_backward_edge_cases(ag, orc):
    import torch
    # all-zero x: every component ZERO, gradients zero
    x = np.zeros(1000)
    y = workloads.vector("a", 1000, 5)
    xt, yt = _dev(x), _dev(y)
    ag.qdot_fn(xt, yt, eps=1e-8, block=32).backward()
    assert not xt.grad.cpu().numpy().any() and not yt.grad.cpu().numpy().any()
    # subnormal and huge components, single-element and tail-only inputs
    for n in (1, 7, 255, 257):
        rng = np.random.default_rng(n)
        x = rng.choice([1e-310, -3e-320, 1.7e308, -1.0, 0.5, 0.0], n)
        y = rng.choice([2.0, -1e-300, 1e-5, 3e300, 0.0], n)
        for block in (0, 1, 32):
            xt, yt = _dev(x), _dev(y)
            ag.qdot_fn(xt, yt, eps=1e-3, block=block).backward()
            ref = orc.qdot(x, y, eps=1e-3, block=block, explain=True)
            gx, gy = orc.backward(x, y, ref.cls, 1.0)
            np.testing.assert_array_equal(_bits(xt.grad.cpu().numpy()), _bits(gx))
            np.testing.assert_array_equal(_bits(yt.grad.cpu().numpy()), _bits(gy))


def _rows(B, L, seed):
    rng = np.random.default_rng(seed)
    X = np.empty((B, L))
    Y = np.empty((B, L))
    for b in range(B):
        X[b], Y[b] = workloads.pair("b", L, int(rng.integers(1 << 30)))
    return X, Y


@pytest.mark.parametrize("block", [32, 64, 256])
def test_batched_backward_matches_oracle(ag, orc, block):
    """Rows of 4098 components: every row 16-byte aligned (the batched forward
    requires it), a ragged last item of 2 components."""
    import torch
    X, Y = _rows(24, 4098, 91)
    Xt, Yt = _dev(X), _dev(Y)
    z = ag.qdot_batch_fn(Xt, Yt, eps=1e-8, block=block)
    (z * z).sum().backward()
    zc = z.detach().cpu().numpy()
    GX, GY = Xt.grad.cpu().numpy(), Yt.grad.cpu().numpy()
    for b in range(X.shape[0]):
        ref = orc.qdot(X[b], Y[b], eps=1e-8, block=block, explain=True)
        assert abs(zc[b] - ref.value) <= 1e-13 * orc.abs_dot_exact(X[b], Y[b])
        gx, gy = orc.backward(X[b], Y[b], ref.cls, 2.0 * zc[b])
        np.testing.assert_array_equal(_bits(GX[b]), _bits(gx))
        np.testing.assert_array_equal(_bits(GY[b]), _bits(gy))


def test_batched_autograd_full_size(ag, orc):
    """1024 pairs of length 2^16, loss sum_b qdot(x_b, y_b)^2: sampled rows
    against the oracle gradient, finite differences on double-class components."""
    import torch
    Bn, L = 1024, 1 << 16
    gen = torch.Generator(device="cuda").manual_seed(2105)
    # distribution (b): lognormal sigma = 4 with random sign, generated on the device
    def lognormal():
        m = torch.randn(Bn, L, generator=gen, device="cuda", dtype=torch.float64) * 4.0
        s = torch.randint(0, 2, (Bn, L), generator=gen, device="cuda").to(torch.float64) * 2 - 1
        return torch.exp(m) * s
    Xt = lognormal().requires_grad_(True)
    Yt = lognormal().requires_grad_(True)
    eps = 1e-8
    z = ag.qdot_batch_fn(Xt, Yt, eps=eps, block=32)
    (z * z).sum().backward()
    zc = z.detach().cpu().numpy()
    for b in (0, 1, 511, 1023):
        x = Xt[b].detach().cpu().numpy()
        y = Yt[b].detach().cpu().numpy()
        ref = orc.qdot(x, y, eps=eps, block=32, explain=True)
        assert abs(zc[b] - ref.value) <= 1e-13 * orc.abs_dot_exact(x, y)
        gx, gy = orc.backward(x, y, ref.cls, 2.0 * zc[b])
        np.testing.assert_array_equal(_bits(Xt.grad[b].cpu().numpy()), _bits(gx))
        np.testing.assert_array_equal(_bits(Yt.grad[b].cpu().numpy()), _bits(gy))
    # central differences of the loss through the GPU forward, step 1e-7
    # relative to |x_i| (an absolute 1e-7 is lost below the rounding of sums
    # of lognormal products), on the double-class components with the largest
    # products (the best-conditioned differences)
    b = 3
    x = Xt[b].detach().cpu().numpy()
    y = Yt[b].detach().cpu().numpy()
    ref = orc.qdot(x, y, eps=eps, block=32, explain=True)
    dbl = np.nonzero(ref.cls == 3)[0]
    dbl = dbl[np.argsort(-np.abs(x[dbl] * y[dbl]))][:20]
    checked = 0
    for i in dbl:
        vals = []
        steps = []
        for s in (+1, -1):
            xp = x.copy()
            xp[i] += s * 1e-7 * abs(x[i])
            steps.append(xp[i])
            if not np.array_equal(orc.qdot(xp, y, eps=eps, block=32, explain=True).cls, ref.cls):
                break  # the perturbation moved the class map; not a point of differentiability
            zp = ag.qdot_batch_fn(torch.from_numpy(xp).cuda()[None, :], Yt[b].detach()[None, :], eps=eps,
                                  block=32).item()
            vals.append(zp * zp)
        if len(vals) < 2:
            continue
        fd = (vals[0] - vals[1]) / (steps[0] - steps[1])
        assert fd == pytest.approx(float(Xt.grad[b, i]), rel=1e-6)
        checked += 1
        if checked == 6:
            break
    assert checked >= 3
