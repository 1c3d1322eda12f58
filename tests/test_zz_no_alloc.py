"""The workspace-free entry point qdot_static_scratch(), for callers that
cannot allocate device memory (the host application owns the allocator, or
allocation after start-up is not allowed).  It must give what qdot() gives,
call after call, while reusing the library's fixed scratch array.

Kept in a file of its own that runs last.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_00115_gb300 import build as qbuild
    qbuild.build()
    import paper_2105_00115_gb300 as q
    return torch, q, q.load()


def _static_call(torch, q, lib, xd, yd, eps, block):
    p = q.params(eps, block, 1, 0, "auto")
    out = torch.empty(80, dtype=torch.uint8, device="cuda")
    st = lib.qdot_static_scratch(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), xd.numel(),
                                 ctypes.byref(p), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.qdot_last_error()
    return q.decode_result(out.cpu().numpy())


def test_static_scratch_matches_qdot_twice_in_a_row(env, orc):
    torch, q, lib = env
    cases = [("b", 300007, 1e-8, 32), ("c", 150001, 1e-3, 0), ("a", 200000, 1e-12, 1), ("b", 70001, 0.5, 256)]
    for kind, n, eps, block in cases:
        x, y = workloads.pair(kind, n, 900 + n)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ref = q.qdot(xd, yd, eps=eps, block=block)
        tol = TOL * orc.abs_dot_exact(x, y)
        for _ in range(2):  # two calls in a row on the shared scratch
            r = _static_call(torch, q, lib, xd, yd, eps, block)
            assert r.status == 0
            assert r.count == ref.count
            assert (r.e_max, r.e_min, r.n_bins, r.f) == (ref.e_max, ref.e_min, ref.n_bins, ref.f)
            assert abs(r.value - ref.value) <= tol


def test_static_scratch_eight_byte_aligned_inputs(env, orc):
    """Inputs that are only 8-byte aligned take the 64-bit load variant; blocks
    of 64 then keep per-block keys in the scratch (2 bytes per block), which
    still fits at this size."""
    torch, q, lib = env
    x, y = workloads.pair("b", 200001, 77)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    xs, ys = xd[1:], yd[1:]
    assert xs.data_ptr() % 16 == 8
    tol = TOL * orc.abs_dot_exact(x[1:], y[1:])
    for block in (32, 64, 0):
        ref = q.qdot(xs, ys, eps=1e-8, block=block)
        for _ in range(2):
            r = _static_call(torch, q, lib, xs, ys, 1e-8, block)
            assert r.count == ref.count and r.n_bins == ref.n_bins
            assert abs(r.value - ref.value) <= tol


def test_static_scratch_rejects_arguments_that_do_not_fit(env):
    torch, q, lib = env
    x = torch.ones(16, dtype=torch.float64, device="cuda")
    p = q.params(1e-8, 128, 1, 0, "auto")
    out = torch.empty(80, dtype=torch.uint8, device="cuda")
    # blocks of 128 keep 2 bytes per block: 2^30 components need 16 MiB (checked before any launch)
    st = lib.qdot_static_scratch(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1 << 30,
                                 ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), None)
    assert st == 5 and b"scratch" in lib.qdot_last_error()
    bad = q.params(-1.0, 32, 1, 0, "auto")
    st = lib.qdot_static_scratch(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 16,
                                 ctypes.byref(bad), ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
