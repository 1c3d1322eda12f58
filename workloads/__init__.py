"""Seeded synthetic inputs for qdot, shared by the GPU path and the oracle.

This module holds no arithmetic of the method: it only draws vectors and
builds sparse matrices.  Every generator takes an integer seed and returns
numpy arrays, so both sides of a comparison consume the very same bytes.

Recipes (value distributions follow the workloads the paper and the
benchmark configuration describe):

* ``config0_pair``: x_i = s * 10**U(-8, 0) with an independent fair sign s.
* ``pair('a')``: U[-1, 1].
* ``pair('b')``: s * exp(4 * N(0, 1)) (lognormal, sigma = 4) with a fair sign.
* ``pair('c')``: U[-1, 1] with each entry, independently with probability
  0.01, multiplied by 1e6 (heavy outliers).
* ``paper_A`` / ``paper_B``: the paper's Sec. 4.1 distributions
  s * 2**p with s ~ U[0.5, 1) and p ~ U[-t/2, t/2] (A) or p ~ N(0, t/2) (B).
* ``batched_lengths``: floor(2**U(8, 20)) pair lengths (log-uniform).
* ``poisson3d`` / ``poisson2d``: SPD variable-coefficient 7-point / 5-point
  operators, coefficient 10**U(-3, 3) per cell, harmonic-mean face
  coefficients, Dirichlet boundary faces adding c_i to the diagonal.
* ``stencil27``: the SPD 27-point operator of the paper's ACG problems (Sec.
  4.2, the HPCCG "chimney" boxes nx x ny x nz): 27 on the diagonal, -1 for
  every grid neighbour within one step along each axis, with
  ``ones_rhs`` = A times the all-ones vector (so x = 1 solves it).
* ``graph_laplacian``: L = D - W of a seeded random undirected graph (every
  vertex draws ``degree`` partners uniformly, unit weights, the edge set
  symmetrised), the stand-in for the paper's random graph Laplacians of
  Sec. 4.3.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_CHUNK = 1 << 22


def _chunked(n: int, seed: int, draw) -> np.ndarray:
    """Fill an n-vector chunk by chunk; chunk k draws from its own stream spawned
    from ``seed`` so the result does not depend on the thread count."""
    out = np.empty(n, dtype=np.float64)
    nchunks = (n + _CHUNK - 1) // _CHUNK
    seqs = np.random.SeedSequence(seed).spawn(max(nchunks, 1))

    def work(k):
        lo, hi = k * _CHUNK, min(n, (k + 1) * _CHUNK)
        out[lo:hi] = draw(np.random.default_rng(seqs[k]), hi - lo)

    if nchunks <= 1:
        if n:
            work(0)
    else:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(work, range(nchunks)))
    return out


def _signs(rng, m):
    return np.where(rng.random(m) < 0.5, -1.0, 1.0)


def vector(kind: str, n: int, seed: int) -> np.ndarray:
    """One length-n vector of distribution ``kind`` ('a', 'b', 'c', 'cfg0')."""
    if kind == "a":
        return _chunked(n, seed, lambda rng, m: rng.uniform(-1.0, 1.0, m))
    if kind == "b":
        return _chunked(n, seed, lambda rng, m: _signs(rng, m) * np.exp(4.0 * rng.standard_normal(m)))
    if kind == "c":
        def draw(rng, m):
            v = rng.uniform(-1.0, 1.0, m)
            v[rng.random(m) < 0.01] *= 1e6
            return v
        return _chunked(n, seed, draw)
    if kind == "cfg0":
        return _chunked(n, seed, lambda rng, m: _signs(rng, m) * 10.0 ** rng.uniform(-8.0, 0.0, m))
    raise ValueError(f"unknown distribution {kind!r}")


def pair(kind: str, n: int, seed: int):
    """(x, y): two independent vectors of distribution ``kind``."""
    return vector(kind, n, 2 * seed + 1), vector(kind, n, 2 * seed + 2)


def config0_pair(n: int = 65536, seed: int = 2105):
    return pair("cfg0", n, seed)


def paper_A(n: int, t: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.5, 1.0, n)
    p = rng.uniform(-0.5 * t, 0.5 * t, n)
    return s * np.exp2(p)


def paper_B(n: int, t: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.5, 1.0, n)
    p = rng.normal(0.0, 0.5 * t, n)
    return s * np.exp2(p)


def batched_lengths(count: int = 4096, seed: int = 2107, lo_log2: float = 8.0, hi_log2: float = 20.0):
    rng = np.random.default_rng(seed)
    return np.floor(np.exp2(rng.uniform(lo_log2, hi_log2, count))).astype(np.int64)


def _assemble(c: np.ndarray, shape: tuple[int, ...]):
    """CSR of the variable-coefficient finite-volume Laplacian on a box grid
    (lexicographic order, first axis fastest), sorted column indices."""
    dims = len(shape)
    c = c.reshape(shape[::-1])  # c[z, y, x] (or c[y, x]); x is the fastest axis
    n = c.size
    idx = np.arange(n, dtype=np.int64).reshape(c.shape)
    diag = np.zeros(c.shape)
    offs = []  # (neighbour index array, coefficient array, valid mask) per direction
    for axis in range(dims):
        for step in (-1, 1):
            nb_c = np.roll(c, -step, axis=axis)
            nb_i = np.roll(idx, -step, axis=axis)
            valid = np.ones(c.shape, dtype=bool)
            sl = [slice(None)] * dims
            sl[axis] = slice(-1, None) if step == 1 else slice(0, 1)
            valid[tuple(sl)] = False
            face = np.where(valid, 2.0 * c * nb_c / (c + nb_c), c)
            diag += face
            offs.append((nb_i, -face, valid))
    # entries per row in ascending column order: axis order reversed (slowest first)
    cols, vals, masks = [], [], []
    neg = [offs[2 * a] for a in range(dims)]              # step -1, slowest axis first
    pos = [offs[2 * a + 1] for a in range(dims)][::-1]    # step +1, fastest axis first
    for nb_i, v, m in neg:
        cols.append(nb_i); vals.append(v); masks.append(m)
    cols.append(idx); vals.append(diag); masks.append(np.ones(c.shape, dtype=bool))
    for nb_i, v, m in pos:
        cols.append(nb_i); vals.append(v); masks.append(m)
    C = np.stack([a.reshape(-1) for a in cols], axis=1)
    V = np.stack([a.reshape(-1) for a in vals], axis=1)
    Mk = np.stack([a.reshape(-1) for a in masks], axis=1)
    counts = Mk.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = C[Mk].astype(np.int32)
    val = V[Mk].astype(np.float64)
    return rowptr, col, val


def coefficients(ncell: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-3.0, 3.0, ncell)


def poisson3d(nx: int, ny: int, nz: int, seed: int = 2108):
    """7-point SPD operator on an nx x ny x nz grid: (rowptr int64, col int32, val f64)."""
    return _assemble(coefficients(nx * ny * nz, seed), (nx, ny, nz))


def laplace3d(nx: int, ny: int, nz: int):
    """Constant-coefficient 7-point operator (every cell coefficient 1)."""
    return _assemble(np.ones(nx * ny * nz), (nx, ny, nz))


def poisson2d(nx: int, ny: int, seed: int = 2109):
    """5-point SPD operator on an nx x ny grid."""
    return _assemble(coefficients(nx * ny, seed), (nx, ny))


def rhs(n: int, seed: int = 2110) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def unit_start(n: int, seed: int = 2111) -> np.ndarray:
    v = np.random.default_rng(seed).uniform(-1.0, 1.0, n)
    return v / np.sqrt(np.dot(v, v))


def block_diagonal(blocks):
    """One CSR matrix with the given (rowptr, col, val) blocks on its diagonal;
    returns (rowptr, col, val, row_off)."""
    rps, cols, vals, offs = [np.zeros(1, dtype=np.int64)], [], [], [0]
    nnz = 0
    for rp, col, val in blocks:
        n = rp.shape[0] - 1
        rps.append(rp[1:] + nnz)
        cols.append(col.astype(np.int64) + offs[-1])
        vals.append(val)
        nnz += int(rp[-1])
        offs.append(offs[-1] + n)
    return (np.concatenate(rps), np.concatenate(cols).astype(np.int32), np.concatenate(vals),
            np.array(offs, dtype=np.int64))


def batched_cg_systems(count: int = 256, lo: int = 16, hi: int = 64, seed: int = 2112):
    """`count` variable-coefficient 7-point systems on cubic grids with edges
    uniform in [lo, hi], block-diagonal; returns (rowptr, col, val, row_off, edges)."""
    rng = np.random.default_rng(seed)
    edges = rng.integers(lo, hi + 1, count)
    blocks = [poisson3d(int(e), int(e), int(e), seed=seed + 1 + i) for i, e in enumerate(edges)]
    return (*block_diagonal(blocks), edges)


def exponent_dist(kind: str, n: int, t: float, seed: int, device="cuda"):
    """The paper's synthetic arrays (Sec. 4.1): components s * 2^p with
    s ~ U[0.5, 1) and p ~ U[-t/2, t/2] (kind 'A') or p ~ N(0, t/2) (kind 'B'),
    drawn on `device` from a seeded torch generator; float64."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    s = torch.rand(n, generator=g, device=device, dtype=torch.float64) * 0.5 + 0.5
    if kind == "A":
        p = (torch.rand(n, generator=g, device=device, dtype=torch.float64) - 0.5) * t
    elif kind == "B":
        p = torch.randn(n, generator=g, device=device, dtype=torch.float64) * (0.5 * t)
    else:
        raise ValueError(kind)
    return s * torch.exp2(p)


def stencil27(nx: int, ny: int, nz: int):
    """27-point operator on an nx x ny x nz box (lexicographic order, x
    fastest): row i has 27 on the diagonal and -1 for each grid point within
    one step of it along every axis; CSR (rowptr int64, col int32, val f64),
    columns ascending.  Strictly diagonally dominant, so SPD.  Built one z
    plane at a time so the 10^7-row boxes stay within a few GB."""
    n = nx * ny * nz
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # ascending columns
    ix = np.tile(np.arange(nx, dtype=np.int64), ny)
    iy = np.repeat(np.arange(ny, dtype=np.int64), nx)
    plane = nx * ny
    cols, vals, counts = [], [], []
    for z in range(nz):
        base = z * plane + iy * nx + ix
        cm, vm, km = [], [], []
        for dz, dy, dx in offs:
            ok = (0 <= ix + dx) & (ix + dx < nx) & (0 <= iy + dy) & (iy + dy < ny) & (0 <= z + dz) & (z + dz < nz)
            cm.append(np.where(ok, base + dx + nx * dy + plane * dz, -1))
            km.append(ok)
            vm.append(27.0 if (dz, dy, dx) == (0, 0, 0) else -1.0)
        C = np.stack(cm, axis=1)
        K = np.stack(km, axis=1)
        V = np.broadcast_to(np.array(vm), C.shape)
        cols.append(C[K].astype(np.int32))
        vals.append(V[K].astype(np.float64))
        counts.append(K.sum(axis=1))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.concatenate(counts), out=rowptr[1:])
    return rowptr, np.concatenate(cols), np.concatenate(vals)


def ones_rhs(rowptr, col, val) -> np.ndarray:
    """b = A 1 (row sums, summed exactly as integers for the 27-point
    operator's integer entries)."""
    sums = np.add.reduceat(val, rowptr[:-1]) if val.size else np.zeros(rowptr.shape[0] - 1)
    sums[rowptr[1:] == rowptr[:-1]] = 0.0
    return sums


def graph_laplacian(n: int, degree: int = 8, seed: int = 2113):
    """L = D - W of a random undirected graph on n vertices: each vertex draws
    `degree` partners uniformly (self loops dropped), every drawn edge is
    made symmetric, weights are 1 (repeated draws count once).  CSR (rowptr
    int64, col int32, val f64), columns ascending.  Symmetric, positive
    semi-definite, rows sum to 0."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(n, dtype=np.int64), degree)
    dst = rng.integers(0, n, src.shape[0])
    keep = src != dst
    src, dst = src[keep], dst[keep]
    W = sp.coo_matrix((np.ones(src.shape[0]), (src, dst)), shape=(n, n)).tocsr()
    W = ((W + W.T) > 0).astype(np.float64)
    deg = np.asarray(W.sum(axis=1)).ravel()
    L = (sp.diags(deg) - W).tocsr()
    L.sort_indices()
    return L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64)
