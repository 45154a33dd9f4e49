"""Seeded synthetic inputs for the interior-SVD workloads.

This module only builds inputs: sparse matrices, seed blocks and intervals.
It holds none of the contour-integral method's arithmetic. The CUDA path and
the CPU oracle both draw their inputs from here, so that they see the same
numbers.

Workload shapes follow the paper's experiments (Sec. 4) and the configured
synthetic stand-ins:

* ``random_sparse``     -- m x n CSR, k distinct uniform-random columns per
                           row, N(0,1) values (the 2000 x 1000 case).
* ``block_permuted``    -- dense blocks on a block diagonal with random row and
                           column permutations; its spectrum is the union of
                           the blocks' spectra, so it is known exactly.
* ``banded_random``     -- m x n CSR with k_band columns near the row's diagonal
                           position and k_rand uniform-random columns per row,
                           U(-1,1) values rounded to bf16 (the 2e6 x 1e6
                           mixed-precision case).
* ``model_problem``     -- the Experiment II model problems
                           A = U diag(sigma) V^T, m = 1000, n = 200 (Sec. 4.2).
* ``gaussian_block``    -- the real Gaussian input block V_in (n x L).
* ``window_interval``   -- an interval [a, b] whose endpoints sit at gap
                           midpoints of a known descending spectrum.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A real sparse matrix in compressed-sparse-row form.

    rowptr: int64[m+1], colidx: int32[nnz] (strictly increasing per row),
    vals: float64[nnz].
    """

    m: int
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        d[rows, self.colidx] = self.vals
        return d


def csr_from_coo(m: int, n: int, rows, cols, vals) -> CSR:
    """Sort COO triplets by (row, col) and compress. Duplicates are rejected."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate (row, col) entries")
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(m, n, rowptr, cols.astype(np.int32), vals)


def csr_from_dense(d: np.ndarray) -> CSR:
    """Every entry of a dense matrix stored explicitly (zeros included)."""
    m, n = d.shape
    rowptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    colidx = np.tile(np.arange(n, dtype=np.int32), m)
    return CSR(m, n, rowptr, colidx, np.ascontiguousarray(d, dtype=np.float64).ravel())


def transpose(A: CSR) -> CSR:
    rows = np.repeat(np.arange(A.m, dtype=np.int64), np.diff(A.rowptr))
    return csr_from_coo(A.n, A.m, A.colidx, rows, A.vals)


def _distinct_columns(rng: np.random.Generator, m: int, n: int, k: int) -> np.ndarray:
    """k distinct columns per row, uniform without replacement, sorted."""
    if k > n:
        raise ValueError("k > n")
    cols = np.sort(rng.integers(0, n, size=(m, k)), axis=1)
    while True:
        bad = np.nonzero((np.diff(cols, axis=1) == 0).any(axis=1))[0]
        if bad.size == 0:
            return cols
        cols[bad] = np.sort(rng.integers(0, n, size=(bad.size, k)), axis=1)


def random_sparse(m: int = 2000, n: int = 1000, k: int = 8, seed: int = 0) -> CSR:
    """m x n CSR with k distinct uniform-random columns per row, N(0,1) values."""
    rng = np.random.default_rng(seed)
    cols = _distinct_columns(rng, m, n, k)
    vals = rng.standard_normal(m * k)
    rowptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    return CSR(m, n, rowptr, cols.ravel().astype(np.int32), vals)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16-representable value (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@dataclass
class BlockPermuted:
    """A block-diagonal matrix hidden by random row/column permutations.

    Block b occupies rows row_perm[b*bm:(b+1)*bm] and columns
    col_perm[b*bn:(b+1)*bn]; ``blocks[b]`` holds its dense values.
    """

    A: CSR
    blocks: np.ndarray      # (nb, bm, bn)
    row_perm: np.ndarray    # (nb*bm,)
    col_perm: np.ndarray    # (nb*bn,)

    def block_sigmas(self) -> np.ndarray:
        """Singular values of every block, shape (nb, min(bm, bn)), descending.

        The matrix's spectrum is the union of these values (the permutations
        are orthogonal), which is what makes the construction's spectrum known.
        """
        return np.linalg.svd(self.blocks, compute_uv=False)

    def sigmas_desc(self) -> np.ndarray:
        return np.sort(self.block_sigmas().ravel())[::-1]


def block_permuted(nb: int, bm: int, bn: int, seed: int, dist: str = "normal") -> BlockPermuted:
    """nb dense bm x bn blocks, permuted. dist: 'normal' N(0,1) or 'uniform_bf16'
    U(-1,1) rounded to bf16-representable values."""
    rng = np.random.default_rng(seed)
    if dist == "normal":
        blocks = rng.standard_normal((nb, bm, bn))
    elif dist == "uniform_bf16":
        blocks = bf16_round(rng.uniform(-1.0, 1.0, size=(nb, bm, bn)))
    else:
        raise ValueError(dist)
    row_perm = rng.permutation(nb * bm)
    col_perm = rng.permutation(nb * bn)
    bi, ii, jj = np.meshgrid(np.arange(nb), np.arange(bm), np.arange(bn), indexing="ij")
    rows = row_perm[bi * bm + ii].ravel()
    cols = col_perm[bi * bn + jj].ravel()
    A = csr_from_coo(nb * bm, nb * bn, rows, cols, blocks.ravel())
    return BlockPermuted(A, blocks, row_perm, col_perm)


def banded_random(m: int = 2_000_000, n: int = 1_000_000, k_band: int = 8, k_rand: int = 8,
                  half_width: int = 5000, seed: int = 10) -> CSR:
    """m x n CSR with k_band + k_rand distinct columns per row (the 2e6 x 1e6 case).

    Row i's "band" columns are uniform in [c_i - half_width, c_i + half_width] clipped to
    [0, n), with c_i = floor(i n / m); its other k_rand columns are uniform over [0, n).
    A row whose draws collide is drawn again as a whole. Values are U(-1, 1) rounded to
    bf16-representable numbers, so FP64, FP32 and bf16 storage hold the same matrix.
    """
    rng = np.random.default_rng(seed)
    k = k_band + k_rand
    c = (np.arange(m, dtype=np.int64) * n) // m
    lo = np.maximum(c - half_width, 0)
    width = np.minimum(c + half_width, n - 1) - lo + 1

    def draw(rows):
        cols = np.empty((rows.size, k), dtype=np.int64)
        cols[:, :k_band] = lo[rows, None] + (rng.random((rows.size, k_band)) * width[rows, None]).astype(np.int64)
        cols[:, k_band:] = rng.integers(0, n, size=(rows.size, k_rand))
        cols.sort(axis=1)
        return cols

    cols = draw(np.arange(m))
    while True:
        bad = np.nonzero((np.diff(cols, axis=1) == 0).any(axis=1))[0]
        if bad.size == 0:
            break
        cols[bad] = draw(bad)
    vals = bf16_round(rng.uniform(-1.0, 1.0, size=m * k))
    rowptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    return CSR(m, n, rowptr, cols.ravel().astype(np.int32), vals)


def _haar_orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((rows, cols)))
    return q * np.sign(np.diag(r))


def model_problem(which: int, m: int = 1000, n: int = 200, seed: int = 7):
    """Experiment II (Sec. 4.2): A = U diag(sigma) V^T with random orthogonal U, V.

    which=1: sigma = 0.005, 0.015, ..., 1.995 (uniform, Eq. model1).
    which=2: sigma = 10^-10.0, 10^-9.95, ..., 10^-0.05 (log-uniform, Eq. model2).
    Returns (dense A, sigma ascending).
    """
    rng = np.random.default_rng(seed)
    if which == 1:
        sig = 0.005 + 0.01 * np.arange(n)
    elif which == 2:
        sig = 10.0 ** (-10.0 + 0.05 * np.arange(n))
    else:
        raise ValueError(which)
    U = _haar_orthonormal(rng, m, n)
    V = _haar_orthonormal(rng, n, n)
    return (U * sig) @ V.T, sig


def gaussian_block(n: int, L: int, seed: int) -> np.ndarray:
    """Real N(0,1) input block V_in, n x L, row-major float64."""
    return np.random.default_rng(seed).standard_normal((n, L))


def window_interval(sig_desc: np.ndarray, first: int, count: int,
                    min_rel_gap: float = 0.0, max_shift: int = 0):
    """Interval holding sig_desc[first:first+count] (0-based, descending order).

    a and b are the midpoints of the gaps just outside the window. With
    min_rel_gap > 0 the window start moves by at most max_shift positions
    (nearest first) until both bounding gaps are >= min_rel_gap * sigma.
    Returns (a, b, first).
    """
    s = np.asarray(sig_desc, dtype=np.float64)
    for d in sorted(range(-max_shift, max_shift + 1), key=lambda x: (abs(x), x)):
        f = first + d
        if f < 1 or f + count >= s.size:
            continue
        hi_gap = s[f - 1] - s[f]
        lo_gap = s[f + count - 1] - s[f + count]
        if hi_gap >= min_rel_gap * s[f - 1] and lo_gap >= min_rel_gap * s[f + count - 1]:
            b = 0.5 * (s[f - 1] + s[f])
            a = 0.5 * (s[f + count - 1] + s[f + count])
            return float(a), float(b), f
    raise ValueError("no window with the requested gaps")


def digits_like(m: int = 60000, side: int = 28, classes: int = 10, nnz_row: float = 150.0, seed: int = 8) -> CSR:
    """A stand-in with the shape of the Experiment III matrix (Sec. 4.3: 60000 x 784 images of
    handwritten digits, 149.9 nonzeros per row on average, nonnegative, scaled to ||A||_2 = 1).

    Columns are the pixels of a side x side grid. Each class has a prototype of six Gaussian
    strokes in the central 16 x 16 pixels. A row is one "drawing" of its class: every stroke
    is moved by N(0, 1.5^2) pixels, its widths are scaled by exp(N(0, 0.15^2)) and its
    amplitude drawn from U(0.6, 1). The row keeps its K brightest pixels, with
    K = round(nnz_row exp(N(0, 0.2^2))) clipped to [60, 300]. The values are the intensities
    relative to the row's maximum, quantized to k/255 with k >= 1. Smooth deformations of a
    few prototypes give a spectrum that decays like that of real digit images. The matrix is
    divided by its largest singular value. That value is found by 40 steps of power iteration
    on A^T A; the matrix is nonnegative, so the top value is simple and well separated.
    """
    rng = np.random.default_rng(seed)
    n = side * side
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    yy, xx = yy.ravel(), xx.ravel()
    ctr = (side - 1) / 2.0
    ns = 6
    proto = np.empty((classes, ns, 4))                      # cy, cx, sy, sx
    proto[:, :, 0:2] = rng.uniform(ctr - 8.0, ctr + 8.0, size=(classes, ns, 2))
    proto[:, :, 2:4] = rng.uniform(1.2, 3.5, size=(classes, ns, 2))
    labels = rng.integers(0, classes, size=m)
    K = np.clip(np.rint(nnz_row * np.exp(0.2 * rng.standard_normal(m))), 60, 300).astype(np.int64)
    rows_l, cols_l, vals_l = [], [], []
    chunk = 4096
    for r0 in range(0, m, chunk):
        r1 = min(m, r0 + chunk)
        st = proto[labels[r0:r1]].copy()                      # (c, ns, 4)
        st[:, :, 0:2] += 1.5 * rng.standard_normal((r1 - r0, ns, 2))
        st[:, :, 2:4] *= np.exp(0.15 * rng.standard_normal((r1 - r0, ns, 2)))
        amp = rng.uniform(0.6, 1.0, size=(r1 - r0, ns))
        img = np.zeros((r1 - r0, n))
        for k in range(ns):
            dy = (yy[None, :] - st[:, k, 0:1]) / st[:, k, 2:3]
            dx = (xx[None, :] - st[:, k, 1:2]) / st[:, k, 3:4]
            img += amp[:, k:k + 1] * np.exp(-0.5 * (dy * dy + dx * dx))
        srt = -np.sort(-img, axis=1)
        thr = srt[np.arange(r1 - r0), K[r0:r1] - 1]
        keep = img >= thr[:, None]
        q = np.maximum(1.0, np.rint(255.0 * img / srt[:, :1])) / 255.0
        rr, cc = np.nonzero(keep)
        rows_l.append(rr + r0)
        cols_l.append(cc)
        vals_l.append(q[rr, cc])
    A = csr_from_coo(m, n, np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(vals_l))
    # ||A||_2 by power iteration on A^T A (sparse products written out with numpy)
    rr = np.repeat(np.arange(m), np.diff(A.rowptr))
    x = np.ones(n) / np.sqrt(n)
    lam = 0.0
    for _ in range(40):
        y = np.bincount(rr, weights=A.vals * x[A.colidx], minlength=m)
        z = np.bincount(A.colidx, weights=A.vals * y[rr], minlength=n)
        lam = float(np.linalg.norm(z))
        x = z / lam
    A.vals = A.vals / np.sqrt(lam)
    return A


def batched_problems(count: int = 64, seed: int = 4, n_min: int = 2000, n_max: int = 80000):
    """Many independent problems of the block-permuted kind (10 x 4 N(0,1) blocks, m = 2.5 n).

    n_i = 4 round(exp(U(ln n_min, ln n_max)) / 4). L_i is drawn from {16, 32}, N = 32 and
    M = 4. (With N = 16 the oracle saturates the L M = 128 subspace on exterior windows and
    finds none of their values: the 16-point filter decays too slowly below a.) t0 = floor(L M / 3) (L M ~ 3 t, as in Sec. 4.3). Every second problem is exterior:
    b = 1.01 sigma_max, and a sits at the midpoint of the widest relative gap below the t-th
    largest value, t within t0 +- 10. The others are interior: a window of t0 values at a
    uniform position, moved by at most 10 places to the position whose two bounding gaps have
    the widest smaller relative gap. An endpoint close to a singular value leaves that value's
    filter near 1/2 (Sec. 4, Exp I). With N = 16 that saturates the L M subspace, and the
    oracle itself then finds nothing. Returns a list of dicts with keys A, sigma (descending),
    a, b, t, N, L, M, kind, seed_v (the seed of V_in).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(4 * round(np.exp(rng.uniform(np.log(n_min), np.log(n_max))) / 4))
        rng.choice([16, 32])                        # (former N draw, kept so the stream stays aligned)
        N = 32
        L = int(rng.choice([16, 32]))
        M = 4
        t0 = (L * M) // 3
        bp = block_permuted(n // 4, 10, 4, seed=int(rng.integers(1 << 30)))
        s = bp.sigmas_desc()
        rel_gap = (s[:-1] - s[1:]) / s[1:]          # gap below s[k], relative
        if i % 2 == 0:
            t = max(range(t0 - 10, t0 + 11), key=lambda k: (rel_gap[k - 1], -abs(k - t0)))
            a, b, kind = 0.5 * (s[t - 1] + s[t]), 1.01 * float(s[0]), "exterior"
        else:
            t = t0
            first0 = int(rng.integers(t + 20, s.size - 2 * t - 20))
            first = max(range(first0 - 10, first0 + 11),
                        key=lambda f: (min(rel_gap[f - 1], rel_gap[f + t - 1]), -abs(f - first0)))
            a, b = 0.5 * (s[first + t - 1] + s[first + t]), 0.5 * (s[first - 1] + s[first])
            kind = "interior"
        out.append(dict(A=bp.A, sigma=s, a=float(a), b=float(b), t=t, N=N, L=L, M=M, kind=kind, seed_v=1000 + i))
    return out
