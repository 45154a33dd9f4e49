"""GPU parity of the SpMM variants (row a3): FP32 and double-float products, bf16 and FP32
storage of A, the autotuner, and the 2e6 x 1e6 banded-plus-random matrix at full size.

Reference: the product computed on the host in extended precision (numpy longdouble), so
that its own rounding is far below the bounds tested.

Bounds, for a row with k nonzeros and s = sum_j |a_ij| |x_j|:
* double-float (cmsvd_spmm_df): x = x_hi + x_lo and a = a_hi + a_lo carry 2^-48 relative
  each; a_hi x_hi is exact (two_prod); the cross terms are rounded at 2^-24 of a 2^-23
  quantity; the high sum is exact (two_sum); the low accumulator holds at most
  (k + 4) 2^-24 s and rounds at 2^-24 of that per addition. Together
  |y - A x| <= (k (k + 4) + 8) 2^-48 s.
* FP32: (k + 2) 2^-24 s (FP32-rounded operands and k rounded multiply-adds).
"""
import numpy as np
import pytest

from paper_2109_13655_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U48 = 2.0 ** -48
U24 = 2.0 ** -24


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_13655_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context()
    yield c
    c.close()


def ragged(m, n, seed, values="normal"):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(m):
        k = int(rng.integers(0, 18))
        c = np.sort(rng.choice(n, size=min(k, n), replace=False))
        rows += [i] * c.size
        cols += list(c)
    v = rng.standard_normal(len(rows))
    if values == "bf16":
        v = synth.bf16_round(rng.uniform(-1, 1, len(rows)))
    return synth.csr_from_coo(m, n, rows, cols, v)


def split(X):
    """x -> (hi, lo) FP32 with hi = fl32(x), lo = fl32(x - hi); rows [hi | lo]."""
    hi = X.astype(np.float32)
    lo = (X - hi.astype(np.float64)).astype(np.float32)
    return np.ascontiguousarray(np.concatenate([hi, lo], axis=1))


def join(Y, L):
    Y = Y.astype(np.float64)
    return Y[:, :L] + Y[:, L:]


def exact_product(A, X):
    """A X in extended precision (longdouble), row by row from the CSR."""
    Xl = X.astype(np.longdouble)
    out = np.zeros((A.m, X.shape[1]), dtype=np.longdouble)
    for i in range(A.m):
        s, e = A.rowptr[i], A.rowptr[i + 1]
        if e > s:
            out[i] = A.vals[s:e].astype(np.longdouble) @ Xl[A.colidx[s:e]]
    return out


def abs_product(A, X):
    Ad = np.abs(A.to_dense())
    return Ad @ np.abs(X)


def max_row(A):
    return int(np.max(np.diff(A.rowptr))) if A.m else 0


@pytest.mark.parametrize("L", [1, 4, 5, 16, 32, 33, 64])
@pytest.mark.parametrize("values", ["normal", "bf16"])
def test_spmm_df_parity(B, ctx, L, values):
    """Double-float product against the extended-precision product, both directions; general
    FP64 values take the split a = a_hi + a_lo path, bf16 values the exact single path."""
    A = ragged(613, 257, seed=L, values=values)
    M = B.Matrix.from_csr(ctx, A)
    At = synth.transpose(A)
    for Mat, rows, cols, tr, seed in ((A, A.m, A.n, False, 1), (At, A.n, A.m, True, 2)):
        X = np.random.default_rng(seed).standard_normal((cols, L))
        Xs = torch.from_numpy(split(X)).cuda()
        Y = join(M.spmm_df(Xs, transpose=tr).cpu().numpy(), L)
        ref = exact_product(Mat, X)
        k = max_row(Mat)
        bound = (k * (k + 4) + 8) * U48 * abs_product(Mat, X) + 1e-300
        err = np.abs((Y.astype(np.longdouble) - ref).astype(np.float64))
        assert np.all(err <= bound), float(np.max(err / bound))
        # and far below what FP32 reaches: typical error a few 2^-48 of s
        rel = err / (abs_product(Mat, X) + 1e-300)
        assert float(np.median(rel[abs_product(Mat, X) > 0])) < 16 * U48
    M.close()


def test_spmm_df_normalized_and_deterministic(B, ctx):
    A = ragged(500, 300, seed=11)
    M = B.Matrix.from_csr(ctx, A)
    X = torch.from_numpy(split(np.random.default_rng(3).standard_normal((300, 32)))).cuda()
    y1 = M.spmm_df(X)
    y2 = M.spmm_df(X)
    assert torch.equal(y1, y2)
    hi, lo = y1[:, :32].double(), y1[:, 32:].double()
    # |lo| <= ulp(hi) / 2 = 2^-24 |hi| (after Fast2Sum)
    assert bool(torch.all(lo.abs() <= hi.abs() * 2.0 ** -24 + 1e-300))
    M.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_storage_rounds_values(B, ctx, storage):
    """Values are rounded to the storage precision at creation: every product on the matrix
    (here the FP64 SpMM) is the product of the rounded matrix."""
    A = ragged(400, 200, seed=7)
    M = B.Matrix.from_csr(ctx, A, storage=storage)
    r = synth.bf16_round(A.vals) if storage == "bf16" else A.vals.astype(np.float32).astype(np.float64)
    Ar = synth.CSR(A.m, A.n, A.rowptr, A.colidx, r)
    X = np.random.default_rng(5).standard_normal((200, 16))
    Y = M.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = exact_product(Ar, X).astype(np.float64)
    assert np.max(np.abs(Y - ref) / (abs_product(Ar, X) + 1e-300)) < 20 * 2.0 ** -53
    M.close()


def test_bf16_storage_f32_and_df(B, ctx):
    """bf16 storage: the FP32 and double-float products stream the 2-byte values exactly."""
    A = ragged(600, 300, seed=9, values="bf16")
    M = B.Matrix.from_csr(ctx, A, storage="bf16")
    X = np.random.default_rng(6).standard_normal((300, 32))
    ref = exact_product(A, X)
    s = abs_product(A, X) + 1e-300
    k = max_row(A)
    y32 = M.spmm_f32(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(y32 - ref.astype(np.float64)) / s) < (k + 2) * U24
    ydf = join(M.spmm_df(torch.from_numpy(split(X)).cuda()).cpu().numpy(), 32)
    assert np.all(np.abs((ydf.astype(np.longdouble) - ref).astype(np.float64)) <= (k * (k + 4) + 8) * U48 * s)
    M.close()


def test_storage_overflow_rejected(B, ctx):
    A = ragged(50, 40, seed=2)
    A.vals[3] = 1e300
    with pytest.raises(RuntimeError, match="storage"):
        B.Matrix.from_csr(ctx, A, storage="fp32")
    with pytest.raises(RuntimeError):
        B.Matrix.from_csr(ctx, A, storage=7)


def test_autotuned_equals_first_call(B, ctx):
    """The first call on a (matrix, kind, L) runs the autotuner (every variant on the call's
    buffers); later calls use the cached pick. Every variant sums in the same order, so the
    results are bitwise equal."""
    A = synth.banded_random(40000, 20000, half_width=200, seed=3)
    for storage in ("fp64", "bf16"):
        M = B.Matrix.from_csr(ctx, A, storage=storage)
        X = torch.from_numpy(np.random.default_rng(8).standard_normal((20000, 32))).cuda()
        y0 = M.spmm(X)
        assert torch.equal(y0, M.spmm(X))
        Xf = X.float()
        f0 = M.spmm_f32(Xf)
        assert torch.equal(f0, M.spmm_f32(Xf))
        Xd = torch.from_numpy(split(X.cpu().numpy())).cuda()
        d0 = M.spmm_df(Xd)
        assert torch.equal(d0, M.spmm_df(Xd))
        M.close()


def test_spmm_full_size_banded_random(B, ctx):
    """The 2e6 x 1e6 banded-plus-random matrix (32M nonzeros, bf16 storage) at full size, L = 32:
    FP64, FP32 and double-float products on 2000 sampled rows of A X and of A^T Y against the
    extended-precision row sums."""
    A = synth.banded_random()
    M = B.Matrix.from_csr(ctx, A, storage="bf16")
    rng = np.random.default_rng(12)
    X = rng.standard_normal((A.n, 32))
    Xd = torch.from_numpy(X).cuda()
    rows = np.sort(rng.choice(A.m, 2000, replace=False))
    y64 = M.spmm(Xd).cpu().numpy()[rows]
    y32 = M.spmm_f32(Xd.float()).cpu().numpy()[rows].astype(np.float64)
    ydf = join(M.spmm_df(torch.from_numpy(split(X)).cuda()).cpu().numpy()[rows], 32)
    del Xd
    for r_i, r in enumerate(rows):
        s, e = A.rowptr[r], A.rowptr[r + 1]
        a = A.vals[s:e]
        xr = X[A.colidx[s:e]]
        ref = a.astype(np.longdouble) @ xr.astype(np.longdouble)
        sc = np.abs(a) @ np.abs(xr) + 1e-300
        k = e - s
        assert np.all(np.abs((y64[r_i] - ref).astype(np.float64)) <= (k + 1) * 2.0 ** -53 * sc)
        assert np.all(np.abs((y32[r_i] - ref).astype(np.float64)) <= (k + 2) * U24 * sc)
        assert np.all(np.abs((ydf[r_i].astype(np.longdouble) - ref).astype(np.float64)) <= (k * (k + 4) + 8) * U48 * sc)
    # A^T Y on sampled columns of A (rows of A^T)
    Y = rng.standard_normal((A.m, 32))
    zdf = M.spmm_df(torch.from_numpy(split(Y)).cuda(), transpose=True).cpu().numpy()
    cols = np.sort(rng.choice(A.n, 500, replace=False))
    z = join(zdf[cols], 32)
    rr = np.repeat(np.arange(A.m), np.diff(A.rowptr))
    for c_i, c in enumerate(cols):
        hit = np.nonzero(A.colidx == c)[0]
        a = A.vals[hit]
        yr = Y[rr[hit]]
        ref = a.astype(np.longdouble) @ yr.astype(np.longdouble)
        sc = np.abs(a) @ np.abs(yr) + 1e-300
        k = hit.size
        assert np.all(np.abs((z[c_i].astype(np.longdouble) - ref).astype(np.float64)) <= (k * (k + 4) + 8) * U48 * sc)
    M.close()
