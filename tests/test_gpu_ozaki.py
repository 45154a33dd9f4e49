"""The tall dense products of the rank truncation and of qr(A V~) (Alg. 1 steps 3-4) computed
from exact BF16 tensor-core slice products (context dense arithmetic 0, the default, for
n >= 16384 rows), against the product in extended precision (numpy longdouble) and against the
FP64-pipe kernels (dense arithmetic 1).

Bound: every operand is cut into 8 slices of 7 bits under a power-of-two scale 2^e > max|x| of
its row or column, so each emulated term x_i y_i is within ~3 * 2^-53 * 2^(e_x + e_y) of the
exact one, and a sum of n terms within 4 n 2^-53 2^(e_x + e_y) (checked), while its typical
error, like the FP64 Gram's, grows like sqrt(n) (checked against the FP64 kernels' own error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_13655_gb300 import binding
    return binding


def graded(rng, n, c, axis):
    """Gaussian entries with scales spread over 10^-3 .. 10^3 across columns (axis 1) or rows."""
    X = rng.standard_normal((n, c))
    s = 10.0 ** rng.uniform(-3, 3, size=c if axis == 1 else n)
    return X * (s[None, :] if axis == 1 else s[:, None])


def pow2_scale(v):
    """2^e with 2^(e-1) <= max|v| < 2^e (the slicing's scale) for each entry of max|v|."""
    return 2.0 ** (np.floor(np.log2(np.maximum(v, 1e-300))) + 1)


def gram_ref(X, Y):
    return X.astype(np.longdouble).T @ Y.astype(np.longdouble)


@pytest.mark.parametrize("n,c1,c2,same", [(20000, 40, 36, False), (16384, 48, 48, True), (33001, 33, 34, False)])
def test_ozaki_gram(B, n, c1, c2, same):
    rng = np.random.default_rng(n + c1)
    X = graded(rng, n, c1, 1)
    Y = X if same else graded(rng, n, c2, 1)
    ref = gram_ref(X, Y)
    out = {}
    for mode in (0, 1):
        ctx = B.Context()
        ctx.set_dense_arith(mode)
        Xd = torch.from_numpy(X).cuda()
        Yd = Xd if same else torch.from_numpy(Y).cuda()
        G = torch.empty((c1, c2), dtype=torch.float64, device="cuda")
        ws = torch.empty(B.cmsvd_gram_workspace_size(ctx.handle, n, c1, c2), dtype=torch.uint8, device="cuda")
        B.cmsvd_gram(ctx.handle, Xd, Yd, G, ws)
        torch.cuda.synchronize()
        out[mode] = G.cpu().numpy()
        ctx.close()
    err = {m: np.abs((out[m].astype(np.longdouble) - ref).astype(np.float64)) for m in (0, 1)}
    sx, sy = pow2_scale(np.abs(X).max(axis=0)), pow2_scale(np.abs(Y).max(axis=0))
    assert np.all(err[0] <= 4 * n * U * np.outer(sx, sy))
    absdot = np.abs(X).T @ np.abs(Y)
    # typical accuracy: within a small factor of the FP64 kernels' own error on the same product
    assert np.median(err[0] / absdot) <= 8 * max(np.median(err[1] / absdot), U)
    if same:
        assert np.array_equal(out[0], out[0].T)


@pytest.mark.parametrize("n,c1,c2", [(20000, 64, 48), (17000, 300, 40), (16384, 1024, 33)])
def test_ozaki_product(B, n, c1, c2):
    """Z = X W (cmsvd_gemm) with rows of X graded over 10^-3..10^3 and columns of W graded:
    each entry within 4 c1 2^-53 2^(e_i + f_l) of the extended-precision product (e_i, f_l the
    row and column scales), and typically within a small factor of the FP64 kernels' error."""
    rng = np.random.default_rng(n + c1 + c2)
    X = graded(rng, n, c1, 0)
    W = graded(rng, c1, c2, 1)
    rows = np.sort(rng.choice(n, 1500, replace=False))     # extended-precision reference on sampled rows
    ref = X[rows].astype(np.longdouble) @ W.astype(np.longdouble)
    out = {}
    for mode in (0, 1):
        ctx = B.Context()
        ctx.set_dense_arith(mode)
        Z = torch.empty((n, c2), dtype=torch.float64, device="cuda")
        B.cmsvd_gemm(ctx.handle, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(), Z)
        torch.cuda.synchronize()
        out[mode] = Z.cpu().numpy()[rows]
        ctx.close()
    err = {m: np.abs((out[m].astype(np.longdouble) - ref).astype(np.float64)) for m in (0, 1)}
    sx, sw = pow2_scale(np.abs(X[rows]).max(axis=1)), pow2_scale(np.abs(W).max(axis=0))
    assert np.all(err[0] <= 4 * c1 * U * np.outer(sx, sw))
    absprod = np.abs(X[rows]) @ np.abs(W)
    assert np.median(err[0] / absprod) <= 8 * max(np.median(err[1] / absprod), U)
