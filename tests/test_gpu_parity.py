"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (floating point, FP64 everywhere):
* SpMM: same per-row summation order as a sequential CSR loop; allowed
  difference 1e-14 relative to sum |a_ij| |x_j| (fused vs separate rounding).
* quadrature: 1e-15 relative.
* moment block S^: 1e-9 relative to max |S| for the Krylov solver (its
  solves stop at relative residual tol_solve = 1e-12 and the block is
  amplified by at most 1 / min Im s_j), 1e-12 for the direct solver.
* triplets: count exact; sigma relative error <= 1e-10; residuals
  ||A^T u - sigma v|| / ||A||_2 <= 1e-10; vectors match the oracle's up to the
  common sign rule within max(1e-7, 10 ||A|| (res_gpu + res_oracle) / gap_i),
  gap_i the distance from sigma_i to the nearest other singular value
  (a singular vector is determined only to residual / gap).
"""
import numpy as np
import pytest

from oracle import cmsvd_oracle as O
from paper_2109_13655_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def ragged_sparse(m, n, seed):
    """Rows with 0..17 nonzeros at random columns (empty rows included)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(m):
        k = int(rng.integers(0, 18))
        c = np.sort(rng.choice(n, size=min(k, n), replace=False))
        rows += [i] * c.size
        cols += list(c)
    return synth.csr_from_coo(m, n, rows, cols, rng.standard_normal(len(rows)))


# ----------------------------------------------------------------------------- SpMM (row a3)
@pytest.mark.parametrize("L", [1, 5, 16, 20, 32, 33, 64, 257])
def test_spmm_parity(B, ctx, L):
    A = ragged_sparse(777, 301, seed=L)
    M = B.Matrix.from_csr(ctx, A)
    X = np.random.default_rng(1).standard_normal((301, L))
    Y = M.spmm(dev(X)).cpu().numpy()
    Ad = A.to_dense()
    ref = Ad @ X
    scale = np.abs(Ad) @ np.abs(X) + 1e-300
    assert np.max(np.abs(Y - ref) / scale) < 1e-14
    Xt = np.random.default_rng(2).standard_normal((777, L))
    Yt = M.spmm(dev(Xt), transpose=True).cpu().numpy()
    assert np.max(np.abs(Yt - Ad.T @ Xt) / (np.abs(Ad.T) @ np.abs(Xt) + 1e-300)) < 1e-14
    M.close()


@pytest.mark.parametrize("L", [3, 15, 32, 120])
def test_spmm_long_rows(B, ctx, L):
    """Rows far longer than 2048 nonzeros (the transpose of a tall matrix: 20 rows of ~5000)
    take the one-CTA-per-row kernel, deterministically. The bound scales with the row length:
    a sum of n = 5000 products carries ~sqrt(n) u of sum |a||x| (1e-14 for rows of 17)."""
    A = synth.random_sparse(20000, 20, 5, seed=L)
    M = B.Matrix.from_csr(ctx, A)
    Ad = A.to_dense()
    X = np.random.default_rng(4).standard_normal((20000, L))
    Yt = M.spmm(dev(X), transpose=True)
    ref = Ad.T @ X
    assert np.max(np.abs(Yt.cpu().numpy() - ref) / (np.abs(Ad.T) @ np.abs(X) + 1e-300)) < 2e-13
    assert torch.equal(Yt, M.spmm(dev(X), transpose=True))
    Z = np.random.default_rng(5).standard_normal((20, L))
    assert np.max(np.abs(M.spmm(dev(Z)).cpu().numpy() - Ad @ Z) / (np.abs(Ad) @ np.abs(Z) + 1e-300)) < 1e-14
    M.close()


@pytest.mark.parametrize("L", [1, 16, 33, 120])
def test_spmm_f32_parity(B, ctx, L):
    """FP32 SpMM (mixed path): FP32 values and accumulation in row order. Bound: a sum of
    k products of FP32-rounded operands is within ~(k + 2) u32 sum |a||x| of the exact sum
    (rows here hold at most 17 nonzeros; long rows of ~5000 in the transpose below)."""
    A = ragged_sparse(777, 301, seed=L)
    M = B.Matrix.from_csr(ctx, A)
    X = np.random.default_rng(1).standard_normal((301, L)).astype(np.float32)
    Y = M.spmm_f32(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    Ad = A.to_dense()
    ref = Ad @ X.astype(np.float64)
    scale = np.abs(Ad) @ np.abs(X.astype(np.float64)) + 1e-300
    assert np.max(np.abs(Y - ref) / scale) < 20 * 2.0 ** -24
    Bl = synth.random_sparse(20000, 20, 5, seed=L)
    Ml = B.Matrix.from_csr(ctx, Bl)
    Z = np.random.default_rng(2).standard_normal((20000, L)).astype(np.float32)
    Yt = Ml.spmm_f32(torch.from_numpy(Z).cuda(), transpose=True).cpu().numpy().astype(np.float64)
    Bd = Bl.to_dense()
    assert np.max(np.abs(Yt - Bd.T @ Z) / (np.abs(Bd.T) @ np.abs(Z) + 1e-300)) < 400 * 2.0 ** -24
    M.close()
    Ml.close()


def test_spmm_transpose_deterministic(B, ctx):
    A = synth.random_sparse(3000, 1000, 12, seed=5)
    M = B.Matrix.from_csr(ctx, A)
    X = dev(np.random.default_rng(3).standard_normal((3000, 16)))
    y1 = M.spmm(X, transpose=True)
    y2 = M.spmm(X, transpose=True)
    assert torch.equal(y1, y2)
    M.close()


# ----------------------------------------------------------------------------- Gram (rows a7-a8)
@pytest.mark.parametrize("n,c1,c2", [(1, 1, 1), (37, 5, 9), (1000, 64, 64), (3001, 80, 80), (20000, 256, 256),
                                      (777, 130, 7)])
def test_gram_parity(B, ctx, n, c1, c2):
    rng = np.random.default_rng(n + c1)
    X = dev(rng.standard_normal((n, c1 + 3)))[:, :c1]      # leading dimension c1 + 3
    Xh = X.cpu().numpy()
    Y = X if c1 == c2 else dev(rng.standard_normal((n, c2)))
    Yh = Y.cpu().numpy()
    G = torch.empty((c1, c2), dtype=torch.float64, device="cuda")
    ws = torch.empty(B.cmsvd_gram_workspace_size(ctx.handle, n, c1, c2), dtype=torch.uint8, device="cuda")
    B.cmsvd_gram(ctx.handle, X, Y, G, ws)
    ref = Xh.T @ Yh
    scale = np.abs(Xh).T @ np.abs(Yh)
    assert np.max(np.abs(G.cpu().numpy() - ref) / scale) < 1e-13
    G2 = torch.empty_like(G)
    B.cmsvd_gram(ctx.handle, X, Y, G2, ws)
    assert torch.equal(G, G2)                                 # deterministic
    if c1 == c2:
        assert torch.equal(G, G.T)                            # symmetric Gram: exactly symmetric


# ----------------------------------------------------------------------------- quadrature (row a1)
@pytest.mark.parametrize("variant", ["linear", "nt"])
@pytest.mark.parametrize("N", [2, 16, 32, 128])
def test_quadrature_parity(B, ctx, variant, N):
    a, b = 0.37, 1.9
    sh, w, sc = B.cmsvd_quadrature(ctx.handle, a, b, N, variant, 0.1)
    q = O.quadrature(a, b, N, variant, 0.1)
    for x, y in ((sh, q.shift), (w, q.weight), (sc, q.scaled)):
        assert np.max(np.abs(x - y) / np.abs(y)) < 1e-14


# ----------------------------------------------------------------------------- moments (rows a3-a6)
@pytest.mark.parametrize("variant,ell", [("linear", 1), ("nt", 1), ("linear", 2)])
def test_moments_krylov_vs_oracle(B, ctx, variant, ell):
    A = synth.random_sparse(400, 200, 8, seed=11)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b, _ = synth.window_interval(s, 60, 6)
    N, L, Mm = 16, 8, 4
    Vin = synth.gaussian_block(200, L, 12)
    M = B.Matrix.from_csr(ctx, A)
    p = B.params(N=N, L=L, M=Mm, ell=ell, variant=variant, solver="krylov")
    S, status, st = M.moments(a, b, p, dev(Vin))
    assert status == B.OK and st["converged"] == 1
    ref = O.moments(O.ShiftedSolver(A), O.quadrature(a, b, N, variant), Vin, Mm, ell=ell, extra=1)
    S = S.cpu().numpy()
    assert np.max(np.abs(S - ref)) <= 1e-9 * np.max(np.abs(ref))
    M.close()


@pytest.mark.parametrize("variant,ell", [("linear", 1), ("nt", 1), ("nt", 2)])
def test_moments_direct_vs_oracle(B, ctx, variant, ell):
    bp = synth.block_permuted(300, 8, 4, seed=21)
    sig = bp.sigmas_desc()
    a, b, _ = synth.window_interval(sig, 500, 12, min_rel_gap=1e-6, max_shift=10)
    N, L, Mm = 32, 8, 4
    Vin = synth.gaussian_block(bp.A.n, L, 22)
    M = B.Matrix.from_csr(ctx, bp.A)
    p = B.params(N=N, L=L, M=Mm, ell=ell, variant=variant, solver="direct")
    S, status, st = M.moments(a, b, p, dev(Vin))
    assert status == B.OK and st["solver_used"] == B.SOLVER_DIRECT
    ref = O.moments(O.ShiftedSolver(bp.A), O.quadrature(a, b, N, variant), Vin, Mm, ell=ell, extra=1)
    assert np.max(np.abs(S.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    M.close()


def test_auto_picks_direct_for_small_components(B, ctx):
    bp = synth.block_permuted(50, 8, 4, seed=23)
    M = B.Matrix.from_csr(ctx, bp.A)
    s = bp.sigmas_desc()
    a, b, _ = synth.window_interval(s, 50, 5)
    _, _, st = M.moments(a, b, B.params(N=16, L=4, M=2), dev(synth.gaussian_block(200, 4, 1)))
    assert st["solver_used"] == B.SOLVER_DIRECT and st["max_component"] == 4
    M.close()


# ----------------------------------------------------------------------------- end to end (rows a1-a9)
def compare(out, ref, truth=None, vec_tol=1e-7, spectrum=None, norm_A=1.0, res_tol=1e-10):
    assert out.sigma.size == ref.sigma.size
    if truth is not None:
        assert out.sigma.size == truth.size
        assert np.max(np.abs(out.sigma - truth) / truth) <= 1e-10
    assert np.max(np.abs(out.sigma - ref.sigma) / ref.sigma) <= 1e-10
    assert out.res_u.max() <= res_tol and out.res_v.max() <= res_tol
    tol = np.full(out.sigma.size, vec_tol)
    if spectrum is not None:
        sp = np.sort(spectrum)
        for i, s in enumerate(ref.sigma):
            k = np.searchsorted(sp, s)
            nb = sp[max(k - 2, 0):k + 2]
            nb = nb[np.abs(nb - s) > 1e-13 * s]
            gap = np.min(np.abs(nb - s)) if nb.size else s
            tol[i] = max(vec_tol, 10 * norm_A * (out.res_u[i] + ref.res_u[i] + 1e-16) / gap)
    assert np.all(np.max(np.abs(out.V - ref.V), axis=0) <= tol)
    assert np.all(np.max(np.abs(out.U - ref.U), axis=0) <= tol)
    assert np.max(np.abs(out.V.T @ out.V - np.eye(out.sigma.size))) <= 1e-10


@pytest.mark.parametrize("solver", ["auto", "krylov"])
def test_solve_random_sparse_2000x1000(B, ctx, solver):
    """The 2000 x 1000, 8 nnz/row workload: sigma ranked 400-419, N=16, L=16, M=4. AUTO takes
    the dense direct solver (n = 1000 <= 1024, one connected component); the Krylov solver is
    checked on the same case."""
    A = synth.random_sparse(2000, 1000, 8, seed=0)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b, _ = synth.window_interval(s, 400, 20)
    Vin = synth.gaussian_block(1000, 16, 1)
    ref = O.solve_interval(A, a, b, 16, 16, 4, Vin, norm_A=s[0])
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, B.params(N=16, L=16, M=4, solver=solver), dev(Vin))
    assert out.status in (B.OK,)
    want = B.SOLVER_DENSE if solver == "auto" else B.SOLVER_KRYLOV
    assert out.stats["solver_used"] == want and out.stats["converged"] == 1
    assert abs(out.stats["norm_A"] - s[0]) <= 1e-8 * s[0]
    compare(out, ref, truth=s[400:420][::-1])
    M.close()


def refine_floor(Ad, a, b, N, variant, Vin):
    """The rounding floor of an FP64 residual R_j = X - (s_j I - H) Y_j: evaluating H Y_j in
    FP64 leaves ~u ||H|| ||Y_j|| of error whatever Y_j is, so max_j,l u ||H||_2 ||Y_j[:, l]|| /
    ||X[:, l]|| is what a refined solve can be shown to reach (Y_j exact, from the oracle)."""
    q = O.quadrature(a, b, N, variant)
    solver = O.ShiftedSolver(Ad)
    nH = np.linalg.norm(Ad, 2) ** 2
    xn = np.linalg.norm(Vin, axis=0)
    worst = 0.0
    for j in range(q.shift.size):
        Y = solver.solve(q.shift[j], Vin)
        worst = max(worst, float(np.max(np.linalg.norm(Y, axis=0) / xn)))
    return 2.0 ** -53 * nH * worst


@pytest.mark.parametrize("which,variant,refine", [(1, "linear", 0), (1, "nt", 0), (2, "nt", 2), (1, "linear", 1)])
def test_solve_model_problems(B, ctx, which, variant, refine):
    """Exp II (Sec. 4.2). FP64 Lanczos, with and without FP64 iterative refinement of every
    shifted solve. Refinement stops at tol_solve = 1e-12 or at the rounding floor of its own
    FP64 residual (refine_floor): on model 1 the floor is far below 1e-12 and the tolerance is
    reached; on model 2 the NT shifts near sigma^2 ~ 1e-6 make ||Y_j|| large, and the check is
    against 64 times the floor."""
    Ad, sig = synth.model_problem(which)
    a, b = (0.8, 1.2) if which == 1 else (10 ** -3.025, 10 ** -1.025)
    truth = sig[(sig >= a) & (sig <= b)]
    Vin = synth.gaussian_block(200, 20, 3)
    # model 2's residuals at L M = 80 sit near 1e-10 (the oracle's own reach 7e-11), so both
    # sides use 1e-9 there to keep the count robust; sigma is still checked at 1e-10.
    # test_model2_at_the_target shows 1e-10 on model 2 with L = 40.
    tt = 1e-10 if which == 1 else 1e-9
    ref = O.solve_interval(Ad, a, b, 32, 20, 4, Vin, variant=variant, norm_A=sig.max(), tol_triplet=tt)
    A = synth.csr_from_dense(Ad)
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, B.params(N=32, L=20, M=4, variant=variant, solver="krylov", refine=refine,
                                          tol_triplet=tt), dev(Vin))
    if refine:
        assert out.stats["refine_rounds"] <= refine
        bound = max(1e-12, 64 * refine_floor(Ad, a, b, 32, variant, Vin))
        assert out.stats["refine_residual"] <= bound, (out.stats["refine_residual"], bound)
        if which == 1:
            assert out.stats["refine_residual"] <= 1e-12
    compare(out, ref, truth=truth, vec_tol=1e-6, spectrum=sig, norm_A=sig.max(), res_tol=tt)
    M.close()


@pytest.mark.parametrize("solver,precision", [("dense", "fp64"), ("krylov", "fp64"), ("krylov", "mixed")])
def test_model2_at_the_target(B, ctx, solver, precision):
    """Exp II model 2 (Sec. 4.2, NT) at the 1e-10 residual target: with L = 40 (L M = 160) the
    oracle's residuals reach 1.5e-11, and every side returns all 40 values with residual
    <= 1e-10 and sigma within 1e-10."""
    Ad, sig = synth.model_problem(2)
    a, b = 10 ** -3.025, 10 ** -1.025
    truth = sig[(sig >= a) & (sig <= b)]
    Vin = synth.gaussian_block(200, 40, 3)
    ref = O.solve_interval(Ad, a, b, 32, 40, 4, Vin, variant="nt", norm_A=sig.max())
    assert ref.sigma.size == 40
    M = B.Matrix.from_csr(ctx, synth.csr_from_dense(Ad))
    prec = B.MIXED if precision == "mixed" else B.FP64
    out = M.solve_interval(a, b, B.params(N=32, L=40, M=4, variant="nt", solver=solver, precision=prec,
                                          refine=2 if solver == "krylov" else 0), dev(Vin))
    compare(out, ref, truth=truth, vec_tol=1e-6, spectrum=sig, norm_A=sig.max(), res_tol=1e-10)
    M.close()


def test_forced_breakdown_returns_breakdown(B, ctx):
    """The test hook fault_breakdown_at makes the Krylov solver treat a Lanczos coefficient as
    non-finite at that step; the solve then reports CMSVD_BREAKDOWN (no GPU fault is made)."""
    A = synth.random_sparse(400, 200, 8, seed=11)
    M = B.Matrix.from_csr(ctx, A)
    Vin = dev(synth.gaussian_block(200, 8, 12))
    for prec in (B.FP64, B.MIXED):
        p = B.params(N=16, L=8, M=4, solver="krylov", precision=prec, fault_breakdown_at=5)
        with pytest.raises(RuntimeError) as ei:
            M.moments(1.0, 2.0, p, Vin)
        assert ei.value.status == B.BREAKDOWN
    # the context stays usable
    S, status, st = M.moments(1.0, 2.0, B.params(N=16, L=8, M=4, solver="krylov"), Vin)
    assert status == B.OK
    M.close()


@pytest.mark.parametrize("which,variant", [(1, "linear"), (1, "nt"), (2, "nt")])
def test_solve_model_problems_dense(B, ctx, which, variant):
    """Exp II (Sec. 4.2) with the dense direct solver: A^T A (200 x 200) eigendecomposed once,
    every shifted solve exact, as in the oracle."""
    Ad, sig = synth.model_problem(which)
    a, b = (0.8, 1.2) if which == 1 else (10 ** -3.025, 10 ** -1.025)
    truth = sig[(sig >= a) & (sig <= b)]
    Vin = synth.gaussian_block(200, 20, 3)
    tt = 1e-10 if which == 1 else 1e-9
    ref = O.solve_interval(Ad, a, b, 32, 20, 4, Vin, variant=variant, norm_A=sig.max(), tol_triplet=tt)
    M = B.Matrix.from_csr(ctx, synth.csr_from_dense(Ad))
    out = M.solve_interval(a, b, B.params(N=32, L=20, M=4, variant=variant, solver="dense", tol_triplet=tt), dev(Vin))
    assert out.stats["solver_used"] == B.SOLVER_DENSE
    compare(out, ref, truth=truth, vec_tol=1e-6, spectrum=sig, norm_A=sig.max(), res_tol=tt)
    M.close()


def test_dense_solver_rejects_wide_matrix(B, ctx):
    A = synth.random_sparse(3000, 1500, 4, seed=3)
    M = B.Matrix.from_csr(ctx, A)
    with pytest.raises(RuntimeError):
        M.solve_interval(1.0, 2.0, B.params(N=16, L=8, M=4, solver="dense"), dev(synth.gaussian_block(1500, 8, 1)))
    M.close()


@pytest.mark.parametrize("case,refine", [("random_sparse", 2), ("model1", 2), ("model2_nt", 2), ("random_sparse", 0),
                                         ("model1", 0)])
def test_solve_mixed_precision(B, ctx, case, refine):
    """Mixed path: double-float Lanczos vectors, SpMM and panel accumulation on the FP32 pipe
    (A's values as FP32 hi + lo pairs here, since these values are not FP32-exact); with
    refine > 0 an FP64 check of every shifted solve with corrections while the residual
    exceeds tol_solve; FP64 truncation and Rayleigh-Ritz. Same parity bar as FP64, and the
    checked FP64 residual reaches tol_solve = 1e-12 (model 2: 64 times its FP64 rounding
    floor, see refine_floor)."""
    if case == "random_sparse":
        A = synth.random_sparse(2000, 1000, 8, seed=0)
        Ad = A.to_dense()
        s = np.linalg.svd(Ad, compute_uv=False)
        a, b, _ = synth.window_interval(s, 400, 20)
        Vin = synth.gaussian_block(1000, 16, 1)
        ref = O.solve_interval(A, a, b, 16, 16, 4, Vin, norm_A=s[0])
        p = B.params(N=16, L=16, M=4, solver="krylov", precision=B.MIXED, refine=refine)
        truth, spec, nA, N, variant = s[400:420][::-1], s, s[0], 16, "linear"
    else:
        which, variant = (1, "linear") if case == "model1" else (2, "nt")
        Ad, sig = synth.model_problem(which)
        a, b = (0.8, 1.2) if which == 1 else (10 ** -3.025, 10 ** -1.025)
        Vin = synth.gaussian_block(200, 20, 3)
        tt = 1e-10 if which == 1 else 1e-9
        ref = O.solve_interval(Ad, a, b, 32, 20, 4, Vin, variant=variant, norm_A=sig.max(), tol_triplet=tt)
        A = synth.csr_from_dense(Ad)
        p = B.params(N=32, L=20, M=4, variant=variant, solver="krylov", precision=B.MIXED, tol_triplet=tt,
                     refine=refine)
        truth, spec, nA, N = sig[(sig >= a) & (sig <= b)], sig, sig.max(), 32
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, p, dev(Vin))
    if refine:
        assert out.stats["refine_residual"] > 0.0        # the FP64 check ran
        bound = max(1e-12, 64 * refine_floor(Ad, a, b, N, variant, Vin))
        assert out.stats["refine_residual"] <= bound, (out.stats["refine_residual"], bound)
        if case != "model2_nt":
            assert out.stats["refine_residual"] <= 1e-12 and out.stats["converged"] == 1
    compare(out, ref, truth=truth, vec_tol=1e-6, spectrum=spec, norm_A=nA, res_tol=p.tol_triplet)
    M.close()


def c2_case():
    bp = synth.block_permuted(25000, 8, 4, seed=2)
    s = bp.sigmas_desc()
    a, b, f = synth.window_interval(s, 50000, 200, min_rel_gap=1e-6, max_shift=10)
    return bp, s, a, b, f


def test_solve_block_permuted_200000x100000(B, ctx):
    """The known-spectrum workload at full size: 25000 permuted 8x4 blocks, 200
    interior sigma, N=32, L=32, M=8, ell=2 (the launch configuration of bench.py)."""
    bp, s, a, b, f = c2_case()
    Vin = synth.gaussian_block(bp.A.n, 32, 3)
    M = B.Matrix.from_csr(ctx, bp.A)
    out = M.solve_interval(a, b, B.params(N=32, L=32, M=8, ell=2), dev(Vin))
    assert out.stats["solver_used"] == B.SOLVER_DIRECT
    truth = np.sort(s[f:f + 200])
    ref = O.solve_interval(bp.A, a, b, 32, 32, 8, Vin, ell=2, norm_A=s[0])
    compare(out, ref, truth=truth, spectrum=s, norm_A=s[0])
    M.close()


@pytest.mark.parametrize("variant", ["linear", "nt"])
@pytest.mark.parametrize("solver", ["krylov", "direct"])
def test_residual_estimate_parity(B, ctx, variant, solver):
    """Sec. 3.4.1 estimate through S_+ against the oracle, on a small subspace (residuals
    O(0.1), far above rounding): Exp II model 1 (Krylov) and a block-permuted matrix (direct)."""
    if solver == "krylov":
        Ad, sig = synth.model_problem(1)
        A, a, b, nA, L, M_ = synth.csr_from_dense(Ad), 0.8, 1.2, sig.max(), 4, 2
    else:
        bp = synth.block_permuted(300, 8, 4, seed=21)
        sig = bp.sigmas_desc()
        a, b, _ = synth.window_interval(sig, 200, 40, min_rel_gap=1e-6, max_shift=10)
        A, nA, L, M_ = bp.A, sig[0], 4, 2
    Vin = synth.gaussian_block(A.n, L, 3)
    ref = O.solve_interval(A, a, b, 32, L, M_, Vin, variant=variant, norm_A=nA, with_estimate=True, tol_triplet=1.0)
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, B.params(N=32, L=L, M=M_, variant=variant, solver=solver, estimate=1, tol_triplet=1.0,
                                          norm_A=nA), dev(Vin))
    assert out.sigma.size == ref.sigma.size >= 3
    assert np.max(np.abs(out.sigma - ref.sigma) / ref.sigma) <= 1e-9
    assert np.max(np.abs(out.res_u - ref.res_u) / ref.res_u) <= 1e-7
    assert np.max(np.abs(out.res_est - ref.res_est) / ref.res_est) <= 1e-7
    if variant == "linear":
        assert np.max(np.abs(out.res_est - out.res_u) / out.res_u) <= 1e-9
    M.close()


def test_residual_estimate_full_size(B, ctx):
    """At the 200000 x 100000 bench configuration the linear estimate tracks the exact
    residual below the 1e-10 triplet tolerance. The estimate reaches v through
    S_+ W_S1 Sigma_S1^{-1} q, so its rounding error grows like u ||A|| ||S|| / sigma_S,r with
    the smallest kept sigma_S (here ~1e-12 of the largest): 2.5e-11 measured, against
    residuals of 1e-13."""
    bp, s, a, b, f = c2_case()
    Vin = synth.gaussian_block(bp.A.n, 32, 3)
    M = B.Matrix.from_csr(ctx, bp.A)
    out = M.solve_interval(a, b, B.params(N=32, L=32, M=8, ell=2, estimate=1), dev(Vin))
    assert out.sigma.size == 200
    assert np.all(np.isfinite(out.res_est))
    assert np.max(np.abs(out.res_est - out.res_u)) <= 1e-10
    with pytest.raises(Exception):
        # a solve without estimate=1 has no estimate to copy
        st, r = B.cmsvd_solve_interval(M.handle, a, b, B.params(N=32, L=32, M=8, ell=2), dev(Vin),
                                       M.workspace(B.params(N=32, L=32, M=8, ell=2)))
        try:
            B.cmsvd_result_copy_estimate(r, np.zeros(200))
        finally:
            B.cmsvd_result_destroy(r)
    M.close()


def test_empty_interval(B, ctx):
    A = synth.random_sparse(300, 150, 6, seed=41)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b = 1.05 * s[0], 2.0 * s[0]          # above the spectrum
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, B.params(N=16, L=4, M=4), dev(synth.gaussian_block(150, 4, 1)))
    assert out.sigma.size == 0
    M.close()


def test_exterior_interval_and_ragged_L(B, ctx):
    A = synth.random_sparse(300, 150, 6, seed=43)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b = 0.5 * (s[6] + s[7]), 1.01 * s[0]
    Vin = synth.gaussian_block(150, 5, 2)
    ref = O.solve_interval(A, a, b, 16, 5, 5, Vin, norm_A=s[0])
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, B.params(N=16, L=5, M=5), dev(Vin))
    compare(out, ref, truth=s[:7][::-1])
    M.close()


def test_determinism_and_seed_invariance(B, ctx):
    A = synth.random_sparse(600, 300, 8, seed=51)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b, _ = synth.window_interval(s, 100, 6)
    M = B.Matrix.from_csr(ctx, A)
    p = B.params(N=16, L=8, M=4)
    V1 = dev(synth.gaussian_block(300, 8, 1))
    o1 = M.solve_interval(a, b, p, V1)
    o2 = M.solve_interval(a, b, p, V1)
    assert np.array_equal(o1.sigma, o2.sigma) and np.array_equal(o1.V, o2.V)
    o3 = M.solve_interval(a, b, p, dev(synth.gaussian_block(300, 8, 99)))
    assert o3.sigma.size == o1.sigma.size == 6
    assert np.max(np.abs(o3.sigma - o1.sigma) / o1.sigma) <= 1e-12
    M.close()


def test_not_converged_status(B, ctx):
    A = synth.random_sparse(600, 300, 8, seed=51)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b, _ = synth.window_interval(s, 100, 6)
    M = B.Matrix.from_csr(ctx, A)
    out = M.solve_interval(a, b, B.params(N=16, L=8, M=4, max_iter=5, solver="krylov"),
                           dev(synth.gaussian_block(300, 8, 1)))
    assert out.status == B.NOT_CONVERGED and out.stats["converged"] == 0
    assert out.stats["krylov_iters"] == 5
    M.close()


def test_invalid_arguments(B, ctx):
    A = synth.random_sparse(60, 30, 4, seed=1)
    M = B.Matrix.from_csr(ctx, A)
    V = dev(synth.gaussian_block(30, 4, 1))
    for kw, (a, b) in [({}, (2.0, 1.0)), ({"N": 15}, (0.1, 1.0)), ({"M": 16, "N": 16}, (0.1, 1.0)),
                       ({"variant": "nt"}, (0.0, 1.0)), ({"L": 0}, (0.1, 1.0))]:
        with pytest.raises(B.CmsvdError) as e:
            M.solve_interval(a, b, B.params(N=kw.get("N", 16), L=kw.get("L", 4), M=kw.get("M", 2),
                                            variant=kw.get("variant", "linear")), V)
        assert e.value.status == B.INVALID_ARG
    M.close()


def test_invalid_matrix_rejected(B, ctx):
    rowptr = np.array([0, 2, 3], dtype=np.int64)
    bad_cols = [np.array([0, 5, 1], dtype=np.int32),    # column out of range
                np.array([1, 0, 1], dtype=np.int32),    # unsorted row
                np.array([1, 1, 0], dtype=np.int32)]    # duplicate
    for cols in bad_cols:
        with pytest.raises(B.CmsvdError) as e:
            B.cmsvd_csr_create(ctx.handle, 2, 3, rowptr, cols, np.ones(3))
        assert e.value.status == B.INVALID_MATRIX
    with pytest.raises(B.CmsvdError) as e:
        B.cmsvd_csr_create(ctx.handle, 2, 3, rowptr, np.array([0, 1, 2], dtype=np.int32),
                           np.array([1.0, np.nan, 1.0]))
    assert e.value.status == B.INVALID_MATRIX
    with pytest.raises(B.CmsvdError) as e:
        B.cmsvd_csr_create(ctx.handle, 2, 3, np.array([0, 2, 1], dtype=np.int64),   # rowptr not monotone
                           np.array([0], dtype=np.int32), np.ones(1))
    assert e.value.status == B.INVALID_MATRIX
