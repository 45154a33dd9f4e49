"""Pins for the CPU oracle: each check compares it with something other than itself.

* the quadrature exactness condition (Eq. cond, Sec. 3.2),
* the conjugate-symmetry halving against the full N-point sum (Sec. 3.1),
* Prop. 1 (S_k = (A^T A)^k S_0, linear variant),
* closed-form moments from a dense SVD (first equality of Prop. 1; Sec. 3.3 for NT),
* the contour-integral limit of Thm. 1 (spectral projector) for both variants,
* the error bound of Thm. 2 (subspace distances of the exact singular vectors),
* the Exp I filter statements (tests/golden/exp1_filter.txt),
* triplets against numpy's dense SVD, and the Exp II model problems (Sec. 4.2),
* the spurious index tau on inputs solvable by hand and on the 2000 x 1000
  workload (Sec. 3.4.2),
* the residual estimate through S_+ (Sec. 3.4.1): equal to the exact residual for the
  linear variant, equal to the ln(A^T A) form for NT, and mu fixed by one exact residual;
  on the Exp II model problems it follows the exact residuals (Sec. 4.2).

The mutation tests at the end plant plausible mistakes in the oracle and
check that at least one of these pins fails.
"""
import os

import numpy as np
import pytest

from oracle import cmsvd_oracle as O
from paper_2109_13655_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- helpers
def _svd_matrix(sig, m, seed):
    """Dense m x n matrix with prescribed singular values and Haar singular vectors."""
    rng = np.random.default_rng(seed)
    n = len(sig)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (U * sig) @ V.T


def exactness_error(N, a=0.8, b=1.2, variant="linear"):
    """max_k<=N-2 |sum_{j=1}^N omega_j m_j^k| / sum|omega_j| and the k=N-1 value."""
    q = O.quadrature(a, b, N, variant, full=True)
    w = q.weight if variant == "linear" else q.weight / np.exp(q.node)  # omega_j
    scale = np.sum(np.abs(w))
    errs = [abs(np.sum(w * q.scaled ** k)) / scale for k in range(N - 1)]
    last = abs(np.sum(w * q.scaled ** (N - 1))) / scale
    return max(errs), last


def halving_error(variant="linear"):
    """2 Re sum_{j<=N/2} vs the full sum over j = 1..N (both through the direct solves)."""
    A = synth.random_sparse(40, 20, 5, seed=11)
    V = synth.gaussian_block(20, 3, 12)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b = 0.5 * (s[5] + s[6]), 0.5 * (s[1] + s[2])
    N, M = 16, 3
    solver = O.ShiftedSolver(A)
    half = O.moments(solver, O.quadrature(a, b, N, variant), V, M)
    qf = O.quadrature(a, b, N, variant, full=True)
    full = []
    for k in range(M):
        acc = np.zeros(V.shape, dtype=complex)
        for j in range(N):
            acc += qf.weight[j] * qf.scaled[j] ** k * solver.solve(qf.shift[j], V)
        full.append(acc)
    full = np.concatenate(full, axis=1)
    return np.max(np.abs(half - full)) / np.max(np.abs(full)), np.max(np.abs(full.imag)) / np.max(np.abs(full))


def closed_form_error(variant="linear", ell=1):
    """S^ from direct solves vs sum_i c_k(sigma_i) f(sigma_i)^(ell-1) v_i v_i^T V_in from numpy's SVD."""
    A = synth.random_sparse(60, 30, 6, seed=21)
    Ad = A.to_dense()
    _, s, Vt = np.linalg.svd(Ad, full_matrices=False)
    a, b = 0.5 * (s[9] + s[10]), 0.5 * (s[3] + s[4])
    N, M, L = 16, 4, 4
    Vin = synth.gaussian_block(30, L, 22)
    q = O.quadrature(a, b, N, variant)
    S = O.moments(O.ShiftedSolver(A), q, Vin, M, ell=ell)
    C = Vt @ Vin                    # v_i^T V_in
    ref = []
    for k in range(M):
        c = O.moment_filter(s, q, k) * O.filter_value(s, q) ** (ell - 1)
        ref.append(Vt.T @ (c[:, None] * C))
    ref = np.concatenate(ref, axis=1)
    return np.max(np.abs(S - ref)) / np.max(np.abs(ref))


def prop1_error(scaled=True):
    """Prop. 1: S_k = (A^T A)^k S_0 (literal z^k) or ((A^T A - gamma)/rho)^k S_0 (scaled)."""
    A = synth.random_sparse(50, 25, 6, seed=31)
    H = A.to_dense().T @ A.to_dense()
    s = np.sqrt(np.linalg.eigvalsh(H))[::-1]
    a, b = 0.5 * (s[7] + s[8]), 0.5 * (s[2] + s[3])
    N, M, L = 8, 7, 3                  # k up to N-1
    Vin = synth.gaussian_block(25, L, 32)
    q = O.quadrature(a, b, N)
    S = O.moments(O.ShiftedSolver(A), q, Vin, M, scaled=scaled)
    T = (H - q.gamma * np.eye(25)) / q.rho if scaled else H
    S0 = S[:, :L]
    err = 0.0
    for k in range(1, M):
        pred = np.linalg.matrix_power(T, k) @ S0
        err = max(err, np.max(np.abs(S[:, k * L:(k + 1) * L] - pred)) / np.max(np.abs(pred)))
    return err


def contour_limit_error(variant="linear"):
    """Thm. 1 / Sec. 3.3: as N grows, S_k -> sum_{sigma_i in [a,b]} x_i^k v_i v_i^T V_in,
    x_i = (sigma_i^2 - gamma)/rho (linear) or (log sigma_i^2 - gamma)/rho (NT)."""
    sig = np.array([3.0, 2.2, 1.6, 1.5, 1.4, 1.0, 0.6, 0.3, 0.1, 0.05])
    Ad = _svd_matrix(sig, 16, 41)
    _, s, Vt = np.linalg.svd(Ad, full_matrices=False)
    a, b = 1.2, 1.9                     # holds 1.6, 1.5, 1.4
    N, M, L = 512, 3, 2
    Vin = synth.gaussian_block(10, L, 42)
    q = O.quadrature(a, b, N, variant, alpha=1.0)
    S = O.moments(O.ShiftedSolver(Ad), q, Vin, M)
    inside = (s >= a) & (s <= b)
    x = (s ** 2 - q.gamma) / q.rho if variant == "linear" else (np.log(s ** 2) - q.gamma) / q.rho
    ref = np.concatenate([Vt[inside].T @ ((x[inside] ** k)[:, None] * (Vt[inside] @ Vin)) for k in range(M)], axis=1)
    return np.max(np.abs(S - ref)) / np.max(np.abs(ref))


def theorem2_excess(variant="linear", ell=1):
    """Thm. 2 on a 60 x 30 matrix with known singular vectors (L = 2, M = 3, N = 16, three
    values inside [a, b]). With f ordered by decreasing |f(sigma_i)|, K the block Krylov
    matrix (of A^T A, or of g^{-1}(A^T A) = ln(A^T A) for NT, where the theorem holds
    approximately), s_i in R(K) with P_LM s_i = v_i and beta_i = ||v_i - s_i||, the distances
    of v_i from R(S) and of u_i from R(A S) must stay below beta_i |f(sigma_LM+1)/f(sigma_i)|^ell
    and alpha_i times that. Returns the largest ratio of distance to bound over i <= LM
    (<= 1 when the theorem holds)."""
    sig = np.linspace(0.1, 3.0, 30)[::-1]
    Ad = _svd_matrix(sig, 60, 5)
    U, s, Vt = np.linalg.svd(Ad, full_matrices=False)
    L, M, N = 2, 3, 16
    q = O.quadrature(1.42, 1.78, N, variant)
    Vin = synth.gaussian_block(30, L, 6)
    S = O.moments(O.ShiftedSolver(Ad), q, Vin, M, ell=ell)
    f = O.filter_value(s, q)
    order = np.argsort(-np.abs(f), kind="stable")
    V, U, so, fo = Vt.T[:, order], U[:, order], s[order], f[order]
    H = Ad.T @ Ad
    if variant == "nt":
        lam, W = np.linalg.eigh(H)
        H = (W * np.log(lam)) @ W.T
    K = np.concatenate([np.linalg.matrix_power(H, k) @ Vin for k in range(M)], axis=1)
    LM = L * M
    QV, _ = np.linalg.qr(S)
    QU, _ = np.linalg.qr(Ad @ S)
    worst = 0.0
    for i in range(LM):
        si = K @ np.linalg.solve(V[:, :LM].T @ K, np.eye(LM)[:, i])
        bound_v = np.linalg.norm(V[:, i] - si) * abs(fo[LM] / fo[i]) ** ell
        bound_u = bound_v * so[LM:].max() / so[i]
        dv = np.linalg.norm(V[:, i] - QV @ (QV.T @ V[:, i]))
        du = np.linalg.norm(U[:, i] - QU @ (QU.T @ U[:, i]))
        worst = max(worst, (dv - 1e-13) / bound_v, (du - 1e-13) / bound_u)
    return worst


@pytest.mark.parametrize("variant,ell", [("linear", 1), ("linear", 2), ("nt", 1), ("nt", 2)])
def test_theorem2_error_bound(variant, ell):
    assert theorem2_excess(variant, ell) <= 1.0


def dense_triplet_errors(variant="linear", ell=1, m=120, n=60, first=20, count=6, seed=51):
    """Triplets of the oracle vs numpy's dense SVD on a small sparse matrix."""
    A = synth.random_sparse(m, n, 6, seed=seed)
    Ad = A.to_dense()
    U, s, Vt = np.linalg.svd(Ad, full_matrices=False)
    a, b, _ = synth.window_interval(s, first, count)
    Vin = synth.gaussian_block(n, 8, seed + 1)
    r = O.solve_interval(A, a, b, 32, 8, 4, Vin, ell=ell, variant=variant, norm_A=s[0])
    truth = s[first:first + count][::-1]
    if r.sigma.size != count:
        return r.sigma.size, np.inf, np.inf, np.inf
    sig_err = np.max(np.abs(r.sigma - truth) / truth)
    vt = Vt[first:first + count][::-1]
    cosv = np.abs(np.sum(vt.T * r.V, axis=0))
    return r.sigma.size, sig_err, float(np.max(1 - cosv)), float(np.max(r.res_u))


# ----------------------------------------------------------------------------- pins
@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_quadrature_exactness_condition(N):
    """Eq. cond: sum_j omega_j z_j^k = 0 for k = 0..N-2 (checked on the scaled nodes,
    which span the same polynomials). At k = N-1 the trapezoidal sum picks up the
    e^{+-iN theta} Fourier terms: writing cos + i alpha sin = c1 e^{i theta} + c2 e^{-i theta}
    with c1 = (1+alpha)/2, c2 = (1-alpha)/2 and sum_j e^{iN theta_j} = -N, it equals
    -rho (c1^N - c2^N), which is nonzero."""
    err, last = exactness_error(N)
    assert err < 1e-14
    q = O.quadrature(0.8, 1.2, N, full=True)
    c1, c2 = (1 + q.alpha) / 2, (1 - q.alpha) / 2
    expect = q.rho * (c1 ** N - c2 ** N) / np.sum(np.abs(q.weight))
    assert abs(last - expect) <= 1e-14 + 1e-9 * expect
    if N <= 32:
        assert expect > 1e-12


def test_quadrature_literal_exactness():
    """Eq. cond in the literal form sum_j omega_j z_j^k for moderate |z|."""
    N = 16
    q = O.quadrature(0.8, 1.2, N, "linear", full=True)
    for k in range(N - 1):
        terms = q.weight * q.node ** k
        assert abs(np.sum(terms)) <= 1e-13 * np.sum(np.abs(terms))


def test_quadrature_conjugate_pairs():
    """(z_j, omega_j) and (z_{N+1-j}, omega_{N+1-j}) are complex conjugates (Sec. 3.1, pairing reading)."""
    q = O.quadrature(1.0, 2.0, 16, full=True)
    assert np.allclose(q.node[::-1], np.conj(q.node), rtol=0, atol=1e-15)
    assert np.allclose(q.weight[::-1], np.conj(q.weight), rtol=0, atol=1e-15)
    assert np.all(q.node[:8].imag > 0)


@pytest.mark.parametrize("variant", ["linear", "nt"])
def test_halving_matches_full_sum(variant):
    err, imag = halving_error(variant)
    assert err < 1e-12
    assert imag < 1e-12          # the full sum is real (Sec. 3.1)


def test_prop1_linear_scaled():
    assert prop1_error(scaled=True) < 1e-9


def test_prop1_linear_literal():
    assert prop1_error(scaled=False) < 1e-8


@pytest.mark.parametrize("variant", ["linear", "nt"])
@pytest.mark.parametrize("ell", [1, 2])
def test_closed_form_moments(variant, ell):
    assert closed_form_error(variant, ell) < 1e-11


@pytest.mark.parametrize("variant", ["linear", "nt"])
def test_contour_integral_limit(variant):
    assert contour_limit_error(variant) < 1e-10


def test_filter_values_exp1():
    rows = []
    with open(os.path.join(GOLDEN, "exp1_filter.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                rows.append(line)
    assert len(rows) >= 10
    for a, b, variant, sig, lo, hi in rows:
        q = O.quadrature(float(a), float(b), 32, variant)
        val = abs(float(O.filter_value(float(sig), q)))
        assert float(lo) <= val <= float(hi), (a, b, variant, sig, val)


@pytest.mark.parametrize("variant,ell", [("linear", 1), ("nt", 1), ("linear", 2)])
def test_triplets_match_dense_svd(variant, ell):
    count, sig_err, vec_err, res = dense_triplet_errors(variant, ell)
    assert count == 6
    assert sig_err < 1e-12
    assert vec_err < 1e-10
    assert res < 1e-10


def test_exterior_interval():
    A = synth.random_sparse(100, 50, 6, seed=61)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b = 0.5 * (s[7] + s[8]), 1.01 * s[0]
    Vin = synth.gaussian_block(50, 8, 62)
    r = O.solve_interval(A, a, b, 32, 8, 4, Vin, norm_A=s[0])
    assert r.sigma.size == 8
    assert np.max(np.abs(r.sigma - s[:8][::-1]) / s[:8][::-1]) < 1e-12


def test_two_sided_identity():
    """A v = sigma u holds by construction of the two-sided projection (Sec. 3.4.1)."""
    A = synth.random_sparse(120, 60, 6, seed=51)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b, _ = synth.window_interval(s, 20, 6)
    r = O.solve_interval(A, a, b, 32, 8, 4, synth.gaussian_block(60, 8, 52), norm_A=s[0])
    assert np.max(r.res_v) < 1e-14
    # the returned bases are orthonormal
    assert np.max(np.abs(r.U.T @ r.U - np.eye(6))) < 1e-12
    assert np.max(np.abs(r.V.T @ r.V - np.eye(6))) < 1e-12


def test_model_problems_exp2():
    """Sec. 4.2: 40 triplets each; model 1 accurate for both variants; on model 2
    the NT variant is accurate and the linear one is not."""
    Vin = synth.gaussian_block(200, 20, 3)
    A1, s1 = synth.model_problem(1)
    truth1 = s1[(s1 >= 0.8) & (s1 <= 1.2)]
    assert truth1.size == 40
    for variant in ("linear", "nt"):
        r = O.solve_interval(A1, 0.8, 1.2, 32, 20, 4, Vin, variant=variant, norm_A=s1.max())
        assert r.sigma.size == 40
        assert np.max(np.abs(r.sigma - truth1) / truth1) < 1e-13
    # model 2, interval endpoints moved to gap midpoints (endpoint reading): 40 values
    a, b = 10 ** -3.025, 10 ** -1.025
    A2, s2 = synth.model_problem(2)
    truth2 = s2[(s2 >= a) & (s2 <= b)]
    assert truth2.size == 40
    # model 2's residuals sit near 1e-10 (filter-limited at L M = 80): the count uses 1e-9
    rn = O.solve_interval(A2, a, b, 32, 20, 4, Vin, variant="nt", norm_A=s2.max(), tol_triplet=1e-9)
    assert rn.sigma.size == 40
    assert np.max(np.abs(rn.sigma - truth2) / truth2) < 1e-13
    rl = O.solve_interval(A2, a, b, 32, 20, 4, Vin, variant="linear", norm_A=s2.max(), tol_triplet=1e-9)
    assert rl.sigma.size < 40


def c1_result():
    """The 2000 x 1000 workload (8 nnz/row, sigma ranked 400-419) through the oracle."""
    A = synth.random_sparse(2000, 1000, 8, seed=0)
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    a, b, _ = synth.window_interval(s, 400, 20)
    Vin = synth.gaussian_block(1000, 16, 1)
    return O.solve_interval(A, a, b, 16, 16, 4, Vin, norm_A=s[0]), s, a, b


def test_c1_tau_detects_spurious():
    """2000 x 1000, 8 nnz/row, sigma ranked 400-419: 20 found; one Ritz value in
    [a, b] is spurious (tiny tau, large residual) and tau removes it (Sec. 3.4.2)."""
    r, s, a, b = c1_result()
    truth = s[400:420][::-1]
    assert r.sigma.size == 20
    assert np.max(np.abs(r.sigma - truth) / truth) < 1e-13
    inside = (r.all_phi >= a) & (r.all_phi <= b)
    spurious = inside & (r.all_tau < 1e-8)
    assert spurious.sum() >= 1
    assert np.all(r.all_res[spurious] > 1e-6)
    assert np.all(r.all_tau[inside & ~spurious] > 1e-3)


def tau_special_case_error():
    """tau of Sec. 3.4.2 on inputs solvable by hand. For q = e_k it is sigma_S,k (relative:
    sigma_S,k / sigma_S,1). For q with equal weight on directions k and l it is the harmonic
    mean 2 s_k s_l / (s_k + s_l), whatever the scale of q, so a Ritz vector with half its
    weight on a rounding-level direction of S is spurious."""
    sS = np.array([4.0, 2.0, 1.0, 1e-12])
    Q = np.zeros((4, 3))
    Q[1, 0] = 1.0                                    # e_2
    Q[0, 1] = Q[3, 1] = np.sqrt(0.5)                 # half on the noise direction
    Q[0, 2] = Q[2, 2] = 3.0                          # equal weight, scaled by 3
    expect = np.array([2.0, 2 * 4.0 * 1e-12 / (4.0 + 1e-12), 2 * 4.0 * 1.0 / 5.0]) / 4.0
    tau = O.spurious_index(Q, sS, 4)
    return float(np.max(np.abs(tau - expect) / expect))


def test_tau_special_cases():
    assert tau_special_case_error() < 1e-14


def estimate_errors(variant):
    """Residual estimate through S_+ (Sec. 3.4.1) on Exp II model 1 with a deliberately small
    subspace (L = 4, M = 2 for 40 wanted values), so that the residuals are O(0.1) and far
    above rounding. Linear: the estimate must equal the exact residual (Prop. 1 makes
    A^T A S_k = rho S_{k+1} + gamma S_k exact with scaled nodes). NT: r~ must equal
    || ln(A^T A) v - ln(sigma^2) v || / sigma computed from a dense eigendecomposition."""
    A, sig = synth.model_problem(1)
    Vin = synth.gaussian_block(200, 4, 3)
    r = O.solve_interval(A, 0.8, 1.2, 32, 4, 2, Vin, variant=variant, norm_A=sig.max(), with_estimate=True,
                         tol_triplet=1.0)
    assert r.sigma.size >= 4 and r.res_u.min() > 1e-3
    if variant == "linear":
        return np.max(np.abs(r.res_est - r.res_u) / r.res_u), r
    lam, W = np.linalg.eigh(A.T @ A)
    lnH = (W * np.log(lam)) @ W.T
    direct = np.linalg.norm(lnH @ r.V - r.V * np.log(r.sigma ** 2), axis=0) / r.sigma / sig.max()
    return np.max(np.abs(r.res_tilde - direct) / direct), r


def test_residual_estimate_linear_equals_exact():
    err, r = estimate_errors("linear")
    assert err < 1e-10
    # and at rounding-level residuals (the full Exp II setting) the two agree to 1e-15
    A, sig = synth.model_problem(1)
    rr = O.solve_interval(A, 0.8, 1.2, 32, 20, 4, synth.gaussian_block(200, 20, 3), norm_A=sig.max(),
                          with_estimate=True)
    assert rr.sigma.size == 40 and np.max(np.abs(rr.res_est - rr.res_u)) < 1e-14


def test_residual_estimate_nt_log_form_and_mu():
    err, r = estimate_errors("nt")
    assert err < 1e-10
    # mu is fixed by one exact residual (Eq. res_nonlinear): there the estimate is exact
    ratio = r.res_est / r.res_u
    assert np.min(np.abs(ratio - 1.0)) < 1e-12
    # i' is the candidate with the largest r~: every other estimate scales r~ by the same mu
    mu = r.res_est / r.res_tilde
    assert np.max(np.abs(mu - mu[0])) <= 1e-12 * mu[0]


@pytest.mark.parametrize("which", [1, 2])
@pytest.mark.parametrize("variant", ["linear", "nt"])
def test_residual_estimate_tracks_exact_on_exp2(which, variant):
    """Sec. 4.2 (the figure of residuals and their estimates): on both model problems, with
    the paper's (L, M, N, ell) = (20, 4, 32, 1), the estimates of Sec. 3.4.1 follow the exact
    residual norms. Here the residuals span two orders of magnitude (model 2). Every estimate
    lies within a factor of 20 of its exact residual, and the median ratio within 2."""
    Vin = synth.gaussian_block(200, 20, 3)
    a, b = (0.8, 1.2) if which == 1 else (10 ** -3.025, 10 ** -1.025)
    A, sig = synth.model_problem(which)
    r = O.solve_interval(A, a, b, 32, 20, 4, Vin, variant=variant, norm_A=sig.max(), with_estimate=True,
                         tol_triplet=1.0)
    assert r.sigma.size >= 30
    ratio = r.res_est / r.res_u
    assert np.all(ratio > 1 / 20) and np.all(ratio < 20)
    assert 0.5 < np.median(ratio) < 2.0


def test_exp3_digits_standin():
    """Sec. 4.3 shape (60000 x 784, ~150 nonzeros per row, ||A||_2 = 1): the exterior
    interval holding the 21 largest values and the interior window of 17 values starting at
    the 41st are found exactly by the NT variant, with L = 15, M = 4, N = 32 (Table 1's first
    row), against numpy's dense SVD. The linear variant misses the exterior values."""
    A = synth.digits_like()
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    assert abs(s[0] - 1.0) < 1e-12
    Vin = synth.gaussian_block(A.n, 15, 5)
    a, b = 0.5 * (s[20] + s[21]), 1.01 * s[0]
    r = O.solve_interval(A, a, b, 32, 15, 4, Vin, variant="nt", norm_A=s[0])
    assert r.sigma.size == 21
    assert np.max(np.abs(r.sigma - s[:21][::-1]) / s[:21][::-1]) < 1e-13
    rl = O.solve_interval(A, a, b, 32, 15, 4, Vin, variant="linear", norm_A=s[0])
    assert rl.sigma.size < 21
    a, b, _ = synth.window_interval(s, 40, 17)
    r = O.solve_interval(A, a, b, 32, 15, 4, Vin, variant="nt", norm_A=s[0])
    assert r.sigma.size == 17
    assert np.max(np.abs(r.sigma - s[40:57][::-1]) / s[40:57][::-1]) < 1e-13


# ----------------------------------------------------------------------------- mutations
def _mutant_quadrature(kind):
    orig = O.quadrature

    def q(a, b, N, variant="linear", alpha=0.1, full=False):
        r = orig(a, b, N, variant, alpha, full)
        if kind == "no_alpha_in_weight":
            r.weight = r.weight / (alpha * np.cos(r.theta) + 1j * np.sin(r.theta)) * (np.cos(r.theta) + 1j * np.sin(r.theta))
        elif kind == "psi_without_exp" and variant == "nt":
            r.weight = r.weight / np.exp(r.node)
        elif kind == "theta_without_half":
            th = r.theta + np.pi / N
            r.node = r.gamma + r.rho * (np.cos(th) + 1j * alpha * np.sin(th))
            r.shift = r.node if variant == "linear" else np.exp(r.node)
        return r
    return q


@pytest.mark.parametrize("kind,check", [
    ("no_alpha_in_weight", lambda: exactness_error(16)[0] > 1e-6),
    ("psi_without_exp", lambda: contour_limit_error("nt") > 1e-3),
    ("theta_without_half", lambda: closed_form_error("linear") > 1e-6 or halving_error()[1] > 1e-6),
])
def test_mutation_quadrature_caught(monkeypatch, kind, check):
    monkeypatch.setattr(O, "quadrature", _mutant_quadrature(kind))
    assert check()


def test_mutation_shift_sign_caught(monkeypatch):
    orig = O.ShiftedSolver.solve
    monkeypatch.setattr(O.ShiftedSolver, "solve", lambda self, s, X: -orig(self, s, X))
    assert closed_form_error("linear") > 1.0


def test_mutation_dropped_factor_two_caught(monkeypatch):
    orig = O.moments

    def half(solver, q, V, M, ell=1, scaled=True, extra=0):
        return 0.5 * orig(solver, q, V, M, ell, scaled, extra)
    monkeypatch.setattr(O, "moments", half)
    assert closed_form_error("linear") > 0.1


def test_mutation_moment_index_caught(monkeypatch):
    """Using the literal node instead of the scaled one in one factor breaks Prop. 1 (scaled form)."""
    monkeypatch.setattr(O, "moment_factor", lambda q, k, scaled=True: q.node ** k)
    assert prop1_error(scaled=True) > 1e-3


def test_mutation_estimate_dropped_gamma_caught(monkeypatch):
    """f(A^T A) v written as rho S_+ Z alone (the gamma v term dropped)."""
    monkeypatch.setattr(O, "shifted_moment_operator", lambda q, Splus, Z, V: q.rho * (Splus @ Z))
    assert estimate_errors("linear")[0] > 1e-3
    assert estimate_errors("nt")[0] > 1e-3


def test_mutation_estimate_log_of_sigma_caught(monkeypatch):
    """g^{-1} applied to sigma instead of sigma^2 in the NT form."""
    orig = O.spectral_map
    monkeypatch.setattr(O, "spectral_map", lambda v, x: orig(v, x) if v == "linear" else np.log(np.sqrt(x)))
    assert estimate_errors("nt")[0] > 1e-3


# Steps 3-5 (truncation, qr(A V~), SVD of B, tau, residuals): each planted mistake must
# make a pin above fail.
def _svd_B(B):
    return np.linalg.svd(B)


@pytest.mark.parametrize("kind", ["Q_not_transposed", "P_transposed"])
def test_mutation_ritz_factors_caught(monkeypatch, kind):
    """B = P Phi Q (G9) read the wrong way: v^ = V~ Q^T, or u^ = U~ P^T."""
    def ritz(Ut, B, Vt):
        P, phi, Qt = _svd_B(B)
        if kind == "Q_not_transposed":
            return phi, Ut @ P, Vt @ Qt, Qt
        return phi, Ut @ P.T, Vt @ Qt.T, Qt.T
    monkeypatch.setattr(O, "ritz_triplets", ritz)
    assert dense_triplet_errors("linear", 1)[0] != 6


def test_mutation_residual_without_sigma_caught(monkeypatch):
    monkeypatch.setattr(O, "exact_residuals", lambda A, uh, vh, phi, nA: (
        np.linalg.norm(A.T @ uh - vh, axis=0) / nA, np.linalg.norm(A @ vh - uh, axis=0) / nA))
    assert dense_triplet_errors("linear", 1)[0] != 6


@pytest.mark.parametrize("kind", ["arithmetic_mean", "not_relative"])
def test_mutation_tau_caught(monkeypatch, kind):
    def tau(Q, sS, r):
        if kind == "arithmetic_mean":
            return np.sum(Q * Q * sS[:r, None], axis=0) / np.sum(Q * Q, axis=0) / sS[0]
        return np.sum(Q * Q, axis=0) / np.sum(Q * Q / sS[:r, None], axis=0)
    monkeypatch.setattr(O, "spurious_index", tau)
    assert tau_special_case_error() > 1e-3


@pytest.mark.parametrize("kind", ["delta_absolute", "keep_every_column", "residual_not_normalised"])
def test_mutation_truncation_and_normalisation_caught(monkeypatch, kind):
    """delta read as absolute, no truncation at all (the paper's 1e-20 in effect), or the
    residual test without the division by ||A||_2: the 2000 x 1000 count changes."""
    if kind == "residual_not_normalised":
        monkeypatch.setattr(O, "exact_residuals", lambda A, uh, vh, phi, nA: (
            np.linalg.norm(A.T @ uh - vh * phi, axis=0), np.linalg.norm(A @ vh - uh * phi, axis=0)))
    else:
        def trunc(S, delta):
            US, sS, WSt = np.linalg.svd(S, full_matrices=False)
            r = int(np.count_nonzero(sS > delta)) if kind == "delta_absolute" else sS.size
            return US, sS, WSt, r
        monkeypatch.setattr(O, "truncate", trunc)
    assert c1_result()[0].sigma.size != 20


def test_mutation_iteration_skipped_caught(monkeypatch):
    """The iteration technique (Eqs. iter1-iter2) dropped: ell = 2 then gives only the ell = 1
    subspace, which misses the bound of Thm. 2 for ell = 2."""
    orig = O.moments
    monkeypatch.setattr(O, "moments", lambda solver, q, V, M, ell=1, scaled=True, extra=0:
                        orig(solver, q, V, M, 1, scaled, extra))
    assert theorem2_excess("linear", 2) > 1.0


# ---------------------------------------------------------------------------
# Largest singular values (expected values of an exterior interval at the top)
# ---------------------------------------------------------------------------
def test_largest_singular_values_against_dense_svd():
    """oracle.largest_singular_values (ARPACK on A^T A) against numpy's dense SVD on small
    instances of the banded-plus-random construction: the k largest values, descending."""
    for seed, (m, n, hw) in enumerate([(1200, 600, 40), (3000, 1000, 100)]):
        A = synth.banded_random(m, n, half_width=hw, seed=seed)
        d = np.linalg.svd(A.to_dense(), compute_uv=False)
        for k in (1, 12, 40):
            s = O.largest_singular_values(A, k)
            assert s.shape == (k,)
            assert np.all(np.diff(s) <= 0)
            assert np.max(np.abs(s - d[:k]) / d[:k]) < 1e-12


def test_exterior_interval_top_values_match_method():
    """For [a, b] with b above sigma_max the method (direct solves) returns exactly the values
    above a, which are the largest ones: the two oracles agree."""
    A = synth.banded_random(1500, 500, half_width=30, seed=5)
    top = O.largest_singular_values(A, 12)
    a, b = 0.5 * (top[9] + top[10]), 1.01 * top[0]
    r = O.solve_interval(A, a, b, 32, 16, 4, synth.gaussian_block(500, 16, 1), norm_A=top[0])
    assert r.sigma.size == 10
    assert np.max(np.abs(np.sort(r.sigma)[::-1] - top[:10]) / top[:10]) < 1e-12
