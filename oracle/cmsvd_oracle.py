"""CPU FP64 oracle for the complex moment-based interior SVD (Imakura & Sakurai).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module. The library never calls
it: the product path runs on the GPU or fails.

It restates the paper's method in plain NumPy/SciPy, step by step, with no
blocking, fusion or reordering beyond what the method states:

* quadrature on an ellipse with the N-point trapezoidal rule (Sec. 4),
* one direct complex solve per quadrature point in the upper half plane,
  (s_j I - A^T A) Y_j = X (Alg. 1 steps 1-2; the paper also solves directly),
* moment accumulation with the conjugate-symmetry halving (Sec. 3.1),
* the iteration technique for ell > 1 (Eqs. iter1, iter2),
* rank truncation by an SVD with threshold delta (Eq. low-rank, Alg. 1 step 3),
* QR of A V~ (Eq. avub, Alg. 1 step 4),
* SVD of B and the Ritz triplets (Eq. bsvd, Alg. 1 step 5),
* the spurious-value index tau (Sec. 3.4.2) and exact residuals (Sec. 3.4.1).

For a matrix too large for direct solves (the 2e6 x 1e6 banded-plus-random case)
and an exterior interval [a, b] with b above sigma_max, the triplets the method
must return are the t largest singular triplets of A (Thm. 1 with Omega holding
the top of the spectrum). ``largest_singular_values`` computes those values
with a library Lanczos routine (ARPACK through scipy's eigsh on A^T A); it is
pinned against numpy's dense SVD on small instances of the same construction.

Readings of points the paper leaves open (each is stated where it is used):
the moment weights use the scaled nodes ((zeta_j - gamma)/rho)^k; delta and
the tau threshold are relative to the largest singular value of S^; a triplet
is "found" when sigma is in [a, b], it is not spurious, and its residual
||A^T u - sigma v|| / ||A||_2 is at most tol_triplet.

Every function is pinned by the non-GPU tests against facts the paper and the
mathematics fix (quadrature exactness, Prop. 1, closed-form moments from a
dense SVD, the contour-integral limit of Thm. 1, the error bound of Thm. 2,
dense-SVD triplets, tau on inputs solvable by hand, the statements of the
experiments of Sec. 4), and mutation tests show that planted mistakes in each
step make one of those pins fail.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.sparse import csgraph


# ---------------------------------------------------------------------------
# Quadrature (Sec. 4, experimental set-up; Alg. 1 and Alg. 2 inputs)
# ---------------------------------------------------------------------------
@dataclass
class Quadrature:
    variant: str          # "linear" (Alg. 1) or "nt" (Alg. 2, g(t) = exp(t))
    N: int
    alpha: float
    gamma: float
    rho: float
    theta: np.ndarray     # theta_j
    node: np.ndarray      # z_j (linear) or t_j (nt)
    shift: np.ndarray     # z_j (linear) or g(t_j) = exp(t_j) (nt)
    weight: np.ndarray    # omega_j (linear) or psi_j (nt)

    @property
    def scaled(self) -> np.ndarray:
        """(node_j - gamma) / rho = cos(theta_j) + i alpha sin(theta_j)."""
        return (self.node - self.gamma) / self.rho


def quadrature(a: float, b: float, N: int, variant: str = "linear",
               alpha: float = 0.1, full: bool = False) -> Quadrature:
    """Trapezoidal points on the ellipse around the target interval (Sec. 4).

    theta_j = 2 pi (j - 1/2) / N;  node_j = gamma + rho (cos theta_j + i alpha sin theta_j);
    omega_j = (rho / N)(alpha cos theta_j + i sin theta_j);  psi_j = omega_j exp(t_j).
    Linear (Alg. 1): gamma = (a^2 + b^2)/2, rho = (b^2 - a^2)/2, shift = z_j.
    NT (Alg. 2):     gamma = log a + log b, rho = log b - log a, shift = exp(t_j).
    ``full=False`` returns j = 1..N/2, the points with Im > 0; the point
    conjugate to j is N+1-j (the pairing reading of Sec. 3.1).
    """
    if not (0 <= a < b):
        raise ValueError("need 0 <= a < b")
    if N < 2 or N % 2:
        raise ValueError("N must be even and >= 2")
    count = N if full else N // 2
    j = np.arange(1, count + 1)
    theta = 2.0 * np.pi / N * (j - 0.5)
    if variant == "linear":
        gamma, rho = 0.5 * (a * a + b * b), 0.5 * (b * b - a * a)
    elif variant == "nt":
        if a <= 0:
            raise ValueError("the exp transform needs a > 0")
        gamma, rho = np.log(a) + np.log(b), np.log(b) - np.log(a)
    else:
        raise ValueError(variant)
    node = gamma + rho * (np.cos(theta) + 1j * alpha * np.sin(theta))
    omega = rho / N * (alpha * np.cos(theta) + 1j * np.sin(theta))
    if variant == "linear":
        shift, weight = node, omega
    else:
        shift = np.exp(node)
        weight = omega * np.exp(node)
    return Quadrature(variant, N, alpha, gamma, rho, theta, node, shift, weight)


def moment_factor(q: Quadrature, k: int, scaled: bool = True) -> np.ndarray:
    """Per-point factor of the k-th moment: ((node-gamma)/rho)^k, or node^k (literal)."""
    base = q.scaled if scaled else q.node
    return base ** k


def filter_value(sigma, q: Quadrature) -> np.ndarray:
    """f(sigma) = sum_{j=1}^N w_j / (s_j - sigma^2) (Sec. 3.2; f_g for the NT variant).

    Evaluated with the conjugate halving, 2 Re sum over the upper-half points.
    """
    s2 = np.asarray(sigma, dtype=np.float64)[..., None] ** 2
    return 2.0 * np.real(np.sum(q.weight / (q.shift - s2), axis=-1))


def moment_filter(sigma, q: Quadrature, k: int, scaled: bool = True) -> np.ndarray:
    """c_k(sigma) = 2 Re sum_j w_j m_j^k / (s_j - sigma^2): the scalar that multiplies
    v_i v_i^T V_in in S^_k when sigma = sigma_i (first equality of Prop. 1)."""
    s2 = np.asarray(sigma, dtype=np.float64)[..., None] ** 2
    return 2.0 * np.real(np.sum(q.weight * moment_factor(q, k, scaled) / (q.shift - s2), axis=-1))


# ---------------------------------------------------------------------------
# Direct shifted solves (Alg. 1 steps 1-2, solver as in Sec. 4: a direct solve)
# ---------------------------------------------------------------------------
def as_scipy(A) -> sp.csr_matrix:
    if sp.issparse(A):
        return sp.csr_matrix(A)
    if isinstance(A, np.ndarray):
        return sp.csr_matrix(A)
    # synth.CSR-like object
    return sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.m, A.n))


class ShiftedSolver:
    """Exact solves of (s I - A^T A) Y = X by dense LU on each connected component
    of the column graph of A (columns sharing a row are connected).

    A^T A is block diagonal over these components, so each block is solved
    exactly with no fill; a matrix with one component is solved densely.
    """

    def __init__(self, A, max_dense: int = 6000):
        A = as_scipy(A)
        m, n = A.shape
        self.n = n
        bip = sp.bmat([[None, A.T], [A, None]], format="csr")  # nodes: n cols, then m rows
        _, labels = csgraph.connected_components(bip, directed=False)
        col_lab = labels[:n]
        uniq, comp = np.unique(col_lab, return_inverse=True)
        order = np.argsort(comp, kind="stable")
        sizes = np.bincount(comp)
        if sizes.max() > max_dense:
            raise ValueError(f"component of size {sizes.max()} too large for a dense direct solve")
        starts = np.concatenate([[0], np.cumsum(sizes)])
        local = np.empty(n, dtype=np.int64)
        local[order] = np.arange(n) - starts[comp[order]]
        H = (A.T @ A).tocoo()
        # group components by size; each group is a batch of dense blocks
        self.groups = []
        for s in np.unique(sizes):
            cids = np.nonzero(sizes == s)[0]
            slot = -np.ones(sizes.size, dtype=np.int64)
            slot[cids] = np.arange(cids.size)
            cols = np.empty((cids.size, s), dtype=np.int64)
            sel = slot[comp] >= 0
            cols[slot[comp[sel]], local[sel]] = np.nonzero(sel)[0]
            Hb = np.zeros((cids.size, s, s))
            e = slot[comp[H.row]] >= 0
            Hb[slot[comp[H.row[e]]], local[H.row[e]], local[H.col[e]]] = H.data[e]
            self.groups.append((cols, Hb))

    def solve(self, shift: complex, X: np.ndarray) -> np.ndarray:
        """Y = (shift I - A^T A)^{-1} X for a real or complex n x L block X."""
        Y = np.zeros(X.shape, dtype=np.complex128)
        for cols, Hb in self.groups:
            s = cols.shape[1]
            Ms = shift * np.eye(s) - Hb
            Y[cols] = np.linalg.solve(Ms, X[cols].astype(np.complex128))
        return Y


# ---------------------------------------------------------------------------
# Moments (Alg. 1 / Alg. 2 steps 1-2, with the halving of Sec. 3.1)
# ---------------------------------------------------------------------------
def moments(solver: ShiftedSolver, q: Quadrature, V_in: np.ndarray, M: int,
            ell: int = 1, scaled: bool = True, extra: int = 0) -> np.ndarray:
    """S^(ell) = [S_0, ..., S_{M-1+extra}] (n x L(M+extra)).

    Step 1: S_0^(nu) = 2 Re sum_j w_j (s_j I - A^T A)^{-1} S_0^(nu-1), nu < ell.
    Step 2: S_k = 2 Re sum_j w_j m_j^k (s_j I - A^T A)^{-1} S_0^(ell-1).
    extra=1 adds S_M, the last block of S_+ (Sec. 3.4.1).
    """
    X = np.asarray(V_in, dtype=np.float64)
    for _ in range(ell - 1):
        acc = np.zeros_like(X)
        for j in range(q.shift.size):
            acc += 2.0 * np.real(q.weight[j] * solver.solve(q.shift[j], X))
        X = acc
    K = M + extra
    out = [np.zeros_like(X) for _ in range(K)]
    for j in range(q.shift.size):
        Y = solver.solve(q.shift[j], X)
        for k in range(K):
            out[k] += 2.0 * np.real(q.weight[j] * moment_factor(q, k, scaled)[j] * Y)
    return np.concatenate(out, axis=1)


# ---------------------------------------------------------------------------
# Rayleigh-Ritz extraction (Alg. 1 steps 3-5) and the practical techniques
# ---------------------------------------------------------------------------
@dataclass
class Result:
    sigma: np.ndarray        # found singular values, ascending
    U: np.ndarray            # m x t
    V: np.ndarray            # n x t
    res_u: np.ndarray        # ||A^T u - sigma v|| / ||A||_2
    res_v: np.ndarray        # ||A v - sigma u|| / ||A||_2
    tau: np.ndarray          # tau_i / sigma_S,1
    rank: int                # columns kept by the truncation
    sigma_S: np.ndarray      # singular values of S^
    S: np.ndarray            # the moment block S^ (n x LM), and S_M if requested
    all_phi: np.ndarray = field(default=None)    # every Ritz value, before selection
    all_tau: np.ndarray = field(default=None)
    all_res: np.ndarray = field(default=None)
    res_est: np.ndarray = field(default=None)    # residual estimate through S_+ (Sec. 3.4.1), / ||A||_2
    res_tilde: np.ndarray = field(default=None)  # ||r~_i|| / ||A||_2 before the NT scaling mu


def spectral_map(variant: str, x):
    """f in f(A^T A) S_k = rho S_{k+1} + gamma S_k: f(x) = x for the linear variant (Prop. 1)
    and f(x) = g^{-1}(x) = ln x for NT (Eq. sk=aks_nonlinear)."""
    return x if variant == "linear" else np.log(x)


def shifted_moment_operator(q: Quadrature, Splus: np.ndarray, Z: np.ndarray, V: np.ndarray) -> np.ndarray:
    """f(A^T A) V for V = S W_S1 Sigma_S1^{-1} Q = S Z (Eq. residual): rho S_+ Z + gamma V."""
    return q.rho * (Splus @ Z) + q.gamma * V


def truncate(S: np.ndarray, delta: float):
    """Alg. 1 step 3 (Eq. low-rank): S = U_S Sigma_S W_S^T, keep sigma_S > delta * sigma_S,1
    (the relative reading of delta). Returns U_S, sigma_S, W_S^T and the kept rank r."""
    US, sS, WSt = np.linalg.svd(S, full_matrices=False)
    r = int(np.count_nonzero(sS > delta * sS[0]))
    return US, sS, WSt, r


def project(A, Vt: np.ndarray):
    """Alg. 1 step 4 (Eq. avub): [U~, B] = qr(A V~)."""
    return np.linalg.qr(A @ Vt)


def ritz_triplets(Ut: np.ndarray, B: np.ndarray, Vt: np.ndarray):
    """Alg. 1 step 5 (Eq. bsvd): B = P Phi Q^T and (sigma^, u^, v^) = (phi, U~ p, V~ q).
    Returns phi, u^, v^ and Q."""
    P, phi, Qt = np.linalg.svd(B)
    Q = Qt.T
    return phi, Ut @ P, Vt @ Q, Q


def spurious_index(Q: np.ndarray, sS: np.ndarray, r: int) -> np.ndarray:
    """Sec. 3.4.2: tau_i = q_i^T q_i / (q_i^T Sigma_S1^{-1} q_i), relative to sigma_S,1."""
    tau = np.sum(Q * Q, axis=0) / np.sum(Q * Q / sS[:r, None], axis=0)
    return tau / sS[0]


def exact_residuals(A, uh: np.ndarray, vh: np.ndarray, phi: np.ndarray, norm_A: float):
    """Sec. 3.4.1, first line: ||A^T u - sigma v|| / ||A||_2 and ||A v - sigma u|| / ||A||_2."""
    res_u = np.linalg.norm(A.T @ uh - vh * phi, axis=0) / norm_A
    res_v = np.linalg.norm(A @ vh - uh * phi, axis=0) / norm_A
    return res_u, res_v


def rayleigh_ritz(A, S: np.ndarray, a: float, b: float, L: int, M: int, delta: float,
                  eps_tau: float, tol_triplet: float, norm_A: float,
                  q: Quadrature | None = None, S_plus_last: np.ndarray | None = None) -> Result:
    """Alg. 1 steps 3-5 on the moment block S, the tau test and the exact residuals."""
    A = as_scipy(A)
    US, sS, WSt, r = truncate(S, delta)
    Vt = US[:, :r]
    Ut, B = project(A, Vt)
    phi, uh, vh, Q = ritz_triplets(Ut, B, Vt)
    tau_rel = spurious_index(Q, sS, r)
    res_u, res_v = exact_residuals(A, uh, vh, phi, norm_A)
    # Residual estimate through S_+ (Sec. 3.4.1). With scaled moment nodes the shifted
    # moments satisfy  f(A^T A) S'_k = rho S'_{k+1} + gamma S'_k,  with f(x) = x for the
    # linear variant (Prop. 1, exact) and f(x) = g^{-1}(x) = ln x for NT (approximate,
    # Eq. sk=aks_nonlinear). Since U_S1 = S' W_S1 Sigma_S1^{-1}:
    #   f(A^T A) v = rho S'_+ W_S1 Sigma_S1^{-1} q + gamma v,   v = U_S1 q,
    #   r~_i = || f(A^T A) v_i - f(sigma_i^2) v_i || / sigma_i      (Eq. residual).
    # Linear: ||r_i|| = ||r~_i||. NT (Eq. res_nonlinear): ||r_i|| ~ mu ||r~_i|| with mu the
    # ratio of one exact residual to its r~; the paper leaves the index i' open, and the
    # candidate (in [a, b], not spurious) with the largest ||r~|| is taken.
    res_est = rt = None
    if S_plus_last is not None and q is not None:
        Splus = np.concatenate([S[:, L:], S_plus_last], axis=1)
        Wm = WSt[:r].T / sS[:r]
        FV = shifted_moment_operator(q, Splus, Wm @ Q, vh)
        fphi = spectral_map(q.variant, np.maximum(phi, 1e-300) ** 2)
        rt = np.linalg.norm(FV - vh * fphi, axis=0) / np.maximum(phi, 1e-300)
        if q.variant == "linear":
            res_est = rt / norm_A
        else:
            cand = np.nonzero((phi >= a) & (phi <= b) & (tau_rel >= eps_tau))[0]
            res_est = np.full(phi.size, np.nan)
            if cand.size:
                ip = cand[np.argmax(rt[cand])]
                if rt[ip] > 0:
                    res_est = res_u[ip] * (rt / rt[ip])
    keep = (phi >= a) & (phi <= b) & (tau_rel >= eps_tau) & (res_u <= tol_triplet)
    idx = np.nonzero(keep)[0]
    idx = idx[np.argsort(phi[idx], kind="stable")]
    U_out, V_out = uh[:, idx].copy(), vh[:, idx].copy()
    # sign rule: the largest-magnitude entry of each v is positive (first one on ties)
    for c in range(idx.size):
        p = int(np.argmax(np.abs(V_out[:, c])))
        if V_out[p, c] < 0:
            V_out[:, c] *= -1.0
            U_out[:, c] *= -1.0
    return Result(phi[idx], U_out, V_out, res_u[idx], res_v[idx], tau_rel[idx], r, sS, S,
                  all_phi=phi, all_tau=tau_rel, all_res=res_u,
                  res_est=None if res_est is None else res_est[idx],
                  res_tilde=None if rt is None else rt[idx] / norm_A)


def solve_interval(A, a: float, b: float, N: int, L: int, M: int, V_in: np.ndarray,
                   ell: int = 1, delta: float = 1e-12, eps_tau: float = 1e-8,
                   variant: str = "linear", alpha: float = 0.1, tol_triplet: float = 1e-10,
                   norm_A: float | None = None, scaled: bool = True,
                   solver: ShiftedSolver | None = None, with_estimate: bool = False) -> Result:
    """Algorithm 1 (variant='linear') or Algorithm 2 (variant='nt'), end to end."""
    A = as_scipy(A)
    if V_in.shape != (A.shape[1], L):
        raise ValueError("V_in must be n x L")
    if M > N - 1:
        raise ValueError("M must be <= N-1 (Prop. 1)")
    if norm_A is None:
        norm_A = float(np.linalg.norm(A.toarray(), 2))
    q = quadrature(a, b, N, variant, alpha)
    solver = solver or ShiftedSolver(A)
    S_all = moments(solver, q, V_in, M, ell, scaled, extra=1 if with_estimate else 0)
    S = S_all[:, :L * M]
    S_last = S_all[:, L * M:] if with_estimate else None
    return rayleigh_ritz(A, S, a, b, L, M, delta, eps_tau, tol_triplet, norm_A, q, S_last)


# ---------------------------------------------------------------------------
# Largest singular values (the expected values for an exterior interval at the top)
# ---------------------------------------------------------------------------
def largest_singular_values(A, k: int, tol: float = 1e-14) -> np.ndarray:
    """The k largest singular values of A, descending.

    For [a, b] with b > sigma_max, the singular values in [a, b] are the largest ones
    (problem statement, Sec. 1), so this is the oracle of the method's values there when
    the direct solves of ``ShiftedSolver`` are out of reach. ARPACK's implicitly restarted
    Lanczos (scipy.sparse.linalg.eigsh) on A^T A, applied as A^T (A x) and never formed;
    sigma = sqrt(lambda).
    """
    from scipy.sparse.linalg import LinearOperator, eigsh
    A = as_scipy(A)
    At = A.T.tocsr()
    n = A.shape[1]
    H = LinearOperator((n, n), matvec=lambda x: At @ (A @ x), dtype=np.float64)
    v0 = np.ones(n) / np.sqrt(n)
    lam = eigsh(H, k=k, which="LA", tol=tol, v0=v0, ncv=min(n, max(2 * k + 1, k + 64)),
                return_eigenvectors=False)
    return np.sqrt(np.sort(np.maximum(lam, 0.0))[::-1])
