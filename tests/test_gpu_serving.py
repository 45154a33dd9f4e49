"""Serving loop (cmsvd_server_*): requests on resident matrices, admitted in arrival order
as slots and HBM budget allow, overlapping on the GPU. Every result must be bit for bit
the result of the same request solved alone (deterministic kernels, no state shared
between slots), and match the closed-form spectrum."""
import numpy as np
import pytest

from paper_2109_13655_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_13655_gb300 import binding
    return binding


def resident_bytes(A):
    # A and A^T: row pointers, int32 columns, FP64 values and their FP32 copy
    return 8 * (A.m + A.n + 2) + 32 * A.nnz


def test_serving_mixed_equals_alone(B):
    rng = np.random.default_rng(21)
    mats = []
    for k, c in enumerate((8, 16, 8, 16)):
        nb = int(rng.integers(300, 1200))
        mats.append(synth.block_permuted(nb, 2 * c, c, seed=100 + k, dist="uniform_bf16"))
    reqs = []
    for i in range(18):
        mi = i % 4
        s = mats[mi].sigmas_desc()
        t = int(rng.integers(10, 41))
        first = int(rng.integers(t + 5, s.size - 2 * t - 5))
        a, b, _ = synth.window_interval(s, first, t, min_rel_gap=1e-6, max_shift=10)
        reqs.append((mi, a, b, t, 500 + i))
    p = B.params(N=32, L=32, M=4)
    # the budget holds the matrices and at most two requests at a time (three slots)
    ctx = B.Context()
    alone_mats = [B.Matrix.from_csr(ctx, bp.A) for bp in mats]
    ws_max = max(M.workspace(p).numel() for M in alone_mats) + 8 * max(bp.A.n for bp in mats) * 32
    budget = sum(resident_bytes(bp.A) for bp in mats) + int(2.5 * ws_max)
    srv = B.Server(slots=3, hbm_budget=budget)
    ids = [srv.add_matrix(bp.A) for bp in mats]
    tickets = []
    for (mi, a, b, t, seed) in reqs:
        V = synth.gaussian_block(mats[mi].A.n, 32, seed)
        tickets.append(srv.submit(ids[mi], a, b, p, V))
    results, queue_ms = [], []
    for tk, (mi, a, b, t, seed) in zip(tickets, reqs):
        done, nt, st, lat, q = srv.wait(tk)
        assert done and st in (B.OK, B.SUBSPACE_SATURATED) and lat >= q >= 0.0
        queue_ms.append(q)
        results.append(srv.take(tk, ids[mi], nt, st))
    srv.close()
    assert max(queue_ms) > 0.0
    for (mi, a, b, t, seed), r in zip(reqs, results):
        s = mats[mi].sigmas_desc()
        truth = np.sort(s[(s >= a) & (s <= b)])
        assert r.sigma.size == truth.size == t
        assert np.max(np.abs(r.sigma - truth) / truth) <= 1e-10
        assert r.res_u.max() <= 1e-10 and r.res_v.max() <= 1e-10
        V = torch.from_numpy(synth.gaussian_block(mats[mi].A.n, 32, seed)).cuda()
        alone = alone_mats[mi].solve_interval(a, b, p, V)
        assert np.array_equal(alone.sigma, r.sigma) and np.array_equal(alone.V, r.V) and np.array_equal(alone.U, r.U)
    for M in alone_mats:
        M.close()
    ctx.close()


def test_serving_rejects_oversized_and_unknown(B):
    bp = synth.block_permuted(200, 16, 8, seed=7, dist="uniform_bf16")
    srv = B.Server(slots=1, hbm_budget=resident_bytes(bp.A) + (1 << 20))
    mid = srv.add_matrix(bp.A)
    with pytest.raises(RuntimeError):
        srv.submit(mid, 0.1, 0.2, B.params(N=32, L=32, M=4), np.zeros((bp.A.n, 32)))   # workspace above the budget
    with pytest.raises(RuntimeError):
        srv.submit(mid + 5, 0.1, 0.2, B.params(), np.zeros((bp.A.n, 16)))
    with pytest.raises(RuntimeError):
        srv.wait(12345)
    srv.close()


def test_serving_matches_the_oracle(B):
    """Two requests served side by side on one resident matrix, each against the oracle's solve
    of the same problem (same A, interval, N, L, M and V_in): the exact count, sigma within
    1e-10, residuals <= 1e-10, and U, V within residual / gap of the oracle's vectors."""
    from oracle import cmsvd_oracle as O
    bp = synth.block_permuted(300, 16, 8, seed=41, dist="uniform_bf16")
    s = bp.sigmas_desc()
    p = B.params(N=32, L=32, M=4)
    reqs = []
    for k, (first, t) in enumerate(((60, 20), (900, 25))):
        a, b, _ = synth.window_interval(s, first, t, min_rel_gap=1e-6, max_shift=10)
        reqs.append((a, b, t, 700 + k))
    srv = B.Server(slots=2, hbm_budget=1 << 30)
    mid = srv.add_matrix(bp.A)
    tickets = [srv.submit(mid, a, b, p, synth.gaussian_block(bp.A.n, 32, seed)) for (a, b, t, seed) in reqs]
    results = []
    for tk in tickets:
        done, nt, st, lat, q = srv.wait(tk)
        assert done and st == B.OK
        results.append(srv.take(tk, mid, nt, st))
    srv.close()
    sp = np.sort(s)
    for (a, b, t, seed), r in zip(reqs, results):
        ref = O.solve_interval(bp.A, a, b, 32, 32, 4, synth.gaussian_block(bp.A.n, 32, seed), norm_A=s[0])
        assert r.sigma.size == ref.sigma.size == t
        assert np.max(np.abs(r.sigma - ref.sigma) / ref.sigma) <= 1e-10
        assert r.res_u.max() <= 1e-10 and r.res_v.max() <= 1e-10
        for i, sig in enumerate(ref.sigma):
            k = np.searchsorted(sp, sig)
            nb = sp[max(k - 2, 0):k + 2]
            nb = nb[np.abs(nb - sig) > 1e-13 * sig]
            gap = np.min(np.abs(nb - sig)) if nb.size else sig
            tol = max(1e-7, 10 * s[0] * (r.res_u[i] + ref.res_u[i] + 1e-16) / gap)
            assert np.max(np.abs(r.V[:, i] - ref.V[:, i])) <= tol
            assert np.max(np.abs(r.U[:, i] - ref.U[:, i])) <= tol
