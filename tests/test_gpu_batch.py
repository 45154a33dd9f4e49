"""Batched solves (cmsvd_solve_batch): many independent block-permuted problems spread over
several contexts (streams) run concurrently from one call. Each problem's result must be
the same alone and in the batch, bit for bit, because every kernel is deterministic and
contexts share no state. The counts and sigma are checked against the closed-form spectra,
and two problems against the oracle."""
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


def test_batch_equals_alone(B):
    probs = synth.batched_problems(count=8, seed=11, n_min=2000, n_max=8000)
    ctxs = [B.Context(torch.cuda.Stream()) for _ in range(4)]
    mats = [B.Matrix.from_csr(ctxs[i % 4], p["A"]) for i, p in enumerate(probs)]
    items = []
    for M, p in zip(mats, probs):
        prm = B.params(N=p["N"], L=p["L"], M=p["M"], norm_A=float(p["sigma"][0]))
        V = torch.from_numpy(synth.gaussian_block(p["A"].n, p["L"], p["seed_v"])).cuda()
        items.append((M, p["a"], p["b"], prm, V))
    torch.cuda.synchronize()
    alone = [M.solve_interval(a, b, prm, V) for (M, a, b, prm, V) in items]
    torch.cuda.synchronize()
    batch = B.solve_batch(items)
    torch.cuda.synchronize()
    for p, x, y in zip(probs, alone, batch):
        s = p["sigma"]
        truth = np.sort(s[(s >= p["a"]) & (s <= p["b"])])
        assert x.sigma.size == y.sigma.size == truth.size == p["t"]
        assert np.array_equal(x.sigma, y.sigma) and np.array_equal(x.V, y.V) and np.array_equal(x.U, y.U)
        assert np.max(np.abs(y.sigma - truth) / truth) <= 1e-10
        assert y.res_u.max() <= 1e-10 and y.res_v.max() <= 1e-10
    for i in (0, 1):   # one exterior and one interior problem against the oracle
        p = probs[i]
        ref = O.solve_interval(p["A"], p["a"], p["b"], p["N"], p["L"], p["M"],
                               synth.gaussian_block(p["A"].n, p["L"], p["seed_v"]), norm_A=float(p["sigma"][0]))
        assert ref.sigma.size == batch[i].sigma.size
        assert np.max(np.abs(batch[i].sigma - ref.sigma) / ref.sigma) <= 1e-10
    for M in mats:
        M.close()
    for c in ctxs:
        c.close()


def test_batch_reports_failing_problem(B):
    """A problem with invalid arguments fails alone; the others still run and return."""
    probs = synth.batched_problems(count=3, seed=12, n_min=2000, n_max=3000)
    ctxs = [B.Context(torch.cuda.Stream()) for _ in range(2)]
    mats = [B.Matrix.from_csr(ctxs[i % 2], p["A"]) for i, p in enumerate(probs)]
    items = []
    for k, (M, p) in enumerate(zip(mats, probs)):
        prm = B.params(N=p["N"], L=p["L"], M=p["M"], norm_A=float(p["sigma"][0]))
        V = torch.from_numpy(synth.gaussian_block(p["A"].n, p["L"], p["seed_v"])).cuda()
        a, b = (p["a"], p["b"]) if k != 1 else (p["b"], p["a"])     # problem 1: a > b
        items.append((M, a, b, prm, V))
    ws = [M.workspace(prm) for (M, a, b, prm, V) in items]
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError):
        B.cmsvd_solve_batch([M.handle for (M, *_r) in items], [x[1] for x in items], [x[2] for x in items],
                            [x[3] for x in items], [x[4] for x in items], ws)
    for M in mats:
        M.close()
    for c in ctxs:
        c.close()
