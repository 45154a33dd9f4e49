"""cmsvd_gram_noalloc: the allocation-free Gram entry point.

Callers that cannot allocate device memory at call time (memory owned by
another allocator, real-time loops where an allocation would synchronize the
device) call it without a workspace; its scratch is a fixed array inside the
library. This file checks it against cmsvd_gram, the entry point with a caller
workspace, on two calls in a row, and that sizes beyond the array are rejected.
It is named to run last, and also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n,c1,c2,same", [(5000, 64, 64, True), (3001, 80, 7, False), (20000, 512, 512, True),
                                          (20000, 512, 300, False), (1, 3, 5, False), (3000, 1, 4096, False)])
def test_noalloc_matches_workspace_gram(B, ctx, n, c1, c2, same):
    rng = np.random.default_rng(n + c1 + c2)
    X = torch.from_numpy(rng.standard_normal((n, c1))).cuda()
    Y = X if same else torch.from_numpy(rng.standard_normal((n, c2))).cuda()
    ref = torch.empty((c1, c2), dtype=torch.float64, device="cuda")
    ws = torch.empty(B.cmsvd_gram_workspace_size(ctx.handle, n, c1, c2), dtype=torch.uint8, device="cuda")
    B.cmsvd_gram(ctx.handle, X, Y, ref, ws)
    scale = (X.abs().T @ Y.abs()).cpu().numpy()
    for _ in range(2):          # two calls in a row share the fixed scratch
        G = torch.full((c1, c2), float("nan"), dtype=torch.float64, device="cuda")
        B.cmsvd_gram_noalloc(ctx.handle, X, Y, G)
        torch.cuda.synchronize()
        assert np.max(np.abs(G.cpu().numpy() - ref.cpu().numpy()) / scale) < 1e-13


def test_noalloc_rejects_oversize(B, ctx):
    X = torch.zeros((4, 1025), dtype=torch.float64, device="cuda")
    G = torch.zeros((1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(B.CmsvdError) as e:
        B.cmsvd_gram_noalloc(ctx.handle, X, X, G)
    assert e.value.status == B.INVALID_ARG
    # the same column limit as cmsvd_gram (c2 <= 4096), whatever c1 * c2
    X1 = torch.zeros((4, 1), dtype=torch.float64, device="cuda")
    Y1 = torch.zeros((4, 4097), dtype=torch.float64, device="cuda")
    G1 = torch.zeros((1, 4097), dtype=torch.float64, device="cuda")
    with pytest.raises(B.CmsvdError) as e:
        B.cmsvd_gram_noalloc(ctx.handle, X1, Y1, G1)
    assert e.value.status == B.INVALID_ARG


def test_noalloc_restores_current_device(B, ctx):
    """The call makes the context's device current only while it runs."""
    X = torch.ones((64, 8), dtype=torch.float64, device="cuda")
    G = torch.empty((8, 8), dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    B.cmsvd_gram_noalloc(ctx.handle, X, X, G)
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == before
    assert torch.allclose(G, torch.full((8, 8), 64.0, dtype=torch.float64, device="cuda"))
