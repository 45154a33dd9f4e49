"""Host-side checks of the seeded input generators (no GPU): the known-spectrum
constructions really have the spectrum they claim, the intervals hold the counts the
workloads state, and the generators are deterministic. The generators hold none of the
method's arithmetic; these tests pin the inputs that both the oracle and the GPU path use."""
import numpy as np

from paper_2109_13655_gb300 import synth


def test_block_permuted_spectrum_is_the_union_of_block_spectra():
    for dist in ("normal", "uniform_bf16"):
        bp = synth.block_permuted(40, 8, 4, seed=3, dist=dist)
        dense = np.linalg.svd(bp.A.to_dense(), compute_uv=False)
        assert np.max(np.abs(np.sort(dense)[::-1][:160] - bp.sigmas_desc())) < 1e-12 * dense[0]
        assert bp.A.nnz == 40 * 8 * 4 and bp.A.m == 320 and bp.A.n == 160
    bf = synth.block_permuted(10, 4, 2, seed=1, dist="uniform_bf16").A.vals
    assert np.array_equal(bf, synth.bf16_round(bf))            # values are bf16-representable


def test_generators_are_deterministic():
    a1, a2 = synth.random_sparse(300, 100, 6, seed=9), synth.random_sparse(300, 100, 6, seed=9)
    assert np.array_equal(a1.colidx, a2.colidx) and np.array_equal(a1.vals, a2.vals)
    assert np.all(np.diff(a1.rowptr) == 6)
    for i in range(a1.m):                                        # distinct, sorted columns per row
        c = a1.colidx[a1.rowptr[i]:a1.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    g1, g2 = synth.gaussian_block(50, 4, 3), synth.gaussian_block(50, 4, 3)
    assert np.array_equal(g1, g2) and g1.shape == (50, 4)


def test_window_interval_counts_and_gaps():
    s = np.sort(np.random.default_rng(0).uniform(0, 1, 500))[::-1]
    a, b, f = synth.window_interval(s, 100, 20, min_rel_gap=1e-4, max_shift=10)
    inside = np.nonzero((s >= a) & (s <= b))[0]
    assert inside.size == 20 and inside[0] == f
    assert (s[f - 1] - b) / b > 0 and (a - s[f + 20]) / a > 0


def test_model_problems_have_the_prescribed_spectrum():
    for which in (1, 2):
        A, sig = synth.model_problem(which)
        assert A.shape == (1000, 200)
        got = np.sort(np.linalg.svd(A, compute_uv=False))
        # a dense SVD resolves every sigma to ~u sigma_max (absolute), also model 2's 1e-10 ones
        assert np.max(np.abs(got - sig)) < 1e-14 * sig.max()


def test_batched_problems_counts():
    probs = synth.batched_problems(count=6, seed=13, n_min=2000, n_max=4000)
    for i, p in enumerate(probs):
        s = p["sigma"]
        assert p["A"].m == 10 * p["A"].n // 4 and p["A"].n % 4 == 0
        assert int(((s >= p["a"]) & (s <= p["b"])).sum()) == p["t"]
        assert p["N"] == 32 and p["M"] == 4 and p["L"] in (16, 32)
        assert p["kind"] == ("exterior" if i % 2 == 0 else "interior")
        assert abs(p["t"] - p["L"] * p["M"] // 3) <= 10


def test_banded_random_structure():
    """The 2e6 x 1e6 banded-plus-random construction (here at a small size): k_band columns
    within half_width of floor(i n / m), k_rand further distinct columns, sorted, bf16 values."""
    m, n, hw = 4000, 2000, 50
    A = synth.banded_random(m, n, half_width=hw, seed=3)
    assert (A.m, A.n, A.nnz) == (m, n, 16 * m)
    cols = A.colidx.reshape(m, 16).astype(np.int64)
    assert np.all(np.diff(cols, axis=1) > 0)
    c = (np.arange(m) * n) // m
    near = np.abs(cols - c[:, None]) <= hw
    assert np.all(near.sum(axis=1) >= 8)            # the 8 band columns (random ones may fall in too)
    assert np.all(synth.bf16_round(A.vals) == A.vals)
    assert np.all(np.abs(A.vals) <= 1.0)
    B = synth.banded_random(m, n, half_width=hw, seed=3)
    assert np.array_equal(A.colidx, B.colidx) and np.array_equal(A.vals, B.vals)
