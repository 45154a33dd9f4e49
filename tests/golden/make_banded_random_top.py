"""Writes banded_random_2000000x1000000_top.txt: the 128 largest singular values of the
2e6 x 1e6 banded-plus-random matrix (synth.banded_random, seed 10), computed by the oracle
(oracle.largest_singular_values: ARPACK Lanczos on A^T A). These are the expected values of
an exterior interval at the top of its spectrum. Runs on the CPU only:

    python tests/golden/make_banded_random_top.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cmsvd_oracle as O  # noqa: E402
from paper_2109_13655_gb300 import synth  # noqa: E402

K = 128


def main():
    t0 = time.time()
    A = synth.banded_random()
    s = O.largest_singular_values(A, K)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "banded_random_2000000x1000000_top.txt")
    with open(out, "w") as f:
        f.write("# 128 largest singular values of synth.banded_random() (2000000 x 1000000, 16 nnz/row: 8 within\n")
        f.write("# +-5000 of the row's diagonal position, 8 uniform; U(-1,1) rounded to bf16; seed 10), descending.\n")
        f.write("# Written by tests/golden/make_banded_random_top.py with oracle.largest_singular_values\n")
        f.write("# (ARPACK Lanczos on A^T A, tol 1e-14): the expected values of an exterior interval at the top.\n")
        for v in s:
            f.write(f"{v:.17e}\n")
    print(f"wrote {out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
