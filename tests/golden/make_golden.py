"""Writes the stored expected values under tests/golden/ from the oracle only.

h1_seed<seed>_s<s>_z<zeta>.txt: the first 64 columns of the sparse sign map
(§2.3.2, eq. (sparse-map)) under the counter hash H1 described in
oracle/hashing.py: per line, zeta row indices then zeta signs (+1/-1).
srht_rows_seed<seed>_np<n_p>_s<s>.txt: the SRHT's sampled Hadamard rows.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import hashing  # noqa: E402


def main():
    for seed, s, zeta in ((0, 80, 8), (7, 600, 12)):
        rows, signs = hashing.sparse_sign_indices(seed, 64, s, zeta)
        out = np.concatenate([rows, signs.astype(np.int64)], axis=1)
        np.savetxt(os.path.join(HERE, f"h1_seed{seed}_s{s}_z{zeta}.txt"), out, fmt="%d")
    for seed, n_p, s in ((7, 1 << 20, 600), (0, 1 << 12, 80)):
        rows = hashing.srht_rows(seed, n_p, s)
        np.savetxt(os.path.join(HERE, f"srht_rows_seed{seed}_np{n_p}_s{s}.txt"), rows, fmt="%d")


if __name__ == "__main__":
    main()
