"""Sketching maps: sparse sign embedding and SRHT, plus distortion measurement.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np
import scipy.sparse as sp

from . import hashing


def sparse_sign_matrix(seed, n, s, zeta):
    """S = (1/sqrt(zeta)) [s_1 ... s_n] as an s x n scipy CSC matrix.

    §2.3.2, eq. (sparse-map): column i has exactly zeta nonzero entries in
    distinct uniformly random rows; Rademacher (+-1) entries for the real
    field (§8.1.1).  The paper writes the scale as 1/sqrt(s); with zeta
    unit-modulus entries per column that gives E||Sx||^2 = (zeta/s)||x||^2,
    so the embedding would not be an approximate isometry.  This library
    reads the scale as 1/sqrt(zeta), the normalisation under which the
    distortion bound of Def. (subspace-embed) is meant; sGMRES/sRR outputs
    (y-hat, M-hat, Ritz values) are invariant to the scalar.
    """
    rows, signs = hashing.sparse_sign_indices(seed, n, s, zeta)
    cols = np.repeat(np.arange(n), zeta)
    vals = signs.reshape(-1) / np.sqrt(zeta)
    return sp.csc_matrix((vals, (rows.reshape(-1), cols)), shape=(s, n))


def sparse_sign_apply(seed, s, zeta, M):
    """S @ M for an n (or n x c) float64 array M."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    S = sparse_sign_matrix(seed, n, s, zeta)
    return S @ M


def fwht(x):
    """Unnormalised Walsh-Hadamard transform along axis 0 (Sylvester order).

    y[r] = sum_i (-1)^{popcount(r & i)} x[i]; length must be a power of two.
    Plain radix-2 butterflies, one stage per bit.
    """
    y = np.array(x, dtype=np.float64, copy=True)
    n = y.shape[0]
    rest = y.shape[1:]
    if n & (n - 1):
        raise ValueError("length must be a power of two")
    h = 1
    while h < n:
        y = y.reshape((n // (2 * h), 2, h) + rest)
        top = y[:, 0] + y[:, 1]
        bot = y[:, 0] - y[:, 1]
        y = np.stack([top, bot], axis=1).reshape((n,) + rest)
        h *= 2
    return y


def srht_apply(seed, s, M):
    """SRHT sketch sqrt(n_p/s) * D * H * E applied to the columns of M.

    §2.3.1, eq. (SRFT) with the unitary Walsh-Hadamard matrix H = H_raw/sqrt(n_p)
    standing in for the DFT (n zero-padded to n_p = 2^ceil(log2 n)), E the
    Rademacher diagonal and D the restriction to s distinct sampled rows.
    Output row q is Hadamard row rows[q].
    """
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    n_p = 1 << max(0, int(np.ceil(np.log2(max(n, 1)))))
    E = hashing.srht_signs(seed, n)
    pad = np.zeros((n_p,) + M.shape[1:])
    pad[:n] = (E.reshape((n,) + (1,) * (M.ndim - 1))) * M
    Hx = fwht(pad) / np.sqrt(n_p)
    rows = hashing.srht_rows(seed, n_p, s)
    return np.sqrt(n_p / s) * Hx[rows]


def apply(kind, seed, s, zeta, M):
    if kind == "sparse":
        return sparse_sign_apply(seed, s, zeta, M)
    if kind == "srht":
        return srht_apply(seed, s, M)
    raise ValueError(kind)


def distortion(SQ):
    """Distortion of S on range(Q) for orthonormal Q, from sigma(SQ).

    Def. (subspace-embed): (1-eps)||Qy|| <= ||SQy|| <= (1+eps)||Qy||, so
    eps = max(sigma_max - 1, 1 - sigma_min).
    """
    sv = np.linalg.svd(SQ, compute_uv=False)
    return max(sv[0] - 1.0, 1.0 - sv[-1]), sv
