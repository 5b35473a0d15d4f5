"""Counter-based hash H1 that places the nonzeros of the sketching maps.

Test infrastructure only (see oracle/__init__.py).

The paper (§2.3.2, eq. (sparse-map)) asks for a sparse map whose columns are
statistically independent and carry exactly zeta nonzeros in uniformly random
coordinates; for the real field the entries are Rademacher signs (§8.1.1).  It
does not fix a generator.  H1 is this library's definition, implemented here
and, independently, in the CUDA library; both must agree bit for bit:

  mix64(z)   : the SplitMix64 output finalizer (Steele, Lea & Flood 2014):
               z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
               z *= 0x94D049BB133111EB; z ^= z>>31            (mod 2^64)
  key        = (seed * 0x9E3779B97F4A7C15) XOR (i<<8 | t<<4 | a)   (mod 2^64)
  x          = mix64(key)
  row        = ((x mod 2^32) * s) >> 32            (multiply-shift range map)
  sign       = +1 if bit 63 of x is 0 else -1

  i = column (coordinate) index, t = slot (0 <= t < zeta <= 14), a = attempt.
  Slot t of column i takes the first attempt a = 0,1,...,15 whose row differs
  from the rows of slots 0..t-1 ("exactly zeta nonzeros" read as zeta distinct
  rows).  Slot value 15 is reserved for the SRHT sign of coordinate i and slot
  value 14 (with i = step q) for the SRHT row sampler below.

SRHT (§2.3.1, eq. (SRFT), with the Walsh-Hadamard transform in place of the
DFT and Rademacher E as in §8.1.1):
  E_i   = sign of mix64(key(seed, i, 15, 0))
  rows  = the first s entries of a partial Fisher-Yates shuffle of 0..n_p-1:
          for q = 0..s-1: x = mix64(key(seed, q, 14, 0));
          j = q + (((x mod 2^32) * (n_p - q)) >> 32); swap(perm[q], perm[j])
"""
import numpy as np

M64 = (1 << 64) - 1
PHI64 = 0x9E3779B97F4A7C15
MIX_C1 = 0xBF58476D1CE4E5B9
MIX_C2 = 0x94D049BB133111EB
MAX_ATTEMPTS = 16
MAX_ZETA = 14
SRHT_SIGN_SLOT = 15
SRHT_ROW_SLOT = 14


def mix64(z):
    """SplitMix64 finalizer on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(MIX_C1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(MIX_C2)
        z ^= z >> np.uint64(31)
    return z


def seed_key(seed):
    return np.uint64((int(seed) * PHI64) & M64)


def h1(seed, i, t, a):
    """x = mix64(seed*phi XOR (i<<8 | t<<4 | a)) for arrays i (broadcast t, a)."""
    i = np.asarray(i, dtype=np.uint64)
    low = (i << np.uint64(8)) | (np.uint64(t) << np.uint64(4)) | np.asarray(a, dtype=np.uint64)
    return mix64(seed_key(seed) ^ low)


def row_of(x, s):
    return ((x & np.uint64(0xFFFFFFFF)) * np.uint64(s)) >> np.uint64(32)


def sign_of(x):
    return np.where((x >> np.uint64(63)) == 0, 1.0, -1.0)


def sparse_sign_indices(seed, n, s, zeta, i0=0):
    """Rows (n x zeta, int64) and signs (n x zeta, +-1.0) of columns i0..i0+n-1.

    §2.3.2: column i of S has zeta nonzeros in distinct uniformly random rows.
    """
    if not (1 <= zeta <= MAX_ZETA) or zeta > s:
        raise ValueError("need 1 <= zeta <= min(14, s)")
    i = np.arange(i0, i0 + n, dtype=np.uint64)
    rows = np.empty((n, zeta), dtype=np.int64)
    signs = np.empty((n, zeta), dtype=np.float64)
    for t in range(zeta):
        a = np.zeros(n, dtype=np.uint64)
        pending = np.ones(n, dtype=bool)
        for attempt in range(MAX_ATTEMPTS):
            idx = np.nonzero(pending)[0]
            if idx.size == 0:
                break
            x = h1(seed, i[idx], t, attempt)
            r = row_of(x, s).astype(np.int64)
            clash = np.zeros(idx.size, dtype=bool)
            for tp in range(t):
                clash |= rows[idx, tp] == r
            ok = ~clash
            rows[idx[ok], t] = r[ok]
            signs[idx[ok], t] = sign_of(x[ok])
            pending[idx[ok]] = False
        if pending.any():
            raise RuntimeError("sparse-sign hash: no distinct row after 16 attempts")
    return rows, signs


def srht_signs(seed, n):
    """Rademacher diagonal E of the SRHT for coordinates 0..n-1 (§2.3.1)."""
    return sign_of(h1(seed, np.arange(n, dtype=np.uint64), SRHT_SIGN_SLOT, 0))


def srht_rows(seed, n_p, s):
    """s distinct Hadamard rows out of n_p by a partial Fisher-Yates shuffle."""
    if s > n_p:
        raise ValueError("s > n_p")
    perm = {}
    out = np.empty(s, dtype=np.int64)
    for q in range(s):
        x = int(h1(seed, np.array([q], dtype=np.uint64), SRHT_ROW_SLOT, 0)[0])
        j = q + (((x & 0xFFFFFFFF) * (n_p - q)) >> 32)
        vq = perm.get(q, q)
        vj = perm.get(j, j)
        perm[q], perm[j] = vj, vq
        out[q] = vj
    return out


def default_zeta(d):
    """zeta = ceil(2 log(1 + d)) with the natural log (§2.3.2)."""
    return int(np.ceil(2.0 * np.log1p(d)))
