"""k-truncated Arnoldi, Chebyshev and block Chebyshev bases, Householder QR,
sGMRES (Algorithm 1, restarted and iterative) and GMRES.

Test infrastructure only (see oracle/__init__.py).

Everything is float64.  ``A`` is any object with ``A @ x`` (a scipy sparse
matrix or a dense array).  ``sketch`` is a callable mapping an n-vector or an
n x c array to its s-row sketch (oracle.sketch.*).
"""
import numpy as np


# ---------------------------------------------------------------------------
# Basis generation: §1.2.2 eq. (partorth), Algorithm 1 (truncated Arnoldi
# loop, "double Gram-Schmidt" implementation note), §4.2.
# ---------------------------------------------------------------------------
def _partorth(W, m, passes):
    """w = (I - W W^T) m by ``passes`` classical Gram-Schmidt passes against
    the columns of W (the k previous basis vectors); returns w, the summed
    coefficients h and ||w||."""
    w = m.copy()
    h = np.zeros(W.shape[1])
    for _ in range(passes):
        c = W.T @ w
        w = w - W @ c
        h += c
    return w, h, np.linalg.norm(w)


def trunc_arnoldi(A, r, d, k, passes=2, breakdown=1e-13):
    """Basis B = [b_1..b_d] and reduced matrix AB = [m_1..m_d].

    b_1 = r/||r||, m_1 = A b_1; for j = 2..d
        w_j = (I - b_{j-1}b_{j-1}^T - ... - b_{j-k}b_{j-k}^T) m_{j-1}
    with b_{-i} = 0 (only existing vectors), applied as ``passes`` classical
    Gram-Schmidt passes against the same vectors (2 = double Gram-Schmidt);
    b_j = w_j/||w_j||, m_j = A b_j.

    If ||w_j|| <= breakdown*||m_{j-1}||, A b_{j-1} lies (numerically) in the
    span of the basis: the Krylov space is invariant and the basis stops at
    d_used = j-1 columns.

    Returns B (n x d_used), M = AB (n x d_used), Hc (d_used+1 x d_used) with
    m_j = sum_i Hc[i, j] b_i (the truncated Hessenberg coefficients), d_used.
    """
    n = r.shape[0]
    B = np.zeros((n, d))
    M = np.zeros((n, d))
    Hc = np.zeros((d + 1, d))
    beta = np.linalg.norm(r)
    B[:, 0] = r / beta
    M[:, 0] = A @ B[:, 0]
    d_used = d
    for j in range(1, d):
        lo = max(0, j - k)
        w, h, nu = _partorth(B[:, lo:j], M[:, j - 1], passes)
        if nu <= breakdown * np.linalg.norm(M[:, j - 1]):
            d_used = j
            break
        Hc[lo:j, j - 1] = h
        Hc[j, j - 1] = nu
        B[:, j] = w / nu
        M[:, j] = A @ B[:, j]
    return B[:, :d_used], M[:, :d_used], Hc[: d_used + 1, :d_used], d_used


# ---------------------------------------------------------------------------
# Shifted-and-scaled Chebyshev basis: §4.3, eq. (Chebrecurse).
# ---------------------------------------------------------------------------
def chebyshev_basis(A, r, d, c, dx, dy=0.0):
    """Chebyshev basis of K_{d+1}(A; r) for a spectrum inside the rectangle
    [c - dx, c + dx] x [-dy, dy] (rho = max(dx, dy)):

        b_1 = r/||r||,   b_2 = (2 rho)^{-1} (A - c I) b_1,
        b_j = rho^{-1} [ (A - c I) b_{j-1} - (dx^2 - dy^2)/(4 rho) b_{j-2} ],

    every vector rescaled to unit norm after it has served in the recurrence.
    Returns B (n x (d+1), unit columns), M = A B[:, :d] (formed directly), and
    Hbar ((d+1) x d, tridiagonal) with A B[:, :d] = B Hbar, read off the
    recurrence: A u_1 = c u_1 + 2 rho u_2 and
    A u_j = c u_j + rho u_{j+1} + gamma u_{j-1} (gamma = (dx^2-dy^2)/(4 rho))
    for the unscaled vectors u, then rescaled by the norms.
    """
    rho = max(dx, dy)
    gamma = (dx * dx - dy * dy) / (4.0 * rho)
    n = r.shape[0]
    U = np.zeros((n, d + 1))
    U[:, 0] = r / np.linalg.norm(r)
    if d >= 1:
        U[:, 1] = (A @ U[:, 0] - c * U[:, 0]) / (2.0 * rho)
    for j in range(2, d + 1):
        U[:, j] = ((A @ U[:, j - 1] - c * U[:, j - 1]) - gamma * U[:, j - 2]) / rho
    sig = np.linalg.norm(U, axis=0)
    B = U / sig
    Hbar = np.zeros((d + 1, d))
    for j in range(d):
        Hbar[j, j] = c
        Hbar[j + 1, j] = (2.0 * rho if j == 0 else rho) * sig[j + 1] / sig[j]
        if j >= 1:
            Hbar[j - 1, j] = gamma * sig[j - 1] / sig[j]
    M = A @ B[:, :d]
    return B, M, Hbar


# ---------------------------------------------------------------------------
# Block Chebyshev basis: §7.5 (the recurrence of §4.3 on an n x b block).
# ---------------------------------------------------------------------------
def block_chebyshev_basis(A, Omega, p, c, dx, dy=0.0):
    """Block Chebyshev basis [B_1, ..., B_p] of K_p(A; Omega) for a spectrum
    inside [c - dx, c + dx] x [-dy, dy] (rho = max(dx, dy),
    gamma = (dx^2 - dy^2) / (4 rho)):

        B_1 = Omega,   B_2 = (2 rho)^{-1} (A - c I) Omega,
        B_j = rho^{-1} [ (A - c I) B_{j-1} - gamma B_{j-2} ],

    as printed (no rescaling).  Returns the n x (b p) matrix, block-major.
    """
    rho = max(dx, dy)
    gamma = (dx * dx - dy * dy) / (4.0 * rho)
    blocks = [np.array(Omega, dtype=np.float64, copy=True)]
    if p >= 2:
        blocks.append((A @ blocks[0] - c * blocks[0]) / (2.0 * rho))
    for _ in range(2, p):
        blocks.append(((A @ blocks[-1] - c * blocks[-1]) - gamma * blocks[-2]) / rho)
    return np.hstack(blocks)


# ---------------------------------------------------------------------------
# Dense Householder QR and the sketched least-squares solve: §3.3 eqs.
# (sgmres-yhat), (sgmres-rhat); Algorithm 1 (QR, triangular substitution).
# ---------------------------------------------------------------------------
def householder_qr(C):
    """Thin QR C = U T by Householder reflectors (no pivoting).

    Reflector j maps R[j:, j] to alpha e_1 with alpha = -sign(x_0)||x||.
    Returns (V, T): V[j] the unit reflector vector acting on rows j.., T the
    d x d upper triangle.
    """
    R = np.array(C, dtype=np.float64, copy=True)
    s, d = R.shape
    V = []
    for j in range(d):
        x = R[j:, j]
        nx = np.linalg.norm(x)
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            V.append(np.zeros_like(v))
            continue
        v /= nv
        R[j:, j:] -= 2.0 * np.outer(v, v @ R[j:, j:])
        V.append(v)
    return V, np.triu(R[:d, :d])


def apply_qt(V, g):
    """Q^T g for the reflectors of householder_qr (all s entries)."""
    z = np.array(g, dtype=np.float64, copy=True)
    for j, v in enumerate(V):
        z[j:] -= 2.0 * v * (v @ z[j:])
    return z


def form_u(V, s):
    """The s x d orthonormal factor U = H_1 ... H_d [I; 0]."""
    d = len(V)
    U = np.zeros((s, d))
    U[:d, :d] = np.eye(d)
    for j in reversed(range(d)):
        v = V[j]
        U[j:, :] -= 2.0 * np.outer(v, v @ U[j:, :])
    return U


def back_substitute(T, z):
    """Solve T y = z for upper-triangular T by substitution."""
    d = T.shape[0]
    y = np.zeros(d)
    for i in reversed(range(d)):
        y[i] = (z[i] - T[i, i + 1:] @ y[i + 1:]) / T[i, i]
    return y


def cond2(T):
    sv = np.linalg.svd(T, compute_uv=False)
    return np.inf if sv[-1] == 0 else sv[0] / sv[-1]


def sketched_ls(C, g, stab_tol=np.inf):
    """min ||C y - g|| via C = U T: y = T^{-1}(U^T g), rhat = ||(I-UU^T)g||.

    §3.3 eqs. (sgmres-yhat), (sgmres-rhat).  If kappa_2(T) > stab_tol the
    solve keeps only the longest leading block of columns whose triangle has
    kappa_2 <= stab_tol (§5.3: restart from the residual of the last
    acceptable basis; kappa_2 of a leading block is non-decreasing in its
    width, so the block is found by bisection).
    Returns y (length of C's columns, zero-padded), rhat, kappa_2(T), width.
    """
    s, d = C.shape
    V, T = householder_qr(C)
    z = apply_qt(V, g)
    kappa = cond2(T)
    width = d
    if kappa > stab_tol:
        lo, hi = 0, d  # cond(T[:lo,:lo]) <= tol < cond(T[:hi,:hi])
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if cond2(T[:mid, :mid]) <= stab_tol:
                lo = mid
            else:
                hi = mid
        width = max(lo, 1)
    y = np.zeros(d)
    y[:width] = back_substitute(T[:width, :width], z[:width])
    rhat = np.sqrt(np.sum(z[width:] ** 2))
    return y, rhat, kappa, width


# ---------------------------------------------------------------------------
# sGMRES: Algorithm 1 with the solution built from B (§3.2 eq. (sgmres),
# §3.3: x-hat = x_0 + B y-hat), restarted as in §3.5.
# ---------------------------------------------------------------------------
def sgmres_cycle(A, f, x, d, k, sketch, passes=2, stab_tol=1e14, breakdown=1e-13, cheb=None):
    """One cycle of Algorithm 1 from the current iterate x.  ``cheb`` =
    (c, dx, dy) takes the Chebyshev basis (§4.3) instead of truncated
    Arnoldi."""
    r = f - A @ x
    g = sketch(r)
    if cheb is not None:
        B, M, _ = chebyshev_basis(A, r, d, *cheb)
        B, d_used = B[:, :d], d
    else:
        B, M, _, d_used = trunc_arnoldi(A, r, d, k, passes=passes, breakdown=breakdown)
    C = sketch(M)
    y, rhat, kappa, width = sketched_ls(C, g, stab_tol)
    x_new = x + B @ y
    return x_new, dict(rhat=rhat, kappa=kappa, d_used=d_used, width=width, r0norm=np.linalg.norm(r))


def sgmres(A, f, x0, d, k, sketch, tol, maxit=10000, passes=2, stab_tol=1e14, breakdown=1e-13, cheb=None):
    """Restarted sGMRES (§3.5) until ||f - A x||/||f|| <= tol or maxit cycles.

    Returns x, relres history (one entry per cycle, after the cycle), infos.
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    fn = np.linalg.norm(f)
    hist = []
    infos = []
    rel = np.linalg.norm(f - A @ x) / fn
    cycles = 0
    while rel > tol and cycles < maxit:
        x, info = sgmres_cycle(A, f, x, d, k, sketch, passes, stab_tol, breakdown, cheb)
        rel = np.linalg.norm(f - A @ x) / fn
        hist.append(rel)
        infos.append(info)
        cycles += 1
    return x, hist, infos


# ---------------------------------------------------------------------------
# Iterative sGMRES (§5.2): each reduced-matrix column is sketched as soon as
# it exists, the QR of S(A B_j) grows by one Householder reflector, and the
# cycle stops on the residual estimate; adaptive restart (§5.3): the cycle
# also ends, one column early, when kappa_2(T_j) first exceeds stab_tol.
# ---------------------------------------------------------------------------
def sgmres_iterative_cycle(A, f, x, dmax, k, sketch, tol_rel, passes=2, stab_tol=1e14, breakdown=1e-13):
    """One cycle from the iterate x with at most dmax basis vectors.

    g = S r_0.  For j = 1, 2, ..: b_j from the truncated recurrence of eq.
    (partorth), m_j = A b_j, c_j = S m_j; reflectors H_1..H_{j-1} are
    applied to c_j, H_j is formed from its entries j.. (the new column of
    T_j is the top j entries), and z = H_j ... H_1 g.  Then
        y_j = T_j^{-1} z[:j],   rhat_j = ||z[j:]|| = ||(I - U_j U_j^T) g||.
    The cycle stops at the first j with rhat_j <= tol_rel * ||g|| (both
    sides are sketched norms, so the sketch's distortion cancels to first
    order; an absolute threshold on rhat_j alone lets a restart stop at j = 1
    without progress once ||S r|| < threshold < ||r||), at a breakdown of
    the recurrence (the Krylov space is invariant), at j = dmax, or -- when
    kappa_2(T_j) > stab_tol -- with the previous solution y_{j-1}.
    Returns x + B_j y_j and a dict: ``j`` (columns used), ``rhat`` (the
    estimate for every j formed), ``kappa`` (kappa_2(T_j) likewise),
    ``stop`` in {"tol", "kappa", "breakdown", "dmax"}, ``r0norm``.
    """
    r = f - A @ x
    g = sketch(r)
    n, s = r.shape[0], g.shape[0]
    if not 1 <= dmax < s:
        raise ValueError("need 1 <= dmax < s (the paper takes s = 2(dmax + 1))")
    B = np.zeros((n, dmax))
    T = np.zeros((dmax, dmax))
    z = np.array(g, dtype=np.float64, copy=True)
    gnorm = np.linalg.norm(g)
    V = []
    rhats, kappas = [], []
    y = np.zeros(0)
    stop = "dmax"
    B[:, 0] = r / np.linalg.norm(r)
    m = A @ B[:, 0]
    j = 0  # columns in the QR so far
    while True:
        c = np.array(sketch(m), dtype=np.float64, copy=True)
        for i, v in enumerate(V):
            c[i:] -= 2.0 * v * (v @ c[i:])
        v, alpha = _reflector(c[j:])
        T[:j, j] = c[:j]
        T[j, j] = alpha
        z[j:] -= 2.0 * v * (v @ z[j:])
        V.append(v)
        j += 1
        kappa = cond2(T[:j, :j])
        kappas.append(kappa)
        if kappa > stab_tol:
            j -= 1  # keep y_{j-1}: restart from the previous residual
            stop = "kappa"
            break
        y = back_substitute(T[:j, :j], z[:j])
        rhats.append(np.sqrt(np.sum(z[j:] ** 2)))
        if rhats[-1] <= tol_rel * gnorm:
            stop = "tol"
            break
        if j == dmax:
            break
        lo = max(0, j - k)
        w, _, nu = _partorth(B[:, lo:j], m, passes)
        if nu <= breakdown * np.linalg.norm(m):
            stop = "breakdown"
            break
        B[:, j] = w / nu
        m = A @ B[:, j]
    if stop == "kappa":
        y = back_substitute(T[:j, :j], z[:j])
    x_new = x + B[:, :j] @ y
    return x_new, dict(j=j, rhat=rhats, kappa=kappas, stop=stop, r0norm=np.linalg.norm(r))


def sgmres_iterative(A, f, x0, dmax, k, sketch, tol, maxit=10000, passes=2, stab_tol=1e14, breakdown=1e-13):
    """Restarted iterative sGMRES: cycles of sgmres_iterative_cycle, each
    asked for the reduction tol ||f|| / ||r_0|| that would meet the target,
    until ||f - A x||/||f|| <= tol or maxit cycles.  Returns x, the relres
    history (after each cycle) and the per-cycle infos."""
    x = np.array(x0, dtype=np.float64, copy=True)
    fn = np.linalg.norm(f)
    hist, infos = [], []
    rel = np.linalg.norm(f - A @ x) / fn
    while rel > tol and len(hist) < maxit:
        x, info = sgmres_iterative_cycle(A, f, x, dmax, k, sketch, tol / rel, passes, stab_tol, breakdown)
        rel = np.linalg.norm(f - A @ x) / fn
        hist.append(rel)
        infos.append(info)
    return x, hist, infos


# ---------------------------------------------------------------------------
# GMRES with the Householder Arnoldi process (§3.1, §4.2; Walker 1988): the
# classic O(nd^2) method sGMRES is compared with.
# ---------------------------------------------------------------------------
def _reflector(x):
    nx = np.linalg.norm(x)
    alpha = -nx if x[0] >= 0 else nx
    v = x.copy()
    v[0] -= alpha
    nv = np.linalg.norm(v)
    return (v / nv if nv > 0 else v), alpha


def gmres_householder(A, f, x0, d):
    """d steps of GMRES from x0; returns x_d and ||f - A x_d||.

    Householder Arnoldi: P_1 r_0 = beta e_1; for j = 1..d, q_j = P_1..P_j e_j,
    z = P_j..P_1 A q_j, P_{j+1} zeroes z below entry j+1, and column j of the
    (d+1) x d Hessenberg H is the top j+1 entries of P_{j+1} z.  Then
    y = argmin ||beta e_1 - H y|| and x_d = x_0 + [q_1..q_d] y.
    """
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[0]
    x0 = np.asarray(x0, dtype=np.float64)
    r0 = f - A @ x0
    refl = []  # (offset, v)

    def apply_p(z, upto):  # P_upto ... P_1 z
        z = z.copy()
        for off, v in refl[:upto]:
            z[off:] -= 2.0 * v * (v @ z[off:])
        return z

    def apply_p_rev(z, upto):  # P_1 ... P_upto z
        z = z.copy()
        for off, v in reversed(refl[:upto]):
            z[off:] -= 2.0 * v * (v @ z[off:])
        return z

    v, beta = _reflector(r0)
    refl.append((0, v))
    m = min(d, n)
    H = np.zeros((m + 1, m))
    Q = np.zeros((n, m))
    for j in range(m):
        e = np.zeros(n)
        e[j] = 1.0
        q = apply_p_rev(e, j + 1)
        Q[:, j] = q
        z = apply_p(A @ q, j + 1)
        if j + 1 < n:
            v, alpha = _reflector(z[j + 1:])
            refl.append((j + 1, v))
            z[j + 1:] = 0.0
            z[j + 1] = alpha
        top = min(j + 2, n)
        H[:top, j] = z[:top]
    rhs = np.zeros(m + 1)
    rhs[0] = beta
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    x = x0 + Q @ y
    return x, np.linalg.norm(f - A @ x)
