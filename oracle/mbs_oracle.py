"""Plain, slow, FP64 CPU implementation of the paper's multibody MFS solve.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

What it follows, step by step, in the paper's order and notation:

  phi            fundamental solution phi_kappa                (Sec. 3.1, eq. FundamentalSol)
  cpqr_id        column-pivoted QR of B halted at k or eps,
                 interpolative decomposition B ~ B(:,I) Z*     (Sec. 4.2, eq. B_fac)
  cpqr_id_sketch the same ID computed from a Gaussian sketch Omega B
                 (randomized ID of the ID framework the paper
                 cites for Sec. 4.2; Omega from philox4x32_10 and
                 gaussian_sketch, a counter-based generator from
                 its published definition)
  tsvd_solve     backward-stable least squares by truncated SVD (Sec. 3.1; Sec. 4.3-4.4)
  build_shape    S = Z* C A^+ U, W = Z* C A^+                  (Sec. 4.2-4.5, eq. scattering-matrix)
  layout         skeleton points x_hat of every placed body    (Sec. 4.2; reuse of S per shape, Sec. 5.1 Ex. 4)
  G_dense / G_matvec   G_hat(i,j) = phi(x_hat_i - x_hat_j), zero diagonal blocks
                                                               (Sec. 1 eq. Gmtx-entries; Sec. 2.2 eq. mbody2)
  apply_operator q -> q + S G_hat q                            (Sec. 2.2, eq. mbody2)
  rhs            b_tau = Z* C A^+ v_tau  (= S v_hat)           (Sec. 4.5, last display)
  solve_dense    (I + S G_hat) q_hat = b by LU                 (Sec. 2.2)
  gmres          unrestarted GMRES, MGS Arnoldi + Givens       (Sec. 2.4; Saad & Schultz 1986)
  field          u(x) = sum_i phi(x - x_hat_i) q_hat_i          (Sec. 4.1, eq. out_skel)
  reconstruct_mfs  q_mfs_tau = A^+ (v_tau - U_tau G_hat_{tau,tau^c} q_hat_{tau^c})
                                                               (Sec. 4.6, MFS-surface reconstruction)
  field_near     u(x) anywhere outside the MFS curves: skeleton sums of the bodies
                 whose proxy surface x lies outside, MFS sums of the one it lies in
                                                               (Sec. 4.6)

Readings where the paper is silent:
  * pivot rule: largest remaining column norm, recomputed in full at every
    step; ties (norm >= (1 - 1e-10) * max) go to the lowest original index;
  * eps mode stops when the largest remaining column norm is <= eps times the
    largest initial column norm;
  * A^+ and the "stabilised" C use a truncated SVD with relative cutoff 1e-14;
  * the right-hand side uses all m collocation values: b = Z* C A^+ v.

Pins (tests, -m "not gpu"): separation-of-variables closed forms for a circle
(2D) and a sphere (3D), reciprocity, dense LU vs GMRES, a brute-force global
MFS on tiny inputs, the ID identities, rigid-motion invariance, and textbook
values of H0; for the reconstruction, the circle series between Gamma and the
proxy, the sound-soft condition on Gamma between collocation points (and its
spectral decay), and agreement of MFS and skeleton sources away from a body;
for the randomized ID, the generator's published known-answer vectors, the
moments of the Gaussian sketch, exactness on low-rank matrices, the identity
sketch reducing to the pivoted-QR ID, and an ID error within a small factor of
the deterministic one.  No function here is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
from scipy.special import hankel1

__all__ = [
    "phi", "kernel_matrix", "cpqr_id", "cpqr_id_sketch", "philox4x32_10", "gaussian_sketch", "tsvd_solve", "tsvd_pinv", "build_shape", "build_all",
    "layout", "apply_W", "G_dense", "G_matvec", "G_rows", "apply_operator", "rhs", "solve_dense", "gmres",
    "field", "solve_workload", "incoming_on_boundary", "reconstruct_mfs", "field_near",
    "proxy_body",
]

TIE_TOL = 1e-10
LS_RCOND = 1e-14


# ----------------------------------------------------------------------------
# Sec. 3.1: the fundamental solution
# ----------------------------------------------------------------------------
def phi(dim: int, kappa: float, r):
    """phi_kappa at distance r: (i/4) H0^(1)(kappa r) in 2D, e^{i kappa r}/(4 pi r) in 3D."""
    r = np.asarray(r, dtype=np.float64)
    if dim == 2:
        return 0.25j * hankel1(0, kappa * r)
    return np.exp(1j * kappa * r) / (4.0 * math.pi * r)


def _dist(T: np.ndarray, S: np.ndarray) -> np.ndarray:
    diff = T[:, None, :] - S[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=2))


def kernel_matrix(dim: int, kappa: float, targets: np.ndarray, sources: np.ndarray) -> np.ndarray:
    """Matrix with entries phi(t_i - s_j) (the A, B, D matrices of Sec. 4)."""
    return phi(dim, kappa, _dist(targets, sources))


# ----------------------------------------------------------------------------
# Sec. 4.2: skeletons by column-pivoted QR, converted to an ID
# ----------------------------------------------------------------------------
def cpqr_id(B: np.ndarray, k: int = 0, eps: float = 0.0, tie_tol: float = TIE_TOL):
    """Householder QR of B with column pivoting, halted at rank k (k > 0) or once
    the largest remaining column norm falls to eps times the largest initial
    one.  Returns (skel, Zs, perm, R, eps_achieved):

      skel = the first k pivot columns (the skeleton index vector I_hat),
      Zs   = Z* (k x m) with Zs[:, skel] = I_k and Zs[:, perm[k:]] = R11^{-1} R12,
             so that B ~ B[:, skel] @ Zs,
      eps_achieved = largest remaining column norm / largest initial norm.
    """
    A = np.array(B, dtype=np.complex128, copy=True)
    p, m = A.shape
    perm = np.arange(m)
    nmax0 = float(np.max(np.linalg.norm(A, axis=0)))
    kmax = min(p, m)
    rank = kmax
    eps_ach = 0.0
    for j in range(kmax):
        cn = np.linalg.norm(A[j:, j:], axis=0)  # full recomputation, no downdating
        mx = float(cn.max())
        eps_ach = mx / nmax0
        if (k > 0 and j == k) or (k <= 0 and mx <= eps * nmax0):
            rank = j
            break
        cand = np.nonzero(cn >= (1.0 - tie_tol) * mx)[0]
        q = int(cand[np.argmin(perm[j + cand])]) + j
        if q != j:
            A[:, [j, q]] = A[:, [q, j]]
            perm[[j, q]] = perm[[q, j]]
        x = A[j:, j].copy()
        nx = np.linalg.norm(x)
        ph = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -ph * nx
        v = x
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv > 0:
            v /= nv
            A[j:, j:] -= 2.0 * np.outer(v, v.conj() @ A[j:, j:])
        A[j + 1:, j] = 0.0
        A[j, j] = alpha
    else:
        eps_ach = 0.0
    if k > 0:
        rank = min(k, kmax)
    R = np.triu(A[:rank, :])
    T = sla.solve_triangular(R[:, :rank], R[:, rank:], lower=False)
    Zs = np.zeros((rank, m), dtype=np.complex128)
    Zs[:, perm[:rank]] = np.eye(rank)
    Zs[:, perm[rank:]] = T
    return perm[:rank].copy(), Zs, perm, R, eps_ach


# ----------------------------------------------------------------------------
# Randomized ID: the skeleton from a Gaussian sketch of B
# ----------------------------------------------------------------------------
_PHILOX_M = (0xD2511F53, 0xCD9E8D57)
_PHILOX_W = (0x9E3779B9, 0xBB67AE85)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11): ctr is
    (..., 4) and key (..., 2), unsigned 32-bit; returns (..., 4) uint32.  Each
    round multiplies counter words 0 and 2 by the two constants, swaps and
    xors the high halves with the other words and the key; the key is bumped
    by the two Weyl constants between rounds."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    m32 = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(_PHILOX_W[0])) & m32
            k1 = (k1 + np.uint64(_PHILOX_W[1])) & m32
        p0 = np.uint64(_PHILOX_M[0]) * c[0]
        p1 = np.uint64(_PHILOX_M[1]) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & m32, (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & m32]
    return np.stack(c, axis=-1).astype(np.uint32)


def gaussian_sketch(d: int, p: int, seed: int, shape_index: int) -> np.ndarray:
    """d x p complex Gaussian test matrix (unit variance: real and imaginary
    parts N(0, 1/2)).  Entry (i, l) takes counter (l, i, 0, 0) and key
    (seed, shape_index); the four output words give two 53-bit uniforms
    u = (w_a 2^21 + floor(w_b / 2^11) + 1/2) 2^-53 in (0, 1), and the
    Box-Muller transform gives sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2)."""
    ii, ll = np.meshgrid(np.arange(d), np.arange(p), indexing="ij")
    ctr = np.stack([ll, ii, np.zeros_like(ii), np.zeros_like(ii)], axis=-1).astype(np.uint64)
    key = np.empty(ii.shape + (2,), dtype=np.uint64)
    key[..., 0] = seed & 0xFFFFFFFF
    key[..., 1] = shape_index & 0xFFFFFFFF
    w = philox4x32_10(ctr, key).astype(np.uint64)
    two53 = 2.0 ** -53
    u1 = ((w[..., 0] << np.uint64(21)) + (w[..., 1] >> np.uint64(11))).astype(np.float64) * two53 + 0.5 * two53
    u2 = ((w[..., 2] << np.uint64(21)) + (w[..., 3] >> np.uint64(11))).astype(np.float64) * two53 + 0.5 * two53
    rad = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * math.pi * u2
    return (rad * np.cos(th) + 1j * rad * np.sin(th)) / math.sqrt(2.0)


def cpqr_id_sketch(B: np.ndarray, k: int, Omega: np.ndarray, tie_tol: float = TIE_TOL):
    """Randomized interpolative decomposition: the column-pivoted QR of the
    sketch Y = Omega B (d x m, d >= k rows, Omega a Gaussian test matrix),
    halted at k, gives the skeleton I_hat and Z* = [I | R11^{-1} R12] of Y,
    which is also an ID of B: B ~ B(:, I_hat) Z* (the columns of Y are the
    columns of B seen through Omega, so a column subset that spans Y's
    columns spans B's to about the same error).  Returns what cpqr_id does."""
    return cpqr_id(Omega @ B, k=k, tie_tol=tie_tol)


# ----------------------------------------------------------------------------
# Sec. 3.1 / 4.3 / 4.4: backward-stable least squares (truncated SVD)
# ----------------------------------------------------------------------------
def _tsvd(A: np.ndarray, rcond: float = LS_RCOND):
    """Thin SVD of A keeping singular values above rcond * s_max."""
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    r = int(np.sum(s > rcond * s[0]))
    return U[:, :r], s[:r], Vh[:r]


def tsvd_solve(A: np.ndarray, Y: np.ndarray, rcond: float = LS_RCOND) -> np.ndarray:
    """Minimum-norm solution of A X = Y with singular values below rcond * s_max
    dropped; the projections U^H Y are formed before the division by s."""
    U, s, Vh = _tsvd(A, rcond)
    return Vh.conj().T @ ((U.conj().T @ Y) / s[:, None])


def tsvd_pinv(A: np.ndarray, rcond: float = LS_RCOND) -> np.ndarray:
    """Truncated-SVD pseudo-inverse A^+ (n x m for an m x n matrix)."""
    return tsvd_solve(A, np.eye(A.shape[0], dtype=np.complex128), rcond)


# ----------------------------------------------------------------------------
# Sec. 4.2-4.5: the local scattering matrix of one shape
# ----------------------------------------------------------------------------
def build_shape(dim: int, kappa: float, x, y, z, k: int = 0, eps: float = 0.0,
                rcond: float = LS_RCOND, sketch=None) -> dict:
    """S = Z* C A^+ U (k x k) and W = Z* C A^+ (k x m) for one shape.

    B(i,j) = phi(z_i - x_j) (p x m, eq. B-matrix); CPQR/ID of B gives I_hat and Z*;
    U = conj(Z) = (Z*)^T (Sec. 4.2); A(i,j) = phi(x_i - y_j) (m x n, Sec. 4.3);
    D(i,j) = phi(z_i - y_j) (p x n) and C solves B C = D (Sec. 4.4)."""
    B = kernel_matrix(dim, kappa, z, x)
    if sketch is not None and k > 0 and k + sketch[2] < B.shape[0]:
        # randomized ID: sketch = (seed, shape index, oversampling)
        Omega = gaussian_sketch(k + sketch[2], B.shape[0], sketch[0], sketch[1])
        skel, Zs, perm, R, eps_ach = cpqr_id_sketch(B, k, Omega)
    else:
        skel, Zs, perm, R, eps_ach = cpqr_id(B, k=k, eps=eps)
    A = kernel_matrix(dim, kappa, x, y)
    D = kernel_matrix(dim, kappa, z, y)
    C = tsvd_solve(B, D, rcond)
    # Order of evaluation (a reading; the paper gives only the product):
    # A^+ = V diag(1/s) U_A^H is never formed on its own, since an explicit
    # pseudo-inverse of the ill-conditioned MFS matrix carries rounding of size
    # u / s_min in every direction.  S is formed as ((Z* C V) / s) (U_A^H U): the
    # division by s acts on the well-determined rows of Z* C V and is then
    # multiplied by the small projections of U on the rough modes.  The explicit
    # W = Z* C A^+ is kept for inspection only; right-hand sides are formed
    # right to left by apply_W.
    Ua, sa, Vh = _tsvd(A, rcond)
    U = Zs.T
    Gc = ((Zs @ C) @ Vh.conj().T) / sa[None, :]
    S = Gc @ (Ua.conj().T @ U)
    W = Gc @ Ua.conj().T
    return {"skel": skel, "Zs": Zs, "S": S, "W": W, "C": C, "B": B,
            "A_svd": (Ua, sa, Vh), "eps": eps_ach, "k": len(skel)}


def build_all(wl, sketch=None) -> list:
    """Scattering data for every distinct shape of a workload (reuse per shape, Sec. 5.1 Ex. 4).
    sketch = (seed, oversampling) selects the randomized ID for fixed-k shapes."""
    used = sorted(set(int(s) for s in wl.body_shape))
    out = [None] * len(wl.shapes)
    for s in used:
        sh = wl.shapes[s]
        sk = None if sketch is None else (sketch[0], s, sketch[1])
        out[s] = build_shape(wl.dim, wl.kappa, sh.x, sh.y, sh.z, k=sh.k, eps=sh.eps, sketch=sk)
    return out


# ----------------------------------------------------------------------------
# global system (Sec. 2.2)
# ----------------------------------------------------------------------------
def layout(wl, sdata) -> dict:
    """Skeleton points x_hat = c_tau + R_tau x_local(I_hat) of every body, in body order."""
    d = wl.dim
    pts, bid, off = [], [], [0]
    for t in range(wl.T):
        s = int(wl.body_shape[t])
        xl = wl.shapes[s].x[sdata[s]["skel"]]
        pts.append(wl.centres[t, :d] + xl @ wl.rots[t, :d, :d].T)
        bid.append(np.full(len(xl), t, dtype=np.int64))
        off.append(off[-1] + len(xl))
    return {"xhat": np.concatenate(pts), "body": np.concatenate(bid), "offsets": np.array(off)}


def G_dense(dim, kappa, xhat, body) -> np.ndarray:
    """Dense G_hat: phi between skeleton points of different bodies, zero diagonal blocks."""
    same = body[:, None] == body[None, :]
    r = _dist(xhat, xhat)
    r[same] = 1.0
    G = phi(dim, kappa, r)
    G[same] = 0.0
    return G


def G_rows(dim, kappa, xhat, body, q, rows) -> np.ndarray:
    """(G_hat q)[rows] for a list of target rows."""
    rows = np.asarray(rows)
    r = _dist(xhat[rows], xhat)
    same = body[rows][:, None] == body[None, :]
    r[same] = 1.0
    G = phi(dim, kappa, r)
    G[same] = 0.0
    return G @ q


def G_matvec(dim, kappa, xhat, body, q, chunk_elems: int = 4_000_000) -> np.ndarray:
    """Matrix-free G_hat q, in row chunks."""
    N = xhat.shape[0]
    q2 = q.reshape(N, -1)
    out = np.zeros_like(q2, dtype=np.complex128)
    step = max(1, chunk_elems // max(1, N))
    for a in range(0, N, step):
        rows = np.arange(a, min(N, a + step))
        out[rows] = G_rows(dim, kappa, xhat, body, q2, rows)
    return out.reshape(q.shape)


def _apply_blocks(wl, sdata, lay, name, X, rows_in):
    """Block-diagonal product: out_tau = M_{shape(tau)} X_tau, blocks of S (or W)."""
    outs = []
    off_in = 0
    for t in range(wl.T):
        M = sdata[int(wl.body_shape[t])][name]
        ni = rows_in[t]
        outs.append(M @ X[off_in:off_in + ni])
        off_in += ni
    return np.concatenate(outs, axis=0)


def apply_operator(wl, sdata, lay, q, G=None) -> np.ndarray:
    """(I + S G_hat) q  (eq. mbody2)."""
    Gq = G @ q if G is not None else G_matvec(wl.dim, wl.kappa, lay["xhat"], lay["body"], q)
    ks = np.diff(lay["offsets"])
    return q + _apply_blocks(wl, sdata, lay, "S", Gq, ks)


def apply_W(sd: dict, v: np.ndarray) -> np.ndarray:
    """Z* C A^+ v for one body, right to left: q_mfs = A^+ v as a solve, then C, then Z*."""
    Ua, sa, Vh = sd["A_svd"]
    qm = Vh.conj().T @ ((Ua.conj().T @ v) / sa[:, None])
    return sd["Zs"] @ (sd["C"] @ qm)


def rhs(wl, sdata, lay, v, explicit_W: bool = False) -> np.ndarray:
    """b_tau = Z* C A^+ v_tau (= S_tau v_hat_tau up to the ID error) with v = -u_inc at
    all m collocation points of body tau (Sec. 4.5, last display).  With
    explicit_W the stored matrix W is used instead (for injected-W tests)."""
    if explicit_W:
        return _apply_blocks(wl, sdata, lay, "W", v, wl.m_of_body())
    out, off = [], 0
    for t in range(wl.T):
        sd = sdata[int(wl.body_shape[t])]
        m = sd["Zs"].shape[1]
        out.append(apply_W(sd, v[off:off + m]))
        off += m
    return np.concatenate(out, axis=0)


def system_matrix(wl, sdata, lay) -> np.ndarray:
    G = G_dense(wl.dim, wl.kappa, lay["xhat"], lay["body"])
    Sblk = sla.block_diag(*[sdata[int(s)]["S"] for s in wl.body_shape])
    return np.eye(G.shape[0]) + Sblk @ G


def solve_dense(wl, sdata, lay, b) -> np.ndarray:
    """q_hat = (I + S G_hat)^{-1} b by LU (small N)."""
    return np.linalg.solve(system_matrix(wl, sdata, lay), b)


def gmres(matvec, b: np.ndarray, tol: float = 1e-13, maxiter: int | None = None):
    """Unrestarted GMRES for one right-hand side: modified Gram-Schmidt Arnoldi,
    Givens rotations on the Hessenberg matrix, stop when ||b - A x|| / ||b|| <= tol
    (the residual norm tracked by the rotations).  Returns (x, iterations, relres)."""
    N = b.shape[0]
    maxiter = maxiter or N
    beta = np.linalg.norm(b)
    if beta == 0:
        return np.zeros_like(b), 0, 0.0
    V = np.zeros((maxiter + 1, N), dtype=np.complex128)
    H = np.zeros((maxiter + 1, maxiter), dtype=np.complex128)
    cs = np.zeros(maxiter, dtype=np.complex128)
    sn = np.zeros(maxiter, dtype=np.complex128)
    g = np.zeros(maxiter + 1, dtype=np.complex128)
    g[0] = beta
    V[0] = b / beta
    j_done = 0
    rel = 1.0
    for j in range(maxiter):
        w = matvec(V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0:
            V[j + 1] = w / H[j + 1, j]
        # rotation i acts on rows (i, i+1) as [[conj(c), conj(s)], [-s, c]]
        for i in range(j):
            t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        a, bb = H[j, j], H[j + 1, j]
        den = math.sqrt(abs(a) ** 2 + abs(bb) ** 2)
        cs[j] = a / den if den else 1.0
        sn[j] = bb / den if den else 0.0
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = np.conj(cs[j]) * g[j]
        j_done = j + 1
        rel = abs(g[j + 1]) / beta
        if rel <= tol:
            break
    y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done], lower=False)
    x = V[:j_done].T @ y
    return x, j_done, rel


def field(dim, kappa, targets, xhat, qhat, chunk_elems: int = 4_000_000) -> np.ndarray:
    """Scattered field u(t) = sum_i phi(t - x_hat_i) q_hat_i (eq. out_skel)."""
    M = targets.shape[0]
    N = xhat.shape[0]
    q2 = qhat.reshape(N, -1)
    out = np.zeros((M, q2.shape[1]), dtype=np.complex128)
    step = max(1, chunk_elems // max(1, N))
    for a in range(0, M, step):
        b = min(M, a + step)
        out[a:b] = kernel_matrix(dim, kappa, targets[a:b], xhat) @ q2
    return out.reshape((M,) + qhat.shape[1:])


def incoming_on_boundary(wl, sdata, lay, qhat, v) -> np.ndarray:
    """Local incoming data w_tau = v_tau - sum_{sigma != tau} G_{tau,sigma} q_hat_sigma at the
    full collocation points of every body (eq. w_in, evaluated on Gamma_tau)."""
    d = wl.dim
    out = []
    off = 0
    xhat, body = lay["xhat"], lay["body"]
    q2 = qhat.reshape(xhat.shape[0], -1)
    for t in range(wl.T):
        X = wl.body_points(t, "x")
        r = _dist(X, xhat)
        K = phi(d, wl.kappa, np.where(body[None, :] == t, 1.0, r))
        K[:, body == t] = 0.0
        m = X.shape[0]
        out.append(v[off:off + m] - K @ q2)
        off += m
    return np.concatenate(out, axis=0)


def reconstruct_mfs(wl, sdata, lay, qhat, v) -> list:
    """Full local solution on the MFS curve/surface of every body (Sec. 4.6):
    q_mfs_tau = A_tau^+ (v_tau - U_tau G_hat_{tau,tau^c} q_hat_{tau^c}), where
    G_hat_{tau,tau^c} q_hat_{tau^c} is the incoming field at tau's skeleton points
    from every other body and U_tau = (Z*_tau)^T interpolates it to all m
    collocation points (Sec. 4.3, eq. inc_field).  A^+ is the truncated-SVD
    solve.  Returns one (n_tau, nrhs) array per body."""
    xhat, body = lay["xhat"], lay["body"]
    q2 = qhat.reshape(xhat.shape[0], -1)
    v2 = v.reshape(v.shape[0], -1)
    w_hat = G_matvec(wl.dim, wl.kappa, xhat, body, q2)
    out, voff = [], 0
    for t in range(wl.T):
        sd = sdata[int(wl.body_shape[t])]
        a, b = lay["offsets"][t], lay["offsets"][t + 1]
        m = sd["Zs"].shape[1]
        resid = v2[voff:voff + m] - sd["Zs"].T @ w_hat[a:b]
        Ua, sa, Vh = sd["A_svd"]
        out.append(Vh.conj().T @ ((Ua.conj().T @ resid) / sa[:, None]))
        voff += m
    return out


def proxy_body(wl, targets) -> np.ndarray:
    """Index of the body whose proxy surface strictly contains each target, or -1."""
    d = wl.dim
    tb = np.full(targets.shape[0], -1, dtype=np.int64)
    rp = wl.proxy_radius_of_body()
    for t in range(wl.T):
        inside = np.sum((targets - wl.centres[t, :d]) ** 2, axis=1) < rp[t] ** 2 * (1.0 - 1e-12)
        tb[inside] = t
    return tb


def field_near(wl, sdata, lay, qhat, qmfs, targets) -> np.ndarray:
    """Scattered field at targets anywhere outside the MFS curves (Sec. 4.6): a
    target inside the proxy surface of body tau gets the MFS sum of tau plus the
    skeleton sums (eq. out_skel) of every other body; any other target gets the
    skeleton sums of all bodies."""
    d = wl.dim
    xhat, body = lay["xhat"], lay["body"]
    q2 = qhat.reshape(xhat.shape[0], -1)
    tb = proxy_body(wl, targets)
    out = np.zeros((targets.shape[0], q2.shape[1]), dtype=np.complex128)
    for i in range(targets.shape[0]):
        x = targets[i:i + 1]
        t = tb[i]
        keep = body != t
        out[i] = (kernel_matrix(d, wl.kappa, x, xhat[keep]) @ q2[keep])[0]
        if t >= 0:
            qm = qmfs[t].reshape(qmfs[t].shape[0], -1)
            out[i] += (kernel_matrix(d, wl.kappa, x, wl.body_points(int(t), "y")) @ qm)[0]
    return out


def solve_workload(wl, method: str = "auto", tol: float = 1e-13, sketch=None):
    """Full oracle pipeline: S per shape, layout, b = W v, solve.  Returns a dict.
    sketch = (seed, oversampling): randomized ID (see build_all)."""
    sdata = build_all(wl, sketch=sketch)
    lay = layout(wl, sdata)
    v = wl.boundary_data()
    b = rhs(wl, sdata, lay, v)
    N = lay["xhat"].shape[0]
    if method == "auto":
        method = "lu" if N <= 8192 else "gmres"
    if method == "lu":
        q = solve_dense(wl, sdata, lay, b)
        its = [0] * b.shape[1]
    else:
        q = np.zeros_like(b)
        its = []
        G = G_dense(wl.dim, wl.kappa, lay["xhat"], lay["body"]) if N <= 8192 else None
        for c in range(b.shape[1]):
            mv = (lambda x: apply_operator(wl, sdata, lay, x[:, None], G)[:, 0])
            q[:, c], it, _ = gmres(mv, b[:, c], tol=tol)
            its.append(it)
    return {"sdata": sdata, "layout": lay, "v": v, "b": b, "q": q, "iterations": its}
