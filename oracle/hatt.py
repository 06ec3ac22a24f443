"""HaTT-1 (Hadamard-avoiding TT recompression), plain float64 numpy.

Indexing is 0-based: core k has shape (r_k, n_k, r_{k+1}); bond k (1..d-1)
sits between cores k-1 and k. The sketch of bond k is
  W[k] = H(A_{k:d-1}) H(R_{k:d-1})^T,  shape (r_k s_k, l_k)      (Eq. (3.1))
with A = Y ⊙ Z never formed: entries of the PKP cores are products
Y_k(alpha, i, alpha') Z_k(beta, i, beta') with the combined index alpha*s+beta.

Readings of the paper taken here (the paper is silent or fixed-rank only):
  * ranks are clamped, l_k = min(l_req, r_k s_k, n_0..n_{k-1}, n_k..n_{d-1}),
    then l_k <= l_{k-1} n_{k-1} (left to right) and l_k <= n_k l_{k+1}
    (right to left), so every economy QR of Algorithm 4 is well posed;
  * each W[k] is divided by its Frobenius norm (a positive scale of C W, so
    Q is unchanged) to keep the chain in range;
  * QR uses the sign convention diag(R) >= 0;
  * an optional truncation sweep (right to left, SVD of each H(X_k) of the
    left-orthogonal result) enforces max_rank / tol with
    delta = tol * ||X|| / sqrt(d-1);
  * low-precision sketches (not in the paper, which is FP64 throughout) are
    emulated by rounding every operand of the three HPCRL-1 products to the
    named format and accumulating exactly in float64; everything after the
    sketches stays float64.
"""
from __future__ import annotations

import numpy as np

from . import philox
from .randorth import qr_pos
from .rounding import choose_rank
from .tt import H, V, pkp_core

_BIG = 1 << 62


def plan_ranks(n, r, s, ell_req):
    """Sketch / target ranks l_0..l_d for HaTT (the clamps described above)."""
    d = len(n)
    ell = [1] * (d + 1)
    for k in range(1, d):
        left = 1
        for v in n[:k]:
            left = min(left * int(v), _BIG)
        right = 1
        for v in n[k:]:
            right = min(right * int(v), _BIG)
        ell[k] = int(min(int(ell_req), int(r[k]) * int(s[k]), left, right))
    for k in range(1, d):
        ell[k] = min(ell[k], ell[k - 1] * int(n[k - 1]))
    for k in range(d - 1, 0, -1):
        ell[k] = min(ell[k], int(n[k]) * ell[k + 1])
    return ell


def requested_sketch_rank(r, s, max_rank=0, sketch_rank=0, oversample=10):
    """l before clamping: sketch_rank if given, else max_rank + oversample,
    else the PKP rank max_k r_k s_k (exact recompression)."""
    if sketch_rank > 0:
        return int(sketch_rank)
    if max_rank > 0:
        return int(max_rank) + int(oversample)
    return max(int(a) * int(b) for a, b in zip(r, s))


# ---------------------------------------------------------------- HPCRL-1 ---

def hpcrl1_wlwr(Y, Z, R, normalize=True):
    """HPCRL-1 in the paper's W_L / W_R form (Eq. (3.4)-(3.5) with S = I,
    Algorithm 3). For each column index (i, gamma):
      U_gamma = W^{(k)}(:, gamma) folded to s_k x r_k  (U_gamma[beta', alpha'] =
                W[alpha' s_k + beta', gamma]),
      W_L(:, (i, gamma)) = vec(Z_k(i) U_gamma Y_k(i)^T)   (column-major vec),
      W_R(:, (i, gamma)) = R_k(i)(:, gamma),
    and W^{(k-1)} = W_L W_R^T. Returns W[0..d] with W[d] = [[1]]."""
    d = len(Y)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1))
    for k in range(d - 1, 0, -1):
        yk, zk, rk = Y[k], Z[k], R[k]
        r0, n, r1 = yk.shape
        s0, _, s1 = zk.shape
        l0, _, l1 = rk.shape
        Wn = W[k + 1]
        WL = np.empty((r0 * s0, n * l1))
        WR = np.empty((l0, n * l1))
        for i in range(n):
            for g in range(l1):
                Ug = Wn[:, g].reshape(r1, s1).T              # s1 x r1
                P = zk[:, i, :] @ Ug @ yk[:, i, :].T          # s0 x r0
                WL[:, i * l1 + g] = P.reshape(-1, order="F")  # vec: index alpha*s0 + beta
                WR[:, i * l1 + g] = rk[:, i, g]
        w = WL @ WR.T
        if normalize:
            nw = np.linalg.norm(w)
            if nw > 0:
                w = w / nw
        W[k] = w
    return W


FORMATS = ("fp64", "fp32", "tf32", "bf16")


def round_operand(x, fmt="fp64"):
    """The value a low-precision multiplier receives for the float64 x:
    float64 -> binary32 (round to nearest even), then
      tf32: 10 explicit mantissa bits, round to nearest, ties away from zero;
      bf16: 7 explicit mantissa bits (the top half of binary32), round to
            nearest, ties to even.
    Both are written on the binary32 bit pattern: adding half of the dropped
    part (plus the kept lsb for ties-to-even) and clearing the dropped bits."""
    if fmt == "fp64":
        return np.asarray(x, dtype=np.float64)
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    if fmt == "fp32":
        return f.astype(np.float64)
    u = f.view(np.uint32).astype(np.uint64)
    if fmt == "tf32":
        u = (u + 0x1000) & 0xFFFFE000
    elif fmt == "bf16":
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    else:
        raise ValueError(fmt)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def hpcrl1_contract(Y, Z, R, normalize=True, fmt="fp64"):
    """HPCRL-1 as a plain index contraction in three stages (Eq. (3.6)):
      T1[a', b', i, l] = sum_g  W[a' s + b', g] R_k(l, i, g)
      T2[a', b,  i, l] = sum_b' Z_k(b, i, b') T1[a', b', i, l]
      W'[a s + b, l]   = sum_{a', i} Y_k(a, i, a') T2[a', b, i, l].
    With fmt != "fp64" every operand of the three products is rounded by
    round_operand (exact float64 accumulation)."""
    q = lambda x: round_operand(x, fmt)
    d = len(Y)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1))
    for k in range(d - 1, 0, -1):
        yk, zk, rk = Y[k], Z[k], R[k]
        r0, n, r1 = yk.shape
        s0, _, s1 = zk.shape
        l0, _, l1 = rk.shape
        Wm = W[k + 1].reshape(r1, s1, l1)
        T1 = np.einsum("abg,lig->abil", q(Wm), q(rk))
        T2 = np.einsum("cib,abil->acil", q(zk), q(T1))
        T3 = np.einsum("xia,acil->xcl", q(yk), q(T2))
        w = T3.reshape(r0 * s0, l0)
        if normalize:
            nw = np.linalg.norm(w)
            if nw > 0:
                w = w / nw
        W[k] = w
    return W


def hpcrl2(Y, Z, R, ep, normalize=True):
    """HPCRL-2 (Eq. (3.7), Algorithm 3 with the truncated SVD): at each step
    W^{(k)} = U S V^T is cut to the R singular values above ep * ||W^{(k)}||_2
    and the recursion runs on the R rank-one terms,
      W_L(:, (i, g)) = vec(Z_k(i) U_g Y_k(i)^T),  W_R(:, (i, g)) = R_k(i) V(:, g) s_g,
      W^{(k-1)} = W_L W_R^T.
    Reading: the returned sketches are the matrices the recursion computes
    (l columns each); the truncation only shortens the next contraction.
    Returns (W, Rk) with Rk[k] the rank kept when forming W^{(k-1)}."""
    d = len(Y)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1))
    kept = [0] * (d + 1)
    for k in range(d - 1, 0, -1):
        yk, zk, rk = Y[k], Z[k], R[k]
        r0, n, r1 = yk.shape
        s0, _, s1 = zk.shape
        l0, _, l1 = rk.shape
        Wn = W[k + 1]
        u, sv, vt = np.linalg.svd(Wn, full_matrices=False)
        Rn = max(1, int(np.sum(sv > ep * sv[0]))) if sv[0] > 0 else 1
        kept[k + 1] = Rn
        WL = np.empty((r0 * s0, n * Rn))
        WR = np.empty((l0, n * Rn))
        for i in range(n):
            for g in range(Rn):
                Ug = u[:, g].reshape(r1, s1).T                  # s1 x r1
                P = zk[:, i, :] @ Ug @ yk[:, i, :].T            # s0 x r0
                WL[:, i * Rn + g] = P.reshape(-1, order="F")    # index alpha * s0 + beta
                WR[:, i * Rn + g] = rk[:, i, :] @ vt[g] * sv[g]
        w = WL @ WR.T
        if normalize:
            nw = np.linalg.norm(w)
            if nw > 0:
                w = w / nw
        W[k] = w
    return W, kept


# ----------------------------------------------------- left-to-right pass ---

def core_update_paper(M, yk, zk):
    """Eq. (3.10): X_{k+1}(gamma, i, :) = vec(Z_{k+1}(i)^T M_gamma Y_{k+1}(i))^T,
    M_gamma = M(gamma, :) folded to s_k x r_k."""
    r0, n, r1 = yk.shape
    s0, _, s1 = zk.shape
    L = M.shape[0]
    out = np.empty((L, n, r1 * s1))
    for g in range(L):
        Mg = M[g].reshape(r0, s0).T                       # s0 x r0
        for i in range(n):
            P = zk[:, i, :].T @ Mg @ yk[:, i, :]          # s1 x r1
            out[g, i, :] = P.reshape(-1, order="F")       # index alpha'*s1 + beta'
    return out


def core_update_contract(M, yk, zk):
    """The same update as an index contraction:
    C[g, i, a' s' + b'] = sum_{a, b} M[g, a s + b] Y(a, i, a') Z(b, i, b')."""
    r0, n, r1 = yk.shape
    s0, _, s1 = zk.shape
    L = M.shape[0]
    Mm = M.reshape(L, r0, s0)
    U1 = np.einsum("gab,bic->gaic", Mm, zk)               # over beta
    C = np.einsum("gaic,aix->gixc", U1, yk)               # over alpha
    return C.reshape(L, n, r1 * s1)


def hatt1_sweep(Y, Z, W, paper_form=False):
    """Algorithm 4 left-to-right pass: X_1 = Y_1 ⊠ Z_1; for k: QR of C_k W^{(k)},
    M = Q^T C_k, C_{k+1} = M x (Y_{k+1} ⊠ Z_{k+1}) without forming the PKP core.
    Returns the left-orthogonal cores X (last core carries the norm)."""
    d = len(Y)
    if d == 1:
        return [Y[0] * Z[0]]
    update = core_update_paper if paper_form else core_update_contract
    C = pkp_core(Y[0], Z[0])
    X = []
    for k in range(d - 1):
        a, n, _ = C.shape
        Cm = V(C)
        q, _ = qr_pos(Cm @ W[k + 1])
        M = q.T @ Cm
        X.append(q.reshape(a, n, q.shape[1]))
        C = update(M, Y[k + 1], Z[k + 1])
    X.append(C)
    return X


# ------------------------------------------------------------- truncation ---

def truncate_rl(X, max_rank=0, tol=0.0):
    """Right-to-left truncation of a left-orthogonal TT: SVD of H(X_k),
    keep rho by `choose_rank`, X_k <- V^T, X_{k-1} <- X_{k-1} U Sigma.
    Returns (cores, ranks)."""
    X = [np.array(c, dtype=np.float64) for c in X]
    d = len(X)
    if d == 1:
        return X, [1, 1]
    nrm = float(np.linalg.norm(X[-1]))
    delta = tol * nrm / np.sqrt(d - 1)
    for k in range(d - 1, 0, -1):
        a, n, b = X[k].shape
        u, sv, vt = np.linalg.svd(H(X[k]), full_matrices=False)
        rho = choose_rank(sv, delta, max_rank)
        X[k] = vt[:rho].reshape(rho, n, b)
        X[k - 1] = np.einsum("aib,bc->aic", X[k - 1], u[:, :rho] * sv[None, :rho])
    return X, [1] + [int(c.shape[2]) for c in X]


# ------------------------------------------------------------ end to end ---

def hadamard_recompress(Y, Z, max_rank=0, tol=0.0, sketch_rank=0, oversample=10,
                        seed=0, normalize=True, coding="contract", return_info=False,
                        fmt="fp64", variant=1, ep=0.0):
    """Recompress Y ⊙ Z with HaTT-1 (Algorithm 4) and the optional truncation.

    coding="contract" uses the three-stage contraction for HPCRL and the core
    update; coding="paper" uses the W_L/W_R form and Eq. (3.10)."""
    d = len(Y)
    n = [int(c.shape[1]) for c in Y]
    r = [int(Y[0].shape[0])] + [int(c.shape[2]) for c in Y]
    s = [int(Z[0].shape[0])] + [int(c.shape[2]) for c in Z]
    lreq = requested_sketch_rank(r, s, max_rank, sketch_rank, oversample)
    ell = plan_ranks(n, r, s, lreq)
    R = philox.sketch_tt(seed, n, ell)
    if variant == 2:
        W, _ = hpcrl2(Y, Z, R, ep, normalize)
    elif coding == "paper":
        W = hpcrl1_wlwr(Y, Z, R, normalize)
    else:
        W = hpcrl1_contract(Y, Z, R, normalize, fmt)
    X = hatt1_sweep(Y, Z, W, paper_form=(coding == "paper"))
    cap = int(max_rank) if max_rank > 0 else 0
    need_trunc = d > 1 and (tol > 0 or (cap > 0 and any(e > cap for e in ell)))
    if need_trunc:
        X, out_r = truncate_rl(X, cap, tol)
    else:
        out_r = [1] + [int(c.shape[2]) for c in X]
    if return_info:
        return X, dict(ell=ell, R=R, W=W, ranks=out_r)
    return X
