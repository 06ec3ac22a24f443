"""RandOrth (Algorithm 2, Al Daas et al.) on explicit TT cores.

Right-to-left partial contraction (Eq. (3.2)):
  W^{(d-1)} = H(A_d) H(R_d)^T,
  V(Z_k) = V(A_k) W^{(k)},  W^{(k-1)} = H(Z_k) H(R_k)^T,
then left to right: QR of B^{(k)} W^{(k)}, M^{(k)} = Q^T B^{(k)},
H(B_{k+1}) = M^{(k)} H(A_{k+1}).

Applied to the explicit PKP cores of Y ⊙ Z this is the algebraic twin of
HaTT-1: the same sketches W^{(k)} and, with the same QR sign convention, the
same output cores (Section 3.1 derivation of Eq. (3.3)).
With normalize=True each W^{(k)} is divided by its Frobenius norm; that scales
C W by a positive constant and leaves Q unchanged.
"""
from __future__ import annotations

import numpy as np

from .tt import H, V


def qr_pos(a):
    """Thin Householder QR with the sign convention diag(R) >= 0."""
    q, r = np.linalg.qr(a)
    sgn = np.sign(np.diag(r))
    sgn[sgn == 0] = 1.0
    return q * sgn[None, :], r * sgn[:, None]


def partial_contraction_rl(A, R, normalize=True):
    """Sketches W[k] for bonds k = 1..d-1 (0-based core indexing: W[k] has
    shape (rank_k of A, ell_k) and contracts cores k..d-1). W[d] = [[1]]."""
    d = len(A)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1))
    for k in range(d - 1, 0, -1):
        a, n, b = A[k].shape
        Zk = (V(A[k]) @ W[k + 1]).reshape(a, n, W[k + 1].shape[1])   # V(Z_k) = V(A_k) W
        w = H(Zk) @ H(R[k]).T                                         # H(Z_k) H(R_k)^T
        if normalize:
            nw = np.linalg.norm(w)
            if nw > 0:
                w = w / nw
        W[k] = w
    return W


def randorth(A, R, normalize=True):
    """Algorithm 2. Returns (cores, W)."""
    d = len(A)
    W = partial_contraction_rl(A, R, normalize)
    B = [np.array(c, dtype=np.float64) for c in A]
    for k in range(d - 1):
        a, n, b = B[k].shape
        Bk = V(B[k])
        q, _ = qr_pos(Bk @ W[k + 1])
        M = q.T @ Bk
        B[k] = q.reshape(a, n, q.shape[1])
        a1, n1, b1 = A[k + 1].shape
        B[k + 1] = (M @ H(A[k + 1])).reshape(M.shape[0], n1, b1)
    return B, W
