"""TT tensor basics in plain float64 numpy (Section 2.1-2.2).

Layout: core k is an array (r_{k-1}, n_k, r_k). The multi-index is row-major
(last index fastest, Section 2.1), so the horizontal unfolding H(T) is
T.reshape(r_{k-1}, n_k r_k) and the vertical unfolding V(T) is
T.reshape(r_{k-1} n_k, r_k). The partial Kronecker product combines a Y index
alpha (slow) and a Z index beta (fast) as alpha*s + beta.
"""
from __future__ import annotations

import numpy as np


def ranks(cores):
    return [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]


def modes(cores):
    return [int(c.shape[1]) for c in cores]


def H(core):
    """Horizontal matricization (mode-1 unfolding) of a core."""
    a, n, b = core.shape
    return core.reshape(a, n * b)


def V(core):
    """Vertical matricization of a core."""
    a, n, b = core.shape
    return core.reshape(a * n, b)


def tt_full(cores):
    """Dense tensor from its TT cores, A(i_1..i_d) = A_1(i_1) ... A_d(i_d)
    (Eq. (2.2)); for tiny cases only."""
    t = cores[0]
    for c in cores[1:]:
        t = np.tensordot(t, c, axes=([t.ndim - 1], [0]))
    return t.reshape(t.shape[1:-1])


def pkp_core(yk, zk):
    """Partial Kronecker product along modes 1 and 3:
    (Y ⊠ Z)(alpha*s+beta, i, alpha'*s'+beta') = Y(alpha,i,alpha') Z(beta,i,beta')
    (Section 2.1)."""
    r0, n, r1 = yk.shape
    s0, n2, s1 = zk.shape
    assert n == n2
    out = np.einsum("aib,cid->acibd", yk, zk)
    return out.reshape(r0 * s0, n, r1 * s1)


def hadamard_pkp(Y, Z):
    """Exact TT of Y ⊙ Z with cores Y_k ⊠ Z_k and ranks r_k s_k (Section 2.2)."""
    assert len(Y) == len(Z)
    return [pkp_core(y, z) for y, z in zip(Y, Z)]


def tt_dot(A, B):
    """<A, B> = sum over all entries of A*B, by the left-to-right contraction
    G_k = sum_i A_k(i)^T G_{k-1} B_k(i), G_0 = [[1]]."""
    g = np.ones((1, 1))
    for a, b in zip(A, B):
        g = np.einsum("xy,xiu,yiv->uv", g, a, b)
    return float(g[0, 0])


def tt_norm(A):
    """Frobenius norm via the left-orthogonalizing QR sweep (no cancellation)."""
    return float(np.linalg.norm(left_orthogonalize(A)[-1]))


def tt_add(A, B, beta=1.0):
    """TT of A + beta*B with block cores (ranks add)."""
    d = len(A)
    if d == 1:
        return [A[0] + beta * B[0]]
    out = []
    for k in range(d):
        a, b = A[k], B[k]
        if k == 0:
            out.append(np.concatenate([a, beta * b], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            ra0, n, ra1 = a.shape
            rb0, _, rb1 = b.shape
            c = np.zeros((ra0 + rb0, n, ra1 + rb1))
            c[:ra0, :, :ra1] = a
            c[ra0:, :, ra1:] = b
            out.append(c)
    return out


def left_orthogonalize(A):
    """Left-to-right QR sweep: cores 1..d-1 get orthonormal vertical
    unfoldings, the last core carries the norm (Section 2.2, left-orthogonal
    cores). Returns new cores; the tensor is unchanged."""
    cores = [np.array(c, dtype=np.float64) for c in A]
    for k in range(len(cores) - 1):
        a, n, b = cores[k].shape
        q, r = np.linalg.qr(V(cores[k]))
        cores[k] = q.reshape(a, n, q.shape[1])
        cores[k + 1] = np.einsum("xy,yiz->xiz", r, cores[k + 1])
    return cores


def tt_diff_norm(A, B):
    """||A - B||_F computed stably: form A - B in TT form (block cores),
    left-orthogonalize by QR and take the norm of the last core. Avoids the
    cancellation of <A,A> - 2<A,B> + <B,B>."""
    return tt_norm(tt_add(A, B, -1.0))


def tt_rel_error(X, A):
    """||X - A||_F / ||A||_F (the paper's relative error, Section 5.1)."""
    return tt_diff_norm(X, A) / tt_norm(A)


def is_left_orthogonal(cores, atol=1e-12):
    """True if V(X_k)^T V(X_k) = I for k < d."""
    for c in cores[:-1]:
        v = V(c)
        if not np.allclose(v.T @ v, np.eye(v.shape[1]), atol=atol, rtol=0):
            return False
    return True


def bond_singular_values(A):
    """Singular values of the unfoldings A_<k> (rows: modes 1..k, columns:
    modes k+1..d) for k = 1..d-1: left-orthogonalize, then sweep right to
    left taking the SVD of H(X_k) and moving U S into core k-1 (the left
    factor is orthonormal, so these are the unfolding's singular values).
    Returns a list of d-1 arrays, bond k at index k-1."""
    cores = left_orthogonalize(A)
    out = [None] * (len(cores) - 1)
    for k in range(len(cores) - 1, 0, -1):
        a, n, b = cores[k].shape
        u, sv, vt = np.linalg.svd(H(cores[k]), full_matrices=False)
        out[k - 1] = sv
        cores[k] = vt.reshape(vt.shape[0], n, b)
        cores[k - 1] = np.einsum("xiy,yz->xiz", cores[k - 1], u * sv)
    return out
