"""The Section 4 cost model of HaTT-1 and TT-Rounding, summed core by core.

Per HPCRL-1 step (core k, sketches W^{(k)} -> W^{(k-1)}):
  W_L:        n r s l (2 r + 2 s - 2)
  W_L W_R^T:  2 n r s l^2 - r s l
Per left-to-right step:
  C W:        n l^2 (2 r s - 1)
  econ-QR:    (4 n - 4/3) l^3       (Householder, Q only: 4 m l^2 - 4 l^3/3)
  M = Q^T C:  r s l (2 l n - 1)
  update:     n r s l (2 r + 2 s - 2)
With uniform ranks the total is (d-2) n r s l (4 r + 4 s + 6 l) to leading
order (Table 4.1).
"""
from __future__ import annotations


def hatt1_flops(n, r, s, ell):
    """Total HaTT-1 flops for mode sizes n[0..d-1] and ranks r, s, ell[0..d].
    HPCRL runs for cores 1..d-1; the left-to-right pass for bonds 1..d-1."""
    d = len(n)
    total_hp = 0.0
    total_lr = 0.0
    for k in range(1, d):
        # HPCRL step consuming core k: contracts W[k+1] (r[k+1] s[k+1] x l[k+1])
        # into W[k] (r[k] s[k] x l[k])
        hp = (n[k] * r[k] * s[k] * ell[k + 1] * (2 * r[k + 1] + 2 * s[k + 1] - 2)
              + 2 * n[k] * r[k] * s[k] * ell[k + 1] * ell[k] - r[k] * s[k] * ell[k])
        total_hp += hp
    for k in range(d - 1):
        # left-to-right step on core k: C_k is (l[k] n[k]) x (r[k+1] s[k+1])
        m = ell[k] * n[k]
        l1 = ell[k + 1]
        rs1 = r[k + 1] * s[k + 1]
        lr = (m * l1 * (2 * rs1 - 1)                    # C W
              + 4 * m * l1 * l1 - 4.0 / 3.0 * l1 ** 3     # econ-QR, Q only
              + rs1 * l1 * (2 * m - 1)                    # M = Q^T C
              + n[k + 1] * rs1 * l1 * (2 * r[k + 1] + 2 * s[k + 1] - 2))  # core update
        total_lr += lr
    return total_hp, total_lr


def table41_hatt1(d, n, r, s, l):
    """Table 4.1 entry for HaTT-1 with uniform ranks."""
    return (d - 2) * (n * r * s * l * (4 * r + 4 * s + 6 * l))


def table41_tt_rounding(d, n, r, s, l):
    """Table 4.1 entry for TT-Rounding applied to the PKP ranks r*s."""
    return (d - 2) * n * (5 * r ** 3 * s ** 3 + 6 * r ** 2 * s ** 2 * l + 2 * r * s * l ** 2)
