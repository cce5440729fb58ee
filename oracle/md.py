"""FP64 oracle of the multidimensional-reconciliation front end (test
infrastructure; the decoder never imports it).

The step before the decoder in the paper's reconciliation (Results,
"Information reconciliation for CV-QKD system", Fig. 1): Bob and Alice turn
their correlated Gaussian samples Y = X + Z into a binary string U (Bob) and
its noisy form V (Alice) by rotating blocks of d = 8 samples, which makes a
virtual binary-input AWGN channel.  The paper cites the method and gives no
formulas; this module writes it out from its definition:

* Octonions are pairs of quaternions with the Cayley-Dickson product
  (a, b)(c, d) = (ac - d*b, da + bc*) (* = conjugate); A_i is the 8x8 matrix
  of left multiplication by the i-th basis octonion e_i (A_0 = identity).
  Because the octonion norm is multiplicative, every A_i is orthogonal and
  A_i^T A_j + A_j^T A_i = 2 delta_ij I, so for any unit vector y' the vectors
  A_0 y', ..., A_7 y' are an orthonormal basis.
* Bob: y' = y / |y| per block of 8; his 8 key bits b give u = (-1)^b / sqrt 8;
  alpha_i = <A_i y', u> are the coordinates of u in that basis, so
  M = sum_i alpha_i A_i is orthogonal (|alpha| = 1) and M y' = u.  He sends
  alpha and |y|.
* Alice: v = M x / |y| = u - M z / |y|.  For Gaussian modulation, given Bob's
  y, x = g y + n' with g = sigma_x^2 / sigma_y^2 and n' ~ N(0, sigma_x^2
  sigma_z^2 / sigma_y^2) independent of y, so v = g u + M n' / |y|: a binary
  input +-1/sqrt 8 with gain g and noise variance sigma_x^2 sigma_z^2 /
  (sigma_y^2 |y|^2) per coordinate (signal-to-noise sigma_x^2 / sigma_z^2,
  the physical channel's).  The LLR of bit i is 2 g (1/sqrt 8) v_i / that
  variance = 2 |y|^2 v_i / (sqrt 8 sigma_z^2) = 2 |y| (M x)_i / (sqrt 8
  sigma_z^2): only sigma_z^2 enters.

Parity status: pinned by the octonion identities (unit e_0, e_i^2 = -1,
norm multiplicativity), the orthogonality and anticommutation of the A_i,
M y' = u and M orthogonal, the noiseless limit (v = u exactly) and the
statistics of the virtual channel: |v - u| = |z| / |y| per block and the gain
E<v, u> = sigma_x^2 / sigma_y^2 (tests/test_oracle_md.py).
"""
from __future__ import annotations

import numpy as np

D = 8


def _qmul(p, q):
    """Quaternion product, (w, x, y, z) components."""
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _qconj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])


def omul(p, q):
    """Octonion product of 8-vectors by Cayley-Dickson: (a,b)(c,d) = (ac - d*b, da + bc*)."""
    a, b = np.asarray(p[:4], float), np.asarray(p[4:], float)
    c, d = np.asarray(q[:4], float), np.asarray(q[4:], float)
    return np.concatenate([_qmul(a, c) - _qmul(_qconj(d), b), _qmul(d, a) + _qmul(b, _qconj(c))])


def left_mult_matrices() -> np.ndarray:
    """A[i] (8x8): v -> e_i v."""
    E = np.eye(D)
    A = np.zeros((D, D, D))
    for i in range(D):
        for j in range(D):
            A[i][:, j] = omul(E[i], E[j])
    return A


A_MATS = left_mult_matrices()


def bits_to_u(bits: np.ndarray) -> np.ndarray:
    return (1.0 - 2.0 * np.asarray(bits, dtype=np.float64)) / np.sqrt(D)


def bob(y: np.ndarray, bits: np.ndarray):
    """y, bits: [..., 8k].  Returns alpha [..., 8k] (8 per block) and |y| [..., k]."""
    y = np.asarray(y, dtype=np.float64)
    blocks = y.reshape(-1, D)
    norm = np.linalg.norm(blocks, axis=1)
    yp = blocks / norm[:, None]
    u = bits_to_u(np.asarray(bits).reshape(-1, D))
    # alpha_i = <A_i y', u>
    Ay = np.einsum("iab,nb->nia", A_MATS, yp)          # [n, i, 8] = A_i y'
    alpha = np.einsum("nia,na->ni", Ay, u)
    return alpha.reshape(y.shape), norm.reshape(y.shape[:-1] + (y.shape[-1] // D,))


def rotation(alpha_block: np.ndarray) -> np.ndarray:
    """M = sum_i alpha_i A_i for one block."""
    return np.einsum("i,iab->ab", np.asarray(alpha_block, dtype=np.float64), A_MATS)


def alice(x: np.ndarray, alpha: np.ndarray, ynorm: np.ndarray, noise_var) -> np.ndarray:
    """LLRs of Bob's bits from Alice's samples: 2 |y| (M x)_i / (sqrt 8 sigma_z^2).
    x, alpha: [rows, 8k]; ynorm: [rows, k]; noise_var: scalar or [rows]."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    rows, n = x.shape
    al = np.asarray(alpha, dtype=np.float64).reshape(rows, n // D, D)
    xb = x.reshape(rows, n // D, D)
    M = np.einsum("rki,iab->rkab", al, A_MATS)
    mx = np.einsum("rkab,rkb->rka", M, xb)
    nv = np.broadcast_to(np.asarray(noise_var, dtype=np.float64).reshape(-1), (rows,))
    scale = 2.0 * np.asarray(ynorm, dtype=np.float64).reshape(rows, n // D) / (np.sqrt(D) * nv[:, None])
    return (mx * scale[:, :, None]).reshape(rows, n)
