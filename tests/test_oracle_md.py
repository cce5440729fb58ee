"""Pins for the multidimensional-reconciliation oracle (oracle/md.py).

Checked against the algebra that fixes the construction, not against the
oracle itself: octonion units (e_0 = 1, e_i^2 = -1), the multiplicative norm
|pq| = |p||q| (which fails for a wrong sign anywhere in the product table),
the orthogonality and anticommutation of the left-multiplication matrices,
M y' = u with M orthogonal, the noiseless limit v = u, and the variance of
the virtual channel's noise, sigma_z^2 / |y|^2.
"""
import numpy as np
import pytest

from oracle import md


def test_octonion_units_and_norm_multiplicativity():
    E = np.eye(8)
    assert np.allclose(md.omul(E[0], E[5]), E[5]) and np.allclose(md.omul(E[5], E[0]), E[5])
    for i in range(1, 8):
        assert np.allclose(md.omul(E[i], E[i]), -E[0])
    rng = np.random.default_rng(1)
    for _ in range(200):
        p, q = rng.normal(size=8), rng.normal(size=8)
        assert np.linalg.norm(md.omul(p, q)) == pytest.approx(np.linalg.norm(p) * np.linalg.norm(q), rel=1e-12)
    # octonions are not associative (a quaternion-only table would be)
    a, b, c = E[1], E[2], E[4]
    assert not np.allclose(md.omul(md.omul(a, b), c), md.omul(a, md.omul(b, c)))


def test_left_multiplication_matrices():
    A = md.A_MATS
    assert np.allclose(A[0], np.eye(8))
    for i in range(8):
        assert np.allclose(A[i].T @ A[i], np.eye(8))
        assert set(np.unique(A[i])) <= {-1.0, 0.0, 1.0}      # signed permutations
        for j in range(8):
            if i != j:
                assert np.allclose(A[i].T @ A[j] + A[j].T @ A[i], 0.0)
    rng = np.random.default_rng(2)
    y = rng.normal(size=8)
    y /= np.linalg.norm(y)
    basis = np.stack([A[i] @ y for i in range(8)])
    assert np.allclose(basis @ basis.T, np.eye(8))


def test_rotation_maps_y_to_u_and_is_orthogonal():
    rng = np.random.default_rng(3)
    y = rng.normal(size=(50, 8))
    bits = rng.integers(0, 2, (50, 8))
    alpha, norm = md.bob(y, bits)
    for k in range(50):
        M = md.rotation(alpha[k])
        assert np.allclose(M @ M.T, np.eye(8), atol=1e-12)
        assert np.allclose(M @ (y[k] / norm[k, 0]), md.bits_to_u(bits[k]), atol=1e-12)
        assert norm[k, 0] == pytest.approx(np.linalg.norm(y[k]))


def test_noiseless_limit_gives_u_and_the_bits():
    rng = np.random.default_rng(4)
    y = rng.normal(size=(3, 64))
    bits = rng.integers(0, 2, (3, 64))
    alpha, norm = md.bob(y, bits)
    llr = md.alice(y, alpha, norm, noise_var=0.5)
    v = llr * 0.5 * np.sqrt(8) / (2 * np.repeat(norm, 8, axis=1) ** 2)
    assert np.allclose(v, md.bits_to_u(bits), atol=1e-12)
    assert np.array_equal((llr < 0).astype(int), bits)


def test_virtual_channel_noise_variance():
    rng = np.random.default_rng(5)
    rows, n = 4, 8 * 20000
    sx, sz = 1.0, 0.7
    x = rng.normal(0, sx, (rows, n))
    y = x + rng.normal(0, sz, (rows, n))
    bits = rng.integers(0, 2, (rows, n))
    alpha, norm = md.bob(y, bits)
    llr = md.alice(x, alpha, norm, noise_var=sz ** 2)
    nrm = np.repeat(norm, 8, axis=1)
    v = llr * sz ** 2 * np.sqrt(8) / (2 * nrm ** 2)
    u = md.bits_to_u(bits)
    w = (v - u) * nrm / sz      # = -(M z)_i / sigma_z: M orthogonal keeps |z| per block
    assert abs(w.mean()) < 0.01
    assert w.var() == pytest.approx(1.0, abs=0.01)
    # the gain of the virtual channel: E<v, u> over a block = sigma_x^2 / sigma_y^2
    gain = (v * u).reshape(rows, -1, 8).sum(axis=2).mean()
    assert gain == pytest.approx(sx ** 2 / (sx ** 2 + sz ** 2), abs=0.005)
