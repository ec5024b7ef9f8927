"""Pins for oracle.ewald / oracle.wavesum (dense classical Ewald, Sec. 2.2).

xi-independence of M = M_r + M_w (the split is exact), positivity of each part
(App. C), Hasimoto's periodic self-mobility of a sphere, free-space limits of
the self mobilities, and symmetry of the grand mobility.
"""
import math

import numpy as np
import pytest

import pse_inputs
from oracle import ewald, wavesum


def test_xi_independence_with_overlaps():
    pos = pse_inputs.random_positions(6, 7.0, seed=5)
    Ms = [ewald.dense_mobility(pos, 7.0, xi=xi, tol=1e-15) for xi in (0.35, 0.6, 0.9)]
    scale = np.abs(Ms[0]).max()
    for M in Ms[1:]:
        assert np.abs(M - Ms[0]).max() / scale < 1e-12


def test_xi_independence_rsa():
    pos, L = pse_inputs.rsa_positions(20, 0.2, seed=11)
    M1 = ewald.dense_mobility(pos, L, xi=0.45, tol=1e-15)
    M2 = ewald.dense_mobility(pos, L, xi=0.8, tol=1e-15)
    assert np.abs(M1 - M2).max() / np.abs(M1).max() < 1e-12


def test_symmetric_and_positive_parts():
    # random (overlapping) configuration with min separation > 0.3a
    rng = np.random.default_rng(3)
    L = 6.0
    pts = []
    while len(pts) < 10:
        x = rng.uniform(0, L, 3)
        ok = True
        for q in pts:
            d = x - q
            d -= L * np.rint(d / L)
            ok &= np.linalg.norm(d) > 0.3
        if ok:
            pts.append(x)
    pos = np.array(pts)
    for xi in (0.5, 1.0):
        Mr, Mw = ewald.dense_mobility(pos, L, xi=xi, tol=1e-15, parts=True)
        for M in (Mr, Mw, Mr + Mw):
            assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
            np.linalg.cholesky(M)            # positive definite (App. C)
            assert np.linalg.eigvalsh(M)[0] > -1e-12 * np.abs(M).max()


def test_hasimoto_self_mobility():
    """6 pi eta a M_UF,self = 1 - c1 (a/L) + (4 pi/3)(a/L)^3 + O((a/L)^6), c1 = 2.837297."""
    Ls = np.array([12.0, 16.0, 24.0, 32.0, 48.0])
    vals = []
    for L in Ls:
        M = ewald.dense_mobility(np.zeros((1, 3)), L, tol=1e-15)
        vals.append(6 * math.pi * M[0, 0])
        assert np.allclose(M[:3, :3], M[0, 0] * np.eye(3), atol=1e-15)
    e = 1.0 / Ls
    y = np.array(vals) - 1 - (4 * math.pi / 3) * e ** 3
    c1 = -np.sum(y * e) / np.sum(e * e)
    assert c1 == pytest.approx(2.837297, abs=1e-6)


def test_free_space_limit_single_sphere():
    L = 400.0
    M = ewald.dense_mobility(np.zeros((1, 3)), L, xi=0.05, tol=1e-15)
    assert 6 * math.pi * M[0, 0] == pytest.approx(1 - 2.837297 / L, abs=1e-7)
    # ES self mobility 3/(20 pi eta a^3) in the orthonormal basis; periodic correction O((a/L)^3)
    assert M[3, 3] * 20 * math.pi / 3 == pytest.approx(1.0, abs=1e-6)
    assert np.allclose(M[3:, 3:], M[3, 3] * np.eye(5), atol=1e-12)


def test_wave_sum_is_hermitian_half_space():
    # sum over the half space x 2 Re equals the full-space complex sum
    pos = pse_inputs.random_positions(3, 5.0, seed=8)
    ks = wavesum.kset_sphere(5.0, 3.0)
    Mh = wavesum.dense_wave(pos, 5.0, 1.0, 1.0, 0.7, ks)
    full = np.concatenate([ks, -ks])
    # complex evaluation of the full-space sum with a one-sided routine
    V = 125.0
    acc = np.zeros((24, 24), complex)
    from oracle.basis import Y
    for k in full:
        kk = np.linalg.norm(k)
        kh = k / kk
        s0, s1 = wavesum.shape_factors(np.array([kk]), 1.0)
        u = kk * kk / (4 * 0.49)
        c = (1 + u) * np.exp(-u) / (V * kk * kk)
        A = np.zeros((3, 8), complex)
        A[:, :3] = s0[0] * np.eye(3)
        A[:, 3:] = -3j * s1[0] * np.einsum('lmn,n->ml', Y, k)
        A = (np.eye(3) - np.outer(kh, kh)) @ A
        for al in range(3):
            for be in range(3):
                ph = np.exp(1j * k @ (pos[al] - pos[be]))
                acc[8 * al:8 * al + 8, 8 * be:8 * be + 8] += c * ph * (A.conj().T @ A)
    assert np.abs(acc.imag).max() < 1e-14
    assert np.abs(acc.real - Mh).max() < 1e-14
