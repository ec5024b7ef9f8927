"""Pins for oracle.pse (the PSE algorithm, Secs. 2.3 and 3).

* NUFFT wave space equals the direct k-sum on the same k set (to the quadrature
  error; to 1e-9 at tight quadrature parameters).
* The full PSE product lies within eps of the dense Ewald sum.
* The wave-space noise covariance equals the NUFFT wave-space operator exactly.
* Lanczos equals the dense symmetric square root; GMRES reproduces the dense
  Schur complement (stresslet-constrained mobility, Eq. constrained_vel).
"""
import math

import numpy as np
import pytest
from scipy.linalg import sqrtm

import pse_inputs
from oracle import ewald, params, pse, wavesum


def _vec(U, E):
    return np.concatenate([U, E], axis=1).ravel()


def _dense_op(fn, N):
    cols = []
    for c in range(8 * N):
        e = np.zeros(8 * N)
        e[c] = 1.0
        cols.append(fn(e))
    return np.array(cols).T


@pytest.mark.parametrize('tol,bound', [(1e-3, 1e-2), (1e-12, 1e-9)])
def test_nufft_equals_direct_ksum(tol, bound):
    N, L, xi = 12, 9.0, 0.6
    pos = pse_inputs.random_positions(N, L, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, rule='paper', rcut=0.5 * L)
    w = pse.wave_apply(pos, F, S, p)
    Mw = wavesum.dense_wave(pos, L, 1.0, 1.0, xi, wavesum.kset_grid(L, p.Ng))
    ref = Mw @ np.concatenate([F, S], 1).ravel()
    err = np.linalg.norm(_vec(w['U'], w['E']) - ref) / np.linalg.norm(ref)
    assert err < bound


@pytest.mark.parametrize('tol,xi', [(1e-3, 0.5), (1e-3, 0.7), (1e-4, 0.6)])
def test_pse_within_tolerance_of_ewald(tol, xi):
    N, phi = 100, 0.1
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15)
    ref = M @ np.concatenate([F, S], 1).ravel()
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol)
    U, E = pse.mobility_apply(pos, F, S, p)
    assert np.linalg.norm(_vec(U, E) - ref) / np.linalg.norm(ref) < tol


def test_wave_noise_covariance_is_wave_operator():
    N, L = 3, 9.0
    pos = pse_inputs.random_positions(N, L, seed=4)
    p = params.choose(N, L, 1.0, 1.0, 1.0, 0.8, 1e-3, Ng=8, P=4, rcut=0.5 * L)
    shape = (3, p.Ng, p.Ng, p.Ng // 2 + 1, 2)
    n = int(np.prod(shape))
    A = np.zeros((8 * N, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        A[:, c] = pse.wave_noise(pos, e.reshape(shape), p).ravel()
    cov = A @ A.T
    Mw = _dense_op(lambda v: _vec(**{k: x for k, x in zip(('U', 'E'), (
        pse.wave_apply(pos, v.reshape(N, 8)[:, :3], v.reshape(N, 8)[:, 3:], p)['U'],
        pse.wave_apply(pos, v.reshape(N, 8)[:, :3], v.reshape(N, 8)[:, 3:], p)['E']))}), N)
    assert np.abs(cov - Mw).max() < 1e-12 * np.abs(Mw).max()
    assert np.abs(Mw - Mw.T).max() < 1e-12 * np.abs(Mw).max()


def test_lanczos_equals_dense_sqrt():
    N = 40
    pos, L = pse_inputs.rsa_positions(N, 0.25, seed=6)
    p = params.choose(N, L, 1.0, 1.0, 1.0, 1.1, 1e-3)
    op = pse.RealOp(pos, p)
    z = pse_inputs.lanczos_noise(N, seed=7).ravel()
    y, it, err = pse.lanczos_sqrt(lambda v: op.apply(v.reshape(N, 8)).ravel(), z, 1e-13, 200)
    Mr = op.dense()
    ref = np.real(sqrtm(Mr)) @ z
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-10
    assert it < 60
    # fixed iteration count (tol = 0) runs exactly that many steps
    _, it5, _ = pse.lanczos_sqrt(lambda v: op.apply(v.reshape(N, 8)).ravel(), z, 0.0, 5)
    assert it5 == 5


def test_gmres_reproduces_schur_complement():
    """Zero noise: the mid-point step moves by dt (M_UF - M_US M_ES^-1 M_EF) F^P."""
    N = 30
    pos, L = pse_inputs.rsa_positions(N, 0.15, seed=9)
    F, _ = pse_inputs.moments(N, seed=10)
    p = params.choose(N, L, 1.0, 1.0, 1.0, 1.0, 1e-4)
    dt = 1e-3
    w1 = np.zeros((N, 8))
    w2 = np.zeros((3, p.Ng, p.Ng, p.Ng // 2 + 1, 2))
    x1, S, st = pse.constrained_step(pos, F, dt, w1, w2, p, krylov_tol=1e-12, krylov_maxiter=200)
    op = pse.RealOp(pos, p)

    def full(v):
        v = v.reshape(N, 8)
        U, E = pse.mobility_apply(pos, v[:, :3], v[:, 3:], p, real_op=op)
        return _vec(U, E)

    M = _dense_op(full, N)
    iu = np.concatenate([np.arange(8 * i, 8 * i + 3) for i in range(N)])
    ie = np.concatenate([np.arange(8 * i + 3, 8 * i + 8) for i in range(N)])
    Muf, Mus, Mef, Mes = M[np.ix_(iu, iu)], M[np.ix_(iu, ie)], M[np.ix_(ie, iu)], M[np.ix_(ie, ie)]
    R_inv = Muf - Mus @ np.linalg.solve(Mes, Mef)
    U = R_inv @ F.ravel()
    S_ref = -np.linalg.solve(Mes, Mef @ F.ravel())
    d = x1 - pos
    d -= L * np.rint(d / L)
    assert np.linalg.norm(d.ravel() / dt - U) / np.linalg.norm(U) < 1e-9
    assert np.linalg.norm(S.ravel() - S_ref) / np.linalg.norm(S_ref) < 1e-9
    assert st['krylov_iters'] < 60
    # constrained mobility is symmetric positive definite
    assert np.abs(R_inv - R_inv.T).max() < 1e-8 * np.abs(R_inv).max()
    np.linalg.cholesky(0.5 * (R_inv + R_inv.T))


def test_constrained_velocity_against_dense_ewald():
    """The PSE Schur complement lies within a few eps of the exact (Ewald) one."""
    N = 60
    pos, L = pse_inputs.rsa_positions(N, 0.1, seed=12)
    F, _ = pse_inputs.moments(N, seed=13)
    M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15)
    iu = np.concatenate([np.arange(8 * i, 8 * i + 3) for i in range(N)])
    ie = np.concatenate([np.arange(8 * i + 3, 8 * i + 8) for i in range(N)])
    U_ref = (M[np.ix_(iu, iu)] - M[np.ix_(iu, ie)] @ np.linalg.solve(M[np.ix_(ie, ie)], M[np.ix_(ie, iu)])) @ F.ravel()
    p = params.choose(N, L, 1.0, 1.0, 1.0, 0.7, 1e-4)
    w1 = np.zeros((N, 8))
    w2 = np.zeros((3, p.Ng, p.Ng, p.Ng // 2 + 1, 2))
    x1, S, st = pse.constrained_step(pos, F, 1.0, w1, w2, p, krylov_tol=1e-10)
    d = x1 - pos
    d -= L * np.rint(d / L)
    assert np.linalg.norm(d.ravel() - U_ref) / np.linalg.norm(U_ref) < 2e-4


def test_brownian_sample_covariance_statistical():
    N, L = 3, 9.0
    pos = pse_inputs.random_positions(N, L, seed=21)
    p = params.choose(N, L, 1.0, 1.0, 1.0, 1.0, 1e-3, Ng=8, P=5)
    op = pse.RealOp(pos, p)

    def full(v):
        v = v.reshape(N, 8)
        U, E = pse.mobility_apply(pos, v[:, :3], v[:, 3:], p, real_op=op)
        return _vec(U, E)

    M = _dense_op(full, N)
    dt, K = 0.5, 3000
    rng = np.random.default_rng(22)
    X = np.zeros((K, 8 * N))
    for s in range(K):
        w1 = rng.standard_normal((N, 8))
        w2 = rng.standard_normal((3, 8, 8, 5, 2))
        B, _ = pse.brownian_sample(pos, dt, w1, w2, p, lanczos_tol=1e-10, real_op=op)
        X[s] = B.ravel()
    C = X.T @ X / K
    target = (2 * p.kT / dt) * M
    d = np.sqrt(np.outer(np.diag(target), np.diag(target)))
    assert np.max(np.abs(C - target) / d) < 6.0 / math.sqrt(K) * 1.5
    assert np.max(np.abs(X.mean(0)) / np.sqrt(np.diag(target))) < 5.0 / math.sqrt(K)
