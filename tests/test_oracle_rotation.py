"""Pins for the 11-moment (force, torque, stresslet) form of the oracle (Sec. 2.2.1).

* Restricted to [U, E] x [F, S], every 11-moment block equals the 8-moment one.
* Dense Ewald: the total is independent of xi, symmetric, SPD, and its real-
  and wave-space parts are each SPD (Sec. 2.2, App. C).
* Free space: the self mobilities are 1/(6 pi eta a), 1/(8 pi eta a^3) (rotation)
  and 3/(20 pi eta a^3); far apart, the rotation of one sphere due to a force on
  the other is half the curl of the Oseen flow (checked by finite differences),
  and due to a torque the rotlet gradient (3 rr - I)/(16 pi eta r^3).
* One sphere in a periodic box: the rotational self mobility tends to the free
  value as L grows, with a correction of order (a/L)^3.
* The 11-grid PSE product equals the direct k-sum over the same k set within the
  quadrature error (1e-9 at tight parameters) and lies within eps of dense Ewald.
"""
import numpy as np
import pytest

import pse_inputs
from oracle import ewald, params, pse as opse, realspace as R, wavesum
from oracle.basis import A, G, Y

A_R, ETA = 1.0, 1.0


def _sel8(N):
    return np.array([11 * n + c for n in range(N) for c in list(range(3)) + list(range(6, 11))])


def test_eleven_moment_blocks_restrict_to_eight():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(40, 3)) * 2.5                        # includes overlapping pairs
    B11 = R.pair_blocks11(x, 0.6, A_R, ETA)
    B8 = R.pair_blocks(x, 0.6, A_R, ETA)
    keep = list(range(3)) + list(range(6, 11))
    assert np.abs(B11[:, keep][:, :, keep] - B8).max() < 1e-14
    S11, S8 = R.self_block11(0.6, A_R, ETA), R.self_block(0.6, A_R, ETA)
    assert np.abs(S11[np.ix_(keep, keep)] - S8).max() < 1e-15
    # basis: A antisymmetric with A_k : A_l = delta/2, orthogonal to Y
    assert np.allclose(np.einsum('kij,lij->kl', A, A), 0.5 * np.eye(3))
    assert np.allclose(np.einsum('kij,lij->kl', A, Y), 0.0) and np.allclose(A, -A.transpose(0, 2, 1))


def test_dense_eleven_moment_ewald():
    L = 9.0
    pos = pse_inputs.random_positions(5, L, seed=8)
    M1 = ewald.dense_mobility(pos, L, xi=0.5, tol=1e-14, torque=True)
    M2 = ewald.dense_mobility(pos, L, xi=0.9, tol=1e-14, torque=True)
    assert np.abs(M1 - M2).max() < 1e-12 * np.abs(M1).max()
    assert np.abs(M1 - M1.T).max() < 1e-14
    Mr, Mw = ewald.dense_mobility(pos, L, xi=0.7, tol=1e-14, parts=True, torque=True)
    for Mx in (Mr, Mw, M1):
        np.linalg.cholesky(Mx + 1e-13 * np.eye(Mx.shape[0]))
    M8 = ewald.dense_mobility(pos, L, xi=0.5, tol=1e-14)
    s = _sel8(5)
    assert np.abs(M1[np.ix_(s, s)] - M8).max() < 1e-14


def test_free_space_rotation_mobilities():
    S = R.self_block11(0.5, A_R, ETA, free_only=True)
    assert S[0, 0] == pytest.approx(1 / (6 * np.pi), rel=1e-12)
    assert S[3, 3] == pytest.approx(1 / (8 * np.pi), rel=1e-12)
    assert S[6, 6] == pytest.approx(3 / (20 * np.pi), rel=1e-12)
    x = np.array([[3.0, -40.0, 90.0]])
    r = np.linalg.norm(x[0])
    rh = x[0] / r
    B = R.pair_blocks11(x, 0.5, A_R, ETA, free_only=True)[0]

    def oseen(y):
        q = np.linalg.norm(y)
        return (np.eye(3) / q + np.outer(y, y) / q ** 3) / (8 * np.pi * ETA)
    h = 1e-4
    half_curl = np.zeros((3, 3))
    for m in range(3):
        grad = np.zeros((3, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            grad[:, j] = (oseen(x[0] + e)[:, m] - oseen(x[0] - e)[:, m]) / (2 * h)
        half_curl[:, m] = 0.5 * np.array([grad[2, 1] - grad[1, 2], grad[0, 2] - grad[2, 0], grad[1, 0] - grad[0, 1]])
    OF = B[3:6, :3]
    assert np.abs(OF - half_curl).max() < 1e-3 * np.abs(half_curl).max()       # finite-size terms O((a/r)^2)
    OL = B[3:6, 3:6]
    ref = (3 * np.outer(rh, rh) - np.eye(3)) / (16 * np.pi * ETA * r ** 3)
    assert np.abs(OL - ref).max() < 1e-3 * np.abs(ref).max()
    Bneg = R.pair_blocks11(-x, 0.5, A_R, ETA, free_only=True)[0]
    assert np.abs(B[:3, 3:6] - Bneg[3:6, :3].T).max() < 1e-15                # M_UL(r) = M_OF(-r)^T


def test_periodic_rotational_self_mobility_tends_to_free_value():
    vals = []
    Ls = np.array([12.0, 18.0, 27.0])
    for L in Ls:
        M = ewald.dense_mobility(np.array([[1.0, 2.0, 3.0]]), L, xi=None, tol=1e-14, torque=True)
        vals.append(8 * np.pi * M[3, 3])
    dev = 1.0 - np.array(vals)
    # deviation of order (a/L)^3: scaling L by 3/2 scales it by about (2/3)^3
    assert np.all(np.abs(dev) < 10 * (1.0 / Ls) ** 3)
    assert abs(dev[1] / dev[0] - (2 / 3) ** 3) < 0.05 and abs(dev[2] / dev[1] - (2 / 3) ** 3) < 0.05


@pytest.mark.parametrize('tol,bound', [(1e-3, 2e-2), (1e-12, 1e-9)])
def test_eleven_grid_nufft_equals_direct_ksum(tol, bound):
    N, L, xi = 12, 9.0, 0.6
    pos = pse_inputs.random_positions(N, L, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    Lt = np.random.default_rng(3).standard_normal((N, 3))
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, rule='paper', rcut=0.5 * L)
    got = np.concatenate(opse.wave_apply11(pos, F, Lt, S, p), axis=1).ravel()
    Mw = wavesum.dense_wave(pos, L, 1.0, 1.0, xi, wavesum.kset_grid(L, p.Ng), basis=G)
    ref = Mw @ np.concatenate([F, Lt, S], 1).ravel()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < bound


@pytest.mark.parametrize('tol,xi', [(1e-3, 0.5), (1e-4, 0.6)])
def test_eleven_moment_pse_within_tolerance_of_ewald(tol, xi):
    N, phi = 100, 0.1
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    rng = np.random.default_rng(2)
    F, Lt, S = rng.standard_normal((N, 3)), rng.standard_normal((N, 3)), rng.standard_normal((N, 5))
    M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15, torque=True)
    ref = M @ np.concatenate([F, Lt, S], 1).ravel()
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol)
    got = np.concatenate(opse.mobility_apply11(pos, F, Lt, S, p), axis=1).ravel()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    # restricted to forces and stresslets it is the 8-moment product
    U, _, E = opse.mobility_apply11(pos, F, 0 * Lt, S, p)
    U8, E8 = opse.mobility_apply(pos, F, S, p)
    assert np.abs(np.concatenate([U - U8, E - E8], 1)).max() < 1e-12 * np.abs(U8).max()
