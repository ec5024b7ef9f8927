"""Pins for the oracle's integrators: the mid-point scheme (oracle.pse.midpoint_step,
Sec. 3.4) and the Euler-Maruyama scheme with a random-finite-difference drift
(oracle.pse.rfd_em_step, the alternative discussed in Sec. 3.4).

App. B states the one-step statistics of the scheme for a smooth SPD grand
mobility M(x): with [U^B; E^B] of covariance (2kT/dt) M drawn at x_k,

    <dx>     = kT dt div R_FU^{-1}  (+ dt R_FU^{-1} F^P with a force)  + O(dt^2)
    <dx dx>  = 2 kT dt R_FU^{-1}                                       + O(dt^2)

with R_FU^{-1} = M_UF - M_US M_ES^{-1} M_EF (Eq. constrained_vel).  The scheme is
driven here with the free-space grand mobility of two and three spheres (the
unsplit real-space functions of an unbounded fluid, oracle.realspace with
free_only=True, pinned against the textbook Faxen forms), the divergence is
taken by central finite differences of the dense Schur complement, and the
expectations are formed two ways:

* a Gaussian cubature of degree 3 (the 2n points +-sqrt(n) e_i over the n = 8N
  noise components), exact for the terms up to cubic order in the noise, so the
  remaining error is O(dt) relative and must shrink in proportion to dt;
* Monte Carlo with antithetic pairs (w, -w), within 5 standard errors.

Planted mistakes (a solve at x_k instead of x_{k+1/2}; a slip of dt instead of
dt/2) are shown to miss the mean by order one.

The RFD scheme evaluates the Brownian and deterministic velocity at x_k (exact
covariance 2 kT dt R_FU^{-1} at fixed x_k) and adds the drift
(kT/delta) [R_FU^{-1}(x + delta/2 W) - R_FU^{-1}(x - delta/2 W)] W, whose mean over
the standard normal W is kT div R_FU^{-1} + O(delta^2); the same cubature over the
joint noise (8N + 3N components) checks both moments, and a drift taken at x_k, or
with the two points swapped, misses the mean.
"""
import math

import numpy as np
import pytest

from oracle import pse as opse
from oracle import realspace as R

A, ETA, KT = 1.0, 1.0, 1.0
BOX = 1.0e4                     # positions wrap in the scheme; far from any edge
SELF = R.self_block(0.5, A, ETA, free_only=True)


def grand_mobility(x):
    """Free-space grand mobility, 8N x 8N, [F(3), s(5)] per particle."""
    N = x.shape[0]
    M = np.zeros((8 * N, 8 * N))
    for n in range(N):
        M[8 * n:8 * n + 8, 8 * n:8 * n + 8] = SELF
    ii, jj = np.triu_indices(N, 1)
    B = R.pair_blocks(x[ii] - x[jj], 0.5, A, ETA, free_only=True)
    for p, (i, j) in enumerate(zip(ii, jj)):
        M[8 * i:8 * i + 8, 8 * j:8 * j + 8] = B[p]
        M[8 * j:8 * j + 8, 8 * i:8 * i + 8] = B[p].T
    return M


def _rows(N):
    iu = np.array([8 * n + c for n in range(N) for c in range(3)])
    ie = np.array([8 * n + 3 + c for n in range(N) for c in range(5)])
    return iu, ie


def constrained_mobility(x):
    """R_FU^{-1} = M_UF - M_US M_ES^{-1} M_EF (3N x 3N)."""
    iu, ie = _rows(x.shape[0])
    M = grand_mobility(x)
    return M[np.ix_(iu, iu)] - M[np.ix_(iu, ie)] @ np.linalg.solve(M[np.ix_(ie, ie)], M[np.ix_(ie, iu)])


def divergence(x, h=1e-5):
    """(div R)_i = sum_j d R_ij / d x_j by central differences."""
    n = x.size
    d = np.zeros(n)
    for j in range(n):
        xp, xm = x.ravel().copy(), x.ravel().copy()
        xp[j] += h
        xm[j] -= h
        d += (constrained_mobility(xp.reshape(x.shape))[:, j] - constrained_mobility(xm.reshape(x.shape))[:, j]) / (2 * h)
    return d


def mobility_at(x):
    M = grand_mobility(x)
    N = x.shape[0]

    def apply(F, S):
        o = (M @ np.concatenate([F, S], 1).ravel()).reshape(N, 8)
        return o[:, :3], o[:, 3:]
    return apply


def dense_solve(A_op, b):
    Mat = np.array([A_op(e) for e in np.eye(b.size)]).T
    return (np.linalg.solve(Mat, b),)


def sqrt_spd(M):
    ev, V = np.linalg.eigh(M)
    assert ev.min() > 0
    return (V * np.sqrt(ev)) @ V.T


def displacements(x0, dt, noises, FP=None, mob=mobility_at):
    """x_{k+1} - x_k of the scheme for each noise vector w (B = sqrt(2kT/dt) M^{1/2} w)."""
    N = x0.shape[0]
    Mh = sqrt_spd(grand_mobility(x0))
    out = []
    for w in noises:
        B = math.sqrt(2 * KT / dt) * (Mh @ w).reshape(N, 8)
        x1, _, _ = opse.midpoint_step(x0, FP, dt, B, mob, dense_solve, BOX)
        out.append((x1 - x0).ravel())
    return np.array(out)


def cubature_points(n):
    pts = []
    for i in range(n):
        for s in (1.0, -1.0):
            w = np.zeros(n)
            w[i] = s * math.sqrt(n)
            pts.append(w)
    return pts


CONFIGS = {
    'pair': np.array([[5000.0, 5000.0, 5000.0], [5002.25, 5000.3, 4999.8]]),
    'triplet': np.array([[5000.0, 5000.0, 5000.0], [5002.2, 5000.4, 5000.1], [5001.0, 5002.1, 4999.6]]),
}


@pytest.mark.parametrize('name', sorted(CONFIGS))
def test_midpoint_mean_and_covariance_by_cubature(name):
    x0 = CONFIGS[name]
    N = x0.shape[0]
    R0 = constrained_mobility(x0)
    drift = KT * divergence(x0)
    assert np.linalg.norm(drift) > 1e-3 * np.abs(np.diag(R0)).max()    # a drift worth testing
    pts = cubature_points(8 * N)
    errs = []
    for dt in (0.02, 0.01):
        D = displacements(x0, dt, pts)
        mean, cov = D.mean(0), D.T @ D / len(D)
        errs.append(np.linalg.norm(mean / dt - drift) / np.linalg.norm(drift))
        assert np.linalg.norm(cov - 2 * KT * dt * R0) < 1e-3 * np.linalg.norm(2 * KT * dt * R0)
    assert errs[1] < 0.01
    assert 0.3 < errs[1] / errs[0] < 0.7         # the remaining error is O(dt)
    # a conservative force adds dt R_FU^{-1} F^P to the mean
    FP = np.array([[0.3, -0.2, 0.1]] * N) * np.arange(1, N + 1)[:, None]
    D = displacements(x0, 0.01, pts, FP=FP)
    expect = R0 @ FP.ravel() + drift
    assert np.linalg.norm(D.mean(0) / 0.01 - expect) < 0.01 * np.linalg.norm(expect)


def test_midpoint_planted_mistakes_miss_the_drift():
    """The two mistakes an implementation of the scheme could make change the mean at O(1)."""
    x0 = CONFIGS['pair']
    drift = KT * divergence(x0)
    pts = cubature_points(16)
    dt = 0.01

    def at_start(x):                  # constrained solve at x_k
        return mobility_at(x0)

    def full_slip(x):                 # x_{k+1/2} = x_k + dt U^B
        return mobility_at(x0 + 2.0 * (x - x0))
    for mob in (at_start, full_slip):
        mean = displacements(x0, dt, pts, mob=mob).mean(0)
        assert np.linalg.norm(mean / dt - drift) > 0.5 * np.linalg.norm(drift)


def test_midpoint_statistics_monte_carlo():
    """Seeded Monte Carlo with antithetic pairs: mean and covariance within 5 standard errors."""
    x0 = CONFIGS['pair']
    R0 = constrained_mobility(x0)
    drift = KT * divergence(x0)
    dt, K = 0.05, 3000
    rng = np.random.default_rng(2024)
    W = rng.standard_normal((K, 16))
    Dp = displacements(x0, dt, W)
    Dm = displacements(x0, dt, -W)
    anti = 0.5 * (Dp + Dm) / dt
    se = anti.std(0, ddof=1) / math.sqrt(K)
    assert np.all(np.abs(anti.mean(0) - drift) < 5 * se)
    prod = 0.5 * (np.einsum('ki,kj->kij', Dp, Dp) + np.einsum('ki,kj->kij', Dm, Dm))   # K independent pairs
    cov = prod.mean(0)
    cse = prod.std(0, ddof=1) / math.sqrt(K)
    assert np.all(np.abs(cov - 2 * KT * dt * R0) < 5 * cse + 1e-12)


def rfd_displacements(x0, dt, noises, delta=1e-4, FP=None, mob=mobility_at):
    """x_{k+1} - x_k of the RFD scheme for joint noise vectors [w (8N); W (3N)]."""
    N = x0.shape[0]
    Mh = sqrt_spd(grand_mobility(x0))
    out = []
    for z in noises:
        w, wt = z[:8 * N], z[8 * N:].reshape(N, 3)
        B = math.sqrt(2 * KT / dt) * (Mh @ w).reshape(N, 8)
        x1, _, _, _ = opse.rfd_em_step(x0, FP, dt, B, wt, delta, KT, mob, dense_solve, BOX)
        out.append((x1 - x0).ravel())
    return np.array(out)


@pytest.mark.parametrize('name', sorted(CONFIGS))
def test_rfd_mean_and_covariance_by_cubature(name):
    x0 = CONFIGS[name]
    N = x0.shape[0]
    R0 = constrained_mobility(x0)
    drift = KT * divergence(x0)
    pts = cubature_points(11 * N)
    dt = 0.01
    D = rfd_displacements(x0, dt, pts)
    mean, cov = D.mean(0), D.T @ D / len(D)
    assert np.linalg.norm(mean / dt - drift) < 1e-4 * np.linalg.norm(drift)
    # the RFD estimate's own spread adds dt^2 <drift drift^T>, O(dt) relative to 2 kT dt R_FU^{-1}
    assert np.linalg.norm(cov - 2 * KT * dt * R0) < 1e-3 * np.linalg.norm(2 * KT * dt * R0)
    FP = np.array([[0.3, -0.2, 0.1]] * N) * np.arange(1, N + 1)[:, None]
    mean = rfd_displacements(x0, dt, pts, FP=FP).mean(0)
    expect = R0 @ FP.ravel() + drift
    assert np.linalg.norm(mean / dt - expect) < 1e-4 * np.linalg.norm(expect)


def test_rfd_planted_mistakes_miss_the_drift():
    x0 = CONFIGS['pair']
    drift = KT * divergence(x0)
    pts = cubature_points(22)

    def at_start(x):                  # both finite-difference points at x_k
        return mobility_at(x0)

    def swapped(x):                   # x_k + delta/2 W and x_k - delta/2 W exchanged
        return mobility_at(2.0 * x0 - x)
    for mob in (at_start, swapped):
        mean = rfd_displacements(x0, 0.01, pts, mob=mob).mean(0)
        assert np.linalg.norm(mean / 0.01 - drift) > 0.5 * np.linalg.norm(drift)
