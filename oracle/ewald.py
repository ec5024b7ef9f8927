"""Dense classical Ewald grand mobility (oracle, test infrastructure only).

The exact periodic mobility of Eqs. MUF-MDC (Hasimoto's sum, Eq. hasimoto),
restricted to (U, E) x (F, S) in the stresslet basis, split as in Sec. 2.2:
    M = sum_images M^(r)(x_a - x_b + n L)  +  sum_{k != 0} H M_hat(k) e^{ik.r}/V,
with the real-space part from ``realspace`` (all periodic images with
|r| < rmax, including a particle's own images, plus the r -> 0 self term) and
the wave-space part from ``wavesum`` (all |k| <= kmax).  Both truncations are
chosen from the splitting parameter so the neglected terms are below ``tol``.

With a deformation A (Sec. 2.3.3) the images are x + L A n and the wave vectors
those of the lattice L A (``wavesum``).

Parity: pinned (tests/test_oracle_ewald.py: xi-independence, Cholesky of each
part, Hasimoto's periodic self-mobility, free-space limits, symmetry;
tests/test_oracle_lattice.py: the same lattice in two descriptions, replicated
cells, xi-independence on sheared and extended lattices).
"""
import itertools
import math

import numpy as np

from . import realspace, wavesum
from .basis import G, Y


def cutoffs(xi, tol):
    """rmax, kmax with exp(-xi^2 rmax^2) and H(kmax) below tol (generous margins)."""
    rmax = math.sqrt(math.log(1.0 / tol)) / xi + 2.0
    u = math.log(1.0 / tol) + 6.0
    kmax = 2.0 * xi * math.sqrt(u)
    return rmax, kmax


def dense_real(pos, L, a, eta, xi, rmax, torque=False, A=None):
    N = pos.shape[0]
    nb = 11 if torque else 8
    blocks = realspace.pair_blocks11 if torque else realspace.pair_blocks
    M = np.zeros((nb * N, nb * N))
    if A is None:
        nimg = int(math.ceil(rmax / L))
        shift = lambda n: L * np.array(n, dtype=float)
    else:  # |L A n| >= L sigma_min(A) |n|, and the positions may lie anywhere in the cell
        A = np.asarray(A, float)
        smin = math.sqrt(np.linalg.eigvalsh(A.T @ A)[0])
        span = np.linalg.norm(pos - pos[0], axis=1).max() if N > 1 else 0.0
        nimg = int(math.ceil((rmax + 2 * span) / (L * smin))) + 1
        shift = lambda n: L * (A @ np.array(n, dtype=float))
    rng = range(-nimg, nimg + 1)
    ia, ib = np.meshgrid(np.arange(N), np.arange(N), indexing='ij')
    ia, ib = ia.ravel(), ib.ravel()
    for n in itertools.product(rng, rng, rng):
        d = pos[ia] - pos[ib] + shift(n)
        r = np.linalg.norm(d, axis=1)
        sel = (r < rmax) & (r > 0)
        if not np.any(sel):
            continue
        B = blocks(d[sel], xi, a, eta)
        for (p, q, blk) in zip(ia[sel], ib[sel], B):
            M[nb * p:nb * p + nb, nb * q:nb * q + nb] += blk
    S = realspace.self_block11(xi, a, eta) if torque else realspace.self_block(xi, a, eta)
    for p in range(N):
        M[nb * p:nb * p + nb, nb * p:nb * p + nb] += S
    return M


def dense_mobility(pos, L, a=1.0, eta=1.0, xi=None, tol=1e-14, parts=False, torque=False, A=None):
    """Exact (to ~tol) periodic grand mobility, 8N x 8N with ordering [F(3), s(5)] per particle,
    or with torque=True 11N x 11N with ordering [F(3), L(3), s(5)] (outputs [U, Omega, e]).
    A: deformation of the periodic cell (columns of L A span it; None = cube of side L)."""
    if xi is None:
        xi = math.sqrt(math.pi) / L * 2.0
    rmax, kmax = cutoffs(xi, tol)
    V = None if A is None else L ** 3 * float(np.linalg.det(np.asarray(A, float)))
    Mr = dense_real(np.asarray(pos, float), L, a, eta, xi, rmax, torque, A=A)
    Mw = wavesum.dense_wave(np.asarray(pos, float), L, a, eta, xi, wavesum.kset_sphere(L, kmax, A=A),
                            basis=G if torque else Y, V=V)
    if parts:
        return Mr, Mw
    return Mr + Mw
