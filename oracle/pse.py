"""The PSE algorithm in plain FP64 NumPy/SciPy (oracle, test infrastructure only).

Steps, in the paper's order:

* Real space (Sec. 2.3.1): pair sum over all pairs with r < r_cut of the
  real-space blocks (``realspace``), plus the self term (App. A, Case 3).
* Wave space (Sec. 2.3.2, Eq. WSops2):  M_w = sigma Q^T F^+ P^+ B P F Q.
  - Q: Gaussian spreading of every moment component onto its own grid with
    K(r) = (2 xi^2/(pi eta_g))^{3/2} exp(-2 xi^2 r^2/eta_g) on the P^3 grid
    points nearest the particle.
  - F: FFT.  The spread density approximates the particles' point moments
    filtered by K_hat(k) = exp(-eta_g k^2 / (8 xi^2)); spreading and
    interpolation together filter by exp(-eta_g k^2/(4 xi^2)), which the
    scaling step divides out (a reading of the normalisation, which the paper leaves implicit).
  - P, B: f = s0 F_hat - 3i s1 S_hat.k;  u = H/(eta V k^2) (I - kk) f;
    U_hat = s0 u;  D_hat = 3i s1 u k^T;  E = Y-projection of D.
  - k = 0 and every mode with an index at the Nyquist plane are excluded.
  - F^+: inverse FFT;  sigma Q^T: interpolation weighted by the cell volume.
* Split sampling (Sec. 3, Eq. split): M^{1/2} dW =d M_r^{1/2} dW1 + M_w^{1/2} dW2.
  - M_r^{1/2} z by the Lanczos method (Sec. 3.2) with full reorthogonalisation
    and the stopping rule |y_m - y_{m-1}| / |y_m| <= tol.
  - M_w^{1/2} dW2 = sigma^{1/2} Q^T F^+ P^+ B^{1/2} dW2 (Eq. FFTsqrt) with
    Hermitian dW2(-k) = conj dW2(k) (Re, Im ~ N(0, 1/2)).
  - Velocities are scaled by sqrt(2 kT / dt) (App. B covariance).
* Mid-point step (Sec. 3.4, App. B): sample [U^B; E^B] at x_k, move to
  x_{k+1/2} = x_k + dt/2 U^B, solve M_ES S = -E^B - M_EF F^P at x_{k+1/2} by
  unrestarted GMRES (x0 = 0), then U = U^B + M_UF F^P + M_US S and
  x_{k+1} = x_k + dt U.
* The alternative the paper weighs against it (Sec. 3.4): Euler-Maruyama with
  the drift kT div R_FU^{-1} from a random finite difference, three constraint
  solves per step.

* Deformed lattices (Sec. 2.3.3): with the cell spanned by the columns of L A,
  the grid nodes sit at h A n; the support is taken in lattice coordinates
  z = A^{-1} x, the Gaussian weight is K(A d) for the lattice displacement d
  (not separable), the wave vectors are (2 pi/L) A^{-T} m, V = L^3 det A,
  sigma = h^3 det A, and the real-space pairs are found over the lattice images.

Layout conventions shared with the product through the documented C ABI (not
through code): grid arrays are [component][z][y][x]; the R2C half spectrum
halves x; 8-vectors per particle are [F_x, F_y, F_z, s_1..s_5].

Parity: pinned against the dense Ewald oracle (within tol) and the direct
k-sum on the same k set (tests/test_oracle_pse.py); Lanczos against a dense
symmetric square root; GMRES against the dense Schur complement; the mid-point
scheme (midpoint_step, shared by constrained_step) against the one-step mean
kT dt div R_FU^{-1} and covariance 2 kT dt R_FU^{-1} of App. B
(tests/test_oracle_midpoint.py); rfd_em_step, with the same App. B statistics
(tests/test_oracle_midpoint.py).
"""
import math

import numpy as np
from scipy.linalg import eigh_tridiagonal
from scipy.spatial import cKDTree

from . import realspace
from .basis import G, Y
from .wavesum import shape_factors


# ---------------------------------------------------------------- wave space
def lattice_coords(pos, p):
    """Wrapped lattice coordinates in [0, L)^3: the positions themselves in the cubic
    box; on a deformed lattice (Sec. 2.3.3, nodes at h A n) z = A^{-1} x mod L, the
    particle's place relative to the undeformed grid."""
    if p.A is None:
        return np.mod(pos, p.L)
    z = np.mod(pos @ np.linalg.inv(p.A).T, p.L)
    return np.where(z >= p.L, z - p.L, z)


def wrap_positions(pos, p):
    """Positions moved into the periodic cell: [0, L)^3 for the cube, A [0, L)^3 on a
    deformed lattice (a lattice translation of each particle)."""
    if p.A is None:
        return np.mod(pos, p.L)
    return lattice_coords(pos, p) @ p.A.T


def _support(pos, p):
    """Base index i0 and displacements of the P support points per dimension.

    Reading: the P grid points nearest the particle; i0 = round(x/h) - (P-1)/2 for
    odd P, floor(x/h) - P/2 + 1 for even P (taken mod Ng).  On a deformed lattice
    x is the lattice coordinate z and the displacements are those of z.
    """
    x = lattice_coords(pos, p)
    q = x / p.h
    if p.P % 2:
        i0 = np.rint(q).astype(np.int64) - (p.P - 1) // 2
    else:
        i0 = np.floor(q).astype(np.int64) - p.P // 2 + 1
    j = np.arange(p.P)
    idx = i0[:, :, None] + j[None, None, :]                    # (N, 3, P)
    disp = idx * p.h - x[:, :, None]                           # (N, 3, P)
    return np.mod(idx, p.Ng), disp


def _weights(pos, p):
    idx, disp = _support(pos, p)
    alpha = 2 * p.xi ** 2 / p.eta_g
    pref = (2 * p.xi ** 2 / (np.pi * p.eta_g)) ** 1.5
    if p.A is None:
        w1 = np.exp(-alpha * disp ** 2)                        # (N, 3, P)
        W = pref * np.einsum('ni,nj,nk->nijk', w1[:, 2], w1[:, 1], w1[:, 0])   # [z][y][x]
    else:  # K(A d): |A d|^2 = d . (A^T A) d, not separable on a deformed lattice
        Gm = p.A.T @ p.A
        d = [disp[:, 0][:, None, None, :], disp[:, 1][:, None, :, None], disp[:, 2][:, :, None, None]]
        q = sum(Gm[i, j] * d[i] * d[j] for i in range(3) for j in range(3))
        W = pref * np.exp(-alpha * q)                          # (N, P, P, P) [z][y][x]
    flat = ((idx[:, 2, :, None, None] * p.Ng + idx[:, 1, None, :, None]) * p.Ng
            + idx[:, 0, None, None, :])
    return flat.reshape(pos.shape[0], -1), W.reshape(pos.shape[0], -1)


def spread(pos, comps, p):
    """Q: spread (N, C) moment components onto C grids of shape (Ng, Ng, Ng)."""
    flat, W = _weights(pos, p)
    n3 = p.Ng ** 3
    C = comps.shape[1]
    grid = np.empty((C, n3))
    for c in range(C):
        grid[c] = np.bincount(flat.ravel(), weights=(W * comps[:, c:c + 1]).ravel(), minlength=n3)
    return grid.reshape(C, p.Ng, p.Ng, p.Ng)


def interpolate(grid, pos, p):
    """Q^T (without sigma): sum over the support of K times the grid values."""
    flat, W = _weights(pos, p)
    C = grid.shape[0]
    g = grid.reshape(C, -1)
    return np.stack([np.sum(W * g[c][flat], axis=1) for c in range(C)], axis=1)


def kgrid(p):
    """Wave vectors of the R2C half spectrum [z][y][x-half] and the Nyquist/zero mask."""
    n = p.Ng
    f = np.fft.fftfreq(n, d=1.0 / n)
    fx = np.arange(n // 2 + 1)
    kz, ky, kx = np.meshgrid(f, f, fx, indexing='ij')
    keep = (np.abs(kz) != n // 2) & (np.abs(ky) != n // 2) & (kx != n // 2)
    keep &= ~((kz == 0) & (ky == 0) & (kx == 0))
    scale = 2 * np.pi / p.L
    if p.A is not None:  # k = (2 pi/L) A^{-T} m
        B = np.linalg.inv(p.A).T
        kx, ky, kz = (B[i, 0] * kx + B[i, 1] * ky + B[i, 2] * kz for i in range(3))
    return kx * scale, ky * scale, kz * scale, keep


def _project_out(uh, kvec, kk, keep, s0, s1, want):
    """P^+: U_hat = s0 u, E_hat_l = Y_l : (3i s1 u k^T)."""
    out = []
    if 'U' in want:
        out += [s0 * uh[i] for i in range(3)]
    if 'E' in want:
        D = 3j * s1[None, None] * uh[:, None] * kvec[None, :]       # [i][j]
        out += [np.einsum('ij...,ij->...', D, Y[l]) for l in range(5)]
    return [np.where(keep, o, 0.0) for o in out]


def _k_arrays(p):
    kx, ky, kz, keep = kgrid(p)
    kvec = np.stack([kx, ky, kz])
    kk2 = kx ** 2 + ky ** 2 + kz ** 2
    kk = np.sqrt(np.where(keep, kk2, 1.0))
    s0, s1 = shape_factors(kk.ravel(), p.a)
    return kvec, kk, keep, s0.reshape(kk.shape), s1.reshape(kk.shape)


def wave_apply(pos, F, S, p, want=('U', 'E')):
    """Wave-space part M_w [F; S] by the NUFFT route of Eq. WSops2."""
    N = pos.shape[0]
    comps = np.concatenate([F, S], axis=1)
    grid = spread(pos, comps, p)
    gh = np.fft.rfftn(grid, axes=(1, 2, 3))
    kvec, kk, keep, s0, s1 = _k_arrays(p)
    Sh = np.einsum('l...,lij->ij...', gh[3:], Y)                     # (3,3,...)
    f = s0[None] * gh[:3] - 3j * s1[None] * np.einsum('ij...,j...->i...', Sh, kvec)
    u = kk ** 2 / (4 * p.xi ** 2)
    c = (p.sigma ** 2 / p.V) / p.eta * (1 + u) * np.exp(-(1 - p.eta_g) * u) / kk ** 2
    kh = kvec / kk[None]
    f = f - kh * np.sum(kh * f, axis=0)[None]
    uh = c[None] * f
    outs = _project_out(uh, kvec, kk, keep, s0, s1, want)
    n = p.Ng
    grids = np.stack([np.fft.irfftn(o, s=(n, n, n), axes=(0, 1, 2)) * n ** 3 for o in outs])
    vals = interpolate(grids, pos, p)
    res = {}
    col = 0
    if 'U' in want:
        res['U'] = vals[:, :3]
        col = 3
    if 'E' in want:
        res['E'] = vals[:, col:col + 5]
    return res


def hermitian_noise(w2, p):
    """dW2 on the half spectrum from standard normals w2 of shape (3, Ng, Ng, Ng/2+1, 2).

    dW2 = (re + i im)/sqrt(2) on representatives; on the kx = 0 plane the entry
    (z, y) with z > Ng/2, or z = 0 and y > Ng/2, is the conjugate of entry
    (-z, -y) mod Ng; Nyquist modes and k = 0 are zero.
    """
    n = p.Ng
    dw = (w2[..., 0] + 1j * w2[..., 1]) / math.sqrt(2.0)
    dw = dw.copy()
    z = np.arange(n)[:, None]
    y = np.arange(n)[None, :]
    partner = (z > n // 2) | ((z == 0) & (y > n // 2))
    zm = (-np.arange(n)) % n
    plane = dw[:, :, :, 0]
    mirror = np.conj(plane[:, zm][:, :, zm])
    plane = np.where(partner[None], mirror, plane)
    dw[:, :, :, 0] = plane
    _, _, _, keep = kgrid(p)
    return np.where(keep[None], dw, 0.0)


def wave_noise(pos, w2, p):
    """M_w^{1/2} dW2 (Eq. FFTsqrt), returned as (N, 8) [U, E] without sqrt(2kT/dt)."""
    dw = hermitian_noise(w2, p)
    kvec, kk, keep, s0, s1 = _k_arrays(p)
    u = kk ** 2 / (4 * p.xi ** 2)
    Hk = (1 + u) * np.exp(-u)
    c = p.sigma * np.exp(p.eta_g * u / 2.0) * np.sqrt(Hk / (p.eta * p.V * kk ** 2))
    kh = kvec / kk[None]
    dw = dw - kh * np.sum(kh * dw, axis=0)[None]
    uh = c[None] * dw
    outs = _project_out(uh, kvec, kk, keep, s0, s1, ('U', 'E'))
    n = p.Ng
    grids = np.stack([np.fft.irfftn(o, s=(n, n, n), axes=(0, 1, 2)) * n ** 3 for o in outs])
    return interpolate(grids, pos, p)


# ---------------------------------------------------------------- real space
def _lattice_pairs(pos, p):
    """Pairs (i < j) and separations x_i - x_j + L A n closer than r_cut on a deformed
    lattice.  Candidates: pairs whose lattice coordinates lie within r_cut/sigma_min
    (|A dz| >= sigma_min |dz|); for each, every image n in {-1, 0, 1}^3 around the
    nearest lattice image is tested in Cartesian space."""
    z = lattice_coords(pos, p)
    smin = math.sqrt(np.linalg.eigvalsh(p.A.T @ p.A)[0])
    tree = cKDTree(z, boxsize=p.L)
    pr = tree.query_pairs(p.rcut / smin * (1 + 1e-12), output_type='ndarray')
    if pr.size == 0:
        return np.zeros((0, 2), dtype=np.int64), np.zeros((0, 3))
    dz = z[pr[:, 0]] - z[pr[:, 1]]
    dz -= p.L * np.rint(dz / p.L)
    ps, ds = [], []
    for n in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing='ij')).reshape(3, -1).T:
        r = (dz + p.L * n) @ p.A.T
        keep = np.linalg.norm(r, axis=1) < p.rcut
        ps.append(pr[keep])
        ds.append(r[keep])
    return np.concatenate(ps), np.concatenate(ds)


class RealOp:
    """Real-space operator M_r for a fixed configuration (pairs with r < r_cut); with
    torque=True the 11-moment form [F, L, S] -> [U, Omega, E]."""

    def __init__(self, pos, p, chunk=20000, torque=False):
        self.N = pos.shape[0]
        if p.A is None:
            x = np.mod(pos, p.L)
            tree = cKDTree(x, boxsize=p.L)
            pr = tree.query_pairs(p.rcut, output_type='ndarray')
            if pr.size == 0:
                pr = np.zeros((0, 2), dtype=np.int64)
            d = x[pr[:, 0]] - x[pr[:, 1]]
            d -= p.L * np.rint(d / p.L)
            keep = np.linalg.norm(d, axis=1) < p.rcut
            pr, d = pr[keep], d[keep]
        else:
            pr, d = _lattice_pairs(pos, p)
        nb = 11 if torque else 8
        fn = realspace.pair_blocks11 if torque else realspace.pair_blocks
        blocks = np.empty((pr.shape[0], nb, nb))
        for c0 in range(0, pr.shape[0], chunk):
            blocks[c0:c0 + chunk] = fn(d[c0:c0 + chunk], p.xi, p.a, p.eta)
        self.nb = nb
        self.i, self.j, self.B = pr[:, 0], pr[:, 1], blocks
        self.self = (realspace.self_block11 if torque else realspace.self_block)(p.xi, p.a, p.eta)

    def apply(self, v):
        """(N, nb) -> (N, nb) real-space product."""
        out = v @ self.self.T
        np.add.at(out, self.i, np.einsum('pab,pb->pa', self.B, v[self.j]))
        np.add.at(out, self.j, np.einsum('pba,pb->pa', self.B, v[self.i]))
        return out

    def dense(self):
        nb = self.nb
        M = np.zeros((nb * self.N, nb * self.N))
        for n in range(self.N):
            M[nb * n:nb * n + nb, nb * n:nb * n + nb] = self.self
        for i, j, b in zip(self.i, self.j, self.B):
            M[nb * i:nb * i + nb, nb * j:nb * j + nb] += b
            M[nb * j:nb * j + nb, nb * i:nb * i + nb] += b.T
        return M


def mobility_apply(pos, F, S, p, parts=('real', 'wave'), real_op=None):
    """[U; E] = M [F; S] with the PSE split (Sec. 2.3)."""
    N = pos.shape[0]
    U = np.zeros((N, 3))
    E = np.zeros((N, 5))
    if 'real' in parts:
        op = real_op if real_op is not None else RealOp(pos, p)
        v = op.apply(np.concatenate([F, S], axis=1))
        U += v[:, :3]
        E += v[:, 3:]
    if 'wave' in parts:
        w = wave_apply(pos, F, S, p)
        U += w['U']
        E += w['E']
    return U, E


def wave_apply11(pos, F, Lt, S, p):
    """Wave-space part of the 11-moment product [U; Omega; E] = M_w [F; L; S] (Sec. 2.3.2, the
    paper's 11 grids: 3 force + 8 couplet).  The couplet is C = sum_k L_k A_k + sum_l s_l Y_l
    (basis G), f = s0 F_hat - 3i s1 C.k, u = c (I - kk) f, and the outputs are U = s0 u and the
    components G_l : D of D = 3i s1 u k^T (the rotation rate through A, the strain through Y)."""
    comps = np.concatenate([F, Lt, S], axis=1)
    grid = spread(pos, comps, p)
    gh = np.fft.rfftn(grid, axes=(1, 2, 3))
    kvec, kk, keep, s0, s1 = _k_arrays(p)
    Ch = np.einsum('l...,lij->ij...', gh[3:], G)
    f = s0[None] * gh[:3] - 3j * s1[None] * np.einsum('ij...,j...->i...', Ch, kvec)
    u = kk ** 2 / (4 * p.xi ** 2)
    c = (p.sigma ** 2 / p.V) / p.eta * (1 + u) * np.exp(-(1 - p.eta_g) * u) / kk ** 2
    kh = kvec / kk[None]
    f = f - kh * np.sum(kh * f, axis=0)[None]
    uh = c[None] * f
    D = 3j * s1[None, None] * uh[:, None] * kvec[None, :]
    outs = [s0 * uh[i] for i in range(3)] + [np.einsum('ij...,ij->...', D, G[l]) for l in range(8)]
    outs = [np.where(keep, o, 0.0) for o in outs]
    n = p.Ng
    grids = np.stack([np.fft.irfftn(o, s=(n, n, n), axes=(0, 1, 2)) * n ** 3 for o in outs])
    vals = interpolate(grids, pos, p)
    return vals[:, :3], vals[:, 3:6], vals[:, 6:]


def mobility_apply11(pos, F, Lt, S, p, parts=('real', 'wave'), real_op=None):
    """[U; Omega; E] = M [F; L; S], the 11-moment grand mobility with the PSE split."""
    N = pos.shape[0]
    out = np.zeros((N, 11))
    if 'real' in parts:
        op = real_op if real_op is not None else RealOp(pos, p, torque=True)
        out += op.apply(np.concatenate([F, Lt, S], axis=1))
    if 'wave' in parts:
        out += np.concatenate(wave_apply11(pos, F, Lt, S, p), axis=1)
    return out[:, :3], out[:, 3:6], out[:, 6:]


# ---------------------------------------------------------------- Lanczos
def lanczos_sqrt(apply, z, tol, maxiter):
    """y ~= M^{1/2} z by the Lanczos method with full reorthogonalisation (Sec. 3.2).

    Stops when |c_m - [c_{m-1}; 0]| / |c_m| <= tol where y_m = |z| V_m c_m and
    c_m = T_m^{1/2} e_1 (V_m orthonormal); tol = 0 runs exactly maxiter steps.
    Returns (y, iterations, last relative change).
    """
    n = z.size
    beta0 = np.linalg.norm(z)
    if beta0 == 0.0:
        return np.zeros_like(z), 0, 0.0
    V = np.zeros((maxiter + 1, n))
    V[0] = z / beta0
    alpha, beta = [], []
    c_prev = None
    err = np.inf
    it = 0
    for j in range(maxiter):
        it = j + 1
        w = apply(V[j])
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        a_j = V[j] @ w
        w = w - a_j * V[j]
        for _ in range(2):                       # full reorthogonalisation
            w = w - V[:j + 1].T @ (V[:j + 1] @ w)
        alpha.append(a_j)
        b_j = np.linalg.norm(w)
        if j == 0:
            c = np.array([math.sqrt(max(a_j, 0.0))])
        else:
            th, Q = eigh_tridiagonal(np.array(alpha), np.array(beta))
            c = Q @ (np.sqrt(np.maximum(th, 0.0)) * Q[0])
        if c_prev is not None:
            err = np.linalg.norm(c - np.append(c_prev, 0.0)) / np.linalg.norm(c)
            if tol > 0 and err <= tol:
                break
        c_prev = c
        if b_j == 0.0 or j == maxiter - 1:
            break
        beta.append(b_j)
        V[j + 1] = w / b_j
    y = beta0 * (V[:it].T @ c)
    return y, it, err


# ---------------------------------------------------------------- GMRES
def gmres(apply, b, tol, maxiter):
    """Unrestarted GMRES with x0 = 0; stops at |r|/|b| <= tol (reading of the
    unnamed Krylov solve, Sec. 4 text on 8-10 iterations).  Returns (x, iters, relres)."""
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b), 0, 0.0
    n = b.size
    V = np.zeros((maxiter + 1, n))
    Hm = np.zeros((maxiter + 1, maxiter))
    V[0] = b / beta
    rel = 1.0
    it = 0
    y = np.zeros(0)
    for j in range(maxiter):
        it = j + 1
        w = apply(V[j])
        for _ in range(2):
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            Hm[:j + 1, j] += h
        Hm[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(Hm[:j + 2, :j + 1], e1, rcond=None)
        rel = np.linalg.norm(e1 - Hm[:j + 2, :j + 1] @ y) / beta
        if rel <= tol or Hm[j + 1, j] == 0.0:
            break
        V[j + 1] = w / Hm[j + 1, j]
    x = V[:it].T @ y
    return x, it, rel


# ---------------------------------------------------------------- sampling / step
def brownian_sample(pos, dt, w1, w2, p, lanczos_tol=None, lanczos_maxiter=100, real_op=None):
    """[U^B; E^B] = sqrt(2kT/dt) (M_r^{1/2} w1 + M_w^{1/2} dW2(w2)) as (N, 8)."""
    op = real_op if real_op is not None else RealOp(pos, p)
    N = pos.shape[0]
    tol = p.tol if lanczos_tol is None else lanczos_tol
    yr, it, err = lanczos_sqrt(lambda v: op.apply(v.reshape(N, 8)).ravel(), w1.reshape(-1), tol,
                               lanczos_maxiter)
    yw = wave_noise(pos, w2, p)
    scale = math.sqrt(2 * p.kT / dt)
    return scale * (yr.reshape(N, 8) + yw), {'lanczos_iters': it, 'lanczos_err': err}


def midpoint_step(x0, FP, dt, B, mobility_at, solve, L):
    """Slip, constrained solve and full step of the mid-point scheme (Sec. 3.4, App. B).

    For any mobility: B = [U^B; E^B] (N, 8) is the Brownian slip drawn at x_k;
    mobility_at(x) returns the product (F, S) -> (U, E) at configuration x;
    solve(mes, rhs) returns (S, *info) with mes(S) = rhs.  The scheme moves to
    x_{k+1/2} = x_k + dt/2 U^B, solves M_ES S = -E^B - M_EF F^P there (E = 0 at the
    mid-point), takes U = U^B + M_UF F^P + M_US S and x_{k+1} = x_k + dt U.
    Positions are wrapped into [0, L) (L a number) or by the callable L.  Returns
    (x_{k+1}, S, info).
    """
    N = x0.shape[0]
    wrap = L if callable(L) else (lambda x: np.mod(x, L))
    UB, EB = B[:, :3], B[:, 3:]
    xh = wrap(x0 + 0.5 * dt * UB)
    mob = mobility_at(xh)
    zF = np.zeros((N, 3)) if FP is None else FP
    rhs = -EB
    if FP is not None:
        rhs = rhs - mob(zF, np.zeros((N, 5)))[1]
    S, *info = solve(lambda s: mob(np.zeros((N, 3)), s.reshape(N, 5))[1].ravel(), rhs.ravel())
    S = S.reshape(N, 5)
    U = UB + mob(zF, S)[0]
    x1 = wrap(x0 + dt * U)
    return x1, S, info


def constrained_step(pos, FP, dt, w1, w2, p, lanczos_tol=None, lanczos_maxiter=100,
                     krylov_tol=None, krylov_maxiter=50):
    """One mid-point step (Sec. 3.4) with the PSE mobility.  Returns (x_{k+1}, S_{k+1/2}, stats)."""
    x0 = wrap_positions(pos, p)
    B, st = brownian_sample(x0, dt, w1, w2, p, lanczos_tol, lanczos_maxiter)

    def mobility_at(x):
        op = RealOp(x, p)
        return lambda F, S: mobility_apply(x, F, S, p, real_op=op)

    ktol = p.tol if krylov_tol is None else krylov_tol
    x1, S, (kit, rel) = midpoint_step(x0, FP, dt, B, mobility_at,
                                      lambda A, b: gmres(A, b, ktol, krylov_maxiter),
                                      p.L if p.A is None else (lambda x: wrap_positions(x, p)))
    st.update({'krylov_iters': kit, 'krylov_relres': rel})
    return x1, S, st


# ---------------------------------------------------------------- RFD + Euler-Maruyama
def constrained_apply(mob, v, solve):
    """R_FU^{-1} v = M_UF v - M_US M_ES^{-1} M_EF v (Eq. constrained_vel) for one mobility product mob."""
    N = v.shape[0]
    U1, E1 = mob(v, np.zeros((N, 5)))
    S, *info = solve(lambda s: mob(np.zeros((N, 3)), s.reshape(N, 5))[1].ravel(), -E1.ravel())
    U2, _ = mob(np.zeros((N, 3)), S.reshape(N, 5))
    return U1 + U2, info


def rfd_em_step(x0, FP, dt, B, wt, delta, kT, mobility_at, solve, L):
    """Euler-Maruyama step with a random-finite-difference drift (Sec. 3.4, the RFD alternative).

    Deterministic and Brownian velocity from one constrained solve at x_k:
    M_ES S = -E^B - M_EF F^P, U = U^B + M_UF F^P + M_US S (covariance (2kT/dt) R_FU^{-1}).
    Drift by RFD with the standard normal vector wt (N, 3):
    kT div R_FU^{-1} ~ (kT/delta) [R_FU^{-1}(x_k + delta/2 wt) - R_FU^{-1}(x_k - delta/2 wt)] wt,
    two more solves.  x_{k+1} = x_k + dt (U + drift), wrapped into [0, L) (L a number)
    or by the callable L.
    Returns (x_{k+1}, S, drift, info) with info the solve outputs of the three solves.
    """
    N = x0.shape[0]
    wrap = L if callable(L) else (lambda x: np.mod(x, L))
    UB, EB = B[:, :3], B[:, 3:]
    mob = mobility_at(x0)
    zF = np.zeros((N, 3)) if FP is None else FP
    rhs = -EB
    if FP is not None:
        rhs = rhs - mob(zF, np.zeros((N, 5)))[1]
    S, *i0 = solve(lambda s: mob(np.zeros((N, 3)), s.reshape(N, 5))[1].ravel(), rhs.ravel())
    S = S.reshape(N, 5)
    U = UB + mob(zF, S)[0]
    Rp, ip = constrained_apply(mobility_at(wrap(x0 + 0.5 * delta * wt)), wt, solve)
    Rm, im = constrained_apply(mobility_at(wrap(x0 - 0.5 * delta * wt)), wt, solve)
    drift = (kT / delta) * (Rp - Rm)
    x1 = wrap(x0 + dt * (U + drift))
    return x1, S, drift, (i0, ip, im)


def rfd_step(pos, FP, dt, w1, w2, wt, delta, p, lanczos_tol=None, lanczos_maxiter=100, krylov_tol=None,
             krylov_maxiter=50):
    """rfd_em_step with the PSE mobility.  Returns (x_{k+1}, S_k, drift, stats)."""
    x0 = wrap_positions(pos, p)
    B, st = brownian_sample(x0, dt, w1, w2, p, lanczos_tol, lanczos_maxiter)

    def mobility_at(x):
        op = RealOp(x, p)
        return lambda F, S: mobility_apply(x, F, S, p, real_op=op)

    ktol = p.tol if krylov_tol is None else krylov_tol
    x1, S, drift, info = rfd_em_step(x0, FP, dt, B, wt, delta, p.kT, mobility_at,
                                     lambda A, b: gmres(A, b, ktol, krylov_maxiter),
                                     p.L if p.A is None else (lambda x: wrap_positions(x, p)))
    st.update({'krylov_iters': sum(i[0] for i in info), 'krylov_relres': max(i[1] for i in info)})
    return x1, S, drift, st
