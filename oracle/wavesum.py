"""Direct wave-space sum of the split mobility (oracle, test infrastructure only).

Follows Eqs. MUFw-MDCw (Sec. 2.2): for every reciprocal lattice vector k != 0
    M^(w),ab = (1/(eta V)) sum_k exp(i k.(x_a - x_b)) H(k, xi)/k^2 P(k)^+ (I - kk) P(k)
with the projector of Sec. 2.3.2 (Eq. for P_ii):
    P(k) [F; C] = s0 F - 3i s1 C.k ,  s0 = sin(ka)/ka, s1 = (sin ka - ka cos ka)/(ka)^3,
restricted to the (U, E) x (F, S) block in the stresslet basis Y.  The k and -k
terms are complex conjugates, so the sum is taken over a half space as 2 Re(.).

On a deformed lattice (Sec. 2.3.3, cell spanned by the columns of L A) the
reciprocal vectors are k = (2 pi/L) A^{-T} m for integer m and V = L^3 det A.

Parity: pinned (xi-independence of the total with the real-space part, and
equality with the NUFFT evaluation on the same k set; on deformed lattices the
same, plus lattice identities in tests/test_oracle_lattice.py).
"""
import numpy as np

from .basis import Y


def shape_factors(k, a):
    x = k * a
    s0 = np.sin(x) / x
    s1 = (np.sin(x) - x * np.cos(x)) / x ** 3
    small = x < 1e-2
    if np.any(small):
        xs = x[small]
        s0[small] = 1 - xs ** 2 / 6 + xs ** 4 / 120
        s1[small] = 1.0 / 3 - xs ** 2 / 30 + xs ** 4 / 840
    return s0, s1


def half_space(n):
    """Mask of integer vectors in the half space used for +-k pairing."""
    n1, n2, n3 = n[:, 0], n[:, 1], n[:, 2]
    return (n3 > 0) | ((n3 == 0) & (n2 > 0)) | ((n3 == 0) & (n2 == 0) & (n1 > 0))


def _to_k(n, L, A):
    """Wave vectors (2 pi/L) A^{-T} n of integer vectors n (rows); A None: 2 pi n/L."""
    if A is None:
        return 2 * np.pi * n / L
    return (2 * np.pi / L) * (n @ np.linalg.inv(np.asarray(A, float)))


def kset_sphere(L, kmax, A=None):
    """Half-space reciprocal vectors with 0 < |k| <= kmax (cubic, or of the lattice L A)."""
    if A is None:
        nm = [int(np.ceil(kmax * L / (2 * np.pi)))] * 3
    else:  # |m_i| = (L/2pi) |A e_i . k| <= (L/2pi) |A e_i| kmax
        nm = [int(np.ceil(kmax * L * np.linalg.norm(np.asarray(A, float)[:, i]) / (2 * np.pi))) for i in range(3)]
    gx, gy, gz = (np.arange(-q, q + 1) for q in nm)
    n = np.stack(np.meshgrid(gx, gy, gz, indexing='ij'), -1).reshape(-1, 3)
    k = _to_k(n, L, A)
    kk = np.linalg.norm(k, axis=1)
    keep = half_space(n) & (kk <= kmax) & (kk > 0)
    return k[keep]


def kset_grid(L, Ng, A=None):
    """Half-space wave vectors of an Ng^3 FFT grid without Nyquist modes and k = 0."""
    g = np.arange(-Ng // 2 + 1, Ng // 2)
    n = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    keep = half_space(n)
    return _to_k(n[keep], L, A)


def dense_wave(pos, L, a, eta, xi, kvecs, chunk=400, basis=Y, V=None):
    """Dense nN x nN wave-space mobility over the half-space k set kvecs, n = 3 + len(basis):
    8 with the stresslet basis Y, 11 with the torque + stresslet basis G.  V: cell
    volume (default L^3)."""
    N = pos.shape[0]
    V = L ** 3 if V is None else V
    nb = 3 + basis.shape[0]
    M = np.zeros((nb * N, nb * N))
    for c0 in range(0, kvecs.shape[0], chunk):
        k = kvecs[c0:c0 + chunk]
        kk = np.linalg.norm(k, axis=1)
        kh = k / kk[:, None]
        s0, s1 = shape_factors(kk, a)
        u = kk ** 2 / (4 * xi * xi)
        H = (1 + u) * np.exp(-u)
        c = H / (eta * V * kk ** 2)
        proj = np.eye(3)[None] - np.einsum('pi,pj->pij', kh, kh)        # (p,3,3)
        # columns: F_m -> s0 e_m ; s_l -> -3i s1 Y_l k
        A = np.zeros((k.shape[0], 3, nb), dtype=complex)
        A[:, :, :3] = s0[:, None, None] * np.eye(3)[None]
        A[:, :, 3:] = (-3j * s1)[:, None, None] * np.einsum('lmn,pn->pml', basis, k)
        A = np.einsum('pij,pjc->pic', proj, A) * np.sqrt(c)[:, None, None]
        phase = np.exp(-1j * pos @ k.T)                                # (N, p)
        Phi = np.einsum('bp,pic->pibc', phase, A).reshape(k.shape[0] * 3, nb * N)
        M += 2.0 * np.real(Phi.conj().T @ Phi)
    return M
