"""Equilibrium distributions of the validation runs of Sec. 4 (oracle, test infrastructure only).

* Two spheres joined by the potential U(r) = k |r - r0| (r the centre-to-centre
  distance): the Boltzmann density of r is proportional to r^2 exp(-U/kT), which
  the paper writes out as
      f(r) = kt^3 / (2 (2 + kt^2 r0^2)) r^2 exp(-kt |r - r0|),   kt = k / kT,
  normalised on the whole line (the mass on r < 0, O(exp(-kt r0)), is dropped).
  ``pair_pdf`` is that formula; ``pair_cdf`` its integral from 0, written out
  piecewise.
* Non-interacting spheres: positions are uniform and independent at
  equilibrium, so the static structure factor S(q) = |sum_j exp(i q.x_j)|^2 / N
  has mean 1 at every q != 0 of the box's reciprocal lattice; ``structure_factor``
  evaluates the definition directly.

Parity: pinned (tests/test_oracle_equilibrium.py) by quadrature of the
Boltzmann weight r^2 exp(-U/kT), the closed-form CDF against the quadrature of
the PDF, and the mean of S(q) over uniform random positions.
"""
import numpy as np


def pair_pdf(r, k, r0, kT=1.0):
    """f(r) of the pair-distance distribution under U = k |r - r0| (Sec. 4)."""
    kt = k / kT
    r = np.asarray(r, dtype=float)
    return kt ** 3 / (2.0 * (2.0 + kt ** 2 * r0 ** 2)) * r ** 2 * np.exp(-kt * np.abs(r - r0))


def pair_cdf(r, k, r0, kT=1.0):
    """Integral of pair_pdf from 0 to r (closed form, piecewise at r0)."""
    kt = k / kT
    c = kt ** 3 / (2.0 * (2.0 + kt ** 2 * r0 ** 2))
    r = np.asarray(r, dtype=float)

    def prim_below(x):          # antiderivative of x^2 exp(kt (x - r0)) for x <= r0
        return np.exp(kt * (x - r0)) * (x ** 2 / kt - 2 * x / kt ** 2 + 2 / kt ** 3)

    def prim_above(x):          # antiderivative of x^2 exp(-kt (x - r0)) for x >= r0
        return -np.exp(-kt * (x - r0)) * (x ** 2 / kt + 2 * x / kt ** 2 + 2 / kt ** 3)

    lo = np.minimum(r, r0)
    below = prim_below(lo) - prim_below(0.0)
    above = np.where(r > r0, prim_above(np.maximum(r, r0)) - prim_above(r0), 0.0)
    return c * (below + above)


def structure_factor(x, L, qvecs):
    """S(q) = |sum_j exp(i q.x_j)|^2 / N for each wave vector q (rows of qvecs)."""
    x = np.asarray(x, dtype=float)
    ph = np.exp(1j * (x @ np.asarray(qvecs, dtype=float).T))
    return np.abs(ph.sum(axis=0)) ** 2 / x.shape[0]


def q_shells(L, nmax):
    """Wave vectors 2 pi n / L with integer n, grouped by |n|^2 <= nmax^2 (half space, q != 0).

    Returns (qvecs, shell index per vector, |q| per shell)."""
    g = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    n2 = (n ** 2).sum(1)
    half = (n[:, 2] > 0) | ((n[:, 2] == 0) & (n[:, 1] > 0)) | ((n[:, 2] == 0) & (n[:, 1] == 0) & (n[:, 0] > 0))
    keep = half & (n2 > 0) & (n2 <= nmax ** 2)
    n, n2 = n[keep], n2[keep]
    vals, shell = np.unique(n2, return_inverse=True)
    return 2 * np.pi * n / L, shell, 2 * np.pi * np.sqrt(vals) / L
