"""Equilibrium validation runs of Sec. 4 through the library's own steps.

* ``pair_distance_run``: two spheres joined by U(r) = k |r - r0| (minimum-image
  centre distance r), advanced by the constrained mid-point step (or the RFD
  Euler-Maruyama step) with the spring force F = -k sign(r - r0) r^ passed as the
  conservative force at x_k; returns the sampled distances, whose distribution
  must be the Boltzmann density r^2 exp(-U/kT) (normalised).
* ``ideal_structure_factor_run``: non-interacting spheres (no force, overlaps
  allowed) advanced by constrained steps; returns the static structure factor
  S(q) = |sum_j exp(i q.x_j)|^2 / N per shell of the box's wave vectors, averaged
  over snapshots, which must stay 1 at equilibrium.

The forces and the structure factor are evaluated with torch tensor operations on
the device (analysis around the steps, not part of the method); every step is a
call of the C ABI.
"""
import math

import numpy as np


def _torch():
    import torch
    return torch


def boltzmann_pair_reference(k, r0, kT=1.0, rmax=None, n=200001):
    """Grid (r, CDF, mean) of the density r^2 exp(-k |r - r0| / kT) on [0, rmax],
    normalised numerically (trapezoid rule): the reference of the bench line."""
    kt = k / kT
    rmax = r0 + 40.0 / kt if rmax is None else rmax
    r = np.linspace(0.0, rmax, n)
    w = r * r * np.exp(-kt * np.abs(r - r0))
    c = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(r))])
    Z = c[-1]
    mean = np.sum(0.5 * (r[1:] * w[1:] + r[:-1] * w[:-1]) * np.diff(r)) / Z
    return r, c / Z, mean


def spring_force(x, L, k, r0, dtype):
    """F (2, 3) on the two spheres from U = k |r - r0| (torch, on x's device)."""
    torch = _torch()
    d = x[0] - x[1]
    d = d - L * torch.round(d / L)
    r = torch.linalg.norm(d)
    f = -k * torch.sign(r - r0) * d / r
    return torch.stack([f, -f]).to(dtype).contiguous()


def pair_distance_run(h, x, L, k, r0, dt, steps, every=1, seed=0, scheme='midpoint', delta=0.0, burn=0):
    """Distances |x_0 - x_1| (minimum image) after every `every`-th step past `burn`."""
    torch = _torch()
    dtype = torch.float64 if h.dtype == np.float64 else torch.float32
    out = []
    for n in range(burn + steps):
        F = spring_force(x, L, k, r0, dtype)
        if scheme == 'rfd':
            h.rfd_step(x, dt, FP=F, delta=delta, seed=seed, step=n)
        else:
            h.step(x, dt, FP=F, seed=seed, step=n)
        if n >= burn and (n - burn) % every == 0:
            d = x[0] - x[1]
            d = d - L * torch.round(d / L)
            out.append(torch.linalg.norm(d))
    return torch.stack(out).cpu().numpy()


def _qshells(L, nmax, device):
    torch = _torch()
    g = torch.arange(-nmax, nmax + 1, device=device)
    n = torch.stack(torch.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    n2 = (n * n).sum(1)
    half = (n[:, 2] > 0) | ((n[:, 2] == 0) & (n[:, 1] > 0)) | ((n[:, 2] == 0) & (n[:, 1] == 0) & (n[:, 0] > 0))
    keep = half & (n2 > 0) & (n2 <= nmax * nmax)
    n, n2 = n[keep], n2[keep]
    vals, shell = torch.unique(n2, return_inverse=True)
    return (2 * math.pi / L) * n.double(), shell, (2 * math.pi / L) * torch.sqrt(vals.double())


def structure_factor(x, L, nmax):
    """Shell averages of S(q) for |n| <= nmax (q = 2 pi n / L); returns (|q|, S, vectors per shell)."""
    torch = _torch()
    q, shell, qs = _qshells(L, nmax, x.device)
    ph = x.double() @ q.T                                  # (N, nq)
    re, im = torch.cos(ph).sum(0), torch.sin(ph).sum(0)
    S = (re * re + im * im) / x.shape[0]
    cnt = torch.zeros(len(qs), device=x.device, dtype=torch.float64).index_add_(0, shell, torch.ones_like(S))
    Ssh = torch.zeros(len(qs), device=x.device, dtype=torch.float64).index_add_(0, shell, S) / cnt
    return qs.cpu().numpy(), Ssh.cpu().numpy(), cnt.cpu().numpy()


def ideal_structure_factor_run(h, x, L, dt, steps, every, nmax, seed=0):
    """S(q) shell averages over the snapshots after every `every`-th step (no forces)."""
    snaps = []
    for n in range(steps):
        h.step(x, dt, seed=seed, step=n)
        if (n + 1) % every == 0:
            snaps.append(structure_factor(x, L, nmax))
    qs = snaps[0][0]
    S = np.array([s[1] for s in snaps])
    return qs, S, snaps[0][2]
