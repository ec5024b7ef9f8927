"""Pins for the oracle on deformed lattices (Sec. 2.3.3).

The periodic cell is spanned by the columns of L A (simple shear, planar
extension, or any A with det A > 0).  What fixes the oracle here, independently
of its own formulas:

* the lattice metrics against the closed forms of Eqs. lmax1 and lmax2;
* exact identities of the periodic sum: a shear with integer strain describes
  the cubic lattice again, and a sheared cell with its particles copied by one
  lattice vector is an orthorhombic cell, which copied again is a cube: the
  dense Ewald mobilities of these descriptions agree to rounding;
* xi-independence of the dense sum on sheared, extended and general lattices,
  and positivity of each part of the split (App. C);
* the NUFFT on the deformed grid equals the direct sum over the same wave
  vectors (tight quadrature: to 1e-10);
* the oracle's real-space pair list equals a brute-force image sum;
* the PSE product lies within the tolerance of the dense sum when the support
  follows Eq. (bound) with lambda_max, and is worse with the orthorhombic rule
  lambda_max = 1 (the comparison of Fig. fig:shear; for the extension past the
  tolerance by an order of magnitude);
* wrapping moves every particle by a lattice vector into the cell.
"""
import math

import numpy as np
import pytest

import pse_inputs
from oracle import ewald, params, pse, wavesum


def _vec(U, E):
    return np.concatenate([U, E], axis=1).ravel()


GENERAL = np.array([[1.0, 0.2, 0.1], [0.0, 1.1, 0.15], [0.05, 0.0, 0.9]])


@pytest.mark.parametrize('gamma', [0.0, 0.1, 0.5, 1.0, 2.0])
def test_shear_metrics_closed_form(gamma):
    lmin, lmax, det, _ = params.lattice_metrics(params.shear_tensor(gamma))
    assert abs(lmax - params.lambda_max_shear(gamma)) < 1e-12 * lmax
    assert abs(det - 1.0) < 1e-14
    assert abs(lmin * lmax - 1.0) < 1e-12          # det(A^T A) = 1 with z untouched


@pytest.mark.parametrize('eps', [0.5, 0.8, 1.0, 1.1, 1.5, 2.0])
def test_extension_metrics_closed_form(eps):
    lmin, lmax, det, _ = params.lattice_metrics(params.extension_tensor(eps))
    assert abs(lmax - params.lambda_max_ext(eps)) < 1e-12 * lmax
    assert abs(det - 1.0) < 1e-14


@pytest.mark.parametrize('gamma', [1.0, -1.0, 2.0])
def test_integer_shear_is_the_cubic_lattice(gamma):
    pos = pse_inputs.random_positions(4, 7.0, seed=5)
    M0 = ewald.dense_mobility(pos, 7.0, xi=0.6, tol=1e-15)
    M1 = ewald.dense_mobility(pos, 7.0, xi=0.6, tol=1e-15, A=params.shear_tensor(gamma))
    assert np.abs(M1 - M0).max() / np.abs(M0).max() < 1e-12
    M2 = ewald.dense_mobility(pos, 7.0, xi=0.6, tol=1e-15, A=params.shear_tensor(0.4))
    assert np.abs(M2 - M0).max() / np.abs(M0).max() > 1e-3  # a non-integer strain is another lattice


def test_replicated_cells():
    """Sheared cell (strain 1/2) == orthorhombic (L, 2L, L) cell with the particles
    copied by L A e_2 == cube of side 2L with those copied by L e_x and L e_z."""
    L, N = 6.0, 2
    A = params.shear_tensor(0.5)
    pos = pse_inputs.random_positions(N, L, seed=7)
    v = np.random.default_rng(1).standard_normal(8 * N)
    Ms = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15, A=A)
    pos2 = np.concatenate([pos, pos + L * A[:, 1]])
    Mo = ewald.dense_mobility(pos2, L, xi=0.6, tol=1e-15, A=np.diag([1.0, 2.0, 1.0]))
    pos8 = np.concatenate([pos2 + np.array([i * L, 0.0, k * L]) for i in (0, 1) for k in (0, 1)])
    Mc = ewald.dense_mobility(pos8, 2 * L, xi=0.6, tol=1e-15)
    u_s = Ms @ v
    u_o = (Mo @ np.concatenate([v, v]))[:8 * N]
    u_c = (Mc @ np.tile(np.concatenate([v, v]), 4))[:8 * N]
    scale = np.abs(u_s).max()
    assert np.abs(u_o - u_s).max() < 1e-12 * scale
    assert np.abs(u_c - u_o).max() < 1e-12 * scale


@pytest.mark.parametrize('A', [params.shear_tensor(0.3), params.extension_tensor(1.3), GENERAL],
                         ids=['shear', 'extension', 'general'])
def test_xi_independence_deformed(A):
    pos = pse_inputs.random_positions(5, 7.0, seed=3)
    Ma = ewald.dense_mobility(pos, 7.0, xi=0.5, tol=1e-15, A=A)
    Mb = ewald.dense_mobility(pos, 7.0, xi=0.9, tol=1e-15, A=A)
    assert np.abs(Ma - Mb).max() / np.abs(Ma).max() < 1e-12


def test_parts_positive_deformed():
    pos = pse_inputs.random_positions(6, 7.0, seed=9)
    Mr, Mw = ewald.dense_mobility(pos, 7.0, xi=0.7, tol=1e-15, parts=True, A=params.shear_tensor(0.5))
    for M in (Mr, Mw):
        assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
        np.linalg.cholesky(M)


@pytest.mark.parametrize('A', [params.shear_tensor(0.5), params.extension_tensor(1.5), GENERAL],
                         ids=['shear', 'extension', 'general'])
@pytest.mark.parametrize('tight', [False, True])
def test_nufft_equals_direct_ksum_deformed(A, tight):
    N, L, xi = 12, 9.0, 0.6
    pos = pse_inputs.random_positions(N, L, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    if tight:
        p = params.choose(N, L, 1.0, 1.0, 1.0, xi, 1e-12, rule='paper', rcut=0.3 * L, A=A, Ng=48)
    else:
        p = params.choose(N, L, 1.0, 1.0, 1.0, xi, 1e-3, rule='paper', rcut=0.3 * L, A=A)
    assert p.P <= p.Ng
    w = pse.wave_apply(pos, F, S, p)
    Mw = wavesum.dense_wave(pos, L, 1.0, 1.0, xi, wavesum.kset_grid(L, p.Ng, A=A), V=p.V)
    ref = Mw @ np.concatenate([F, S], 1).ravel()
    err = np.linalg.norm(_vec(w['U'], w['E']) - ref) / np.linalg.norm(ref)
    assert err < (1e-10 if tight else 1e-2)


@pytest.mark.parametrize('A', [params.shear_tensor(0.5), GENERAL], ids=['shear', 'general'])
def test_real_pairs_equal_image_sum(A):
    N = 100
    pos, L = pse_inputs.rsa_positions(N, 0.2, seed=4)
    p = params.choose(N, L, 1.0, 1.0, 1.0, 1.0, 1e-3, A=A)
    M_oracle = pse.RealOp(pos, p).dense()
    M_images = ewald.dense_real(pos, L, 1.0, 1.0, 1.0, p.rcut, A=A)
    assert np.abs(M_oracle - M_images).max() < 1e-12 * np.abs(M_images).max()


@pytest.fixture(scope='module')
def dense_case():
    N, phi = 100, 0.1
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    out = {}
    for name, A in (('shear', params.shear_tensor(0.5)), ('extension', params.extension_tensor(1.5))):
        M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15, A=A)
        out[name] = (A, M @ np.concatenate([F, S], 1).ravel())
    return pos, L, F, S, out


@pytest.mark.parametrize('name', ['shear', 'extension'])
def test_lambda_aware_support_meets_tolerance(dense_case, name):
    pos, L, F, S, out = dense_case
    A, ref = out[name]
    tol = 1e-3
    errs = {}
    for aware in (True, False):
        p = params.choose(pos.shape[0], L, 1.0, 1.0, 1.0, 0.7, tol, A=A, lambda_aware=aware)
        U, E = pse.mobility_apply(pos, F, S, p)
        errs[aware] = np.linalg.norm(_vec(U, E) - ref) / np.linalg.norm(ref)
    assert errs[True] < tol
    assert errs[False] > 3 * errs[True]
    if name == 'extension':  # lambda_max = 2.25: the orthorhombic rule misses the tolerance by 10x
        assert errs[False] > 10 * tol


def test_wrap_is_a_lattice_translation():
    A = params.shear_tensor(0.5)
    p = params.choose(50, 20.0, 1.0, 1.0, 1.0, 0.8, 1e-3, A=A)
    x = np.random.default_rng(3).uniform(-50, 50, (50, 3))
    xw = pse.wrap_positions(x, p)
    z = xw @ np.linalg.inv(A).T
    assert np.all(z >= 0) and np.all(z < p.L)
    n = (x - xw) @ np.linalg.inv(A).T / p.L
    assert np.abs(n - np.rint(n)).max() < 1e-10
