"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/pse.h declares, and its host-side pieces (real-space table generator,
tridiagonal square root) agree with the oracle.  No GPU compute is issued."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1709_06946_gb300 as pkg
from oracle import realspace as R
from oracle.basis import Y

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def lib():
    pkg.build()
    return pkg.load()


def test_exports_every_header_symbol(lib):
    hdr = open(os.path.join(ROOT, 'include', 'pse.h')).read()
    names = set(re.findall(r'^(?:pse_status|void|const char|int32_t)\s*\*?\s*(pse_[a-z_0-9]+)\s*\(', hdr, re.M))
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    declared = {n for n, _, _ in pkg.binding.SIGNATURES}
    assert names == declared


def test_default_options(lib):
    o = pkg.binding.Options()
    lib.pse_default_options(ctypes.byref(o))
    assert o.rule == 0 and o.lanczos_maxiter == 100 and o.krylov_maxiter == 50 and o.grid_ladder == 1
    assert o.lanczos_tol < 0 and o.krylov_tol < 0


def test_invalid_arguments_rejected(lib):
    h = ctypes.c_void_p()
    o = pkg.binding.Options()
    lib.pse_default_options(ctypes.byref(o))
    # r_cut = 1 + sqrt(ln(1e4))/0.5 = 7.07 > L/2 = 5: rejected before any device call
    assert lib.pse_create(ctypes.byref(h), 10, 10.0, 1.0, 1.0, 1.0, 0.5, 1e-3, 0, ctypes.byref(o)) == 1
    assert b'exceeds the half-width 5.0' in lib.pse_last_error(None)
    # a sheared cell (strain 1/2) is narrower: L sqrt(lambda_min)/2 = 7.81 < r_cut 7.98 at L = 20, xi = 0.43
    for i, v in enumerate([1.0, 0.5, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0]):
        o.deform[i] = v
    assert lib.pse_create(ctypes.byref(h), 10, 20.0, 1.0, 1.0, 1.0, 0.43, 1e-3, 0, ctypes.byref(o)) == 1
    assert b'half-width 7.8' in lib.pse_last_error(None)
    # det A <= 0 is refused
    for i, v in enumerate([1.0, 0.0, 0.0, 0.0, -1.0, 0.0, 0.0, 0.0, 1.0]):
        o.deform[i] = v
    assert lib.pse_create(ctypes.byref(h), 10, 20.0, 1.0, 1.0, 1.0, 0.8, 1e-3, 0, ctypes.byref(o)) == 1
    assert b'det A > 0' in lib.pse_last_error(None)
    lib.pse_default_options(ctypes.byref(o))
    assert lib.pse_create(ctypes.byref(h), 0, 30.0, 1.0, 1.0, 1.0, 0.5, 1e-3, 0, ctypes.byref(o)) == 1
    assert lib.pse_create(ctypes.byref(h), 10, 30.0, 1.0, 1.0, 1.0, 0.5, 0.5, 0, ctypes.byref(o)) == 1
    assert lib.pse_status_string(4) == b'Krylov iteration cap reached'


def _yv(M):
    return np.einsum('ij,kij->k', M, Y)


def _block(f, rh):
    fp, fr, gS, gR, kS, kX, kR = f
    B = np.zeros((8, 8))
    for c in range(8):
        e = np.zeros(8)
        e[c] = 1
        F, s = e[:3], e[3:]
        S = np.einsum('k,kij->ij', s, Y)
        v = S @ rh
        q = rh @ v
        U = fp * F + (fr - fp) * (rh @ F) * rh + gS * v + gR * q * rh
        E = (-(gS / 2) * _yv(np.outer(F, rh) + np.outer(rh, F)) - gR * (rh @ F) * _yv(np.outer(rh, rh))
             + kS * s + kX * _yv(np.outer(v, rh) + np.outer(rh, v)) + kR * q * _yv(np.outer(rh, rh)))
        B[:, c] = np.concatenate([U, E])
    return B


@pytest.mark.parametrize('xi,eta,a', [(0.5, 1.0, 1.0), (0.8, 1.7, 1.3)])
def test_table_functions_match_oracle(lib, xi, eta, a):
    rs = np.array([0.5, 1.0, 1.7, 1.999, 2.0, 2.001, 2.6, 3.5, 5.0, 7.0]) * a
    out = np.zeros((rs.size, 7))
    self2 = np.zeros(2)
    lib.pse_internal_real_functions(ctypes.c_double(a), ctypes.c_double(eta), ctypes.c_double(xi), rs.size,
                                    rs.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                    self2.ctypes.data_as(ctypes.c_void_p))
    Bs = R.self_block(xi, a, eta)
    assert self2[0] == pytest.approx(Bs[0, 0], rel=1e-13)
    assert self2[1] == pytest.approx(Bs[3, 3], rel=1e-13)
    rng = np.random.default_rng(0)
    for r, f in zip(rs, out):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Bo = R.pair_blocks((d * r)[None], xi, a, eta)[0]
        assert np.abs(_block(f, d) - Bo).max() < 1e-13 * max(1.0, np.abs(Bo).max() / 1e-3)


def test_tridiagonal_square_root(lib):
    rng = np.random.default_rng(1)
    for n in (1, 2, 7, 40):
        d = rng.uniform(0.5, 2.0, n)
        e = rng.uniform(-0.4, 0.4, max(n - 1, 1))[:max(n - 1, 0)]
        c = np.zeros(n)
        ep = e if n > 1 else np.zeros(1)
        assert lib.pse_internal_tridiag_sqrt_e1(n, d.ctypes.data_as(ctypes.c_void_p),
                                                ep.ctypes.data_as(ctypes.c_void_p),
                                                c.ctypes.data_as(ctypes.c_void_p)) == 0
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        w, Q = np.linalg.eigh(T)
        assert np.abs(c - Q @ (np.sqrt(w) * Q[0])).max() < 1e-13


def _tile(lib, Ng, P, ts, caps, fixed=(0, 0, 0)):
    c = (ctypes.c_int * 3)(*caps)
    f = (ctypes.c_int * 3)(*fixed)
    out = (ctypes.c_int * 4)()
    rc = lib.pse_internal_choose_tile(Ng, P, ts, c, f, out)
    return rc, list(out)


def test_spreading_tile_rules(lib):
    """The tile chosen for every 2^i 3^j grid, support and real size under the
    autotuner's caps divides N_g, spans at least P - 1 points (or the whole
    side), fits the shared-memory budget with 8 components, and its rows are
    padded by the documented rule (rows of 16 or more: length = P mod 8)."""
    grids = sorted({2 ** i * 3 ** j for i in range(1, 10) for j in range(0, 6) if 8 <= 2 ** i * 3 ** j <= 512})
    caps_list = [(16, 16, 16), (16, 8, 16), (8, 8, 16), (8, 16, 16), (16, 16, 32), (16, 8, 32), (32, 8, 16)]
    for Ng in grids:
        for P in (4, 5, 6, 8, 10):
            for ts in (4, 8):
                for caps in caps_list:
                    rc, (tx, ty, tz, row) = _tile(lib, Ng, P, ts, caps)
                    if rc:  # refused only when even the smallest admissible tile is too large
                        m = min(d for d in range(1, Ng + 1) if Ng % d == 0 and (d >= P - 1 or d == Ng))
                        mrow = m + ((P - m) % 8 if m >= 16 else (2 if m % 4 == 0 else 0))
                        assert 8 * m * m * mrow * ts > 220 * 1024, (Ng, P, ts, caps)
                        continue
                    for t in (tx, ty, tz):
                        assert Ng % t == 0 and (t >= P - 1 or t == Ng) and t <= 256
                    if tx >= 16:
                        assert row % 8 == P % 8 and tx <= row < tx + 8
                    else:
                        assert row == tx + (2 if tx % 4 == 0 else 0)
                    assert 8 * tz * ty * row * ts <= 220 * 1024, (Ng, P, ts, caps, tx, ty, tz)
    # the benchmark's grid: 16^3 tiles in mixed precision, rows of 22 points for P = 6
    assert _tile(lib, 256, 6, 4, (16, 16, 16)) == (0, [16, 16, 16, 22])
    # a forced tile that cannot fit is refused
    assert _tile(lib, 256, 6, 8, (16, 16, 16), fixed=(32, 32, 32))[0] == 1


def test_batch_arguments_checked_on_host(lib):
    """Batch creation checks every suspension before touching the device and
    names the one that fails; the memory estimate needs no device."""
    h = ctypes.c_void_p()
    o = pkg.binding.Options()
    lib.pse_default_options(ctypes.byref(o))
    N = np.array([100, 10, 50], dtype=np.int64)
    L = np.array([16.2, 9.0, 20.0])
    assert lib.pse_create_batch(ctypes.byref(h), 3, N.ctypes.data, L.ctypes.data, 1.0, 1.0, 1.0, 0.5, 1e-3, 0,
                                ctypes.byref(o)) == 1
    assert b'suspension 1' in lib.pse_last_error(None)
    assert lib.pse_create_batch(ctypes.byref(h), 0, N.ctypes.data, L.ctypes.data, 1.0, 1.0, 1.0, 0.5, 1e-3, 0,
                                ctypes.byref(o)) == 1
    assert lib.pse_num_systems(None) == 0


def test_memory_estimate(lib):
    est = pkg.binding.estimate_bytes
    one = est(100000, 80.0, xi=0.5, tol=1e-3)
    assert one > 100000 * 8 * 4 * 100          # at least the Krylov basis
    assert est(200000, 100.8, xi=0.5, tol=1e-3) > 1.8 * one
    assert est(100000, 80.0, xi=0.5, tol=1e-3, precision='fp64') > 1.5 * one   # reals double, indices do not
    both = est([100000, 100000], [80.0, 80.0], xi=0.5, tol=1e-3)
    assert abs(both - 2 * one) < 0.05 * one
    with pytest.raises(pkg.PSEError):
        est([100, 10], [16.2, 9.0])


def test_grid_ladder_rounds_to_three_smooth(lib):
    """With grid_ladder the grid is the next even 2^i 3^j size at or above the rule's grid."""
    h = ctypes.c_void_p()
    for L in (20.0, 37.0, 61.0, 118.0):
        b0 = pkg.binding.estimate_bytes(1000, L, xi=0.5, grid_ladder=0)
        b1 = pkg.binding.estimate_bytes(1000, L, xi=0.5, grid_ladder=1)
        assert b1 >= b0


def test_server_needs_a_device(lib):
    """Without a GPU the server refuses to start (CUDA error), it does not crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip('a device is present')
    srv = ctypes.c_void_p()
    assert lib.pse_server_create(ctypes.byref(srv), 2, 1 << 30) == 3
    assert lib.pse_server_create(ctypes.byref(srv), 0, 1 << 30) == 1
