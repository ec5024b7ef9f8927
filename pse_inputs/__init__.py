"""Seeded synthetic inputs for the PSE tests and benchmark.

Holds none of the method's arithmetic: hard-sphere configurations by random
sequential addition (RSA, compiled C in rsa.c), standard-normal forces and
stresslets, and standard-normal noise arrays in the layouts of the C ABI.
Both the oracle side and the CUDA side of a test receive the same arrays.

Workload recipe: a = eta = kT = 1, box L = (4 pi N / (3 phi))^{1/3},
positions by RSA for phi <= 0.35 and, above (RSA jams near phi = 0.38), by
overlap removal from uniform centres followed by hard-sphere Monte Carlo
sweeps; forces and stresslet components (orthonormal basis) i.i.d. N(0, 1)
from numpy's PCG64 with the given seed.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, '_rsa.so')
_lib = None


def build():
    """Compile the RSA generator in place (gcc, no architecture flags)."""
    src = os.path.join(_HERE, 'rsa.c')
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + '.%d.tmp' % os.getpid()
        subprocess.check_call(['gcc', '-O2', '-shared', '-fPIC', src, '-o', tmp, '-lm'])
        os.replace(tmp, _LIB)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.pse_rsa.restype = ctypes.c_int64
        lib.pse_rsa.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                ctypes.c_int64, ctypes.c_void_p]
        lib.pse_pack.restype = ctypes.c_int64
        lib.pse_pack.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                 ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        _lib = lib
    return _lib


def box_length(N, phi, a=1.0):
    return (4.0 * math.pi * N * a ** 3 / (3.0 * phi)) ** (1.0 / 3.0)


def rsa_positions(N, phi, seed=1, a=1.0, L=None):
    """(N, 3) float64 hard-sphere centres in [0, L)^3 and the box length L."""
    if L is None:
        L = box_length(N, phi, a)
    pos = np.empty((N, 3), dtype=np.float64)
    got = _load().pse_rsa(N, L, a, seed, 2000 * N + 10000, pos.ctypes.data)
    if got != N:
        raise RuntimeError('RSA placed %d of %d spheres (phi too high for RSA?)' % (got, N))
    return pos, L


def packed_positions(N, phi, seed=1, a=1.0, sweeps=100):
    """Hard-sphere centres at densities RSA cannot reach: overlap removal from
    uniform centres, then `sweeps` Monte Carlo sweeps.  Returns (pos, L)."""
    L = box_length(N, phi, a)
    pos = np.empty((N, 3), dtype=np.float64)
    if _load().pse_pack(N, L, a, seed, sweeps, 20000, pos.ctypes.data) != 0:
        raise RuntimeError('could not remove the overlaps at phi = %g' % phi)
    return pos, L


def hard_sphere_positions(N, phi, seed=1, a=1.0):
    """RSA for phi <= 0.35, packed_positions above."""
    return rsa_positions(N, phi, seed, a) if phi <= 0.35 else packed_positions(N, phi, seed, a)


def random_positions(N, L, seed=1):
    """Uniform (possibly overlapping) positions, for positivity tests."""
    return np.random.default_rng(seed).uniform(0.0, L, size=(N, 3))


def moments(N, seed=2):
    """Forces F (N,3) and stresslet components S (N,5), i.i.d. N(0,1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, 3)), rng.standard_normal((N, 5))


def lanczos_noise(N, seed=3):
    """w1: (N, 8) standard normals (Lanczos start vector)."""
    return np.random.default_rng(seed).standard_normal((N, 8))


def wave_noise(Ng, seed=4):
    """w2: (3, Ng, Ng, Ng/2+1, 2) standard normals (real, imaginary parts)."""
    return np.random.default_rng(seed).standard_normal((3, Ng, Ng, Ng // 2 + 1, 2))
