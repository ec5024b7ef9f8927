"""Pins for oracle.philox: Random123 known-answer vectors of Philox4x32-10."""
import numpy as np

from oracle.philox import normals, philox4x32_10


def test_kat_zero():
    out = philox4x32_10(np.zeros(4, np.uint32), np.zeros(2, np.uint32))
    assert [int(v) for v in out] == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]


def test_kat_ones():
    out = philox4x32_10(np.full(4, 0xffffffff, np.uint32), np.full(2, 0xffffffff, np.uint32))
    assert [int(v) for v in out] == [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]


def test_normals_moments():
    z0, z1 = normals(12345, 7, 2, np.arange(200000))
    for z in (z0, z1):
        assert abs(z.mean()) < 0.01
        assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z0 * z1)) < 0.01
