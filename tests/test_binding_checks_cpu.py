"""The Python binding refuses, before any library call, arrays whose element type,
shape or element count differ from what the C ABI reads (positions FP64 N x 3;
forces, w1 (N x 8), w2 (6 Ng^2 (Ng/2 + 1) per suspension) and wt in the handle's
precision): such an array would be read past its end on the device.  Checked on
the CPU with a handle-less object, since creating a handle needs a GPU."""
import numpy as np
import pytest

from paper_1709_06946_gb300 import binding


class _Unreachable:
    """Stands in for the library: any call means a check let a bad array through."""

    def __getattr__(self, name):
        raise AssertionError('library call %s reached with an invalid argument' % name)


def _handle(Ns, Ngs, precision='mixed'):
    h = binding.PSE.__new__(binding.PSE)
    h.Ns = list(Ns)
    h.N = int(sum(Ns))
    h.nsys = len(Ns)
    h.prec = binding._precision(precision)
    h.dtype = np.float64 if h.prec == binding.PSE_FP64 else np.float32
    h._lib = _Unreachable()
    h._h = None
    h.system_info = lambda s: {'Ng': Ngs[s]}
    return h


def _nk(g):
    return g * g * (g // 2 + 1)


@pytest.mark.parametrize('precision', ['mixed', 'fp64'])
def test_valid_arguments_pass(precision):
    h = _handle([50, 70], [24, 32], precision)
    dt = h.dtype
    N = 120
    pos = np.zeros((N, 3))
    w2 = np.zeros(6 * (_nk(24) + _nk(32)), dtype=dt)
    h._check_step_args(pos, np.zeros((N, 3), dt), np.zeros((N, 8), dt), w2, np.zeros((N, 3), dt))
    # w1 flattened and w2 in the (3, Ng, Ng, Ng/2 + 1, 2) layout of a single suspension
    h1 = _handle([N], [24], precision)
    h1._check_step_args(pos, None, np.zeros(8 * N, dt), np.zeros((3, 24, 24, 13, 2), dt))


def test_positions_must_be_fp64_n_by_3():
    h = _handle([100], [24])
    for bad in (np.zeros((100, 3), np.float32), np.zeros((99, 3)), np.zeros((100, 4)), np.zeros(300)):
        with pytest.raises(ValueError, match='pos'):
            h._check_step_args(bad)
    for call in (lambda p: h.brownian(p, 1e-3), lambda p: h.step(p, 1e-3), lambda p: h.rfd_step(p, 1e-3),
                 lambda p: h.overlap_force(p, 1.0), lambda p: h.autotune(p)):
        with pytest.raises(ValueError, match='pos'):
            call(np.zeros((100, 3), np.float32))


def test_forces_and_noise_follow_the_handle_precision():
    h = _handle([100], [24], 'mixed')
    pos = np.zeros((100, 3))
    with pytest.raises(ValueError, match='FP'):
        h.step(pos, 1e-3, FP=np.zeros((100, 3)))                      # FP64 forces on a mixed handle
    with pytest.raises(ValueError, match='w1'):
        h.brownian(pos, 1e-3, w1=np.zeros((100, 8)), w2=np.zeros(6 * _nk(24), np.float32))
    with pytest.raises(ValueError, match='w1'):
        h.step(pos, 1e-3, w1=np.zeros((100, 7), np.float32), w2=np.zeros(6 * _nk(24), np.float32))
    with pytest.raises(ValueError, match='w2'):
        h.step(pos, 1e-3, w1=np.zeros((100, 8), np.float32), w2=np.zeros(6 * _nk(24) - 2, np.float32))
    with pytest.raises(ValueError, match='wt'):
        h.rfd_step(pos, 1e-3, w1=np.zeros((100, 8), np.float32), w2=np.zeros(6 * _nk(24), np.float32),
                   wt=np.zeros((100, 3)))


def test_batch_noise_counts_every_suspension():
    h = _handle([40, 60], [24, 36], 'fp64')
    pos = np.zeros((100, 3))
    w1 = np.zeros((100, 8))
    with pytest.raises(ValueError, match='w2'):                     # only the first suspension's block
        h.brownian(pos, 1e-3, w1=w1, w2=np.zeros(6 * _nk(24)))
    h._check_step_args(pos, None, w1, np.zeros(6 * (_nk(24) + _nk(36))))


def test_server_requests_are_checked():
    srv = binding.Server.__new__(binding.Server)
    srv._lib = _Unreachable()
    pos = np.zeros((64, 3))
    with pytest.raises(ValueError, match='pos'):
        srv.submit('mobility', pos.astype(np.float32), 30.0)
    with pytest.raises(ValueError, match='F'):
        srv.submit('mobility', pos, 30.0, F=np.zeros((64, 3)), S=np.zeros((64, 5), np.float32))
    with pytest.raises(ValueError, match='S'):
        srv.submit('mobility', pos, 30.0, precision='fp64', F=np.zeros((64, 3)), S=np.zeros((64, 4)))
