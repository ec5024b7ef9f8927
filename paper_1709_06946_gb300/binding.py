"""Thin ctypes binding of the C ABI in include/pse.h (argument marshalling only).

Every computation runs in the CUDA library ``libpse.so`` built in this
directory; importing this module never falls back to anything else, and the
first call fails with an explicit error if the library is missing.
Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must be
C-contiguous with float64 positions and float32 (PSE_MIXED) / float64
(PSE_FP64) moments.  Results are returned as torch tensors on the device of
``pos`` (torch input) or as numpy arrays (numpy input).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'libpse.so')

PSE_MIXED, PSE_FP64 = 0, 1
PSE_RULE_STRICT, PSE_RULE_PAPER = 0, 1
PARTS = {'real': 1, 'wave': 2, 'all': 3}
STATUS = {0: 'ok', 1: 'invalid argument', 2: 'out of device memory', 3: 'CUDA error',
          4: 'Krylov iteration cap reached', 5: 'non-finite input', 6: 'device wait timed out'}


class Options(ctypes.Structure):
    _fields_ = [('rule', ctypes.c_int32), ('Ng', ctypes.c_int32), ('P', ctypes.c_int32),
                ('table_points', ctypes.c_int32), ('rcut', ctypes.c_double),
                ('lanczos_tol', ctypes.c_double), ('lanczos_maxiter', ctypes.c_int32),
                ('krylov_tol', ctypes.c_double), ('krylov_maxiter', ctypes.c_int32),
                ('tile', ctypes.c_int32 * 3), ('real_lanes', ctypes.c_int32), ('grid_ladder', ctypes.c_int32),
                ('use_graph', ctypes.c_int32), ('wave_kernel', ctypes.c_int32), ('torque', ctypes.c_int32),
                ('lambda_support', ctypes.c_int32), ('reserved', ctypes.c_int32 * 2),
                ('deform', ctypes.c_double * 9)]


class Info(ctypes.Structure):
    _fields_ = [('N', ctypes.c_int64), ('L', ctypes.c_double), ('a', ctypes.c_double),
                ('eta', ctypes.c_double), ('kT', ctypes.c_double), ('xi', ctypes.c_double),
                ('tol', ctypes.c_double), ('precision', ctypes.c_int32), ('rule', ctypes.c_int32),
                ('rcut', ctypes.c_double), ('kcut', ctypes.c_double), ('h', ctypes.c_double),
                ('eta_g', ctypes.c_double), ('m', ctypes.c_double), ('Ng', ctypes.c_int32),
                ('P', ctypes.c_int32), ('cells_per_side', ctypes.c_int32), ('tile', ctypes.c_int32 * 3),
                ('table_len', ctypes.c_int32), ('table_dr', ctypes.c_double),
                ('device_bytes', ctypes.c_int64), ('deformed', ctypes.c_int32), ('tile_kernels', ctypes.c_int32),
                ('deform', ctypes.c_double * 9), ('lambda_max', ctypes.c_double),
                ('lambda_min_cells', ctypes.c_double), ('colnorm_max', ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [('lanczos_iters', ctypes.c_int32), ('krylov_iters', ctypes.c_int32),
                ('lanczos_change', ctypes.c_double), ('krylov_relres', ctypes.c_double),
                ('neighbor_pairs', ctypes.c_int64), ('products', ctypes.c_int32),
                ('reserved', ctypes.c_int32 * 5)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != 'reserved'}


NSTAGES = 8
STAGES = ['setup', 'real', 'spread', 'fft', 'scale', 'interp', 'noise', 'vector']


NVARIANTS = 4
VARIANTS = ('full', 'se', 'fsu', 'su')


class Profile(ctypes.Structure):
    _fields_ = [('ms', ctypes.c_double * NSTAGES), ('calls', ctypes.c_int64 * NSTAGES),
                ('launches', ctypes.c_int64), ('fft_execs', ctypes.c_int64),
                ('variant_ms', (ctypes.c_double * NVARIANTS) * NSTAGES),
                ('variant_calls', (ctypes.c_int64 * NVARIANTS) * NSTAGES)]


class Request(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32), ('precision', ctypes.c_int32), ('N', ctypes.c_int64),
                ('L', ctypes.c_double), ('a', ctypes.c_double), ('eta', ctypes.c_double), ('kT', ctypes.c_double),
                ('xi', ctypes.c_double), ('tol', ctypes.c_double), ('options', ctypes.POINTER(Options)),
                ('pos', ctypes.c_void_p), ('F', ctypes.c_void_p), ('S', ctypes.c_void_p), ('U', ctypes.c_void_p),
                ('E', ctypes.c_void_p), ('S_out', ctypes.c_void_p), ('dt', ctypes.c_double),
                ('seed', ctypes.c_uint64), ('counter', ctypes.c_uint64), ('stats', ctypes.POINTER(Stats))]


class ServerStats(ctypes.Structure):
    _fields_ = [('completed', ctypes.c_int64), ('queued', ctypes.c_int64), ('running', ctypes.c_int32),
                ('peak_running', ctypes.c_int32), ('p50_ms', ctypes.c_double), ('p99_ms', ctypes.c_double),
                ('wait_p50_ms', ctypes.c_double), ('wait_p99_ms', ctypes.c_double),
                ('service_p50_ms', ctypes.c_double), ('requests_per_s', ctypes.c_double),
                ('resident_bytes', ctypes.c_int64), ('peak_resident_bytes', ctypes.c_int64),
                ('resident_handles', ctypes.c_int32), ('handles_created', ctypes.c_int64),
                ('handles_reused', ctypes.c_int64), ('handles_evicted', ctypes.c_int64),
                ('rejected', ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_KINDS = {'mobility': 0, 'sample': 1, 'step': 2}


class Tuning(ctypes.Structure):
    _fields_ = [('real_lanes', ctypes.c_int32), ('real_smem_table', ctypes.c_int32), ('real_smem_ms', ctypes.c_double),
                ('tile', ctypes.c_int32 * 3), ('best_real_ms', ctypes.c_double),
                ('best_wave_ms', ctypes.c_double), ('n_lanes', ctypes.c_int32), ('n_tiles', ctypes.c_int32),
                ('real_ms', ctypes.c_double * 8), ('tiles', (ctypes.c_int32 * 3) * 8), ('wave_ms', ctypes.c_double * 8)]

# (name, restype, argtypes) of every symbol declared in include/pse.h
_P = ctypes.c_void_p
_D = ctypes.c_double
_U64 = ctypes.c_uint64
SIGNATURES = [
    ('pse_default_options', None, [ctypes.POINTER(Options)]),
    ('pse_create', ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, _D, _D, _D, _D, _D, _D, ctypes.c_int,
                                  ctypes.POINTER(Options)]),
    ('pse_create_batch', ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P, _P, _D, _D, _D, _D, _D,
                                        ctypes.c_int, ctypes.POINTER(Options)]),
    ('pse_estimate_bytes', ctypes.c_int, [ctypes.c_int32, _P, _P, _D, _D, _D, _D, _D, ctypes.c_int,
                                          ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_int64)]),
    ('pse_destroy', ctypes.c_int, [_P]),
    ('pse_get_info', ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    ('pse_set_deformation', ctypes.c_int, [_P, _P, _P]),
    ('pse_num_systems', ctypes.c_int32, [_P]),
    ('pse_graph_ready', ctypes.c_int32, [_P]),
    ('pse_graph_error', ctypes.c_char_p, [_P]),
    ('pse_get_system_info', ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Info)]),
    ('pse_get_system_stats', ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Stats)]),
    ('pse_mobility_apply', ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ('pse_mobility_apply_parts', ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    ('pse_mobility_apply11', ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    ('pse_brownian_sample', ctypes.c_int, [_P, _P, _D, _U64, _U64, _P, _P, _P, _P, ctypes.POINTER(Stats), _P]),
    ('pse_constrained_step', ctypes.c_int, [_P, _P, _P, _D, _U64, _U64, _P, ctypes.POINTER(Stats), _P]),
    ('pse_constrained_step_noise', ctypes.c_int, [_P, _P, _P, _D, _P, _P, _P, ctypes.POINTER(Stats), _P]),
    ('pse_rfd_step', ctypes.c_int, [_P, _P, _P, _D, _D, _U64, _U64, _P, ctypes.POINTER(Stats), _P]),
    ('pse_rfd_step_noise', ctypes.c_int, [_P, _P, _P, _D, _D, _P, _P, _P, _P, ctypes.POINTER(Stats), _P]),
    ('pse_mobility_real_noalloc', ctypes.c_int, [ctypes.c_int64, _D, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P]),
    ('pse_noalloc_last_error', ctypes.c_char_p, []),
    ('pse_server_create', ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int64]),
    ('pse_server_submit', ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    ('pse_server_wait', ctypes.c_int, [_P, ctypes.c_uint64, _D, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(_D)]),
    ('pse_server_get_stats', ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    ('pse_server_reset_stats', ctypes.c_int, [_P]),
    ('pse_server_destroy', ctypes.c_int, [_P]),
    ('pse_overlap_force', ctypes.c_int, [_P, _P, _D, _P, _P]),
    ('pse_autotune', ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(Tuning), _P]),
    ('pse_set_profiling', ctypes.c_int, [_P, ctypes.c_int32]),
    ('pse_get_profile', ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    ('pse_stage_name', ctypes.c_char_p, [ctypes.c_int32]),
    ('pse_sync', ctypes.c_int, [_P]),
    ('pse_status_string', ctypes.c_char_p, [ctypes.c_int]),
    ('pse_last_error', ctypes.c_char_p, [_P]),
]

_lib = None


def load():
    """Loads libpse.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError('libpse.so is not built: run paper_1709_06946_gb300.build() '
                               '(nvcc for sm_103a); there is no CPU fallback')
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class PSEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s: %s' % (STATUS.get(code, code), msg))
        self.code = code


def _torch():
    import torch
    return torch


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags['C_CONTIGUOUS']:
            raise ValueError('arrays must be C-contiguous')
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError('tensors must be contiguous')
    return x.data_ptr()


def _checked(x, shape, dtype, name):
    """x itself after checking its shape and element type (numpy array or torch tensor)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        ok = x.dtype == np.dtype(dtype)
    else:
        torch = _torch()
        ok = x.dtype == (torch.float64 if dtype == np.float64 else torch.float32)
    if not ok:
        raise ValueError(f'{name} must hold {np.dtype(dtype).name} elements, not {x.dtype}')
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f'{name} must have shape {tuple(shape)}, not {tuple(x.shape)}')
    return x


def _checked_size(x, n, dtype, name):
    """x itself after checking its element type and element count (any shape)."""
    if x is None:
        return None
    size = x.size if isinstance(x, np.ndarray) else x.numel()
    _checked(x.reshape(-1), (size,), dtype, name)
    if size != n:
        raise ValueError(f'{name} must hold {n} elements, not {size}')
    return x


def _stream(x):
    try:
        torch = _torch()
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return torch.cuda.current_stream(x.device).cuda_stream
    except ImportError:
        pass
    return None


def mobility_real_noalloc(pos, F, S, L, a=1.0, eta=1.0, xi=0.5, tol=1e-3):
    """Real-space product M_r [F; S] without device allocation (CUDA tensors, float32 moments).

    For callers that cannot allocate device memory: the scratch is a fixed static
    device array inside the library (N <= 65536).  Calls that overlap on the GPU race.
    """
    torch = _torch()
    lib = load()
    if not isinstance(pos, torch.Tensor) or not pos.is_cuda:
        raise ValueError('pos must be a CUDA tensor')
    if pos.dtype != torch.float64 or pos.dim() != 2 or pos.shape[1] != 3 or not pos.is_contiguous():
        raise ValueError('pos must be a contiguous float64 tensor of shape (N, 3)')
    N = pos.shape[0]
    for name, x, ncol in (('F', F, 3), ('S', S, 5)):
        if x is None:
            continue
        if not isinstance(x, torch.Tensor) or x.device != pos.device:
            raise ValueError('%s must be a tensor on %s' % (name, pos.device))
        if x.dtype != torch.float32 or tuple(x.shape) != (N, ncol) or not x.is_contiguous():
            raise ValueError('%s must be a contiguous float32 tensor of shape (%d, %d)' % (name, N, ncol))
    U = torch.empty((N, 3), dtype=torch.float32, device=pos.device)
    E = torch.empty((N, 5), dtype=torch.float32, device=pos.device)
    with torch.cuda.device(pos.device):       # the library uses the current device's scratch
        st = lib.pse_mobility_real_noalloc(int(N), float(L), float(a), float(eta), float(xi), float(tol),
                                           _ptr(pos), _ptr(F), _ptr(S), _ptr(U), _ptr(E), _stream(pos))
    if st != 0:
        raise PSEError(st, lib.pse_noalloc_last_error().decode())
    return U, E


def _options(rule='strict', Ng=0, P=0, rcut=0.0, lanczos_tol=-1.0, lanczos_maxiter=100, krylov_tol=-1.0,
             krylov_maxiter=50, table_points=0, tile=(0, 0, 0), real_lanes=0, grid_ladder=1, use_graph=0,
             wave_kernel=0, torque=0, deform=None, lambda_support=1):
    o = Options()
    load().pse_default_options(ctypes.byref(o))
    o.rule = PSE_RULE_PAPER if rule == 'paper' else PSE_RULE_STRICT
    o.Ng, o.P, o.rcut = int(Ng), int(P), float(rcut)
    o.lanczos_tol, o.lanczos_maxiter = float(lanczos_tol), int(lanczos_maxiter)
    o.krylov_tol, o.krylov_maxiter = float(krylov_tol), int(krylov_maxiter)
    o.table_points = int(table_points)
    o.real_lanes = int(real_lanes)
    o.grid_ladder = int(grid_ladder)
    o.use_graph = int(use_graph)
    o.wave_kernel = int(wave_kernel)
    o.torque = int(torque)
    o.lambda_support = int(lambda_support)
    if deform is not None:
        A = np.asarray(deform, dtype=np.float64).reshape(9)
        for i in range(9):
            o.deform[i] = float(A[i])
    for d in range(3):
        o.tile[d] = int(tile[d])
    return o


def _precision(precision):
    return PSE_FP64 if precision in ('fp64', 'double', PSE_FP64) else PSE_MIXED


def estimate_bytes(N, L, a=1.0, eta=1.0, kT=1.0, xi=0.5, tol=1e-3, precision='mixed', **opts):
    """Device bytes a handle for suspensions N[i], L[i] would allocate (upper estimate)."""
    lib = load()
    Ns = np.ascontiguousarray(np.atleast_1d(N), dtype=np.int64)
    Ls = np.ascontiguousarray(np.atleast_1d(L), dtype=np.float64)
    out = ctypes.c_int64(0)
    o = _options(**opts)
    st = lib.pse_estimate_bytes(len(Ns), Ns.ctypes.data, Ls.ctypes.data, float(a), float(eta), float(kT), float(xi),
                                float(tol), _precision(precision), ctypes.byref(o), ctypes.byref(out))
    if st != 0:
        raise PSEError(st, lib.pse_last_error(None).decode())
    return int(out.value)


class PSE:
    """One PSE handle: N particles in a cubic periodic box of side L, or (N and L
    sequences) a batch of independent suspensions whose arrays are concatenated."""

    def __init__(self, N, L, a=1.0, eta=1.0, kT=1.0, xi=0.5, tol=1e-3, precision='mixed', **opts):
        lib = load()
        o = _options(**opts)
        self.prec = _precision(precision)
        self.dtype = np.float64 if self.prec == PSE_FP64 else np.float32
        h = _P()
        self.batch = np.ndim(N) > 0
        if self.batch:
            Ns = np.ascontiguousarray(N, dtype=np.int64)
            Ls = np.ascontiguousarray(L, dtype=np.float64)
            if Ns.shape != Ls.shape:
                raise ValueError('N and L must have the same length')
            st = lib.pse_create_batch(ctypes.byref(h), len(Ns), Ns.ctypes.data, Ls.ctypes.data, float(a), float(eta),
                                      float(kT), float(xi), float(tol), self.prec, ctypes.byref(o))
            self.Ns = [int(v) for v in Ns]
        else:
            st = lib.pse_create(ctypes.byref(h), int(N), float(L), float(a), float(eta), float(kT), float(xi),
                                float(tol), self.prec, ctypes.byref(o))
            self.Ns = [int(N)]
        if st != 0:
            raise PSEError(st, lib.pse_last_error(None).decode())
        self._h = h
        self._lib = lib
        self.N = int(sum(self.Ns))
        self.nsys = int(lib.pse_num_systems(h))
        self.offsets = np.concatenate([[0], np.cumsum(self.Ns)]).astype(np.int64)
        self.info = self.get_info()

    def graph_ready(self):
        """(captured, reason capture was given up or '')."""
        return bool(self._lib.pse_graph_ready(self._h)), self._lib.pse_graph_error(self._h).decode()

    def system_info(self, s):
        """Parameters of suspension s (grid, cells, tiles, ...)."""
        inf = Info()
        self._check(self._lib.pse_get_system_info(self._h, int(s), ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in Info._fields_}
        d['tile'] = tuple(inf.tile)
        d['deform'] = np.array(inf.deform[:]).reshape(3, 3)
        return d

    def system_stats(self, s):
        """Statistics of suspension s in the last sample or step call."""
        st = Stats()
        self._check(self._lib.pse_get_system_stats(self._h, int(s), ctypes.byref(st)))
        return st.as_dict()

    def _check(self, st):
        if st not in (0,):
            raise PSEError(st, self._lib.pse_last_error(self._h).decode())

    def get_info(self):
        inf = Info()
        self._check(self._lib.pse_get_info(self._h, ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in Info._fields_}
        d['tile'] = tuple(inf.tile)
        d['deform'] = np.array(inf.deform[:]).reshape(3, 3)
        return d

    def set_deformation(self, A, stream=None):
        """Lattice deformation A (3 x 3; the cell is spanned by the columns of L A) for
        the following calls; the handle must have been created with deform=..."""
        Am = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        st = self._lib.pse_set_deformation(self._h, Am.ctypes.data, stream)
        self._check(st)
        self.info = self.get_info()

    def close(self):
        if getattr(self, '_h', None):
            self._lib.pse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- helpers
    def _like(self, ref, shape, dtype):
        if isinstance(ref, np.ndarray):
            return np.zeros(shape, dtype=dtype)
        torch = _torch()
        tdt = torch.float64 if dtype == np.float64 else torch.float32
        return torch.zeros(shape, dtype=tdt, device=ref.device)

    def mobility(self, pos, F=None, S=None, parts='all', want=('U', 'E')):
        """[U, E] = M [F; S] (or its real / wave part)."""
        _checked(pos, (self.N, 3), np.float64, 'pos')
        _checked(F, (self.N, 3), self.dtype, 'F')
        _checked(S, (self.N, 5), self.dtype, 'S')
        U = self._like(pos, (self.N, 3), self.dtype) if 'U' in want else None
        E = self._like(pos, (self.N, 5), self.dtype) if 'E' in want else None
        st = self._lib.pse_mobility_apply_parts(self._h, _ptr(pos), _ptr(F), _ptr(S), _ptr(U), _ptr(E),
                                                PARTS[parts], _stream(pos))
        self._check(st)
        return U, E

    def mobility11(self, pos, F=None, Lt=None, S=None, parts='all'):
        """[U, Omega, E] = M [F; L; S] with torques (handle created with torque=1)."""
        N, dt = self.N, self.dtype
        _checked(pos, (N, 3), np.float64, 'pos')
        F, Lt, S = _checked(F, (N, 3), dt, 'F'), _checked(Lt, (N, 3), dt, 'L'), _checked(S, (N, 5), dt, 'S')
        U, Om, E = self._like(pos, (N, 3), dt), self._like(pos, (N, 3), dt), self._like(pos, (N, 5), dt)
        st = self._lib.pse_mobility_apply11(self._h, _ptr(pos), _ptr(F), _ptr(Lt), _ptr(S), _ptr(U), _ptr(Om),
                                            _ptr(E), PARTS[parts], _stream(pos))
        self._check(st)
        return U, Om, E

    def _noise_points(self):
        """Half-spectrum points of all suspensions, sum of Ng^2 (Ng/2 + 1)."""
        ngs = [self.system_info(s)['Ng'] for s in range(self.nsys)]
        return int(sum(g * g * (g // 2 + 1) for g in ngs))

    def _check_step_args(self, pos, FP=None, w1=None, w2=None, wt=None):
        """Shapes and element types of the arrays a sample or step reads (positions FP64; forces and
        noise in the handle's precision): a wrong one would be read past its end."""
        _checked(pos, (self.N, 3), np.float64, 'pos')
        _checked(FP, (self.N, 3), self.dtype, 'FP')
        _checked_size(w1, 8 * self.N, self.dtype, 'w1')
        if w2 is not None:
            _checked_size(w2, 6 * self._noise_points(), self.dtype, 'w2')
        _checked(wt, (self.N, 3), self.dtype, 'wt')

    def brownian(self, pos, dt, seed=0, counter=0, w1=None, w2=None):
        """Brownian slip velocities (U^B, E^B) with covariance (2kT/dt) M."""
        self._check_step_args(pos, w1=w1, w2=w2)
        U = self._like(pos, (self.N, 3), self.dtype)
        E = self._like(pos, (self.N, 5), self.dtype)
        stats = Stats()
        st = self._lib.pse_brownian_sample(self._h, _ptr(pos), float(dt), int(seed), int(counter), _ptr(w1),
                                           _ptr(w2), _ptr(U), _ptr(E), ctypes.byref(stats), _stream(pos))
        if st not in (0, 4):
            self._check(st)
        return U, E, stats.as_dict()

    def step(self, pos, dt, FP=None, seed=0, step=0, w1=None, w2=None, want_S=False, allow_cap=True):
        """One constrained mid-point step; pos (N x 3 float64) is updated in place."""
        self._check_step_args(pos, FP, w1, w2)
        S = self._like(pos, (self.N, 5), self.dtype) if want_S else None
        stats = Stats()
        if w1 is not None or w2 is not None:
            st = self._lib.pse_constrained_step_noise(self._h, _ptr(pos), _ptr(FP), float(dt), _ptr(w1), _ptr(w2),
                                                      _ptr(S), ctypes.byref(stats), _stream(pos))
        else:
            st = self._lib.pse_constrained_step(self._h, _ptr(pos), _ptr(FP), float(dt), int(seed), int(step),
                                                _ptr(S), ctypes.byref(stats), _stream(pos))
        if not (st == 0 or (allow_cap and st == 4)):
            self._check(st)
        d = stats.as_dict()
        d['status'] = st
        return S, d

    def rfd_step(self, pos, dt, FP=None, delta=0.0, seed=0, step=0, w1=None, w2=None, wt=None, want_S=False,
                 allow_cap=True):
        """One Euler-Maruyama step with a random-finite-difference drift (three stresslet solves);
        pos is updated in place.  External noise needs w1, w2 and wt together."""
        self._check_step_args(pos, FP, w1, w2, wt)
        S = self._like(pos, (self.N, 5), self.dtype) if want_S else None
        stats = Stats()
        if w1 is not None or w2 is not None or wt is not None:
            st = self._lib.pse_rfd_step_noise(self._h, _ptr(pos), _ptr(FP), float(dt), float(delta), _ptr(w1),
                                              _ptr(w2), _ptr(wt), _ptr(S), ctypes.byref(stats), _stream(pos))
        else:
            st = self._lib.pse_rfd_step(self._h, _ptr(pos), _ptr(FP), float(dt), float(delta), int(seed), int(step),
                                        _ptr(S), ctypes.byref(stats), _stream(pos))
        if not (st == 0 or (allow_cap and st == 4)):
            self._check(st)
        d = stats.as_dict()
        d['status'] = st
        return S, d

    def overlap_force(self, pos, k):
        """Harmonic overlap repulsion k (2a - r) rh summed over pairs closer than contact."""
        _checked(pos, (self.N, 3), np.float64, 'pos')
        F = self._like(pos, (self.N, 3), self.dtype)
        self._check(self._lib.pse_overlap_force(self._h, _ptr(pos), float(k), _ptr(F), _stream(pos)))
        return F

    def autotune(self, pos, reps=3):
        """Times the pair-sum lanes and spreading-tile candidates on `pos` and keeps the fastest."""
        _checked(pos, (self.N, 3), np.float64, 'pos')
        t = Tuning()
        self._check(self._lib.pse_autotune(self._h, _ptr(pos), int(reps), ctypes.byref(t), _stream(pos)))
        self.info = self.get_info()
        lanes = [1, 4, 8, 16, 32][:t.n_lanes]
        return {'real_lanes': t.real_lanes, 'real_smem_table': t.real_smem_table, 'real_smem_ms': t.real_smem_ms,
                'tile': tuple(t.tile), 'best_real_ms': t.best_real_ms,
                'best_wave_ms': t.best_wave_ms, 'real_ms': dict(zip(lanes, list(t.real_ms)[:t.n_lanes])),
                'wave_ms': {tuple(t.tiles[k]): t.wave_ms[k] for k in range(t.n_tiles)}}

    def set_profiling(self, enable=True):
        self._check(self._lib.pse_set_profiling(self._h, 1 if enable else 0))

    def profile(self):
        """{'ms': {stage: ms}, 'calls': {stage: n}, 'launches': n, 'fft_execs': n,
        'variant_ms': {stage: {variant: ms}}, 'variant_calls': {stage: {variant: n}}} (variants:
        'full' [F; S] -> [U; E] and the noise interpolation, 'se' S -> E, 'fsu' [F; S] -> U, 'su' S -> U)."""
        pr = Profile()
        self._check(self._lib.pse_get_profile(self._h, ctypes.byref(pr)))
        return {'ms': {STAGES[i]: pr.ms[i] for i in range(NSTAGES)},
                'calls': {STAGES[i]: pr.calls[i] for i in range(NSTAGES)},
                'launches': pr.launches, 'fft_execs': pr.fft_execs,
                'variant_ms': {STAGES[i]: {VARIANTS[v]: pr.variant_ms[i][v] for v in range(NVARIANTS)}
                               for i in range(NSTAGES)},
                'variant_calls': {STAGES[i]: {VARIANTS[v]: pr.variant_calls[i][v] for v in range(NVARIANTS)}
                                  for i in range(NSTAGES)}}

    def sync(self):
        self._check(self._lib.pse_sync(self._h))


class Server:
    """Serving loop of the C ABI: `slots` concurrent workers (one CUDA stream each)
    under a device-memory budget; suspension state stays resident between
    requests with the same parameters.  Arrays are numpy (host) or torch tensors
    and must stay alive until the request completes (the Server keeps them)."""

    def __init__(self, slots=4, budget_bytes=64 << 30):
        self._lib = load()
        h = _P()
        st = self._lib.pse_server_create(ctypes.byref(h), int(slots), int(budget_bytes))
        if st != 0:
            raise PSEError(st, 'cannot create the server')
        self._h = h
        self._keep = {}

    def submit(self, kind, pos, L, a=1.0, eta=1.0, kT=1.0, xi=0.5, tol=1e-3, precision='mixed', F=None, S=None,
               dt=1e-3, seed=0, counter=0, **opts):
        """Queues a request; returns (ticket, outputs).  kind: 'mobility' (outputs U, E),
        'sample' (U^B, E^B), 'step' (pos updated in place; outputs S_out)."""
        prec = _precision(precision)
        dtype = np.float64 if prec == PSE_FP64 else np.float32
        N = pos.shape[0]
        _checked(pos, (N, 3), np.float64, 'pos')
        _checked(F, (N, 3), dtype, 'F')
        _checked(S, (N, 5), dtype, 'S')
        out = {}
        r = Request()
        r.kind = REQ_KINDS[kind]
        r.precision = prec
        r.N, r.L, r.a, r.eta, r.kT, r.xi, r.tol = int(N), float(L), float(a), float(eta), float(kT), float(xi), float(tol)
        o = _options(**opts) if opts else None
        if o is not None:
            r.options = ctypes.pointer(o)
        r.pos = _ptr(pos)
        r.dt, r.seed, r.counter = float(dt), int(seed), int(counter)
        stats = Stats()
        r.stats = ctypes.pointer(stats)

        def like(shape):
            if isinstance(pos, np.ndarray):
                return np.zeros(shape, dtype=dtype)
            torch = _torch()
            return torch.zeros(shape, dtype=torch.float64 if dtype == np.float64 else torch.float32,
                               device=pos.device)
        if kind in ('mobility', 'sample'):
            out['U'], out['E'] = like((N, 3)), like((N, 5))
            r.U, r.E = _ptr(out['U']), _ptr(out['E'])
            if kind == 'mobility':
                r.F, r.S = _ptr(F), _ptr(S)
        else:
            r.F = _ptr(F)
            out['S'] = like((N, 5))
            r.S_out = _ptr(out['S'])
        t = ctypes.c_uint64(0)
        st = self._lib.pse_server_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        if st != 0:
            raise PSEError(st, 'request rejected')
        out['stats'] = stats
        self._keep[t.value] = (r, o, stats, pos, F, S, out)
        return t.value, out

    def wait(self, ticket, timeout_ms=600000.0):
        """(status, latency_ms) of a request; raises TimeoutError if it has not completed in time."""
        res = ctypes.c_int(0)
        lat = ctypes.c_double(0)
        st = self._lib.pse_server_wait(self._h, int(ticket), float(timeout_ms), ctypes.byref(res), ctypes.byref(lat))
        if st == 6:
            raise TimeoutError('request %d still running' % ticket)
        if st != 0:
            raise PSEError(st, 'unknown ticket')
        self._keep.pop(ticket, None)
        return res.value, lat.value

    def stats(self):
        s = ServerStats()
        self._lib.pse_server_get_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    def reset_stats(self):
        self._lib.pse_server_reset_stats(self._h)

    def set_deformation(self, A, stream=None):
        """Lattice deformation A (3 x 3; the cell is spanned by the columns of L A) for
        the following calls; the handle must have been created with deform=..."""
        Am = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        st = self._lib.pse_set_deformation(self._h, Am.ctypes.data, stream)
        self._check(st)
        self.info = self.get_info()

    def close(self):
        if getattr(self, '_h', None):
            self._lib.pse_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
