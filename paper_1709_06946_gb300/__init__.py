"""GB300-native positively-split Ewald (PSE) mobility with stresslet constraints.

The compute path is the CUDA library ``libpse.so`` (sm_103a kernels + cuFFT)
behind the C ABI in ``include/pse.h``; this package only builds it and binds it.
"""
from .binding import PSE, PSEError, Server, estimate_bytes, load, LIB_PATH, PSE_MIXED, PSE_FP64  # noqa: F401


def build(verbose=False, force=False):
    from .builder import build as _build
    return _build(verbose=verbose, force=force)
