"""ctypes binding of libnfft_gb300.so: the C ABI of include/nfft_gb300.h under
the same names, argument marshalling only.

Every function takes plain integers (pointers as ints) and returns the C
status code; ``check`` turns a non-zero status into ``NFFTError``.  Loading
fails loudly if the library has not been built: there is no fallback path.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libnfft_gb300.so")

NFFT_OK = 0
NFFT_ERR_INVALID_ARG = -1
NFFT_ERR_NO_NODES = -2
NFFT_ERR_OOM = -3
NFFT_ERR_CUFFT = -4
NFFT_ERR_CUDA = -5
NFFT_ERR_TIMEOUT = -6
NFFT_ERR_DEVICE_CHECK = -7
NFFT_ERR_UNSUPPORTED = -8

NFFT_C64 = 0
NFFT_C128 = 1
NFFT_FLAG_CLOSED_SUPPORT = 0x1
NFFT_FLAG_COMPENSATED = 0x2
NFFT_FLAG_FULL_MATRIX = 0x4
NFFT_FLAG_WIDE_WINDOW = 0x8
NFFT_FLAG_LIBRARY_FFT = 0x10
NFFT_FLAG_WINDOW_DIRECT = 0x20
NFFT_FLAG_WINDOW_LINEAR = 0x40
NFFT_FLAG_WINDOW_POLYNOMIAL = 0x80

_p = ctypes.c_void_p
_i = ctypes.c_int
_i64p = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes), in header order
SIGNATURES = {
    "nfft_plan_create": (_i, [ctypes.POINTER(_p), _i, _i64p, ctypes.c_int64, ctypes.c_double, _i, _i,
                              ctypes.c_uint32, _p]),
    "nfft_plan_destroy": (_i, [_p]),
    "nfft_set_nodes": (_i, [_p, _p, _i]),
    "nfft_forward": (_i, [_p, _p, _p]),
    "nfft_adjoint": (_i, [_p, _p, _p]),
    "nfft_grad": (_i, [_p, _p, _p, _p]),
    "nfft_plan_sync": (_i, [_p]),
    "nfft_strerror": (ctypes.c_char_p, [_i]),
    "nfft_plan_info": (_i, [_p, _i64p, _i64p, _i64p]),
    "nfft_plan_grid": (_p, [_p]),
    "nfft_plan_set_tile": (_i, [_p, _i64p]),
    "nfft_step_deconv_pad": (_i, [_p, _p]),
    "nfft_step_fft": (_i, [_p, _i]),
    "nfft_step_gather": (_i, [_p, _p]),
    "nfft_step_scatter": (_i, [_p, _p]),
    "nfft_step_crop_deconv": (_i, [_p, _p]),
    "nfft_step_pad_fft": (_i, [_p, _p]),
    "nfft_step_fft_crop": (_i, [_p, _p]),
    "nfft_plan_set_graph": (_i, [_p, _i]),
    "nfft_plan_set_async": (_i, [_p, _i]),
    "nfft_plan_paths": (_i, [_p, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "nfft_step_grad_gather": (_i, [_p, _p, _p]),
    "nfft_plan_autotune": (_i, [_p, _p, _i, _i64p]),
    "nfft_batch_create": (_i, [ctypes.POINTER(_p), _i, _i, _i64p, ctypes.POINTER(ctypes.c_int32), _i, _i64p,
                               ctypes.c_double, _i, _i, ctypes.c_uint32, _p]),
    "nfft_batch_destroy": (_i, [_p]),
    "nfft_batch_set_nodes": (_i, [_p, _p, _i]),
    "nfft_batch_forward": (_i, [_p, _p, _p]),
    "nfft_batch_adjoint": (_i, [_p, _p, _p]),
    "nfft_batch_set_graph": (_i, [_p, _i]),
    "nfft_batch_set_tile": (_i, [_p, _i64p]),
    "nfft_batch_info": (_i, [_p, _i64p, _i64p, _i64p]),
    "nfft_batch_autotune": (_i, [_p, _p, _i, _i64p]),
    "nfft_spread_noalloc": (_i, [_i, _i64p, ctypes.c_double, _i, ctypes.c_int64, _p, _p, _p, _p]),
}

NFFT_NOALLOC_MAX_NODES = 262144
NFFT_NOALLOC_MAX_TILES = 65536

_lib = None


class NFFTError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where or "nfft", strerror(code), code))


def lib():
    """Load the library once; raise if it is missing (no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libnfft_gb300.so is not built (expected at %s); run "
                "paper_2208_00049_gb300.build.build() first" % LIB_PATH)
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def strerror(code):
    return lib().nfft_strerror(int(code)).decode()


def check(code, where=""):
    if code != NFFT_OK:
        raise NFFTError(code, where)
    return code


def _i64_array(vals, n=3):
    arr = (ctypes.c_int64 * n)()
    for i, v in enumerate(vals):
        arr[i] = int(v)
    return arr


def nfft_plan_create(D, N, M, sigma, m, dtype, flags, stream):
    """Returns (status, plan handle as int or None)."""
    out = _p()
    Narr = _i64_array(N, max(3, len(N)))
    s = lib().nfft_plan_create(ctypes.byref(out), int(D), Narr, int(M), float(sigma), int(m),
                               int(dtype), int(flags), _p(stream or None))
    return s, out.value


def nfft_plan_destroy(plan):
    return lib().nfft_plan_destroy(_p(plan))


def nfft_set_nodes(plan, k_ptr, k_is_fp64):
    return lib().nfft_set_nodes(_p(plan), _p(k_ptr), int(k_is_fp64))


def nfft_forward(plan, f_ptr, fhat_ptr):
    return lib().nfft_forward(_p(plan), _p(f_ptr), _p(fhat_ptr))


def nfft_adjoint(plan, fhat_ptr, y_ptr):
    return lib().nfft_adjoint(_p(plan), _p(fhat_ptr), _p(y_ptr))


def nfft_grad(plan, f_ptr, cot_ptr, gk_ptr):
    return lib().nfft_grad(_p(plan), _p(f_ptr), _p(cot_ptr), _p(gk_ptr))


def nfft_plan_sync(plan):
    return lib().nfft_plan_sync(_p(plan))


def nfft_strerror(code):
    return strerror(code)


def nfft_plan_info(plan):
    """Returns (status, Ntilde3, tile3, n_items)."""
    nt = (ctypes.c_int64 * 3)()
    tl = (ctypes.c_int64 * 3)()
    ni = ctypes.c_int64()
    s = lib().nfft_plan_info(_p(plan), nt, tl, ctypes.byref(ni))
    return s, tuple(nt), tuple(tl), ni.value


def nfft_plan_grid(plan):
    return lib().nfft_plan_grid(_p(plan))


def nfft_plan_set_tile(plan, tile3):
    return lib().nfft_plan_set_tile(_p(plan), _i64_array(list(tile3) + [1] * (3 - len(tile3))))


def nfft_step_deconv_pad(plan, f_ptr):
    return lib().nfft_step_deconv_pad(_p(plan), _p(f_ptr))


def nfft_step_fft(plan, sign):
    return lib().nfft_step_fft(_p(plan), int(sign))


def nfft_step_gather(plan, fhat_ptr):
    return lib().nfft_step_gather(_p(plan), _p(fhat_ptr))


def nfft_step_scatter(plan, fhat_ptr):
    return lib().nfft_step_scatter(_p(plan), _p(fhat_ptr))


def nfft_step_crop_deconv(plan, y_ptr):
    return lib().nfft_step_crop_deconv(_p(plan), _p(y_ptr))


def nfft_step_pad_fft(plan, f_ptr):
    return lib().nfft_step_pad_fft(_p(plan), _p(f_ptr))


def nfft_step_fft_crop(plan, y_ptr):
    return lib().nfft_step_fft_crop(_p(plan), _p(y_ptr))


def nfft_plan_set_graph(plan, enable):
    return lib().nfft_plan_set_graph(_p(plan), int(bool(enable)))


def nfft_plan_set_async(plan, enable):
    return lib().nfft_plan_set_async(_p(plan), int(bool(enable)))


def nfft_plan_paths(plan):
    """Returns (status, fast_gather, fast_scatter, fft_form) with fft_form 0 =
    library FFT + separate correction, 1 = pruned 3D FFT, 2 = direct sums."""
    a = _i()
    b = _i()
    s = lib().nfft_plan_paths(_p(plan), ctypes.byref(a), ctypes.byref(b))
    return s, bool(a.value & 1), bool(a.value & 2), int(b.value)


def nfft_step_grad_gather(plan, cot_ptr, gk_ptr):
    return lib().nfft_step_grad_gather(_p(plan), _p(cot_ptr), _p(gk_ptr))


def nfft_plan_autotune(plan, k_ptr, k_is_fp64):
    """Returns (status, chosen tile3)."""
    t = (ctypes.c_int64 * 3)()
    s = lib().nfft_plan_autotune(_p(plan), _p(k_ptr), int(k_is_fp64), t)
    return s, tuple(t)


def nfft_batch_create(D, N_flat, set_of, M_set, sigma, m, dtype, flags, stream):
    """Returns (status, batch handle or None)."""
    out = _p()
    B = len(set_of)
    Narr = _i64_array(N_flat, len(N_flat))
    sarr = (ctypes.c_int32 * B)(*[int(v) for v in set_of])
    Marr = _i64_array(M_set, len(M_set))
    s = lib().nfft_batch_create(ctypes.byref(out), int(D), B, Narr, sarr, len(M_set), Marr, float(sigma),
                                int(m), int(dtype), int(flags), _p(stream or None))
    return s, out.value


def nfft_batch_destroy(batch):
    return lib().nfft_batch_destroy(_p(batch))


def nfft_batch_set_nodes(batch, k_ptr, k_is_fp64):
    return lib().nfft_batch_set_nodes(_p(batch), _p(k_ptr), int(k_is_fp64))


def nfft_batch_forward(batch, f_ptr, fhat_ptr):
    return lib().nfft_batch_forward(_p(batch), _p(f_ptr), _p(fhat_ptr))


def nfft_batch_adjoint(batch, fhat_ptr, y_ptr):
    return lib().nfft_batch_adjoint(_p(batch), _p(fhat_ptr), _p(y_ptr))


def nfft_batch_set_graph(batch, enable):
    return lib().nfft_batch_set_graph(_p(batch), int(enable))


def nfft_batch_set_tile(batch, tile3):
    return lib().nfft_batch_set_tile(_p(batch), _i64_array(list(tile3) + [1] * (3 - len(tile3))))


def nfft_batch_info(batch):
    """Returns (status, tile3, n_items, n_fft_classes)."""
    t = (ctypes.c_int64 * 3)()
    ni = ctypes.c_int64()
    nc = ctypes.c_int64()
    s = lib().nfft_batch_info(_p(batch), t, ctypes.byref(ni), ctypes.byref(nc))
    return s, tuple(t), ni.value, nc.value


def nfft_batch_autotune(batch, k_ptr, k_is_fp64):
    """Returns (status, chosen tile3)."""
    t = (ctypes.c_int64 * 3)()
    s = lib().nfft_batch_autotune(_p(batch), _p(k_ptr), int(k_is_fp64), t)
    return s, tuple(t)


def nfft_spread_noalloc(D, N, sigma, m, M, k_ptr, fhat_ptr, grid_ptr, stream):
    """Adjoint resampling onto a caller grid with no device allocation (see the header)."""
    return lib().nfft_spread_noalloc(int(D), _i64_array(N, max(3, len(N))), float(sigma), int(m),
                                     int(M), _p(k_ptr), _p(fhat_ptr), _p(grid_ptr), _p(stream or None))
