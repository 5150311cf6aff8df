"""ctypes binding of the C ABI in ``include/celes.h`` (argument marshalling only).

Every entry point of the C library has a Python function of the same name
here.  Host arrays are NumPy arrays; device buffers for the matvec / apply
calls are any objects exposing ``data_ptr()`` (torch CUDA tensors) or raw
integer device addresses.  No arithmetic on problem data happens in Python:
if the shared library is missing this module raises instead of falling back.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libceles_gb300.so")

CELES_OK = 0
CELES_EINVAL = -1
CELES_ENOMEM = -2
CELES_ECUDA = -3
CELES_ENOCONV = -4
CELES_ENUMERIC = -5
CELES_EOVERLAP = -6
CELES_ETIMEOUT = -7
CELES_ESTATE = -8
CELES_ETOOBIG = -9
STATUS_NAMES = {0: "CELES_OK", -1: "CELES_EINVAL", -2: "CELES_ENOMEM", -3: "CELES_ECUDA", -4: "CELES_ENOCONV",
                -5: "CELES_ENUMERIC", -6: "CELES_EOVERLAP", -7: "CELES_ETIMEOUT", -8: "CELES_ESTATE",
                -9: "CELES_ETOOBIG"}

CELES_FP64 = 0
CELES_FP32 = 1
CELES_PLANE_WAVE = 0
CELES_GAUSSIAN_BEAM = 1
CELES_SOLVE_FP64 = 0
CELES_SOLVE_MIXED = 1
CELES_X0_TA = 0
CELES_X0_USER = 1
CELES_X0_ZERO = 2
CELES_X0_LEARNED = 3
CELES_SOLVER_GMRES = 0
CELES_SOLVER_BICGSTAB = 1


CELES_KERNEL_AUTO = 0
CELES_KERNEL_DIRECT = 1
CELES_KERNEL_RTR = 2


class celes_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("check_overlap", ctypes.c_int), ("chunks", ctypes.c_int),
                ("kernel", ctypes.c_int), ("autotune", ctypes.c_int), ("variant", ctypes.c_int)]


class celes_incident(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("beta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("pol", ctypes.c_int), ("E0_re", ctypes.c_double), ("E0_im", ctypes.c_double),
                ("waist", ctypes.c_double), ("focus", ctypes.c_double * 3), ("alpha_G", ctypes.c_double),
                ("n_beta", ctypes.c_int)]


class celes_solve_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("x0", ctypes.c_int), ("use_precond", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("solver", ctypes.c_int)]


class celes_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer", ctypes.c_int),
                ("matvecs_fp64", ctypes.c_int), ("matvecs_fp32", ctypes.c_int), ("residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int), ("history_len", ctypes.c_int), ("guess_used", ctypes.c_int)]


_c_ctx_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

# (name, restype, argtypes) of every exported symbol of include/celes.h
SIGNATURES = [
    ("celes_coupling_shape", ctypes.c_int, [_c_ctx_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    ("celes_precond_stats", ctypes.c_int, [_c_ctx_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]),
    ("celes_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("celes_create", ctypes.c_int, [ctypes.POINTER(_c_ctx_p), ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.POINTER(celes_options)]),
    ("celes_set_incident", ctypes.c_int, [_c_ctx_p, ctypes.POINTER(celes_incident), ctypes.c_int]),
    ("celes_coupling_matvec", ctypes.c_int, [_c_ctx_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_void_p]),
    ("celes_master_matvec", ctypes.c_int, [_c_ctx_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_void_p]),
    ("celes_precond_build", ctypes.c_int, [_c_ctx_p, ctypes.c_double]),
    ("celes_precond_apply", ctypes.c_int, [_c_ctx_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_void_p]),
    ("celes_set_initial_guess", ctypes.c_int, [_c_ctx_p, _dp]),
    ("celes_solve", ctypes.c_int, [_c_ctx_p, ctypes.c_double, ctypes.POINTER(celes_solve_opts),
                                   ctypes.POINTER(celes_solve_info)]),
    ("celes_get_coefficients", ctypes.c_int, [_c_ctx_p, _dp]),
    ("celes_get_incident_coefficients", ctypes.c_int, [_c_ctx_p, _dp]),
    ("celes_get_tmatrix", ctypes.c_int, [_c_ctx_p, _dp]),
    ("celes_farfield", ctypes.c_int, [_c_ctx_p, _dp, ctypes.c_int64, _dp, ctypes.c_int]),
    ("celes_num_spheres", ctypes.c_int64, [_c_ctx_p]),
    ("celes_nmax", ctypes.c_int, [_c_ctx_p]),
    ("celes_num_rhs", ctypes.c_int, [_c_ctx_p]),
    ("celes_coupling_terms", ctypes.c_int, [ctypes.c_int, _ip, _dp, ctypes.c_int]),
    ("celes_profile", ctypes.c_int, [_c_ctx_p, ctypes.c_int]),
    ("celes_kernel_time", ctypes.c_int, [_c_ctx_p, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64)]),
    ("celes_kernel_launches", ctypes.c_int64, []),
    ("celes_flops_per_pair", ctypes.c_double, [ctypes.c_int, ctypes.c_int]),
    ("celes_coupling_matvec_noalloc", ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_int, ctypes.c_void_p]),
    ("celes_gemm_bf16", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_void_p]),
    ("celes_gnn_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_uint64, ctypes.c_int]),
    ("celes_gnn_train", ctypes.c_int, [ctypes.c_void_p, _c_ctx_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]),
    ("celes_gnn_predict", ctypes.c_int, [ctypes.c_void_p, _c_ctx_p]),
    ("celes_gnn_add_example", ctypes.c_int, [ctypes.c_void_p, _c_ctx_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("celes_gnn_train_example", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]),
    ("celes_gnn_num_examples", ctypes.c_int, [ctypes.c_void_p]),
    ("celes_gnn_clear_examples", ctypes.c_int, [ctypes.c_void_p]),
    ("celes_gnn_num_params", ctypes.c_int, [ctypes.c_void_p]),
    ("celes_gnn_export", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                        ctypes.c_int]),
    ("celes_gnn_destroy", None, [ctypes.c_void_p]),
    ("celes_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_c_ctx_p), ctypes.c_int,
                                          ctypes.c_int]),
    ("celes_batch_num_systems", ctypes.c_int, [ctypes.c_void_p]),
    ("celes_batch_num_unknowns", ctypes.c_longlong, [ctypes.c_void_p]),
    ("celes_batch_master_matvec", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("celes_batch_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(celes_solve_opts),
                                         ctypes.POINTER(celes_solve_info)]),
    ("celes_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("celes_batch_destroy", None, [ctypes.c_void_p]),
    ("celes_s11", ctypes.c_int, [_c_ctx_p, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp]),
    ("celes_power", ctypes.c_int, [_c_ctx_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]),
    ("celes_nearfield", ctypes.c_int, [_c_ctx_p, _dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp]),
    ("celes_destroy", None, [_c_ctx_p]),
    ("celes_last_error", ctypes.c_char_p, [_c_ctx_p]),
    ("celes_version", ctypes.c_char_p, []),
]

_lib = None


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class CelesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code, ctx=None):
    if code != CELES_OK:
        msg = ""
        if ctx is not None:
            m = load().celes_last_error(ctx)
            msg = m.decode() if m else ""
        raise CelesError(code, msg)
    return code


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _devptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _check_vec(name, t, n_complex, precision, device=None):
    """Check a device coefficient buffer before its pointer crosses the C ABI,
    which cannot see sizes: a contiguous CUDA tensor of at least n_complex
    entries of the dtype that `precision` names (complex128 for FP64,
    complex64 for FP32), on `device` when given.  Raw integer pointers are
    passed through unchecked."""
    if t is None or isinstance(t, int):
        return
    want = "complex128" if precision == CELES_FP64 else "complex64"
    dt = str(t.dtype).replace("torch.", "")
    if dt != want:
        raise CelesError(CELES_EINVAL, f"{name}: dtype {dt}, expected {want} for this precision")
    if not t.is_cuda:
        raise CelesError(CELES_EINVAL, f"{name}: not a CUDA tensor")
    if device is not None and t.device.index != device:
        raise CelesError(CELES_EINVAL, f"{name}: on cuda:{t.device.index}, expected cuda:{device}")
    if not t.is_contiguous():
        raise CelesError(CELES_EINVAL, f"{name}: not contiguous")
    if t.numel() < n_complex:
        raise CelesError(CELES_EINVAL, f"{name}: {t.numel()} entries, needs {n_complex}")


def _ctx_vec_checks(ctx, x, y, nrhs, precision):
    n = int(load().celes_num_spheres(ctx)) * int(load().celes_nmax(ctx)) * int(nrhs)
    dev = None
    for name, t in (("x", x), ("y", y)):
        _check_vec(name, t, n, precision)
        if t is not None and not isinstance(t, int):
            if dev is None:
                dev = t.device.index
            elif t.device.index != dev:
                raise CelesError(CELES_EINVAL, "x and y are on different devices")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# one Python function per C entry point
# ---------------------------------------------------------------------------

def celes_create(positions, radii, n_i, n0, k0, lmax, device=0, check_overlap=True, chunks=0,
                 kernel=CELES_KERNEL_AUTO, autotune=True, variant=-1):
    pos = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1, 3)
    rad = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    ni = np.ascontiguousarray(np.asarray(n_i, dtype=np.complex128).reshape(-1)).view(np.float64)
    opt = celes_options(int(device), int(bool(check_overlap)), int(chunks), int(kernel), int(bool(autotune)),
                        int(variant))
    ctx = _c_ctx_p()
    code = load().celes_create(ctypes.byref(ctx), pos.shape[0], _dptr(pos), _dptr(rad), _dptr(ni),
                               float(n0), float(k0), int(lmax), ctypes.byref(opt))
    if code != CELES_OK:
        raise CelesError(code, "celes_create failed")
    return ctx


def make_incident(kind="plane", beta=0.0, alpha=0.0, pol=2, E0=1.0, waist=0.0, focus=(0.0, 0.0, 0.0),
                  alpha_G=-np.pi / 2, n_beta=0):
    d = celes_incident()
    d.kind = CELES_PLANE_WAVE if kind == "plane" else CELES_GAUSSIAN_BEAM
    d.beta, d.alpha, d.pol = float(beta), float(alpha), int(pol)
    d.E0_re, d.E0_im = float(np.real(E0)), float(np.imag(E0))
    d.waist = float(waist)
    for q in range(3):
        d.focus[q] = float(focus[q])
    d.alpha_G = float(alpha_G)
    d.n_beta = int(n_beta)
    return d


def celes_set_incident(ctx, incidents):
    arr = (celes_incident * len(incidents))(*incidents)
    return _check(load().celes_set_incident(ctx, arr, len(incidents)), ctx)


def celes_coupling_matvec(ctx, x, y, nrhs=1, precision=CELES_FP64, stream=None):
    _ctx_vec_checks(ctx, x, y, nrhs, precision)
    return _check(load().celes_coupling_matvec(ctx, _devptr(x), _devptr(y), int(nrhs), int(precision),
                                               _stream(stream)), ctx)


def celes_master_matvec(ctx, x, y, nrhs=1, precision=CELES_FP64, stream=None):
    _ctx_vec_checks(ctx, x, y, nrhs, precision)
    return _check(load().celes_master_matvec(ctx, _devptr(x), _devptr(y), int(nrhs), int(precision),
                                             _stream(stream)), ctx)


def celes_precond_build(ctx, cuboid_edge):
    return _check(load().celes_precond_build(ctx, float(cuboid_edge)), ctx)


def celes_precond_apply(ctx, x, y, nrhs=1, precision=CELES_FP64, stream=None):
    _ctx_vec_checks(ctx, x, y, nrhs, precision)
    return _check(load().celes_precond_apply(ctx, _devptr(x), _devptr(y), int(nrhs), int(precision),
                                             _stream(stream)), ctx)


def celes_coupling_shape(ctx, precision):
    """(variant, chunks, tuned ms) of the context's coupling kernel in `precision`."""
    v, ch, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().celes_coupling_shape(ctx, int(precision), ctypes.byref(v), ctypes.byref(ch), ctypes.byref(ms)), ctx)
    return v.value, ch.value, ms.value


def celes_precond_stats(ctx):
    """(blocks, largest block dimension, complex entries of all factors) of the built preconditioner."""
    a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().celes_precond_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), ctx)
    return a.value, b.value, c.value


def celes_set_initial_guess(ctx, b0):
    b = np.ascontiguousarray(b0, dtype=np.complex128)
    return _check(load().celes_set_initial_guess(ctx, _dptr(b.view(np.float64))), ctx)


def celes_solve(ctx, tol, mode=CELES_SOLVE_MIXED, restart=100, max_iter=2000, max_outer=20, x0=CELES_X0_TA,
                use_precond=True, inner_tol=1e-5, history_cap=4096, raise_on_noconv=True, solver=0):
    """Returns a dict with the solve statistics and the residual history.
    solver: CELES_SOLVER_GMRES (0) or CELES_SOLVER_BICGSTAB (1)."""
    opts = celes_solve_opts(int(mode), int(restart), int(max_iter), int(max_outer), int(x0), int(bool(use_precond)),
                            float(inner_tol), int(solver))
    hist = np.zeros(max(1, history_cap), dtype=np.float64)
    info = celes_solve_info()
    info.history = _dptr(hist)
    info.history_cap = int(history_cap)
    code = load().celes_solve(ctx, float(tol), ctypes.byref(opts), ctypes.byref(info))
    out = {"status": int(code), "iterations": info.iterations, "outer": info.outer,
           "matvecs_fp64": info.matvecs_fp64, "matvecs_fp32": info.matvecs_fp32, "residual": info.residual,
           "seconds": info.seconds, "history": hist[:info.history_len].copy(), "guess_used": info.guess_used}
    if code != CELES_OK and not (code == CELES_ENOCONV and not raise_on_noconv):
        _check(code, ctx)
    return out


def _host_vec(ctx, getter, shape):
    out = np.zeros(shape, dtype=np.complex128)
    _check(getter(ctx, _dptr(out.view(np.float64))), ctx)
    return out


def celes_get_coefficients(ctx):
    lib = load()
    return _host_vec(ctx, lib.celes_get_coefficients,
                     (lib.celes_num_rhs(ctx), lib.celes_num_spheres(ctx), lib.celes_nmax(ctx)))


def celes_get_incident_coefficients(ctx):
    lib = load()
    return _host_vec(ctx, lib.celes_get_incident_coefficients,
                     (lib.celes_num_rhs(ctx), lib.celes_num_spheres(ctx), lib.celes_nmax(ctx)))


def celes_get_tmatrix(ctx):
    lib = load()
    return _host_vec(ctx, lib.celes_get_tmatrix, (lib.celes_num_spheres(ctx), lib.celes_nmax(ctx)))


def celes_farfield(ctx, dirs, rhs=0):
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 2)
    g = np.zeros((d.shape[0], 2), dtype=np.complex128)
    _check(load().celes_farfield(ctx, _dptr(d), d.shape[0], _dptr(g.view(np.float64)), int(rhs)), ctx)
    return g


def celes_num_spheres(ctx):
    return int(load().celes_num_spheres(ctx))


def celes_nmax(ctx):
    return int(load().celes_nmax(ctx))


def celes_num_rhs(ctx):
    return int(load().celes_num_rhs(ctx))


def celes_coupling_terms(lmax):
    """(idx (T, 5) int32 = (source row, receiving row, p, mu, kind), val (T,)) of the built-in table."""
    lib = load()
    n = lib.celes_coupling_terms(int(lmax), None, None, 0)
    if n < 0:
        raise CelesError(n, "celes_coupling_terms")
    idx = np.zeros((n, 5), dtype=np.int32)
    val = np.zeros(n, dtype=np.float64)
    lib.celes_coupling_terms(int(lmax), idx.ctypes.data_as(_ip), _dptr(val), n)
    return idx, val


def celes_profile(ctx, on):
    return _check(load().celes_profile(ctx, int(bool(on))), ctx)


KERNEL_FP32_COUPLING = 0
KERNEL_FP64_COUPLING = 1
KERNEL_EPILOGUE = 2


def celes_kernel_time(ctx, which):
    """(total milliseconds, launches) recorded since celes_profile(ctx, 1)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().celes_kernel_time(ctx, int(which), ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def celes_kernel_launches():
    return int(load().celes_kernel_launches())


def celes_flops_per_pair(lmax, kernel=CELES_KERNEL_AUTO):
    return float(load().celes_flops_per_pair(int(lmax), int(kernel)))


FMA_FP64 = 0
FMA_FP32 = 1
FMA_FP32_PACKED = 2


def celes_fma_peak(kind):
    """Measured FMA issue peak of the current device: (TFLOP/s, ms of the timed launch)."""
    tf = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    code = load().celes_fma_peak(int(kind), ctypes.byref(tf), ctypes.byref(ms))
    if code != CELES_OK:
        raise CelesError(code, "celes_fma_peak")
    return tf.value, ms.value


def celes_coupling_matvec_noalloc(N, lmax, k, positions4, x, y, precision=CELES_FP64, stream=None,
                                  check=True):
    """y = W x without any device allocation by the library (see include/celes.h).
    positions4, x, y: device buffers ([N][4] float64, [N][nmax] complex).
    Tensors are checked for dtype, size, contiguity and device first (with
    check=False as well: a mismatch there is an out-of-bounds access)."""
    nmax = 2 * int(lmax) * (int(lmax) + 2)
    if int(N) >= 1 and 1 <= int(lmax) <= 5:
        _check_vec("x", x, int(N) * nmax, precision)
        _check_vec("y", y, int(N) * nmax, precision)
        if positions4 is not None and not isinstance(positions4, int):
            if str(positions4.dtype) != "torch.float64" or not positions4.is_cuda or not positions4.is_contiguous() \
                    or positions4.numel() < 4 * int(N):
                raise CelesError(CELES_EINVAL, "positions4: needs a contiguous CUDA float64 tensor of N x 4")
        devs = {t.device.index for t in (x, y, positions4) if t is not None and not isinstance(t, int)}
        if len(devs) > 1:
            raise CelesError(CELES_EINVAL, "positions4, x and y must be on one device")
    code = load().celes_coupling_matvec_noalloc(int(N), int(lmax), float(k), _devptr(positions4), _devptr(x),
                                                 _devptr(y), int(precision), _stream(stream))
    if check and code != CELES_OK:
        raise CelesError(code, "celes_coupling_matvec_noalloc")
    return code


def celes_gemm_bf16(A, B, C, alpha=1.0, beta=0.0, stream=None):
    """C = alpha A B^T + beta C on the tensor cores; A (M, K), B (N, K) bf16 CUDA tensors, C (M, N) float32."""
    M, K = A.shape
    N = B.shape[0]
    code = load().celes_gemm_bf16(M, N, K, _devptr(A), A.stride(0), _devptr(B), B.stride(0), _devptr(C),
                                  C.stride(0), float(alpha), float(beta), _stream(stream))
    if code != CELES_OK:
        raise CelesError(code, "celes_gemm_bf16")
    return C


def celes_gnn_create(lmax, width=128, layers=3, knn=16, seed=0, device=0):
    g = ctypes.c_void_p()
    code = load().celes_gnn_create(ctypes.byref(g), int(lmax), int(width), int(layers), int(knn), int(seed),
                                   int(device))
    if code != CELES_OK:
        raise CelesError(code, "celes_gnn_create")
    return g


def celes_gnn_train(g, ctx, rhs=0, steps=1, lr=1e-3):
    loss = ctypes.c_double(0.0)
    code = load().celes_gnn_train(g, ctx, int(rhs), int(steps), float(lr), ctypes.byref(loss))
    if code != CELES_OK:
        raise CelesError(code, "celes_gnn_train")
    return loss.value


def celes_gnn_add_example(g, ctx, rhs=0):
    """Store a solved context's training example in the network; returns its index."""
    idx = ctypes.c_int(-1)
    code = load().celes_gnn_add_example(g, ctx, int(rhs), ctypes.byref(idx))
    if code != CELES_OK:
        raise CelesError(code, "celes_gnn_add_example")
    return idx.value


def celes_gnn_train_example(g, idx, steps=1, lr=1e-3):
    """Adam steps on stored example idx; returns the last loss."""
    loss = np.zeros(1)
    code = load().celes_gnn_train_example(g, int(idx), int(steps), float(lr), _dptr(loss))
    if code != CELES_OK:
        raise CelesError(code, "celes_gnn_train_example")
    return float(loss[0])


def celes_gnn_num_examples(g):
    return int(load().celes_gnn_num_examples(g))


def celes_gnn_clear_examples(g):
    code = load().celes_gnn_clear_examples(g)
    if code != CELES_OK:
        raise CelesError(code, "celes_gnn_clear_examples")


def celes_gnn_predict(g, ctx):
    return _check(load().celes_gnn_predict(g, ctx), ctx)


def celes_gnn_num_params(g):
    return int(load().celes_gnn_num_params(g))


def celes_gnn_export(g, what=0):
    lib = load()
    n = lib.celes_gnn_export(g, int(what), None, 0)
    if n < 0:
        raise CelesError(n, "celes_gnn_export")
    out = np.zeros(n, dtype=np.float32)
    code = lib.celes_gnn_export(g, int(what), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n)
    if code < 0:
        raise CelesError(code, "celes_gnn_export")
    return out


def celes_gnn_destroy(g):
    if g:
        load().celes_gnn_destroy(g)


def celes_nearfield(ctx, points, rhs=0, what=2):
    """E at points [Np][3]: what 0 scattered, 1 incident, 2 total; returns complex128 [Np][3]."""
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    E = np.zeros((p.shape[0], 3), dtype=np.complex128)
    _check(load().celes_nearfield(ctx, _dptr(p), p.shape[0], int(rhs), int(what), _dptr(E.view(np.float64))), ctx)
    return E


def celes_s11(ctx, betas, rhs_a=0, rhs_b=1, n_alpha=64):
    """Unnormalised S11 at polar angles betas (TE/TM average of the azimuthally averaged far-field intensity)."""
    b = np.ascontiguousarray(betas, dtype=np.float64).ravel()
    out = np.zeros(b.size)
    _check(load().celes_s11(ctx, int(rhs_a), int(rhs_b), _dptr(b), b.size, int(n_alpha), _dptr(out)), ctx)
    return out


def celes_power(ctx, rhs=0, n_beta=128, n_alpha=128):
    """(R, T): reflected and transmitted power fractions of a Gaussian-beam RHS."""
    R, T = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().celes_power(ctx, int(rhs), int(n_beta), int(n_alpha), ctypes.byref(R), ctypes.byref(T)), ctx)
    return R.value, T.value


def celes_batch_create(ctxs, restart=30):
    """Batch of contexts (see include/celes.h): one lockstep solve for every RHS of every context."""
    arr = (_c_ctx_p * len(ctxs))(*ctxs)
    b = ctypes.c_void_p()
    code = load().celes_batch_create(ctypes.byref(b), arr, len(ctxs), int(restart))
    if code != CELES_OK:
        raise CelesError(code, "celes_batch_create")
    return b


def celes_batch_num_systems(b):
    return int(load().celes_batch_num_systems(b))


def celes_batch_num_unknowns(b):
    return int(load().celes_batch_num_unknowns(b))


def celes_batch_master_matvec(b, x, y, precision=CELES_FP64):
    """y = (I - T W) x for every system; x, y flat device tensors of celes_batch_num_unknowns complex entries."""
    code = load().celes_batch_master_matvec(b, _devptr(x), _devptr(y), int(precision))
    if code != CELES_OK:
        raise CelesError(code, "celes_batch_master_matvec: " + celes_batch_last_error(b))


def celes_batch_solve(b, count, tol, mode=CELES_SOLVE_MIXED, restart=30, max_iter=2000, max_outer=8,
                      inner_tol=1e-5, raise_on_noconv=True):
    """Returns (status, list of per-context info dicts)."""
    opts = celes_solve_opts(int(mode), int(restart), int(max_iter), int(max_outer), CELES_X0_TA, 0, float(inner_tol),
                            CELES_SOLVER_GMRES)
    infos = (celes_solve_info * count)()
    code = load().celes_batch_solve(b, float(tol), ctypes.byref(opts), infos)
    out = [{"status": int(i.status), "iterations": i.iterations, "outer": i.outer, "matvecs_fp64": i.matvecs_fp64,
            "matvecs_fp32": i.matvecs_fp32, "residual": i.residual, "seconds": i.seconds} for i in infos]
    if code != CELES_OK and not (code == CELES_ENOCONV and not raise_on_noconv):
        raise CelesError(code, "celes_batch_solve: " + celes_batch_last_error(b))
    return int(code), out


def celes_batch_last_error(b):
    m = load().celes_batch_last_error(b)
    return m.decode() if m else ""


def celes_batch_destroy(b):
    if b:
        load().celes_batch_destroy(b)


def celes_destroy(ctx):
    if ctx:
        load().celes_destroy(ctx)


def celes_last_error(ctx):
    m = load().celes_last_error(ctx)
    return m.decode() if m else ""


def celes_version():
    return load().celes_version().decode()
