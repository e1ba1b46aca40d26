"""Python binding of the GB300 batched IPOP-CMA-ES engine (include/cmaes.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libcmaes_gb300.so``. The functions keep the C names; arrays are numpy,
matrices and population panels are column-major (Fortran order), as in the C
ABI. Importing this package does not need a GPU; loading the library does not
either, but every call that computes needs one. If the library is missing the
calls raise: there is no CPU fallback.
"""
import ctypes
import math
import os

import numpy as np

from . import _build

__all__ = [
    "CmaesError", "cmaes_options", "lib", "lib_path", "cmaes_default_options", "cmaes_create",
    "cmaes_create_batch", "cmaes_count", "cmaes_set_problem", "cmaes_ask", "cmaes_ask_device",
    "cmaes_tell", "cmaes_step_batch", "cmaes_sync", "cmaes_restart", "cmaes_best",
    "cmaes_get_state", "cmaes_set_state", "cmaes_get_generation", "cmaes_query",
    "cmaes_set_profiling", "cmaes_phase_times", "cmaes_kernel_launches", "cmaes_eig_stats",
    "cmaes_eig_stage_times",
    "cmaes_ask_async", "cmaes_tell_async",
    "probe_fma_tflops", "cmaes_ozaki_dgemm", "cmaes_evaluate_noalloc", "cmaes_inject_status", "cmaes_strerror",
    "cmaes_last_error", "cmaes_destroy",
]

FP64, MIXED_TF32, MIXED_BF16 = 0, 1, 2
EIG_AUTO, EIG_JACOBI, EIG_TRIDIAGONAL = 0, 1, 2
OBJ_ELLIPSOID, OBJ_RASTRIGIN, OBJ_SPHERE = 1, 2, 3
PHASES = ("sample", "objective", "update", "cov", "eig", "stop")


class CmaesError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (status %d): %s" % (_STATUS.get(status, "?"), status, message))
        self.status = status


_STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ETIMEOUT",
           6: "ENUMERIC", 7: "EUNSUPPORTED"}


class cmaes_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("ipop_double", ctypes.c_int), ("eig_every", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("stop_mask", ctypes.c_int),
                ("f_target", ctypes.c_double), ("box_lo", ctypes.c_double),
                ("box_hi", ctypes.c_double), ("tol_hist_fun", ctypes.c_double),
                ("tol_x_factor", ctypes.c_double), ("cond_max", ctypes.c_double),
                ("restart_hold", ctypes.c_int), ("eig_method", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)


class cmaes_state(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("lambda_", ctypes.c_int), ("gen", ctypes.c_int),
                ("restart", ctypes.c_int), ("done", ctypes.c_int), ("flags", ctypes.c_int),
                ("hist_count", ctypes.c_int), ("sigma", ctypes.c_double),
                ("best_f", ctypes.c_double), ("m", _DP), ("ps", _DP), ("pc", _DP), ("D", _DP),
                ("best_x", _DP), ("C", _DP), ("B", _DP), ("hist", _DP)]


def lib_path():
    return _build.LIB


_lib = None


def lib():
    """The loaded engine library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise CmaesError(3, "engine library %s is missing; run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    I, D, V = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    IP = ctypes.POINTER(ctypes.c_int)
    sig = {
        "cmaes_default_options": (None, [ctypes.POINTER(cmaes_options)]),
        "cmaes_create": (I, [I, I, _DP, D, ctypes.c_uint64, ctypes.POINTER(cmaes_options),
                             ctypes.POINTER(H)]),
        "cmaes_create_batch": (I, [I, IP, IP, ctypes.POINTER(_DP), _DP, ctypes.c_uint64,
                                   ctypes.POINTER(cmaes_options), ctypes.POINTER(H)]),
        "cmaes_count": (I, [H]),
        "cmaes_set_problem": (I, [H, I, I, _DP, _DP, _DP]),
        "cmaes_ask": (I, [H, I, _DP]),
        "cmaes_ask_device": (I, [H, I, ctypes.POINTER(V), IP]),
        "cmaes_tell": (I, [H, I, _DP]),
        "cmaes_step_batch": (I, [H, I, V]),
        "cmaes_sync": (I, [H]),
        "cmaes_restart": (I, [H, I]),
        "cmaes_best": (I, [H, I, _DP, _DP]),
        "cmaes_get_state": (I, [H, I, ctypes.POINTER(cmaes_state)]),
        "cmaes_set_state": (I, [H, I, ctypes.POINTER(cmaes_state)]),
        "cmaes_get_generation": (I, [H, I, _DP, _DP, IP]),
        "cmaes_query": (I, [H, I, IP, IP, IP, IP, IP]),
        "cmaes_set_profiling": (I, [H, I]),
        "cmaes_phase_times": (I, [H, _DP, ctypes.POINTER(ctypes.c_longlong), I]),
        "cmaes_kernel_launches": (ctypes.c_longlong, [H]),
        "cmaes_eig_stats": (I, [H, I] + [ctypes.POINTER(ctypes.c_longlong)] * 4),
        "cmaes_eig_stage_times": (I, [H, _DP, I]),
        "cmaes_evaluate_noalloc": (I, [I, I, I, V, I, V, I, V, V, V, V]),
        "cmaes_ask_async": (I, [H, I, I, ctypes.POINTER(V), ctypes.POINTER(ctypes.c_int), V]),
        "cmaes_tell_async": (I, [H, I, I, ctypes.POINTER(V), V]),
        "cmaes_inject_status": (I, [H, I]),
        "cmaes_ozaki_dgemm": (I, [I, I, I, D, V, ctypes.c_longlong, V, ctypes.c_longlong, D, V,
                                  ctypes.c_longlong, V]),
        "cmaes_strerror": (ctypes.c_char_p, [I]),
        "cmaes_last_error": (ctypes.c_char_p, [H]),
        "cmaes_destroy": (None, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(h, st):
    if st != 0:
        raise CmaesError(st, lib().cmaes_last_error(h).decode(errors="replace"))


def _dptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _colmajor(a, n):
    a = np.asfortranarray(a, dtype=np.float64)
    if a.shape != (n, n):
        raise ValueError("expected a %dx%d matrix" % (n, n))
    return a


def cmaes_default_options(**overrides):
    o = cmaes_options()
    lib().cmaes_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def cmaes_create(n, lam, x0, sigma0, seed, opt=None):
    h = ctypes.c_void_p()
    x0 = _f64(x0, n)
    st = lib().cmaes_create(n, lam, _dptr(x0), sigma0, seed,
                            ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(None, st)
    return h


def cmaes_create_batch(ns, lams, x0s, sigma0s, seed, opt=None):
    count = len(ns)
    n_arr = (ctypes.c_int * count)(*ns)
    l_arr = (ctypes.c_int * count)(*lams)
    xs = [_f64(x, n) for x, n in zip(x0s, ns)]
    x_arr = (_DP * count)(*[_dptr(x) for x in xs])
    s_arr = _f64(sigma0s, count)
    h = ctypes.c_void_p()
    st = lib().cmaes_create_batch(count, n_arr, l_arr, x_arr, _dptr(s_arr), seed,
                                  ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(None, st)
    return h


def cmaes_count(h):
    return lib().cmaes_count(h)


def cmaes_set_problem(h, s, kind, Q=None, lamdiag=None, xstar=None):
    xstar = _f64(xstar)
    n = xstar.size
    Qc = _colmajor(Q, n) if Q is not None else None
    ld = _f64(lamdiag, n) if lamdiag is not None else None
    _check(h, lib().cmaes_set_problem(h, s, kind, _dptr(Qc), _dptr(ld), _dptr(xstar)))


def cmaes_query(h, s):
    v = [ctypes.c_int() for _ in range(5)]
    _check(h, lib().cmaes_query(h, s, *[ctypes.byref(x) for x in v]))
    return dict(zip(("lam", "gen", "restart", "flags", "done"), (x.value for x in v)))


def cmaes_ask(h, s, n):
    lam = cmaes_query(h, s)["lam"]
    X = np.empty((n, lam), dtype=np.float64, order="F")
    _check(h, lib().cmaes_ask(h, s, _dptr(X)))
    return X


def cmaes_ask_device(h, s):
    p = ctypes.c_void_p()
    ld = ctypes.c_int()
    _check(h, lib().cmaes_ask_device(h, s, ctypes.byref(p), ctypes.byref(ld)))
    return p.value, ld.value


def cmaes_tell(h, s, f):
    f = _f64(f)
    _check(h, lib().cmaes_tell(h, s, _dptr(f)))


def cmaes_step_batch(h, generations, stream=None):
    _check(h, lib().cmaes_step_batch(h, generations, ctypes.c_void_p(stream) if stream else None))


def cmaes_sync(h):
    _check(h, lib().cmaes_sync(h))


def cmaes_restart(h, s):
    _check(h, lib().cmaes_restart(h, s))


def cmaes_ask_async(h, s0, s1, X_ptrs, lam_done_ptr, stream=None):
    """X_ptrs: host addresses (ints) of n x lambda_cap FP64 buffers, one per
    search of [s0, s1); lam_done_ptr: host address of 2 (s1 - s0) ints."""
    arr = (ctypes.c_void_p * max(1, s1 - s0))(*X_ptrs)  # the C side checks the range
    _check(h, lib().cmaes_ask_async(h, s0, s1, arr, ctypes.cast(lam_done_ptr, ctypes.POINTER(ctypes.c_int)),
                                    ctypes.c_void_p(stream) if stream else None))


def cmaes_tell_async(h, s0, s1, f_ptrs, stream=None):
    arr = (ctypes.c_void_p * max(1, s1 - s0))(*f_ptrs)  # the C side checks the range
    _check(h, lib().cmaes_tell_async(h, s0, s1, arr, ctypes.c_void_p(stream) if stream else None))


def cmaes_best(h, s, n):
    x = np.empty(n)
    f = ctypes.c_double()
    _check(h, lib().cmaes_best(h, s, _dptr(x), ctypes.byref(f)))
    return x, f.value


def cmaes_get_state(h, s, n, hist_cap=None):
    if hist_cap is None:
        hist_cap = 10 + int(math.ceil(30.0 * n / 2))
    arr = dict(m=np.empty(n), ps=np.empty(n), pc=np.empty(n), D=np.empty(n), best_x=np.empty(n),
               C=np.empty((n, n), order="F"), B=np.empty((n, n), order="F"), hist=np.empty(hist_cap))
    st = cmaes_state()
    for k, a in arr.items():
        setattr(st, k, _dptr(a))
    _check(h, lib().cmaes_get_state(h, s, ctypes.byref(st)))
    out = {k: np.array(a) for k, a in arr.items()}
    out["hist"] = out["hist"][:st.hist_count].copy()
    out.update(n=st.n, lam=st.lambda_, gen=st.gen, restart=st.restart, done=st.done,
               flags=st.flags, sigma=st.sigma, best_f=st.best_f)
    return out


def cmaes_set_state(h, s, d):
    """d: dict with n, lam, sigma and any of m, ps, pc, D, best_x, C, B, hist,
    gen, restart, done, flags, best_f."""
    n = int(d["n"])
    st = cmaes_state()
    st.n = n
    st.lambda_ = int(d["lam"])
    st.gen = int(d.get("gen", 0))
    st.restart = int(d.get("restart", 0))
    st.done = int(d.get("done", 0))
    st.flags = int(d.get("flags", 0))
    st.sigma = float(d["sigma"])
    st.best_f = float(d.get("best_f", math.inf))
    keep = []
    for k in ("m", "ps", "pc", "D", "best_x"):
        if d.get(k) is not None:
            a = _f64(d[k], n)
            keep.append(a)
            setattr(st, k, _dptr(a))
    for k in ("C", "B"):
        if d.get(k) is not None:
            a = _colmajor(d[k], n)
            keep.append(a)
            setattr(st, k, _dptr(a))
    hist = d.get("hist")
    if hist is not None and len(hist):
        a = _f64(hist)
        keep.append(a)
        st.hist = _dptr(a)
        st.hist_count = a.size
    _check(h, lib().cmaes_set_state(h, s, ctypes.byref(st)))


def cmaes_get_generation(h, s, n):
    lam = cmaes_query(h, s)["lam"]
    X = np.empty((n, lam), order="F")
    f = np.empty(lam)
    order = np.empty(lam, dtype=np.int32)
    _check(h, lib().cmaes_get_generation(h, s, _dptr(X), _dptr(f),
                                         order.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return X, f, order


def cmaes_set_profiling(h, enable):
    _check(h, lib().cmaes_set_profiling(h, 1 if enable else 0))


def cmaes_phase_times(h, reset=False):
    ms = (ctypes.c_double * 6)()
    ln = (ctypes.c_longlong * 6)()
    _check(h, lib().cmaes_phase_times(h, ms, ln, 1 if reset else 0))
    return dict(zip(PHASES, ms)), dict(zip(PHASES, ln))


def cmaes_eig_stats(h, s):
    v = [ctypes.c_longlong() for _ in range(4)]
    _check(h, lib().cmaes_eig_stats(h, s, *[ctypes.byref(x) for x in v]))
    return dict(zip(("decompositions", "sweeps", "rotations", "sweeps32"), (x.value for x in v)))


EIG_STAGES = ("reduction", "eigenvalues", "eigenvectors", "clusters", "orthogonalisation",
              "backtransform")


def cmaes_eig_stage_times(h, reset=False):
    """Device ms of the tridiagonal route's stages over the profiled
    generations (see include/cmaes.h)."""
    ms = (ctypes.c_double * len(EIG_STAGES))()
    _check(h, lib().cmaes_eig_stage_times(h, ms, 1 if reset else 0))
    return dict(zip(EIG_STAGES, ms))


def probe_fma_tflops(precision=64, blocks_per_sm=4, repeats=5):
    """Measured FMA throughput of the current device (TFLOP/s)."""
    L = ctypes.CDLL(_build.PROBE_LIB)
    L.cmaes_probe_fma_tflops.restype = ctypes.c_int
    L.cmaes_probe_fma_tflops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    st = L.cmaes_probe_fma_tflops(precision, blocks_per_sm, repeats, ctypes.byref(out))
    if st != 0:
        raise CmaesError(st, "FMA probe failed")
    return out.value


def cmaes_ozaki_dgemm(M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, stream=None):
    """C = alpha A B + beta C on device arrays (pointers as ints, column-major)
    with the engine's FP64-accurate tensor-core product; see
    include/cmaes_ozaki.h."""
    st = lib().cmaes_ozaki_dgemm(M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, stream)
    if st != 0:
        raise CmaesError({1: 1, 2: 2, 3: 3, 4: 5}.get(st, 3), "cmaes_ozaki_dgemm returned %d" % st)


def cmaes_kernel_launches(h):
    return lib().cmaes_kernel_launches(h)


def cmaes_evaluate_noalloc(kind, n, lam, X_ptr, ld, Q_ptr, ldq, lamdiag_ptr, xstar_ptr, f_ptr,
                           stream=None):
    """Objective values of lam points held in device memory (pointers as
    ints), with no device allocation; see include/cmaes.h."""
    st = lib().cmaes_evaluate_noalloc(kind, n, lam, X_ptr, ld, Q_ptr, ldq, lamdiag_ptr, xstar_ptr,
                                      f_ptr, stream)
    _check(None, st)


def cmaes_inject_status(h, bits):
    """ORs bits into the handle's device status word (host-side fault
    injection; see include/cmaes.h)."""
    _check(h, lib().cmaes_inject_status(h, bits))


def cmaes_strerror(st):
    return lib().cmaes_strerror(st).decode()


def cmaes_last_error(h=None):
    return lib().cmaes_last_error(h).decode(errors="replace")


def cmaes_destroy(h):
    if h:
        lib().cmaes_destroy(h)
