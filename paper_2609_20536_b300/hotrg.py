"""ctypes binding of libhotrg (argument marshalling only).

Entry points keep the C names: hotrg_create, hotrg_destroy, hotrg_init_tensor,
hotrg_step, hotrg_run, hotrg_observables, hotrg_last_error.  Device buffers
are passed as integer addresses (e.g. ``torch.Tensor.data_ptr()``); host
structs are the ctypes mirrors below.  Every numerical step runs in the CUDA
library; there is no Python or CPU fallback, and importing this module fails
when ``libhotrg.so`` is absent.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhotrg.so")

MAX_STEPS = 64

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6
FP64, SPLIT_BF16, SPLIT_BF16_FAST = 0, 1, 2
T_PURE, T_IMP_M, T_IMP_M1, T_ISING = 0, 1, 2, 3


class HotrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libhotrg status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_double), ("delta", ctypes.c_double),
        ("h", ctypes.c_double), ("h1", ctypes.c_double),
        ("n_max", ctypes.c_int32), ("d_cut", ctypes.c_int32), ("n_steps", ctypes.c_int32),
        ("prec", ctypes.c_int32), ("env_policy", ctypes.c_int32), ("m_range", ctypes.c_int32),
        ("eig_max_sweeps", ctypes.c_int32), ("tkind", ctypes.c_int32),
        ("tie_rtol", ctypes.c_double), ("eig_tol", ctypes.c_double), ("side_rtol", ctypes.c_double),
        ("block_sparse", ctypes.c_int32), ("gxy_q", ctypes.c_int32),
        ("eig_mode", ctypes.c_int32), ("eig_fp64_iters", ctypes.c_int32),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [
        ("ln_c", ctypes.c_double), ("eps_left", ctypes.c_double), ("eps_right", ctypes.c_double),
        ("side", ctypes.c_int32), ("dprime", ctypes.c_int32), ("sweeps", ctypes.c_int32),
        ("status", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("lnz_per_site", ctypes.c_double), ("ln_c0", ctypes.c_double), ("ln_trace", ctypes.c_double),
        ("imp_ratio", ctypes.c_double), ("step", StepInfo * MAX_STEPS),
        ("n_steps", ctypes.c_int32), ("status", ctypes.c_int32),
    ]


class Profile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64), ("gemm_calls", ctypes.c_int64 * 3), ("gemm_ms", ctypes.c_double * 3),
        ("gemm_flops", ctypes.c_double * 3), ("slice_ms", ctypes.c_double), ("eig_ms", ctypes.c_double),
        ("step_ms", ctypes.c_double), ("steps", ctypes.c_int64), ("eig_part_ms", ctypes.c_double * 4),
        ("operand_elems", ctypes.c_double * 3), ("output_elems", ctypes.c_double * 3),
    ]


class Obs(ctypes.Structure):
    _fields_ = [
        ("lnz", ctypes.c_double), ("f", ctypes.c_double), ("cv", ctypes.c_double),
        ("m", ctypes.c_double), ("m1", ctypes.c_double), ("chi", ctypes.c_double),
        ("chi1", ctypes.c_double), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


class TcFit(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
        ("a_err", ctypes.c_double), ("b_err", ctypes.c_double), ("c_err", ctypes.c_double),
        ("rss", ctypes.c_double), ("n", ctypes.c_int32), ("at_bound", ctypes.c_int32),
    ]


class PhaseOpts(ctypes.Structure):
    _fields_ = [
        ("field", ctypes.c_int32), ("nstreams", ctypes.c_int32), ("dh", ctypes.c_double),
        ("hb", ctypes.c_double), ("min_prominence", ctypes.c_double), ("c_lo", ctypes.c_double),
        ("c_hi", ctypes.c_double),
    ]


class Scaling(ctypes.Structure):
    _fields_ = [
        ("x_mean", ctypes.c_double * 2), ("x_std", ctypes.c_double * 2),
        ("y_mean", ctypes.c_double * 4), ("y_std", ctypes.c_double * 4),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhotrg.so not built ({LIB_PATH}); run paper_2609_20536_b300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.hotrg_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, vp]
    lib.hotrg_create.restype = ctypes.c_int
    lib.hotrg_destroy.argtypes = [vp]
    lib.hotrg_destroy.restype = None
    lib.hotrg_last_error.argtypes = [vp]
    lib.hotrg_last_error.restype = ctypes.c_char_p
    lib.hotrg_version.argtypes = []
    lib.hotrg_version.restype = ctypes.c_char_p
    lib.hotrg_init_tensor.argtypes = [vp, ctypes.POINTER(Params), i32, vp, vp]
    lib.hotrg_init_tensor.restype = ctypes.c_int
    lib.hotrg_step.argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, i32, i32, vp, vp,
                               ctypes.POINTER(i32), vp, vp, vp]
    lib.hotrg_step.restype = ctypes.c_int
    lib.hotrg_run.argtypes = [vp, ctypes.POINTER(Params), i32, i32, ctypes.POINTER(Result)]
    lib.hotrg_run.restype = ctypes.c_int
    lib.hotrg_observables.argtypes = [vp, ctypes.POINTER(Params), i32, f64, f64, f64, ctypes.POINTER(Obs)]
    lib.hotrg_observables.restype = ctypes.c_int
    lib.hotrg_observables_batch.argtypes = [vp, ctypes.POINTER(Params), i32, f64, f64, f64, i32,
                                            ctypes.POINTER(Obs)]
    lib.hotrg_observables_batch.restype = ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.hotrg_scaling_fit.argtypes = [dp, dp, i32, ctypes.POINTER(Scaling)]
    lib.hotrg_scaling_fit.restype = ctypes.c_int
    lib.hotrg_surrogate_fit.argtypes = [vp, dp, dp, i32, i32, i32, ctypes.c_float, ctypes.POINTER(Scaling),
                                        ctypes.POINTER(ctypes.c_float)]
    lib.hotrg_surrogate_fit.restype = ctypes.c_int
    lib.hotrg_surrogate_predict.argtypes = [vp, ctypes.POINTER(Scaling), dp, i32, dp, dp]
    lib.hotrg_surrogate_predict.restype = ctypes.c_int
    lib.hotrg_surrogate_peaks.argtypes = [vp, ctypes.POINTER(Scaling), dp, i32, f64, f64, i32, i32, f64, dp, dp]
    lib.hotrg_surrogate_peaks.restype = ctypes.c_int
    lib.hotrg_surrogate_refine.argtypes = [vp, vp, ctypes.POINTER(Scaling), ctypes.POINTER(Params), dp, i32, f64,
                                           f64, f64, f64, i32, dp, dp, ip, ip]
    lib.hotrg_surrogate_refine.restype = ctypes.c_int
    lib.hotrg_contract.argtypes = [vp, i32, i32, i32, i32, vp, ctypes.c_int64, vp, ctypes.c_int64, vp,
                                   ctypes.c_int64]
    lib.hotrg_contract.restype = ctypes.c_int
    lib.hotrg_find_peaks.argtypes = [dp, dp, i32, f64, i32, dp, dp, dp, ip]
    lib.hotrg_find_peaks.restype = ctypes.c_int
    lib.hotrg_fit_tc.argtypes = [dp, dp, i32, f64, f64, ctypes.POINTER(TcFit)]
    lib.hotrg_fit_tc.restype = ctypes.c_int
    lib.hotrg_phase_scan.argtypes = [vp, ctypes.POINTER(Params), dp, i32, dp, i32, ctypes.POINTER(PhaseOpts), dp,
                                     dp, dp, ctypes.POINTER(TcFit), ip]
    lib.hotrg_phase_scan.restype = ctypes.c_int
    lib.hotrg_profile_enable.argtypes = [vp, i32]
    lib.hotrg_profile_enable.restype = ctypes.c_int
    lib.hotrg_profile_read.argtypes = [vp, ctypes.POINTER(Profile)]
    lib.hotrg_profile_read.restype = ctypes.c_int
    return lib


lib = _load()


def params(beta, delta, n_max, d_cut, n_steps, h=0.0, h1=0.0, prec=FP64, env_policy=0, m_range=50,
           eig_max_sweeps=0, tkind=T_PURE, tie_rtol=0.0, eig_tol=0.0, side_rtol=0.0, block_sparse=0, q=2,
           eig_mode=0, eig_fp64_iters=0):
    return Params(beta, delta, h, h1, n_max, d_cut, n_steps, prec, env_policy, m_range,
                  eig_max_sweeps, tkind, tie_rtol, eig_tol, side_rtol, block_sparse, q, eig_mode, eig_fp64_iters)


def hotrg_create(workspace_bytes=0, stream=0):
    h = ctypes.c_void_p()
    st = lib.hotrg_create(ctypes.byref(h), workspace_bytes, ctypes.c_void_p(stream or None))
    if st != OK:
        raise HotrgError(st, "hotrg_create failed")
    return h


def hotrg_destroy(ctx):
    lib.hotrg_destroy(ctx)


def hotrg_last_error(ctx):
    return lib.hotrg_last_error(ctx).decode()


def _check(ctx, st):
    if st != OK:
        raise HotrgError(st, hotrg_last_error(ctx))
    return st


def hotrg_init_tensor(ctx, p, kind, T_ptr, labels_ptr):
    return _check(ctx, lib.hotrg_init_tensor(ctx, ctypes.byref(p), kind, ctypes.c_void_p(T_ptr),
                                             ctypes.c_void_p(labels_ptr)))


def hotrg_step(ctx, p, T_in, q_h, q_v, Dh, Dv, T_out, q_out, info_dev=0, T_imp_in=0, T_imp_out=0):
    dp = ctypes.c_int32(0)
    _check(ctx, lib.hotrg_step(ctx, ctypes.byref(p), ctypes.c_void_p(T_in), ctypes.c_void_p(q_h),
                               ctypes.c_void_p(q_v), Dh, Dv, ctypes.c_void_p(T_out), ctypes.c_void_p(q_out),
                               ctypes.byref(dp), ctypes.c_void_p(info_dev or None),
                               ctypes.c_void_p(T_imp_in or None), ctypes.c_void_p(T_imp_out or None)))
    return dp.value


def hotrg_run(ctx, plist, imp_kind=T_PURE, check=True):
    n = len(plist)
    arr = (Params * n)(*plist)
    out = (Result * n)()
    st = lib.hotrg_run(ctx, arr, n, imp_kind, out)
    if check:
        _check(ctx, st)
    return list(out)


def hotrg_run_batch(ctx, plist, imp_kind=T_PURE, nstreams=2, check=True):
    n = len(plist)
    arr = (Params * n)(*plist)
    out = (Result * n)()
    f = lib.hotrg_run_batch
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  ctypes.POINTER(Result)]
    f.restype = ctypes.c_int
    st = f(ctx, arr, n, imp_kind, nstreams, out)
    if check:
        _check(ctx, st)
    return list(out)


def hotrg_autotune_batch(ctx, plist, max_streams=4):
    """Times hotrg_run_batch with 1..max_streams worker streams; returns (best, seconds per count)."""
    n = len(plist)
    arr = (Params * n)(*plist)
    best = ctypes.c_int32(0)
    secs = (ctypes.c_double * max_streams)()
    f = lib.hotrg_autotune_batch
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32,
                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    _check(ctx, f(ctx, arr, n, max_streams, ctypes.byref(best), secs))
    return best.value, list(secs)


def hotrg_set_tiles(ctx, env_tile_n, coarse_tile_n):
    """Tile widths (128 or 64 output columns) of the split forms' block-sparse products."""
    f = lib.hotrg_set_tiles
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
    f.restype = ctypes.c_int
    return _check(ctx, f(ctx, env_tile_n, coarse_tile_n))


def hotrg_autotune_tiles(ctx, plist, nstreams=0):
    """Times the four (env, coarse) tile-width pairs on the sample; returns ((env, coarse), seconds)."""
    n = len(plist)
    arr = (Params * n)(*plist)
    e, c = ctypes.c_int32(0), ctypes.c_int32(0)
    secs = (ctypes.c_double * 4)()
    f = lib.hotrg_autotune_tiles
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32,
                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    _check(ctx, f(ctx, arr, n, nstreams, ctypes.byref(e), ctypes.byref(c), secs))
    return (e.value, c.value), list(secs)


def hotrg_observables(ctx, plist, hb=1e-3, hbar=0.01, dh=1e-3):
    n = len(plist)
    arr = (Params * n)(*plist)
    out = (Obs * n)()
    _check(ctx, lib.hotrg_observables(ctx, arr, n, hb, hbar, dh, out))
    return list(out)


def hotrg_observables_batch(ctx, plist, hb=1e-3, hbar=0.01, dh=1e-3, nstreams=2, check=True):
    n = len(plist)
    arr = (Params * n)(*plist)
    out = (Obs * n)()
    st = lib.hotrg_observables_batch(ctx, arr, n, hb, hbar, dh, nstreams, out)
    if check:
        _check(ctx, st)
    return list(out)


def _f64(a, cols):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, cols)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def hotrg_scaling_fit(X, Y):
    """Column means and standard deviations (host C++; no device work)."""
    X, xp = _f64(X, 2)
    Y, yp = _f64(Y, 4)
    s = Scaling()
    st = lib.hotrg_scaling_fit(xp, yp, len(X), ctypes.byref(s))
    if st != OK:
        raise HotrgError(st, "hotrg_scaling_fit")
    return s


def hotrg_find_peaks(x, y, min_prominence=0.0, cap=8):
    """Peaks of y(x) (host C++): ([(x_v, y_v, prominence), ...] in ascending x, number found)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if x.shape != y.shape or x.ndim != 1:
        raise ValueError("x and y must be 1-D arrays of one length")
    xp, yp, pr = (ctypes.c_double * max(cap, 1))(), (ctypes.c_double * max(cap, 1))(), (ctypes.c_double * max(cap, 1))()
    nf = ctypes.c_int32(0)
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.hotrg_find_peaks(x.ctypes.data_as(dp), y.ctypes.data_as(dp), len(x), min_prominence, cap, xp, yp, pr,
                              ctypes.byref(nf))
    if st != OK:
        raise HotrgError(st, "hotrg_find_peaks")
    return [(xp[i], yp[i], pr[i]) for i in range(min(cap, nf.value))], nf.value


def hotrg_fit_tc(hbar, t_peak, c_lo=0.0, c_hi=0.0):
    """Zero-field fit T_p(hbar) = a + b hbar^c (host C++); returns a TcFit."""
    import numpy as np
    h = np.ascontiguousarray(hbar, dtype=np.float64)
    t = np.ascontiguousarray(t_peak, dtype=np.float64)
    if h.shape != t.shape or h.ndim != 1:
        raise ValueError("hbar and t_peak must be 1-D arrays of one length")
    out = TcFit()
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.hotrg_fit_tc(h.ctypes.data_as(dp), t.ctypes.data_as(dp), len(h), c_lo, c_hi, ctypes.byref(out))
    if st != OK:
        raise HotrgError(st, "hotrg_fit_tc")
    return out


def hotrg_phase_scan(ctx, base, temps, hbars, field=0, dh=1e-3, hb=1e-3, min_prominence=0.0, nstreams=0,
                     c_lo=0.0, c_hi=0.0, with_cv=True, check=True):
    """Temperature scans at one Delta: dict with cv (n_t or None), chi (n_h x n_t), t_peak (n_h), fit, field."""
    import numpy as np
    temps = np.ascontiguousarray(temps, dtype=np.float64)
    hbars = np.ascontiguousarray(hbars, dtype=np.float64)
    nt, nh = len(temps), len(hbars)
    cv = np.zeros(nt) if with_cv else None
    chi = np.zeros((nh, nt))
    tp = np.zeros(nh)
    fit = TcFit()
    used = ctypes.c_int32(0)
    opts = PhaseOpts(field, nstreams, dh, hb, min_prominence, c_lo, c_hi)
    dp = ctypes.POINTER(ctypes.c_double)

    def ptr(a):
        return a.ctypes.data_as(dp) if a is not None and a.size else None
    st = lib.hotrg_phase_scan(ctx, ctypes.byref(base), ptr(temps), nt, ptr(hbars), nh, ctypes.byref(opts),
                              ptr(cv) if with_cv else None, ptr(chi), ptr(tp), ctypes.byref(fit), ctypes.byref(used))
    if check:
        _check(ctx, st)
    return {"cv": cv, "chi": chi, "t_peak": tp, "fit": fit, "field": used.value, "status": st}


def hotrg_contract(ctx, prec, M, N, K, A, lda, B, ldb, C, ldc):
    return _check(ctx, lib.hotrg_contract(ctx, prec, M, N, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(B), ldb,
                                          ctypes.c_void_p(C), ldc))


def hotrg_profile_enable(ctx, enable=True):
    return _check(ctx, lib.hotrg_profile_enable(ctx, 1 if enable else 0))


def hotrg_profile_read(ctx):
    out = Profile()
    _check(ctx, lib.hotrg_profile_read(ctx, ctypes.byref(out)))
    return out


def hotrg_contract_noalloc(prec, M, N, K, A, lda, B, ldb, C, ldc, stream=0):
    """Allocation-free split contraction (static device scratch); returns the status code."""
    f = lib.hotrg_contract_noalloc
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(prec, M, N, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(B), ldb, ctypes.c_void_p(C), ldc,
             ctypes.c_void_p(stream or None))


class MLP:
    """Ensemble of 2-128-128-128-4 networks (libhotrg surrogate kernels)."""

    def __init__(self, ensemble=4, seed=20536, stream=0):
        f = lib.hotrg_mlp_create
        f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p]
        f.restype = ctypes.c_int
        lib.hotrg_mlp_destroy.argtypes = [ctypes.c_void_p]
        lib.hotrg_mlp_destroy.restype = None
        lib.hotrg_mlp_num_params.restype = ctypes.c_int64
        self.handle = ctypes.c_void_p()
        st = f(ctypes.byref(self.handle), ensemble, seed, ctypes.c_void_p(stream or None))
        if st != OK:
            raise HotrgError(st, "hotrg_mlp_create failed")
        self.ensemble = ensemble
        self.nparams = lib.hotrg_mlp_num_params()

    def close(self):
        if self.handle:
            lib.hotrg_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _f32(a):
        import numpy as np
        return np.ascontiguousarray(a, dtype=np.float32)

    def _ptr(self, a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))

    def set_params(self, member, flat):
        a = self._f32(flat)
        lib.hotrg_mlp_set_params.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
        st = lib.hotrg_mlp_set_params(self.handle, member, self._ptr(a))
        if st != OK:
            raise HotrgError(st, "hotrg_mlp_set_params")

    def get_params(self, member):
        import numpy as np
        a = np.zeros(self.nparams, dtype=np.float32)
        lib.hotrg_mlp_get_params.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
        st = lib.hotrg_mlp_get_params(self.handle, member, self._ptr(a))
        if st != OK:
            raise HotrgError(st, "hotrg_mlp_get_params")
        return a

    def gradients(self, member, X, T):
        import numpy as np
        X, T = self._f32(X), self._f32(T)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float()
        f = lib.hotrg_mlp_gradients
        f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                      ctypes.c_int32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
        st = f(self.handle, member, self._ptr(X), self._ptr(T), len(X), ctypes.byref(loss), self._ptr(g))
        if st != OK:
            raise HotrgError(st, "hotrg_mlp_gradients")
        return loss.value, g

    def train(self, X, T, epochs=100, batch=256, lr=1e-3):
        X, T = self._f32(X), self._f32(T)
        loss = ctypes.c_float()
        f = lib.hotrg_mlp_train
        f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                      ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
        st = f(self.handle, self._ptr(X), self._ptr(T), len(X), epochs, batch, lr, ctypes.byref(loss))
        if st != OK:
            raise HotrgError(st, "hotrg_mlp_train")
        return loss.value

    def predict(self, X):
        import numpy as np
        X = self._f32(X)
        mean = np.zeros((len(X), 4), dtype=np.float32)
        spread = np.zeros((len(X), 4), dtype=np.float32)
        f = lib.hotrg_mlp_predict
        f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                      ctypes.POINTER(ctypes.c_float)]
        st = f(self.handle, self._ptr(X), len(X), self._ptr(mean), self._ptr(spread))
        if st != OK:
            raise HotrgError(st, "hotrg_mlp_predict")
        return mean, spread


class Surrogate:
    """MLP ensemble plus its standardisation: fit, predict, refinement
    points near the C_V / chi maxima, and HOTRG re-solves of uncertain
    points (hotrg_surrogate_* entry points)."""

    def __init__(self, ensemble=4, seed=20536, stream=0):
        self.mlp = MLP(ensemble, seed, stream)
        self.scaling = None

    def close(self):
        self.mlp.close()

    def fit(self, X, Y, epochs=200, batch=256, lr=1e-3):
        X, xp = _f64(X, 2)
        Y, yp = _f64(Y, 4)
        self.scaling = Scaling()
        loss = ctypes.c_float()
        st = lib.hotrg_surrogate_fit(self.mlp.handle, xp, yp, len(X), epochs, batch, lr, ctypes.byref(self.scaling),
                                     ctypes.byref(loss))
        if st != OK:
            raise HotrgError(st, "hotrg_surrogate_fit")
        return loss.value

    def predict(self, X):
        import numpy as np
        X, xp = _f64(X, 2)
        y = np.zeros((len(X), 4))
        sd = np.zeros((len(X), 4))
        st = lib.hotrg_surrogate_predict(self.mlp.handle, ctypes.byref(self.scaling), xp, len(X),
                                         y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         sd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if st != OK:
            raise HotrgError(st, "hotrg_surrogate_predict")
        return y, sd

    def peaks(self, deltas, beta_lo, beta_hi, n_beta, per_peak, width):
        import numpy as np
        d, dptr = _f64(deltas, 1)
        X = np.zeros((len(d) * 2 * per_peak, 2))
        pk = np.zeros((len(d), 2))
        st = lib.hotrg_surrogate_peaks(self.mlp.handle, ctypes.byref(self.scaling), dptr, len(d), beta_lo, beta_hi,
                                       n_beta, per_peak, width, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       pk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if st != OK:
            raise HotrgError(st, "hotrg_surrogate_peaks")
        return X, pk

    def refine(self, ctx, base, X, threshold=1e-3, hb=1e-3, hbar=0.01, dh=1e-3, nstreams=2):
        import numpy as np
        X, xp = _f64(X, 2)
        n = len(X)
        y = np.zeros((n, 4))
        sd = np.zeros((n, 4))
        solved = np.zeros(n, dtype=np.int32)
        ns = ctypes.c_int32(0)
        dptr = ctypes.POINTER(ctypes.c_double)
        st = lib.hotrg_surrogate_refine(ctx.handle if isinstance(ctx, Context) else ctx, self.mlp.handle,
                                        ctypes.byref(self.scaling), ctypes.byref(base), xp, n, threshold, hb, hbar,
                                        dh, nstreams, y.ctypes.data_as(dptr), sd.ctypes.data_as(dptr),
                                        solved.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(ns))
        if st != OK:
            raise HotrgError(st, "hotrg_surrogate_refine")
        return y, sd, solved.astype(bool)


class Context:
    """Owns one hotrg_ctx bound to a CUDA stream (0: legacy default)."""

    def __init__(self, workspace_bytes=0, stream=0):
        self.handle = hotrg_create(workspace_bytes, stream)

    def close(self):
        if self.handle:
            hotrg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, plist, imp_kind=T_PURE):
        return hotrg_run(self.handle, plist, imp_kind)

    def run_batch(self, plist, imp_kind=T_PURE, nstreams=2):
        return hotrg_run_batch(self.handle, plist, imp_kind, nstreams)

    def autotune_batch(self, plist, max_streams=4):
        return hotrg_autotune_batch(self.handle, plist, max_streams)

    def set_tiles(self, env_tile_n, coarse_tile_n):
        return hotrg_set_tiles(self.handle, env_tile_n, coarse_tile_n)

    def autotune_tiles(self, plist, nstreams=0):
        return hotrg_autotune_tiles(self.handle, plist, nstreams)

    def observables(self, plist, hb=1e-3, hbar=0.01, dh=1e-3):
        return hotrg_observables(self.handle, plist, hb, hbar, dh)

    def observables_batch(self, plist, hb=1e-3, hbar=0.01, dh=1e-3, nstreams=2):
        return hotrg_observables_batch(self.handle, plist, hb, hbar, dh, nstreams)

    def phase_scan(self, base, temps, hbars, **kw):
        return hotrg_phase_scan(self.handle, base, temps, hbars, **kw)
