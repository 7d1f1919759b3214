"""ctypes binding of libtcprod (include/tcprod.h): argument marshalling only.

Each ``tc_*`` function here calls the C function of the same name with the
device pointers of CUDA torch tensors and the current torch stream. Nothing
is computed in Python; if the library is missing the first call raises.
"""
import ctypes
import os

import torch

from . import build as _build

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p

TC_OK, TC_EINVAL, TC_ECUDA, TC_EBREAKDOWN, TC_ENONFINITE, TC_ETIMEOUT, TC_ENOMEM, \
    TC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
TC_FP32, TC_TF32, TC_BF16, TC_BF16X3 = 0, 1, 2, 3
TC_GCV_PAPER, TC_GCV_FULL = 0, 1
TC_TH, TC_ORTHODCT = 0, 1
TC_M, TC_MINV, TC_MINVT, TC_MT = 0, 1, 2, 3
TC_ROUTE_AUTO, TC_ROUTE_SPATIAL, TC_ROUTE_DUAL = 0, 1, 2
TC_DUAL_U, TC_DUAL_V = 0, 1
TC_STORE_F32, TC_STORE_BF16 = 0, 1
STATUS_NAMES = {0: "maxiter", 1: "converged", TC_EBREAKDOWN: "breakdown",
                TC_ENONFINITE: "nonfinite"}


class tc_opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("gcv_variant", c_int), ("use_graphs", c_int),
                ("product", c_int), ("route", c_int), ("store", c_int),
                ("reserved", c_int * 2)]


class tc_solve_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("status", c_int), ("cycles", c_int), ("fallback", c_int),
                ("resid", c_double), ("lambda_", c_double), ("gcv", c_double),
                ("beta1", c_double), ("kopt", c_int), ("reserved", c_int)]


_SIGS = {
    "tc_version": ([], ctypes.c_char_p),
    "tc_last_error": ([], ctypes.c_char_p),
    "tc_plan_create": ([ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                        ctypes.POINTER(tc_opts), c_void_p], c_int),
    "tc_plan_destroy": ([c_void_p], c_int),
    "tc_cprod": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "tc_cprod_adjoint": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "tc_gkb_init": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                     c_void_p], c_int),
    "tc_gkb_step": ([c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p],
                    c_int),
    "tc_lsqr_c": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_void_p,
                   c_void_p, c_void_p], c_int),
    "tc_lsqr_c_lcurve": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_void_p,
                          c_void_p, c_void_p], c_int),
    "tc_gmres_c": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_double, c_double,
                    c_void_p, c_void_p], c_int),
    "tc_tikhonov_gcv": ([c_void_p, c_int, c_void_p, c_int, c_double, c_void_p, c_void_p,
                         c_void_p, c_void_p], c_int),
    "tc_fro_norm_noalloc": ([c_void_p, ctypes.c_size_t, c_void_p, c_void_p], c_int),
    "tc_check_bounded_wait": ([c_int, c_void_p, c_void_p], c_int),
    "tc_slice_gemm": ([c_void_p, c_void_p, c_void_p, c_int, c_void_p], c_int),
    "tc_transform": ([c_void_p, c_int, c_void_p, c_void_p, ctypes.c_size_t, c_void_p, c_void_p,
                      c_void_p], c_int),
    "tc_transform_bf16in": ([c_void_p, c_int, c_void_p, c_void_p, ctypes.c_size_t, c_void_p,
                             c_void_p, c_int, c_void_p, c_void_p], c_int),
    "tc_slice_gemm_gk": ([c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                          c_void_p, c_void_p], c_int),
    "tc_transform_dual": ([c_void_p, c_int, c_void_p, c_void_p, ctypes.c_size_t, c_void_p,
                           c_void_p], c_int),
    "tc_plan_status": ([c_void_p, ctypes.POINTER(c_int)], c_int),
    "tc_lsqr_graph_kernels": ([c_void_p, ctypes.POINTER(c_int)], c_int),
    "tc_check_recip": ([c_void_p, ctypes.c_size_t, c_void_p, c_void_p, c_void_p], c_int),
    "tc_peak_probe": ([c_int, c_int, c_void_p, c_void_p], c_int),
    "tc_batch_create": ([ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_int),
                         ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_int,
                         ctypes.POINTER(c_void_p), ctypes.POINTER(tc_opts), c_void_p], c_int),
    "tc_batch_destroy": ([c_void_p], c_int),
    "tc_batch_info": ([c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                       ctypes.POINTER(ctypes.c_float)], c_int),
    "tc_mlp_create": ([ctypes.POINTER(c_void_p), ctypes.c_ulonglong, c_void_p], c_int),
    "tc_mlp_destroy": ([c_void_p], c_int),
    "tc_mlp_set_params": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "tc_mlp_get_params": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "tc_mlp_forward": ([c_void_p, c_void_p, c_int, c_void_p, c_void_p], c_int),
    "tc_mlp_loss_grad": ([c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p], c_int),
    "tc_mlp_fit_norm": ([c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p], c_int),
    "tc_mlp_train": ([c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, ctypes.c_float, c_void_p,
                      c_void_p], c_int),
    "tc_lsqr_label": ([c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p], c_int),
    "tc_lsqr_c_learned": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double,
                           c_void_p, c_void_p], c_int),
    "tc_lsqr_c_batched": ([c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                           ctypes.POINTER(c_void_p), c_int, c_double, c_double, c_void_p,
                           c_void_p], c_int),
}

_LIB = None


def lib():
    """Load libtcprod.so (built by build.build()); raise if it is missing."""
    global _LIB
    if _LIB is None:
        path = _build.lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libtcprod.so is not built ({path}); run "
                               "paper_2103_11847_gb300.build.build() first")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


class TcError(RuntimeError):
    def __init__(self, fn, code):
        msg = f"{fn} returned {code}"
        if code == TC_ECUDA:
            msg += ": " + lib().tc_last_error().decode()
        super().__init__(msg)
        self.code = code


def _check(fn, code):
    if code != TC_OK:
        raise TcError(fn, code)


def _ptr(t, dtype=torch.float32, shape=None, name="tensor"):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def tc_version():
    return lib().tc_version().decode()


def tc_plan_create(A, B=None, s=None, precision=TC_FP32, gcv_variant=TC_GCV_PAPER,
                   use_graphs=True, stream=None, product=TC_TH, route=TC_ROUTE_AUTO,
                   store=TC_STORE_F32):
    """A: (n3, n1, n2); B: (n3, s, s) or None (then s must be given)."""
    n3, n1, n2 = A.shape
    if B is not None:
        s = B.shape[1]
        _ptr(B, shape=(n3, s, s), name="B")
    if s is None:
        raise ValueError("s (columns of X) is required for a one-sided plan")
    o = tc_opts(precision, gcv_variant, int(bool(use_graphs)), product, route, store)
    h = c_void_p()
    _check("tc_plan_create", lib().tc_plan_create(ctypes.byref(h), n1, n2, s, n3, _ptr(A, name="A"),
                                                  _ptr(B, name="B"), ctypes.byref(o),
                                                  _stream(stream)))
    return h


def tc_plan_destroy(h):
    _check("tc_plan_destroy", lib().tc_plan_destroy(h))


def tc_cprod(h, X, Y, stream=None):
    _check("tc_cprod", lib().tc_cprod(h, _ptr(X, name="X"), _ptr(Y, name="Y"), _stream(stream)))


def tc_cprod_adjoint(h, Y, X, stream=None):
    _check("tc_cprod_adjoint", lib().tc_cprod_adjoint(h, _ptr(Y, name="Y"), _ptr(X, name="X"),
                                                      _stream(stream)))


def tc_gkb_init(h, C, U, V, alpha, beta, mmax, stream=None):
    _check("tc_gkb_init", lib().tc_gkb_init(h, _ptr(C), _ptr(U), _ptr(V),
                                            _ptr(alpha, torch.float64), _ptr(beta, torch.float64),
                                            mmax, _stream(stream)))


def tc_gkb_step(h, j, U, V, alpha, beta, mmax, stream=None):
    _check("tc_gkb_step", lib().tc_gkb_step(h, j, _ptr(U), _ptr(V), _ptr(alpha, torch.float64),
                                            _ptr(beta, torch.float64), mmax, _stream(stream)))


def new_info():
    """Device buffer for one tc_solve_info."""
    return torch.zeros(ctypes.sizeof(tc_solve_info), dtype=torch.uint8, device="cuda")


def read_info(buf):
    raw = bytes(buf.cpu().numpy().tobytes())
    info = tc_solve_info.from_buffer_copy(raw)
    return dict(iters=info.iters, status=STATUS_NAMES.get(info.status, info.status),
                cycles=info.cycles, fallback=info.fallback, resid=info.resid, lam=info.lambda_, gcv=info.gcv,
                beta1=info.beta1, kopt=info.kopt)


def tc_lsqr_c(h, C, X, X_reg, itermax, tol, lam, phibar_hist, info, stream=None):
    _check("tc_lsqr_c", lib().tc_lsqr_c(h, _ptr(C), _ptr(X), _ptr(X_reg), itermax, tol,
                                        -1.0 if lam is None else float(lam),
                                        _ptr(phibar_hist, torch.float64),
                                        _ptr(info, torch.uint8), _stream(stream)))


def tc_lsqr_c_lcurve(h, C, X, X_opt, kmax, tol, curve, info, stream=None):
    _check("tc_lsqr_c_lcurve", lib().tc_lsqr_c_lcurve(h, _ptr(C), _ptr(X), _ptr(X_opt), kmax, tol,
                                                      _ptr(curve, torch.float64),
                                                      _ptr(info, torch.uint8), _stream(stream)))


def tc_gmres_c(h, C, X0, X, m, itermax, tol, lam, info, stream=None):
    _check("tc_gmres_c", lib().tc_gmres_c(h, _ptr(C), _ptr(X0), _ptr(X), m, itermax, tol,
                                          -1.0 if lam is None else float(lam),
                                          _ptr(info, torch.uint8), _stream(stream)))


def tc_tikhonov_gcv(H, k, beta, variant, lam, lambda_out, y, gcv_out, stream=None):
    _check("tc_tikhonov_gcv", lib().tc_tikhonov_gcv(
        _ptr(H, torch.float64), k, _ptr(beta, torch.float64), variant,
        -1.0 if lam is None else float(lam), _ptr(lambda_out, torch.float64),
        _ptr(y, torch.float64), _ptr(gcv_out, torch.float64), _stream(stream)))


def tc_slice_gemm(h, Xh, Yh, adjoint=False, stream=None):
    """Transform-domain slice products; Xh is FP32, or BF16 for a BF16 plan."""
    dt = torch.bfloat16 if Xh.dtype == torch.bfloat16 else torch.float32
    _check("tc_slice_gemm", lib().tc_slice_gemm(h, _ptr(Xh, dt, name="Xh"), _ptr(Yh, name="Yh"),
                                                int(bool(adjoint)), _stream(stream)))


def tc_transform(h, which, X, Y, prev=None, sumsq=None, stream=None):
    """Y = X x_3 T (+ prev) with T = M, M^-1, M^-T or M^T (which = TC_M ..
    TC_MT); X, Y of shape (n3, ...); sumsq: device double for ||Y||^2 or None."""
    P = X[0].numel()
    if Y.shape != X.shape or (prev is not None and prev.shape != X.shape):
        raise ValueError("X, Y (and prev) must have the same shape")
    _check("tc_transform", lib().tc_transform(h, int(which), _ptr(X, name="X"), _ptr(Y, name="Y"),
                                              P, _ptr(prev, name="prev"),
                                              _ptr(sumsq, torch.float64, name="sumsq"),
                                              _stream(stream)))


def tc_transform_bf16in(h, which, X, Y, prev=None, sumsq=None, which_next=-1, nxt=None,
                        stream=None):
    """Y = X x_3 T (+ prev) from BF16 X (plans with TC_STORE_BF16); Y FP32;
    nxt (BF16, or None) = bf16(Y x_3 T_next)."""
    P = X[0].numel()
    if Y.shape != X.shape or (prev is not None and prev.shape != X.shape):
        raise ValueError("X, Y (and prev) must have the same shape")
    if nxt is not None and nxt.shape != X.shape:
        raise ValueError("nxt must have X's shape")
    _check("tc_transform_bf16in", lib().tc_transform_bf16in(
        h, int(which), _ptr(X, torch.bfloat16, name="X"), _ptr(Y, name="Y"), P,
        _ptr(prev, name="prev"), _ptr(sumsq, torch.float64, name="sumsq"), int(which_next),
        _ptr(nxt, torch.bfloat16, name="nxt"), _stream(stream)))


def tc_slice_gemm_gk(h, Xh, Yh, s0, s1=None, prev=None, sumsq=None, adjoint=False,
                     stream=None):
    """Yh = (1/s0) A~_k Xh_k - (s0/s1) prev (A~^T for adjoint); Xh BF16;
    s0, s1, sumsq: device float64 tensors of one element."""
    _check("tc_slice_gemm_gk", lib().tc_slice_gemm_gk(
        h, _ptr(Xh, torch.bfloat16, name="Xh"), _ptr(Yh, name="Yh"), int(bool(adjoint)),
        _ptr(s0, torch.float64, name="s0"), _ptr(s1, torch.float64, name="s1"),
        _ptr(prev, name="prev"), _ptr(sumsq, torch.float64, name="sumsq"), _stream(stream)))


def tc_transform_dual(h, which, X, Y, sumsq, stream=None):
    """Y = bf16(X x_3 G) (which = TC_DUAL_U) or bf16(X x_3 G^-1) (TC_DUAL_V),
    sumsq = ||X x_3 M^-1||^2 or ||X x_3 M^T||^2; X FP32, Y BF16, same shape
    (n3, ...); sumsq: device double."""
    P = X[0].numel()
    if Y.shape != X.shape:
        raise ValueError("X and Y must have the same shape")
    _check("tc_transform_dual", lib().tc_transform_dual(
        h, int(which), _ptr(X, name="X"), _ptr(Y, torch.bfloat16, name="Y"), P,
        _ptr(sumsq, torch.float64, name="sumsq"), _stream(stream)))


def tc_plan_status(h):
    """The plan's device status word (synchronous): TC_OK or TC_ETIMEOUT."""
    v = c_int(0)
    _check("tc_plan_status", lib().tc_plan_status(h, ctypes.byref(v)))
    return v.value


def tc_lsqr_graph_kernels(h):
    """Kernel launches in the plan's captured c-LSQR graph (0 if none)."""
    v = c_int(0)
    _check("tc_lsqr_graph_kernels", lib().tc_lsqr_graph_kernels(h, ctypes.byref(v)))
    return v.value


def tc_check_recip(x, rcp, rsq, stream=None):
    """rcp = 1/x, rsq = 1/sqrt(x) by the library's FP64 helpers (float64 tensors)."""
    _check("tc_check_recip", lib().tc_check_recip(
        _ptr(x, torch.float64, name="x"), x.numel(), _ptr(rcp, torch.float64, name="rcp"),
        _ptr(rsq, torch.float64, name="rsq"), _stream(stream)))


def tc_peak_probe(kind, iters, status, stream=None):
    """Launch the peak-rate probe `kind` (0 FFMA, 1 DFMA, 2 TF32 MMA, 3 BF16 MMA)."""
    _check("tc_peak_probe", lib().tc_peak_probe(int(kind), int(iters),
                                                _ptr(status, torch.int32, name="status"),
                                                _stream(stream)))


def tc_fro_norm_noalloc(X, out, stream=None):
    """||X||_F into the device double `out`, using no device allocation."""
    _check("tc_fro_norm_noalloc", lib().tc_fro_norm_noalloc(
        _ptr(X, name="X"), X.numel(), _ptr(out, torch.float64, name="out"), _stream(stream)))


def tc_check_bounded_wait(spins, status, stream=None):
    """One bounded mbarrier wait that cannot complete; writes TC_ETIMEOUT to
    the device int32 `status`."""
    _check("tc_check_bounded_wait", lib().tc_check_bounded_wait(
        int(spins), _ptr(status, torch.int32, name="status"), _stream(stream)))


def _ptr_array(ts, name):
    arr = (c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t, name=f"{name}[{i}]")
    return arr


def tc_batch_create(As, ss, precision=TC_FP32, gcv_variant=TC_GCV_PAPER, stream=None,
                    product=TC_TH):
    """As: list of (n3, n1_i, n2_i) CUDA tensors; ss: list of column counts."""
    n = len(As)
    n3 = As[0].shape[0]
    n1 = (c_int * n)(*[a.shape[1] for a in As])
    n2 = (c_int * n)(*[a.shape[2] for a in As])
    sv = (c_int * n)(*ss)
    o = tc_opts(precision, gcv_variant, 1, product)
    h = c_void_p()
    _check("tc_batch_create", lib().tc_batch_create(ctypes.byref(h), n, n1, n2, sv, n3,
                                                    _ptr_array(As, "A"), ctypes.byref(o),
                                                    _stream(stream)))
    return h


def tc_batch_destroy(h):
    _check("tc_batch_destroy", lib().tc_batch_destroy(h))


def tc_batch_info(h, mode=-1):
    """Set the batch's form (mode 0: grouped where eligible, tile autotuned;
    1: child graphs; 2 + t: grouped with tile shape t; -1 leaves it) and
    return (grouped, tile shape in use, autotune times in ms)."""
    g, t = c_int(0), c_int(0)
    ms = (ctypes.c_float * 3)()
    _check("tc_batch_info", lib().tc_batch_info(h, int(mode), ctypes.byref(g), ctypes.byref(t),
                                                ms))
    return bool(g.value), t.value, tuple(ms)


def tc_batch_force_tile(h, tile):
    """The grouped form with tile shape `tile`, no autotuning."""
    return tc_batch_info(h, mode=2 + int(tile))


def tc_lsqr_c_batched(h, Cs, Xs, Xregs, itermax, tol, lam, infos, stream=None):
    """infos: device uint8 tensor of len(Cs) * sizeof(tc_solve_info) bytes."""
    _check("tc_lsqr_c_batched", lib().tc_lsqr_c_batched(
        h, _ptr_array(Cs, "C"), _ptr_array(Xs, "X"),
        _ptr_array(Xregs, "X_reg") if Xregs is not None else None, itermax, tol,
        -1.0 if lam is None else float(lam), _ptr(infos, torch.uint8), _stream(stream)))


def new_infos(count):
    return torch.zeros(count * ctypes.sizeof(tc_solve_info), dtype=torch.uint8, device="cuda")


def read_infos(buf, count):
    sz = ctypes.sizeof(tc_solve_info)
    return [read_info(buf[i * sz:(i + 1) * sz]) for i in range(count)]


MLP_NPARAMS, MLP_NORM = 6658, 76


class Mlp:
    """The learned-lambda network (tc_mlp_*): thin wrapper over the C calls."""

    def __init__(self, seed=0):
        self.handle = c_void_p()
        _check("tc_mlp_create", lib().tc_mlp_create(ctypes.byref(self.handle), seed, _stream(None)))

    def close(self):
        if self.handle is not None:
            lib().tc_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta=None, norm=None):
        _check("tc_mlp_set_params", lib().tc_mlp_set_params(
            self.handle, _ptr(theta, name="theta"), _ptr(norm, name="norm"), _stream(None)))

    def get_params(self):
        theta = torch.empty(MLP_NPARAMS, device="cuda")
        norm = torch.empty(MLP_NORM, device="cuda")
        _check("tc_mlp_get_params", lib().tc_mlp_get_params(self.handle, _ptr(theta), _ptr(norm),
                                                            _stream(None)))
        return theta, norm

    def forward(self, X):
        Y = torch.empty((X.shape[0], 2), device="cuda")
        _check("tc_mlp_forward", lib().tc_mlp_forward(self.handle, _ptr(X), X.shape[0], _ptr(Y),
                                                      _stream(None)))
        return Y

    def loss_grad(self, X, T):
        loss = torch.empty(1, device="cuda")
        grad = torch.empty(MLP_NPARAMS, device="cuda")
        _check("tc_mlp_loss_grad", lib().tc_mlp_loss_grad(self.handle, _ptr(X), _ptr(T), X.shape[0],
                                                          _ptr(loss), _ptr(grad), _stream(None)))
        return loss, grad

    def fit_norm(self, Xraw, Traw):
        Xn, Tn = torch.empty_like(Xraw), torch.empty_like(Traw)
        _check("tc_mlp_fit_norm", lib().tc_mlp_fit_norm(self.handle, _ptr(Xraw), _ptr(Traw),
                                                        Xraw.shape[0], _ptr(Xn), _ptr(Tn),
                                                        _stream(None)))
        return Xn, Tn

    def train(self, Xn, Tn, batch, steps, lr):
        hist = torch.empty(steps, device="cuda")
        _check("tc_mlp_train", lib().tc_mlp_train(self.handle, _ptr(Xn), _ptr(Tn), Xn.shape[0], batch,
                                                  steps, lr, _ptr(hist), _stream(None)))
        return hist


def tc_lsqr_label(h, C, X_true, kmax, feat, target, stream=None):
    _check("tc_lsqr_label", lib().tc_lsqr_label(h, _ptr(C), _ptr(X_true), kmax, _ptr(feat),
                                                _ptr(target), _stream(stream)))


def tc_lsqr_c_learned(h, mlp, C, X, X_reg, kmax, gcv_factor, info, stream=None):
    _check("tc_lsqr_c_learned", lib().tc_lsqr_c_learned(h, mlp.handle, _ptr(C), _ptr(X), _ptr(X_reg),
                                                        kmax, gcv_factor, _ptr(info, torch.uint8),
                                                        _stream(stream)))


class Plan:
    """Owns a tc_plan for A (and B); methods allocate outputs as torch tensors."""

    def __init__(self, A, B=None, s=None, precision=TC_FP32, gcv_variant=TC_GCV_PAPER,
                 use_graphs=True, product=TC_TH, route=TC_ROUTE_AUTO, store=TC_STORE_F32):
        self.n3, self.n1, self.n2 = A.shape
        self.s = B.shape[1] if B is not None else s
        self.two_sided = B is not None
        self.handle = tc_plan_create(A, B, s, precision, gcv_variant, use_graphs,
                                     product=product, route=route, store=store)

    def close(self):
        if self.handle is not None:
            tc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def xshape(self):
        return (self.n3, self.n2, self.s)

    def yshape(self):
        return (self.n3, self.n1, self.s)

    def cprod(self, X, out=None):
        Y = out if out is not None else torch.empty(self.yshape(), device="cuda")
        tc_cprod(self.handle, X, Y)
        return Y

    def adjoint(self, Y, out=None):
        X = out if out is not None else torch.empty(self.xshape(), device="cuda")
        tc_cprod_adjoint(self.handle, Y, X)
        return X

    def lsqr(self, C, itermax, tol=0.0, regularize=False, lam=None, history=False):
        X = torch.empty(self.xshape(), device="cuda")
        Xr = torch.empty(self.xshape(), device="cuda") if regularize else None
        hist = torch.zeros(itermax, dtype=torch.float64, device="cuda") if history else None
        info = new_info()
        tc_lsqr_c(self.handle, C, X, Xr, itermax, tol, lam, hist, info)
        return X, Xr, hist, info

    def lsqr_lcurve(self, C, kmax, tol=0.0):
        """c-LSQR stopped at the L-curve corner: (X_K, X_{k_opt}, curve, info);
        curve[:kmax] holds ||R_k||, curve[kmax:] ||X_k|| for k = 1..K."""
        X = torch.empty(self.xshape(), device="cuda")
        Xo = torch.empty(self.xshape(), device="cuda")
        curve = torch.full((2 * kmax,), float("nan"), dtype=torch.float64, device="cuda")
        info = new_info()
        tc_lsqr_c_lcurve(self.handle, C, X, Xo, kmax, tol, curve, info)
        return X, Xo, curve, info

    def gmres(self, C, m, itermax, tol=0.0, lam=None, X0=None):
        X = torch.empty(self.xshape(), device="cuda")
        info = new_info()
        tc_gmres_c(self.handle, C, X0, X, m, itermax, tol, lam, info)
        return X, info
