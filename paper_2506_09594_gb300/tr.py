"""Thin ctypes binding of libtr (include/tr.h).

Argument marshalling only: every step of the proximal iteration runs in the
CUDA library.  Device buffers are torch CUDA tensors (PyTorch provides the
memory and the stream); their data pointers are passed straight through.
There is no CPU fallback: if libtr.so is missing or fails to load, every call
raises.
"""

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtr.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "tr.h")

# tr_status
TR_OK, TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_ENUMERIC, TR_ETIMEOUT, TR_ENOTCONV, TR_EUNSUPPORTED = range(8)
STATUS_NAMES = ["TR_OK", "TR_EINVAL", "TR_ENOMEM", "TR_ECUDA", "TR_ENUMERIC", "TR_ETIMEOUT",
                "TR_ENOTCONV", "TR_EUNSUPPORTED"]
TR_F32, TR_F64 = 0, 1
TR_PEN_L1, TR_PEN_MCP = 0, 1
TR_NOISE_NONE, TR_NOISE_L1 = 0, 1
TR_LR_FULLSVD, TR_LR_RSVD, TR_LR_ADAPTIVE, TR_LR_LEARNED, TR_LR_TUCKER = 0, 1, 2, 3, 4
TR_PREC_FP32, TR_PREC_TF32, TR_PREC_BF16, TR_PREC_BF16X3 = 0, 1, 2, 3
TR_MLP_FEATURES, TR_MLP_PARAMS = 16, 35329
MODEL_MAGIC = b"TRRANK01"
DEFAULT_MODEL = os.path.join(PKG, "rank_mlp.bin")


class TrError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, msg))


class tr_problem(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("dims", ctypes.c_int64 * 8), ("dtype", ctypes.c_int),
                ("observed", ctypes.c_void_p), ("mask", ctypes.c_void_p)]


class tr_params(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_int), ("phi_theta", ctypes.c_double), ("phi_gamma", ctypes.c_double),
                ("psi", ctypes.c_int), ("psi_theta", ctypes.c_double), ("psi_gamma", ctypes.c_double),
                ("noise", ctypes.c_int), ("lambda_", ctypes.c_double),
                ("mu0", ctypes.c_double), ("mu_max", ctypes.c_double), ("growth", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("engine", ctypes.c_int), ("rank", ctypes.c_int), ("oversample", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("adapt_eps", ctypes.c_double),
                ("adapt_block", ctypes.c_int), ("prec", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("model_path", ctypes.c_char_p)]


class tr_ctv_params(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_uint32), ("phi", ctypes.c_int), ("phi_theta", ctypes.c_double),
                ("phi_gamma", ctypes.c_double), ("psi", ctypes.c_int),
                ("psi_theta", ctypes.c_double), ("psi_gamma", ctypes.c_double),
                ("noise", ctypes.c_int), ("lambda_", ctypes.c_double),
                ("mu0", ctypes.c_double), ("mu_max", ctypes.c_double), ("growth", ctypes.c_double),
                ("rank", ctypes.c_int), ("oversample", ctypes.c_int), ("power_iters", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int)]


class tr_onebit_params(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_uint32), ("lambda_", ctypes.c_double),
                ("theta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("mu0", ctypes.c_double), ("mu_max", ctypes.c_double), ("growth", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("phi", ctypes.c_int), ("phi_theta", ctypes.c_double),
                ("phi_gamma", ctypes.c_double), ("rank", ctypes.c_int),
                ("oversample", ctypes.c_int), ("power_iters", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int)]


class tr_step_info(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int), ("mu", ctypes.c_double), ("tau", ctypes.c_double),
                ("res_inf", ctypes.c_double * 5), ("max_rank", ctypes.c_int),
                ("sum_rank", ctypes.c_int), ("fallback_slices", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"iter": self.iter, "mu": self.mu, "tau": self.tau, "res_inf": list(self.res_inf),
                "max_rank": self.max_rank, "sum_rank": self.sum_rank,
                "fallback_slices": self.fallback_slices, "ms": self.ms}


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "tr_default_params": (None, [ctypes.POINTER(tr_params)]),
    "tr_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(tr_problem),
                               ctypes.POINTER(tr_params), _P]),
    "tr_prox_step": (ctypes.c_int, [_P, ctypes.POINTER(tr_step_info)]),
    "tr_recover": (ctypes.c_int, [_P, _P, ctypes.POINTER(tr_step_info)]),
    "tr_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int)]),
    "tr_set_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int]),
    "tr_transform_forward": (ctypes.c_int, [_P, _P, _P]),
    "tr_transform_inverse": (ctypes.c_int, [_P, _P, _P]),
    "tr_slice_prox": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int]),
    "tr_last_slice_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "tr_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "tr_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "tr_kernel_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "tr_profile_slice_pass": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_char_p), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int)]),
    "tr_slice_prox_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64, ctypes.c_int, _P,
                                             ctypes.c_char_p, ctypes.c_size_t]),
    "tr_slice_prox_ad_tucker": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_uint64, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int), _P, ctypes.c_char_p,
                                               ctypes.c_size_t]),
    "tr_grad": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                               ctypes.c_int, ctypes.c_int, _P, _P, _P, ctypes.c_char_p,
                               ctypes.c_size_t]),
    "tr_gradient_solve": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_uint32, _P, _P,
                                         _P, ctypes.c_char_p, ctypes.c_size_t]),
    "tr_ctv_default_params": (None, [_P]),
    "tr_ctv_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, _P, ctypes.c_char_p,
                                     ctypes.c_size_t]),
    "tr_ctv_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "tr_ctv_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]),
    "tr_ctv_set_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int]),
    "tr_ctv_last_error": (ctypes.c_char_p, [_P]),
    "tr_ctv_free": (ctypes.c_int, [_P]),
    "tr_onebit_default_params": (None, [_P]),
    "tr_onebit_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _P, _P,
                                        _P, _P, ctypes.c_char_p, ctypes.c_size_t]),
    "tr_onebit_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "tr_onebit_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int)]),
    "tr_onebit_set_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int]),
    "tr_onebit_last_error": (ctypes.c_char_p, [_P]),
    "tr_onebit_free": (ctypes.c_int, [_P]),
    "tr_mlp_param_count": (ctypes.c_int64, []),
    "tr_set_model": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "tr_last_slice_widths": (ctypes.c_int, [_P, _P]),
    "tr_slice_features": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _P]),
    "tr_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P]),
    "tr_plan_widths": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                      _P]),
    "tr_mlp_init": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "tr_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "tr_mlp_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, _P, _P, _P]),
    "tr_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, _P]),
    "tr_mlp_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64, _P, _P]),
    "tr_set_observed": (ctypes.c_int, [_P, _P, _P]),
    "tr_read_residuals": (ctypes.c_int, [_P, _P]),
    "tr_slice_prox_tucker": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "tr_graph_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "tr_set_tube_tile": (ctypes.c_int, [_P, ctypes.c_int]),
    "tr_set_slice_groups": (ctypes.c_int, [_P, ctypes.c_int]),
    "tr_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]),
    "tr_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, _P, ctypes.c_int,
                                       _P]),
    "tr_batch_step": (ctypes.c_int, [_P, _P]),
    "tr_batch_handle": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "tr_batch_graph_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "tr_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int]),
    "tr_batch_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "tr_batch_free": (ctypes.c_int, [_P]),
    "tr_batch_last_error": (ctypes.c_char_p, []),
    "tr_free": (ctypes.c_int, [_P]),
    "tr_last_error": (ctypes.c_char_p, [_P]),
}


def load(path=LIB_PATH):
    """Load libtr.so (raises if it is absent: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libtr.so not built at %s; run paper_2506_09594_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(header=HEADER):
    """Names of the functions declared in include/tr.h."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tr_\w+)\s*\(", txt)))


def _check(st, h=None):
    if st != TR_OK:
        msg = load().tr_last_error(h)
        raise TrError(st, msg.decode() if msg else "")


def default_params(**kw):
    p = tr_params()
    load().tr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "lambda":
            k = "lambda_"
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class TrArgError(TrError, ValueError):
    """A tensor argument refused by the binding before the C call (the C ABI
    sees only pointers, so dtype, device, layout and size are checked here)."""

    def __init__(self, msg):
        super().__init__(TR_EINVAL, msg)


def _need(t, name, dtype, numel, device="cuda", optional=False):
    """Check that `t` is a contiguous tensor on `device` of `dtype` (a dtype
    or a tuple of them) holding at least `numel` elements; None passes when
    the C call accepts NULL (optional)."""
    import torch
    if t is None:
        if optional:
            return
        raise TrArgError("%s: a tensor is required" % name)
    if not isinstance(t, torch.Tensor):
        raise TrArgError("%s: expected a torch tensor, got %s" % (name, type(t).__name__))
    if t.device.type != device:
        raise TrArgError("%s: expected a %s tensor, got one on %s" % (name, device, t.device))
    ok = dtype if isinstance(dtype, tuple) else (dtype,)
    if dtype is not None and t.dtype not in ok:
        raise TrArgError("%s: expected %s, got %s" % (name, " or ".join(map(str, ok)), t.dtype))
    if not t.is_contiguous():
        raise TrArgError("%s: must be contiguous" % name)
    if t.numel() < numel:
        raise TrArgError("%s: holds %d elements, the call needs %d" % (name, t.numel(), numel))


def _float_dtype(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype not in (torch.float32, torch.float64):
        raise TrArgError("%s: expected a float32 or float64 tensor" % name)
    return {torch.float32: TR_F32, torch.float64: TR_F64}[t.dtype]


def slice_prox_noalloc(Abar, Gbar, l, q, tau, t, seed=0, phi=TR_PEN_MCP, theta=1.0,
                       gamma=4000.0, stream=None):
    """tr_slice_prox_noalloc: the slice pass with no device allocation.

    For callers that cannot allocate device memory (latency-critical host
    loops, code living in another framework's memory pool).  Abar and Gbar
    are (n, n1, n2) CUDA tensors supplied by the caller; scratch comes from a
    fixed array inside the library.  Raises TrError on failure.
    """
    import torch
    dt = _float_dtype(Abar, "Abar")
    if Abar.dim() != 3:
        raise TrArgError("Abar: expected an (n, n1, n2) tensor")
    n, n1, n2 = Abar.shape
    _need(Abar, "Abar", Abar.dtype, n * n1 * n2)
    _need(Gbar, "Gbar", Abar.dtype, n * n1 * n2)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    buf = ctypes.create_string_buffer(256)
    st = load().tr_slice_prox_noalloc(dt, n, n1, n2, _ptr(Abar), _ptr(Gbar), int(l), int(q),
                                      int(phi), float(theta), float(gamma), float(tau),
                                      int(seed), int(t), ctypes.c_void_p(stream), buf, 256)
    if st != TR_OK:
        raise TrError(st, buf.value.decode())
    return Gbar


def _dims_array(dims):
    arr = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
    n = 1
    for d in dims:
        n *= max(int(d), 0)
    return arr, n


def grad(src, dims, mode, adjoint=False, out=None, stream=None):
    """tr_grad: nabla_mode(src) (or its adjoint) of a face-slice stack of the
    tensor with sizes `dims`; returns `out`."""
    import torch
    dt = _float_dtype(src, "src")
    arr, N = _dims_array(dims)
    _need(src, "src", src.dtype, N)
    if out is None:
        out = torch.empty_like(src)
    _need(out, "out", src.dtype, N)
    buf = ctypes.create_string_buffer(256)
    st = load().tr_grad(dt, len(dims), arr, int(mode), int(bool(adjoint)), _ptr(src), _ptr(out),
                        _stream(stream), buf, 256)
    if st != TR_OK:
        raise TrError(st, buf.value.decode())
    return out


def gradient_solve(rhs, dims, modes, out=None, stream=None):
    """tr_gradient_solve: (I + sum_{k in modes} nabla_k^T nabla_k)^{-1} rhs for
    the modes listed (1-based); returns `out`."""
    import torch
    dt = _float_dtype(rhs, "rhs")
    arr, N = _dims_array(dims)
    _need(rhs, "rhs", rhs.dtype, N)
    if out is None:
        out = torch.empty_like(rhs)
    _need(out, "out", rhs.dtype, N)
    mask = 0
    for k in modes:
        if not 1 <= int(k) <= len(dims):
            raise TrArgError("modes: %r is not a mode of an order-%d tensor" % (k, len(dims)))
        mask |= 1 << (int(k) - 1)
    buf = ctypes.create_string_buffer(256)
    st = load().tr_gradient_solve(dt, len(dims), arr, mask, _ptr(rhs), _ptr(out), _stream(stream),
                                  buf, 256)
    if st != TR_OK:
        raise TrError(st, buf.value.decode())
    return out


def slice_prox_ad_tucker(Abar, tau, eps, b, delta_rel=1e-12, max_rank=0, phi=TR_PEN_MCP,
                         theta=1.0, gamma=4000.0, seed=0, t=0, out=None, stream=None):
    """tr_slice_prox_ad_tucker: the fixed-accuracy shared-Tucker prox of a
    transformed stack Abar (n, n1, n2); returns (Gbar, (r1, r2))."""
    import torch
    dt = _float_dtype(Abar, "Abar")
    if Abar.dim() != 3:
        raise TrArgError("Abar: expected an (n, n1, n2) tensor")
    n, n1, n2 = Abar.shape
    _need(Abar, "Abar", Abar.dtype, n * n1 * n2)
    if out is None:
        out = torch.empty_like(Abar)
    _need(out, "out", Abar.dtype, n * n1 * n2)
    ranks = (ctypes.c_int * 2)()
    buf = ctypes.create_string_buffer(256)
    st = load().tr_slice_prox_ad_tucker(dt, n, n1, n2, _ptr(Abar), _ptr(out), float(tau), int(phi),
                                        float(theta), float(gamma), float(eps), int(b),
                                        float(delta_rel), int(max_rank), int(seed), int(t), ranks,
                                        _stream(stream), buf, 256)
    if st != TR_OK:
        raise TrError(st, buf.value.decode())
    return out, (ranks[0], ranks[1])


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(stream)


def save_model(path, params):
    """Write a weights file (layout documented at tr_set_model in tr.h)."""
    import numpy as np
    w = np.ascontiguousarray(np.asarray(params, dtype="<f4").ravel())
    if w.size != TR_MLP_PARAMS:
        raise ValueError("expected %d parameters, got %d" % (TR_MLP_PARAMS, w.size))
    with open(path, "wb") as f:
        f.write(MODEL_MAGIC)
        f.write(np.array([TR_MLP_FEATURES, 128, 3, 0], dtype="<i4").tobytes())
        f.write(np.array([w.size], dtype="<i8").tobytes())
        f.write(w.tobytes())


def load_model(path):
    """Read a weights file into a float32 numpy array."""
    import numpy as np
    with open(path, "rb") as f:
        raw = f.read()
    if raw[:8] != MODEL_MAGIC:
        raise ValueError("%s: not a rank-predictor weights file" % path)
    dims = np.frombuffer(raw[8:24], dtype="<i4")
    count = int(np.frombuffer(raw[24:32], dtype="<i8")[0])
    if tuple(dims) != (TR_MLP_FEATURES, 128, 3, 0) or count != TR_MLP_PARAMS:
        raise ValueError("%s: unexpected architecture %s / %d" % (path, tuple(dims), count))
    return np.frombuffer(raw[32:32 + 4 * count], dtype="<f4").copy()


def features(sig, rank, width, thr, thr0, tfrac, stream=None):
    """tr_features: (n, 16) float32 features from per-slice singular values."""
    import torch
    dt = _float_dtype(sig, "sig")
    if sig.dim() != 2:
        raise TrArgError("sig: expected an (n, ldsig) tensor")
    n, ldsig = sig.shape
    _need(sig, "sig", sig.dtype, n * ldsig)
    _need(rank, "rank", torch.int32, n)
    _need(width, "width", torch.int32, n)
    out = torch.empty((n, TR_MLP_FEATURES), dtype=torch.float32, device=sig.device)
    _check(load().tr_features(dt, n, _ptr(sig), ldsig, _ptr(rank), _ptr(width), float(thr),
                              float(thr0), float(tfrac), _ptr(out), _stream(stream)))
    return out


def plan_widths(yhat, oversample, lmax, stream=None):
    """tr_plan_widths: (width per slice, ids sorted by class, class counts)."""
    import torch
    _need(yhat, "yhat", torch.float32, 0)
    n = yhat.numel()
    width = torch.empty(n, dtype=torch.int32, device=yhat.device)
    ids = torch.empty(n, dtype=torch.int32, device=yhat.device)
    counts = torch.empty((lmax + 7) // 8, dtype=torch.int32, device=yhat.device)
    _check(load().tr_plan_widths(n, _ptr(yhat), int(oversample), int(lmax), _ptr(width),
                                 _ptr(ids), _ptr(counts), _stream(stream)))
    return width, ids, counts


def mlp_init(seed, device="cuda", stream=None):
    import torch
    prm = torch.empty(TR_MLP_PARAMS, dtype=torch.float32, device=device)
    _check(load().tr_mlp_init(_ptr(prm), int(seed), _stream(stream)))
    return prm


def mlp_forward(params, X, stream=None):
    import torch
    _need(params, "params", torch.float32, TR_MLP_PARAMS)
    _need(X, "X", torch.float32, 0)
    _need(X, "X", torch.float32, X.shape[0] * TR_MLP_FEATURES)
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(load().tr_mlp_forward(_ptr(params), _ptr(X), int(X.shape[0]), _ptr(y), _stream(stream)))
    return y


def mlp_loss_grad(params, X, y, under_weight, stream=None):
    import torch
    _need(params, "params", torch.float32, TR_MLP_PARAMS)
    _need(X, "X", torch.float32, 0)
    _need(X, "X", torch.float32, X.shape[0] * TR_MLP_FEATURES)
    _need(y, "y", torch.float32, X.shape[0])
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(load().tr_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(y), int(X.shape[0]),
                                   float(under_weight), _ptr(grad), _ptr(loss), _stream(stream)))
    return loss, grad


def mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    import torch
    _need(params, "params", torch.float32, 0)
    for t, name in ((grad, "grad"), (m, "m"), (v, "v")):
        _need(t, name, torch.float32, params.numel())
    _check(load().tr_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(params.numel()),
                              float(lr), float(beta1), float(beta2), float(eps), int(step),
                              _stream(stream)))


def mlp_train(params, X, y, batch, steps, lr, under_weight, seed, stream=None):
    """tr_mlp_train in place on `params`; returns the per-step loss (device)."""
    import torch
    _need(params, "params", torch.float32, TR_MLP_PARAMS)
    _need(X, "X", torch.float32, 0)
    _need(X, "X", torch.float32, X.shape[0] * TR_MLP_FEATURES)
    _need(y, "y", torch.float32, X.shape[0])
    hist = torch.empty(max(int(steps), 1), dtype=torch.float32, device=params.device)
    _check(load().tr_mlp_train(_ptr(params), _ptr(X), _ptr(y), int(X.shape[0]), int(batch),
                               int(steps), float(lr), float(under_weight), int(seed), _ptr(hist),
                               _stream(stream)))
    return hist[:int(steps)]


class Handle:
    """One recovery problem on the current CUDA device (tr_init ... tr_free)."""

    def __init__(self, observed, mask, dims, params=None, stream=None, **kw):
        import torch
        lib = load()
        dt = _float_dtype(observed, "observed")
        self.dtype = observed.dtype
        self.dims = tuple(int(d) for d in dims)
        N = 1
        for d in self.dims:
            N *= max(d, 0)
        _need(observed, "observed", observed.dtype, N)
        _need(mask, "mask", torch.uint8, N)
        prob = tr_problem()
        prob.order = len(self.dims)
        for i, d in enumerate(self.dims):
            prob.dims[i] = d
        prob.dtype = dt
        prob.observed = observed.data_ptr()
        prob.mask = mask.data_ptr()
        self._keep = (observed, mask)       # caller-owned buffers stay alive
        self.params = params if params is not None else default_params(**kw)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib.tr_init(ctypes.byref(h), ctypes.byref(prob), ctypes.byref(self.params),
                         ctypes.c_void_p(stream))
        _check(st, None)
        self.h = h
        n = 1
        for d in self.dims[2:]:
            n *= d
        self.shape = (n, self.dims[0], self.dims[1])

    def _new(self):
        import torch
        return torch.empty(self.shape, dtype=self.dtype, device="cuda")

    def _numel(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def _same(self, t, name, optional=False):
        """t must hold one tensor of this problem (N elements of its dtype)."""
        _need(t, name, self.dtype, self._numel(), optional=optional)

    def step(self, info=False):
        if info:
            si = tr_step_info()
            _check(load().tr_prox_step(self.h, ctypes.byref(si)), self.h)
            return si.as_dict()
        _check(load().tr_prox_step(self.h, None), self.h)
        return None

    def recover(self, L_out=None, check=True):
        si = tr_step_info()
        self._same(L_out, "L_out", optional=True)
        st = load().tr_recover(self.h, _ptr(L_out), ctypes.byref(si))
        if check:
            _check(st, self.h)
        return st, si.as_dict()

    def get_state(self):
        L, E, Y, Lam, G = (self._new() for _ in range(5))
        mu = ctypes.c_double()
        t = ctypes.c_int()
        _check(load().tr_get_state(self.h, _ptr(L), _ptr(E), _ptr(Y), _ptr(Lam), _ptr(G),
                                   ctypes.byref(mu), ctypes.byref(t)), self.h)
        return {"L": L, "E": E, "Y": Y, "Lam": Lam, "G": G, "mu": mu.value, "t": t.value}

    def get_L(self):
        """The low-rank iterate L only (completes a deferred step first)."""
        L = self._new()
        _check(load().tr_get_state(self.h, _ptr(L), None, None, None, None, None, None), self.h)
        return L

    def set_state(self, L, E, Y, Lam, G, mu, t):
        for x, name in ((L, "L"), (E, "E"), (Y, "Y"), (Lam, "Lam"), (G, "G")):
            self._same(x, name, optional=True)       # None: keep that tensor
        _check(load().tr_set_state(self.h, _ptr(L), _ptr(E), _ptr(Y), _ptr(Lam), _ptr(G),
                                   float(mu), int(t)), self.h)

    def transform_forward(self, src):
        self._same(src, "src")
        dst = self._new()
        _check(load().tr_transform_forward(self.h, _ptr(src), _ptr(dst)), self.h)
        return dst

    def transform_inverse(self, src):
        self._same(src, "src")
        dst = self._new()
        _check(load().tr_transform_inverse(self.h, _ptr(src), _ptr(dst)), self.h)
        return dst

    def slice_prox(self, Abar, tau, t, out=None):
        self._same(Abar, "Abar")
        Gbar = self._new() if out is None else out
        self._same(Gbar, "out")
        _check(load().tr_slice_prox(self.h, _ptr(Abar), _ptr(Gbar), float(tau), int(t)), self.h)
        return Gbar

    def slice_prox_tucker(self, Abar, tau, ranks, blocks, krylov, G1, G2, out=None,
                          factors=False):
        """tr_slice_prox_tucker: the shared-Tucker randomized prox of a
        transformed stack; returns Gbar (and F1, F2 when factors)."""
        import torch
        self._same(Abar, "Abar")
        Gbar = self._new() if out is None else out
        self._same(Gbar, "out")
        r1, r2 = ranks
        n, n1, n2 = self.shape
        # G1 is (n n2) x b1 and G2 (n r1) x b2, column-major
        _need(G1, "G1", self.dtype, n * n2 * max(int(blocks[0]), 0))
        _need(G2, "G2", self.dtype, n * max(int(r1), 0) * max(int(blocks[1]), 0))
        F1 = F2 = None
        if factors:
            F1 = torch.empty((r1, self.dims[0]), dtype=Abar.dtype, device=Abar.device)
            F2 = torch.empty((r2, self.dims[1]), dtype=Abar.dtype, device=Abar.device)
        _check(load().tr_slice_prox_tucker(self.h, _ptr(Abar), _ptr(Gbar), float(tau), int(r1),
                                           int(r2), int(blocks[0]), int(blocks[1]),
                                           int(krylov[0]), int(krylov[1]), _ptr(G1), _ptr(G2),
                                           _ptr(F1), _ptr(F2)), self.h)
        if factors:
            return Gbar, F1.T, F2.T      # column-major (n_k x r_k) as (r_k, n_k) row-major
        return Gbar

    def slice_stats(self):
        import numpy as np
        l = ctypes.c_int()
        _check(load().tr_last_slice_stats(self.h, None, None, ctypes.byref(l)), self.h)
        n = self.shape[0]
        sig = np.zeros(n * l.value)
        ranks = np.zeros(n, dtype=np.int32)
        _check(load().tr_last_slice_stats(
            self.h, sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            ranks.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), None), self.h)
        return sig.reshape(n, l.value), ranks

    def slice_widths(self):
        import numpy as np
        w = np.zeros(self.shape[0], dtype=np.int32)
        _check(load().tr_last_slice_widths(self.h, ctypes.c_void_p(w.ctypes.data)), self.h)
        return w

    def slice_features(self, tau, t):
        import torch
        out = torch.empty((self.shape[0], TR_MLP_FEATURES), dtype=torch.float32, device="cuda")
        _check(load().tr_slice_features(self.h, float(tau), int(t), _ptr(out)), self.h)
        return out

    def set_model(self, params):
        import numpy as np
        w = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        _check(load().tr_set_model(self.h, ctypes.c_void_p(w.ctypes.data), int(w.size)), self.h)

    def set_observed(self, observed, mask):
        """Point the handle at other observed data (same shape and dtype).
        The binding keeps the last two buffer pairs alive: a step enqueued on
        the previous pair may still be running on the handle's stream."""
        import torch
        self._same(observed, "observed")
        _need(mask, "mask", torch.uint8, self._numel())
        _check(load().tr_set_observed(self.h, _ptr(observed), _ptr(mask)), self.h)
        self._remember((observed, mask))

    def _remember(self, pair):
        self._keep_prev = getattr(self, "_keep", None)
        self._keep = pair

    def graph_mode(self, on=True):
        _check(load().tr_graph_mode(self.h, int(bool(on))), self.h)

    def read_residuals(self, out):
        """tr_read_residuals: enqueue the copy of the last step's residual
        maxima into `out`, a CPU float64 tensor of 10 entries (pinned for an
        asynchronous copy); valid after the handle's stream reaches it."""
        import torch
        if out.device.type != "cpu" or out.dtype != torch.float64 or out.numel() < 10 \
                or not out.is_contiguous():
            raise ValueError("out must be a contiguous CPU float64 tensor of 10 entries")
        _check(load().tr_read_residuals(self.h, _ptr(out)), self.h)
        return out

    def set_tube_tile(self, tp):
        _check(load().tr_set_tube_tile(self.h, int(tp)), self.h)

    def set_slice_groups(self, groups):
        _check(load().tr_set_slice_groups(self.h, int(groups)), self.h)

    def autotune(self, reps=5):
        """Returns (tube tile, slice groups) installed by the autotuner."""
        tile = ctypes.c_int()
        groups = ctypes.c_int()
        _check(load().tr_autotune(self.h, int(reps), ctypes.byref(tile), ctypes.byref(groups)),
               self.h)
        return tile.value, groups.value

    def profile_enable(self, max_steps):
        _check(load().tr_profile_enable(self.h, int(max_steps)), self.h)

    def profile_read(self):
        ms = (ctypes.c_double * 3)()
        steps = ctypes.c_int()
        _check(load().tr_profile_read(self.h, ms, ctypes.byref(steps)), self.h)
        return {"tube_forward": ms[0], "slice_pass": ms[1], "tube_inverse": ms[2],
                "steps": steps.value}

    def profile_slice_pass(self, Abar, tau, t, reps=5, out=None):
        """Mean device ms of every kernel of one eager slice pass
        (tr_profile_slice_pass): a list of (label, ms) in launch order."""
        self._same(Abar, "Abar")
        out = self._new() if out is None else out
        self._same(out, "out")
        cap = 40
        ms = (ctypes.c_double * cap)()
        names = (ctypes.c_char_p * cap)()
        cnt = ctypes.c_int()
        _check(load().tr_profile_slice_pass(self.h, _ptr(Abar), _ptr(out), float(tau), int(t),
                                            int(reps), ms, names, cap, ctypes.byref(cnt)),
               self.h)
        return [(names[k].decode(), ms[k]) for k in range(cnt.value)]

    def kernel_launches(self):
        c = ctypes.c_uint64()
        _check(load().tr_kernel_launches(self.h, ctypes.byref(c)), self.h)
        return int(c.value)

    def close(self):
        if getattr(self, "h", None):
            load().tr_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_batch(st):
    if st != TR_OK:
        msg = load().tr_batch_last_error()
        raise TrError(st, msg.decode() if msg else "")


class BorrowedHandle(Handle):
    """The handle of one problem of a Batch (owned by the batch)."""

    def __init__(self, h, dims, dtype, params, stream, owner=None, index=0):
        self.h = h
        self._owner = owner
        self._index = index
        self.dims = tuple(dims)
        self.dtype = dtype
        self.params = params
        self.stream = stream
        n = 1
        for d in self.dims[2:]:
            n *= d
        self.shape = (n, self.dims[0], self.dims[1])

    def _remember(self, pair):
        if self._owner is not None:
            self._owner._remember(self._index, pair)

    def close(self):
        self.h = None


class Batch:
    """Independent problems of any shapes stepped together (tr_batch_*)."""

    def __init__(self, problems, params, nstreams=8, stream=None):
        """problems: list of (observed, mask, dims) CUDA tensors; params: a
        tr_params per problem (or one for all)."""
        import torch
        lib = load()
        if isinstance(params, tr_params):
            params = [params] * len(problems)
        n = len(problems)
        probs = (tr_problem * n)()
        prms = (tr_params * n)()
        self._keep = []
        self._keep_prev = [None] * len(problems)
        self.meta = []
        for i, (obs, mask, dims) in enumerate(problems):
            N = 1
            for d in dims:
                N *= max(int(d), 0)
            _float_dtype(obs, "problems[%d] observed" % i)
            _need(obs, "problems[%d] observed" % i, obs.dtype, N)
            _need(mask, "problems[%d] mask" % i, torch.uint8, N)
            probs[i].order = len(dims)
            for k, d in enumerate(dims):
                probs[i].dims[k] = int(d)
            probs[i].dtype = {torch.float32: TR_F32, torch.float64: TR_F64}[obs.dtype]
            probs[i].observed = obs.data_ptr()
            probs[i].mask = mask.data_ptr()
            prms[i] = params[i]
            self._keep.append((obs, mask))
            self.meta.append((tuple(dims), obs.dtype, params[i]))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        b = ctypes.c_void_p()
        _check_batch(lib.tr_batch_create(ctypes.byref(b), n, ctypes.cast(probs, _P),
                                         ctypes.cast(prms, _P), int(nstreams),
                                         ctypes.c_void_p(stream)))
        self.b = b
        self.n = n

    def step(self, info=False):
        if info:
            infos = (tr_step_info * self.n)()
            _check_batch(load().tr_batch_step(self.b, ctypes.cast(infos, _P)))
            return [x.as_dict() for x in infos]
        _check_batch(load().tr_batch_step(self.b, None))
        return None

    def handle(self, i):
        h = ctypes.c_void_p()
        _check_batch(load().tr_batch_handle(self.b, int(i), ctypes.byref(h)))
        dims, dtype, prm = self.meta[i]
        return BorrowedHandle(h, dims, dtype, prm, self.stream, owner=self, index=int(i))

    def _remember(self, i, pair):
        # buffers of problem i set through its borrowed handle: keep the
        # current and the previous pair alive as long as the batch
        self._keep_prev[i] = self._keep[i]
        self._keep[i] = pair

    def graph_mode(self, on=True):
        _check_batch(load().tr_batch_graph_mode(self.b, int(bool(on))))

    def autotune(self, reps=3):
        """tr_batch_autotune: tune every problem's tube tile and slice split
        (between steps; values do not change)."""
        if int(reps) < 0:
            raise TrArgError("reps must be >= 0")
        _check_batch(load().tr_batch_autotune(self.b, int(reps)))

    def launches(self):
        c = ctypes.c_uint64()
        _check_batch(load().tr_batch_launches(self.b, ctypes.byref(c)))
        return int(c.value)

    def close(self):
        if getattr(self, "b", None):
            load().tr_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def onebit_params(**kw):
    """tr_onebit_params with the defaults of tr_onebit_default_params, then `kw`
    (`modes` may be a list of 1-based modes; `lambda` stands for lambda_)."""
    p = tr_onebit_params()
    load().tr_onebit_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "lambda":
            k = "lambda_"
        if k == "modes" and not isinstance(v, int):
            bits = 0
            for i in v:
                bits |= 1 << (int(i) - 1)
            v = bits
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class OneBit:
    """One-bit completion (tr_onebit_*): Alg. 6 on dithered one-bit samples."""

    def __init__(self, dims, idx, sign, params=None, dtype=None, stream=None, **kw):
        """dims: tensor sizes (order 3..8); idx: CUDA int64 flat face-slice
        indices of the m samples; sign: CUDA int8 signs (> 0: +1)."""
        import torch
        self.dtype = torch.float32 if dtype is None else dtype
        if self.dtype not in (torch.float32, torch.float64):
            raise TrArgError("dtype must be float32 or float64")
        m = idx.numel() if isinstance(idx, torch.Tensor) else 0
        _need(idx, "idx", torch.int64, max(m, 1))
        _need(sign, "sign", torch.int8, max(m, 1))
        self.dims = tuple(int(d) for d in dims)
        arr, self.N = _dims_array(self.dims)
        self.params = params if params is not None else onebit_params(**kw)
        self.nmodes = bin(int(self.params.modes)).count("1")
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        n = 1
        for d in self.dims[2:]:
            n *= d
        self.shape = (n, self.dims[0], self.dims[1])
        ob = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(256)
        dt = TR_F32 if self.dtype == torch.float32 else TR_F64
        st = load().tr_onebit_create(ctypes.byref(ob), dt, len(self.dims), arr, int(m), _ptr(idx),
                                     _ptr(sign), ctypes.byref(self.params),
                                     ctypes.c_void_p(self.stream), buf, 256)
        if st != TR_OK:
            raise TrError(st, buf.value.decode())
        self.ob = ob

    def _check(self, st):
        if st != TR_OK:
            msg = load().tr_onebit_last_error(self.ob)
            raise TrError(st, msg.decode() if msg else "")

    def step(self, rel=False):
        """One iteration; with rel=True returns the stop quantity (synchronises)."""
        if rel:
            r = ctypes.c_double()
            self._check(load().tr_onebit_step(self.ob, ctypes.byref(r)))
            return r.value
        self._check(load().tr_onebit_step(self.ob, None))
        return None

    def get_state(self):
        import torch
        L, Z, Y = (torch.empty(self.shape, dtype=self.dtype, device="cuda") for _ in range(3))
        G = torch.empty((self.nmodes,) + self.shape, dtype=self.dtype, device="cuda")
        Lam = torch.empty_like(G)
        mu = ctypes.c_double()
        t = ctypes.c_int()
        self._check(load().tr_onebit_get_state(self.ob, _ptr(L), _ptr(Z), _ptr(Y), _ptr(G),
                                               _ptr(Lam), ctypes.byref(mu), ctypes.byref(t)))
        return {"L": L, "Z": Z, "Y": Y, "G": G, "Lam": Lam, "mu": mu.value, "t": t.value}

    def set_state(self, L, Z, Y, G, Lam, mu, t):
        """G, Lam: (|Gamma|, n, n1, n2) tensors, modes ascending; None keeps one."""
        for x, name in ((L, "L"), (Z, "Z"), (Y, "Y")):
            _need(x, name, self.dtype, self.N, optional=True)
        for x, name in ((G, "G"), (Lam, "Lam")):
            _need(x, name, self.dtype, self.N * self.nmodes, optional=True)
        self._check(load().tr_onebit_set_state(self.ob, _ptr(L), _ptr(Z), _ptr(Y), _ptr(G),
                                               _ptr(Lam), float(mu), int(t)))

    def close(self):
        if getattr(self, "ob", None):
            load().tr_onebit_free(self.ob)
            self.ob = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctv_params(**kw):
    """tr_ctv_params with the defaults of tr_ctv_default_params, then `kw`
    (`modes` may be a list of 1-based modes; `lambda` stands for lambda_)."""
    p = tr_ctv_params()
    load().tr_ctv_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "lambda":
            k = "lambda_"
        if k == "modes" and not isinstance(v, int):
            bits = 0
            for i in v:
                bits |= 1 << (int(i) - 1)
            v = bits
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Ctv:
    """The gradient-domain prior (tr_ctv_*): Alg. 5 with a set of gradient
    directions on observed data M and mask (caller-owned CUDA tensors)."""

    def __init__(self, observed, mask, dims, params=None, stream=None, **kw):
        import torch
        dt = _float_dtype(observed, "observed")
        self.dtype = observed.dtype
        self.dims = tuple(int(d) for d in dims)
        arr, self.N = _dims_array(self.dims)
        _need(observed, "observed", observed.dtype, self.N)
        _need(mask, "mask", torch.uint8, self.N)
        self.params = params if params is not None else ctv_params(**kw)
        self.nmodes = bin(int(self.params.modes)).count("1")
        prob = tr_problem()
        prob.order = len(self.dims)
        for i, d in enumerate(self.dims):
            prob.dims[i] = d
        prob.dtype = dt
        prob.observed = observed.data_ptr()
        prob.mask = mask.data_ptr()
        self._keep = (observed, mask)
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        n = 1
        for d in self.dims[2:]:
            n *= d
        self.shape = (n, self.dims[0], self.dims[1])
        c = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(256)
        st = load().tr_ctv_create(ctypes.byref(c), ctypes.byref(prob), ctypes.byref(self.params),
                                  ctypes.c_void_p(self.stream), buf, 256)
        if st != TR_OK:
            raise TrError(st, buf.value.decode())
        self.c = c

    def _check(self, st):
        if st != TR_OK:
            msg = load().tr_ctv_last_error(self.c)
            raise TrError(st, msg.decode() if msg else "")

    def step(self, info=False):
        """One iteration; with info=True returns the five residuals (synchronises)."""
        if info:
            r = (ctypes.c_double * 5)()
            self._check(load().tr_ctv_step(self.c, r))
            return list(r)
        self._check(load().tr_ctv_step(self.c, None))
        return None

    def get_state(self):
        import torch
        L, E, Y = (torch.empty(self.shape, dtype=self.dtype, device="cuda") for _ in range(3))
        G = torch.empty((self.nmodes,) + self.shape, dtype=self.dtype, device="cuda")
        Lam = torch.empty_like(G)
        mu = ctypes.c_double()
        t = ctypes.c_int()
        self._check(load().tr_ctv_get_state(self.c, _ptr(L), _ptr(E), _ptr(Y), _ptr(G), _ptr(Lam),
                                            ctypes.byref(mu), ctypes.byref(t)))
        return {"L": L, "E": E, "Y": Y, "G": G, "Lam": Lam, "mu": mu.value, "t": t.value}

    def set_state(self, L, E, Y, G, Lam, mu, t):
        """G, Lam: (|Gamma|, n, n1, n2) tensors, modes ascending; None keeps one."""
        for x, name in ((L, "L"), (E, "E"), (Y, "Y")):
            _need(x, name, self.dtype, self.N, optional=True)
        for x, name in ((G, "G"), (Lam, "Lam")):
            _need(x, name, self.dtype, self.N * self.nmodes, optional=True)
        self._check(load().tr_ctv_set_state(self.c, _ptr(L), _ptr(E), _ptr(Y), _ptr(G), _ptr(Lam),
                                            float(mu), int(t)))

    def close(self):
        if getattr(self, "c", None):
            load().tr_ctv_free(self.c)
            self.c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
