"""Thin ctypes binding of the C ABI in include/tomo.h (argument marshalling only).

Every function here forwards to the function of the same name in
``_lib/libtomo.so``; all arithmetic runs in that library's CUDA kernels.
Device buffers are passed as torch CUDA tensors (their ``data_ptr()``), host
buffers as numpy arrays.  There is no fallback: if the library is missing or a
call fails, an exception is raised.
"""

import ctypes
import os

import numpy as np

from . import _build

TOMO_OK, TOMO_EINVAL, TOMO_ENOMEM, TOMO_ECUDA, TOMO_ETIMEOUT, TOMO_ERANGE = range(6)
FRAME_CONVERGED, FRAME_MAXIT, FRAME_BREAKDOWN, FRAME_FALLBACK_PLAIN_CG = range(4)
PRECISIONS = {"fp32": 0, "fp64": 1, "mixed": 2}


class tomo_gs(ctypes.Structure):
    _fields_ = [("alpha_x", ctypes.c_double), ("alpha_y", ctypes.c_double),
                ("height", ctypes.c_double), ("noise_sigma", ctypes.c_double)]


class tomo_config(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("obstruction", ctypes.c_double), ("n", ctypes.c_int),
                ("n_gs", ctypes.c_int), ("gs", ctypes.POINTER(tomo_gs)),
                ("n_layers", ctypes.c_int), ("layer_h", ctypes.POINTER(ctypes.c_double)),
                ("layer_frac", ctypes.POINTER(ctypes.c_double)),
                ("r0", ctypes.c_double), ("L0", ctypes.c_double),
                ("n_targets", ctypes.c_int), ("target_x", ctypes.POINTER(ctypes.c_double)),
                ("target_y", ctypes.POINTER(ctypes.c_double)),
                ("fft_P", ctypes.c_int), ("fft_Pcos", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("precond", ctypes.c_int), ("precond_floor", ctypes.c_double), ("mode_removal", ctypes.c_int),
                ("slope_model", ctypes.c_int), ("noise_cov", ctypes.POINTER(ctypes.c_double))]


class tomo_layout_info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in
                ("n", "n_gs", "n_vs", "N", "n_vphi", "n_targets", "n_layers", "P", "Pcos", "n_new", "max_batch")]


class tomo_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("check_every", ctypes.c_int), ("precond", ctypes.c_int),
                ("method", ctypes.c_int), ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("deadline_ms", ctypes.c_double), ("host_loop", ctypes.c_int)]


class tomo_frame_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("status", ctypes.c_int),
                ("pad_", ctypes.c_int), ("relres", ctypes.c_double)]


FRAME_INFO_DTYPE = np.dtype([("iters", np.int32), ("refinements", np.int32), ("status", np.int32),
                             ("pad_", np.int32), ("relres", np.float64)])

EXPORTS = ("tomo_create", "tomo_layout", "tomo_apply_css", "tomo_apply_css_noalloc", "tomo_apply_css_f64",
           "tomo_apply_cos",
           "tomo_solve", "tomo_solve_r0", "tomo_solve_host", "tomo_solve_f64", "tomo_autotune_result",
           "tomo_apply_cos_adjoint", "tomo_reconstructor", "tomo_apply_reconstructor", "tomo_launch_count", "tomo_set_kernel_timing",
           "tomo_apply_precond", "tomo_ws_init", "tomo_ws_param_count", "tomo_ws_set_params", "tomo_ws_get_params", "tomo_ws_apply",
           "tomo_ws_gradient", "tomo_ws_train_step",
           "tomo_get_kernel_timing", "tomo_destroy", "tomo_strerror")
KERNEL_NAMES = ("rows_fwd", "cols_mul", "rows_inv", "cg_scalars")

_lib = None


class TomoError(RuntimeError):
    """A call returned a status other than TOMO_OK.  For TOMO_ETIMEOUT of a solve
    the outputs were written anyway and ``info`` holds the per-frame results."""

    def __init__(self, fn, status, info=None):
        super().__init__(f"{fn} failed: {lib().tomo_strerror(status).decode()} (status {status})")
        self.status = status
        self.info = info


def lib(path=None):
    """Loads libtomo.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with __graft_entry__.build() "
                           "(or python -m paper_1806_07938_gb300._build)")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.tomo_create.argtypes = [ctypes.POINTER(tomo_config), vp, ctypes.POINTER(vp)]
    L.tomo_layout.argtypes = [vp, ctypes.POINTER(tomo_layout_info), vp, vp]
    L.tomo_apply_css.argtypes = [vp, vp, vp, i]
    L.tomo_apply_css_noalloc.argtypes = [vp, vp, vp, i]
    L.tomo_apply_css_f64.argtypes = [vp, vp, vp, i]
    L.tomo_apply_cos.argtypes = [vp, vp, vp, i]
    L.tomo_solve.argtypes = [vp, vp, i, ctypes.POINTER(tomo_solve_opts), vp, vp, vp]
    L.tomo_solve_host.argtypes = [vp, vp, i, ctypes.POINTER(tomo_solve_opts), vp, vp, vp]
    L.tomo_solve_f64.argtypes = [vp, vp, i, ctypes.POINTER(tomo_solve_opts), vp, vp]
    L.tomo_autotune_result.argtypes = [vp, vp, vp, i, ctypes.POINTER(i)]
    L.tomo_apply_cos_adjoint.argtypes = [vp, vp, vp, i]
    L.tomo_reconstructor.argtypes = [vp, i, ctypes.POINTER(tomo_solve_opts), vp, vp, vp]
    L.tomo_apply_reconstructor.argtypes = [vp, vp, i, vp, i, vp]
    L.tomo_solve_r0.argtypes = [vp, vp, i, vp, vp, ctypes.POINTER(tomo_solve_opts), vp, vp, vp]
    L.tomo_launch_count.argtypes = [vp]
    L.tomo_launch_count.restype = ctypes.c_longlong
    L.tomo_ws_init.argtypes = [vp, i, i, ctypes.c_float, ctypes.c_float, i, ctypes.c_float]
    L.tomo_apply_precond.argtypes = [vp, vp, vp, i]
    L.tomo_ws_param_count.argtypes = [vp, ctypes.POINTER(i)]
    L.tomo_ws_set_params.argtypes = [vp, vp, i]
    L.tomo_ws_get_params.argtypes = [vp, vp, i]
    L.tomo_ws_apply.argtypes = [vp, vp, vp, i]
    L.tomo_ws_gradient.argtypes = [vp, vp, vp, i, vp, ctypes.POINTER(d)]
    L.tomo_ws_train_step.argtypes = [vp, vp, vp, i, ctypes.c_float, ctypes.POINTER(d)]
    L.tomo_set_kernel_timing.argtypes = [vp, i]
    L.tomo_get_kernel_timing.argtypes = [vp, vp, vp, vp]
    L.tomo_destroy.argtypes = [vp]
    L.tomo_destroy.restype = None
    L.tomo_strerror.argtypes = [i]
    L.tomo_strerror.restype = ctypes.c_char_p
    for fn in EXPORTS:
        if fn not in ("tomo_launch_count", "tomo_destroy", "tomo_strerror"):
            getattr(L, fn).restype = i
    _lib = L
    return L


def _check(fn, status, info=None):
    if status != TOMO_OK:
        raise TomoError(fn, status, info)


def _dptr(t, dtype):
    """Device pointer of a contiguous CUDA tensor of the given torch dtype."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == dtype):
        raise TypeError(f"expected a contiguous CUDA tensor of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, dtype):
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"] and a.dtype == dtype):
        raise TypeError(f"expected a C-contiguous numpy array of {dtype}")
    return ctypes.c_void_p(a.ctypes.data)


def make_config(cfg, max_batch=1, fft_P=0, fft_Pcos=0, precond=False, precond_floor=0.0, mode_removal=False):
    """tomo_config from the plain-number system description; keeps its arrays alive.

    Keys of ``cfg``: D, obstruction, n, r0, L0; gs = [(alpha_x, alpha_y, H)] (H = 0
    for a natural star); noise_sigma = [sigma per guide star]; layers = [(h, fraction)];
    targets = [(beta_x, beta_y)]; optional slope_model ("hudgin" or "fried") and
    noise_cov ([n_gs][n][n][3] = s_xx, s_yy, s_xy per subaperture, elongated laser
    spots).  Angles in radians, lengths in metres."""
    n_gs = len(cfg["gs"])
    gs = (tomo_gs * n_gs)()
    for g, (ax, ay, H) in enumerate(cfg["gs"]):
        gs[g] = tomo_gs(ax, ay, H, float(cfg["noise_sigma"][g]))
    nl = len(cfg["layers"])
    lh = (ctypes.c_double * nl)(*[h for h, _ in cfg["layers"]])
    lf = (ctypes.c_double * nl)(*[f for _, f in cfg["layers"]])
    nt = len(cfg["targets"])
    tx = (ctypes.c_double * nt)(*[t[0] for t in cfg["targets"]])
    ty = (ctypes.c_double * nt)(*[t[1] for t in cfg["targets"]])
    ncov = cfg.get("noise_cov")
    if ncov is not None:
        ncov = np.ascontiguousarray(ncov, dtype=np.float64)
        if ncov.shape != (n_gs, cfg["n"], cfg["n"], 3):
            raise ValueError("noise_cov must be [n_gs][n][n][3]")
    c = tomo_config(cfg["D"], cfg["obstruction"], cfg["n"], n_gs, gs, nl, lh, lf, cfg["r0"], cfg["L0"],
                    nt, tx, ty, fft_P, fft_Pcos, max_batch, int(bool(precond)), float(precond_floor),
                    int(bool(mode_removal)), SLOPE_MODELS[cfg.get("slope_model", "hudgin")],
                    None if ncov is None else ncov.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    c._keep = (gs, lh, lf, tx, ty, ncov)
    return c


def tomo_create(cfg, stream=None, max_batch=1, fft_P=0, fft_Pcos=0, precond=False, precond_floor=0.0,
                mode_removal=False):
    """Creates a handle; ``stream`` is a torch.cuda.Stream or None (legacy default)."""
    L = lib()
    c = make_config(cfg, max_batch, fft_P, fft_Pcos, precond, precond_floor, mode_removal)
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
    _check("tomo_create", L.tomo_create(ctypes.byref(c), s, ctypes.byref(h)))
    return h


def tomo_autotune_result(h):
    """(sides, ms) the FFT-side autotuner timed; empty when not autotuned."""
    cnt = ctypes.c_int()
    _check("tomo_autotune_result", lib().tomo_autotune_result(h, None, None, 0, ctypes.byref(cnt)))
    sides = np.zeros(cnt.value, np.int32)
    ms = np.zeros(cnt.value, np.float64)
    if cnt.value:
        _check("tomo_autotune_result", lib().tomo_autotune_result(
            h, ctypes.c_void_p(sides.ctypes.data), ctypes.c_void_p(ms.ctypes.data), cnt.value, ctypes.byref(cnt)))
    return sides, ms


def tomo_layout(h):
    info = tomo_layout_info()
    _check("tomo_layout", lib().tomo_layout(h, ctypes.byref(info), None, None))
    sub = np.zeros((info.n, info.n), np.uint8)
    ph = np.zeros((info.n + 1, info.n + 1), np.uint8)
    _check("tomo_layout", lib().tomo_layout(h, ctypes.byref(info), ctypes.c_void_p(sub.ctypes.data),
                                            ctypes.c_void_p(ph.ctypes.data)))
    return info, sub.astype(bool), ph.astype(bool)


def tomo_apply_css(h, x, y, batch):
    import torch
    _check("tomo_apply_css", lib().tomo_apply_css(h, _dptr(x, torch.float32), _dptr(y, torch.float32), batch))


def tomo_apply_css_noalloc(h, x, y, batch):
    """tomo_apply_css without any device allocation (intermediates in the library's static buffer)."""
    import torch
    _check("tomo_apply_css_noalloc",
           lib().tomo_apply_css_noalloc(h, _dptr(x, torch.float32), _dptr(y, torch.float32), batch))


def tomo_apply_css_f64(h, x, y, batch):
    import torch
    _check("tomo_apply_css_f64", lib().tomo_apply_css_f64(h, _dptr(x, torch.float64), _dptr(y, torch.float64), batch))


def tomo_apply_cos(h, zeta, phase, batch):
    import torch
    _check("tomo_apply_cos", lib().tomo_apply_cos(h, _dptr(zeta, torch.float32), _dptr(phase, torch.float32), batch))


METHODS = {"cg": 0, "minres": 1, "block": 2}
SLOPE_MODELS = {"hudgin": 0, "fried": 1}


def solve_opts(tol=1e-4, max_iter=10000, max_refine=2, warm_start=0, check_every=32, precond=False, method="cg",
               precision="fp32", inner_tol=0.0, deadline_ms=0.0, host_loop=False):
    """warm_start: 0 cold, 1 zeta holds the guess, 2 the warm-start network's guess;
    precond: False / True (block-circulant M) or "learned" (flexible PCG with the
    network's correction of M r, plain PCG as fallback);
    method: "cg", "minres" or "block" (block CG over the frames of a chunk);
    precision: "fp32", "fp64" (tomo_solve_f64 only) or "mixed" (FP64 outer
    refinement around FP32 inner solves to inner_tol, 0 = automatic);
    deadline_ms > 0: the call's wall-clock budget (TOMO_ETIMEOUT when spent);
    host_loop: convergence checks on the host instead of the single graph launch."""
    precond = 2 if precond == "learned" else int(precond)
    return tomo_solve_opts(tol, max_iter, max_refine, int(warm_start), check_every, precond,
                           METHODS[method], PRECISIONS[precision], float(inner_tol), float(deadline_ms),
                           int(bool(host_loop)))


def tomo_solve(h, slopes, batch, opts, zeta, phase=None):
    """Device solve; returns the per-frame info as a numpy structured array."""
    import torch
    info = np.zeros(batch, FRAME_INFO_DTYPE)
    _check("tomo_solve", lib().tomo_solve(
        h, _dptr(slopes, torch.float32), batch, ctypes.byref(opts), _dptr(zeta, torch.float32),
        _dptr(phase, torch.float32) if phase is not None else None, ctypes.c_void_p(info.ctypes.data)), info)
    return info


def tomo_solve_f64(h, slopes, batch, opts, zeta):
    """Device solve on FP64 slopes and zeta (opts.precision "fp64" or "mixed");
    returns the per-frame info."""
    import torch
    info = np.zeros(batch, FRAME_INFO_DTYPE)
    _check("tomo_solve_f64", lib().tomo_solve_f64(
        h, _dptr(slopes, torch.float64), batch, ctypes.byref(opts), _dptr(zeta, torch.float64),
        ctypes.c_void_p(info.ctypes.data)), info)
    return info


def tomo_apply_cos_adjoint(h, phase, zeta, batch):
    import torch
    _check("tomo_apply_cos_adjoint", lib().tomo_apply_cos_adjoint(h, _dptr(phase, torch.float32),
                                                                  _dptr(zeta, torch.float32), batch))


def tomo_reconstructor(h, target, opts, R=None, n_rows=None, wfe=False):
    """Builds R [n_vphi][N] (device float32 tensor, or None) of one target.
    Returns the per-row info, and with wfe=True also the analytic error
    (rms [rad], trace term of Sigma_phi_phi, trace term of R Sigma_s_phi)."""
    import torch
    rows = R.shape[0] if R is not None else n_rows
    info = np.zeros(rows, FRAME_INFO_DTYPE)
    w = np.zeros(3, np.float64)
    _check("tomo_reconstructor", lib().tomo_reconstructor(
        h, target, ctypes.byref(opts), _dptr(R, torch.float32) if R is not None else None,
        ctypes.c_void_p(info.ctypes.data), ctypes.c_void_p(w.ctypes.data) if wfe else None))
    return (info, w) if wfe else info


def tomo_apply_reconstructor(h, R, slopes, batch, phase):
    import torch
    _check("tomo_apply_reconstructor", lib().tomo_apply_reconstructor(
        h, _dptr(R, torch.float32), R.shape[0], _dptr(slopes, torch.float32), batch, _dptr(phase, torch.float32)))


def tomo_solve_r0(h, slopes, batch, r0, opts, zeta, phase=None, noise_scale=None):
    """Device solve with a Fried parameter per frame (r0, noise_scale: host
    float64 arrays [batch]); returns the per-frame info."""
    import torch
    r0 = np.ascontiguousarray(r0, dtype=np.float64)
    ns = None if noise_scale is None else np.ascontiguousarray(noise_scale, dtype=np.float64)
    if r0.shape != (batch,) or (ns is not None and ns.shape != (batch,)):
        raise ValueError("r0 and noise_scale need one value per frame")
    info = np.zeros(batch, FRAME_INFO_DTYPE)
    _check("tomo_solve_r0", lib().tomo_solve_r0(
        h, _dptr(slopes, torch.float32), batch, _hptr(r0, np.float64),
        _hptr(ns, np.float64) if ns is not None else None, ctypes.byref(opts), _dptr(zeta, torch.float32),
        _dptr(phase, torch.float32) if phase is not None else None, ctypes.c_void_p(info.ctypes.data)), info)
    return info


def tomo_solve_host(h, slopes, batch, opts, zeta, phase=None):
    """Host-buffer solve (copies inside the call); returns the per-frame info."""
    info = np.zeros(batch, FRAME_INFO_DTYPE)
    _check("tomo_solve_host", lib().tomo_solve_host(
        h, _hptr(slopes, np.float32), batch, ctypes.byref(opts), _hptr(zeta, np.float32),
        _hptr(phase, np.float32) if phase is not None else None, ctypes.c_void_p(info.ctypes.data)), info)
    return info


def tomo_launch_count(h):
    return lib().tomo_launch_count(h)


def tomo_ws_init(h, hidden=32, max_batch=64, in_scale=1.0, out_scale=1.0, precond_input=False, pre_gain=1.0):
    _check("tomo_ws_init", lib().tomo_ws_init(h, hidden, max_batch, in_scale, out_scale, int(bool(precond_input)),
                                              pre_gain))


def tomo_apply_precond(h, x, y, batch):
    import torch
    _check("tomo_apply_precond", lib().tomo_apply_precond(h, _dptr(x, torch.float32), _dptr(y, torch.float32), batch))


def tomo_ws_param_count(h):
    c = ctypes.c_int(0)
    _check("tomo_ws_param_count", lib().tomo_ws_param_count(h, ctypes.byref(c)))
    return c.value


def tomo_ws_set_params(h, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check("tomo_ws_set_params", lib().tomo_ws_set_params(h, _hptr(p, np.float32), p.size))


def tomo_ws_get_params(h):
    p = np.zeros(tomo_ws_param_count(h), np.float32)
    _check("tomo_ws_get_params", lib().tomo_ws_get_params(h, _hptr(p, np.float32), p.size))
    return p


def tomo_ws_apply(h, slopes, zeta, batch):
    import torch
    _check("tomo_ws_apply", lib().tomo_ws_apply(h, _dptr(slopes, torch.float32), _dptr(zeta, torch.float32), batch))


def tomo_ws_gradient(h, slopes, target, batch):
    """Returns (flat parameter gradient, loss) of the supervised loss, without updating."""
    import torch
    g = np.zeros(tomo_ws_param_count(h), np.float32)
    loss = ctypes.c_double(0.0)
    _check("tomo_ws_gradient", lib().tomo_ws_gradient(h, _dptr(slopes, torch.float32), _dptr(target, torch.float32),
                                                      batch, _hptr(g, np.float32), ctypes.byref(loss)))
    return g, loss.value


def tomo_ws_train_step(h, slopes, target, batch, lr):
    import torch
    loss = ctypes.c_double(0.0)
    _check("tomo_ws_train_step", lib().tomo_ws_train_step(h, _dptr(slopes, torch.float32),
                                                          _dptr(target, torch.float32), batch, lr,
                                                          ctypes.byref(loss)))
    return loss.value


def tomo_set_kernel_timing(h, enable):
    _check("tomo_set_kernel_timing", lib().tomo_set_kernel_timing(h, int(bool(enable))))


def tomo_get_kernel_timing(h):
    """Returns ({kernel: total ms}, {kernel: launches}, frame_iterations)."""
    ms = np.zeros(len(KERNEL_NAMES), np.float64)
    n = np.zeros(len(KERNEL_NAMES), np.int64)
    fi = ctypes.c_longlong(0)
    _check("tomo_get_kernel_timing", lib().tomo_get_kernel_timing(
        h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(n.ctypes.data), ctypes.byref(fi)))
    return dict(zip(KERNEL_NAMES, ms.tolist())), dict(zip(KERNEL_NAMES, n.tolist())), fi.value


def tomo_destroy(h):
    if h:
        lib().tomo_destroy(h)


def tomo_strerror(status):
    return lib().tomo_strerror(status).decode()


def valid_slopes(full, mask):
    """Selects the valid subapertures (row-major) from full-grid slopes [..., gs, 2, n, n]
    into the ABI layout [..., N] (input marshalling; no arithmetic)."""
    lead = full.shape[:-4]
    return full[..., mask].reshape(*lead, -1)
