"""Python binding of libvfisv.so, the GB300 Milne-Eddington Stokes inversion.

Argument marshalling only: every step of synthesis and inversion runs in the
library's CUDA kernels.  Functions carry the C-ABI names of ``include/vfisv.h``
and accept numpy arrays (host memory, staged by the library) or torch tensors
(device memory, used in place, asynchronous on the current torch stream).
Importing this module does not load the library; the first call does, and
raises if ``libvfisv.so`` has not been built (``python -m
paper_0901_2702_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "vfisv_create", "vfisv_destroy", "vfisv_synth", "vfisv_invert", "vfisv_check",
    "vfisv_counters",
    "vfisv_strerror", "vfisv_config_default", "vfisv_nn_init", "vfisv_nn_train",
    "vfisv_nn_grad", "vfisv_nn_infer", "vfisv_invert_nn", "vfisv_graph_begin", "vfisv_graph_end",
    "vfisv_graph_launch", "vfisv_graph_kernels", "vfisv_graph_destroy", "vfisv_autotune",
    "vfisv_set_pipeline_chunks", "vfisv_set_sm_limit", "vfisv_set_launch_shape", "vfisv_voigt",
    "vfisv_limb_weights", "vfisv_restart_models", "vfisv_init_models", "vfisv_invert_batch",
    "VfisvError",
    "library_path",
    "load",
    "NN_NBLOB", "NN_NTRAIN",
]

NN_NIN, NN_NHID, NN_NOUT = 24, 256, 11
NN_NTRAIN, NN_NBLOB = 140811, 140879

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libvfisv.so")
_lib = None

VFISV_OK = 0
PIX_CONVERGED, PIX_MAXITER, PIX_STALLED, PIX_BAD_INPUT, PIX_NAN_STATE = range(5)


class VfisvError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {vfisv_strerror(code)} ({code})")
        self.code = code


class vfisv_line(ctypes.Structure):
    _fields_ = [("lambda0_A", ctypes.c_double), ("geff", ctypes.c_double), ("mu", ctypes.c_double)]


class vfisv_config(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("free_mask", ctypes.c_uint32),
                ("conv_rtol", ctypes.c_double), ("conv_eps", ctypes.c_double),
                ("eps0", ctypes.c_double), ("restarts", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("hess_reuse", ctypes.c_double),
                ("wfa_pol", ctypes.c_double), ("fast_solve", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libvfisv.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libvfisv.so not built: {_LIB_PATH} is missing; run "
                           "__graft_entry__.build() or python -m paper_0901_2702_gb300.build")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.vfisv_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    lib.vfisv_create.restype = ctypes.c_int
    lib.vfisv_destroy.argtypes = [P]
    lib.vfisv_destroy.restype = None
    lib.vfisv_config_default.argtypes = [ctypes.POINTER(vfisv_config)]
    lib.vfisv_config_default.restype = None
    lib.vfisv_strerror.argtypes = [ctypes.c_int]
    lib.vfisv_strerror.restype = ctypes.c_char_p
    lib.vfisv_check.argtypes = [P, P]
    lib.vfisv_check.restype = ctypes.c_int
    lib.vfisv_synth.argtypes = [P, P, I64, P, I32, P, I32, ctypes.POINTER(vfisv_line), P, P]
    lib.vfisv_synth.restype = ctypes.c_int
    lib.vfisv_invert.argtypes = [P, P, P, I32, P, I32, P, I32, ctypes.POINTER(vfisv_line), P,
                                 ctypes.POINTER(vfisv_config), I64, P, P, P, P, P, P]
    lib.vfisv_invert.restype = ctypes.c_int
    U64 = ctypes.c_uint64
    lib.vfisv_nn_init.argtypes = [P, P, P, P, I64, U64, P]
    lib.vfisv_nn_init.restype = ctypes.c_int
    lib.vfisv_nn_train.argtypes = [P, P, P, P, I64, I32, I32, ctypes.c_float, U64, P, P]
    lib.vfisv_nn_train.restype = ctypes.c_int
    lib.vfisv_nn_grad.argtypes = [P, P, P, P, I64, P, P, P]
    lib.vfisv_nn_grad.restype = ctypes.c_int
    lib.vfisv_nn_infer.argtypes = [P, P, P, I64, ctypes.POINTER(vfisv_line), P, P, P, P]
    lib.vfisv_nn_infer.restype = ctypes.c_int
    lib.vfisv_invert_nn.argtypes = [P, P, P, P, I32, P, I32, P, I32, ctypes.POINTER(vfisv_line),
                                    ctypes.POINTER(vfisv_config), ctypes.POINTER(vfisv_config),
                                    ctypes.c_double, I32, ctypes.c_double, I64, P, P, P, P, P,
                                    P, P]
    lib.vfisv_invert_nn.restype = ctypes.c_int
    lib.vfisv_counters.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64), I32]
    lib.vfisv_counters.restype = ctypes.c_int
    lib.vfisv_noalloc_check.argtypes = [P]
    lib.vfisv_noalloc_check.restype = ctypes.c_int
    lib.vfisv_graph_begin.argtypes = [P, P]
    lib.vfisv_graph_begin.restype = ctypes.c_int
    lib.vfisv_graph_end.argtypes = [P, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.vfisv_graph_end.restype = ctypes.c_int
    lib.vfisv_graph_launch.argtypes = [P, P]
    lib.vfisv_graph_launch.restype = ctypes.c_int
    lib.vfisv_set_sm_limit.argtypes = [P, I32]
    lib.vfisv_set_sm_limit.restype = ctypes.c_int
    lib.vfisv_set_pipeline_chunks.argtypes = [P, I32]
    lib.vfisv_set_pipeline_chunks.restype = ctypes.c_int
    lib.vfisv_graph_kernels.argtypes = [P, ctypes.POINTER(I64)]
    lib.vfisv_graph_kernels.restype = ctypes.c_int
    lib.vfisv_graph_destroy.argtypes = [P]
    lib.vfisv_graph_destroy.restype = None
    lib.vfisv_autotune.argtypes = [P, P, P, I32, P, I32, P, I32, ctypes.POINTER(vfisv_line),
                                   ctypes.POINTER(vfisv_config), I64, ctypes.POINTER(I32),
                                   ctypes.POINTER(I32), P, P]
    lib.vfisv_autotune.restype = ctypes.c_int
    lib.vfisv_set_launch_shape.argtypes = [P, I32, I32]
    lib.vfisv_set_launch_shape.restype = ctypes.c_int
    lib.vfisv_voigt.argtypes = [P, P, P, I64, I32, P, P, P]
    lib.vfisv_voigt.restype = ctypes.c_int
    lib.vfisv_limb_weights.argtypes = [P, P, P, I64, I32, ctypes.c_float, P, P, P]
    lib.vfisv_limb_weights.restype = ctypes.c_int
    lib.vfisv_invert_batch.argtypes = [P, P, P, P, I32, P, I32, P, I32,
                                       ctypes.POINTER(vfisv_line), P, ctypes.POINTER(vfisv_config),
                                       P, P, P, P, P, P, P]
    lib.vfisv_invert_batch.restype = ctypes.c_int
    lib.vfisv_init_models.argtypes = [P, P, I64, P, I32, P, I32, ctypes.POINTER(vfisv_line), P,
                                      P, P]
    lib.vfisv_init_models.restype = ctypes.c_int
    lib.vfisv_restart_models.argtypes = [P, P, I64, I64, I32, ctypes.c_uint32, U64, P, P]
    lib.vfisv_restart_models.restype = ctypes.c_int
    _lib = lib
    return lib


def vfisv_strerror(code: int) -> str:
    try:
        return load().vfisv_strerror(int(code)).decode()
    except RuntimeError:
        return f"error {code}"


def _check(code, where):
    if code != VFISV_OK:
        raise VfisvError(code, where)


class Handle:
    """Owns a vfisv_handle (workspaces, work queue, constants) on one device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.vfisv_create(ctypes.byref(h), int(device)), "vfisv_create")
        self.ptr = h
        self.device = int(device)

    def close(self):
        if getattr(self, "ptr", None):
            self._lib.vfisv_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vfisv_create(device: int = 0) -> Handle:
    return Handle(device)


def vfisv_destroy(h: Handle) -> None:
    h.close()


def vfisv_config_default(**overrides) -> vfisv_config:
    c = vfisv_config()
    load().vfisv_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def _line(line) -> vfisv_line:
    if isinstance(line, vfisv_line):
        return line
    return vfisv_line(float(line["lambda0_A"]), float(line["geff"]), float(line.get("mu", 1.0)))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keep-alive object) of a C-contiguous array of `dtype`."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def _stream(ref, stream):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if _is_torch(ref) and ref.is_cuda:
        import torch
        return torch.cuda.current_stream(ref.device).cuda_stream
    return 0


def _empty(ref, shape, dtype):
    if _is_torch(ref):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


def vfisv_check(h: Handle, stream=None) -> None:
    _check(load().vfisv_check(h.ptr, ctypes.c_void_p(_stream(None, stream))), "vfisv_check")


def vfisv_counters(h: Handle, stream=None, reset: bool = False) -> dict:
    """Work of the handle's filter-position LM launches: fused passes,
    accepted trials, pixels retired and wavelength points evaluated since
    creation or the last reset."""
    c = (ctypes.c_uint64 * 4)()
    _check(load().vfisv_counters(h.ptr, ctypes.c_void_p(_stream(None, stream)), c,
                                 int(bool(reset))), "vfisv_counters")
    return {"passes": int(c[0]), "accepted": int(c[1]), "retired": int(c[2]),
            "points": int(c[3])}


def vfisv_synth(h: Handle, params, filters, wl_mA, line, stokes=None, stream=None):
    """Filtered Stokes vector [npix, 4, nfilt] of models params [npix, 10]."""
    npix = int(params.shape[0])
    nfilt, nlam = int(filters.shape[0]), int(filters.shape[1])
    if stokes is None:
        stokes = _empty(params, (npix, 4, nfilt), np.float32)
    pp, k1 = _ptr(params, np.float32)
    fp, k2 = _ptr(filters, np.float32)
    wp, k3 = _ptr(wl_mA, np.float32)
    sp, k4 = _ptr(stokes, np.float32)
    ln = _line(line)
    rc = load().vfisv_synth(h.ptr, pp, npix, fp, nfilt, wp, nlam, ctypes.byref(ln), sp,
                            ctypes.c_void_p(_stream(params, stream)))
    _check(rc, "vfisv_synth")
    if k4 is not stokes and not _is_torch(stokes):
        stokes[...] = k4
    return stokes


def vfisv_invert(h: Handle, obs, weights, filters, wl_mA, line, init=None, config=None,
                 want_cov=True, out=None, stream=None):
    """Levenberg-Marquardt inversion of obs [npix, 4*nfilt] (or [npix, 4, nfilt]).

    weights: [npix, 4*nfilt] per pixel or [4*nfilt] for all pixels (w^2/sigma^2).
    Returns dict(params, chi2, iters, status, cov) in the memory kind of obs.
    """
    npix = int(obs.shape[0])
    nfilt, nlam = int(filters.shape[0]), int(filters.shape[1])
    per_pixel = 1 if (len(weights.shape) >= 2 and int(weights.shape[0]) == npix and
                      int(np.prod(weights.shape)) == npix * 4 * nfilt) else 0
    cfg = config if isinstance(config, vfisv_config) else vfisv_config_default(**(config or {}))
    if out is None:
        out = {"params": _empty(obs, (npix, 10), np.float32),
               "chi2": _empty(obs, (npix,), np.float32),
               "iters": _empty(obs, (npix,), np.int32),
               "status": _empty(obs, (npix,), np.int32),
               "cov": _empty(obs, (npix, 10, 10), np.float32) if want_cov else None}
    op, k1 = _ptr(obs, np.float32)
    wp, k2 = _ptr(weights, np.float32)
    fp, k3 = _ptr(filters, np.float32)
    lp, k4 = _ptr(wl_mA, np.float32)
    ip, k5 = _ptr(init, np.float32)
    pp, k6 = _ptr(out["params"], np.float32)
    cp, k7 = _ptr(out["chi2"], np.float32)
    tp, k8 = _ptr(out["iters"], np.int32)
    sp, k9 = _ptr(out["status"], np.int32)
    vp, k10 = _ptr(out.get("cov"), np.float32)
    ln = _line(line)
    rc = load().vfisv_invert(h.ptr, op, wp, per_pixel, fp, nfilt, lp, nlam, ctypes.byref(ln), ip,
                             ctypes.byref(cfg), npix, pp, cp, tp, sp, vp,
                             ctypes.c_void_p(_stream(obs, stream)))
    _check(rc, "vfisv_invert")
    for key, k in (("params", k6), ("chi2", k7), ("iters", k8), ("status", k9), ("cov", k10)):
        dst = out.get(key)
        if dst is not None and not _is_torch(dst) and k is not dst:
            dst[...] = k
    return out


def _out(ref, given, shape, dtype):
    return given if given is not None else _empty(ref, shape, dtype)


def vfisv_nn_init(h: Handle, obs, params, seed: int = 0, blob=None, stream=None):
    """Fresh network blob: random weights and the training set's statistics."""
    n = int(obs.shape[0])
    blob = _out(obs, blob, (NN_NBLOB,), np.float32)
    bp, kb = _ptr(blob, np.float32)
    op, k1 = _ptr(obs, np.float32)
    pp, k2 = _ptr(params, np.float32)
    _check(load().vfisv_nn_init(h.ptr, bp, op, pp, n, int(seed),
                                ctypes.c_void_p(_stream(obs, stream))), "vfisv_nn_init")
    if not _is_torch(blob) and kb is not blob:
        blob[...] = kb
    return blob


def vfisv_nn_train(h: Handle, blob, obs, params, batch: int = 8192, epochs: int = 1,
                   lr0: float = 1e-3, seed: int = 0, want_loss: bool = True, stream=None):
    """Train the blob in place (Adam, cosine decay); returns the per-step loss."""
    n = int(obs.shape[0])
    steps = (n // batch) * epochs
    loss = _empty(obs, (max(steps, 1),), np.float32) if want_loss else None
    bp, kb = _ptr(blob, np.float32)
    op, k1 = _ptr(obs, np.float32)
    pp, k2 = _ptr(params, np.float32)
    lp, kl = _ptr(loss, np.float32)
    _check(load().vfisv_nn_train(h.ptr, bp, op, pp, n, int(batch), int(epochs), float(lr0),
                                 int(seed), lp, ctypes.c_void_p(_stream(obs, stream))),
           "vfisv_nn_train")
    if not _is_torch(blob) and kb is not blob:
        blob[...] = kb
    if loss is not None and not _is_torch(loss) and kl is not loss:
        loss[...] = kl
    return loss[:steps] if loss is not None else None


def vfisv_nn_grad(h: Handle, blob, obs, params, stream=None):
    """(loss, gradient[NN_NTRAIN]) of one batch."""
    n = int(obs.shape[0])
    grad = _empty(obs, (NN_NTRAIN,), np.float32)
    loss = _empty(obs, (1,), np.float32)
    bp, kb = _ptr(blob, np.float32)
    op, k1 = _ptr(obs, np.float32)
    pp, k2 = _ptr(params, np.float32)
    gp, kg = _ptr(grad, np.float32)
    lp, kl = _ptr(loss, np.float32)
    _check(load().vfisv_nn_grad(h.ptr, bp, op, pp, n, gp, lp,
                                ctypes.c_void_p(_stream(obs, stream))), "vfisv_nn_grad")
    return loss, grad


def vfisv_nn_infer(h: Handle, blob, obs, line, want_conf=True, want_raw=False, init=None,
                   stream=None):
    """Initial models [npix, 10] (and confidence / raw outputs) from the network;
    ``init`` may be a preallocated output (needed inside a graph capture)."""
    n = int(obs.shape[0])
    init = _empty(obs, (n, 10), np.float32) if init is None else init
    conf = _empty(obs, (n,), np.float32) if want_conf else None
    raw = _empty(obs, (n, NN_NOUT), np.float32) if want_raw else None
    bp, kb = _ptr(blob, np.float32)
    op, k1 = _ptr(obs, np.float32)
    ip, ki = _ptr(init, np.float32)
    cp, kc = _ptr(conf, np.float32)
    rp, kr = _ptr(raw, np.float32)
    ln = _line(line)
    _check(load().vfisv_nn_infer(h.ptr, bp, op, n, ctypes.byref(ln), ip, cp, rp,
                                 ctypes.c_void_p(_stream(obs, stream))), "vfisv_nn_infer")
    for dst, k in ((init, ki), (conf, kc), (raw, kr)):
        if dst is not None and not _is_torch(dst) and k is not dst:
            dst[...] = k
    return {"init": init, "conf": conf, "raw": raw}


def vfisv_invert_nn(h: Handle, blob, obs, weights, filters, wl_mA, line, config_nn=None,
                    config_plain=None, chi2_flag: float = 3.0, flag_unconverged: bool = True,
                    conf_route: float = float("inf"), want_cov=True, out=None, stream=None):
    """Mixed inversion: network guess + LM, plain LM re-inversion of flagged pixels
    (chi2 > chi2_flag, and with flag_unconverged also those that did not converge);
    pixels whose confidence output exceeds ``conf_route`` go to plain LM directly."""
    npix = int(obs.shape[0])
    nfilt, nlam = int(filters.shape[0]), int(filters.shape[1])
    per_pixel = 1 if (len(weights.shape) >= 2 and int(weights.shape[0]) == npix and
                      int(np.prod(weights.shape)) == npix * 4 * nfilt) else 0
    cn = config_nn if isinstance(config_nn, vfisv_config) else \
        vfisv_config_default(**({"max_iter": 20} | (config_nn or {})))
    cp_ = config_plain if isinstance(config_plain, vfisv_config) else \
        vfisv_config_default(**(config_plain or {}))
    if out is None:
        out = {"params": _empty(obs, (npix, 10), np.float32),
               "chi2": _empty(obs, (npix,), np.float32),
               "iters": _empty(obs, (npix,), np.int32),
               "status": _empty(obs, (npix,), np.int32),
               "cov": _empty(obs, (npix, 10, 10), np.float32) if want_cov else None,
               "flagged": _empty(obs, (npix,), np.int32)}
    ptrs = [_ptr(x, np.float32) for x in (blob, obs, weights, filters, wl_mA)]
    outs = [(k, _ptr(out.get(k), np.int32 if k in ("iters", "status", "flagged") else np.float32))
            for k in ("params", "chi2", "iters", "status", "cov", "flagged")]
    ln = _line(line)
    rc = load().vfisv_invert_nn(h.ptr, ptrs[0][0], ptrs[1][0], ptrs[2][0], per_pixel, ptrs[3][0],
                                nfilt, ptrs[4][0], nlam, ctypes.byref(ln), ctypes.byref(cn),
                                ctypes.byref(cp_), float(chi2_flag), int(bool(flag_unconverged)),
                                float(conf_route), npix,
                                *[p for _, (p, _k) in outs],
                                ctypes.c_void_p(_stream(obs, stream)))
    _check(rc, "vfisv_invert_nn")
    for key, (_, k) in outs:
        dst = out.get(key)
        if dst is not None and not _is_torch(dst) and k is not dst:
            dst[...] = k
    return out


class Graph:
    """An instantiated CUDA graph of captured vfisv_* calls."""

    def __init__(self, ptr):
        self.ptr = ptr

    def launch(self, stream):
        vfisv_graph_launch(self, stream)

    def kernels(self) -> int:
        """Kernel launches one replay performs."""
        return vfisv_graph_kernels(self)

    def close(self):
        if getattr(self, "ptr", None):
            load().vfisv_graph_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vfisv_graph_begin(h: Handle, stream) -> None:
    _check(load().vfisv_graph_begin(h.ptr, ctypes.c_void_p(_stream(None, stream))),
           "vfisv_graph_begin")


def vfisv_graph_end(h: Handle, stream) -> Graph:
    g = ctypes.c_void_p()
    _check(load().vfisv_graph_end(h.ptr, ctypes.c_void_p(_stream(None, stream)), ctypes.byref(g)),
           "vfisv_graph_end")
    return Graph(g)


def vfisv_graph_launch(g: Graph, stream) -> None:
    _check(load().vfisv_graph_launch(g.ptr, ctypes.c_void_p(_stream(None, stream))),
           "vfisv_graph_launch")


def vfisv_set_sm_limit(h: Handle, nsm: int) -> None:
    """At most `nsm` SMs for this handle's persistent launches (0: all)."""
    _check(load().vfisv_set_sm_limit(h.ptr, int(nsm)), "vfisv_set_sm_limit")


def vfisv_set_pipeline_chunks(h: Handle, chunks: int) -> None:
    """Host-buffer pipeline depth of this handle (0: stage the whole map)."""
    _check(load().vfisv_set_pipeline_chunks(h.ptr, int(chunks)), "vfisv_set_pipeline_chunks")


def vfisv_graph_kernels(g: Graph) -> int:
    n = ctypes.c_int64(0)
    _check(load().vfisv_graph_kernels(g.ptr, ctypes.byref(n)), "vfisv_graph_kernels")
    return int(n.value)


def vfisv_graph_destroy(g: Graph) -> None:
    g.close()


def vfisv_autotune(h: Handle, obs, weights, filters, wl_mA, line, config=None, stream=None):
    """Pick the LM kernel's launch shape on a sample; returns (threads per CTA,
    threads per pixel, [ms x 10]: threads-per-pixel-major over 64/128/256 x
    1/2/4, then the warp-specialised 384 x 1)."""
    npix = int(obs.shape[0])
    nfilt, nlam = int(filters.shape[0]), int(filters.shape[1])
    per_pixel = 1 if (len(weights.shape) >= 2 and int(weights.shape[0]) == npix) else 0
    cfg = config if isinstance(config, vfisv_config) else vfisv_config_default(**(config or {}))
    ptrs = [_ptr(x, np.float32) for x in (obs, weights, filters, wl_mA)]
    best, tpp = ctypes.c_int32(), ctypes.c_int32()
    ms = np.zeros(10, np.float32)
    ln = _line(line)
    _check(load().vfisv_autotune(h.ptr, ptrs[0][0], ptrs[1][0], per_pixel, ptrs[2][0], nfilt,
                                 ptrs[3][0], nlam, ctypes.byref(ln), ctypes.byref(cfg), npix,
                                 ctypes.byref(best), ctypes.byref(tpp), ms.ctypes.data,
                                 ctypes.c_void_p(_stream(obs, stream))), "vfisv_autotune")
    return int(best.value), int(tpp.value), ms.tolist()


def vfisv_set_launch_shape(h: Handle, block: int, tpp: int = 1) -> None:
    """Threads per CTA (64, 128, 256) and per pixel (1, 2, 4) of the LM kernel,
    or 384 x 1: the warp-specialised kernel."""
    _check(load().vfisv_set_launch_shape(h.ptr, int(block), int(tpp)), "vfisv_set_launch_shape")


VOIGT_RATIONAL, VOIGT_TAYLOR1, VOIGT_TAYLOR2 = 0, 1, 2


def vfisv_voigt(h: Handle, a, u, method: int = VOIGT_RATIONAL, stream=None):
    """(H, F) = (Re, Im) w(u + i a) for arrays a, u of equal length."""
    n = int(np.prod(u.shape))
    H = _empty(u, tuple(u.shape), np.float32)
    F = _empty(u, tuple(u.shape), np.float32)
    ap, k1 = _ptr(a, np.float32)
    up_, k2 = _ptr(u, np.float32)
    hp, kh = _ptr(H, np.float32)
    fp, kf = _ptr(F, np.float32)
    _check(load().vfisv_voigt(h.ptr, ap, up_, n, int(method), hp, fp,
                              ctypes.c_void_p(_stream(u, stream))), "vfisv_voigt")
    for dst, k in ((H, kh), (F, kf)):
        if not _is_torch(dst) and k is not dst:
            dst[...] = k
    return H, F


def vfisv_limb_weights(h: Handle, obs, mu, ic0: float, sigma4, stream=None):
    """Eq. 14 weights (w^2/sigma^2) [npix, 4*nfilt] for observables obs [npix, 4*nfilt]."""
    npix = int(obs.shape[0])
    nobs = int(np.prod(obs.shape)) // max(npix, 1)
    out = _empty(obs, (npix, nobs), np.float32)
    op, k1 = _ptr(obs, np.float32)
    mp, k2 = _ptr(mu, np.float32)
    outp, ko = _ptr(out, np.float32)
    s4 = np.ascontiguousarray(sigma4, dtype=np.float32)
    _check(load().vfisv_limb_weights(h.ptr, op, mp, npix, nobs // 4, float(ic0), s4.ctypes.data,
                                     outp, ctypes.c_void_p(_stream(obs, stream))),
           "vfisv_limb_weights")
    if not _is_torch(out) and ko is not out:
        out[...] = ko
    return out


def vfisv_restart_models(h: Handle, models, pixel0: int, k: int, free_mask: int = 0x1FF,
                         seed: int = 0, stream=None):
    """Restart number k of pixels pixel0.. from models [n, 10] (Sec. 4.2)."""
    n = int(models.shape[0])
    out = _empty(models, (n, 10), np.float32)
    mp, k1 = _ptr(models, np.float32)
    outp, ko = _ptr(out, np.float32)
    _check(load().vfisv_restart_models(h.ptr, mp, n, int(pixel0), int(k), int(free_mask),
                                       int(seed), outp, ctypes.c_void_p(_stream(models, stream))),
           "vfisv_restart_models")
    if not _is_torch(out) and ko is not out:
        out[...] = ko
    return out


def vfisv_init_models(h: Handle, obs, filters, wl_mA, line, want_pol: bool = True, stream=None):
    """Initial models [npix, 10] from the filtergrams (weak field, wing
    azimuth, centre-of-gravity velocity) and the polarisation level [npix]."""
    npix = int(obs.shape[0])
    nfilt, nlam = int(filters.shape[0]), int(filters.shape[1])
    out = {"init": _empty(obs, (npix, 10), np.float32),
           "pol": _empty(obs, (npix,), np.float32) if want_pol else None}
    op, k1 = _ptr(obs, np.float32)
    fp, k2 = _ptr(filters, np.float32)
    lp, k3 = _ptr(wl_mA, np.float32)
    ip, k4 = _ptr(out["init"], np.float32)
    pp, k5 = _ptr(out["pol"], np.float32)
    ln = _line(line)
    _check(load().vfisv_init_models(h.ptr, op, npix, fp, nfilt, lp, nlam, ctypes.byref(ln), ip, pp,
                                    ctypes.c_void_p(_stream(obs, stream))), "vfisv_init_models")
    for key, k in (("init", k4), ("pol", k5)):
        dst = out.get(key)
        if dst is not None and not _is_torch(dst) and k is not dst:
            dst[...] = k
    return out


def vfisv_invert_batch(h: Handle, obs, weights, map_off, filters, wl_mA, line, init=None,
                       config=None, want_cov=True, want_latency=True, out=None, stream=None):
    """Inversion of many concatenated maps in one launch.

    obs [npix, 4*nfilt]; weights [nmaps, 4*nfilt] per map; map_off host
    int64 [nmaps+1] prefix offsets.  Returns vfisv_invert's outputs plus
    latency_ms [nmaps] (per-map completion time from the call's start)."""
    off = np.ascontiguousarray(np.asarray(map_off, dtype=np.int64))
    nmaps = int(off.size - 1)
    npix = int(off[-1])
    nfilt, nlam = int(filters.shape[0]), int(filters.shape[1])
    cfg = config if isinstance(config, vfisv_config) else vfisv_config_default(**(config or {}))
    if out is None:
        out = {"params": _empty(obs, (npix, 10), np.float32),
               "chi2": _empty(obs, (npix,), np.float32),
               "iters": _empty(obs, (npix,), np.int32),
               "status": _empty(obs, (npix,), np.int32),
               "cov": _empty(obs, (npix, 10, 10), np.float32) if want_cov else None,
               "latency_ms": _empty(obs, (nmaps,), np.float32) if want_latency else None}
    op, k1 = _ptr(obs, np.float32)
    wp, k2 = _ptr(weights, np.float32)
    fp, k3 = _ptr(filters, np.float32)
    lp, k4 = _ptr(wl_mA, np.float32)
    ip, k5 = _ptr(init, np.float32)
    keys = ("params", "chi2", "iters", "status", "cov", "latency_ms")
    dts = (np.float32, np.float32, np.int32, np.int32, np.float32, np.float32)
    ptrs = [_ptr(out.get(k), dt) for k, dt in zip(keys, dts)]
    ln = _line(line)
    _check(load().vfisv_invert_batch(h.ptr, op, wp, off.ctypes.data, nmaps, fp, nfilt, lp, nlam,
                                     ctypes.byref(ln), ip, ctypes.byref(cfg),
                                     *[p for p, _ in ptrs],
                                     ctypes.c_void_p(_stream(obs, stream))),
           "vfisv_invert_batch")
    for k, (_, kk) in zip(keys, ptrs):
        dst = out.get(k)
        if dst is not None and not _is_torch(dst) and kk is not dst:
            dst[...] = kk
    return out
