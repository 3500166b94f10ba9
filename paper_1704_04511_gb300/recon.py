"""Thin ctypes binding of include/recon.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards device pointers of
torch CUDA tensors; all arithmetic runs in librecon.so. Importing this module does not touch the
GPU; the first call that needs the library loads it and raises if it was not built
(`python -m paper_1704_04511_gb300.build`) -- there is no fallback path.

Tensor conventions: image series / k-space are torch.complex64 tensors of shape (T, P, Q)
(bfloat16 k-space: shape (T, P, Q, 2)); masks are torch.uint8 (T, P, Q); the Gram matrix is
torch.complex128 (s, s) stored column-major, i.e. the C array G[i + j*s] is tensor element
[j, i] of a row-major (s, s) tensor (use .T to read it as G[i, j]); S is complex64
(npair, P, Q); lags and summed diagonals are complex128 (npair, 2N1-1, 2N2-1).
Volumes (the *3 calls): series, k-space and masks (T, R, P, Q); filters (N1, N2, N3, M); S
(npair, R, P, Q); lags and summed diagonals (npair, 2N3-1, 2N1-1, 2N2-1).
"""

from __future__ import annotations

import ctypes
import os
import threading

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "librecon.so")

RECON_OK = 0
RECON_EINVAL = -1
RECON_ENOMEM = -2
RECON_ECUDA = -3
RECON_ENUMERIC = -4
RECON_ETIMEOUT = -5
RECON_EBUSY = -6
RECON_WEIGHT_AUTO = 0
RECON_WEIGHT_EIG = 1
RECON_VARIANT_PROPOSED = 0
RECON_VARIANT_GIRAF = 1
RECON_VARIANT_HLR_VOXEL = 2
RECON_VARIANT_DIRECT = 3

_ERR_NAMES = {RECON_EINVAL: "RECON_EINVAL", RECON_ENOMEM: "RECON_ENOMEM",
              RECON_ECUDA: "RECON_ECUDA", RECON_ENUMERIC: "RECON_ENUMERIC",
              RECON_ETIMEOUT: "RECON_ETIMEOUT", RECON_EBUSY: "RECON_EBUSY"}

EXPORTED = ("recon_create", "recon_destroy", "recon_last_error", "recon_bytes_needed",
            "recon_solve", "recon_adjoint", "recon_fft2", "recon_gram", "recon_weight",
            "recon_apply_normal", "recon_apply_w", "recon_cg", "recon_profile",
            "recon_profile_read", "recon_profile_name", "recon_gram_static",
            "recon_solve_batch", "recon_solve_batch_host", "recon_solve_many", "recon_set_option", "recon_submit", "recon_poll", "recon_t2fit",
            "recon_solve_coils", "recon_adjoint_coils", "recon_apply_normal_coils",
            "recon_bytes_needed3", "recon_solve3", "recon_adjoint3", "recon_fft3", "recon_gram3",
            "recon_weight3", "recon_apply_normal3", "recon_solve_variant", "recon_gram_variant",
            "recon_voxel_weight", "recon_weight_direct", "recon_apply_normal_variant",
            "recon_tile_cache", "recon_tile_choice", "recon_fft_schedule_choice")

PROF_KINDS = 13


class ReconError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class recon_dims(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("Q", ctypes.c_int), ("T", ctypes.c_int)]


class recon_filter(ctypes.Structure):
    _fields_ = [("N1", ctypes.c_int), ("N2", ctypes.c_int), ("M", ctypes.c_int)]


class recon_dims3(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("Q", ctypes.c_int), ("R", ctypes.c_int), ("T", ctypes.c_int)]


class recon_filter3(ctypes.Structure):
    _fields_ = [("N1", ctypes.c_int), ("N2", ctypes.c_int), ("N3", ctypes.c_int),
                ("M", ctypes.c_int)]


class recon_params(ctypes.Structure):
    _fields_ = [("irls", ctypes.c_int), ("cg", ctypes.c_int), ("lambda_", ctypes.c_double),
                ("p", ctypes.c_double), ("gamma", ctypes.c_double),
                ("eps0_frac", ctypes.c_double), ("kspace_bf16", ctypes.c_int),
                ("weight_method", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librecon.so (once) and declare the C signatures. Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_1704_04511_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(path)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        dims, filt = recon_dims, recon_filter
        dims3, filt3 = recon_dims3, recon_filter3
        sig = {
            "recon_create": (i, [ctypes.POINTER(vp), i, sz, vp]),
            "recon_destroy": (None, [vp]),
            "recon_last_error": (ctypes.c_char_p, [vp]),
            "recon_bytes_needed": (sz, [dims, filt, i]),
            "recon_solve": (i, [vp, dims, vp, vp, filt, ctypes.POINTER(recon_params), vp]),
            "recon_adjoint": (i, [vp, dims, vp, i, vp, vp]),
            "recon_fft2": (i, [vp, dims, vp, vp, i]),
            "recon_gram": (i, [vp, dims, filt, vp, vp, vp]),
            "recon_weight": (i, [vp, dims, filt, vp, d, d, i, vp, vp, vp, ctypes.POINTER(d)]),
            "recon_apply_normal": (i, [vp, dims, filt, vp, vp, d, vp, vp]),
            "recon_apply_w": (i, [vp, dims, filt, vp, vp, vp]),
            "recon_cg": (i, [vp, dims, filt, vp, vp, vp, d, vp, vp, i, ctypes.POINTER(d)]),
            "recon_profile": (i, [vp, ctypes.c_uint]),
            "recon_profile_read": (i, [vp, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]),
            "recon_profile_name": (ctypes.c_char_p, [i]),
            "recon_gram_static": (i, [dims, filt, vp, vp, vp, vp]),
            "recon_set_option": (i, [vp, i, i]),
            "recon_submit": (i, [vp, dims, vp, vp, filt, ctypes.POINTER(recon_params), vp,
                                 ctypes.POINTER(i)]),
            "recon_poll": (i, [vp, i, ctypes.POINTER(i)]),
            "recon_t2fit": (i, [vp, dims, vp, ctypes.POINTER(d), d, i, vp, vp]),
            "recon_solve_coils": (i, [vp, dims, vp, vp, vp, i, filt, ctypes.POINTER(recon_params),
                                      vp]),
            "recon_adjoint_coils": (i, [vp, dims, vp, vp, vp, i, vp]),
            "recon_apply_normal_coils": (i, [vp, dims, filt, vp, vp, i, vp, d, vp, vp]),
            "recon_solve_batch": (i, [vp, i, dims, ctypes.POINTER(vp), ctypes.POINTER(vp), filt,
                                      ctypes.POINTER(recon_params), ctypes.POINTER(vp)]),
            "recon_solve_batch_host": (i, [vp, i, dims, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           filt, ctypes.POINTER(recon_params), ctypes.POINTER(vp)]),
            "recon_solve_many": (i, [vp, i, ctypes.POINTER(dims), ctypes.POINTER(filt),
                                     ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(recon_params), ctypes.POINTER(vp)]),
            "recon_bytes_needed3": (sz, [dims3, filt3, i]),
            "recon_solve3": (i, [vp, dims3, vp, vp, filt3, ctypes.POINTER(recon_params), vp]),
            "recon_adjoint3": (i, [vp, dims3, vp, i, vp, vp]),
            "recon_fft3": (i, [vp, dims3, vp, vp, i]),
            "recon_gram3": (i, [vp, dims3, filt3, vp, vp, vp]),
            "recon_weight3": (i, [vp, dims3, filt3, vp, d, d, i, vp, vp, vp, ctypes.POINTER(d)]),
            "recon_apply_normal3": (i, [vp, dims3, filt3, vp, vp, d, vp, vp]),
            "recon_solve_variant": (i, [vp, dims, vp, vp, filt, ctypes.POINTER(recon_params), i,
                                        vp]),
            "recon_gram_variant": (i, [vp, dims, filt, i, vp, vp]),
            "recon_voxel_weight": (i, [vp, dims, i, vp, vp, d, vp, vp]),
            "recon_weight_direct": (i, [vp, dims, filt, vp, d, d, i, vp, ctypes.POINTER(d)]),
            "recon_apply_normal_variant": (i, [vp, dims, filt, i, vp, vp, d, vp, vp]),
            "recon_tile_cache": (i, [vp, ctypes.c_char_p]),
            "recon_tile_choice": (i, [vp, dims3, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
            "recon_fft_schedule_choice": (i, [vp, dims3, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(ctx, rc: int):
    if rc != RECON_OK:
        msg = load_library().recon_last_error(ctx).decode(errors="replace")
        raise ReconError(rc, msg)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dims(x) -> recon_dims:
    T, P, Q = x.shape[:3]
    return recon_dims(P=int(P), Q=int(Q), T=int(T))


def _filt(f) -> recon_filter:
    N1, N2, M = f
    return recon_filter(N1=int(N1), N2=int(N2), M=int(M))


# ------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ------------------------------------------------------------------------------------------

def recon_create(device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int | None = None):
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.recon_create(ctypes.byref(h), int(device), int(mem_budget_bytes),
                          ctypes.c_void_p(cuda_stream) if cuda_stream else None)
    if rc != RECON_OK:
        raise ReconError(rc, lib.recon_last_error(None).decode(errors="replace"))
    return h


def recon_destroy(ctx) -> None:
    if ctx:
        load_library().recon_destroy(ctx)


def recon_last_error(ctx) -> str:
    return load_library().recon_last_error(ctx).decode(errors="replace")


def recon_bytes_needed(shape, filt, kspace_bf16: bool = False) -> int:
    T, P, Q = shape
    return int(load_library().recon_bytes_needed(recon_dims(P=P, Q=Q, T=T), _filt(filt),
                                                  int(kspace_bf16)))


def recon_solve(ctx, kspace, masks, filt, lam: float, p: float, irls: int, cg: int,
                image_out, gamma: float = 1.4, eps0_frac: float = 0.01,
                weight_method: int = RECON_WEIGHT_AUTO) -> None:
    import torch
    bf16 = kspace.dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    _check(ctx, load_library().recon_solve(ctx, _dims(masks), _ptr(kspace), _ptr(masks),
                                           _filt(filt), ctypes.byref(prm), _ptr(image_out)))


def recon_solve_coils(ctx, kspace, masks, coils, filt, lam: float, p: float, irls: int, cg: int,
                      image_out, gamma: float = 1.4, eps0_frac: float = 0.01,
                      weight_method: int = RECON_WEIGHT_AUTO) -> None:
    """Multi-coil solve: kspace [Nc, T, P, Q] complex64, coils [Nc, P, Q] complex64."""
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=0,
                       weight_method=int(weight_method))
    _check(ctx, load_library().recon_solve_coils(ctx, _dims(masks), _ptr(kspace), _ptr(masks),
                                                 _ptr(coils), int(coils.shape[0]), _filt(filt),
                                                 ctypes.byref(prm), _ptr(image_out)))


def recon_adjoint_coils(ctx, kspace, masks, coils, x_out) -> None:
    _check(ctx, load_library().recon_adjoint_coils(ctx, _dims(masks), _ptr(kspace), _ptr(masks),
                                                   _ptr(coils), int(coils.shape[0]), _ptr(x_out)))


def recon_apply_normal_coils(ctx, masks, coils, filt, S, lam: float, x, y) -> None:
    _check(ctx, load_library().recon_apply_normal_coils(ctx, _dims(x), _filt(filt), _ptr(masks),
                                                        _ptr(coils), int(coils.shape[0]), _ptr(S),
                                                        float(lam), _ptr(x), _ptr(y)))


def recon_solve_batch(ctx, kspaces, masks_list, filt, lam: float, p: float, irls: int, cg: int,
                      image_outs, gamma: float = 1.4, eps0_frac: float = 0.01,
                      weight_method: int = RECON_WEIGHT_AUTO) -> None:
    """n independent problems of the same shape, solved concurrently (one stream each)."""
    import torch
    n = len(kspaces)
    if not (len(masks_list) == n == len(image_outs)):
        raise ValueError("kspaces, masks_list and image_outs must have the same length")
    bf16 = kspaces[0].dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    arr = ctypes.c_void_p * n
    kp = arr(*[_ptr(t) for t in kspaces])
    mp = arr(*[_ptr(t) for t in masks_list])
    op = arr(*[_ptr(t) for t in image_outs])
    _check(ctx, load_library().recon_solve_batch(ctx, int(n), _dims(masks_list[0]), kp, mp,
                                                 _filt(filt), ctypes.byref(prm), op))


def _host_ptr(t):
    if t.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def recon_solve_batch_host(ctx, kspaces, masks_list, filt, lam: float, p: float, irls: int,
                           cg: int, image_outs, gamma: float = 1.4, eps0_frac: float = 0.01,
                           weight_method: int = RECON_WEIGHT_AUTO) -> None:
    """recon_solve_batch on host tensors (pin them for overlapped copies); image_outs are host
    tensors that hold the results when the call returns."""
    import torch
    n = len(kspaces)
    if not (len(masks_list) == n == len(image_outs)):
        raise ValueError("kspaces, masks_list and image_outs must have the same length")
    bf16 = kspaces[0].dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    arr = ctypes.c_void_p * n
    kp = arr(*[_host_ptr(t) for t in kspaces])
    mp = arr(*[_host_ptr(t) for t in masks_list])
    op = arr(*[_host_ptr(t) for t in image_outs])
    _check(ctx, load_library().recon_solve_batch_host(ctx, int(n), _dims(masks_list[0]), kp, mp,
                                                      _filt(filt), ctypes.byref(prm), op))


def recon_solve_many(ctx, kspaces, masks_list, filts, lam: float, p: float, irls: int, cg: int,
                     image_outs, gamma: float = 1.4, eps0_frac: float = 0.01,
                     weight_method: int = RECON_WEIGHT_AUTO) -> None:
    """n problems of their own shapes and filters (shared parameters), solved as one batch."""
    import torch
    n = len(kspaces)
    if not (len(masks_list) == n == len(image_outs) == len(filts)):
        raise ValueError("kspaces, masks_list, filts and image_outs must have the same length")
    bf16 = kspaces[0].dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    arr = ctypes.c_void_p * n
    dims = (recon_dims * n)(*[_dims(m) for m in masks_list])
    filt = (recon_filter * n)(*[_filt(f) for f in filts])
    kp = arr(*[_ptr(t) for t in kspaces])
    mp = arr(*[_ptr(t) for t in masks_list])
    op = arr(*[_ptr(t) for t in image_outs])
    _check(ctx, load_library().recon_solve_many(ctx, int(n), dims, filt, kp, mp,
                                                ctypes.byref(prm), op))


RECON_OPT_GRAPHS = 1
RECON_OPT_AUTOTUNE = 3
RECON_OPT_INJECT_BARRIER_FAULT = 5
RECON_OPT_TEST_WITHHOLD_ARRIVAL = 6
RECON_OPT_BATCH_GROUP = 7
RECON_OPT_AUTOTUNE_FFT = 8
RECON_OPT_FFT_SCHEDULE = 9


def recon_tile_cache(ctx, path) -> None:
    """Read tuned column-tile choices from `path` and append new ones to it (None: stop)."""
    _check(ctx, load_library().recon_tile_cache(ctx, None if path is None else str(path).encode()))


def recon_tile_choice(ctx, shape, n_coils: int = 1):
    """(colC, depthC) the context uses for shape (T, P, Q) or (T, R, P, Q); 0 = not tuned."""
    if len(shape) == 3:
        T, P, Q = shape
        R = 1
    else:
        T, R, P, Q = shape
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, load_library().recon_tile_choice(ctx, recon_dims3(P=P, Q=Q, R=R, T=T), int(n_coils),
                                                 ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def recon_fft_schedule_choice(ctx, shape, n_coils: int = 1):
    """(colS, depthS) radix schedules the context uses for shape (T, P, Q) or (T, R, P, Q);
    -1 = not tuned."""
    if len(shape) == 3:
        T, P, Q = shape
        R = 1
    else:
        T, R, P, Q = shape
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, load_library().recon_fft_schedule_choice(ctx, recon_dims3(P=P, Q=Q, R=R, T=T),
                                                         int(n_coils), ctypes.byref(a),
                                                         ctypes.byref(b)))
    return a.value, b.value


def recon_set_option(ctx, option: int, value: int) -> None:
    _check(ctx, load_library().recon_set_option(ctx, int(option), int(value)))


def recon_submit(ctx, kspace, masks, filt, lam: float, p: float, irls: int, cg: int, image_out,
                 gamma: float = 1.4, eps0_frac: float = 0.01,
                 weight_method: int = RECON_WEIGHT_AUTO):
    """Queue one reconstruction; returns a ticket, or None when no slot / budget is free now."""
    import torch
    bf16 = kspace.dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    t = ctypes.c_int(0)
    rc = load_library().recon_submit(ctx, _dims(masks), _ptr(kspace), _ptr(masks), _filt(filt),
                                     ctypes.byref(prm), _ptr(image_out), ctypes.byref(t))
    if rc == RECON_EBUSY:
        return None
    _check(ctx, rc)
    return t.value


def recon_poll(ctx, ticket: int) -> bool:
    """True once the request finished (raises its error if it failed), False while it runs."""
    done = ctypes.c_int(0)
    rc = load_library().recon_poll(ctx, int(ticket), ctypes.byref(done))
    _check(ctx, rc)
    return bool(done.value)


def recon_adjoint(ctx, kspace, masks, x_out) -> None:
    import torch
    bf16 = kspace.dtype == torch.bfloat16
    _check(ctx, load_library().recon_adjoint(ctx, _dims(masks), _ptr(kspace), int(bf16),
                                             _ptr(masks), _ptr(x_out)))


def recon_fft2(ctx, x, y, inverse: bool = False) -> None:
    _check(ctx, load_library().recon_fft2(ctx, _dims(x), _ptr(x), _ptr(y), int(inverse)))


def recon_gram(ctx, x, filt, G_out, lags_out=None) -> None:
    _check(ctx, load_library().recon_gram(ctx, _dims(x), _filt(filt), _ptr(x), _ptr(G_out),
                                          _ptr(lags_out)))


def recon_gram_static(x, filt, G_out, lags_out=None, cuda_stream: int | None = None) -> None:
    """Gram matrix and lags as recon_gram, without a context and without allocating device
    memory (scratch in a fixed array inside the library; see include/recon.h)."""
    rc = load_library().recon_gram_static(_dims(x), _filt(filt), _ptr(x), _ptr(G_out),
                                           _ptr(lags_out),
                                           ctypes.c_void_p(cuda_stream) if cuda_stream else None)
    _check(None, rc)


def recon_weight(ctx, shape, filt, G_in, eps_in: float, p: float, S_out, dsum_out=None,
                 evals_out=None, method: int = RECON_WEIGHT_AUTO) -> float:
    T, P, Q = shape
    eps_used = ctypes.c_double(0.0)
    _check(ctx, load_library().recon_weight(ctx, recon_dims(P=P, Q=Q, T=T), _filt(filt),
                                            _ptr(G_in), float(eps_in), float(p), int(method),
                                            _ptr(S_out),
                                            _ptr(dsum_out), _ptr(evals_out),
                                            ctypes.byref(eps_used)))
    return eps_used.value


def recon_apply_normal(ctx, masks, filt, S, lam: float, x, y) -> None:
    _check(ctx, load_library().recon_apply_normal(ctx, _dims(x), _filt(filt), _ptr(masks), _ptr(S),
                                                  float(lam), _ptr(x), _ptr(y)))


def recon_apply_w(ctx, filt, S, x, y) -> None:
    _check(ctx, load_library().recon_apply_w(ctx, _dims(x), _filt(filt), _ptr(S), _ptr(x), _ptr(y)))


def recon_cg(ctx, masks, filt, S_old, S_new, lam: float, x, r, n_cg: int):
    hist = (ctypes.c_double * (n_cg + 1))()
    _check(ctx, load_library().recon_cg(ctx, _dims(x), _filt(filt), _ptr(masks), _ptr(S_old),
                                        _ptr(S_new), float(lam), _ptr(x), _ptr(r), int(n_cg), hist))
    return list(hist)


def recon_t2fit(ctx, x, times_ms, t2_out, amp_out=None, fg_frac: float = 0.1, n_gn: int = 20) -> None:
    """T2 (ms, NaN outside the foreground) and optionally amplitude maps of a [T, P, Q] series."""
    if len(times_ms) != x.shape[0]:
        raise ValueError("need one echo time per frame")
    t = (ctypes.c_double * len(times_ms))(*[float(v) for v in times_ms])
    _check(ctx, load_library().recon_t2fit(ctx, _dims(x), _ptr(x), t, float(fg_frac), int(n_gn),
                                           _ptr(t2_out), _ptr(amp_out)))


# ---- comparison methods (RECON_VARIANT_*) ----

def recon_solve_variant(ctx, kspace, masks, filt, lam: float, p: float, irls: int, cg: int,
                        image_out, variant: int, gamma: float = 1.4, eps0_frac: float = 0.01,
                        weight_method: int = RECON_WEIGHT_AUTO) -> None:
    import torch
    bf16 = kspace.dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    _check(ctx, load_library().recon_solve_variant(ctx, _dims(masks), _ptr(kspace), _ptr(masks),
                                                   _filt(filt), ctypes.byref(prm), int(variant),
                                                   _ptr(image_out)))


def recon_gram_variant(ctx, x, filt, variant: int, G_out) -> None:
    _check(ctx, load_library().recon_gram_variant(ctx, _dims(x), _filt(filt), int(variant),
                                                  _ptr(x), _ptr(G_out)))


def recon_voxel_weight(ctx, x, M: int, eps, p: float, S_out, lmax_out=None) -> None:
    """HLR-Voxel weight: eps (P, Q) float64 CUDA tensor, S_out (npair, P, Q) complex64."""
    _check(ctx, load_library().recon_voxel_weight(ctx, _dims(x), int(M), _ptr(x), _ptr(eps),
                                                  float(p), _ptr(S_out), _ptr(lmax_out)))


def recon_weight_direct(ctx, shape, filt, G_in, eps_in: float, p: float, H_out,
                        method: int = RECON_WEIGHT_AUTO) -> float:
    T, P, Q = shape
    eps_used = ctypes.c_double(0.0)
    _check(ctx, load_library().recon_weight_direct(ctx, recon_dims(P=P, Q=Q, T=T), _filt(filt),
                                                   _ptr(G_in), float(eps_in), float(p),
                                                   int(method), _ptr(H_out),
                                                   ctypes.byref(eps_used)))
    return eps_used.value


def recon_apply_normal_variant(ctx, masks, filt, variant: int, W, lam: float, x, y) -> None:
    _check(ctx, load_library().recon_apply_normal_variant(ctx, _dims(x), _filt(filt), int(variant),
                                                          _ptr(masks), _ptr(W), float(lam),
                                                          _ptr(x), _ptr(y)))


# ---- volumes (T, R, P, Q) ----

def _dims3(x) -> recon_dims3:
    T, R, P, Q = x.shape[:4]
    return recon_dims3(P=int(P), Q=int(Q), R=int(R), T=int(T))


def _filt3(f) -> recon_filter3:
    N1, N2, N3, M = f
    return recon_filter3(N1=int(N1), N2=int(N2), N3=int(N3), M=int(M))


def recon_bytes_needed3(shape, filt, kspace_bf16: bool = False) -> int:
    T, R, P, Q = shape
    return int(load_library().recon_bytes_needed3(recon_dims3(P=P, Q=Q, R=R, T=T), _filt3(filt),
                                                   int(kspace_bf16)))


def recon_solve3(ctx, kspace, masks, filt, lam: float, p: float, irls: int, cg: int,
                 image_out, gamma: float = 1.4, eps0_frac: float = 0.01,
                 weight_method: int = RECON_WEIGHT_AUTO) -> None:
    import torch
    bf16 = kspace.dtype == torch.bfloat16
    prm = recon_params(irls=int(irls), cg=int(cg), lambda_=float(lam), p=float(p),
                       gamma=float(gamma), eps0_frac=float(eps0_frac), kspace_bf16=int(bf16),
                       weight_method=int(weight_method))
    _check(ctx, load_library().recon_solve3(ctx, _dims3(masks), _ptr(kspace), _ptr(masks),
                                            _filt3(filt), ctypes.byref(prm), _ptr(image_out)))


def recon_adjoint3(ctx, kspace, masks, x_out) -> None:
    import torch
    bf16 = kspace.dtype == torch.bfloat16
    _check(ctx, load_library().recon_adjoint3(ctx, _dims3(masks), _ptr(kspace), int(bf16),
                                              _ptr(masks), _ptr(x_out)))


def recon_fft3(ctx, x, y, inverse: bool = False) -> None:
    _check(ctx, load_library().recon_fft3(ctx, _dims3(x), _ptr(x), _ptr(y), int(inverse)))


def recon_gram3(ctx, x, filt, G_out, lags_out=None) -> None:
    _check(ctx, load_library().recon_gram3(ctx, _dims3(x), _filt3(filt), _ptr(x), _ptr(G_out),
                                           _ptr(lags_out)))


def recon_weight3(ctx, shape, filt, G_in, eps_in: float, p: float, S_out, dsum_out=None,
                  evals_out=None, method: int = RECON_WEIGHT_AUTO) -> float:
    T, R, P, Q = shape
    eps_used = ctypes.c_double(0.0)
    _check(ctx, load_library().recon_weight3(ctx, recon_dims3(P=P, Q=Q, R=R, T=T), _filt3(filt),
                                             _ptr(G_in), float(eps_in), float(p), int(method),
                                             _ptr(S_out), _ptr(dsum_out), _ptr(evals_out),
                                             ctypes.byref(eps_used)))
    return eps_used.value


def recon_apply_normal3(ctx, masks, filt, S, lam: float, x, y) -> None:
    _check(ctx, load_library().recon_apply_normal3(ctx, _dims3(x), _filt3(filt), _ptr(masks),
                                                   _ptr(S), float(lam), _ptr(x), _ptr(y)))


PROF_ALL = (1 << 15) - 1


def recon_profile(ctx, kind_mask: int) -> None:
    """Time the launch classes whose bit is set (0 = off, PROF_ALL = all)."""
    _check(ctx, load_library().recon_profile(ctx, int(kind_mask) & PROF_ALL))


def recon_profile_read(ctx, kind: int):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(ctx, load_library().recon_profile_read(ctx, int(kind), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def recon_profile_name(kind: int) -> str:
    return load_library().recon_profile_name(int(kind)).decode()


# ------------------------------------------------------------------------------------------
# convenience wrapper
# ------------------------------------------------------------------------------------------

class Context:
    """Owns one recon context (device workspace, eigensolver handle, stream)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int | None = None):
        self.h = recon_create(device, mem_budget_bytes, cuda_stream)
        self.device = device

    def close(self):
        if self.h:
            recon_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, kspace, masks, filt, lam, p, irls, cg, gamma=1.4, eps0_frac=0.01, out=None,
              weight_method=RECON_WEIGHT_AUTO):
        import torch
        if out is None:
            out = torch.empty(tuple(masks.shape), dtype=torch.complex64, device=masks.device)
        recon_solve(self.h, kspace, masks, filt, lam, p, irls, cg, out, gamma, eps0_frac,
                    weight_method)
        return out
