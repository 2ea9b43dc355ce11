"""ctypes binding of libdehaze.so, one Python function per C entry point of
include/dehaze.h, with the same names.  Argument marshalling only: every step
of the method runs in the library's CUDA kernels.  Array arguments are device
pointers, given as torch tensors (their data_ptr()) or as integers.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libdehaze.so")

DH_OK = 0
DH_WDEGENERATE = 1
DH_WNOCONV = 2
DH_EINVAL = -1
DH_ENONFINITE = -2
DH_EWORKSPACE = -3
DH_ECUDA = -4
DH_ETIMEOUT = -5
DH_PRESET_PAPER = 0
DH_PRESET_STABLE = 1
DH_STORE_F32, DH_STORE_BF16, DH_STORE_F16, DH_STORE_BF16_F32, DH_STORE_F16_F32 = 0, 1, 2, 3, 4
DH_VAR_NO_ADAPTIVE, DH_VAR_NO_EDGE, DH_VAR_NO_NONLOCAL = 1, 2, 4
DH_BOUNDARY_REFLECT, DH_BOUNDARY_ZERO = 0, 1

# Every symbol include/dehaze.h declares.
EXPORTS = ("dh_params_default", "dh_strerror", "dh_version", "dh_workspace_bytes",
           "dh_dark_channel", "dh_atmospheric_light", "dh_transmission", "dh_fixed_point",
           "dh_dehaze", "dh_batch_workspace_bytes", "dh_dehaze_batch", "dh_sweep_variants", "dh_tune",
           "dh_tune_set", "dh_tune_get", "dh_unet_param_count", "dh_unet_workspace_bytes", "dh_unet_init",
           "dh_unet_forward", "dh_unet_backward", "dh_unet_adam", "dh_warm_start", "dh_warm_target",
           "dh_conv3x3_forward",
           "dh_conv3x3_backward_weights", "dh_dehaze_warm", "dh_atmospheric_light_noalloc",
           "dh_semi_implicit_workspace_bytes", "dh_semi_implicit", "dh_transmission_ws",
           "dh_selftest_bounded_wait", "dh_batch_net_workspace_bytes", "dh_dehaze_batch_warm")


class DhParams(ctypes.Structure):
    _fields_ = [
        ("patch", ctypes.c_int),
        ("topk_permille", ctypes.c_int),
        ("omega", ctypes.c_float),
        ("t0", ctypes.c_float),
        ("lambda0", ctypes.c_float),
        ("beta", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("sigma", ctypes.c_float),
        ("radius", ctypes.c_int),
        ("tau", ctypes.c_float),
        ("tol", ctypes.c_float),
        ("max_iter", ctypes.c_int),
        ("tb_depth", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("sweep_variant", ctypes.c_int),
        ("boundary", ctypes.c_int),
        ("dc_scales", ctypes.c_int),
        ("gf_radius", ctypes.c_int),
        ("gf_eps", ctypes.c_float),
    ]

    def replace(self, **kw) -> "DhParams":
        q = DhParams()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(self), ctypes.sizeof(self))
        for k, v in kw.items():
            setattr(q, k, v)
        return q

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class DhReport(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("n_iter", ctypes.c_int),
        ("rho", ctypes.c_float * 3),
        ("A", ctypes.c_float * 3),
        ("a_index", ctypes.c_longlong),
        ("ms", ctypes.c_float),
        ("ms_loop", ctypes.c_float),
        ("launches", ctypes.c_int),
    ]


class DhTuneResult(ctypes.Structure):
    _fields_ = [
        ("best", ctypes.c_int),
        ("count", ctypes.c_int),
        ("variant", ctypes.c_int * 64),
        ("us_per_iter", ctypes.c_float * 64),
    ]


class DhImage(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_void_p),
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("u0", ctypes.c_void_p),
        ("J", ctypes.c_void_p),
        ("u", ctypes.c_void_p),
        ("t", ctypes.c_void_p),
        ("A", ctypes.c_void_p),
    ]


_lock = threading.Lock()
_lib = None


def lib(build_if_missing: bool = True):
    """Loads libdehaze.so, building it first when it is missing or stale.
    Raises when it cannot be built: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build

        if build_if_missing:
            _build.build()
        if not os.path.exists(SO):
            raise RuntimeError(f"CUDA library not built: {SO} is missing")
        L = ctypes.CDLL(SO)
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        PP = ctypes.POINTER(DhParams)
        PR = ctypes.POINTER(DhReport)
        sig = {
            "dh_params_default": ([PP, I], I),
            "dh_strerror": ([I], ctypes.c_char_p),
            "dh_version": ([], I),
            "dh_workspace_bytes": ([I, I, PP], S),
            "dh_dark_channel": ([P, I, I, I, P, P, P], I),
            "dh_atmospheric_light": ([P, P, I, I, I, P, P, P, S, P, PR], I),
            "dh_transmission": ([P, P, I, I, PP, P, P, P, P, P], I),
            "dh_fixed_point": ([P, P, P, I, I, PP, P, P, S, P, PR], I),
            "dh_dehaze": ([P, I, I, PP, P, P, P, P, P, P, S, P, PR], I),
            "dh_atmospheric_light_noalloc": ([P, P, I, I, I, P, P, P], I),
            "dh_batch_workspace_bytes": ([I, ctypes.POINTER(DhImage), PP], S),
            "dh_dehaze_batch": ([I, ctypes.POINTER(DhImage), PP, P, S, P, PR], I),
            "dh_sweep_variants": ([], I),
            "dh_tune": ([P, P, P, I, I, PP, I, P, S, P, ctypes.POINTER(DhTuneResult)], I),
            "dh_tune_set": ([I, I, I, I], I),
            "dh_tune_get": ([I, I, I], I),
            "dh_unet_param_count": ([I], S),
            "dh_unet_workspace_bytes": ([I, I, I, I, I], S),
            "dh_unet_init": ([P, I, ctypes.c_ulonglong, P], I),
            "dh_unet_forward": ([P, I, P, P, P, P, I, I, I, P, P, S, P], I),
            "dh_unet_backward": ([P, I, P, P, P, P, P, I, I, I, P, P, P, S, P], I),
            "dh_unet_adam": ([P, P, P, P, S, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, I, P], I),
            "dh_warm_start": ([P, P, I, I, P, P], I),
            "dh_warm_target": ([P, P, I, I, P, P], I),
            "dh_conv3x3_forward": ([P, I, I, I, I, I, P, P, I, I, P, I, P], I),
            "dh_conv3x3_backward_weights": ([P, I, I, P, I, I, I, I, I, P, P, P, S, P], I),
            "dh_dehaze_warm": ([P, I, P, I, I, PP, P, P, P, P, P, S, P, S, P, PR], I),
            "dh_batch_net_workspace_bytes": ([I, I, ctypes.POINTER(DhImage)], S),
            "dh_dehaze_batch_warm": ([P, I, I, ctypes.POINTER(DhImage), PP, P, S, P, S, P, PR], I),
            "dh_semi_implicit_workspace_bytes": ([I, I], S),
            "dh_transmission_ws": ([P, P, I, I, PP, P, P, P, P, P, S, P], I),
            "dh_selftest_bounded_wait": ([ctypes.c_longlong, P], I),
            "dh_semi_implicit": ([P, P, P, P, I, I, PP, ctypes.c_float, I, P, P, P, S, P, PR], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _p(x):
    """Device pointer of a tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ref(x):
    return None if x is None else ctypes.byref(x)


def dh_params_default(preset: int = DH_PRESET_PAPER) -> DhParams:
    p = DhParams()
    rc = lib().dh_params_default(ctypes.byref(p), preset)
    if rc != DH_OK:
        raise ValueError(dh_strerror(rc))
    return p


def dh_strerror(status: int) -> str:
    return lib().dh_strerror(status).decode()


def dh_version() -> int:
    return lib().dh_version()


def dh_workspace_bytes(H: int, W: int, p: DhParams | None = None) -> int:
    return lib().dh_workspace_bytes(H, W, _ref(p))


def dh_dark_channel(I, H, W, patch, A, out, stream=None) -> int:
    return lib().dh_dark_channel(_p(I), H, W, patch, _p(A), _p(out), _stream(stream))


def dh_atmospheric_light(I, dc, H, W, topk_permille, A_out, index_out, workspace, workspace_bytes,
                         stream=None, report: DhReport | None = None) -> int:
    return lib().dh_atmospheric_light(_p(I), _p(dc), H, W, topk_permille, _p(A_out), _p(index_out),
                                      _p(workspace), workspace_bytes, _stream(stream), _ref(report))


def dh_transmission(I, A, H, W, p: DhParams, td, t, lam, Phi, stream=None) -> int:
    return lib().dh_transmission(_p(I), _p(A), H, W, ctypes.byref(p), _p(td), _p(t), _p(lam), _p(Phi),
                                 _stream(stream))


def dh_transmission_ws(I, A, H, W, p: DhParams, td, t, lam, Phi, workspace, workspace_bytes, stream=None) -> int:
    return lib().dh_transmission_ws(_p(I), _p(A), H, W, ctypes.byref(p), _p(td), _p(t), _p(lam), _p(Phi),
                                    _p(workspace), workspace_bytes, _stream(stream))


def dh_fixed_point(u, Phi, lam, H, W, p: DhParams, rho_hist, workspace, workspace_bytes, stream=None,
                   report: DhReport | None = None) -> int:
    return lib().dh_fixed_point(_p(u), _p(Phi), _p(lam), H, W, ctypes.byref(p), _p(rho_hist),
                                _p(workspace), workspace_bytes, _stream(stream), _ref(report))


def dh_semi_implicit_workspace_bytes(H: int, W: int) -> int:
    return lib().dh_semi_implicit_workspace_bytes(H, W)


def dh_semi_implicit(u, u_lo, Phi, lam, H, W, p: DhParams, step, cg_iters, rho_hist, J, workspace,
                     workspace_bytes, stream=None, report: DhReport | None = None) -> int:
    return lib().dh_semi_implicit(_p(u), _p(u_lo), _p(Phi), _p(lam), H, W, ctypes.byref(p), float(step),
                                  int(cg_iters), _p(rho_hist), _p(J), _p(workspace), workspace_bytes,
                                  _stream(stream), _ref(report))


def dh_dehaze(I, H, W, p: DhParams, u0, J, u, t, A, workspace, workspace_bytes, stream=None,
              report: DhReport | None = None) -> int:
    return lib().dh_dehaze(_p(I), H, W, ctypes.byref(p), _p(u0), _p(J), _p(u), _p(t), _p(A),
                           _p(workspace), workspace_bytes, _stream(stream), _ref(report))


def dh_atmospheric_light_noalloc(I, dc, H, W, topk_permille, A_out, index_out, stream=None) -> int:
    """dh_atmospheric_light with the library's fixed device scratch array in
    place of a caller workspace (for callers that may not allocate)."""
    return lib().dh_atmospheric_light_noalloc(_p(I), _p(dc), H, W, topk_permille, _p(A_out), _p(index_out),
                                              _stream(stream))


def dh_image(I, H, W, u0, J, u, t, A) -> DhImage:
    return DhImage(_p(I), H, W, _p(u0), _p(J), _p(u), _p(t), _p(A))


def dh_batch_workspace_bytes(n, imgs, p: DhParams) -> int:
    arr = (DhImage * n)(*imgs)
    return lib().dh_batch_workspace_bytes(n, arr, ctypes.byref(p))


def dh_dehaze_batch(n, imgs, p: DhParams, workspace, workspace_bytes, stream=None, reports=None) -> int:
    """imgs: sequence of DhImage; reports: ctypes array of n DhReport or None."""
    arr = (DhImage * n)(*imgs)
    return lib().dh_dehaze_batch(n, arr, ctypes.byref(p), _p(workspace), workspace_bytes, _stream(stream), reports)


def dh_sweep_variants() -> int:
    return lib().dh_sweep_variants()


def dh_tune(Phi, lam, u_scratch, H, W, p: DhParams, iters, workspace, workspace_bytes, stream=None,
            out: DhTuneResult | None = None) -> int:
    return lib().dh_tune(_p(Phi), _p(lam), _p(u_scratch), H, W, ctypes.byref(p), iters, _p(workspace),
                         workspace_bytes, _stream(stream), _ref(out))


def dh_tune_set(H, W, storage, variant) -> int:
    return lib().dh_tune_set(H, W, storage, variant)


def dh_tune_get(H, W, storage) -> int:
    return lib().dh_tune_get(H, W, storage)


def dh_unet_param_count(base) -> int:
    return lib().dh_unet_param_count(base)


def dh_unet_workspace_bytes(base, N, H, W, train) -> int:
    return lib().dh_unet_workspace_bytes(base, N, H, W, train)


def dh_unet_init(params, base, seed, stream=None) -> int:
    return lib().dh_unet_init(_p(params), base, seed, _stream(stream))


def dh_unet_forward(params, base, I, t, A, Phi, N, H, W, y, workspace, workspace_bytes, stream=None) -> int:
    return lib().dh_unet_forward(_p(params), base, _p(I), _p(t), _p(A), _p(Phi), N, H, W, _p(y), _p(workspace),
                                 workspace_bytes, _stream(stream))


def dh_unet_backward(params, base, I, t, A, Phi, target, N, H, W, grads, loss, workspace, workspace_bytes,
                     stream=None) -> int:
    return lib().dh_unet_backward(_p(params), base, _p(I), _p(t), _p(A), _p(Phi), _p(target), N, H, W, _p(grads),
                                  _p(loss), _p(workspace), workspace_bytes, _stream(stream))


def dh_unet_adam(params, grads, m, v, n, lr, beta1, beta2, eps, step, stream=None) -> int:
    return lib().dh_unet_adam(_p(params), _p(grads), _p(m), _p(v), n, lr, beta1, beta2, eps, step, _stream(stream))


def dh_warm_start(y, lam, H, W, u0, stream=None) -> int:
    return lib().dh_warm_start(_p(y), _p(lam), H, W, _p(u0), _stream(stream))


def dh_warm_target(u, lam, H, W, y, stream=None) -> int:
    return lib().dh_warm_target(_p(u), _p(lam), H, W, _p(y), _stream(stream))


def dh_conv3x3_forward(x, ldx, C, N, H, W, w, bias, Cout, relu, y, ldy, stream=None) -> int:
    return lib().dh_conv3x3_forward(_p(x), ldx, C, N, H, W, _p(w), _p(bias), Cout, relu, _p(y), ldy, _stream(stream))


def dh_conv3x3_backward_weights(x, ldx, C, dy, lddy, Cout, N, H, W, dw, db, scratch, scratch_bytes,
                                stream=None) -> int:
    return lib().dh_conv3x3_backward_weights(_p(x), ldx, C, _p(dy), lddy, Cout, N, H, W, _p(dw), _p(db),
                                             _p(scratch), scratch_bytes, _stream(stream))


def dh_dehaze_warm(params, base, I, H, W, p: DhParams, J, u, t, A, workspace, workspace_bytes, net_workspace,
                   net_workspace_bytes, stream=None, report: DhReport | None = None) -> int:
    return lib().dh_dehaze_warm(_p(params), base, _p(I), H, W, ctypes.byref(p), _p(J), _p(u), _p(t), _p(A),
                                _p(workspace), workspace_bytes, _p(net_workspace), net_workspace_bytes,
                                _stream(stream), _ref(report))


def dh_batch_net_workspace_bytes(base, n, imgs) -> int:
    arr = (DhImage * n)(*imgs)
    return lib().dh_batch_net_workspace_bytes(base, n, arr)


def dh_dehaze_batch_warm(params, base, n, imgs, p: DhParams, workspace, workspace_bytes, net_workspace,
                         net_workspace_bytes, stream=None, reports=None) -> int:
    """dh_dehaze_batch with the network's u0 for every image; reports: ctypes
    array of n DhReport or None."""
    arr = (DhImage * n)(*imgs)
    return lib().dh_dehaze_batch_warm(_p(params), base, n, arr, ctypes.byref(p), _p(workspace), workspace_bytes,
                                      _p(net_workspace), net_workspace_bytes, _stream(stream), reports)


def dh_selftest_bounded_wait(limit_cycles: int, stream=None) -> int:
    return lib().dh_selftest_bounded_wait(int(limit_cycles), _stream(stream))
