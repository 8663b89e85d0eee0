"""Thin ctypes binding of libcsvc.so (include/csvc.h), same names as the C ABI.

Argument marshalling only: every function forwards to the C entry point of
the same name.  Device buffers may be given as integers (device addresses) or
as objects with ``data_ptr()`` (torch tensors); streams as integers, ``None``
(the legacy default stream) or objects with ``cuda_stream``.  A non-zero
status raises :class:`CsError`.  There is no fallback: if the library is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcsvc.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "csvc.h")

CS_OK = 0
CS_EINVAL = -1
CS_ENOMEM = -2
CS_EAGAIN = -3
CS_ETIMEDOUT = -4
CS_ECUDA = -5
CS_ENOTFOUND = -6
CS_ENODEV = -7

CS_FP32, CS_BF16, CS_BF16X2, CS_FP16 = 0, 1, 2, 3
CS_ENGINE_AUTO, CS_ENGINE_PLAIN, CS_ENGINE_TC, CS_ENGINE_TC_STREAM, CS_ENGINE_TC_CHUNK = 0, 1, 2, 3, 4


class CsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (status %d): %s" % (_strerror_safe(status), status, message))
        self.status = status


class cs_params(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int32), ("width", ctypes.c_int32),
        ("gop", ctypes.c_int32), ("n_gops", ctypes.c_int32),
        ("block", ctypes.c_int32), ("m", ctypes.c_int32),
        ("iters", ctypes.c_int32), ("fp32_tail_iters", ctypes.c_int32),
        ("lambda_rel", ctypes.c_float),
        ("precision", ctypes.c_int32), ("engine", ctypes.c_int32),
    ]


def make_params(height, width, gop, block, m, iters=200, n_gops=1, lambda_rel=0.01,
                precision=CS_FP32, engine=CS_ENGINE_AUTO, fp32_tail_iters=0) -> cs_params:
    return cs_params(int(height), int(width), int(gop), int(n_gops), int(block), int(m),
                     int(iters), int(fp32_tail_iters), float(lambda_rel), int(precision),
                     int(engine))


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_SIGS = {
    "cs_ctx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t]),
    "cs_ctx_destroy": (ctypes.c_int, [_vp]),
    "cs_ctx_status": (ctypes.c_int, [_vp]),
    "cs_ctx_set_debug": (ctypes.c_int, [_vp, _i32]),
    "cs_make_phi": (ctypes.c_int, [_vp, _i32, _i32, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "cs_plan_destroy": (ctypes.c_int, [_vp]),
    "cs_plan_phi": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "cs_plan_a": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "cs_plan_lipschitz": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "cs_encode_gop": (ctypes.c_int, [_vp, ctypes.POINTER(cs_params), _vp, _vp, _vp]),
    "cs_encode_batch": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(cs_params),
                                       _vp, ctypes.POINTER(_vp), _vp]),
    "cs_decode_gop": (ctypes.c_int, [_vp, ctypes.POINTER(cs_params), _vp, _vp, _vp, _vp, _vp]),
    "cs_decode_batch": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(cs_params),
                                       ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                       ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    "cs_decode_gop_tv": (ctypes.c_int, [_vp, ctypes.POINTER(cs_params), ctypes.c_float,
                                        ctypes.c_float, _vp, _vp, _vp, _vp, _vp]),
    "cs_autotune": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                   ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float)]),
    "cs_psnr": (ctypes.c_int, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "cs_total_cr": (ctypes.c_double, [_i32, ctypes.c_double, ctypes.c_double]),
    "cs_raw_key_cr": (ctypes.c_double, [_i32, _i32, _i32, _i32, _i32]),
    "cs_submit": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(cs_params), _vp, _vp, _vp,
                                 ctypes.POINTER(ctypes.c_uint64)]),
    "cs_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32),
                               ctypes.POINTER(ctypes.c_float)]),
    "cs_codec_host": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(cs_params),
                                     _vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    "cs_lambda_max_noalloc": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp]),
    "cs_ctx_set_serving": (ctypes.c_int, [_vp, _i32]),
    "cs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cs_last_error": (ctypes.c_char_p, []),
}


def load():
    """Load libcsvc.so once; raise if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libcsvc.so not built (%s); run python -m "
                                   "paper_1311_1419_gb300.build" % LIB_PATH)
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def header_symbols():
    """Function names declared in include/csvc.h."""
    text = open(HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", text)))


def _strerror_safe(status: int) -> str:
    try:
        return load().cs_strerror(status).decode()
    except Exception:  # the library itself may be what failed to load
        return "error"


def _check(status: int):
    if status != CS_OK:
        raise CsError(status, load().cs_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def cs_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    out = _vp()
    _check(load().cs_ctx_create(ctypes.byref(out), int(device), int(hbm_budget_bytes)))
    return out.value


def cs_ctx_destroy(ctx: int) -> None:
    _check(load().cs_ctx_destroy(ctx))


def cs_ctx_status(ctx: int) -> None:
    _check(load().cs_ctx_status(ctx))


CS_DEBUG_DROP_ARRIVAL = 1


def cs_ctx_set_debug(ctx: int, flags: int) -> None:
    _check(load().cs_ctx_set_debug(ctx, int(flags)))


def cs_autotune(ctx: int, plan: int):
    """Time the decode shapes of the plan's (N, M) and record the fastest;
    returns (engine, plain_threads, plain_blocks_per_cta, ns_per_block_iter)."""
    eng, thr, blk, ns = _i32(), _i32(), _i32(), ctypes.c_float()
    _check(load().cs_autotune(ctx, plan, ctypes.byref(eng), ctypes.byref(thr), ctypes.byref(blk),
                              ctypes.byref(ns)))
    return eng.value, thr.value, blk.value, ns.value


def cs_make_phi(ctx: int, n: int, m: int, seed: int) -> int:
    out = _vp()
    _check(load().cs_make_phi(ctx, int(n), int(m), int(seed) & (2**64 - 1), ctypes.byref(out)))
    return out.value


def cs_plan_destroy(plan: int) -> None:
    _check(load().cs_plan_destroy(plan))


def cs_plan_phi(plan: int) -> int:
    out = _vp()
    _check(load().cs_plan_phi(plan, ctypes.byref(out)))
    return out.value


def cs_plan_a(plan: int) -> int:
    out = _vp()
    _check(load().cs_plan_a(plan, ctypes.byref(out)))
    return out.value


def cs_plan_lipschitz(plan: int) -> float:
    out = ctypes.c_double()
    _check(load().cs_plan_lipschitz(plan, ctypes.byref(out)))
    return out.value


def cs_encode_gop(plan: int, params: cs_params, frames_dev, y_dev, stream=None) -> None:
    _check(load().cs_encode_gop(plan, ctypes.byref(params), _ptr(frames_dev), _ptr(y_dev),
                                _stream(stream)))


def cs_encode_batch(ctx: int, plans, params, frames_dev, y_dev, stream=None) -> None:
    """cs_encode_gop for several plans over one clip; sequences of equal length."""
    n = len(plans)
    pl = (_vp * n)(*plans)
    pa = (cs_params * n)(*params)
    ys = (_vp * n)(*[_ptr(y) for y in y_dev])
    _check(load().cs_encode_batch(ctx, n, pl, pa, _ptr(frames_dev), ys, _stream(stream)))


def cs_decode_gop(plan: int, params: cs_params, key_dev, y_dev, frames_f32_dev=None,
                  frames_u8_dev=None, stream=None) -> None:
    _check(load().cs_decode_gop(plan, ctypes.byref(params), _ptr(key_dev), _ptr(y_dev),
                                _ptr(frames_f32_dev), _ptr(frames_u8_dev), _stream(stream)))


def cs_decode_gop_tv(plan: int, params: cs_params, key_dev, y_dev, frames_f32_dev=None,
                     frames_u8_dev=None, stream=None, beta: float = 0.125, mu: float = 1.0) -> None:
    """TV recovery (the paper's TVAL3 regulariser) of every CS frame of the call."""
    _check(load().cs_decode_gop_tv(plan, ctypes.byref(params), float(beta), float(mu),
                                   _ptr(key_dev), _ptr(y_dev), _ptr(frames_f32_dev),
                                   _ptr(frames_u8_dev), _stream(stream)))


def cs_decode_batch(ctx: int, plans, params, key_dev, y_dev, frames_f32_dev=None,
                    frames_u8_dev=None, stream=None) -> None:
    """Sequences of equal length; device buffers as ints or tensors (None allowed)."""
    n = len(plans)

    def arr(xs):
        if xs is None:
            return None
        a = (_vp * n)()
        for i, x in enumerate(xs):
            a[i] = _ptr(x)
        return a

    pl = (_vp * n)(*plans)
    pa = (cs_params * n)(*params)
    _check(load().cs_decode_batch(ctx, n, pl, pa, arr(key_dev), arr(y_dev), arr(frames_f32_dev),
                                  arr(frames_u8_dev), _stream(stream)))


def cs_psnr(ref_dev, test_dev, n_frames: int, height: int, width: int, psnr_dev,
            stream=None) -> None:
    _check(load().cs_psnr(_ptr(ref_dev), _ptr(test_dev), int(n_frames), int(height), int(width),
                          _ptr(psnr_dev), _stream(stream)))


def cs_total_cr(gop: int, cr_key: float, cr_cs: float) -> float:
    return load().cs_total_cr(int(gop), float(cr_key), float(cr_cs))


def cs_raw_key_cr(gop: int, height: int, width: int, block: int, m: int) -> float:
    return load().cs_raw_key_cr(int(gop), int(height), int(width), int(block), int(m))


def _host_ptr(x):
    """Host buffer address: an int, a numpy array or a CPU tensor."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    return int(x.data_ptr())


def cs_submit(ctx: int, plan: int, params: cs_params, key_host, y_host, frames_u8_host) -> int:
    t = ctypes.c_uint64()
    _check(load().cs_submit(ctx, plan, ctypes.byref(params), _host_ptr(key_host),
                            _host_ptr(y_host), _host_ptr(frames_u8_host), ctypes.byref(t)))
    return t.value


def cs_poll(ctx: int, ticket: int):
    """(done, latency_ms); latency is meaningful once done is True."""
    done = _i32()
    lat = ctypes.c_float()
    _check(load().cs_poll(ctx, int(ticket), ctypes.byref(done), ctypes.byref(lat)))
    return bool(done.value), float(lat.value)


def cs_codec_host(ctx: int, plans, params, clip_host, frames_u8_host, psnr_host,
                  stream=None) -> None:
    """Encode + batched decode + PSNR of one clip under every plan, host memory
    in and out; sequences of equal length (host buffers as arrays, CPU tensors
    or ints)."""
    n = len(plans)
    pl = (_vp * n)(*plans)
    pa = (cs_params * n)(*params)
    fu = (_vp * n)(*[_host_ptr(x) for x in frames_u8_host])
    ps = (_vp * n)(*[_host_ptr(x) for x in psnr_host])
    _check(load().cs_codec_host(ctx, n, pl, pa, _host_ptr(clip_host), fu, ps, _stream(stream)))


CS_SERVING_LAUNCH, CS_SERVING_QUEUE = 0, 1


def cs_ctx_set_serving(ctx: int, mode: int) -> None:
    """CS_SERVING_QUEUE (device work queue, the default) or CS_SERVING_LAUNCH."""
    _check(load().cs_ctx_set_serving(ctx, int(mode)))


def cs_lambda_max_noalloc(phi_dev, n: int, m: int, lambda_max_dev, stream=None) -> None:
    _check(load().cs_lambda_max_noalloc(_ptr(phi_dev), int(n), int(m), _ptr(lambda_max_dev),
                                        _stream(stream)))


def cs_strerror(status: int) -> str:
    return load().cs_strerror(int(status)).decode()


def cs_last_error() -> str:
    return load().cs_last_error().decode()
