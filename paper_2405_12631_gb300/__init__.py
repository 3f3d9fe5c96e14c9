"""Python binding of libpwave (the GB300 pWave++ codec library).

Thin ctypes marshalling over the C ABI declared in include/pwave.h: every
function of the ABI is exposed under the same name (``pw_*``), plus a small
``Codec`` convenience class that converts numpy arrays, bytes and torch
tensors to the ABI's pointers. All computation happens in the CUDA library;
importing this module fails loudly when libpwave.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpwave.so")

PW_OK, PW_EINVAL, PW_ENOMEM, PW_ECORRUPT, PW_EUNSUPPORTED, PW_ETIMEOUT, PW_EAGAIN, PW_ECUDA = range(8)
PW_PREC_FP32, PW_PREC_BF16, PW_PREC_FP8, PW_PREC_INT8 = 0, 1, 2, 3


class PwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pwave error {code}: {msg}")
        self.code = code


class pw_image(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("channels", C.c_int32),
                ("bitdepth", C.c_int32), ("is_device", C.c_int32), ("reserved", C.c_int32),
                ("data", C.c_void_p), ("stride_bytes", C.c_int64)]


class pw_codec_opts(C.Structure):
    _fields_ = [("q", C.c_float), ("lossless", C.c_int32), ("chunk_symbols", C.c_int32)]


class pw_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("rejected", C.c_uint64), ("queued", C.c_uint64), ("batches", C.c_uint64),
                ("held_bytes", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("mpix_per_s", C.c_double)]


class pw_model_cfg(C.Structure):
    _fields_ = [("levels", C.c_int32), ("C", C.c_int32), ("F", C.c_int32),
                ("ll_mode", C.c_int32)]


class pw_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_uint64), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libpwave.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`"
            f" (expected at {LIB_PATH})")
    return C.CDLL(LIB_PATH)


_lib = _load()

_P = C.c_void_p
_u8p = C.POINTER(C.c_uint8)
_sig = {
    "pw_ctx_create": (C.c_int, [C.c_int, _P, C.c_int, C.POINTER(_P)]),
    "pw_ctx_destroy": (None, [_P]),
    "pw_ctx_precision": (C.c_int, [_P]),
    "pw_ctx_set_lane_rule": (C.c_int, [_P, C.c_int]),
    "pw_ctx_launch_count": (C.c_uint64, [_P]),
    "pw_model_load": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(_P)]),
    "pw_model_free": (None, [_P]),
    "pw_model_hash": (C.c_uint64, [_P]),
    "pw_model_mixture": (C.c_int, [_P]),
    "pw_ctx_set_graphs": (C.c_int, [_P, C.c_int]),
    "pw_ctx_graph_replays": (C.c_uint64, [_P]),
    "pw_model_random_blob": (C.c_int, [C.POINTER(pw_model_cfg), C.c_uint64, _P, C.c_size_t,
                                       C.POINTER(C.c_size_t)]),
    "pw_model_init_random": (C.c_int, [_P, C.POINTER(pw_model_cfg), C.c_uint64,
                                       C.POINTER(_P)]),
    "pw_encode_image": (C.c_int, [_P, _P, C.POINTER(pw_image), C.POINTER(pw_codec_opts),
                                  C.POINTER(_u8p), C.POINTER(C.c_size_t)]),
    "pw_decode_image": (C.c_int, [_P, _P, _P, C.c_size_t, C.POINTER(pw_image)]),
    "pw_encode_batch": (C.c_int, [_P, _P, C.c_int, C.POINTER(pw_image),
                                  C.POINTER(pw_codec_opts), C.POINTER(_u8p),
                                  C.POINTER(C.c_size_t)]),
    "pw_decode_batch": (C.c_int, [_P, _P, C.c_int, C.POINTER(_P), C.POINTER(C.c_size_t),
                                  C.c_int, C.POINTER(pw_image)]),
    "pw_cdf_bank": (C.c_int, [_P, _P]),
    "pw_entropy_index": (C.c_int, [_P, _P, _P, C.c_int64, _P]),
    "pw_rans_decode": (C.c_int, [_P, _P, C.c_size_t, C.c_int, _P, _P, _P, _P, _P, _P]),
    "pw_rans_encode": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.POINTER(_u8p),
                                 C.POINTER(C.c_size_t), _P, _P]),
    "pw_rans_decode_noalloc": (C.c_int, [_P, _P, C.c_size_t, C.c_int, _P, _P, _P, _P, _P,
                                         _P]),
    "pw_context_params": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P]),
    "pw_context_mixture": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P]),
    "pw_mix_tables": (C.c_int, [_P, C.c_int64, _P, _P]),
    "pw_lift_forward": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "pw_lift_inverse": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "pw_decode_symbols": (C.c_int, [_P, _P, _P, C.c_size_t, _P]),
    "pw_analyse": (C.c_int, [_P, _P, C.POINTER(pw_image), C.POINTER(pw_codec_opts), _P]),
    "pw_encode_latent": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(pw_codec_opts), C.POINTER(_u8p),
                                   C.POINTER(C.c_size_t)]),
    "pw_conv_bf16": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.c_int, _P, _P, _P, _P]),
    "pw_encode_gop": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(pw_image),
                                C.POINTER(pw_codec_opts), C.POINTER(_u8p),
                                C.POINTER(C.c_size_t)]),
    "pw_decode_gop": (C.c_int, [_P, _P, _P, _P, C.c_size_t, C.c_int, C.POINTER(pw_image)]),
    "pw_temporal_lift": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "pw_temporal_lift_mc": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "pw_motion_search": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "pw_decode_footprint": (C.c_int, [_P, _P, _P, C.c_size_t, C.c_int,
                                      C.POINTER(C.c_uint64)]),
    "pw_server_create": (C.c_int, [_P, _P, C.c_size_t, C.c_int, C.c_int, C.POINTER(_P)]),
    "pw_server_submit": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_uint64)]),
    "pw_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(pw_image), C.c_int]),
    "pw_server_stats": (C.c_int, [_P, C.POINTER(pw_stats)]),
    "pw_server_destroy": (None, [_P]),
    "pw_autotune": (C.c_int, [C.c_int]),
    "pw_autotune_settled": (C.c_int, []),
    "pw_autotune_report": (C.c_int, [C.c_char_p, C.c_size_t]),
    "pw_ctx_profile": (C.c_int, [_P, C.c_int]),
    "pw_ctx_kernel_stats": (C.c_int, [_P, C.POINTER(pw_kernel_stat), C.c_int]),
    "pw_ctx_profile_classes": (C.c_int, [_P, C.c_uint32]),
    "pw_kernel_class": (C.c_int, [C.c_char_p]),
    "pw_free": (None, [_P]),
    "pw_strerror": (C.c_char_p, [C.c_int]),
    "pw_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_sig)


def check(code: int):
    if code != PW_OK:
        raise PwError(code, pw_strerror(code).decode())


def random_model_blob(levels: int = 4, C: int = 64, F: int = 16, ll_mode: int = 0,
                      seed: int = 0) -> bytes:
    """pw_model_random_blob: seeded random-init weights of the architecture as
    a weight blob (host only, no device needed)."""
    import ctypes
    cfg = pw_model_cfg(levels, C, F, ll_mode)
    n = ctypes.c_size_t(0)
    check(pw_model_random_blob(ctypes.byref(cfg), seed, None, 0, ctypes.byref(n)))
    buf = (ctypes.c_uint8 * n.value)()
    check(pw_model_random_blob(ctypes.byref(cfg), seed, ctypes.cast(buf, ctypes.c_void_p),
                               n.value, ctypes.byref(n)))
    return bytes(buf)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _take_bytes(p, n: int) -> bytes:
    b = C.string_at(p, n)
    pw_free(p)
    return b


def _opts(q, lossless, chunk):
    return pw_codec_opts(float(q), int(bool(lossless)), int(chunk))


def _host_image(img: np.ndarray, bitdepth: int | None):
    img = np.ascontiguousarray(img)
    h, w = img.shape[:2]
    ch = 1 if img.ndim == 2 else img.shape[2]
    if bitdepth is None:
        bitdepth = 8 if img.dtype == np.uint8 else 16
    return pw_image(w, h, ch, bitdepth, 0, 0, img.ctypes.data, 0), img


class Model:
    def __init__(self, codec: "Codec", blob: bytes = None, cfg: "pw_model_cfg" = None,
                 seed: int = 0):
        """A loaded model: from a weight blob (pw_model_load), or, with
        blob None, random-init weights of `cfg` (pw_model_init_random)."""
        self.codec = codec
        self._blob = blob
        h = C.c_void_p()
        if blob is not None:
            check(pw_model_load(codec.ctx, blob, len(blob), C.byref(h)))
        else:
            check(pw_model_init_random(codec.ctx, C.byref(cfg), seed, C.byref(h)))
        self.handle = h

    @property
    def hash(self) -> int:
        return int(pw_model_hash(self.handle))

    @property
    def mixture(self) -> bool:
        """Logistic-mixture probability model (else Laplace)."""
        return bool(pw_model_mixture(self.handle))

    def close(self):
        if self.handle:
            pw_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A decode server (pw_server_*): continuous batching over worker lanes."""

    def __init__(self, codec: "Codec", model: Model, hbm_budget: int, lanes: int = 2,
                 max_batch: int = 8):
        self.codec, self.model = codec, model
        h = C.c_void_p()
        check(pw_server_create(codec.ctx, model.handle, int(hbm_budget), int(lanes),
                               int(max_batch), C.byref(h)))
        self.handle = h
        self._shapes = {}

    def submit(self, bs: bytes) -> int:
        t = C.c_uint64()
        check(pw_server_submit(self.handle, bs, len(bs), C.byref(t)))
        self._shapes[t.value] = stream_image_shape(bs)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 60000):
        """Decoded image of a ticket (numpy), or None when not ready yet."""
        shape, dtype = self._shapes[ticket]
        out = np.zeros(shape, dtype=dtype)
        h, w = shape[:2]
        ch = 1 if len(shape) == 2 else shape[2]
        im = pw_image(w, h, ch, 8 if out.dtype == np.uint8 else 16, 0, 0, out.ctypes.data, 0)
        r = pw_server_poll(self.handle, ticket, C.byref(im), int(timeout_ms))
        if r in (PW_EAGAIN, PW_ETIMEOUT):
            return None
        del self._shapes[ticket]
        check(r)
        return out

    def stats(self) -> dict:
        st = pw_stats()
        check(pw_server_stats(self.handle, C.byref(st)))
        return {k: getattr(st, k) for k, _ in pw_stats._fields_}

    def close(self):
        if self.handle:
            pw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Codec:
    """A libpwave context (one CUDA device, one stream, one precision)."""

    def __init__(self, device: int = 0, precision: str | int = "fp32", stream: int = 0):
        prec = {"fp32": PW_PREC_FP32, "bf16": PW_PREC_BF16, "fp8": PW_PREC_FP8,
                "int8": PW_PREC_INT8}.get(precision, precision)
        h = C.c_void_p()
        check(pw_ctx_create(int(device), C.c_void_p(stream or None), int(prec), C.byref(h)))
        self.ctx = h
        self.precision = prec

    def set_lane_rule(self, log2_symbols_per_state: int):
        """pw_ctx_set_lane_rule: streams this context encodes use one rANS
        state per 2^s symbols (s in 5..7; default 7)."""
        check(pw_ctx_set_lane_rule(self.ctx, int(log2_symbols_per_state)))

    def set_graphs(self, enable: bool) -> bool:
        """pw_ctx_set_graphs: replay image decodes from captured CUDA graphs
        (default on); returns the previous setting."""
        old = pw_ctx_set_graphs(self.ctx, int(bool(enable)))
        if old < 0:
            check(-old)
        return bool(old)

    @property
    def graph_replays(self) -> int:
        """Decodes served by a replayed CUDA graph (pw_ctx_graph_replays)."""
        return int(pw_ctx_graph_replays(self.ctx))

    def close(self):
        if self.ctx:
            pw_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(pw_ctx_launch_count(self.ctx))

    def load_model(self, blob: bytes) -> Model:
        return Model(self, blob)

    def init_random_model(self, levels: int = 4, C: int = 64, F: int = 16, ll_mode: int = 0,
                          seed: int = 0) -> Model:
        """pw_model_init_random: the model of random_model_blob(same arguments)."""
        return Model(self, None, pw_model_cfg(levels, C, F, ll_mode), seed)

    # ---- images -----------------------------------------------------------
    def encode_image(self, model: Model, img: np.ndarray, q: float = 8.0,
                     lossless: bool = False, chunk: int = 16384,
                     bitdepth: int | None = None) -> bytes:
        return self.encode_batch(model, [img], q, lossless, chunk, bitdepth)[0]

    def encode_batch(self, model: Model, imgs, q: float = 8.0, lossless: bool = False,
                     chunk: int = 16384, bitdepth: int | None = None) -> list:
        ims, keep = [], []
        for im in imgs:
            s, a = _host_image(im, bitdepth)
            ims.append(s)
            keep.append(a)
        arr = (pw_image * len(ims))(*ims)
        outs = (_u8p * len(ims))()
        lens = (C.c_size_t * len(ims))()
        o = _opts(q, lossless, chunk)
        check(pw_encode_batch(self.ctx, model.handle, len(ims), arr, C.byref(o), outs, lens))
        return [_take_bytes(outs[i], lens[i]) for i in range(len(ims))]

    def decode_image(self, model: Model, bs: bytes, shape=None, dtype=None) -> np.ndarray:
        return self.decode_batch(model, [bs], shape, dtype)[0]

    def decode_ragged_device(self, model: Model, ptrs, lens, out_ptrs, shapes,
                             bitdepth: int = 8):
        """Decode device-resident streams of one format and different sizes
        in one call: out_ptrs[i] is a packed device image of shapes[i]."""
        B = len(ptrs)
        ims = (pw_image * B)(*[pw_image(sh[1], sh[0], 1 if len(sh) == 2 else sh[2], bitdepth, 1,
                                        0, o, 0) for o, sh in zip(out_ptrs, shapes)])
        p = (C.c_void_p * B)(*ptrs)
        n = (C.c_size_t * B)(*lens)
        check(pw_decode_batch(self.ctx, model.handle, B, p, n, 1, ims))

    def decode_image_alloc(self, model: Model, bs: bytes) -> np.ndarray:
        """pw_decode_image with no output buffer: the library allocates the
        image (its size from the stream); copied out and released here."""
        im = pw_image(0, 0, 0, 0, 0, 0, None, 0)
        check(pw_decode_image(self.ctx, model.handle, bs, len(bs), C.byref(im)))
        try:
            dtype = np.uint8 if im.bitdepth <= 8 else np.uint16
            n = im.width * im.height * im.channels
            arr = np.ctypeslib.as_array(C.cast(im.data, C.POINTER(
                C.c_uint8 if dtype == np.uint8 else C.c_uint16)), shape=(n,)).copy()
        finally:
            pw_free(im.data)
        shape = (im.height, im.width) if im.channels == 1 else (im.height, im.width, im.channels)
        return arr.reshape(shape)

    def decode_batch(self, model: Model, streams, shape=None, dtype=None) -> np.ndarray:
        if shape is None or dtype is None:
            shape, dtype = stream_image_shape(streams[0])
        B = len(streams)
        out = np.zeros((B,) + tuple(shape), dtype=dtype)
        h, w = shape[:2]
        ch = 1 if len(shape) == 2 else shape[2]
        bd = 8 if out.dtype == np.uint8 else 16
        item = out[0].nbytes
        ims = (pw_image * B)(*[pw_image(w, h, ch, bd, 0, 0, out.ctypes.data + i * item, 0)
                               for i in range(B)])
        bufs = [C.c_char_p(s) for s in streams]
        ptrs = (C.c_void_p * B)(*[C.cast(b, C.c_void_p) for b in bufs])
        lens = (C.c_size_t * B)(*[len(s) for s in streams])
        check(pw_decode_batch(self.ctx, model.handle, B, ptrs, lens, 0, ims))
        return out

    def decode_ragged(self, model: Model, streams) -> list:
        """Decode host streams of one format whose image sizes differ, in one
        batch call (a ragged batch on a canvas of the largest size); returns
        one array per stream, each exactly what decoding it alone gives."""
        B = len(streams)
        outs = []
        for s in streams:
            shape, dtype = stream_image_shape(s)
            outs.append(np.zeros(shape, dtype=dtype))
        ims = (pw_image * B)(*[pw_image(o.shape[1], o.shape[0], 1 if o.ndim == 2 else o.shape[2],
                                        8 if o.dtype == np.uint8 else 16, 0, 0, o.ctypes.data, 0)
                               for o in outs])
        bufs = [C.c_char_p(s) for s in streams]
        ptrs = (C.c_void_p * B)(*[C.cast(b, C.c_void_p) for b in bufs])
        lens = (C.c_size_t * B)(*[len(s) for s in streams])
        check(pw_decode_batch(self.ctx, model.handle, B, ptrs, lens, 0, ims))
        return outs

    def decode_footprint(self, model: Model, bs: bytes, count: int = 1) -> int:
        """Estimated device workspace bytes to decode `count` streams like bs."""
        b = C.c_uint64()
        check(pw_decode_footprint(self.ctx, model.handle, bs, len(bs), int(count), C.byref(b)))
        return int(b.value)

    def decode_batch_device(self, model: Model, ptrs, lens, out_ptr: int, shape,
                            bitdepth: int = 8):
        """Decode device-resident streams into a contiguous device output.

        ptrs / lens: device addresses and byte lengths of the streams;
        out_ptr: device address of a packed [B, H, W, C] buffer.
        """
        B = len(ptrs)
        h, w = shape[:2]
        ch = 1 if len(shape) == 2 else shape[2]
        item = h * w * ch * (1 if bitdepth <= 8 else 2)
        ims = (pw_image * B)(*[pw_image(w, h, ch, bitdepth, 1, 0, out_ptr + i * item, 0)
                               for i in range(B)])
        p = (C.c_void_p * B)(*ptrs)
        n = (C.c_size_t * B)(*lens)
        check(pw_decode_batch(self.ctx, model.handle, B, p, n, 1, ims))

    def decode_batch_host_ptrs(self, model: Model, ptrs, lens, out_ptr: int, shape,
                               bitdepth: int = 8):
        """Decode host-resident streams (host addresses and byte lengths)
        into a contiguous host output [B, H, W, C] at out_ptr. Page-locked
        buffers (e.g. pinned torch tensors) are copied to and from the device
        directly; pageable ones go through the library's pinned staging."""
        B = len(ptrs)
        h, w = shape[:2]
        ch = 1 if len(shape) == 2 else shape[2]
        item = h * w * ch * (1 if bitdepth <= 8 else 2)
        ims = (pw_image * B)(*[pw_image(w, h, ch, bitdepth, 0, 0, out_ptr + i * item, 0)
                               for i in range(B)])
        p = (C.c_void_p * B)(*ptrs)
        n = (C.c_size_t * B)(*lens)
        check(pw_decode_batch(self.ctx, model.handle, B, p, n, 0, ims))

    # ---- video GOPs -------------------------------------------------------
    def encode_gop(self, m_low: Model, m_high: Model, frames: np.ndarray, q: float = 8.0,
                   chunk: int = 16384) -> bytes:
        frames = np.ascontiguousarray(frames, dtype=np.uint8)
        nf = frames.shape[0]
        ims = (pw_image * nf)(*[_host_image(frames[f], 8)[0] for f in range(nf)])
        o = _opts(q, False, chunk)
        p = _u8p()
        n = C.c_size_t()
        check(pw_encode_gop(self.ctx, m_low.handle, m_high.handle, nf, ims, C.byref(o),
                            C.byref(p), C.byref(n)))
        return _take_bytes(p, n.value)

    def decode_gop(self, m_low: Model, m_high: Model, gs: bytes, nframes: int, shape) -> np.ndarray:
        out = np.zeros((nframes,) + tuple(shape), dtype=np.uint8)
        self.decode_gop_into(m_low, m_high, gs, nframes, shape, out.ctypes.data)
        return out

    def decode_gop_into(self, m_low: Model, m_high: Model, gs: bytes, nframes: int, shape,
                        out_ptr: int, on_device: bool = False):
        """pw_decode_gop into a caller's contiguous [nframes, H, W, C] uint8
        buffer (host, page-locked or not, or device with on_device)."""
        h, w = shape[:2]
        ch = 1 if len(shape) == 2 else shape[2]
        item = h * w * ch
        ims = (pw_image * nframes)(*[pw_image(w, h, ch, 8, int(on_device), 0, out_ptr + f * item, 0)
                                     for f in range(nframes)])
        check(pw_decode_gop(self.ctx, m_low.handle, m_high.handle, gs, len(gs), nframes, ims))

    def temporal_lift(self, model: Model, frames: np.ndarray, forward: bool = True) -> np.ndarray:
        frames = np.ascontiguousarray(frames, dtype=np.float32)
        nf, H, W = frames.shape
        out = np.zeros_like(frames)
        check(pw_temporal_lift(self.ctx, model.handle, nf, H, W, int(forward), _ptr(frames),
                               _ptr(out)))
        return out

    def temporal_lift_mc(self, model: Model, frames: np.ndarray, mv: np.ndarray,
                         forward: bool = True) -> np.ndarray:
        """pw_temporal_lift_mc: frames [nf, H, W] float, mv [nf - 1, nby,
        nbx, 2] int8 (the layout motion_search returns)."""
        frames = np.ascontiguousarray(frames, dtype=np.float32)
        mv = np.ascontiguousarray(mv, dtype=np.int8)
        nf, H, W = frames.shape
        out = np.zeros_like(frames)
        check(pw_temporal_lift_mc(self.ctx, model.handle, nf, H, W, int(forward), _ptr(mv),
                                  _ptr(frames), _ptr(out)))
        return out

    def motion_search(self, luma: np.ndarray) -> np.ndarray:
        """pw_motion_search on integer luma frames [nf, H, W] -> vectors
        [nf - 1, ceil(H/16), ceil(W/16), 2] (int8 dy, dx)."""
        luma = np.ascontiguousarray(luma, dtype=np.int32)
        nf, H, W = luma.shape
        mv = np.zeros((nf - 1, -(-H // 16), -(-W // 16), 2), dtype=np.int8)
        check(pw_motion_search(self.ctx, nf, H, W, _ptr(luma), _ptr(mv)))
        return mv

    # ---- stages -----------------------------------------------------------
    def cdf_bank_device(self, dev_ptr: int):
        check(pw_cdf_bank(self.ctx, C.c_void_p(dev_ptr)))

    def entropy_index(self, mu: np.ndarray, sigma: np.ndarray) -> np.ndarray:
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sigma = np.ascontiguousarray(sigma, dtype=np.float32)
        idx = np.zeros(mu.shape, dtype=np.uint32)
        check(pw_entropy_index(self.ctx, _ptr(mu), _ptr(sigma), mu.size, _ptr(idx)))
        return idx

    def rans_decode(self, payload: bytes, offset, nbytes, count, lanes, idx) -> np.ndarray:
        offset = np.ascontiguousarray(offset, dtype=np.uint32)
        nbytes = np.ascontiguousarray(nbytes, dtype=np.uint32)
        count = np.ascontiguousarray(count, dtype=np.uint32)
        lanes = np.ascontiguousarray(lanes, dtype=np.uint32)
        idx = np.ascontiguousarray(idx, dtype=np.uint32)
        out = np.zeros(int(count.sum()), dtype=np.int32)
        pb = C.create_string_buffer(payload, len(payload))
        check(pw_rans_decode(self.ctx, pb, len(payload), len(count), _ptr(offset),
                             _ptr(nbytes), _ptr(count), _ptr(lanes), _ptr(idx), _ptr(out)))
        return out

    def rans_encode(self, count, lanes, idx, values):
        count = np.ascontiguousarray(count, dtype=np.uint32)
        lanes = np.ascontiguousarray(lanes, dtype=np.uint32)
        idx = np.ascontiguousarray(idx, dtype=np.uint32)
        values = np.ascontiguousarray(values, dtype=np.int32)
        n = len(count)
        offset = np.zeros(n, dtype=np.uint32)
        nbytes = np.zeros(n, dtype=np.uint32)
        p = _u8p()
        pbytes = C.c_size_t()
        check(pw_rans_encode(self.ctx, n, _ptr(count), _ptr(lanes), _ptr(idx), _ptr(values),
                             C.byref(p), C.byref(pbytes), _ptr(offset), _ptr(nbytes)))
        return _take_bytes(p, pbytes.value), offset, nbytes

    def context_params(self, model: Model, H: int, W: int, q: np.ndarray):
        q = np.ascontiguousarray(q, dtype=np.int32)
        mu = np.zeros(q.size, dtype=np.float32)
        sg = np.zeros(q.size, dtype=np.float32)
        check(pw_context_params(self.ctx, model.handle, H, W, _ptr(q), _ptr(mu), _ptr(sg)))
        return mu, sg

    def context_mixture(self, model: Model, H: int, W: int, q: np.ndarray) -> np.ndarray:
        """Mixture parameters (w, mu, sigma) [n, 9] of every position."""
        q = np.ascontiguousarray(q, dtype=np.int32)
        par = np.zeros((q.size, 9), dtype=np.float32)
        check(pw_context_mixture(self.ctx, model.handle, H, W, _ptr(q), _ptr(par)))
        return par

    def mix_tables(self, keys: np.ndarray) -> np.ndarray:
        """CDF tables [n, 128] (uint16) of mixture keys [n, 9] (q, j, g)."""
        keys = np.ascontiguousarray(keys, dtype=np.int32).reshape(-1, 9)
        out = np.zeros((keys.shape[0], 128), dtype=np.uint16)
        check(pw_mix_tables(self.ctx, keys.shape[0], _ptr(keys), _ptr(out)))
        return out

    def lift_forward(self, model: Model, x: np.ndarray, lossless: bool = False) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        H, W = x.shape
        out = np.zeros(H * W, dtype=np.float32)
        check(pw_lift_forward(self.ctx, model.handle, H, W, int(lossless), _ptr(x), _ptr(out)))
        return out

    def lift_inverse(self, model: Model, sb: np.ndarray, H: int, W: int,
                     lossless: bool = False) -> np.ndarray:
        sb = np.ascontiguousarray(sb, dtype=np.float32)
        out = np.zeros((H, W), dtype=np.float32)
        check(pw_lift_inverse(self.ctx, model.handle, H, W, int(lossless), _ptr(sb), _ptr(out)))
        return out

    def conv_bf16(self, x: np.ndarray, w: np.ndarray, b: np.ndarray, act: bool = False):
        """x [P, H, W, cin], w [cout, cin, k, k], b [cout] -> y [P, H, W, cout]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        P, H, W, cin = x.shape
        cout, _, k, _ = w.shape
        y = np.zeros((P, H, W, cout), dtype=np.float32)
        check(pw_conv_bf16(self.ctx, P, H, W, cin, cout, k, int(act), _ptr(x), _ptr(w), _ptr(b),
                           _ptr(y)))
        return y

    def decode_symbols(self, model: Model, bs: bytes) -> np.ndarray:
        hd = parse_stream_header(bs)
        n = hd["ncomp"] * padded_elems(hd)
        q = np.zeros(n, dtype=np.int32)
        check(pw_decode_symbols(self.ctx, model.handle, bs, len(bs), _ptr(q)))
        return q

    def analyse(self, model: Model, img: np.ndarray, q: float = 8.0, lossless: bool = False,
                levels: int = 4, bitdepth: int | None = None) -> np.ndarray:
        s, a = _host_image(img, bitdepth)
        mult = 1 << levels
        Hp = -(-s.height // mult) * mult
        Wp = -(-s.width // mult) * mult
        out = np.zeros(s.channels * Hp * Wp, dtype=np.int32)
        o = _opts(q, lossless, 16384)
        check(pw_analyse(self.ctx, model.handle, C.byref(s), C.byref(o), _ptr(out)))
        return out

    def encode_latent(self, model: Model, q: np.ndarray, width: int, height: int,
                      channels: int, bitdepth: int = 8, colour: int = 0, qstep: float = 8.0,
                      lossless: bool = False, chunk: int = 16384) -> bytes:
        q = np.ascontiguousarray(q, dtype=np.int32)
        o = _opts(qstep, lossless, chunk)
        p = _u8p()
        n = C.c_size_t()
        check(pw_encode_latent(self.ctx, model.handle, _ptr(q), width, height, channels,
                               bitdepth, colour, C.byref(o), C.byref(p), C.byref(n)))
        return _take_bytes(p, n.value)


# ---- stream header helpers (format only) ------------------------------------
def parse_stream_header(bs: bytes) -> dict:
    import struct
    if bs[:4] != b"PWBS":
        raise ValueError("not a PWBS stream")
    (ver, flags, width, height, ncomp, levels, bitdepth, colour, dl, dh, T, log2m, lanes,
     chunk, nch, mhash, pbytes) = struct.unpack_from("<HHIIBBBBffHBBIIQI", bs, 4)
    return dict(version=ver, flags=flags, width=width, height=height, ncomp=ncomp,
                levels=levels, bitdepth=bitdepth, colour=colour, delta_l=dl, delta_h=dh,
                chunk=chunk, n_chunks=nch, model_hash=mhash, payload_bytes=pbytes)


def padded_elems(hd: dict) -> int:
    mult = 1 << hd["levels"]
    return (-(-hd["height"] // mult) * mult) * (-(-hd["width"] // mult) * mult)


def autotune_report() -> list:
    """Tuned convolution classes as dicts (see pw_autotune_report)."""
    n = pw_autotune_report(None, 0)
    buf = C.create_string_buffer(n + 1)
    pw_autotune_report(buf, n + 1)
    keys = ("ks", "kb", "ncta", "epi", "fp8", "log2tiles", "choice")
    out = []
    for line in buf.value.decode().splitlines():
        v = line.split()
        d = {k: int(x) for k, x in zip(keys, v[:7])}
        d["pairs"] = d["choice"] & 1
        d["shape"] = d["choice"] >> 1
        d["us"] = [float(x) for x in v[7:11]]
        out.append(d)
    return out


def stream_image_shape(bs: bytes):
    hd = parse_stream_header(bs)
    dtype = np.uint8 if hd["bitdepth"] <= 8 else np.uint16
    shape = (hd["height"], hd["width"]) if hd["ncomp"] == 1 else (hd["height"], hd["width"], 3)
    return shape, dtype
