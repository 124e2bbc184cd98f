"""ctypes binding of libtabnet.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only
passes pointers, sizes and streams.  PyTorch tensors are accepted for device
buffers (their data_ptr is passed) and numpy arrays for host buffers.  When
the shared library is missing the import of any entry point raises: there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtabnet.so")

TABNET_FP32, TABNET_BF16, TABNET_FP8_E4M3, TABNET_BF16X3, TABNET_BF16X6 = 0, 1, 2, 3, 4
PRECISIONS = {"fp32": TABNET_FP32, "bf16": TABNET_BF16, "fp8": TABNET_FP8_E4M3, "bf16x3": TABNET_BF16X3,
              "bf16x6": TABNET_BF16X6}

OK = 0
ERR = {
    -1: "ARG", -2: "BLOB_MAGIC", -3: "BLOB_VERSION", -4: "BLOB_SIZE", -5: "BLOB_HASH",
    -6: "UNSUPPORTED_DIMS", -7: "CUDA", -8: "OOM", -9: "TIMEOUT", -10: "DEVICE",
}
STATUS_CAT_OOB = 0x1
STATUS_TIMEOUT = 0x2

#: every symbol declared in include/tabnet.h
EXPORTS = (
    "tabnet_abi_version", "tabnet_blob_inspect", "tabnet_create", "tabnet_dims_of",
    "tabnet_precision_of", "tabnet_forward", "tabnet_forward_host", "tabnet_poll_status",
    "tabnet_destroy", "tabnet_status_string", "tabnet_last_error", "tabnet_set_tile_config",
    "tabnet_get_tile_config", "tabnet_forward_segments", "tabnet_forward_segments_device",
    "tabnet_reserve_segments", "tabnet_forward_segments_noalloc",
    "tabnet_server_create", "tabnet_server_submit", "tabnet_server_poll", "tabnet_server_wait",
    "tabnet_server_result", "tabnet_server_result_compact", "tabnet_server_release", "tabnet_server_get_stats", "tabnet_server_reset_stats",
    "tabnet_server_replay", "tabnet_server_destroy", "tabnet_mask_stats", "tabnet_topk_agreement",
    "tabnet_set_input_transform",
)
#: fixed scratch capacity of tabnet_forward_segments_noalloc
NOALLOC_MAX_SEGMENTS = 65536


class TabnetError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {ERR.get(code, code)} ({detail})")


class Segment(ctypes.Structure):
    """tabnet_segment: one request's device buffers (48 bytes)."""
    _fields_ = [
        ("x_num", ctypes.c_void_p), ("x_cat", ctypes.c_void_p), ("rows", ctypes.c_int64),
        ("logits", ctypes.c_void_p), ("step_masks", ctypes.c_void_p), ("agg_mask", ctypes.c_void_p),
    ]


def segment_array(segs):
    """ctypes array of Segment from dicts {x_num, x_cat, rows, logits, masks, agg}
    whose values are torch tensors, raw pointers or None."""
    arr = (Segment * len(segs))()
    for i, g in enumerate(segs):
        arr[i] = Segment(_ptr(g.get("x_num")), _ptr(g.get("x_cat")), int(g["rows"]), _ptr(g.get("logits")),
                         _ptr(g.get("masks")), _ptr(g.get("agg")))
    return arr


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("max_batch_rows", ctypes.c_int),
                ("max_inflight_batches", ctypes.c_int), ("streams_per_model", ctypes.c_int),
                ("batch_min_rows", ctypes.c_int), ("batch_wait_us", ctypes.c_int), ("batch_busy", ctypes.c_int),
                ("mask_slots", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("rows_completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("mean_batch_rows", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p95_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("rows_per_s", ctypes.c_double), ("queue_depth", ctypes.c_int64),
                ("inflight_batches", ctypes.c_int64), ("device_bytes_in_use", ctypes.c_size_t),
                ("engine_staged", ctypes.c_uint64), ("p50_queue_ms", ctypes.c_double),
                ("p99_queue_ms", ctypes.c_double), ("engine_busy", ctypes.c_double),
                ("engine_max_pass_ms", ctypes.c_double), ("replay_max_late_ms", ctypes.c_double),
                ("p50_submit_ms", ctypes.c_double), ("p99_submit_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerRequest(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("x_num", ctypes.c_void_p), ("x_cat", ctypes.c_void_p),
                ("rows", ctypes.c_int64), ("arrival_s", ctypes.c_double)]


class Dims(ctypes.Structure):
    _fields_ = [
        ("n_num", ctypes.c_int32), ("n_cat", ctypes.c_int32), ("d_emb", ctypes.c_int32),
        ("n_feat", ctypes.c_int32), ("n_d", ctypes.c_int32), ("n_a", ctypes.c_int32),
        ("n_steps", ctypes.c_int32), ("n_shared", ctypes.c_int32), ("n_indep", ctypes.c_int32),
        ("n_classes", ctypes.c_int32), ("gamma", ctypes.c_double), ("bn_eps", ctypes.c_double),
        ("content_hash", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libtabnet.so (built in-tree by paper_2510_19689_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2510_19689_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    L.tabnet_abi_version.restype = i32
    L.tabnet_blob_inspect.argtypes = [vp, sz, ctypes.POINTER(Dims)]
    L.tabnet_create.argtypes = [vp, sz, i32, i32, ctypes.POINTER(vp)]
    L.tabnet_dims_of.argtypes = [vp, ctypes.POINTER(Dims)]
    L.tabnet_precision_of.argtypes = [vp]
    L.tabnet_forward.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    L.tabnet_forward_host.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    L.tabnet_poll_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint32)]
    L.tabnet_set_tile_config.argtypes = [vp, i32, i32, i32]
    ip = ctypes.POINTER(ctypes.c_int)
    L.tabnet_get_tile_config.argtypes = [vp, ip, ip, ip]
    L.tabnet_forward_segments.argtypes = [vp, vp, i32, vp]
    L.tabnet_forward_segments_device.argtypes = [vp, vp, i32, vp]
    L.tabnet_reserve_segments.argtypes = [vp, i32]
    L.tabnet_forward_segments_noalloc.argtypes = [vp, vp, i32, vp]
    L.tabnet_mask_stats.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp]
    L.tabnet_set_input_transform.argtypes = [vp, vp, vp, vp]
    L.tabnet_topk_agreement.argtypes = [vp, vp, i64, i32, i32, vp, vp]
    L.tabnet_server_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.tabnet_server_submit.argtypes = [vp, i32, vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
    L.tabnet_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), i32, ctypes.POINTER(ctypes.c_int)]
    L.tabnet_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double]
    fpp = ctypes.POINTER(ctypes.POINTER(ctypes.c_float))
    L.tabnet_server_result.argtypes = [vp, ctypes.c_uint64, fpp, fpp, fpp, ctypes.POINTER(ctypes.c_int64)]
    L.tabnet_server_result_compact.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.POINTER(ctypes.c_uint8)),
                                               ctypes.POINTER(ctypes.POINTER(ctypes.c_uint16)), fpp,
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]
    L.tabnet_server_release.argtypes = [vp, ctypes.c_uint64]
    L.tabnet_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.tabnet_server_reset_stats.argtypes = [vp]
    L.tabnet_server_replay.argtypes = [vp, ctypes.POINTER(ServerRequest), i32, i32, i32, i32]
    L.tabnet_server_destroy.argtypes = [vp]
    L.tabnet_server_destroy.restype = None
    L.tabnet_destroy.argtypes = [vp]
    L.tabnet_destroy.restype = None
    L.tabnet_status_string.argtypes = [i32]
    L.tabnet_status_string.restype = ctypes.c_char_p
    L.tabnet_last_error.restype = ctypes.c_char_p
    for name in ("tabnet_blob_inspect", "tabnet_create", "tabnet_dims_of", "tabnet_precision_of",
                 "tabnet_forward", "tabnet_forward_host", "tabnet_poll_status",
                 "tabnet_set_tile_config", "tabnet_get_tile_config", "tabnet_forward_segments",
                 "tabnet_forward_segments_device", "tabnet_reserve_segments",
                 "tabnet_forward_segments_noalloc", "tabnet_server_create", "tabnet_server_submit",
                 "tabnet_server_poll", "tabnet_server_wait", "tabnet_server_result", "tabnet_server_release",
                 "tabnet_server_get_stats", "tabnet_server_reset_stats", "tabnet_server_replay"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def last_error() -> str:
    return lib().tabnet_last_error().decode()


def _check(code: int, where: str):
    if code != OK:
        raise TabnetError(code, where, last_error())


def blob_inspect(blob: bytes) -> Dims:
    d = Dims()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().tabnet_blob_inspect(buf, len(blob), ctypes.byref(d)), "tabnet_blob_inspect")
    return d


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Model:
    """A model loaded on one device at one precision (tabnet_create)."""

    def __init__(self, blob: bytes, precision="bf16", device: int = 0):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().tabnet_create(buf, len(blob), prec, device, ctypes.byref(h)), "tabnet_create")
        self._h = h
        self.device = device
        self.precision = prec
        d = Dims()
        _check(lib().tabnet_dims_of(h, ctypes.byref(d)), "tabnet_dims_of")
        self.dims = d

    @property
    def handle(self) -> int:
        return self._h.value

    def forward(self, x_num, x_cat, rows: int, logits, masks=None, agg=None, stream=None) -> None:
        """Device buffers (torch tensors or raw pointers); stream-ordered."""
        _check(lib().tabnet_forward(self._h, _ptr(x_num), _ptr(x_cat), int(rows), _ptr(logits),
                                    _ptr(masks), _ptr(agg), _stream(stream)), "tabnet_forward")

    def forward_host(self, x_num: np.ndarray, x_cat: np.ndarray, masks=True, agg=True, stream=0):
        """Host numpy buffers in and out (synchronous)."""
        d = self.dims
        rows = x_num.shape[0] if d.n_num else x_cat.shape[0]
        x_num = np.ascontiguousarray(x_num, dtype=np.float32)
        x_cat = np.ascontiguousarray(x_cat, dtype=np.int32)
        lg = np.empty((rows, d.n_classes), np.float32)
        mk = np.empty((rows, d.n_steps, d.d_emb), np.float32) if masks else None
        ag = np.empty((rows, d.n_feat), np.float32) if agg else None
        _check(lib().tabnet_forward_host(self._h, _ptr(x_num) if d.n_num else None,
                                         _ptr(x_cat) if d.n_cat else None, rows, _ptr(lg),
                                         _ptr(mk), _ptr(ag), stream), "tabnet_forward_host")
        return lg, mk, ag

    def forward_segments(self, segs, stream=None) -> None:
        """Uneven request batches in one launch; segs: list of dicts (see
        segment_array) or a ctypes Segment array in host memory."""
        arr = segs if isinstance(segs, ctypes.Array) else segment_array(segs)
        _check(lib().tabnet_forward_segments(self._h, ctypes.cast(arr, ctypes.c_void_p), len(arr),
                                             _stream(stream)), "tabnet_forward_segments")

    def forward_segments_device(self, dev_descriptors, n_segs: int, stream=None) -> None:
        """Descriptors already in device memory (e.g. a uint8 CUDA tensor
        holding n_segs Segment records); capturable in a CUDA graph."""
        _check(lib().tabnet_forward_segments_device(self._h, _ptr(dev_descriptors), int(n_segs),
                                                    _stream(stream)), "tabnet_forward_segments_device")

    def reserve_segments(self, max_segs: int) -> None:
        _check(lib().tabnet_reserve_segments(self._h, int(max_segs)), "tabnet_reserve_segments")

    def set_tile_config(self, nwg: int = 0, n_slots: int = 0, ctas_per_sm: int = 0) -> None:
        _check(lib().tabnet_set_tile_config(self._h, nwg, n_slots, ctas_per_sm), "tabnet_set_tile_config")

    def tile_config(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().tabnet_get_tile_config(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "tabnet_get_tile_config")
        return dict(nwg=a.value, n_slots=b.value, ctas_per_sm=c.value)

    def set_input_transform(self, num_mean=None, num_scale=None, cat_base=None) -> None:
        """Feed raw inputs: numeric (x - num_mean) * num_scale, categorical
        x - cat_base (tabnet_set_input_transform); None = identity."""
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=t)
                for a, t in ((num_mean, np.float32), (num_scale, np.float32), (cat_base, np.int32))]
        _check(lib().tabnet_set_input_transform(self._h, *[_ptr(a) for a in arrs]), "tabnet_set_input_transform")

    def poll_status(self, stream=None) -> int:
        st = ctypes.c_uint32(0)
        code = lib().tabnet_poll_status(self._h, _stream(stream), ctypes.byref(st))
        if code not in (OK, -9, -10):
            _check(code, "tabnet_poll_status")
        return st.value

    def run(self, x_num, x_cat, stream=None):
        """Allocate torch outputs on the model's device and run forward."""
        import torch
        d = self.dims
        rows = x_num.shape[0] if d.n_num else x_cat.shape[0]
        dev = torch.device("cuda", self.device)
        lg = torch.empty((rows, d.n_classes), dtype=torch.float32, device=dev)
        mk = torch.empty((rows, d.n_steps, d.d_emb), dtype=torch.float32, device=dev)
        ag = torch.empty((rows, d.n_feat), dtype=torch.float32, device=dev)
        self.forward(x_num if d.n_num else None, x_cat if d.n_cat else None, rows, lg, mk, ag, stream)
        return lg, mk, ag

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tabnet_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server over resident models
    (tabnet_server_*).  Inputs are numpy arrays kept alive until release."""

    def __init__(self, models, device_bytes=1 << 30, max_batch_rows=65536, max_inflight_batches=32,
                 streams_per_model=8, batch_min_rows=0, batch_wait_us=0, mask_slots=0, batch_busy=0):
        self.models = list(models)
        arr = (ctypes.c_void_p * len(self.models))(*[m.handle for m in self.models])
        cfg = ServerConfig(device_bytes, max_batch_rows, max_inflight_batches, streams_per_model, batch_min_rows,
                           batch_wait_us, batch_busy, mask_slots)
        h = ctypes.c_void_p()
        _check(lib().tabnet_server_create(arr, len(self.models), ctypes.byref(cfg), ctypes.byref(h)),
               "tabnet_server_create")
        self._h = h
        self._keep = {}

    def submit(self, model: int, x_num: np.ndarray, x_cat: np.ndarray) -> int:
        d = self.models[model].dims
        rows = x_num.shape[0] if d.n_num else x_cat.shape[0]
        x_num = np.ascontiguousarray(x_num, dtype=np.float32)
        x_cat = np.ascontiguousarray(x_cat, dtype=np.int32)
        t = ctypes.c_uint64()
        _check(lib().tabnet_server_submit(self._h, model, _ptr(x_num) if d.n_num else None,
                                          _ptr(x_cat) if d.n_cat else None, rows, ctypes.byref(t)),
               "tabnet_server_submit")
        self._keep[t.value] = (x_num, x_cat, model, rows)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 30.0) -> None:
        _check(lib().tabnet_server_wait(self._h, ticket, timeout_s), "tabnet_server_wait")

    def result(self, ticket: int):
        """Copies of (logits, step_masks, agg_mask) of a completed request."""
        _, _, model, rows = self._keep[ticket]
        d = self.models[model].dims
        pl, pm, pa = (ctypes.POINTER(ctypes.c_float)() for _ in range(3))
        r = ctypes.c_int64()
        _check(lib().tabnet_server_result(self._h, ticket, ctypes.byref(pl), ctypes.byref(pm), ctypes.byref(pa),
                                          ctypes.byref(r)), "tabnet_server_result")
        lg = np.ctypeslib.as_array(pl, shape=(rows, d.n_classes)).copy()
        mk = np.ctypeslib.as_array(pm, shape=(rows, d.n_steps, d.d_emb)).copy()
        ag = np.ctypeslib.as_array(pa, shape=(rows, d.n_feat)).copy()
        return lg, mk, ag

    def result_compact(self, ticket: int):
        """Copies of a completed request's compact step masks (counts
        [rows, n_steps], cols and vals [rows, n_steps, slots]), or None when
        its batch was sent densely."""
        _, _, model, rows = self._keep[ticket]
        d = self.models[model].dims
        pc, pcol = ctypes.POINTER(ctypes.c_uint8)(), ctypes.POINTER(ctypes.c_uint16)()
        pv = ctypes.POINTER(ctypes.c_float)()
        slots, r = ctypes.c_int(), ctypes.c_int64()
        _check(lib().tabnet_server_result_compact(self._h, ticket, ctypes.byref(pc), ctypes.byref(pcol),
                                                  ctypes.byref(pv), ctypes.byref(slots), ctypes.byref(r)),
               "tabnet_server_result_compact")
        if slots.value == 0:
            return None
        k = slots.value
        return (np.ctypeslib.as_array(pc, shape=(rows, d.n_steps)).copy(),
                np.ctypeslib.as_array(pcol, shape=(rows, d.n_steps, k)).copy(),
                np.ctypeslib.as_array(pv, shape=(rows, d.n_steps, k)).copy())

    def release(self, ticket: int) -> None:
        _check(lib().tabnet_server_release(self._h, ticket), "tabnet_server_release")
        self._keep.pop(ticket, None)

    def poll(self, max_tickets: int = 4096):
        buf = (ctypes.c_uint64 * max_tickets)()
        n = ctypes.c_int()
        _check(lib().tabnet_server_poll(self._h, buf, max_tickets, ctypes.byref(n)), "tabnet_server_poll")
        return list(buf[:n.value])

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().tabnet_server_get_stats(self._h, ctypes.byref(st)), "tabnet_server_get_stats")
        return st.as_dict()

    def reset_stats(self) -> None:
        _check(lib().tabnet_server_reset_stats(self._h), "tabnet_server_reset_stats")

    def prepare_replay(self, requests):
        """The C request array for replay_prepared (marshalling only):
        requests is a list of (model, x_num, x_cat, arrival_s), numpy inputs."""
        arr = (ServerRequest * len(requests))()
        keep = []
        for i, (model, xn, xc, t) in enumerate(requests):
            xn = np.ascontiguousarray(xn, dtype=np.float32)
            xc = np.ascontiguousarray(xc, dtype=np.int32)
            keep.append((xn, xc))
            d = self.models[model].dims
            rows = xn.shape[0] if d.n_num else xc.shape[0]
            arr[i] = ServerRequest(model, _ptr(xn) if d.n_num else None, _ptr(xc) if d.n_cat else None, rows, t)
        return arr, keep

    def replay_prepared(self, prepared, release: bool = True, threads: int = 1, warmup: int = 0) -> None:
        arr, _ = prepared
        _check(lib().tabnet_server_replay(self._h, arr, len(arr), 1 if release else 0, threads, warmup),
               "tabnet_server_replay")

    def replay(self, requests, release: bool = True, threads: int = 1, warmup: int = 0) -> None:
        """requests: list of (model, x_num, x_cat, arrival_s) with numpy inputs;
        `threads` submitting threads (clients); the first `warmup` requests
        are left out of the latency statistics."""
        self.replay_prepared(self.prepare_replay(requests), release, threads, warmup)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tabnet_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mask_stats(agg, k: int, stream=None):
    """Per-feature mean, variance and top-k frequency of a [rows, d] float32
    CUDA tensor of aggregated masks (tabnet_mask_stats); returns three [d]
    float32 CUDA tensors."""
    import torch
    rows, d = agg.shape
    mean = torch.empty(d, dtype=torch.float32, device=agg.device)
    var = torch.empty_like(mean)
    frac = torch.empty_like(mean)
    _check(lib().tabnet_mask_stats(_ptr(agg), rows, d, k, _ptr(mean), _ptr(var), _ptr(frac), _stream(stream)),
           "tabnet_mask_stats")
    return mean, var, frac


def topk_agreement(agg_a, agg_b, k: int, stream=None):
    """Mean row-wise overlap of the top-k feature sets of two [rows, d]
    aggregates (tabnet_topk_agreement), as a one-element CUDA tensor."""
    import torch
    rows, d = agg_a.shape
    out = torch.empty(1, dtype=torch.float32, device=agg_a.device)
    _check(lib().tabnet_topk_agreement(_ptr(agg_a), _ptr(agg_b), rows, d, k, _ptr(out), _stream(stream)),
           "tabnet_topk_agreement")
    return out
