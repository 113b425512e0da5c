"""Python binding of libhp (ctypes, argument marshalling only).

Every step of the reconstruction runs in the library's CUDA kernels; this
module converts numpy arrays / torch tensors to pointers and back.  There is
no CPU fallback: importing it without a built ``libhp.so`` raises.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhp.so")

HP_OK, HP_EAGAIN, HP_ENOTREADY, HP_EINVAL, HP_EBADDIGI, HP_EDUP, HP_ECAPACITY, HP_ENOMEM, HP_ETIMEOUT, HP_ECUDA = \
    range(10)
HP_WANT_LABELS = 0x1
HP_INPUT_NOCOPY = 0x2
HP_KEEP_ON_DEVICE = 0x4
HP_LABELS_U16 = 0x8
HP_ALLOW_CPU = 0x10
HP_TRANSFER_CLUSTERS = 0x1
HP_TRANSFER_LABELS = 0x2

# Every function that include/hp.h declares.
EXPORTS = ("hp_status_string", "hp_create", "hp_destroy", "hp_enqueue_event", "hp_enqueue_batch", "hp_on_complete",
           "hp_event_query", "hp_fetch_clusters", "hp_release_event", "hp_event_device", "hp_event_stream",
           "hp_event_cuda_event", "hp_event_latency_ns", "hp_reconstruct_device", "hp_reconstruct_device_noalloc",
           "hp_get_stats",
           "hp_profile_enable", "hp_profile_read", "hp_debug_fail_allocations", "hp_serve_start", "hp_submit",
           "hp_serve_stop", "hp_serve_replay", "hp_set_geometry", "hp_enqueue_hits", "hp_fetch_hits",
           "hp_hits_device", "hp_graph_capture", "hp_graph_launch", "hp_graph_destroy", "hp_tuning_candidates",
           "hp_get_tuning", "hp_set_tuning", "hp_autotune", "hp_event_device_clusters", "hp_enqueue_transfer",
           "hp_debug_expire_waits", "hp_event_provenance", "hp_serve_trace_enable", "hp_serve_trace_read")


class HPError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("n_modules", ctypes.c_uint32), ("rows", ctypes.c_uint32),
                ("cols", ctypes.c_uint32), ("pixel_thr", ctypes.c_int32), ("cluster_thr", ctypes.c_int32),
                ("gain", ctypes.c_void_p), ("pedestal", ctypes.c_void_p), ("device_budget_bytes", ctypes.c_size_t),
                ("max_inflight", ctypes.c_uint32), ("n_streams", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class ClustersView(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint32), ("n_digis", ctypes.c_uint64), ("n_clusters", ctypes.c_uint64),
                ("tag", ctypes.c_uint64), ("cluster_offsets", ctypes.c_void_p), ("event_status", ctypes.c_void_p),
                ("module", ctypes.c_void_p), ("id", ctypes.c_void_p), ("charge", ctypes.c_void_p),
                ("npix", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("label", ctypes.c_void_p), ("label16", ctypes.c_void_p), ("item_first", ctypes.c_void_p)]


class DeviceClusters(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_uint64), ("module", ctypes.c_void_p), ("id", ctypes.c_void_p),
                ("charge", ctypes.c_void_p), ("npix", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("cluster_offsets", ctypes.c_void_p), ("event_status", ctypes.c_void_p),
                ("label", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "device_mallocs", "host_mallocs", "pool_hits", "device_bytes_in_use", "device_bytes_cached",
        "events_enqueued", "events_completed", "inflight", "h2d_bytes", "d2h_bytes", "kernel_launches",
        "serve_batches", "serve_requests", "consumer_stream_reuses", "consumer_stream_waits", "serve_submit_ns",
        "serve_launch_ns", "serve_complete_ns", "serve_max_batch")]


HP_STORE_BITMAP, HP_STORE_HASH = 0, 1


class Tuning(ctypes.Structure):
    _fields_ = [("tile_slots", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32), ("ticket_items", ctypes.c_uint32),
                ("warp_max", ctypes.c_uint32), ("label_store", ctypes.c_uint32), ("item_threads", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Provenance(ctypes.Structure):
    _fields_ = [("device_name", ctypes.c_char * 64), ("device", ctypes.c_int), ("cc_major", ctypes.c_int),
                ("cc_minor", ctypes.c_int), ("library", ctypes.c_char_p), ("path", ctypes.c_uint32),
                ("tuning", Tuning)]


PATHS = {1: "event", 2: "batch", 3: "serving", 4: "hits", 5: "transfer", 6: "cpu"}
HP_PATH_CPU = 6


class HitsView(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint32), ("n_hits", ctypes.c_uint64), ("tag", ctypes.c_uint64),
                ("hit_offsets", ctypes.c_void_p), ("event_status", ctypes.c_void_p), ("module", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_size_t), ("max_batch_events", ctypes.c_uint32),
                ("max_batch_digis", ctypes.c_uint64), ("max_inflight_batches", ctypes.c_uint32),
                ("max_pending", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


# hp_serve_trace_record as a numpy record
TRACE_DTYPE = np.dtype([("t_first_submit", np.uint64), ("t_admit", np.uint64), ("t_launched", np.uint64),
                        ("t_done_start", np.uint64), ("t_done_end", np.uint64), ("n_digis", np.uint64),
                        ("n_events", np.uint32), ("stream", np.uint32), ("t_pooled", np.uint64),
                        ("t_inputs", np.uint64), ("t_kernels", np.uint64), ("gpu_start", np.int64),
                        ("gpu_inputs", np.int64), ("gpu_kernels", np.int64), ("gpu_outputs", np.int64)])

CALLBACK = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int)

_lib = None
_lib_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libhp.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libhp.so not built at {path}; run paper_2004_04334_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, V, U32, U64, I = ctypes.POINTER, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        sig = {
            "hp_status_string": (ctypes.c_char_p, [I]),
            "hp_create": (I, [P(Config), P(V)]),
            "hp_destroy": (I, [V]),
            "hp_enqueue_event": (I, [V, V, V, U64, U64, U32, P(V)]),
            "hp_enqueue_batch": (I, [V, U32, V, V, V, U64, U32, P(V)]),
            "hp_on_complete": (I, [V, CALLBACK, V]),
            "hp_event_query": (I, [V]),
            "hp_fetch_clusters": (I, [V, P(ClustersView)]),
            "hp_release_event": (I, [V]),
            "hp_event_device": (I, [V]),
            "hp_event_stream": (V, [V]),
            "hp_event_cuda_event": (V, [V]),
            "hp_event_latency_ns": (U64, [V]),
            "hp_reconstruct_device": (I, [V, U32, U64, V, V, V, P(DeviceClusters), V]),
            "hp_reconstruct_device_noalloc": (I, [V, U32, U64, V, V, V, P(DeviceClusters), V]),
            "hp_get_stats": (I, [V, P(Stats)]),
            "hp_profile_enable": (I, [V, U32]),
            "hp_serve_trace_enable": (I, [V, U64]),
            "hp_serve_trace_read": (I, [V, V, U64, P(U64)]),
            "hp_profile_read": (I, [V, U32, P(ctypes.c_char_p), P(ctypes.c_double), P(U64), P(U32)]),
            "hp_debug_fail_allocations": (I, [V, U32]),
            "hp_debug_expire_waits": (I, [V, U32]),
            "hp_event_provenance": (I, [V, P(Provenance)]),
            "hp_serve_start": (I, [V, P(ServeConfig)]),
            "hp_submit": (I, [V, V, V, U64, U64, V, V, P(V)]),
            "hp_serve_stop": (I, [V]),
            "hp_serve_replay": (I, [V, U32, U64, V, V, U32, V, V, V, V, V, P(U64)]),
            "hp_set_geometry": (I, [V, V, V, ctypes.c_float, ctypes.c_float]),
            "hp_enqueue_hits": (I, [V, U32, P(V)]),
            "hp_fetch_hits": (I, [V, P(HitsView)]),
            "hp_hits_device": (I, [V, U32, U64, V, V, V, V, V, V, V, V]),
            "hp_graph_capture": (I, [V, U32, U64, V, V, V, P(DeviceClusters), P(V)]),
            "hp_graph_launch": (I, [V, V]),
            "hp_graph_destroy": (I, [V]),
            "hp_tuning_candidates": (I, [V, U32, P(Tuning), P(U32)]),
            "hp_event_device_clusters": (I, [V, P(DeviceClusters)]),
            "hp_enqueue_transfer": (I, [V, U32, P(V)]),
            "hp_get_tuning": (I, [V, U32, U64, P(Tuning)]),
            "hp_set_tuning": (I, [V, U32, U64, P(Tuning)]),
            "hp_autotune": (I, [V, U32, U64, V, V, V, P(DeviceClusters), U32, U32, P(ctypes.c_double), P(Tuning),
                                P(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(st: int) -> str:
    return load().hp_status_string(st).decode()


def _check(st: int, what: str):
    if st != HP_OK:
        raise HPError(st, what)


@dataclass
class Result:
    """Host copy of an event's clusters (see hp_clusters in include/hp.h)."""
    status: int
    n_events: int
    cluster_offsets: np.ndarray
    event_status: np.ndarray
    module: np.ndarray
    id: np.ndarray
    charge: np.ndarray
    npix: np.ndarray
    x: np.ndarray
    y: np.ndarray
    label: np.ndarray | None
    tag: int
    label16: np.ndarray | None = None     # HP_LABELS_U16: rank of the digi's cluster in its module
    item_first: np.ndarray | None = None  # HP_LABELS_U16: [E * M] first cluster of (e, m) from e's first

    @property
    def n_clusters(self) -> int:
        return len(self.id)

    def labels_from_compact(self, digi_offsets, modules) -> np.ndarray:
        """The int32 labels (cluster id, -1, -2) that the compact form
        stands for: digi i of event e on module m is in cluster
        cluster_offsets[e] + item_first[e * M + m] + label16[i]."""
        N = len(self.label16)
        M = len(self.item_first) // max(1, self.n_events)
        offs = np.asarray(digi_offsets, np.int64)
        ev = np.repeat(np.arange(self.n_events), np.diff(offs))
        l16 = self.label16.astype(np.int64)
        out = np.where(l16 == 0xFFFE, -2, -1).astype(np.int32)
        keep = l16 < 0xFFFE
        k = (self.cluster_offsets[ev[keep]].astype(np.int64) +
             self.item_first[ev[keep] * M + np.asarray(modules, np.int64)[keep]].astype(np.int64) + l16[keep])
        out[keep] = self.id[k]
        assert len(out) == N
        return out

    def event(self, e: int) -> "Result":
        a, b = int(self.cluster_offsets[e]), int(self.cluster_offsets[e + 1])
        return Result(int(self.event_status[e]), 1, np.array([0, b - a], np.uint64), self.event_status[e:e + 1],
                      self.module[a:b], self.id[a:b], self.charge[a:b], self.npix[a:b], self.x[a:b], self.y[a:b],
                      None, self.tag)


@dataclass
class HitsResult:
    """Host copy of a hits event (see hp_hits in include/hp.h)."""
    status: int
    n_events: int
    hit_offsets: np.ndarray
    event_status: np.ndarray
    module: np.ndarray
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    tag: int

    @property
    def n_hits(self) -> int:
        return len(self.x)


def _arr(ptr, n, dtype, copy=True):
    if n == 0 or not ptr:
        return np.empty(0, dtype)
    buf = (ctypes.c_char * (n * np.dtype(dtype).itemsize)).from_address(ptr)
    a = np.frombuffer(buf, dtype=dtype, count=n)
    return a.copy() if copy else a


# Python-side completion dispatch: one C callback for all events.
_events: dict = {}
_events_lock = threading.Lock()
_ids = itertools.count(1)


@CALLBACK
def _on_complete(user, ev, st):
    with _events_lock:
        e = _events.get(user)
    if e is not None:
        e._complete(st)


class Event:
    """An enqueued event or batch (a Product<T>-like handle)."""

    def __init__(self, ctx: "Context", handle: int, n_events: int, n_digis: int):
        self._ctx = ctx
        self._h = ctypes.c_void_p(handle)
        self.n_events = n_events
        self.n_digis = n_digis
        self._done = threading.Event()
        self._status = None
        self._callbacks = []
        self._cb_lock = threading.Lock()
        self._id = next(_ids)
        self._released = False
        with _events_lock:
            _events[self._id] = self
        _check(ctx._lib.hp_on_complete(self._h, _on_complete, ctypes.c_void_p(self._id)), "hp_on_complete")

    def _complete(self, st: int):
        with self._cb_lock:
            self._status = st
            cbs = list(self._callbacks)
        self._done.set()
        for fn in cbs:
            fn(self, st)

    def on_complete(self, fn):
        """fn(event, status) runs on the CUDA host-function thread (or here if done)."""
        with self._cb_lock:
            if self._status is None:
                self._callbacks.append(fn)
                return
        fn(self, self._status)

    def query(self) -> int:
        return self._ctx._lib.hp_event_query(self._h)

    def wait(self, timeout: float | None = None) -> int:
        if not self._done.wait(timeout):
            raise TimeoutError("event did not complete")
        return self._status

    @property
    def latency_ns(self) -> int:
        return int(self._ctx._lib.hp_event_latency_ns(self._h))

    @property
    def device(self) -> int:
        return int(self._ctx._lib.hp_event_device(self._h))

    @property
    def stream(self) -> int:
        return int(self._ctx._lib.hp_event_stream(self._h) or 0)

    def provenance(self) -> dict:
        """Device, library build, path and clustering settings that made this product."""
        p = Provenance()
        _check(self._ctx._lib.hp_event_provenance(self._h, ctypes.byref(p)), "hp_event_provenance")
        return {"device_name": p.device_name.decode(), "device": p.device, "cc": (p.cc_major, p.cc_minor),
                "library": p.library.decode() if p.library else "", "path": PATHS.get(p.path, str(p.path)),
                "tuning": p.tuning.as_dict()}

    def fetch(self, copy: bool = True) -> Result:
        """The event's results.  copy=False returns numpy views of the
        library's pinned buffers, valid only until release()."""
        v = ClustersView()
        st = self._ctx._lib.hp_fetch_clusters(self._h, ctypes.byref(v))
        if st == HP_ENOTREADY:
            raise HPError(st, "hp_fetch_clusters")
        if st == HP_EINVAL:
            raise HPError(st, "hp_fetch_clusters")
        E, N, C = v.n_events, v.n_digis, v.n_clusters
        a = lambda p, n, t: _arr(p, n, t, copy)  # noqa: E731
        return Result(st, E, a(v.cluster_offsets, E + 1, np.uint64), a(v.event_status, E, np.int32),
                      a(v.module, C, np.uint32), a(v.id, C, np.int32), a(v.charge, C, np.int32),
                      a(v.npix, C, np.int32), a(v.x, C, np.float32), a(v.y, C, np.float32),
                      a(v.label, N, np.int32) if v.label else None, int(v.tag),
                      a(v.label16, N, np.uint16) if v.label16 else None,
                      a(v.item_first, E * self._ctx.n_modules, np.uint32) if v.item_first else None)

    def transfer(self, what: int = HP_TRANSFER_CLUSTERS) -> "Event":
        """Queue the transfer module of a HP_KEEP_ON_DEVICE event (hp_enqueue_transfer)."""
        h = ctypes.c_void_p()
        _check(self._ctx._lib.hp_enqueue_transfer(self._h, what, ctypes.byref(h)), "hp_enqueue_transfer")
        return Event(self._ctx, h.value, self.n_events, self.n_digis)

    def device_clusters(self) -> DeviceClusters:
        """Device addresses of a HP_KEEP_ON_DEVICE event's results (hp_event_device_clusters)."""
        v = DeviceClusters()
        _check(self._ctx._lib.hp_event_device_clusters(self._h, ctypes.byref(v)), "hp_event_device_clusters")
        return v

    def hits(self) -> "HitsEvent":
        """Queue the clusters -> hits consumer of this event (hp_enqueue_hits)."""
        h = ctypes.c_void_p()
        _check(self._ctx._lib.hp_enqueue_hits(self._h, 0, ctypes.byref(h)), "hp_enqueue_hits")
        return HitsEvent(self._ctx, h.value, self.n_events, self.n_digis)

    def release(self):
        if not self._released:
            self._released = True
            _check(self._ctx._lib.hp_release_event(self._h), "hp_release_event")
            with _events_lock:
                _events.pop(self._id, None)


class HitsEvent(Event):
    """A hits event: the consumer of a clusters event (hp_enqueue_hits)."""

    def fetch(self, copy: bool = True) -> HitsResult:
        v = HitsView()
        st = self._ctx._lib.hp_fetch_hits(self._h, ctypes.byref(v))
        if st in (HP_ENOTREADY, HP_EINVAL):
            raise HPError(st, "hp_fetch_hits")
        E, H = v.n_events, v.n_hits
        a = lambda p, n, t: _arr(p, n, t, copy)  # noqa: E731
        return HitsResult(st, E, a(v.hit_offsets, E + 1, np.uint64), a(v.event_status, E, np.int32),
                          a(v.module, H, np.uint32), a(v.x, H, np.float32), a(v.y, H, np.float32),
                          a(v.z, H, np.float32), int(v.tag))

    def hits(self):
        raise HPError(HP_EINVAL, "hp_enqueue_hits: a hits event is not a clusters product")


class Context:
    """A libhp context on one device (see hp_create)."""

    def __init__(self, n_modules, gain, pedestal, *, device=0, rows=160, cols=416, pixel_thr=1000,
                 cluster_thr=4000, budget_bytes=0, max_inflight=0, n_streams=0, want_labels=False,
                 allow_cpu=False):
        self._lib = load()
        self.n_modules = int(n_modules)
        self.gain = np.ascontiguousarray(gain, np.int32)
        self.pedestal = np.ascontiguousarray(pedestal, np.int32)
        if len(self.gain) != self.n_modules or len(self.pedestal) != self.n_modules:
            raise ValueError("gain/pedestal must have n_modules entries")
        cfg = Config(device, self.n_modules, rows, cols, pixel_thr, cluster_thr, self.gain.ctypes.data,
                     self.pedestal.ctypes.data, budget_bytes, max_inflight, n_streams,
                     (HP_WANT_LABELS if want_labels else 0) | (HP_ALLOW_CPU if allow_cpu else 0))
        h = ctypes.c_void_p()
        _check(self._lib.hp_create(ctypes.byref(cfg), ctypes.byref(h)), "hp_create")
        self._h = h
        self.device = device

    def close(self):
        if self._h:
            st = self._lib.hp_destroy(self._h)
            self._h = None
            _check(st, "hp_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def enqueue_event(self, words, modules, tag=0, flags=0) -> Event:
        words = np.ascontiguousarray(words, np.uint32)
        modules = np.ascontiguousarray(modules, np.uint16)
        if len(words) != len(modules):
            raise ValueError("words and modules differ in length")
        h = ctypes.c_void_p()
        _check(self._lib.hp_enqueue_event(self._h, words.ctypes.data, modules.ctypes.data, len(words), tag, flags,
                                          ctypes.byref(h)), "hp_enqueue_event")
        return Event(self, h.value, 1, len(words))

    def try_enqueue_batch(self, words, modules, offsets, tag=0, flags=0):
        """As enqueue_batch, but returns (status, event-or-None) instead of raising."""
        offsets = np.ascontiguousarray(offsets, np.uint64)
        E = len(offsets) - 1
        h = ctypes.c_void_p()
        wp = words.data_ptr() if hasattr(words, "data_ptr") else np.ascontiguousarray(words, np.uint32).ctypes.data
        mp = modules.data_ptr() if hasattr(modules, "data_ptr") else \
            np.ascontiguousarray(modules, np.uint16).ctypes.data
        st = self._lib.hp_enqueue_batch(self._h, E, offsets.ctypes.data, wp, mp, tag, flags, ctypes.byref(h))
        if st != HP_OK:
            return st, None
        return st, Event(self, h.value, E, int(offsets[-1]))

    def enqueue_batch(self, words, modules, offsets, tag=0, flags=0) -> Event:
        if not hasattr(words, "data_ptr"):
            words = np.ascontiguousarray(words, np.uint32)
            modules = np.ascontiguousarray(modules, np.uint16)
        st, ev = self.try_enqueue_batch(words, modules, offsets, tag, flags)
        _check(st, "hp_enqueue_batch")
        return ev

    def reconstruct_device(self, n_events, n_digis, d_offsets, d_words, d_modules, out: "DeviceOutputs",
                           stream: int = 0):
        """Queue the device-resident pass (all pointers are device addresses)."""
        _check(self._lib.hp_reconstruct_device(self._h, n_events, n_digis, d_offsets, d_words, d_modules,
                                               ctypes.byref(out.struct), ctypes.c_void_p(stream)),
               "hp_reconstruct_device")

    def graph_capture(self, n_events, n_digis, d_offsets, d_words, d_modules, out: "DeviceOutputs") -> "Graph":
        """Capture one device-resident pass into a CUDA graph (hp_graph_capture)."""
        h = ctypes.c_void_p()
        _check(self._lib.hp_graph_capture(self._h, n_events, n_digis, d_offsets, d_words, d_modules,
                                          ctypes.byref(out.struct), ctypes.byref(h)), "hp_graph_capture")
        return Graph(self, h.value)

    def tuning_candidates(self) -> list:
        """The autotuner's search space on this device (list of dicts)."""
        n = ctypes.c_uint32()
        _check(self._lib.hp_tuning_candidates(self._h, 0, None, ctypes.byref(n)), "hp_tuning_candidates")
        arr = (Tuning * max(1, n.value))()
        _check(self._lib.hp_tuning_candidates(self._h, n.value, arr, ctypes.byref(n)), "hp_tuning_candidates")
        return [arr[i].as_dict() for i in range(n.value)]

    def get_tuning(self, n_events, n_digis) -> dict:
        """The clustering-kernel settings a launch of this shape uses."""
        t = Tuning()
        _check(self._lib.hp_get_tuning(self._h, n_events, n_digis, ctypes.byref(t)), "hp_get_tuning")
        return t.as_dict()

    def try_set_tuning(self, n_events, n_digis, tuning) -> int:
        """Set (dict) or clear (None) the settings of this shape's bucket; returns the status."""
        if tuning is None:
            return self._lib.hp_set_tuning(self._h, n_events, n_digis, None)
        t = Tuning(**dict({"label_store": HP_STORE_BITMAP, "item_threads": 512}, **tuning))
        return self._lib.hp_set_tuning(self._h, n_events, n_digis, ctypes.byref(t))

    def set_tuning(self, n_events, n_digis, tuning):
        _check(self.try_set_tuning(n_events, n_digis, tuning), "hp_set_tuning")

    def autotune(self, n_events, n_digis, d_offsets, d_words, d_modules, out: "DeviceOutputs", reps: int = 3):
        """Time every candidate on these device inputs and keep the fastest for
        the shape's bucket.  Returns (best dict, best ms, [ms per candidate])."""
        n = len(self.tuning_candidates())
        ms = (ctypes.c_double * max(1, n))()
        best = Tuning()
        best_ms = ctypes.c_double()
        _check(self._lib.hp_autotune(self._h, n_events, n_digis, d_offsets, d_words, d_modules,
                                     ctypes.byref(out.struct), reps, n, ms, ctypes.byref(best),
                                     ctypes.byref(best_ms)), "hp_autotune")
        return best.as_dict(), best_ms.value, [ms[i] for i in range(n)]

    def set_geometry(self, origin, rot, pitch_row, pitch_col):
        """Install the module placement for hits (origin float[M,3] cm, rot float[M,3,3])."""
        origin = np.ascontiguousarray(origin, np.float32).reshape(-1)
        rot = np.ascontiguousarray(rot, np.float32).reshape(-1)
        if len(origin) != 3 * self.n_modules or len(rot) != 9 * self.n_modules:
            raise ValueError("origin/rot must have n_modules entries")
        _check(self._lib.hp_set_geometry(self._h, origin.ctypes.data, rot.ctypes.data, pitch_row, pitch_col),
               "hp_set_geometry")

    def hits_device(self, n_events, capacity, d_cluster_offsets, d_module, d_x, d_y, d_hx, d_hy, d_hz,
                    stream: int = 0):
        """Queue the device-resident clusters -> hits pass (device addresses)."""
        _check(self._lib.hp_hits_device(self._h, n_events, capacity, d_cluster_offsets, d_module, d_x, d_y, d_hx,
                                        d_hy, d_hz, ctypes.c_void_p(stream)), "hp_hits_device")

    def serve_start(self, budget_bytes=0, max_batch_events=0, max_batch_digis=0, max_inflight_batches=0,
                    max_pending=0, want_labels=False, nocopy=False, compact_labels=False):
        """Start the continuous-batching serving loop (see hp_serve_start)."""
        cfg = ServeConfig(budget_bytes, max_batch_events, max_batch_digis, max_inflight_batches, max_pending,
                          (HP_WANT_LABELS if want_labels else 0) | (HP_INPUT_NOCOPY if nocopy else 0) |
                          (HP_LABELS_U16 if compact_labels else 0))
        _check(self._lib.hp_serve_start(self._h, ctypes.byref(cfg)), "hp_serve_start")

    def try_submit(self, words, modules, tag=0):
        """Queue one event for serving: (status, Event-or-None)."""
        words = np.ascontiguousarray(words, np.uint32)
        modules = np.ascontiguousarray(modules, np.uint16)
        h = ctypes.c_void_p()
        st = self._lib.hp_submit(self._h, words.ctypes.data, modules.ctypes.data, len(words), tag, None, None,
                                 ctypes.byref(h))
        if st != HP_OK:
            return st, None
        return st, Event(self, h.value, 1, len(words))

    def submit(self, words, modules, tag=0) -> "Event":
        st, ev = self.try_submit(words, modules, tag)
        _check(st, "hp_submit")
        return ev

    def serve_replay(self, pool, arrival_s, event_index, n_threads=4):
        """Replay an arrival schedule with native submitter threads (see
        hp_serve_replay).  pool: list of (words, modules).  Returns
        (latency seconds[n], status[n], span seconds)."""
        ws = [np.ascontiguousarray(w, np.uint32) for w, _ in pool]
        ms = [np.ascontiguousarray(m, np.uint16) for _, m in pool]
        P = len(pool)
        pw = (ctypes.c_void_p * P)(*[w.ctypes.data for w in ws])
        pm = (ctypes.c_void_p * P)(*[m.ctypes.data for m in ms])
        pn = np.array([len(w) for w in ws], np.uint64)
        arr = np.ascontiguousarray(np.round(np.asarray(arrival_s) * 1e9), np.uint64)
        idx = np.ascontiguousarray(event_index, np.uint32)
        n = len(arr)
        lat = np.zeros(n, np.uint64)
        st = np.zeros(n, np.int32)
        span = ctypes.c_uint64()
        _check(self._lib.hp_serve_replay(self._h, n_threads, n, arr.ctypes.data, idx.ctypes.data, P, pw, pm,
                                         pn.ctypes.data, lat.ctypes.data, st.ctypes.data, ctypes.byref(span)),
               "hp_serve_replay")
        return lat * 1e-9, st, span.value * 1e-9

    def serve_trace_enable(self, cap: int):
        """Record the next `cap` serving batches (hp_serve_trace_enable; 0 stops and clears)."""
        _check(self._lib.hp_serve_trace_enable(self._h, cap), "hp_serve_trace_enable")

    def serve_trace(self) -> np.ndarray:
        """The serving trace records (hp_serve_trace_read), as a structured array."""
        dt = TRACE_DTYPE
        n = ctypes.c_uint64()
        _check(self._lib.hp_serve_trace_read(self._h, None, 0, ctypes.byref(n)), "hp_serve_trace_read")
        out = np.zeros(n.value, dt)
        if n.value:
            _check(self._lib.hp_serve_trace_read(self._h, out.ctypes.data, n.value, ctypes.byref(n)),
                   "hp_serve_trace_read")
        return out[:n.value]

    def serve_stop(self):
        """Launch what is queued and wait for every batch."""
        _check(self._lib.hp_serve_stop(self._h), "hp_serve_stop")

    def debug_expire_waits(self, count: int):
        """Test hook: the next `count` launches let their bounded device wait expire (HP_ETIMEOUT)."""
        _check(self._lib.hp_debug_expire_waits(self._h, count), "hp_debug_expire_waits")

    def debug_fail_allocations(self, count: int):
        _check(self._lib.hp_debug_fail_allocations(self._h, count), "hp_debug_fail_allocations")

    def profile_enable(self, max_launches: int):
        """Record CUDA events around each kernel of the next max_launches launches."""
        _check(self._lib.hp_profile_enable(self._h, max_launches), "hp_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} of the timed launches (blocks)."""
        cap = 16
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_uint64 * cap)()
        n = ctypes.c_uint32()
        _check(self._lib.hp_profile_read(self._h, cap, names, ms, cnt, ctypes.byref(n)), "hp_profile_read")
        return {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(min(cap, n.value))}

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.hp_get_stats(self._h, ctypes.byref(s)), "hp_get_stats")
        return {n: int(getattr(s, n)) for n, _ in Stats._fields_}


class Graph:
    """A captured device-resident pass (see hp_graph_capture)."""

    def __init__(self, ctx: "Context", handle: int):
        self._ctx = ctx
        self._h = ctypes.c_void_p(handle)

    def launch(self, stream: int = 0):
        _check(self._ctx._lib.hp_graph_launch(self._h, ctypes.c_void_p(stream)), "hp_graph_launch")

    def destroy(self):
        if self._h:
            h, self._h = self._h, None
            _check(self._ctx._lib.hp_graph_destroy(h), "hp_graph_destroy")


class DeviceOutputs:
    """Caller-owned device output tensors for Context.reconstruct_device (torch)."""

    def __init__(self, n_events: int, n_digis: int, device, capacity: int | None = None, labels: bool = True):
        import torch
        cap = max(1, n_digis if capacity is None else capacity)
        kw = dict(device=device)
        self.module = torch.empty(cap, dtype=torch.int32, **kw)
        self.id = torch.empty(cap, dtype=torch.int32, **kw)
        self.charge = torch.empty(cap, dtype=torch.int32, **kw)
        self.npix = torch.empty(cap, dtype=torch.int32, **kw)
        self.x = torch.empty(cap, dtype=torch.float32, **kw)
        self.y = torch.empty(cap, dtype=torch.float32, **kw)
        self.cluster_offsets = torch.empty(n_events + 1, dtype=torch.int64, **kw)
        self.event_status = torch.empty(n_events, dtype=torch.int32, **kw)
        self.label = torch.empty(max(1, n_digis), dtype=torch.int32, **kw) if labels else None
        self.struct = DeviceClusters(cap, self.module.data_ptr(), self.id.data_ptr(), self.charge.data_ptr(),
                                     self.npix.data_ptr(), self.x.data_ptr(), self.y.data_ptr(),
                                     self.cluster_offsets.data_ptr(), self.event_status.data_ptr(),
                                     self.label.data_ptr() if labels else None)

    def to_result(self, n_digis: int) -> Result:
        offs = self.cluster_offsets.cpu().numpy().astype(np.uint64)
        C = int(offs[-1])
        es = self.event_status.cpu().numpy()
        return Result(int(next((s for s in es if s), 0)), len(es), offs, es,
                      self.module[:C].cpu().numpy().astype(np.uint32), self.id[:C].cpu().numpy(),
                      self.charge[:C].cpu().numpy(), self.npix[:C].cpu().numpy(), self.x[:C].cpu().numpy(),
                      self.y[:C].cpu().numpy(),
                      self.label[:n_digis].cpu().numpy() if self.label is not None else None, 0)
