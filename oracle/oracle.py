"""TEST INFRASTRUCTURE — Python front end of the CPU oracle (``hp_oracle.c``).

The oracle is the plain, single-threaded CPU definition of silicon-pixel local
reconstruction (decode, calibrate and threshold, 8-connected clustering per
module, charge and charge-weighted centroid, cluster threshold, ordered
output).  Only the tests, the smoke check and the benchmark's CPU-baseline leg
use it; the GPU library never imports, links or calls it, and the two share no
code.  ``build()`` compiles ``hp_oracle.c`` with gcc into ``oracle/_lib``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hp_oracle.c")
_SO = os.path.join(_HERE, "_lib", "libhp_oracle.so")
_lock = threading.Lock()
_lib = None

# Status codes returned by the oracle (numbering chosen to line up with the
# library's public status enum so that tests can compare them directly).
OK, EINVAL, EBADDIGI, EDUP, ECAPACITY, ENOMEM = 0, 3, 4, 5, 6, 7
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", EBADDIGI: "EBADDIGI", EDUP: "EDUP", ECAPACITY: "ECAPACITY",
                ENOMEM: "ENOMEM"}

ROWS, COLS = 160, 416
PIXEL_THR, CLUSTER_THR = 1000, 4000


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _Geometry(ctypes.Structure):
    _fields_ = [("n_modules", ctypes.c_uint32), ("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32),
                ("pixel_thr", ctypes.c_int32), ("cluster_thr", ctypes.c_int32),
                ("gain", ctypes.c_void_p), ("pedestal", ctypes.c_void_p)]


class _Out(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_uint64), ("n_clusters", ctypes.c_uint64),
                ("module", ctypes.c_void_p), ("id", ctypes.c_void_p), ("charge", ctypes.c_void_p),
                ("npix", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("label", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_event.argtypes = [ctypes.POINTER(_Geometry), ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(_Out)]
            lib.oracle_event.restype = ctypes.c_int
            lib.oracle_batch.argtypes = [ctypes.POINTER(_Geometry), ctypes.c_uint32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Out),
                                         ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_batch.restype = ctypes.c_int
            lib.oracle_hits.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
            lib.oracle_hits.restype = None
            _lib = lib
    return _lib


@dataclass
class Clusters:
    """Reconstructed clusters of one event or a batch (cluster arrays ordered
    by event, then module, then id)."""
    status: int
    module: np.ndarray   # uint32[C]
    id: np.ndarray       # int32[C]   smallest linear pixel index row*cols+col
    charge: np.ndarray   # int32[C]
    npix: np.ndarray     # int32[C]
    x: np.ndarray        # float64[C] charge-weighted mean row
    y: np.ndarray        # float64[C] charge-weighted mean column
    label: np.ndarray    # int32[N]
    cluster_offsets: np.ndarray  # uint64[E+1]
    event_status: np.ndarray     # int32[E]

    @property
    def n_clusters(self) -> int:
        return len(self.id)

    def event(self, e: int) -> "Clusters":
        a, b = int(self.cluster_offsets[e]), int(self.cluster_offsets[e + 1])
        return Clusters(int(self.event_status[e]), self.module[a:b], self.id[a:b], self.charge[a:b],
                        self.npix[a:b], self.x[a:b], self.y[a:b], self.label,
                        np.array([0, b - a], np.uint64), self.event_status[e:e + 1])


def reconstruct_batch(words, modules, offsets, n_modules, gain, pedestal, pixel_thr=PIXEL_THR,
                      cluster_thr=CLUSTER_THR, rows=ROWS, cols=COLS) -> Clusters:
    """Run the oracle over a batch (events [offsets[e], offsets[e+1]))."""
    lib = _load()
    words = np.ascontiguousarray(words, np.uint32)
    modules = np.ascontiguousarray(modules, np.uint16)
    offsets = np.ascontiguousarray(offsets, np.uint64)
    gain = np.ascontiguousarray(gain, np.int32)
    pedestal = np.ascontiguousarray(pedestal, np.int32)
    assert len(gain) == n_modules and len(pedestal) == n_modules
    n = int(offsets[-1]) if len(offsets) else 0
    E = len(offsets) - 1
    cap = max(n, 1)
    mod = np.empty(cap, np.uint32)
    cid = np.empty(cap, np.int32)
    chg = np.empty(cap, np.int32)
    npx = np.empty(cap, np.int32)
    x = np.empty(cap, np.float64)
    y = np.empty(cap, np.float64)
    label = np.empty(max(n, 1), np.int32)
    coff = np.zeros(E + 1, np.uint64)
    est = np.zeros(max(E, 1), np.int32)
    g = _Geometry(n_modules, rows, cols, pixel_thr, cluster_thr, gain.ctypes.data, pedestal.ctypes.data)
    o = _Out(cap, 0, mod.ctypes.data, cid.ctypes.data, chg.ctypes.data, npx.ctypes.data, x.ctypes.data,
             y.ctypes.data, label.ctypes.data)
    st = lib.oracle_batch(ctypes.byref(g), E, offsets.ctypes.data, words.ctypes.data, modules.ctypes.data,
                          ctypes.byref(o), coff.ctypes.data, est.ctypes.data)
    c = int(o.n_clusters)
    return Clusters(int(st), mod[:c].copy(), cid[:c].copy(), chg[:c].copy(), npx[:c].copy(), x[:c].copy(),
                    y[:c].copy(), label[:n].copy(), coff, est[:E].copy())


def reconstruct_event(words, modules, n_modules, gain, pedestal, **kw) -> Clusters:
    """Run the oracle on one event."""
    n = len(words)
    return reconstruct_batch(words, modules, np.array([0, n], np.uint64), n_modules, gain, pedestal, **kw)


def reconstruct_workload(w, events=None, **kw) -> Clusters:
    """Run the oracle on a ``synth.Workload`` (or a subset of its events)."""
    if events is not None:
        w = w.subset(events)
    return reconstruct_batch(w.words, w.modules, w.offsets, w.n_modules, w.gain, w.pedestal, **kw)


def hits(module, x, y, origin, rot, pitch_row, pitch_col, rows=ROWS, cols=COLS):
    """Global hit positions (double[n] x 3) of clusters (module, centroid x, y)."""
    lib = _load()
    module = np.ascontiguousarray(module, np.uint32)
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    origin = np.ascontiguousarray(origin, np.float32)
    rot = np.ascontiguousarray(rot, np.float32)
    n = len(module)
    gx, gy, gz = (np.empty(n, np.float64) for _ in range(3))
    lib.oracle_hits(rows, cols, pitch_row, pitch_col, origin.ctypes.data, rot.ctypes.data, n, module.ctypes.data,
                    x.ctypes.data, y.ctypes.data, gx.ctypes.data, gy.ctypes.data, gz.ctypes.data)
    return gx, gy, gz
