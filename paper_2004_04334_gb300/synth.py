"""Seeded synthetic workloads for silicon-pixel local reconstruction.

This module only *generates inputs*: packed digi words, 16-bit module ids,
per-event offsets and per-module gain/pedestal tables.  It holds none of the
reconstruction arithmetic, so both the CPU oracle and the GPU library consume
exactly the same bytes from here.  The generator itself is plain C
(``synth.c``), compiled on first use with gcc.

Digi word layout (the input encoding of the workload): bits 0-7 row (0-159),
bits 8-16 column (0-415), bits 17-24 ADC (1-255), bits 25-31 zero.

Named workloads (module geometry 160 x 416 everywhere):

``tiny``        one event, 64 modules, Poisson(3) random-walk blobs of 1-12
                pixels, Poisson(2) noise pixels per module (~1.4k digis).
``full``        one event, 1856 modules, blobs of 1-20 pixels, the 20 inner
                modules at 4x the cluster rate, noise = 1% of the event's digis;
                the cluster rate is scaled so that E[N] ~ 60k digis.
``full_literal`` as ``full`` but with 12 clusters per module and 1% noise
                occupancy of every module (~1.5M digis).
``batched``     256 events on the 64-module geometry, per-event cluster rate
                scaled so that digi counts are uniform in 10k-200k (~27M).
``occupancy``   64 events, 1856 modules, Poisson(80) clusters of 1-40 pixels
                (10% of them 1x30 column streaks), 2% of modules "hot" at 20%
                occupancy (~3.6M digis per event).
``serving``     event sizes lognormal (median 80k, sigma 0.8, capped 500k),
                generated as ``tiny`` with the cluster rate scaled to the size.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, replace

import numpy as np

ROWS, COLS = 160, 416
BASE_SEED = 2004_04334 * 10

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "libhp_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to this file."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _EventCfg(ctypes.Structure):
    _fields_ = [
        ("n_modules", ctypes.c_uint32), ("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32),
        ("lambda_clusters", ctypes.c_double),
        ("n_inner", ctypes.c_uint32), ("inner_factor", ctypes.c_double),
        ("size_min", ctypes.c_uint32), ("size_max", ctypes.c_uint32), ("walk_cap", ctypes.c_uint32),
        ("streak_frac", ctypes.c_double), ("streak_len", ctypes.c_uint32),
        ("lambda_noise", ctypes.c_double),
        ("hot_frac", ctypes.c_double), ("hot_occupancy", ctypes.c_double),
        ("adc_mu", ctypes.c_double), ("adc_sigma", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.synth_event.argtypes = [P(_EventCfg), ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_uint64]
            lib.synth_event.restype = ctypes.c_int64
            lib.synth_calib.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_calib.restype = None
            for fn in (lib.synth_uniform, lib.synth_lognormal):
                fn.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                               ctypes.c_void_p]
                fn.restype = None
            lib.synth_exponential.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                              ctypes.c_void_p]
            lib.synth_exponential.restype = None
            lib.synth_barrel_geometry.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_barrel_geometry.restype = None
            lib.synth_child_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_child_seed.restype = ctypes.c_uint64
            _lib = lib
    return _lib


@dataclass(frozen=True)
class EventCfg:
    """Generation parameters of one event (per module unless stated)."""
    n_modules: int = 64
    lambda_clusters: float = 3.0
    n_inner: int = 0
    inner_factor: float = 1.0
    size_min: int = 1
    size_max: int = 12
    walk_cap: int = 64
    streak_frac: float = 0.0
    streak_len: int = 30
    lambda_noise: float = 2.0
    hot_frac: float = 0.0
    hot_occupancy: float = 0.0
    adc_mu: float = 3.5
    adc_sigma: float = 0.6

    def _c(self) -> _EventCfg:
        return _EventCfg(self.n_modules, ROWS, COLS, self.lambda_clusters, self.n_inner, self.inner_factor,
                         self.size_min, self.size_max, self.walk_cap, self.streak_frac, self.streak_len,
                         self.lambda_noise, self.hot_frac, self.hot_occupancy, self.adc_mu, self.adc_sigma)

    def expected_digis(self) -> float:
        """Rough upper estimate of E[N] (used to size buffers and scale rates)."""
        eff = self.n_modules + self.n_inner * (self.inner_factor - 1.0)
        blob = 0.5 * (self.size_min + self.size_max)
        per_cl = self.streak_frac * self.streak_len + (1.0 - self.streak_frac) * blob
        hot = self.hot_frac * self.n_modules * self.hot_occupancy * ROWS * COLS
        return eff * self.lambda_clusters * per_cl + self.n_modules * self.lambda_noise + hot


TINY = EventCfg()
FULL_LITERAL = EventCfg(n_modules=1856, lambda_clusters=12.0, n_inner=20, inner_factor=4.0, size_max=20,
                        lambda_noise=0.01 * ROWS * COLS)
# "about 60k digis": the cluster rate is scaled by a common factor and the noise is
# 1% of the event's digis (0.99 * 60000 cluster digis over 1916 module-equivalents
# of mean blob size 10.5; 600 noise digis over 1856 modules).
FULL = replace(FULL_LITERAL, lambda_clusters=0.99 * 60000 / (1916 * 10.5), lambda_noise=600 / 1856)
OCCUPANCY = EventCfg(n_modules=1856, lambda_clusters=80.0, size_max=40, walk_cap=160, streak_frac=0.1,
                     streak_len=30, lambda_noise=0.0, hot_frac=0.02, hot_occupancy=0.2)


def child_seed(base: int, index: int) -> int:
    return int(_load().synth_child_seed(base & (2**64 - 1), index))


def make_event(cfg: EventCfg, seed: int):
    """Return (words uint32[N], modules uint16[N]) for one event."""
    lib = _load()
    cap = int(cfg.expected_digis() * 1.5) + 4096
    c = cfg._c()
    while True:
        words = np.empty(cap, np.uint32)
        mods = np.empty(cap, np.uint16)
        n = lib.synth_event(ctypes.byref(c), seed & (2**64 - 1), words.ctypes.data, mods.ctypes.data, cap)
        if n >= 0:
            return words[:n].copy(), mods[:n].copy()
        cap *= 2


def calibration(n_modules: int, seed: int):
    """Per-module int32 gain in [60, 80] e/ADC and pedestal in [0, 200] e."""
    lib = _load()
    gain = np.empty(n_modules, np.int32)
    ped = np.empty(n_modules, np.int32)
    lib.synth_calib(n_modules, seed & (2**64 - 1), 60, 80, 0, 200, gain.ctypes.data, ped.ctypes.data)
    return gain, ped


def uniform(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().synth_uniform(seed & (2**64 - 1), n, lo, hi, out.ctypes.data)
    return out


def lognormal(seed: int, n: int, mu: float, sigma: float) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().synth_lognormal(seed & (2**64 - 1), n, mu, sigma, out.ctypes.data)
    return out


def exponential(seed: int, n: int, rate: float) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().synth_exponential(seed & (2**64 - 1), n, rate, out.ctypes.data)
    return out


def scaled_tiny(target_digis: float) -> EventCfg:
    """The ``tiny`` recipe with its cluster rate scaled so that E[N] ~ target_digis."""
    per_module = target_digis / TINY.n_modules - TINY.lambda_noise
    return replace(TINY, lambda_clusters=max(0.0, per_module / (0.5 * (TINY.size_min + TINY.size_max))))


@dataclass
class Workload:
    """A batch of events sharing one module geometry and calibration."""
    name: str
    n_modules: int
    words: np.ndarray     # uint32[N_total]
    modules: np.ndarray   # uint16[N_total]
    offsets: np.ndarray   # uint64[E+1]
    gain: np.ndarray      # int32[M]
    pedestal: np.ndarray  # int32[M]

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_digis(self) -> int:
        return int(self.offsets[-1])

    def event(self, e: int):
        a, b = int(self.offsets[e]), int(self.offsets[e + 1])
        return self.words[a:b], self.modules[a:b]

    def subset(self, events) -> "Workload":
        ws, ms, offs = [], [], [0]
        for e in events:
            w, m = self.event(e)
            ws.append(w)
            ms.append(m)
            offs.append(offs[-1] + len(w))
        return Workload(self.name, self.n_modules, np.concatenate(ws) if ws else np.empty(0, np.uint32),
                        np.concatenate(ms) if ms else np.empty(0, np.uint16), np.asarray(offs, np.uint64),
                        self.gain, self.pedestal)


def _assemble(name, cfgs, seeds, n_modules, calib_seed):
    ws, ms = [], []
    offs = np.zeros(len(cfgs) + 1, np.uint64)
    for i, (cfg, s) in enumerate(zip(cfgs, seeds)):
        w, m = make_event(cfg, s)
        ws.append(w)
        ms.append(m)
        offs[i + 1] = offs[i] + len(w)
    gain, ped = calibration(n_modules, calib_seed)
    words = np.concatenate(ws) if ws else np.empty(0, np.uint32)
    mods = np.concatenate(ms) if ms else np.empty(0, np.uint16)
    return Workload(name, n_modules, words, mods, offs, gain, ped)


WORKLOADS = ("tiny", "full", "full_literal", "batched", "occupancy", "serving")
_CONFIG_INDEX = {"tiny": 1, "full": 2, "full_literal": 2, "batched": 3, "occupancy": 4, "serving": 5}


def workload(name: str, n_events: int | None = None, seed: int | None = None) -> Workload:
    """Build a named workload.  ``n_events`` truncates/extends the event count."""
    k = _CONFIG_INDEX[name]
    base = BASE_SEED + k if seed is None else seed
    calib_seed = child_seed(base, 1 << 40)
    if name in ("tiny", "full", "full_literal"):
        cfg = {"tiny": TINY, "full": FULL, "full_literal": FULL_LITERAL}[name]
        E = 1 if n_events is None else n_events
        return _assemble(name, [cfg] * E, [child_seed(base, e) for e in range(E)], cfg.n_modules, calib_seed)
    if name == "batched":
        E = 256 if n_events is None else n_events
        targets = uniform(child_seed(base, 1 << 41), E, 10_000, 200_000)
        cfgs = [scaled_tiny(t) for t in targets]
        return _assemble(name, cfgs, [child_seed(base, e) for e in range(E)], TINY.n_modules, calib_seed)
    if name == "occupancy":
        E = 64 if n_events is None else n_events
        return _assemble(name, [OCCUPANCY] * E, [child_seed(base, e) for e in range(E)], OCCUPANCY.n_modules,
                         calib_seed)
    if name == "serving":
        E = 1000 if n_events is None else n_events
        sizes = np.minimum(lognormal(child_seed(base, 1 << 41), E, np.log(80_000.0), 0.8), 500_000.0)
        cfgs = [scaled_tiny(t) for t in sizes]
        return _assemble(name, cfgs, [child_seed(base, e) for e in range(E)], TINY.n_modules, calib_seed)
    raise KeyError(name)


PITCH_ROW, PITCH_COL = 0.01, 0.015  # cm: 100 um x 150 um pixels


def barrel_geometry(n_modules: int, pitch_row: float = PITCH_ROW, pitch_col: float = PITCH_COL):
    """Synthetic module placement: (origin float32[M, 3], rotation float32[M, 3, 3])
    with global = origin + R @ (u, v, 0) for local (u, v) in cm."""
    lib = _load()
    origin = np.empty((n_modules, 3), np.float32)
    rot = np.empty((n_modules, 3, 3), np.float32)
    lib.synth_barrel_geometry(n_modules, ROWS, COLS, pitch_row, pitch_col, origin.ctypes.data, rot.ctypes.data)
    return origin, rot


def pack(row, col, adc) -> np.ndarray:
    """Pack (row, col, adc) into digi words (the input encoding)."""
    row = np.asarray(row, np.uint32)
    col = np.asarray(col, np.uint32)
    adc = np.asarray(adc, np.uint32)
    return (row | (col << 8) | (adc << 17)).astype(np.uint32)
