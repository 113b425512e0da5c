"""Comparison helpers for GPU-vs-oracle parity tests."""
import concurrent.futures as cf
import os

import numpy as np

# Centroids: FP32 on the GPU vs the FP64 oracle, within 1e-4 pixel.
CENTROID_TOL = 1e-4


def assert_event_matches(got, ref, e_got, e_ref=None, labels_got=None, labels_ref=None, tol=CENTROID_TOL):
    """Compare event e of a GPU result with event e_ref of an oracle result."""
    e_ref = e_got if e_ref is None else e_ref
    sg = int(got.event_status[e_got])
    sr = int(ref.event_status[e_ref])
    assert sg == sr, f"event {e_got}: status {sg} != oracle {sr}"
    if sr != 0:
        return
    a, b = int(got.cluster_offsets[e_got]), int(got.cluster_offsets[e_got + 1])
    c, d = int(ref.cluster_offsets[e_ref]), int(ref.cluster_offsets[e_ref + 1])
    assert b - a == d - c, f"event {e_got}: {b - a} clusters != oracle {d - c}"
    for f in ("module", "id", "charge", "npix"):
        g = getattr(got, f)[a:b].astype(np.int64)
        r = getattr(ref, f)[c:d].astype(np.int64)
        if not np.array_equal(g, r):
            i = int(np.flatnonzero(g != r)[0])
            raise AssertionError(f"event {e_got}: {f}[{i}] {g[i]} != oracle {r[i]}")
    for f in ("x", "y"):
        dev = np.abs(getattr(got, f)[a:b].astype(np.float64) - getattr(ref, f)[c:d])
        assert dev.size == 0 or dev.max() <= tol, f"event {e_got}: {f} off by {dev.max()}"
    if labels_got is not None:
        assert np.array_equal(labels_got, labels_ref), f"event {e_got}: labels differ"


def assert_batch_matches(got, ref, offsets, check_labels=True):
    assert got.n_events == len(ref.event_status)
    for e in range(got.n_events):
        lg = lr = None
        if check_labels and got.label is not None and int(ref.event_status[e]) == 0:
            s, t = int(offsets[e]), int(offsets[e + 1])
            lg, lr = got.label[s:t], ref.label[s:t]
        assert_event_matches(got, ref, e, labels_got=lg, labels_ref=lr)


def oracle_events(w, events=None, **kw):
    """The oracle's result for each event of workload w (one oracle call per
    event, on the host's cores; the oracle releases the GIL)."""
    from oracle import oracle

    events = list(range(w.n_events)) if events is None else list(events)

    def one(e):
        words, mods = w.event(e)
        return oracle.reconstruct_event(words, mods, w.n_modules, w.gain, w.pedestal, **kw)

    with cf.ThreadPoolExecutor(min(len(events), os.cpu_count() or 1) or 1) as ex:
        return list(ex.map(one, events))


def assert_events_match(got, refs, offsets, events=None):
    """Compare every event e of a GPU batch result with refs[j], the oracle's
    result for that event alone (j-th of `events`, default all)."""
    events = range(got.n_events) if events is None else events
    for j, e in enumerate(events):
        s, t = int(offsets[e]), int(offsets[e + 1])
        ref = refs[j]
        lg = got.label[s:t] if got.label is not None and int(ref.event_status[0]) == 0 else None
        lr = ref.label if lg is not None else None
        assert_event_matches(got, ref, e, 0, lg, lr)
