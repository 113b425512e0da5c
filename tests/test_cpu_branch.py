"""The CPU case of libhp (Sec. 3, the SwitchProducer), on a host without a
GPU (or with HP_FORCE_CPU): the same product as the GPU path, checked event
by event and digi by digi against the oracle on every workload shape, plus
the invalid-event statuses, the compact labels, provenance, callbacks and
the calls a CPU context refuses.  These tests need no GPU."""
import ctypes
import threading

import numpy as np
import pytest

from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_events_match, oracle_events


@pytest.fixture(autouse=True)
def force_cpu(monkeypatch):
    monkeypatch.setenv("HP_FORCE_CPU", "1")
    monkeypatch.setenv("HP_CPU_THREADS", "4")


def _run(w, flags=hp.HP_WANT_LABELS):
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=flags)
        st = ev.wait(120)
        r = ev.fetch()
        prov = ev.provenance()
        ev.release()
    return st, r, prov


@pytest.mark.parametrize("name,n", [("tiny", 6), ("full", 2), ("batched", 6), ("serving", 8)])
def test_cpu_case_equals_the_oracle(name, n):
    w = synth.workload(name, n_events=n)
    st, r, prov = _run(w)
    assert st == hp.HP_OK and prov["path"] == "cpu" and prov["device"] == -1
    assert_events_match(r, oracle_events(w), w.offsets)
    # the compact form stands for the same labels
    _, r16, _ = _run(w, hp.HP_LABELS_U16)
    assert r16.label is None
    assert np.array_equal(r16.labels_from_compact(w.offsets, w.modules), r.label)
    assert np.array_equal(r16.id, r.id) and np.array_equal(r16.x, r.x)


def test_cpu_case_on_heavy_modules():
    # one high-occupancy event: hot modules, long streaks, clusters of tens of pixels
    w = synth.workload("occupancy", n_events=1)
    st, r, _ = _run(w)
    assert st == hp.HP_OK
    assert_events_match(r, oracle_events(w), w.offsets)


def test_invalid_and_empty_events():
    w = synth.workload("tiny", n_events=5)
    words, mods, offs = w.words.copy(), w.modules.copy(), w.offsets.copy()
    a1 = int(offs[1])
    words[a1 + 3] = words[a1 + 3] | (1 << 26)                           # event 1: a word with high bits set
    a2 = int(offs[2])
    words[a2 + 1], mods[a2 + 1] = words[a2], mods[a2]                   # event 2: a position twice
    a3 = int(offs[3])
    mods[a3] = w.n_modules                                              # event 3: a module out of range
    # event 4 emptied: drop its digis
    keep = np.ones(len(words), bool)
    keep[int(offs[4]):int(offs[5])] = False
    words, mods = words[keep], mods[keep]
    offs = offs.copy()
    offs[5] = offs[4]
    bad = synth.Workload(w.name, w.n_modules, words, mods, offs, w.gain, w.pedestal)
    st, r, _ = _run(bad)
    assert list(r.event_status) == [hp.HP_OK, hp.HP_EBADDIGI, hp.HP_EDUP, hp.HP_EBADDIGI, hp.HP_OK]
    assert st == hp.HP_EBADDIGI  # the first failing event's status
    for e in (1, 2, 3):
        assert r.cluster_offsets[e + 1] == r.cluster_offsets[e]
        assert (r.label[int(offs[e]):int(offs[e + 1])] == -1).all()
    assert r.cluster_offsets[5] == r.cluster_offsets[4]
    refs = oracle_events(bad)
    for e in (0, 1, 2, 3, 4):
        assert int(refs[e].event_status[0]) == int(r.event_status[e])
    assert_events_match(r, [refs[0], refs[4]], offs, events=[0, 4])


def test_callbacks_order_and_release_before_completion():
    w = synth.workload("batched", n_events=3)
    seen = []
    lock = threading.Lock()
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        evs = []
        for k in range(6):
            ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, tag=k)
            ev.on_complete(lambda e, st, k=k: (lock.acquire(), seen.append((k, st)), lock.release()))
            evs.append(ev)
        # the first one released before it completed: the library frees it
        # once it has run (the binding drops its handle, and its callback, now)
        evs[0].release()
        for ev in evs[1:]:
            assert ev.wait(60) == hp.HP_OK
            ev.release()
        stats = ctx.stats()
    assert stats["events_completed"] == 6 and stats["inflight"] == 0
    assert [k for k, _ in seen] == [k for k in range(6) if k > 0 or (0, hp.HP_OK) in seen]
    assert all(st == hp.HP_OK for _, st in seen)


def test_calls_a_cpu_context_refuses():
    w = synth.workload("tiny", n_events=1)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        lib, h = ctx._lib, ctx._h
        st, ev = ctx.try_enqueue_batch(w.words, w.modules, w.offsets, flags=hp.HP_KEEP_ON_DEVICE)
        assert st == hp.HP_EINVAL and ev is None
        out = hp.DeviceClusters()
        one = ctypes.c_void_p(16)  # never dereferenced: refused first
        assert lib.hp_reconstruct_device(h, 1, 1, one, one, one, ctypes.byref(out), None) == hp.HP_EINVAL
        cfg = hp.ServeConfig(0, 0, 0, 0, 0, 0)
        assert lib.hp_serve_start(h, ctypes.byref(cfg)) == hp.HP_EINVAL
        o = np.zeros(3 * w.n_modules, np.float32)
        rot = np.zeros(9 * w.n_modules, np.float32)
        assert lib.hp_set_geometry(h, o.ctypes.data, rot.ctypes.data, ctypes.c_float(0.01),
                                   ctypes.c_float(0.015)) == hp.HP_EINVAL


def test_no_silent_fallback_to_the_host(monkeypatch):
    """Without HP_FORCE_CPU or HP_ALLOW_CPU a context on a host without a
    usable GPU is an error, never a CPU context; with HP_ALLOW_CPU it is the
    CPU case (the runtime choice of Sec. 3, asked for by the caller)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the missing-device case cannot be made here")
    monkeypatch.delenv("HP_FORCE_CPU")
    w = synth.workload("tiny", n_events=1)
    with pytest.raises(hp.HPError) as e:
        hp.Context(w.n_modules, w.gain, w.pedestal)
    assert e.value.status == hp.HP_ECUDA
    with hp.Context(w.n_modules, w.gain, w.pedestal, allow_cpu=True) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        assert ev.wait(60) == hp.HP_OK and ev.provenance()["path"] == "cpu"
        ev.release()
