"""GPU tests of the execution contract (arXiv:2004.04334 Sec. 2 and Sec. 4):
exactly-once completion callbacks, non-blocking acquire, no allocation once
the pools are warm, errors delivered with the callback, admission control,
host-side fault injection, draining teardown."""
import ctypes
import threading
import time

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_batch_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return synth.workload("tiny", n_events=8)


def _ctx(w, **kw):
    return hp.Context(w.n_modules, w.gain, w.pedestal, **kw)


def test_callback_exactly_once_both_orders(tiny):
    lib = hp.load()
    calls = []
    lock = threading.Lock()

    @hp.CALLBACK
    def cb(user, ev, st):
        with lock:
            calls.append((user, st))

    with _ctx(tiny) as ctx:
        words, mods = tiny.event(0)
        for order in range(20):
            h = ctypes.c_void_p()
            assert lib.hp_enqueue_event(ctx._h, words.ctypes.data, mods.ctypes.data, len(words), 0, 0,
                                        ctypes.byref(h)) == hp.HP_OK
            if order % 2:  # register after completion
                t0 = time.time()
                while lib.hp_event_query(h) == hp.HP_ENOTREADY:
                    assert time.time() - t0 < 30
                    time.sleep(0.0005)
            assert lib.hp_on_complete(h, cb, ctypes.c_void_p(order + 1)) == hp.HP_OK
            assert lib.hp_on_complete(h, cb, ctypes.c_void_p(99)) == hp.HP_EINVAL  # only one callback
            t0 = time.time()
            while True:
                with lock:
                    n = sum(1 for u, _ in calls if u == order + 1)
                if n:
                    break
                assert time.time() - t0 < 30
                time.sleep(0.0005)
            assert lib.hp_release_event(h) == hp.HP_OK
        time.sleep(0.05)
        with lock:
            users = [u for u, _ in calls]
        assert sorted(users) == list(range(1, 21))
        assert all(st == hp.HP_OK for _, st in calls)


def test_release_before_completion_is_deferred(tiny):
    with _ctx(tiny, want_labels=True) as ctx:
        evs = [ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets) for _ in range(8)]
        for ev in evs[:4]:
            ev.release()  # deferred until each completes
        for ev in evs[4:]:
            assert ev.wait(30) == hp.HP_OK
            ev.release()
        s = ctx.stats()
        t0 = time.time()
        while ctx.stats()["events_completed"] < 8:
            assert time.time() - t0 < 30
            time.sleep(0.001)
        assert s["events_enqueued"] == 8


def test_no_allocation_in_steady_state(tiny):
    with _ctx(tiny, want_labels=True) as ctx:
        for _ in range(3):  # warm the pools
            ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
            ev.wait(30)
            ev.release()
        before = ctx.stats()
        for _ in range(50):
            ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
            ev.wait(30)
            ev.release()
        after = ctx.stats()
        assert after["device_mallocs"] == before["device_mallocs"]
        assert after["host_mallocs"] == before["host_mallocs"]
        assert after["pool_hits"] >= before["pool_hits"] + 100


def test_acquire_does_not_wait_for_the_device():
    """Enqueue time stays small and flat while device time grows with the event."""
    torch = pytest.importorskip("torch")
    w = synth.workload("occupancy", n_events=4)
    pinned_w = torch.from_numpy(w.words.view(np.int32)).pin_memory()
    pinned_m = torch.from_numpy(w.modules.view(np.int16)).pin_memory()
    with _ctx(w, want_labels=True) as ctx:
        ev = ctx.enqueue_batch(pinned_w, pinned_m, w.offsets, flags=hp.HP_INPUT_NOCOPY)
        ev.wait(60)
        ev.release()
        t0 = time.perf_counter()
        ev = ctx.enqueue_batch(pinned_w, pinned_m, w.offsets, flags=hp.HP_INPUT_NOCOPY)
        t_enq = time.perf_counter() - t0
        ev.wait(60)
        t_all = time.perf_counter() - t0
        ev.release()
    assert t_enq < 0.25 * t_all, (t_enq, t_all)


def test_errors_arrive_with_the_callback(tiny):
    words, mods = tiny.event(0)
    bad = words.copy()
    bad[0] |= 1 << 30
    dup_w = np.concatenate([words, words[5:6]])
    dup_m = np.concatenate([mods, mods[5:6]])
    got = {}
    done = threading.Event()
    with _ctx(tiny) as ctx:
        e1 = ctx.enqueue_event(bad, mods)
        e2 = ctx.enqueue_event(dup_w, dup_m)
        for name, ev in (("bad", e1), ("dup", e2)):
            ev.on_complete(lambda e, st, name=name: (got.__setitem__(name, st), len(got) == 2 and done.set()))
        assert done.wait(30)
        assert got == {"bad": hp.HP_EBADDIGI, "dup": hp.HP_EDUP}
        assert e1.fetch().n_clusters == 0 or e1.fetch().status == hp.HP_EBADDIGI
        e1.release()
        e2.release()


def test_inflight_limit_returns_eagain():
    w = synth.workload("full_literal")
    with _ctx(w, max_inflight=1) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        statuses = []
        for _ in range(5):
            st, e2 = ctx.try_enqueue_batch(w.words, w.modules, w.offsets)
            statuses.append(st)
            if e2 is not None:
                e2.wait(60)
                e2.release()
        ev.wait(60)
        ev.release()
        assert hp.HP_EAGAIN in statuses
        # after completion the slot is free again
        st, e3 = ctx.try_enqueue_batch(w.words, w.modules, w.offsets)
        assert st == hp.HP_OK
        e3.wait(60)
        e3.release()


def test_device_budget_returns_eagain():
    w = synth.workload("full_literal")
    with _ctx(w, budget_bytes=1 << 20) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)  # larger than the budget but alone: admitted
        st, e2 = ctx.try_enqueue_batch(w.words, w.modules, w.offsets)
        if e2 is not None:  # the first one already finished
            e2.wait(60)
            e2.release()
        ev.wait(60)
        ev.release()
        assert st in (hp.HP_EAGAIN, hp.HP_OK)


def test_injected_allocation_failure(tiny):
    with _ctx(tiny) as ctx:
        ctx.debug_fail_allocations(1)
        st, ev = ctx.try_enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
        assert st == hp.HP_ENOMEM and ev is None
        st, ev = ctx.try_enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
        assert st == hp.HP_OK
        assert ev.wait(30) == hp.HP_OK
        ev.release()
        assert ctx.stats()["inflight"] == 0


def test_destroy_drains_inflight_events(tiny):
    ref = oracle.reconstruct_workload(tiny)
    results = []
    ctx = _ctx(tiny, want_labels=True)
    for _ in range(16):
        ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
        ev.on_complete(lambda e, st: results.append(e.fetch()))
    ctx.close()  # blocks until every event has completed and its callback ran
    assert len(results) == 16
    for r in results:
        assert_batch_matches(r, ref, tiny.offsets)


def test_concurrent_submitters_share_a_context(tiny):
    ref = oracle.reconstruct_workload(tiny)
    errors = []
    with _ctx(tiny, want_labels=True, n_streams=4) as ctx:
        def worker():
            try:
                for _ in range(10):
                    ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
                    ev.wait(30)
                    assert_batch_matches(ev.fetch(), ref, tiny.offsets)
                    ev.release()
            except Exception as exc:  # noqa: BLE001
                errors.append(exc)

        ts = [threading.Thread(target=worker) for _ in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    assert not errors, errors[0]


def test_product_metadata(tiny):
    with _ctx(tiny) as ctx:
        ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
        assert ev.device == 0 and ev.stream != 0
        ev.wait(30)
        assert ev.latency_ns > 0
        ev.release()


def test_labels_cross_the_link_only_when_asked(tiny):
    """D2H on demand (Sec. 4.3): without HP_WANT_LABELS no label bytes are copied."""
    N = tiny.n_digis
    with _ctx(tiny) as ctx:
        d0 = ctx.stats()["d2h_bytes"]
        ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets)
        assert ev.wait(30) == hp.HP_OK and ev.fetch().label is None
        ev.release()
        d1 = ctx.stats()["d2h_bytes"]
        # what was copied is leading cluster records (24 bytes each, at most
        # a quarter of the digis' worth: the DMA part of the cluster output)
        assert (d1 - d0) % 24 == 0 and d1 - d0 <= 24 * (N // 4)
        ev = ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets, flags=hp.HP_WANT_LABELS)
        assert ev.wait(30) == hp.HP_OK and ev.fetch().label is not None
        ev.release()
        d2 = ctx.stats()["d2h_bytes"]
        assert d2 - d1 >= 4 * N and (d2 - d1 - 4 * N) % 24 == 0 and d2 - d1 - 4 * N <= 24 * (N // 4)


def test_events_in_flight_use_different_streams(tiny):
    """One stream per event in flight (Sec. 4.1): consecutive enqueues take
    different streams of the pool, so their copies and kernels may overlap."""
    with _ctx(tiny, n_streams=4) as ctx:
        evs = [ctx.enqueue_batch(tiny.words, tiny.modules, tiny.offsets) for _ in range(4)]
        assert len({ev.stream for ev in evs}) == 4
        for ev in evs:
            assert ev.wait(30) == hp.HP_OK
            ev.release()
