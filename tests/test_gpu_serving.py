"""GPU tests of the serving loop (continuous batching): requests submitted
from several threads while others run are admitted as batch slots and
device budget free up, and every result equals the result of the same event
processed alone (and the oracle)."""
import threading
import time

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_batch_matches, oracle_events

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # serving-recipe events (lognormal sizes), a few of them small for speed
    w = synth.workload("serving", n_events=24)
    return w


def _alone(ctx, w, e):
    words, mods = w.event(e)
    ev = ctx.enqueue_event(words, mods)
    assert ev.wait(60) == hp.HP_OK
    r = ev.fetch()
    ev.release()
    return r


def test_mix_equals_alone(pool):
    w = pool
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True, n_streams=4) as ctx:
        alone = [_alone(ctx, w, e) for e in range(w.n_events)]
        ctx.serve_start(budget_bytes=16 << 30, want_labels=True)
        order = [e for _ in range(3) for e in np.random.default_rng(2).permutation(w.n_events)]
        results = [None] * len(order)
        errors = []

        def submitter(tid):
            try:
                evs = []
                for i in range(tid, len(order), 4):
                    words, mods = w.event(order[i])
                    evs.append((i, ctx.submit(words, mods, tag=i)))
                for i, ev in evs:
                    assert ev.wait(120) == hp.HP_OK
                    results[i] = ev.fetch()
                    assert ev.latency_ns > 0
                    ev.release()
            except Exception as exc:  # noqa: BLE001
                errors.append(exc)

        ts = [threading.Thread(target=submitter, args=(t,)) for t in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errors, errors[0]
        stats = ctx.stats()
        ctx.serve_stop()
    assert stats["serve_requests"] == len(order)
    assert stats["serve_batches"] < len(order)  # requests were batched together
    for i, e in enumerate(order):
        r, a = results[i], alone[e]
        for f in ("module", "id", "charge", "npix", "x", "y", "label"):
            assert np.array_equal(getattr(r, f), getattr(a, f)), (i, f)
    # and the alone results (so the mixed ones too) are the oracle's, for
    # every event of the pool
    refs = oracle_events(w)
    for e in range(w.n_events):
        assert_batch_matches(alone[e], refs[e], np.array([0, int(w.offsets[e + 1] - w.offsets[e])], np.uint64))


def test_budget_admits_one_batch_at_a_time(pool):
    w = pool
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        ctx.serve_start(budget_bytes=1 << 20, max_batch_events=2)
        evs = [ctx.submit(*w.event(e)) for e in range(8)]
        for ev in evs:
            assert ev.wait(120) == hp.HP_OK
        s = ctx.stats()
        assert s["serve_batches"] >= 4
        for e, ev in enumerate(evs):
            r = ev.fetch()
            a = _alone(ctx, w, e)
            assert np.array_equal(r.id, a.id) and np.array_equal(r.charge, a.charge)
            ev.release()
        ctx.serve_stop()


def test_backpressure_and_draining_stop(pool):
    w = pool
    done = []
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        ctx.serve_start(max_pending=4, max_inflight_batches=1, max_batch_events=1)
        statuses, evs = [], []
        for e in range(40):
            st, ev = ctx.try_submit(*w.event(e % w.n_events))
            statuses.append(st)
            if ev is not None:
                ev.on_complete(lambda ev, st: done.append(st))
                evs.append(ev)
        assert hp.HP_EAGAIN in statuses
        ctx.serve_stop()  # launches what is queued and waits
        assert len(done) == len(evs) and all(st == hp.HP_OK for st in done)
        for ev in evs:
            ev.release()


def test_bad_request_does_not_disturb_its_batch(pool):
    w = pool
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        a0 = _alone(ctx, w, 0)
        ctx.serve_start(max_inflight_batches=1)
        words, mods = w.event(1)
        bad = words.copy()
        bad[7] |= 1 << 27
        time.sleep(0.01)
        evs = [ctx.submit(*w.event(0)), ctx.submit(bad, mods), ctx.submit(*w.event(0))]
        sts = [ev.wait(60) for ev in evs]
        assert sts == [hp.HP_OK, hp.HP_EBADDIGI, hp.HP_OK]
        for ev in (evs[0], evs[2]):
            r = ev.fetch()
            assert np.array_equal(r.id, a0.id) and np.array_equal(r.x, a0.x)
        for ev in evs:
            ev.release()
        ctx.serve_stop()


def test_native_replay_driver(pool):
    """hp_serve_replay: 4 native submitter threads on a Poisson schedule."""
    w = pool
    events = [w.event(e) for e in range(w.n_events)]
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        ctx.serve_start(budget_bytes=16 << 30, want_labels=True)
        rng = np.random.default_rng(4)
        arrival = np.cumsum(rng.exponential(1 / 5000.0, 200))
        lat, st, span = ctx.serve_replay(events, arrival, np.arange(200) % len(events), 4)
        s = ctx.stats()
        ctx.serve_stop()
    assert np.all(st == 0) and np.all(lat > 0)
    assert span >= arrival[-1] - arrival[0]
    assert s["serve_requests"] == 200 and s["serve_batches"] <= 200


def test_nocopy_serving_reads_pinned_inputs_in_place(pool):
    """HP_INPUT_NOCOPY serving: hp_submit keeps the caller's (pinned) buffers,
    the batch copies them by DMA; results equal the event processed alone."""
    import torch

    w = pool
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True, n_streams=4) as ctx:
        alone = [_alone(ctx, w, e) for e in range(w.n_events)]
        pinned = []
        for e in range(w.n_events):
            words, mods = w.event(e)
            pw = torch.from_numpy(words.view(np.int32).copy()).pin_memory()
            pm = torch.from_numpy(mods.view(np.int16).copy()).pin_memory()
            pinned.append((pw, pm))
        ctx.serve_start(budget_bytes=16 << 30, want_labels=True, nocopy=True)
        before = ctx.stats()["serve_submit_ns"]
        order = [e for _ in range(2) for e in np.random.default_rng(3).permutation(w.n_events)]
        evs = []
        for i, e in enumerate(order):
            pw, pm = pinned[e]
            words = pw.numpy().view(np.uint32)
            mods = pm.numpy().view(np.uint16)
            evs.append(ctx.submit(words, mods, tag=i))
        for i, ev in enumerate(evs):
            assert ev.wait(120) == hp.HP_OK
            r, a = ev.fetch(), alone[order[i]]
            for f in ("module", "id", "charge", "npix", "x", "y", "label"):
                assert np.array_equal(getattr(r, f), getattr(a, f)), (i, f)
            ev.release()
        assert ctx.stats()["serve_submit_ns"] > before
        # the native driver in the same mode (it submits from a pinned copy of its pool)
        events = [w.event(e) for e in range(w.n_events)]
        arrival = np.cumsum(np.random.default_rng(5).exponential(1 / 5000.0, 100))
        lat, st, _ = ctx.serve_replay(events, arrival, np.arange(100) % len(events), 4)
        assert np.all(st == 0) and np.all(lat > 0)
        ctx.serve_stop()


def test_serving_trace_records_every_batch_in_order(pool):
    """hp_serve_trace_*: one record per batch with its host timestamps in
    causal order, the device marks in stream order, and the batches'
    event counts adding up to the requests; disabling clears it."""
    w = pool
    with hp.Context(w.n_modules, w.gain, w.pedestal, n_streams=4) as ctx:
        ctx.serve_start(budget_bytes=8 << 30, nocopy=False)
        ctx.serve_trace_enable(1 << 16)
        n = 60
        evs = [ctx.submit(*w.event(i % w.n_events)) for i in range(n)]
        for ev in evs:
            assert ev.wait(120) == hp.HP_OK
            ev.release()
        ctx.serve_stop()
        tr = ctx.serve_trace()
        assert len(tr) >= 1 and int(tr["n_events"].sum()) == n
        assert int(tr["n_digis"].sum()) == sum(len(w.event(i % w.n_events)[0]) for i in range(n))
        order = ["t_first_submit", "t_admit", "t_pooled", "t_inputs", "t_kernels", "t_launched", "t_done_start",
                 "t_done_end"]
        for a, b in zip(order, order[1:]):
            assert (tr[a].astype(np.int64) <= tr[b].astype(np.int64)).all(), (a, b)
        marks = ["gpu_start", "gpu_inputs", "gpu_kernels", "gpu_outputs"]
        assert (tr["gpu_start"] >= 0).all()
        for a, b in zip(marks, marks[1:]):
            assert (tr[a] <= tr[b]).all(), (a, b)
        assert set(int(s) for s in tr["stream"]) <= {0, 1, 2, 3}
        ctx.serve_trace_enable(0)
        assert len(ctx.serve_trace()) == 0
