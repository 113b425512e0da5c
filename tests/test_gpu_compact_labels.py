"""GPU tests of the compact label form (HP_LABELS_U16): each digi's cluster
as its rank among its module's clusters, plus every (event, module) item's
first cluster.  Expanded back to cluster ids it must equal the oracle's
labels, digi by digi, on the batch, single-event and serving paths; the
clusters themselves are unchanged."""
import numpy as np
import pytest

from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_event_matches, oracle_events

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _check(r, w, refs, events=None):
    events = range(w.n_events) if events is None else events
    assert r.label is None and r.label16 is not None and r.item_first is not None
    assert r.label16.dtype == np.uint16 and len(r.label16) == int(w.offsets[-1])
    assert len(r.item_first) == r.n_events * w.n_modules
    lab = r.labels_from_compact(w.offsets, w.modules)
    for j, e in enumerate(events):
        s, t = int(w.offsets[e]), int(w.offsets[e + 1])
        ref = refs[j]
        ok = int(ref.event_status[0]) == 0
        assert_event_matches(r, ref, e, 0, lab[s:t] if ok else None, ref.label if ok else None)
        if ok:  # both markers occur and map back exactly
            assert np.array_equal(r.label16[s:t] == 0xFFFF, ref.label == -1)
            assert np.array_equal(r.label16[s:t] == 0xFFFE, ref.label == -2)


def test_batch_compact_labels_equal_the_oracle(torch_cuda):
    w = synth.workload("batched", n_events=24)
    refs = oracle_events(w)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=hp.HP_LABELS_U16)
        assert ev.wait(120) == hp.HP_OK
        r = ev.fetch()
        ev.release()
    _check(r, w, refs)
    assert (r.label16 == 0xFFFE).any() and (r.label16 == 0xFFFF).any()


def test_single_events_with_many_modules_and_empty_events(torch_cuda):
    # the 1856-module geometry (most items empty), then an event of no digis
    w = synth.workload("full", n_events=2)
    refs = oracle_events(w)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        for e in range(w.n_events):
            words, mods = w.event(e)
            ev = ctx.enqueue_event(words, mods, flags=hp.HP_LABELS_U16)
            assert ev.wait(120) == hp.HP_OK
            r = ev.fetch()
            ev.release()
            one = w.subset([e])
            _check(r, one, [refs[e]])
        ev = ctx.enqueue_event(np.zeros(0, np.uint32), np.zeros(0, np.uint16), flags=hp.HP_LABELS_U16)
        assert ev.wait(60) == hp.HP_OK
        r = ev.fetch()
        ev.release()
        assert r.n_clusters == 0 and len(r.label16) == 0
        assert len(r.item_first) == w.n_modules and not r.item_first.any()


def test_compact_labels_with_device_resident_results_are_refused(torch_cuda):
    w = synth.workload("batched", n_events=2)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        st, ev = ctx.try_enqueue_batch(w.words, w.modules, w.offsets,
                                       flags=hp.HP_LABELS_U16 | hp.HP_KEEP_ON_DEVICE)
        assert st == hp.HP_EINVAL and ev is None


def test_serving_requests_carry_compact_labels(torch_cuda):
    w = synth.workload("serving", n_events=16)
    refs = oracle_events(w)
    with hp.Context(w.n_modules, w.gain, w.pedestal, n_streams=4) as ctx:
        ctx.serve_start(budget_bytes=8 << 30, compact_labels=True)
        evs = [ctx.submit(*w.event(e % w.n_events), tag=e) for e in range(3 * w.n_events)]
        results = []
        for ev in evs:
            assert ev.wait(120) == hp.HP_OK
            results.append(ev.fetch())
            ev.release()
        assert ctx.stats()["serve_batches"] < len(evs)
        ctx.serve_stop()
    for i, r in enumerate(results):
        e = i % w.n_events
        _check(r, w.subset([e]), [refs[e]])


@pytest.mark.parametrize("name,n", [("occupancy", 1), ("batched", 6)])
def test_compact_labels_in_every_tier(torch_cuda, name, n):
    """Every clustering setting (tile sizes that push the hot modules into the
    shared-memory tile or the global-memory tier, warp-tier limits, the hash
    label store at each group size), compact
    labels through the host path: the same labels as the oracle."""
    w = synth.workload(name, n_events=n)
    refs = oracle_events(w)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        cands = ctx.tuning_candidates()
        # one setting per (tile, blocks per SM, warp-tier limit): the ticket size does not change the tiers
        seen = set()
        for c in cands:
            key = (c["tile_slots"], c["blocks_per_sm"], c["warp_max"], c["label_store"], c["item_threads"])
            if key in seen:
                continue
            seen.add(key)
            ctx.set_tuning(w.n_events, w.n_digis, c)
            ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=hp.HP_LABELS_U16)
            assert ev.wait(120) == hp.HP_OK
            r = ev.fetch()
            ev.release()
            _check(r, w, refs)
        assert len(seen) >= 3
