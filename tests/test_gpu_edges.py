"""GPU edge cases of the API surface: batches whose events are all empty go
through every entry point (host, device, graph, hits, transfer) and give
empty, OK results; a single-digi event and a batch mixing empty and
non-empty events match the oracle."""
import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_batch_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ctx(w):
    ctx = hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True)
    origin, rot = synth.barrel_geometry(w.n_modules)
    ctx.set_geometry(origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
    return ctx


def test_all_empty_batch_through_every_entry(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("tiny")
    E = 5
    offs = np.zeros(E + 1, np.uint64)
    words = np.empty(0, np.uint32)
    mods = np.empty(0, np.uint16)
    with _ctx(w) as ctx:
        ev = ctx.enqueue_batch(words, mods, offs)
        assert ev.wait(60) == hp.HP_OK
        r = ev.fetch()
        assert r.n_clusters == 0 and np.all(r.cluster_offsets == 0) and np.all(r.event_status == 0)
        h = ev.hits()
        assert h.wait(60) == hp.HP_OK and h.fetch().n_hits == 0
        h.release()
        ev.release()
        kept = ctx.enqueue_batch(words, mods, offs, flags=hp.HP_KEEP_ON_DEVICE | hp.HP_WANT_LABELS)
        t = kept.transfer(hp.HP_TRANSFER_CLUSTERS | hp.HP_TRANSFER_LABELS)
        assert t.wait(60) == hp.HP_OK
        tr = t.fetch()
        assert tr.n_clusters == 0 and np.all(tr.cluster_offsets == 0)
        t.release()
        kept.release()
        single = ctx.enqueue_event(words, mods)
        assert single.wait(60) == hp.HP_OK and single.fetch().n_clusters == 0
        single.release()
        d_offs = torch.zeros(E + 1, dtype=torch.int64, device=dev)
        d_w = torch.zeros(1, dtype=torch.int32, device=dev)
        d_m = torch.zeros(1, dtype=torch.int16, device=dev)
        out = hp.DeviceOutputs(E, 0, dev)
        out.cluster_offsets.fill_(-1)
        ctx.reconstruct_device(E, 0, d_offs.data_ptr(), d_w.data_ptr(), d_m.data_ptr(), out,
                               torch.cuda.current_stream(dev).cuda_stream)
        g = ctx.graph_capture(E, 0, d_offs.data_ptr(), d_w.data_ptr(), d_m.data_ptr(), out)
        g.launch(torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize(dev)
        g.destroy()
        res = out.to_result(0)
        assert res.n_clusters == 0 and np.all(res.cluster_offsets == 0) and np.all(res.event_status == 0)


def test_single_digi_and_mixed_empty_events(torch_cuda):
    w = synth.workload("tiny", n_events=3)
    # event 0: one digi above both thresholds (ADC 255); event 1: empty; event 2: a normal event
    gain, ped = int(w.gain[7]), int(w.pedestal[7])
    assert 255 * gain - ped >= 4000
    one = np.array([(255 << 17) | (100 << 8) | 42], np.uint32)
    one_m = np.array([7], np.uint16)
    w2, m2 = w.event(2)
    words = np.concatenate([one, w2])
    mods = np.concatenate([one_m, m2])
    offs = np.array([0, 1, 1, 1 + len(w2)], np.uint64)
    ref = oracle.reconstruct_batch(words, mods, offs, w.n_modules, w.gain, w.pedestal)
    assert ref.cluster_offsets[1] == 1 and ref.id[0] == 42 * 416 + 100
    with _ctx(w) as ctx:
        ev = ctx.enqueue_batch(words, mods, offs)
        assert ev.wait(60) == hp.HP_OK
        assert_batch_matches(ev.fetch(), ref, offs)
        ev.release()


def test_provenance_of_products(torch_cuda):
    w = synth.workload("tiny", n_events=4)
    with _ctx(w) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        assert ev.wait(60) == hp.HP_OK
        p = ev.provenance()
        assert p["path"] == "batch" and p["device"] == 0 and p["device_name"]
        assert p["cc"][0] >= 10 and "sm_103a" in p["library"]
        assert p["tuning"] == ctx.get_tuning(w.n_events, w.n_digis)
        h = ev.hits()
        assert h.wait(60) == hp.HP_OK
        ph = h.provenance()
        assert ph["path"] == "hits" and ph["tuning"]["tile_slots"] == 0
        h.release()
        ev.release()
        single = ctx.enqueue_event(*w.event(0))
        assert single.wait(60) == hp.HP_OK and single.provenance()["path"] == "event"
        single.release()
        ctx.serve_start()
        r = ctx.submit(*w.event(1))
        assert r.wait(60) == hp.HP_OK
        pr = r.provenance()
        assert pr["path"] == "serving" and pr["tuning"]["tile_slots"] > 0
        r.release()
        ctx.serve_stop()


def test_destroy_with_unreleased_products_and_consumers(torch_cuda):
    """hp_destroy drains and frees products whose consumers (hits, transfers)
    were never released, in any state."""
    w = synth.workload("full", n_events=2)
    ctx = _ctx(w)
    ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
    h = ev.hits()
    kept = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=hp.HP_KEEP_ON_DEVICE | hp.HP_WANT_LABELS)
    t = kept.transfer(hp.HP_TRANSFER_CLUSTERS | hp.HP_TRANSFER_LABELS)
    h2 = kept.hits()
    assert t.wait(60) == hp.HP_OK
    ctx.close()  # nothing released: everything is drained and freed here
    # a fresh context on the same device works
    with _ctx(w) as ctx2:
        e2 = ctx2.enqueue_batch(w.words, w.modules, w.offsets)
        assert e2.wait(60) == hp.HP_OK
        e2.release()
