"""GPU tests of transfer on demand (Sec. 4.3): an event enqueued with
HP_KEEP_ON_DEVICE moves nothing but per-event status and offsets to the
host; device consumers (hits) read its clusters in place; a transfer
consumer brings clusters and/or labels to the host only when asked, under
the same stream rules as any consumer (Sec. 4.2), with the oracle's
results."""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_batch_matches
from tests.test_gpu_hits import HIT_TOL

pytestmark = pytest.mark.gpu

KEEP = hp.HP_KEEP_ON_DEVICE


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def work():
    w = synth.workload("full", n_events=3)
    return w, oracle.reconstruct_workload(w)


def test_kept_event_moves_only_status_and_offsets(torch_cuda, work):
    w, ref = work
    E, N = w.n_events, w.n_digis
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        d0 = ctx.stats()["d2h_bytes"]
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=KEEP | hp.HP_WANT_LABELS)
        assert ev.wait(60) == hp.HP_OK
        assert ctx.stats()["d2h_bytes"] - d0 == 8 * (E + 1) + 4 * E
        with pytest.raises(hp.HPError) as e:
            ev.fetch()
        assert e.value.status == hp.HP_EINVAL
        v = ev.device_clusters()
        assert v.capacity == N and v.module and v.x and v.label
        # labels then clusters, each on demand
        t_lab = ev.transfer(hp.HP_TRANSFER_LABELS)
        assert t_lab.stream == ev.stream  # first consumer: the product's stream
        t_cl = ev.transfer(hp.HP_TRANSFER_CLUSTERS)
        assert t_cl.stream != ev.stream
        assert t_lab.wait(60) == hp.HP_OK and t_cl.wait(60) == hp.HP_OK
        lab = t_lab.fetch()
        assert lab.label is not None and np.array_equal(lab.label, ref.label)
        assert lab.id.size == 0  # clusters not transferred
        got = t_cl.fetch()
        assert got.label is None
        assert_batch_matches(got, ref, w.offsets, check_labels=False)
        assert ctx.stats()["d2h_bytes"] - d0 == 8 * (E + 1) + 4 * E + 4 * N  # the labels' copy
        for x in (t_lab, t_cl, ev):
            x.release()


def test_hits_read_a_kept_product_in_place(torch_cuda, work):
    w, ref = work
    origin, rot = synth.barrel_geometry(w.n_modules)
    gx, gy, gz = oracle.hits(ref.module, ref.x, ref.y, origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        ctx.set_geometry(origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=KEEP)
        h = ev.hits()
        ev.release()  # the hits consumer holds the kept clusters until it has run
        assert h.wait(60) == hp.HP_OK
        r = h.fetch()
        assert np.array_equal(r.hit_offsets, ref.cluster_offsets) and np.array_equal(r.module, ref.module)
        for a, b in ((r.x, gx), (r.y, gy), (r.z, gz)):
            assert np.abs(a.astype(np.float64) - b).max() <= HIT_TOL
        h.release()


def test_transfer_errors_and_early_release(torch_cuda, work):
    w, ref = work
    lib = hp.load()
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        plain = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        out = ctypes.c_void_p()
        assert lib.hp_enqueue_transfer(plain._h, hp.HP_TRANSFER_CLUSTERS, ctypes.byref(out)) == hp.HP_EINVAL
        assert lib.hp_event_device_clusters(plain._h, ctypes.byref(hp.DeviceClusters())) == hp.HP_EINVAL
        kept = ctx.enqueue_batch(w.words, w.modules, w.offsets, flags=KEEP)  # no labels computed
        assert lib.hp_enqueue_transfer(kept._h, hp.HP_TRANSFER_LABELS, ctypes.byref(out)) == hp.HP_EINVAL
        assert lib.hp_enqueue_transfer(kept._h, 0, ctypes.byref(out)) == hp.HP_EINVAL
        assert lib.hp_enqueue_transfer(kept._h, 8, ctypes.byref(out)) == hp.HP_EINVAL
        ts = [kept.transfer() for _ in range(3)]
        kept.release()  # before its transfers ran
        for t in ts:
            assert t.wait(60) == hp.HP_OK
            assert_batch_matches(t.fetch(), ref, w.offsets, check_labels=False)
            t.release()
        assert plain.wait(60) == hp.HP_OK
        plain.release()
        # every kept block went back: nothing is charged to the budget any more
        assert ctx.stats()["device_bytes_in_use"] == 0
