"""GPU tests of the clusters -> hits stage (the step after the clusters in
the paper's Fig. 1) and of the Product<T> / ScopedContext consumer rules of
Sec. 4.2: the first consumer of a product runs on the product's stream, a
later one on another stream behind cudaStreamWaitEvent (none once the
product's event has completed), results identical either way, and the
product lives until every consumer's work has run.

Hit positions: FP32 on the GPU from FP32 centroids, against the FP64 oracle
from its FP64 centroids.  The centroids agree within 1e-4 pixel, i.e.
1.5e-6 cm at the 150 um column pitch; the FP32 evaluation of
origin + R (u, v, 0) with |terms| <= 20 cm adds at most a few ulp(16 cm)
(about 1e-6 cm each), so 1e-5 cm (0.1 um) bounds the difference.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth

pytestmark = pytest.mark.gpu

HIT_TOL = 1e-5  # cm


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ctx(w, geometry=True, **kw):
    ctx = hp.Context(w.n_modules, w.gain, w.pedestal, **kw)
    if geometry:
        origin, rot = synth.barrel_geometry(w.n_modules)
        ctx.set_geometry(origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
    return ctx


def _oracle_hits(w):
    ref = oracle.reconstruct_workload(w)
    origin, rot = synth.barrel_geometry(w.n_modules)
    gx, gy, gz = oracle.hits(ref.module, ref.x, ref.y, origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
    return ref, gx, gy, gz


def _assert_hits(got, ref, gx, gy, gz):
    assert np.array_equal(got.event_status, ref.event_status)
    assert np.array_equal(got.hit_offsets, ref.cluster_offsets)
    assert np.array_equal(got.module, ref.module)
    for a, r in ((got.x, gx), (got.y, gy), (got.z, gz)):
        d = np.abs(a.astype(np.float64) - r)
        assert d.size == 0 or d.max() <= HIT_TOL, d.max()


def _with_empty_event(w):
    """The workload with an empty event inserted second."""
    offs = np.concatenate([w.offsets[:2], w.offsets[1:]]).astype(np.uint64)
    return synth.Workload(w.name, w.n_modules, w.words, w.modules, offs, w.gain, w.pedestal)


def test_hits_chain_matches_oracle(torch_cuda):
    w = _with_empty_event(synth.workload("full", n_events=3))
    ref, gx, gy, gz = _oracle_hits(w)
    assert ref.n_clusters > 1000
    with _ctx(w) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets, tag=7)
        hits = ev.hits()
        assert hits.wait(60) == hp.HP_OK
        got = hits.fetch()
        assert got.tag == 7 and got.n_events == w.n_events
        _assert_hits(got, ref, gx, gy, gz)
        assert got.hit_offsets[1] == got.hit_offsets[2]  # the empty event has no hits
        hits.release()
        ev.wait(60)
        ev.release()


def test_first_consumer_reuses_the_stream_later_ones_wait(torch_cuda):
    w = synth.workload("full", n_events=2)
    with _ctx(w) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        s0 = ctx.stats()
        first = ev.hits()
        second = ev.hits()
        assert first.stream == ev.stream
        assert second.stream != ev.stream and second.stream != 0
        s1 = ctx.stats()
        assert s1["consumer_stream_reuses"] == s0["consumer_stream_reuses"] + 1
        waited = s1["consumer_stream_waits"] - s0["consumer_stream_waits"]
        assert waited in (0, 1)  # 0 only if the product had already completed
        assert ev.wait(60) == hp.HP_OK
        # product complete: a third consumer takes another stream and queues no wait
        third = ev.hits()
        assert third.stream != ev.stream
        assert ctx.stats()["consumer_stream_waits"] == s1["consumer_stream_waits"]
        res = [h.fetch() for h in (first, second, third) if h.wait(60) == hp.HP_OK]
        assert len(res) == 3
        for r in res[1:]:
            for f in ("hit_offsets", "event_status", "module", "x", "y", "z"):
                assert np.array_equal(getattr(r, f), getattr(res[0], f)), f
        for h in (first, second, third):
            h.release()
        ev.release()


def test_product_released_before_its_consumers_ran(torch_cuda):
    w = synth.workload("full", n_events=2)
    ref, gx, gy, gz = _oracle_hits(w)
    with _ctx(w) as ctx:
        for trial in range(6):
            ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
            consumers = [ev.hits() for _ in range(1 + trial % 3)]
            ev.release()  # deferred until every consumer's kernel has read the clusters
            if trial % 2:
                consumers[-1].release()  # a consumer released before it completes
                consumers = consumers[:-1]
            for h in consumers:
                assert h.wait(60) == hp.HP_OK
                _assert_hits(h.fetch(), ref, gx, gy, gz)
                h.release()
        torch_cuda.cuda.synchronize()


def test_hits_consumer_errors(torch_cuda):
    w = synth.workload("tiny", n_events=2)
    lib = hp.load()
    with _ctx(w, geometry=False) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        with pytest.raises(hp.HPError) as e:
            ev.hits()  # no geometry
        assert e.value.status == hp.HP_EINVAL
        origin, rot = synth.barrel_geometry(w.n_modules)
        assert lib.hp_set_geometry(ctx._h, origin.ctypes.data, rot.ctypes.data, 0.0, 0.015) == hp.HP_EINVAL
        assert lib.hp_set_geometry(ctx._h, origin.ctypes.data, rot.ctypes.data, float("nan"), 0.015) == hp.HP_EINVAL
        ctx.set_geometry(origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
        h = ev.hits()
        assert h.wait(60) == hp.HP_OK
        out = ctypes.c_void_p()
        assert lib.hp_enqueue_hits(h._h, 0, ctypes.byref(out)) == hp.HP_EINVAL  # not a clusters product
        assert lib.hp_enqueue_hits(ev._h, 1, ctypes.byref(out)) == hp.HP_EINVAL  # reserved flags
        assert lib.hp_fetch_clusters(h._h, ctypes.byref(hp.ClustersView())) == hp.HP_EINVAL
        assert lib.hp_fetch_hits(ev._h, ctypes.byref(hp.HitsView())) == hp.HP_EINVAL
        h.release()
        ev.release()


def test_new_geometry_applies_to_later_consumers_only(torch_cuda):
    w = synth.workload("full", n_events=1)
    ref = oracle.reconstruct_workload(w)
    origin, rot = synth.barrel_geometry(w.n_modules)
    shifted = origin + np.float32(1.0)
    with _ctx(w) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        a = ev.hits()
        ctx.set_geometry(shifted, rot, synth.PITCH_ROW, synth.PITCH_COL)
        b = ev.hits()
        assert a.wait(60) == hp.HP_OK and b.wait(60) == hp.HP_OK
        ha, hb = a.fetch(), b.fetch()
        gx, gy, gz = oracle.hits(ref.module, ref.x, ref.y, shifted, rot, synth.PITCH_ROW, synth.PITCH_COL)
        _assert_hits(hb, ref, gx, gy, gz)
        np.testing.assert_allclose(hb.x.astype(np.float64) - ha.x, 1.0, atol=1e-5)
        for h in (a, b, ev):
            h.release()


def test_device_chain_batched_workload(torch_cuda):
    """raw -> clusters -> hits device-resident on one stream, 256 events."""
    torch = torch_cuda
    w = synth.workload("batched")
    ref, gx, gy, gz = _oracle_hits(w)
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    with _ctx(w) as ctx:
        out = hp.DeviceOutputs(w.n_events, w.n_digis, dev, labels=False)
        cap = out.struct.capacity
        hx, hy, hz = (torch.full((cap,), -1.0, dtype=torch.float32, device=dev) for _ in range(3))
        stream = torch.cuda.current_stream(dev).cuda_stream
        ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                               out, stream)
        ctx.hits_device(w.n_events, cap, out.cluster_offsets.data_ptr(), out.module.data_ptr(), out.x.data_ptr(),
                        out.y.data_ptr(), hx.data_ptr(), hy.data_ptr(), hz.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.to_result(w.n_digis)
        C = got.n_clusters
        res = hp.HitsResult(got.status, w.n_events, got.cluster_offsets, got.event_status, got.module,
                            hx[:C].cpu().numpy(), hy[:C].cpu().numpy(), hz[:C].cpu().numpy(), 0)
        _assert_hits(res, ref, gx, gy, gz)
        if C < cap:  # nothing written past the clusters
            assert float(hx[C:].max()) == -1.0 and float(hx[C:].min()) == -1.0


def test_device_hits_module_outside_the_table_is_nan(torch_cuda):
    torch = torch_cuda
    w = synth.workload("tiny")
    dev = torch.device("cuda:0")
    with _ctx(w) as ctx:
        offs = torch.tensor([0, 3], dtype=torch.int64, device=dev)
        mod = torch.tensor([0, w.n_modules, w.n_modules - 1], dtype=torch.int32, device=dev)
        x = torch.tensor([79.5, 10.0, 79.5], dtype=torch.float32, device=dev)
        y = torch.tensor([207.5, 10.0, 207.5], dtype=torch.float32, device=dev)
        h = [torch.zeros(3, dtype=torch.float32, device=dev) for _ in range(3)]
        ctx.hits_device(1, 3, offs.data_ptr(), mod.data_ptr(), x.data_ptr(), y.data_ptr(), h[0].data_ptr(),
                        h[1].data_ptr(), h[2].data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize()
        hx, hy, hz = (t.cpu().numpy() for t in h)
        origin, _ = synth.barrel_geometry(w.n_modules)
        assert np.isnan(hx[1]) and np.isnan(hy[1]) and np.isnan(hz[1])
        # a centroid at the module centre lands on the module origin
        for i, m in ((0, 0), (2, w.n_modules - 1)):
            np.testing.assert_allclose([hx[i], hy[i], hz[i]], origin[m], atol=1e-6)
