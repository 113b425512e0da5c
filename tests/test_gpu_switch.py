"""GPU tests of the runtime choice of technology (Sec. 3, the SwitchProducer):
on a host with a GPU, HP_FORCE_CPU selects the CPU case, and both cases
give the same product on the one-event, full-geometry and batched workloads:
offsets, statuses, cluster ids, charges, sizes and labels identical, the
float centroids within the 1e-4 pixel tolerance (each case rounds its
quotient once; the GPU's warp tier rounds relative to the seed pixel), and
the provenance names the case that ran."""
import numpy as np
import pytest

from paper_2004_04334_gb300 import hp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _product(w, monkeypatch, force, flags, per_event=False):
    monkeypatch.setenv("HP_FORCE_CPU", force)
    out = []
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        jobs = [w.subset([e]) for e in range(w.n_events)] if per_event else [w]
        for j in jobs:
            if per_event:
                ev = ctx.enqueue_event(j.words, j.modules, flags=flags)
            else:
                ev = ctx.enqueue_batch(j.words, j.modules, j.offsets, flags=flags)
            assert ev.wait(120) == hp.HP_OK
            out.append((ev.fetch(), ev.provenance()))
            ev.release()
    return out


@pytest.mark.parametrize("name,n", [("tiny", 8), ("full", 2), ("batched", 16)])
@pytest.mark.parametrize("per_event", [False, True])
def test_both_cases_give_the_same_product(torch_cuda, monkeypatch, name, n, per_event):
    w = synth.workload(name, n_events=n)
    for flags in (hp.HP_WANT_LABELS, hp.HP_LABELS_U16):
        gpu = _product(w, monkeypatch, "0", flags, per_event)
        cpu = _product(w, monkeypatch, "1", flags, per_event)
        for (g, pg), (c, pc) in zip(gpu, cpu):
            assert pg["path"] == ("event" if per_event else "batch") and pg["device"] >= 0
            assert pc["path"] == "cpu" and pc["device"] == -1
            for f in ("cluster_offsets", "event_status", "module", "id", "charge", "npix", "label", "label16",
                      "item_first"):
                a, b = getattr(g, f), getattr(c, f)
                assert (a is None) == (b is None), f
                assert a is None or np.array_equal(a, b), f
            for f in ("x", "y"):
                d = np.abs(getattr(g, f).astype(np.float64) - getattr(c, f))
                assert d.size == 0 or d.max() <= 1e-4, (f, d.max())


def test_allow_cpu_still_takes_the_gpu_when_there_is_one(torch_cuda, monkeypatch):
    """HP_ALLOW_CPU only permits the CPU case where no device is usable: on a
    host with a GPU the context is the GPU case."""
    monkeypatch.delenv("HP_FORCE_CPU", raising=False)
    w = synth.workload("tiny", n_events=2)
    with hp.Context(w.n_modules, w.gain, w.pedestal, allow_cpu=True) as ctx:
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        assert ev.wait(60) == hp.HP_OK
        prov = ev.provenance()
        ev.release()
    assert prov["path"] == "batch" and prov["device"] >= 0
