"""GPU tests of the split cluster transfer of the host paths: the leading
positions go through device columns and one DMA each, sized from the
clusters-per-digi ratio of recent launches, the rest straight to mapped host
memory.  Launches far below and far above the estimate (one blob, isolated
pixels) alternate with ordinary ones, and every result equals the oracle."""
import numpy as np
import pytest

from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_events_match, oracle_events

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _events(w):
    """Three batches on w's geometry: isolated pixels (a cluster per digi),
    one large blob per module (almost no clusters), and w's own events."""
    rows, cols = np.meshgrid(np.arange(0, synth.ROWS, 2), np.arange(0, synth.COLS, 2), indexing="ij")
    r, c = rows.ravel()[:3000], cols.ravel()[:3000]
    iso_w = np.concatenate([synth.pack(r, c, np.full(len(r), 200)) for _ in range(8)])
    iso_m = np.repeat(np.arange(8, dtype=np.uint16), len(r))
    br, bc = np.meshgrid(np.arange(20, 80), np.arange(30, 130), indexing="ij")
    blob_w = np.concatenate([synth.pack(br.ravel(), bc.ravel(), np.full(br.size, 200)) for _ in range(8)])
    blob_m = np.repeat(np.arange(8, dtype=np.uint16), br.size)
    out = []
    for words, mods in ((iso_w, iso_m), (blob_w, blob_m)):
        half = len(words) // 2
        out.append(synth.Workload(w.name, w.n_modules, words.astype(np.uint32), mods,
                                  np.array([0, half, len(words)], np.uint64), w.gain, w.pedestal))
    out.append(w)
    return out


def test_split_transfer_matches_the_oracle_when_the_estimate_is_off(torch_cuda):
    w = synth.workload("batched", n_events=6)
    batches = _events(w)
    refs = [oracle_events(b) for b in batches]
    order = [2, 0, 0, 2, 1, 1, 0, 2, 1, 2]  # ratio ~0.14, then ~1 (capped), ~0, back
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        for k in order:
            b = batches[k]
            ev = ctx.enqueue_batch(b.words, b.modules, b.offsets)
            assert ev.wait(120) == hp.HP_OK
            r = ev.fetch()
            ev.release()
            assert_events_match(r, refs[k], b.offsets)
        # the serving path splits the same way
        ctx.serve_start(budget_bytes=4 << 30, want_labels=True)
        evs = []
        for k in order:
            b = batches[k]
            for e in range(b.n_events):
                s, t = int(b.offsets[e]), int(b.offsets[e + 1])
                evs.append((k, e, ctx.submit(b.words[s:t], b.modules[s:t])))
        for k, e, ev in evs:
            assert ev.wait(120) == hp.HP_OK
            r = ev.fetch()
            ev.release()
            b = batches[k]
            assert_events_match(r, [refs[k][e]], np.array([0, int(b.offsets[e + 1] - b.offsets[e])], np.uint64))
        ctx.serve_stop()
