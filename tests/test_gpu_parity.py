"""GPU parity: the sm_103a library against the CPU oracle, element by element.

Labels, cluster sets, ids, pixel counts and integer charges must be
bit-identical; FP32 centroids within 1e-4 pixel of the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests import shapes
from tests.gpu_util import CENTROID_TOL, assert_batch_matches, assert_event_matches, assert_events_match, \
    oracle_events

pytestmark = pytest.mark.gpu

SF = shapes.load()


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


_ctx_cache = {}


def ctx_for(n_modules, gain, pedestal, **kw):
    key = (n_modules, gain.tobytes(), pedestal.tobytes(), tuple(sorted(kw.items())))
    if key not in _ctx_cache:
        _ctx_cache[key] = hp.Context(n_modules, gain, pedestal, want_labels=True, **kw)
    return _ctx_cache[key]


def teardown_module(module):
    for c in _ctx_cache.values():
        c.close()
    _ctx_cache.clear()


def run_batch(ctx, words, mods, offsets, flags=0):
    ev = ctx.enqueue_batch(words, mods, offsets, flags=flags)
    ev.wait(120)
    res = ev.fetch()
    ev.release()
    return res


def test_hand_shapes_one_event_each(torch_cuda):
    ctx = ctx_for(SF.n_modules, SF.gain, SF.pedestal)
    for s in SF.shapes:
        w, m = s.arrays()
        ev = ctx.enqueue_event(w, m)
        st = ev.wait(60)
        got = ev.fetch()
        ev.release()
        assert st == s.status, s.name
        if st != 0:
            continue
        assert list(zip(got.module.tolist(), got.id.tolist(), got.charge.tolist(), got.npix.tolist())) == \
            [t[:4] for t in s.clusters], s.name
        for xg, yg, t in zip(got.x, got.y, s.clusters):
            assert abs(float(xg) - float(t[4])) <= CENTROID_TOL and abs(float(yg) - float(t[5])) <= CENTROID_TOL
        if s.labels is not None:
            assert got.label.tolist() == s.labels, s.name


def test_hand_shapes_as_one_batch(torch_cuda):
    ctx = ctx_for(SF.n_modules, SF.gain, SF.pedestal)
    w, m, offs, sel = SF.batch()
    got = run_batch(ctx, w, m, offs)
    ref = oracle.reconstruct_batch(w, m, offs, SF.n_modules, SF.gain, SF.pedestal)
    assert got.event_status.tolist() == [s.status for s in sel]
    assert_batch_matches(got, ref, offs)


@pytest.mark.parametrize("name", ["tiny", "full"])
def test_plain_event_matches_oracle(torch_cuda, name):
    w = synth.workload(name)
    words, mods = w.event(0)
    ref = oracle.reconstruct_event(words, mods, w.n_modules, w.gain, w.pedestal)
    ctx = ctx_for(w.n_modules, w.gain, w.pedestal)
    ev = ctx.enqueue_event(words, mods)
    assert ev.wait(60) == hp.HP_OK
    got = ev.fetch()
    ev.release()
    assert_batch_matches(got, ref, np.array([0, len(words)], np.uint64))


def test_full_literal_event(torch_cuda):
    """1% noise occupancy of all 1856 modules: ~1.5M digis in one event."""
    w = synth.workload("full_literal")
    ref = oracle.reconstruct_workload(w)
    got = run_batch(ctx_for(w.n_modules, w.gain, w.pedestal), w.words, w.modules, w.offsets)
    assert_batch_matches(got, ref, w.offsets)


def test_batched_uneven_events(torch_cuda):
    w = synth.workload("batched", n_events=24)
    ref = oracle.reconstruct_workload(w)
    got = run_batch(ctx_for(w.n_modules, w.gain, w.pedestal), w.words, w.modules, w.offsets)
    assert_batch_matches(got, ref, w.offsets)


def test_occupancy_events_with_hot_modules(torch_cuda):
    """Hot modules (13,312 pixels) exercise the global-scratch tier."""
    w = synth.workload("occupancy", n_events=2)
    ref = oracle.reconstruct_workload(w)
    got = run_batch(ctx_for(w.n_modules, w.gain, w.pedestal), w.words, w.modules, w.offsets)
    assert_batch_matches(got, ref, w.offsets)


def _module_with(n, rng, r0=10, c0=10, span=None):
    """n distinct pixels packed in a square window (dense enough to cluster)."""
    side = span or max(2, int(np.ceil(np.sqrt(n / 0.45))))
    side = min(side, 150)
    cells = rng.choice(side * min(side, 400), size=n, replace=False)
    rr = r0 + cells // min(side, 400)
    cc = c0 + cells % min(side, 400)
    assert rr.max() < 160 and cc.max() < 416
    adc = rng.integers(1, 60, n)
    return synth.pack(rr, cc, adc)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 63, 64, 65, 2048, 4095, 4096, 4097, 9000, 20000])
def test_tier_boundaries(torch_cuda, n):
    """Module sizes around the warp tiers (32, 64 digis) and the shared-memory tier (4096)."""
    rng = np.random.default_rng(n)
    gain = np.array([70, 75, 80], np.int32)
    ped = np.array([100, 0, 200], np.int32)
    words = _module_with(n, rng) if n else np.empty(0, np.uint32)
    other = _module_with(7, rng, r0=100, c0=300)
    w = np.concatenate([words, other])
    m = np.concatenate([np.ones(n, np.uint16), np.zeros(7, np.uint16)])
    perm = rng.permutation(len(w))
    w, m = w[perm], m[perm]
    offs = np.array([0, len(w)], np.uint64)
    ref = oracle.reconstruct_batch(w, m, offs, 3, gain, ped)
    got = run_batch(ctx_for(3, gain, ped), w, m, offs)
    assert_batch_matches(got, ref, offs)


def test_ragged_batch_with_empty_events(torch_cuda):
    base = synth.workload("tiny", n_events=6)
    sizes = [0, 1, 0, 33, 500, 0]
    ws, ms, offs = [], [], [0]
    for e, k in enumerate(sizes):
        w, m = base.event(e)
        ws.append(w[:k])
        ms.append(m[:k])
        offs.append(offs[-1] + k)
    w, m, offs = np.concatenate(ws), np.concatenate(ms), np.asarray(offs, np.uint64)
    ref = oracle.reconstruct_batch(w, m, offs, base.n_modules, base.gain, base.pedestal)
    got = run_batch(ctx_for(base.n_modules, base.gain, base.pedestal), w, m, offs)
    assert_batch_matches(got, ref, offs)


def test_bad_events_do_not_disturb_good_ones(torch_cuda):
    base = synth.workload("tiny", n_events=5)
    ws, ms, offs = [], [], [0]
    for e in range(5):
        w, m = base.event(e)
        w, m = w.copy(), m.copy()
        if e == 1:
            w[3] = w[3] | (1 << 25)            # high bits set
        if e == 2:
            m[0] = base.n_modules              # module out of range
        if e == 3:
            w = np.concatenate([w, w[:1]])     # duplicate position
            m = np.concatenate([m, m[:1]])
        ws.append(w)
        ms.append(m)
        offs.append(offs[-1] + len(w))
    w, m, offs = np.concatenate(ws), np.concatenate(ms), np.asarray(offs, np.uint64)
    ref = oracle.reconstruct_batch(w, m, offs, base.n_modules, base.gain, base.pedestal)
    assert ref.event_status.tolist() == [0, 4, 4, 5, 0]
    got = run_batch(ctx_for(base.n_modules, base.gain, base.pedestal), w, m, offs)
    assert got.event_status.tolist() == [0, 4, 4, 5, 0]
    assert_batch_matches(got, ref, offs)


def test_permutation_invariance(torch_cuda):
    w = synth.workload("full")
    words, mods = w.event(0)
    ctx = ctx_for(w.n_modules, w.gain, w.pedestal)
    offs = np.array([0, len(words)], np.uint64)
    a = run_batch(ctx, words, mods, offs)
    perm = np.random.default_rng(9).permutation(len(words))
    b = run_batch(ctx, words[perm], mods[perm], offs)
    for f in ("module", "id", "charge", "npix", "x", "y"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert np.array_equal(a.label[perm], b.label)


@pytest.mark.parametrize("pixel_thr,cluster_thr", [(1, 1), (2500, 6000), (1000, 100000)])
def test_other_thresholds(torch_cuda, pixel_thr, cluster_thr):
    w = synth.workload("tiny", n_events=3)
    ref = oracle.reconstruct_workload(w, pixel_thr=pixel_thr, cluster_thr=cluster_thr)
    ctx = ctx_for(w.n_modules, w.gain, w.pedestal, pixel_thr=pixel_thr, cluster_thr=cluster_thr)
    got = run_batch(ctx, w.words, w.modules, w.offsets)
    assert_batch_matches(got, ref, w.offsets)


def test_device_path_full_batched_workload(torch_cuda):
    """The 256-event batched workload, device-resident, as the benchmark runs it."""
    torch = torch_cuda
    w = synth.workload("batched")
    ref = oracle.reconstruct_workload(w)
    ctx = ctx_for(w.n_modules, w.gain, w.pedestal)
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):  # the second call reuses the warmed workspace
        ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                               out, stream.cuda_stream)
    torch.cuda.synchronize()
    got = out.to_result(w.n_digis)
    assert_batch_matches(got, ref, w.offsets)


def _device_run(torch, ctx, w):
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
    ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out,
                           torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    return out.to_result(w.n_digis)


def test_device_path_occupancy_every_event(torch_cuda):
    """All 64 high-occupancy events (~229M digis, hot modules at 20%
    occupancy) in one device launch with the autotuned settings, every event
    element by element against the oracle (run event by event on the host's
    cores)."""
    torch = torch_cuda
    w = synth.workload("occupancy")
    ctx = ctx_for(w.n_modules, w.gain, w.pedestal)
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
    ctx.autotune(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out, reps=1)
    got = _device_run(torch, ctx, w)
    assert np.all(got.event_status == 0)
    assert_events_match(got, oracle_events(w), w.offsets)


def test_many_small_events_on_large_geometry(torch_cuda):
    """Events of 1856 modules with ~100 digis each, so that one histogram
    range spans more (event, module) keys than a shared histogram holds (the
    one-by-one counting path), between ranges of large events that reserve
    their runs in bulk; device and host paths."""
    torch = torch_cuda
    big = synth.workload("full", n_events=3)
    ws, ms, offs = [], [], [0]
    for e in range(3):
        words, mods = big.event(e)
        ws.append(words)
        ms.append(mods)
        offs.append(offs[-1] + len(words))
        if e < 2:
            for k in range(40):
                sub_w, sub_m = big.event((e + 1) % 3)
                sel = np.random.default_rng(100 * e + k).choice(len(sub_w), 100, replace=False)
                ws.append(sub_w[sel])
                ms.append(sub_m[sel])
                offs.append(offs[-1] + 100)
    words, mods, offs = np.concatenate(ws), np.concatenate(ms), np.asarray(offs, np.uint64)
    ref = oracle.reconstruct_batch(words, mods, offs, big.n_modules, big.gain, big.pedestal)
    ctx = ctx_for(big.n_modules, big.gain, big.pedestal)
    got = run_batch(ctx, words, mods, offs)
    assert_batch_matches(got, ref, offs)
    dev = torch.device("cuda:0")
    out = hp.DeviceOutputs(len(offs) - 1, len(words), dev)
    d_offs = torch.from_numpy(offs.view(np.int64)).to(dev)  # held until the pass has run
    d_words = torch.from_numpy(words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(mods.view(np.int16)).to(dev)
    ctx.reconstruct_device(len(offs) - 1, len(words), d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out,
                           torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    assert_batch_matches(out.to_result(len(words)), ref, offs)


@pytest.mark.parametrize("kind", ["short_last", "decreasing", "nonzero_first"])
def test_malformed_offsets_report_einval(torch_cuda, kind):
    """Device entry with event offsets that do not run 0 <= ... <= N (all
    within the digi arrays, so nothing is read out of bounds): every event
    reports HP_EINVAL with no clusters, and the next call with good offsets
    is exact."""
    torch = torch_cuda
    w = synth.workload("tiny", n_events=4)
    ctx = ctx_for(w.n_modules, w.gain, w.pedestal)
    offs = w.offsets.copy()
    if kind == "short_last":
        offs[-1] -= 5
    elif kind == "decreasing":
        offs[2] = offs[1] - 1
    else:
        offs[0] = 1
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    d_offs = torch.from_numpy(offs.view(np.int64)).to(dev)  # held until the pass has run
    ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out,
                           stream)
    torch.cuda.synchronize()
    bad = out.to_result(w.n_digis)
    assert bad.event_status.tolist() == [hp.HP_EINVAL] * w.n_events
    assert int(bad.cluster_offsets[-1]) == 0
    got = _device_run(torch, ctx, w)
    assert_batch_matches(got, oracle.reconstruct_workload(w), w.offsets)


@pytest.mark.parametrize("rows,cols", [(40, 100), (50, 120)])
def test_heavy_cluster_exact_moments(torch_cuda, rows, cols):
    """One dense cluster whose moments overflow 32 bits (Q ~ 1.3e8): the 64-bit
    fallback, in the shared-memory tier (4000 digis) and the global tier (6000)."""
    rr, cc = np.meshgrid(np.arange(rows) + 60, np.arange(cols) + 200, indexing="ij")
    rr, cc = rr.ravel(), cc.ravel()
    rng = np.random.default_rng(rows)
    adc = rng.integers(200, 256, rr.size)
    words = synth.pack(rr, cc, adc)
    gain = np.array([126, 70], np.int32)
    ped = np.array([0, 100], np.int32)
    extra = synth.pack([3, 150], [3, 400], [90, 90])
    w = np.concatenate([words, extra])
    m = np.concatenate([np.zeros(rr.size, np.uint16), np.array([1, 1], np.uint16)])
    perm = rng.permutation(len(w))
    w, m = w[perm], m[perm]
    offs = np.array([0, len(w)], np.uint64)
    ref = oracle.reconstruct_batch(w, m, offs, 2, gain, ped)
    assert ref.charge[0] > 0x7FFFFFFF // 512
    got = run_batch(ctx_for(2, gain, ped), w, m, offs)
    assert_batch_matches(got, ref, offs)


def test_duplicates_in_block_tier_items(torch_cuda):
    """Items of ~1,400 digis (clustered by the whole block): a duplicate of a
    surviving pixel, of a dropped pixel, and a surviving and a dropped pixel
    at one position each flag their event HP_EDUP; the other events are
    unaffected."""
    base = synth.workload("batched", n_events=4)
    ws, ms, offs = [], [], [0]
    for e in range(4):
        w, m = base.event(e)
        w, m = w.copy(), m.copy()
        q = ((w >> 17) & 0xFF).astype(np.int64) * base.gain[m] - base.pedestal[m]
        if e == 0:
            i = int(np.flatnonzero(q >= 1000)[0])      # survivor twice
            extra_w, extra_m = w[i:i + 1], m[i:i + 1]
        elif e == 1:
            i = int(np.flatnonzero(q < 1000)[0])       # dropped pixel twice
            extra_w, extra_m = w[i:i + 1], m[i:i + 1]
        elif e == 2:
            i = int(np.flatnonzero(q >= 1000)[0])      # survivor and a dropped pixel (ADC 1) at one position
            extra_w = (w[i:i + 1] & np.uint32(0x1FFFF)) | np.uint32(1 << 17)
            extra_m = m[i:i + 1]
            assert int(base.gain[extra_m[0]]) - int(base.pedestal[extra_m[0]]) < 1000
        if e < 3:
            w, m = np.concatenate([w, extra_w]), np.concatenate([m, extra_m])
        ws.append(w)
        ms.append(m)
        offs.append(offs[-1] + len(w))
    w, m, offs = np.concatenate(ws), np.concatenate(ms), np.asarray(offs, np.uint64)
    ref = oracle.reconstruct_batch(w, m, offs, base.n_modules, base.gain, base.pedestal)
    assert ref.event_status.tolist() == [hp.HP_EDUP] * 3 + [0]
    got = run_batch(ctx_for(base.n_modules, base.gain, base.pedestal), w, m, offs)
    assert got.event_status.tolist() == [hp.HP_EDUP] * 3 + [0]
    assert_batch_matches(got, ref, offs)
