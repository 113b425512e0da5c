"""GPU tests of the hash label store of the clustering kernel (tuning
label_store = HP_STORE_HASH, item_threads = 128, 256 or 512 threads an
item): the hand-worked shapes pushed out of the warp tier, a cluster heavy
enough for the exact 64-bit moments, items on both sides of the store's
capacity in one launch, and duplicate or invalid digis inside its items,
each against the oracle or the stated clusters."""
import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests import shapes
from tests.gpu_util import CENTROID_TOL, assert_batch_matches

pytestmark = pytest.mark.gpu

SF = shapes.load()


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _hash_settings(ctx):
    cands = [c for c in ctx.tuning_candidates() if c["label_store"] == hp.HP_STORE_HASH]
    assert {c["item_threads"] for c in cands} == {128, 256, 512}
    return cands


def _run(ctx, words, mods, offs, tuning, flags=hp.HP_WANT_LABELS):
    E, N = len(offs) - 1, int(offs[-1])
    ctx.set_tuning(E, N, tuning)
    assert ctx.get_tuning(E, N) == tuning
    ev = ctx.enqueue_batch(words, mods, offs, flags=flags)
    st = ev.wait(120)
    r = ev.fetch()
    prov = ev.provenance()
    ev.release()
    assert prov["tuning"] == tuning
    return st, r


def _smem(t, rows=synth.ROWS, cols=synth.COLS):
    nwords = (rows * cols + 31) // 32
    return t["tile_slots"] * 20 + nwords * 12


def _capacity(t):
    """The hash store's largest item for setting t (its slice of shared memory
    at 28 bytes a digi plus 256 row counters, its share of the tile, at most
    8 digis a thread, 5 at three blocks per SM, at most 4096)."""
    groups = 512 // t["item_threads"]
    per_thread = 5 if t["blocks_per_sm"] >= 3 else 8
    sl = (_smem(t) // groups) & ~15
    return min((sl - 1024) // 28, t["tile_slots"] // groups, per_thread * t["item_threads"], 4096)


def _padded(s, n_pad=80, seed=0):
    """Shape s with n_pad isolated pixels below the pixel threshold added to
    the module of its first digi, at positions the shape does not use, so
    that the item leaves the warp tier (more than 64 digis) while its
    clusters stay the same.  Shapes already above the warp tier (or empty)
    are returned as they are."""
    w, m = s.arrays()
    if len(w) == 0 or len(w) > 64:
        return w, m
    mod = int(m[0])
    used = {(int(x) & 0xFF, (int(x) >> 8) & 0x1FF) for x, mm in zip(w, m) if int(mm) == mod}
    adc = 1
    assert adc * int(SF.gain[mod]) - int(SF.pedestal[mod]) < SF.pixel_thr
    rng = np.random.default_rng(seed)
    pad = []
    while len(pad) < n_pad:
        r, c = int(rng.integers(0, SF.rows)), int(rng.integers(0, SF.cols))
        if (r, c) in used:
            continue
        used.add((r, c))
        pad.append(synth.pack([r], [c], [adc])[0])
    pw = np.concatenate([w, np.asarray(pad, np.uint32)])
    pm = np.concatenate([m, np.full(n_pad, mod, np.uint16)])
    perm = rng.permutation(len(pw))
    return pw[perm], pm[perm]


def test_hand_shapes_through_the_hash_store(torch_cuda):
    with hp.Context(SF.n_modules, SF.gain, SF.pedestal, want_labels=True) as ctx:
        for t in _hash_settings(ctx):
            for s in SF.shapes:
                if s.status != 0 or not s.words:
                    continue
                w, m = _padded(s)
                offs = np.array([0, len(w)], np.uint64)
                st, got = _run(ctx, w, m, offs, t)
                assert st == hp.HP_OK, s.name
                assert list(zip(got.module.tolist(), got.id.tolist(), got.charge.tolist(), got.npix.tolist())) == \
                    [c[:4] for c in s.clusters], (s.name, t)
                for xg, yg, c in zip(got.x, got.y, s.clusters):
                    assert abs(float(xg) - float(c[4])) <= CENTROID_TOL, s.name
                    assert abs(float(yg) - float(c[5])) <= CENTROID_TOL, s.name


@pytest.mark.parametrize("rows,cols", [(20, 40), (30, 50)])
def test_heavy_cluster_in_the_hash_store(torch_cuda, rows, cols):
    """One dense cluster (800 or 1,500 digis, Q ~ 2e7-4e7) whose moments
    overflow 32 bits: the hash store's exact 64-bit pass, at every group size
    whose capacity holds it (the others send it to the bitmap tiers)."""
    rr, cc = np.meshgrid(np.arange(rows) + 60, np.arange(cols) + 200, indexing="ij")
    rr, cc = rr.ravel(), cc.ravel()
    rng = np.random.default_rng(rows)
    adc = rng.integers(200, 256, rr.size)
    gain = np.array([126, 70], np.int32)
    ped = np.array([0, 100], np.int32)
    words = np.concatenate([synth.pack(rr, cc, adc), synth.pack([3, 150], [3, 400], [90, 90])])
    mods = np.concatenate([np.zeros(rr.size, np.uint16), np.array([1, 1], np.uint16)])
    perm = rng.permutation(len(words))
    words, mods = words[perm], mods[perm]
    offs = np.array([0, len(words)], np.uint64)
    ref = oracle.reconstruct_batch(words, mods, offs, 2, gain, ped)
    assert ref.charge[0] > 0x7FFFFFFF // 512
    with hp.Context(2, gain, ped, want_labels=True) as ctx:
        held = 0
        for t in _hash_settings(ctx):
            held += rr.size <= _capacity(t)
            st, got = _run(ctx, words, mods, offs, t)
            assert st == hp.HP_OK
            assert_batch_matches(got, ref, offs)
        assert held > 0


def test_items_on_both_sides_of_the_capacity(torch_cuda):
    """In one launch: items of exactly the capacity, one digi over it, and
    one digi over the warp tier, for every hash setting; compact and 32-bit
    labels."""
    rng = np.random.default_rng(7)
    gain = np.full(4, 70, np.int32)
    ped = np.full(4, 50, np.int32)
    with hp.Context(4, gain, ped, want_labels=True) as ctx:
        for t in _hash_settings(ctx):
            cap = _capacity(t)
            ws, ms = [], []
            for mod, n in enumerate((cap, cap + 1, t["warp_max"] + 1, 3)):
                lin = rng.choice(synth.ROWS * synth.COLS, size=n, replace=False)
                adc = rng.integers(1, 256, n)
                ws.append(synth.pack(lin // synth.COLS, lin % synth.COLS, adc))
                ms.append(np.full(n, mod, np.uint16))
            words, mods = np.concatenate(ws), np.concatenate(ms)
            perm = rng.permutation(len(words))
            words, mods = words[perm], mods[perm]
            offs = np.array([0, len(words)], np.uint64)
            ref = oracle.reconstruct_batch(words, mods, offs, 4, gain, ped)
            st, got = _run(ctx, words, mods, offs, t)
            assert st == hp.HP_OK
            assert_batch_matches(got, ref, offs)
            st, g16 = _run(ctx, words, mods, offs, t, flags=hp.HP_LABELS_U16)
            assert st == hp.HP_OK
            assert np.array_equal(g16.labels_from_compact(offs, mods), ref.label)


def test_duplicates_and_invalid_digis_in_hash_items(torch_cuda):
    """Events whose items run in the hash store: a duplicated surviving
    pixel, a duplicated pixel below threshold, and an ADC of zero flag their
    own event only; the unflagged event matches the oracle."""
    base = synth.workload("full", n_events=4)
    ws, ms, offs = [], [], [0]
    for e in range(4):
        w, m = base.event(e)
        w, m = w.copy(), m.copy()
        counts = np.bincount(m, minlength=base.n_modules)
        big = int(np.argmax(counts))  # an inner module: well over the warp tier
        idx = np.nonzero(m == big)[0]
        assert len(idx) > 64
        q = ((w[idx] >> 17) & 0xFF).astype(np.int64) * int(base.gain[big]) - int(base.pedestal[big])
        if e == 1:  # a surviving pixel twice
            k = idx[np.argmax(q)]
            w = np.append(w, w[k])
            m = np.append(m, m[k])
        if e == 2:  # a pixel below threshold twice (added, then repeated)
            free = set(range(synth.ROWS * synth.COLS)) - {int(x & 0xFF) * synth.COLS + int((x >> 8) & 0x1FF)
                                                          for x in w[idx]}
            lin = min(free)
            low = synth.pack([lin // synth.COLS], [lin % synth.COLS], [1])
            w = np.concatenate([w, low, low])
            m = np.concatenate([m, [big, big]]).astype(np.uint16)
        if e == 3:  # an ADC of zero
            w[idx[0]] = w[idx[0]] & ~np.uint32(0xFF << 17)
        ws.append(w)
        ms.append(m)
        offs.append(offs[-1] + len(w))
    words, mods = np.concatenate(ws).astype(np.uint32), np.concatenate(ms).astype(np.uint16)
    offs = np.asarray(offs, np.uint64)
    with hp.Context(base.n_modules, base.gain, base.pedestal, want_labels=True) as ctx:
        for t in _hash_settings(ctx):
            st, got = _run(ctx, words, mods, offs, t)
            assert list(got.event_status) == [hp.HP_OK, hp.HP_EDUP, hp.HP_EDUP, hp.HP_EBADDIGI], t
            ref0 = oracle.reconstruct_batch(words[:int(offs[1])], mods[:int(offs[1])], offs[:2], base.n_modules,
                                            base.gain, base.pedestal)
            a, b = int(got.cluster_offsets[0]), int(got.cluster_offsets[1])
            assert np.array_equal(got.id[a:b], ref0.id) and np.array_equal(got.charge[a:b], ref0.charge)
            assert np.array_equal(got.label[:int(offs[1])], ref0.label)
            # (the cluster slices of the flagged events are unspecified)
