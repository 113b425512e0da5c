"""Pins of the CPU oracle against facts fixed independently of it.

* hand-worked shapes with expected values written by hand (tests/golden);
* exhaustive brute force: every subset of a 4x4 window, flood fill vs oracle;
* random tiny modules placed in the real 160 x 416 frame, flood fill vs oracle;
* scipy.ndimage.label with a full 3x3 structure on dense random grids;
* invariants on the synthetic workloads (permutation, batch = concatenation,
  charge conservation, labels vs npix, centroid inside the bounding box).

A plausible slip in the oracle (a dropped neighbour direction, a wrap across a
module edge, a wrong calibration sign, x and y swapped, a strict instead of
inclusive threshold, a cluster id that is not the minimum) fails at least one
of these.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import synth
from tests import shapes
from tests.bruteforce import bfs_reconstruct

SF = shapes.load()


def _oracle_shape(s, **kw):
    w, m = s.arrays()
    return oracle.reconstruct_event(w, m, SF.n_modules, SF.gain, SF.pedestal, pixel_thr=SF.pixel_thr,
                                    cluster_thr=SF.cluster_thr, **kw)


def _check_against_expected(c, exp_clusters, exp_labels, exp_status, tol=1e-12):
    assert c.status == exp_status
    got = list(zip(c.module.tolist(), c.id.tolist(), c.charge.tolist(), c.npix.tolist()))
    assert got == [t[:4] for t in exp_clusters]
    for xg, yg, t in zip(c.x, c.y, exp_clusters):
        assert abs(xg - float(t[4])) <= tol and abs(yg - float(t[5])) <= tol
    if exp_labels is not None:
        assert c.label.tolist() == list(exp_labels)


@pytest.mark.parametrize("name", [s.name for s in SF.shapes])
def test_hand_shape(name):
    s = next(s for s in SF.shapes if s.name == name)
    c = _oracle_shape(s)
    _check_against_expected(c, s.clusters, s.labels, s.status)


@pytest.mark.parametrize("name", [s.name for s in SF.shapes if s.name != "full_module"])
def test_bruteforce_agrees_with_hand_shapes(name):
    """The flood fill used below is itself pinned by the hand-worked values."""
    s = next(s for s in SF.shapes if s.name == name)
    w, m = s.arrays()
    st, cl, lab = bfs_reconstruct(w, m, SF.n_modules, SF.gain, SF.pedestal)
    assert st == s.status
    if st == 0:
        assert cl == s.clusters
        if s.labels is not None:
            assert lab == s.labels


def test_hand_shapes_as_one_batch():
    w, m, offs, sel = SF.batch()
    c = oracle.reconstruct_batch(w, m, offs, SF.n_modules, SF.gain, SF.pedestal)
    assert c.event_status.tolist() == [s.status for s in sel]
    for e, s in enumerate(sel):
        ce = c.event(e)
        _check_against_expected(ce, s.clusters, None, s.status)
        if s.labels is not None:
            assert c.label[int(offs[e]):int(offs[e + 1])].tolist() == s.labels


def _compare_with_bfs(words, modules, n_modules, gain, ped, **kw):
    c = oracle.reconstruct_event(words, modules, n_modules, gain, ped, **kw)
    st, cl, lab = bfs_reconstruct(words, modules, n_modules, gain, ped, **kw)
    assert c.status == st
    got = list(zip(c.module.tolist(), c.id.tolist(), c.charge.tolist(), c.npix.tolist()))
    assert got == [t[:4] for t in cl]
    for xg, yg, t in zip(c.x, c.y, cl):
        assert abs(xg - float(t[4])) <= 1e-9 and abs(yg - float(t[5])) <= 1e-9
    assert c.label.tolist() == lab
    return c


def test_exhaustive_4x4_window():
    """All 65536 subsets of a 4x4 window (8 x 8 geometry), one event each."""
    R = C = 8
    pos = [(2 + i // 4, 3 + i % 4) for i in range(16)]
    adc = [15 + 2 * i for i in range(16)]  # q = 1500..4500: some single pixels pass Q >= 4000
    gain = np.array([100], np.int32)
    ped = np.array([0], np.int32)
    words, offs = [], [0]
    for mask in range(1 << 16):
        for i in range(16):
            if mask >> i & 1:
                r, c = pos[i]
                words.append(r | (c << 8) | (adc[i] << 17))
        offs.append(len(words))
    words = np.asarray(words, np.uint32)
    mods = np.zeros(len(words), np.uint16)
    offs = np.asarray(offs, np.uint64)
    res = oracle.reconstruct_batch(words, mods, offs, 1, gain, ped, rows=R, cols=C)
    assert res.status == 0
    for mask in range(1 << 16):
        a, b = int(offs[mask]), int(offs[mask + 1])
        st, cl, lab = bfs_reconstruct(words[a:b], mods[a:b], 1, gain, ped, rows=R, cols=C)
        ca, cb = int(res.cluster_offsets[mask]), int(res.cluster_offsets[mask + 1])
        got = list(zip(res.module[ca:cb].tolist(), res.id[ca:cb].tolist(), res.charge[ca:cb].tolist(),
                       res.npix[ca:cb].tolist()))
        assert got == [t[:4] for t in cl], mask
        for xg, yg, t in zip(res.x[ca:cb], res.y[ca:cb], cl):
            assert abs(xg - float(t[4])) <= 1e-12 and abs(yg - float(t[5])) <= 1e-12
        assert res.label[a:b].tolist() == lab, mask


def test_window_subsets_at_module_corners():
    """Random subsets of 4x4 windows touching every corner of the real frame."""
    rng = np.random.default_rng(11)
    corners = [(0, 0), (0, 412), (156, 0), (156, 412), (78, 206)]
    gain = np.array([70, 100], np.int32)
    ped = np.array([150, 0], np.int32)
    for _ in range(400):
        r0, c0 = corners[rng.integers(len(corners))]
        words, mods = [], []
        for m in range(2):
            mask = rng.integers(1 << 16)
            for i in range(16):
                if mask >> i & 1:
                    words.append((r0 + i // 4) | ((c0 + i % 4) << 8) | (int(rng.integers(1, 80)) << 17))
                    mods.append(m)
        perm = rng.permutation(len(words))
        _compare_with_bfs(np.asarray(words, np.uint32)[perm], np.asarray(mods, np.uint16)[perm], 2, gain, ped)


@pytest.mark.parametrize("size", [8, 16, 32])
def test_random_tiny_modules(size):
    rng = np.random.default_rng(size)
    M = 6
    for trial in range(30):
        gain = rng.integers(60, 81, M).astype(np.int32)
        ped = rng.integers(0, 201, M).astype(np.int32)
        words, mods = [], []
        for m in range(M):
            r0 = int(rng.integers(0, 160 - size + 1))
            c0 = int(rng.integers(0, 416 - size + 1))
            occ = rng.uniform(0.05, 0.6)
            cells = np.flatnonzero(rng.uniform(size=size * size) < occ)
            for p in cells:
                words.append((r0 + p // size) | ((c0 + p % size) << 8) | (int(rng.integers(1, 60)) << 17))
                mods.append(m)
        perm = rng.permutation(len(words))
        _compare_with_bfs(np.asarray(words, np.uint32)[perm], np.asarray(mods, np.uint16)[perm], M, gain, ped)


def test_scipy_label_partition():
    """Connected components match scipy.ndimage.label with a full 3x3 structure."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    for occ in (0.2, 0.35, 0.5):
        grid = rng.uniform(size=(160, 416)) < occ
        rr, cc = np.nonzero(grid)
        adc = rng.integers(10, 40, len(rr))
        words = synth.pack(rr, cc, adc)
        mods = np.zeros(len(words), np.uint16)
        gain = np.array([100], np.int32)
        ped = np.array([0], np.int32)
        # cluster_thr 1: every component is kept, so the partition is complete
        c = oracle.reconstruct_event(words, mods, 1, gain, ped, cluster_thr=1)
        lab, nlab = ndimage.label(grid, structure=np.ones((3, 3), int))
        assert c.n_clusters == nlab
        comp_ids = lab[rr, cc]
        # two digis share an oracle label iff they share a scipy label
        pairs = {}
        for ol, sl in zip(c.label.tolist(), comp_ids.tolist()):
            assert pairs.setdefault(sl, ol) == ol
        assert len(set(pairs.values())) == nlab
        # each cluster id is the smallest linear index of its scipy component
        lin = rr * 416 + cc
        mins = np.full(nlab + 1, 1 << 30)
        np.minimum.at(mins, comp_ids, lin)
        assert sorted(c.id.tolist()) == sorted(mins[1:].tolist())


def _q(words, modules, gain, ped):
    adc = (words.astype(np.int64) >> 17) & 0xFF
    return adc * gain[modules].astype(np.int64) - ped[modules].astype(np.int64)


@pytest.mark.parametrize("name,events", [("tiny", None), ("full", None), ("batched", [0, 1, 2])])
def test_invariants_on_workloads(name, events):
    w = synth.workload(name, n_events=None if events is None else max(events) + 1)
    if events is not None:
        w = w.subset(events)
    c = oracle.reconstruct_workload(w)
    assert c.status == 0
    for e in range(w.n_events):
        words, mods = w.event(e)
        ce = c.event(e)
        lab = c.label[int(w.offsets[e]):int(w.offsets[e + 1])]
        q = _q(words, mods, w.gain, w.pedestal)
        # survivors are exactly the pixels at or above the pixel threshold
        assert np.array_equal(lab != -1, q >= 1000)
        # kept charge equals the charge of the labelled pixels
        assert int(ce.charge.astype(np.int64).sum()) == int(q[lab >= 0].sum())
        # strictly ordered by (module, id)
        key = ce.module.astype(np.int64) * (1 << 20) + ce.id
        assert np.all(np.diff(key) > 0)
        # every kept cluster above threshold; labels point to clusters of the right size
        assert np.all(ce.charge >= 4000)
        key_of_digi = mods.astype(np.int64) * (1 << 20) + lab
        kept = lab >= 0
        uniq, cnt = np.unique(key_of_digi[kept], return_counts=True)
        assert np.array_equal(uniq, key) and np.array_equal(cnt, ce.npix)
        # centroid lies in the bounding box of its pixels
        rows = (words & 0xFF).astype(np.int64)
        cols = ((words >> 8) & 0x1FF).astype(np.int64)
        order = np.argsort(key_of_digi[kept], kind="stable")
        kr, kc = rows[kept][order], cols[kept][order]
        starts = np.concatenate([[0], np.cumsum(ce.npix)[:-1]])
        assert np.all(ce.x >= np.minimum.reduceat(kr, starts) - 1e-9)
        assert np.all(ce.x <= np.maximum.reduceat(kr, starts) + 1e-9)
        assert np.all(ce.y >= np.minimum.reduceat(kc, starts) - 1e-9)
        assert np.all(ce.y <= np.maximum.reduceat(kc, starts) + 1e-9)
        # id is a member's linear index and the smallest one
        klin = (kr * 416 + kc)
        assert np.array_equal(np.minimum.reduceat(klin, starts), ce.id)


@pytest.mark.parametrize("name", ["tiny", "full"])
def test_bruteforce_on_workload(name):
    w = synth.workload(name)
    words, mods = w.event(0)
    _compare_with_bfs(words, mods, w.n_modules, w.gain, w.pedestal)


def test_permutation_invariance():
    w = synth.workload("full")
    words, mods = w.event(0)
    c0 = oracle.reconstruct_event(words, mods, w.n_modules, w.gain, w.pedestal)
    rng = np.random.default_rng(3)
    for _ in range(3):
        perm = rng.permutation(len(words))
        c1 = oracle.reconstruct_event(words[perm], mods[perm], w.n_modules, w.gain, w.pedestal)
        for f in ("module", "id", "charge", "npix", "x", "y"):
            assert np.array_equal(getattr(c0, f), getattr(c1, f))
        assert np.array_equal(c0.label[perm], c1.label)


def test_batch_is_concatenation():
    w = synth.workload("batched", n_events=4)
    cb = oracle.reconstruct_workload(w)
    for e in range(4):
        words, mods = w.event(e)
        ce = oracle.reconstruct_event(words, mods, w.n_modules, w.gain, w.pedestal)
        cbe = cb.event(e)
        for f in ("module", "id", "charge", "npix", "x", "y"):
            assert np.array_equal(getattr(ce, f), getattr(cbe, f))
        assert np.array_equal(ce.label, cb.label[int(w.offsets[e]):int(w.offsets[e + 1])])


@pytest.mark.parametrize("pixel_thr,cluster_thr", [(1, 1), (1500, 1), (1000, 10000), (2500, 6000)])
def test_other_thresholds_against_bruteforce(pixel_thr, cluster_thr):
    w = synth.workload("tiny")
    words, mods = w.event(0)
    _compare_with_bfs(words, mods, w.n_modules, w.gain, w.pedestal, pixel_thr=pixel_thr,
                      cluster_thr=cluster_thr)


def test_invalid_configuration():
    w = synth.workload("tiny")
    words, mods = w.event(0)
    assert oracle.reconstruct_event(words, mods, w.n_modules, w.gain, w.pedestal, pixel_thr=0).status == \
        oracle.EINVAL
    bad_gain = w.gain.copy()
    bad_gain[3] = 127  # 255 * 127 exceeds INT32_MAX / 66560 = 32263
    assert oracle.reconstruct_event(words, mods, w.n_modules, bad_gain, w.pedestal * 0).status == oracle.EINVAL
    assert oracle.reconstruct_event(words, mods, w.n_modules, w.gain * 0 + 126, w.pedestal * 0).status == oracle.OK


def test_centroid_is_exact_division():
    """x = sum(q*row)/Q in double, i.e. the correctly rounded quotient."""
    s = next(s for s in SF.shapes if s.name == "spiral")
    c = _oracle_shape(s)
    assert c.x[0] == float(Fraction(8591, 123)) and c.y[0] == float(Fraction(38338, 123))
