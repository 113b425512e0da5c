"""CPU test of the hash label store's algorithm (the clustering kernel's
`hash_item`), written as a sequential model of its phases: the table of 2n
slots with multiplicative hashing and linear probing, union-find on packed
(pixel index, digi index) keys with the smaller key as the root, the
neighbour rule (left and up; without up, upper-left unless left survives,
and upper-right), and ordinals from per-row counts of kept roots, a scan
in groups of eight rows and a rank by column within the row.  The model
takes the digis of each item in a random order and must give the oracle's
clusters, in the oracle's order, and the oracle's labels.  This checks the
design on CPU; the kernel itself is compared with the oracle by the GPU
tests."""
import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import synth

IDX = 12  # digi index bits of a packed key


def _home(lin, H):
    return (((lin * 0x9E3779B1) & 0xFFFFFFFF) * H) >> 32


def _model_item(words, gain, ped, rows, cols, pixel_thr, cluster_thr, rng):
    """Clusters (id, charge, npix, sum q*row, sum q*col) in ordinal order and
    the label of every digi of one item, by the hash store's phases."""
    n = len(words)
    H = 2 * n
    table = [0] * H
    par = [None] * n
    for j in rng.permutation(n):                    # insertion in any order
        x = int(words[j])
        r, c, adc = x & 0xFF, (x >> 8) & 0x1FF, (x >> 17) & 0xFF
        lin = r * cols + c
        surv = adc * gain - ped >= pixel_thr
        e = ((lin + 1) << 13) | (int(surv) << 12) | int(j)
        s = _home(lin, H)
        for _ in range(H):
            if table[s] == 0:
                table[s] = e
                break
            assert (table[s] >> 13) != lin + 1
            s = (s + 1) % H
        else:
            raise AssertionError("table full")
        if surv:
            par[j] = (lin << IDX) | int(j)

    def survivor(lin):
        s = _home(lin, H)
        for _ in range(H):
            e = table[s]
            if e == 0:
                return 0
            if (e >> 13) == lin + 1:
                return e if (e >> 12) & 1 else 0
            s = (s + 1) % H
        return 0

    def key(e):
        return (((e >> 13) - 1) << IDX) | (e & ((1 << IDX) - 1))

    def find(x):
        while par[x & ((1 << IDX) - 1)] != x:
            x = par[x & ((1 << IDX) - 1)]
        return x

    def union(a, b):
        a, b = find(a), find(b)
        if a != b:
            a, b = max(a, b), min(a, b)
            par[a & ((1 << IDX) - 1)] = b

    mine = {}
    for j in rng.permutation(n):                    # unions in any order
        if par[j] is None:
            continue
        x = int(words[j])
        r, c = x & 0xFF, (x >> 8) & 0x1FF
        lin = r * cols + c
        mine[j] = (lin << IDX) | int(j)
        e_left = survivor(lin - 1) if c > 0 else 0
        e1, e2 = e_left, 0
        if r > 0:
            e_up = survivor(lin - cols)
            if e_up:
                e2 = e_up
            else:
                if not e_left and c > 0:
                    e1 = survivor(lin - cols - 1)
                if c + 1 < cols:
                    e2 = survivor(lin - cols + 1)
        for e in (e1, e2):
            if e:
                union(mine[j], key(e))

    root = {j: find(k) for j, k in mine.items()}
    sums = {}
    for j, rt in root.items():
        x = int(words[j])
        q = ((x >> 17) & 0xFF) * gain - ped
        s = sums.setdefault(rt, [0, 0, 0, 0])
        s[0] += q
        s[1] += 1
        s[2] += q * (x & 0xFF)
        s[3] += q * ((x >> 8) & 0x1FF)
    labels = [-1] * n
    rowcnt = [0] * 256
    arrival = {}
    for j in rng.permutation(n):                    # kept roots counted per row
        if j not in root:
            continue
        kept = sums[root[j]][0] >= cluster_thr
        labels[j] = root[j] >> IDX if kept else -2
        if kept and root[j] == mine[j]:
            r = int(words[j]) & 0xFF
            arrival[j] = rowcnt[r]
            rowcnt[r] += 1
    eight = [sum(rowcnt[8 * l:8 * l + 8]) for l in range(32)]
    base8 = np.concatenate([[0], np.cumsum(eight)[:-1]])
    K = sum(eight)
    lists = [None] * K
    pre = {}
    for j, a in arrival.items():
        x = int(words[j])
        r = x & 0xFF
        pre[j] = int(base8[r >> 3]) + sum(rowcnt[r & ~7:r])
        lists[pre[j] + a] = (x >> 8) & 0x1FF
    out = [None] * K
    for j, p in pre.items():
        x = int(words[j])
        r, c = x & 0xFF, (x >> 8) & 0x1FF
        o = p + sum(1 for i in range(p, p + rowcnt[r]) if lists[i] < c)
        assert out[o] is None
        out[o] = (root[j] >> IDX, *sums[root[j]])
    return out, labels


@pytest.mark.parametrize("name,n_events,lo,hi", [("tiny", 3, 1, 4096), ("full", 1, 33, 917)])
def test_hash_store_model_matches_the_oracle(name, n_events, lo, hi):
    w = synth.workload(name, n_events=n_events)
    ref = oracle.reconstruct_workload(w)
    rng = np.random.default_rng(11)
    checked = 0
    for e in range(w.n_events):
        a, b = int(w.offsets[e]), int(w.offsets[e + 1])
        ev = ref.event(e)
        mods, words = w.modules[a:b], w.words[a:b]
        for m in np.unique(mods):
            idx = rng.permutation(np.flatnonzero(mods == m))
            if not lo <= len(idx) <= hi:
                continue
            out, labels = _model_item(words[idx], int(w.gain[m]), int(w.pedestal[m]), synth.ROWS, synth.COLS,
                                      oracle.PIXEL_THR, oracle.CLUSTER_THR, rng)
            sel = ev.module == m
            assert [o[0] for o in out] == ev.id[sel].tolist()
            assert [o[1] for o in out] == ev.charge[sel].tolist()
            assert [o[2] for o in out] == ev.npix[sel].tolist()
            assert np.allclose([o[3] / o[1] for o in out], ev.x[sel], rtol=0, atol=1e-9)
            assert np.allclose([o[4] / o[1] for o in out], ev.y[sel], rtol=0, atol=1e-9)
            assert labels == ref.label[a + idx].tolist()
            checked += 1
    assert checked > 0
