"""Brute-force flood fill: an independent, obviously-correct restatement of
8-connected pixel clustering used to pin the oracle on small inputs.

It decodes digi words with Python integers, calibrates each pixel, and grows
every cluster by breadth-first search over a dict of surviving pixels; the
centroid is kept as an exact Fraction.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction


def bfs_reconstruct(words, modules, n_modules, gain, ped, pixel_thr=1000, cluster_thr=4000, rows=160, cols=416):
    """Return (status, clusters, labels); clusters are tuples
    (module, id, charge, npix, Fraction x, Fraction y) sorted by (module, id)."""
    n = len(words)
    dec = []
    for i in range(n):
        w = int(words[i])
        m = int(modules[i])
        r, c, a = w & 0xFF, (w >> 8) & 0x1FF, (w >> 17) & 0xFF
        if r >= rows or c >= cols or a < 1 or (w >> 25) or m >= n_modules:
            return 4, [], [-1] * n
        dec.append((m, r, c, a))
    seen = set()
    for m, r, c, _ in dec:
        if (m, r, c) in seen:
            return 5, [], [-1] * n
        seen.add((m, r, c))
    alive = {}
    labels = [-1] * n
    for i, (m, r, c, a) in enumerate(dec):
        q = a * int(gain[m]) - int(ped[m])
        if q >= pixel_thr:
            alive[(m, r, c)] = (i, q)
    visited = set()
    clusters = []
    members_of = []
    for key in sorted(alive):
        if key in visited:
            continue
        comp = []
        dq = deque([key])
        visited.add(key)
        while dq:
            m, r, c = dq.popleft()
            comp.append((m, r, c))
            for dr in (-1, 0, 1):
                for dc in (-1, 0, 1):
                    nb = (m, r + dr, c + dc)
                    if (dr or dc) and nb in alive and nb not in visited:
                        visited.add(nb)
                        dq.append(nb)
        m = comp[0][0]
        cid = min(r * cols + c for _, r, c in comp)
        Q = sum(alive[p][1] for p in comp)
        sr = sum(alive[p][1] * p[1] for p in comp)
        sc = sum(alive[p][1] * p[2] for p in comp)
        members_of.append((comp, Q >= cluster_thr, cid))
        if Q >= cluster_thr:
            clusters.append((m, cid, Q, len(comp), Fraction(sr, Q), Fraction(sc, Q)))
    for comp, kept, cid in members_of:
        for p in comp:
            labels[alive[p][0]] = cid if kept else -2
    clusters.sort(key=lambda t: (t[0], t[1]))
    return 0, clusters, labels
