"""Parser for the hand-worked cluster shapes in tests/golden/hand_shapes.txt."""
from __future__ import annotations

import os
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_shapes.txt")
STATUS = {"OK": 0, "EBADDIGI": 4, "EDUP": 5}


@dataclass
class Shape:
    name: str
    words: list = field(default_factory=list)
    modules: list = field(default_factory=list)
    clusters: list = field(default_factory=list)  # (module, id, charge, npix, Fraction x, Fraction y)
    labels: list | None = None
    status: int = 0

    def arrays(self):
        return np.asarray(self.words, np.uint32), np.asarray(self.modules, np.uint16)


@dataclass
class ShapeFile:
    n_modules: int
    rows: int
    cols: int
    pixel_thr: int
    cluster_thr: int
    gain: np.ndarray
    pedestal: np.ndarray
    shapes: list

    def batch(self, names=None):
        """Concatenate shapes into one batch: (words, modules, offsets, shapes)."""
        sel = [s for s in self.shapes if names is None or s.name in names]
        ws, ms, offs = [], [], [0]
        for s in sel:
            w, m = s.arrays()
            ws.append(w)
            ms.append(m)
            offs.append(offs[-1] + len(w))
        return (np.concatenate(ws).astype(np.uint32), np.concatenate(ms).astype(np.uint16),
                np.asarray(offs, np.uint64), sel)


def _word(row, col, adc):
    return int(row) | (int(col) << 8) | (int(adc) << 17)


def load(path: str = GOLDEN) -> ShapeFile:
    shapes, cur = [], None
    geom = None
    calib = {}
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            t = line.split()
            k = t[0]
            if k == "geometry":
                geom = [int(v) for v in t[1:]]
            elif k == "calib":
                calib[int(t[1])] = (int(t[2]), int(t[3]))
            elif k == "event":
                cur = Shape(t[1])
            elif k == "digi":
                m, r, c, a = (int(v) for v in t[1:])
                cur.words.append(_word(r, c, a))
                cur.modules.append(m)
            elif k == "word":
                cur.modules.append(int(t[1]))
                cur.words.append(int(t[2], 16))
            elif k == "fill":
                m, a = int(t[1]), int(t[2])
                for r in range(geom[1]):
                    for c in range(geom[2]):
                        cur.words.append(_word(r, c, a))
                        cur.modules.append(m)
            elif k == "hseg":
                m, r, c0, c1, a = (int(v) for v in t[1:])
                for c in range(c0, c1 + 1):
                    cur.words.append(_word(r, c, a))
                    cur.modules.append(m)
            elif k == "vseg":
                m, c, r0, r1, a = (int(v) for v in t[1:])
                for r in range(r0, r1 + 1):
                    cur.words.append(_word(r, c, a))
                    cur.modules.append(m)
            elif k == "cluster":
                cur.clusters.append((int(t[1]), int(t[2]), int(t[3]), int(t[4]), Fraction(t[5]), Fraction(t[6])))
            elif k == "labels":
                cur.labels = [int(v) for v in t[1:]]
            elif k == "status":
                cur.status = STATUS[t[1]]
            elif k == "end":
                shapes.append(cur)
                cur = None
            else:
                raise ValueError(f"bad record {line!r}")
    M = geom[0]
    gain = np.array([calib[m][0] for m in range(M)], np.int32)
    ped = np.array([calib[m][1] for m in range(M)], np.int32)
    return ShapeFile(M, geom[1], geom[2], geom[3], geom[4], gain, ped, shapes)
