"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a
standalone driver (tests/oracle_sanitize_main.c) built with
-fsanitize=address,undefined runs the hand-worked shapes, invalid and
duplicate digis, empty events and synthetic batches; it must report nothing
and give exactly the results of the normal build."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import synth
from tests import shapes

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    exe = str(tmp_path_factory.mktemp("san") / "oracle_san")
    r = subprocess.run([gcc, "-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        "-fno-omit-frame-pointer", os.path.join(HERE, "oracle_sanitize_main.c"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitizer build unavailable: " + r.stderr[-200:])
    return exe


def _run(driver, tmp_path, words, mods, offs, n_modules, gain, ped, pthr=1000, cthr=4000, rows=160, cols=416):
    inp, outp = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    E, N = len(offs) - 1, int(offs[-1])
    with open(inp, "wb") as f:
        f.write(np.array([n_modules, rows, cols], np.uint32).tobytes())
        f.write(np.array([pthr, cthr], np.int32).tobytes())
        f.write(np.array([E], np.uint32).tobytes())
        f.write(np.array([N], np.uint64).tobytes())
        for a, t in ((gain, np.int32), (ped, np.int32), (offs, np.uint64), (words, np.uint32), (mods, np.uint16)):
            f.write(np.ascontiguousarray(a, t).tobytes())
    r = subprocess.run([driver, inp, outp], capture_output=True, text=True,
                       env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1"))
    assert r.returncode == 0, r.stderr[-2000:]
    assert "runtime error" not in r.stderr and "ERROR:" not in r.stderr, r.stderr[-2000:]
    b = open(outp, "rb").read()
    pos = 0

    def get(dtype, n):
        nonlocal pos
        a = np.frombuffer(b, dtype, n, pos)
        pos += a.nbytes
        return a

    st = int(get(np.int32, 1)[0])
    C = int(get(np.uint64, 1)[0])
    res = dict(status=st, cluster_offsets=get(np.uint64, E + 1), event_status=get(np.int32, E),
               module=get(np.uint32, C), id=get(np.int32, C), charge=get(np.int32, C), npix=get(np.int32, C),
               x=get(np.float64, C), y=get(np.float64, C), label=get(np.int32, N))
    return res


def _same(res, ref):
    assert res["status"] == ref.status
    for f in ("cluster_offsets", "event_status", "module", "id", "charge", "npix", "x", "y", "label"):
        assert np.array_equal(res[f], getattr(ref, f)), f


def test_hand_shapes_under_sanitizers(driver, tmp_path):
    sf = shapes.load()
    words, mods, offs, _ = sf.batch()
    ref = oracle.reconstruct_batch(words, mods, offs, sf.n_modules, sf.gain, sf.pedestal, sf.pixel_thr,
                                   sf.cluster_thr, sf.rows, sf.cols)
    _same(_run(driver, tmp_path, words, mods, offs, sf.n_modules, sf.gain, sf.pedestal, sf.pixel_thr,
               sf.cluster_thr, sf.rows, sf.cols), ref)


@pytest.mark.parametrize("name,n_events", [("tiny", 6), ("full", 1), ("batched", 2)])
def test_synthetic_batches_under_sanitizers(driver, tmp_path, name, n_events):
    w = synth.workload(name, n_events=n_events)
    # add an empty event and an event with an invalid word
    bad = np.array([(1 << 25) | 5], np.uint32)
    words = np.concatenate([w.words, bad])
    mods = np.concatenate([w.modules, np.array([0], np.uint16)])
    offs = np.concatenate([w.offsets, [w.offsets[-1], w.offsets[-1] + 1]]).astype(np.uint64)
    ref = oracle.reconstruct_batch(words, mods, offs, w.n_modules, w.gain, w.pedestal)
    _same(_run(driver, tmp_path, words, mods, offs, w.n_modules, w.gain, w.pedestal), ref)
