"""The allocation-free entry point, called through the C ABI, against the
allocating device entry point.

hp_reconstruct_device_noalloc is for callers that may not allocate device
memory (cudaMalloc/cudaFree synchronise the device and are off limits in
some hosting frameworks): its scratch is a fixed array inside the library.
Two calls in a row must both give the results of hp_reconstruct_device on
the same input (integers bit-exact, centroids within the tests' 1e-4 px),
and a call beyond the array's limits must be refused with HP_ECAPACITY.
This file is collected last so that a failure here leaves every other test
already run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import CENTROID_TOL

pytestmark = pytest.mark.gpu

MAX_DIGIS = 131072


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _results(torch, lib, fn, ctx, w, d_offs, d_words, d_mods, dev):
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
    out.cluster_offsets.fill_(-1)
    out.event_status.fill_(-1)
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = getattr(lib, fn)(ctx._h, w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                          ctypes.byref(out.struct), ctypes.c_void_p(stream))
    assert st == hp.HP_OK, hp.status_string(st)
    torch.cuda.synchronize(dev)
    return out.to_result(w.n_digis)


def _same(a, b):
    assert a.event_status.tolist() == b.event_status.tolist()
    assert np.array_equal(a.cluster_offsets, b.cluster_offsets)
    for f in ("module", "id", "charge", "npix"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    for f in ("x", "y"):
        d = np.abs(getattr(a, f).astype(np.float64) - getattr(b, f))
        assert d.size == 0 or d.max() <= CENTROID_TOL, f
    assert np.array_equal(a.label, b.label)


@pytest.mark.parametrize("name,n_events", [("full", 1), ("tiny", 40)])
def test_noalloc_matches_allocating_entry_twice(torch_cuda, name, n_events):
    torch = torch_cuda
    lib = hp.load()
    w = synth.workload(name, n_events=n_events)
    assert w.n_digis <= MAX_DIGIS
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        ref = _results(torch, lib, "hp_reconstruct_device", ctx, w, d_offs, d_words, d_mods, dev)
        assert ref.status == hp.HP_OK and ref.n_clusters > 0
        before = ctx.stats()["device_mallocs"]
        first = _results(torch, lib, "hp_reconstruct_device_noalloc", ctx, w, d_offs, d_words, d_mods, dev)
        second = _results(torch, lib, "hp_reconstruct_device_noalloc", ctx, w, d_offs, d_words, d_mods, dev)
        assert ctx.stats()["device_mallocs"] == before
    _same(first, ref)
    _same(second, ref)


def test_noalloc_refuses_oversized_calls(torch_cuda):
    torch = torch_cuda
    lib = hp.load()
    w = synth.workload("tiny")
    dev = torch.device("cuda:0")
    d_words = torch.zeros(MAX_DIGIS + 1, dtype=torch.int32, device=dev)
    d_mods = torch.zeros(MAX_DIGIS + 1, dtype=torch.int16, device=dev)
    d_offs = torch.tensor([0, MAX_DIGIS + 1], dtype=torch.int64, device=dev)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        out = hp.DeviceOutputs(1, MAX_DIGIS + 1, dev, labels=False)
        st = lib.hp_reconstruct_device_noalloc(ctx._h, 1, MAX_DIGIS + 1, d_offs.data_ptr(), d_words.data_ptr(),
                                               d_mods.data_ptr(), ctypes.byref(out.struct),
                                               ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
        assert st == hp.HP_ECAPACITY
        # too many (event, module) items
        many = 16384 // w.n_modules + 1
        offs = torch.zeros(many + 1, dtype=torch.int64, device=dev)
        out2 = hp.DeviceOutputs(many, 1, dev, labels=False)
        st = lib.hp_reconstruct_device_noalloc(ctx._h, many, 0, offs.data_ptr(), d_words.data_ptr(),
                                               d_mods.data_ptr(), ctypes.byref(out2.struct),
                                               ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
        assert st == hp.HP_ECAPACITY
