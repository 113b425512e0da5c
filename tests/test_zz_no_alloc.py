"""The allocation-free entry point, called through the C ABI, against the
CPU oracle.

hp_reconstruct_device_noalloc serves callers that must not allocate device
memory: a cudaMalloc or cudaFree synchronises the whole device (stalling
every stream a hosting framework has in flight), and some frameworks own
all of the device's memory through their own allocator.  Its scratch is a
fixed array inside the library instead.  Two calls in a row must both give
the oracle's result (integers bit-exact, centroids within the tests' 1e-4
px), including an item larger than the shared-memory tile (its scratch is in
the fixed array too), the second call must leave the device's free memory
unchanged, and a call beyond the array's limits must be refused with
HP_ECAPACITY.  This file is collected last so that a failure here leaves
every other test already run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_batch_matches

pytestmark = pytest.mark.gpu

MAX_DIGIS = 131072


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _call(torch, lib, ctx, n_events, n_digis, d_offs, d_words, d_mods, out, dev):
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = lib.hp_reconstruct_device_noalloc(ctx._h, n_events, n_digis, d_offs.data_ptr(), d_words.data_ptr(),
                                           d_mods.data_ptr(), ctypes.byref(out.struct), ctypes.c_void_p(stream))
    assert st == hp.HP_OK, hp.status_string(st)
    torch.cuda.synchronize(dev)


def _big_module_input():
    """One event on a 3-module geometry: a 9,000-digi module (beyond the
    4,096-slot shared-memory tile), a 2,000-digi one and a small one."""
    rng = np.random.default_rng(4334)
    parts, mods = [], []
    for m, (n, r0, c0, side) in enumerate([(9000, 5, 5, 140), (2000, 40, 200, 70), (7, 150, 400, 4)]):
        cells = rng.choice(side * side, size=n, replace=False)
        rr, cc = r0 + cells // side, c0 + cells % side
        rr, cc = np.minimum(rr, 159), np.minimum(cc, 415)
        keep = np.unique(rr * 416 + cc, return_index=True)[1]
        parts.append(synth.pack(rr[keep], cc[keep], rng.integers(1, 60, keep.size)))
        mods.append(np.full(keep.size, m, np.uint16))
    w, m = np.concatenate(parts), np.concatenate(mods)
    perm = rng.permutation(len(w))
    gain = np.array([70, 75, 80], np.int32)
    ped = np.array([100, 0, 200], np.int32)
    return w[perm], m[perm], np.array([0, len(w)], np.uint64), 3, gain, ped


def _case(name):
    if name == "big_module":
        return _big_module_input()
    w = synth.workload(name, n_events=40 if name == "tiny" else 1)
    return w.words, w.modules, w.offsets, w.n_modules, w.gain, w.pedestal


@pytest.mark.parametrize("name", ["full", "tiny", "big_module"])
def test_noalloc_matches_oracle_twice_without_allocating(torch_cuda, name):
    torch = torch_cuda
    lib = hp.load()
    words, mods, offs, n_modules, gain, ped = _case(name)
    E, N = len(offs) - 1, len(words)
    assert N <= MAX_DIGIS
    ref = oracle.reconstruct_batch(words, mods, offs, n_modules, gain, ped)
    assert ref.n_clusters > 0
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(mods.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(offs.view(np.int64)).to(dev)
    outs = [hp.DeviceOutputs(E, N, dev) for _ in range(2)]
    for o in outs:
        o.cluster_offsets.fill_(-1)
        o.event_status.fill_(-1)
    with hp.Context(n_modules, gain, ped, want_labels=True) as ctx:
        _call(torch, lib, ctx, E, N, d_offs, d_words, d_mods, outs[0], dev)
        free_before = torch.cuda.mem_get_info(dev)[0]
        _call(torch, lib, ctx, E, N, d_offs, d_words, d_mods, outs[1], dev)
        free_after = torch.cuda.mem_get_info(dev)[0]
    assert free_after == free_before, "the second call changed the device's free memory"
    for o in outs:
        assert_batch_matches(o.to_result(N), ref, offs)


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
