"""GPU tests of the CUDA-graph form of the device-resident pass
(hp_graph_capture / hp_graph_launch / hp_graph_destroy): a replay gives the
results of a direct call, reads its input buffers at launch time, allocates
nothing, and graphs left over are destroyed with their context."""
import numpy as np
import pytest

from oracle import oracle
from paper_2004_04334_gb300 import hp, synth
from tests.gpu_util import assert_batch_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _device_inputs(torch, w, dev):
    return (torch.from_numpy(w.offsets.view(np.int64)).to(dev), torch.from_numpy(w.words.view(np.int32)).to(dev),
            torch.from_numpy(w.modules.view(np.int16)).to(dev))


def test_graph_replay_matches_direct_call_and_reads_buffers_at_launch(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("batched", n_events=24)
    d_offs, d_words, d_mods = _device_inputs(torch, w, dev)
    stream = torch.cuda.Stream(dev)
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        direct = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
        ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                               direct, stream.cuda_stream)
        out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
        g = ctx.graph_capture(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out)
        torch.cuda.synchronize(dev)
        before = ctx.stats()
        for _ in range(3):
            g.launch(stream.cuda_stream)
        torch.cuda.synchronize(dev)
        after = ctx.stats()
        assert after["device_mallocs"] == before["device_mallocs"]
        assert after["kernel_launches"] - before["kernel_launches"] == 3 * 6
        a, b = direct.to_result(w.n_digis), out.to_result(w.n_digis)
        for f in ("cluster_offsets", "event_status", "module", "id", "charge", "npix", "x", "y", "label"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
        # same sizes, new contents: every event's digis reversed in place
        rev = w.words.copy()
        revm = w.modules.copy()
        for e in range(w.n_events):
            s, t = int(w.offsets[e]), int(w.offsets[e + 1])
            rev[s:t] = rev[s:t][::-1]
            revm[s:t] = revm[s:t][::-1]
        d_words.copy_(torch.from_numpy(rev.view(np.int32)).to(dev))
        d_mods.copy_(torch.from_numpy(revm.view(np.int16)).to(dev))
        torch.cuda.synchronize(dev)
        g.launch(stream.cuda_stream)
        torch.cuda.synchronize(dev)
        ref = oracle.reconstruct_batch(rev, revm, w.offsets, w.n_modules, w.gain, w.pedestal)
        assert_batch_matches(out.to_result(w.n_digis), ref, w.offsets)
        g.destroy()
        g.destroy()  # a second destroy is a no-op in the binding


def test_graph_left_over_is_destroyed_with_the_context(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("tiny", n_events=4)
    d_offs, d_words, d_mods = _device_inputs(torch, w, dev)
    ctx = hp.Context(w.n_modules, w.gain, w.pedestal)
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev, labels=False)
    g = ctx.graph_capture(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out)
    g.launch(torch.cuda.current_stream(dev).cuda_stream)
    ctx.close()  # waits for the replay, frees the graph
    ref = oracle.reconstruct_workload(w)
    got = out.to_result(w.n_digis)
    assert np.array_equal(got.cluster_offsets, ref.cluster_offsets)
    assert np.array_equal(got.id, ref.id)


def test_graph_capture_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("tiny")
    lib = hp.load()
    import ctypes
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        out = hp.DeviceOutputs(1, w.n_digis, dev, labels=False)
        h = ctypes.c_void_p()
        assert lib.hp_graph_capture(ctx._h, 0, 0, 8, 0, 0, ctypes.byref(out.struct), ctypes.byref(h)) == hp.HP_EINVAL
        assert lib.hp_graph_capture(ctx._h, 1, 10, None, None, None, ctypes.byref(out.struct),
                                    ctypes.byref(h)) == hp.HP_EINVAL
        assert lib.hp_graph_launch(None, None) == hp.HP_EINVAL
        assert lib.hp_graph_destroy(None) == hp.HP_EINVAL
