"""Failure detection on the GPU without a fault: the clustering kernel's one
kind of device-side wait (the ordered output waiting for earlier tickets'
cluster counts) is bounded by one second of wall time.  A test hook keeps
one ticket's count back so that the wait expires; the launch must end with
HP_ETIMEOUT on every event, in bounded time, and the context must stay
usable (the next launch gives the oracle's results)."""
import time

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


def test_expired_wait_reports_timeout_and_the_context_survives(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("batched", n_events=8)
    ref = oracle.reconstruct_workload(w)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)

        def run():
            ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                                   out, stream)
            torch.cuda.synchronize(dev)
            return out.to_result(w.n_digis)

        run()  # warm (workspace allocated)
        ctx.debug_expire_waits(1)
        t0 = time.monotonic()
        bad = run()
        dt = time.monotonic() - t0
        assert np.all(bad.event_status == hp.HP_ETIMEOUT)
        assert 0.5 < dt < 60  # the wait's one-second limit, not a hang
        assert_batch_matches(run(), ref, w.offsets)  # the next launch is exact again

        # host path: the completion callback delivers the status
        ctx.debug_expire_waits(1)
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        assert ev.wait(60) == hp.HP_ETIMEOUT
        assert ev.fetch().status == hp.HP_ETIMEOUT
        ev.release()
        ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
        assert ev.wait(60) == hp.HP_OK
        assert_batch_matches(ev.fetch(), ref, w.offsets)
        ev.release()
