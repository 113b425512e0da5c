"""GPU tests of the autotuner: every candidate setting of the clustering
kernel gives the oracle's results (on shapes that exercise the warp tier,
the hash label store at each group size, the shared-memory tile and the
global-memory tier), hp_autotune keeps the fastest per shape bucket, and the
cache file round-trips across contexts."""
import json
import os

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


def _run(torch, ctx, w, dev):
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    out = hp.DeviceOutputs(w.n_events, w.n_digis, dev)
    ctx.reconstruct_device(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out,
                           torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize(dev)
    return out.to_result(w.n_digis), (d_offs, d_words, d_mods, out)


WORKLOADS = [("batched", 12), ("full", 2), ("occupancy", 1)]
DEFAULT = {"tile_slots": 4096, "blocks_per_sm": 2, "ticket_items": 16, "warp_max": 64,
           "label_store": hp.HP_STORE_BITMAP, "item_threads": 512}


@pytest.mark.parametrize("name,n_events", WORKLOADS)
def test_every_candidate_matches_the_oracle(torch_cuda, name, n_events):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload(name, n_events=n_events)
    ref = oracle.reconstruct_workload(w)
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        cands = ctx.tuning_candidates()
        assert len(cands) >= 4
        assert dict(DEFAULT) in cands
        # both label stores, and the hash store at every group size
        assert {(c["label_store"], c["item_threads"]) for c in cands} == \
            {(hp.HP_STORE_BITMAP, 512), (hp.HP_STORE_HASH, 128), (hp.HP_STORE_HASH, 256), (hp.HP_STORE_HASH, 512)}
        for c in cands:
            ctx.set_tuning(w.n_events, w.n_digis, c)
            assert ctx.get_tuning(w.n_events, w.n_digis) == c
            got, _ = _run(torch, ctx, w, dev)
            assert_batch_matches(got, ref, w.offsets)


def test_autotune_keeps_the_fastest_and_results_stay_exact(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("batched", n_events=32)
    ref = oracle.reconstruct_workload(w)
    with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
        default = ctx.get_tuning(w.n_events, w.n_digis)
        far = ctx.get_tuning(1, 10)
        _, (d_offs, d_words, d_mods, out) = _run(torch, ctx, w, dev)
        best, best_ms, ms = ctx.autotune(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(),
                                         d_mods.data_ptr(), out, reps=2)
        cands = ctx.tuning_candidates()
        assert len(ms) == len(cands) and all(m > 0 for m in ms)
        assert best == cands[int(np.argmin(ms))] and best_ms == min(ms)
        assert ctx.get_tuning(w.n_events, w.n_digis) == best
        assert_batch_matches(out.to_result(w.n_digis), ref, w.offsets)  # autotune leaves a valid result
        got, _ = _run(torch, ctx, w, dev)
        assert_batch_matches(got, ref, w.offsets)
        # another bucket is untouched; clearing restores the defaults
        assert ctx.get_tuning(1, 10) == far
        ctx.set_tuning(w.n_events, w.n_digis, None)
        assert ctx.get_tuning(w.n_events, w.n_digis) == default
        bad = dict(default, blocks_per_sm=5)
        assert ctx.try_set_tuning(w.n_events, w.n_digis, bad) == hp.HP_EINVAL
        assert ctx.try_set_tuning(w.n_events, w.n_digis, dict(default, tile_slots=100)) == hp.HP_EINVAL
        assert ctx.try_set_tuning(w.n_events, w.n_digis, dict(default, warp_max=48)) == hp.HP_EINVAL
        assert ctx.try_set_tuning(w.n_events, w.n_digis, dict(default, label_store=2)) == hp.HP_EINVAL
        # the bitmap store takes a block an item; the hash store 128, 256 or 512 threads
        assert ctx.try_set_tuning(w.n_events, w.n_digis,
                                  dict(default, label_store=hp.HP_STORE_BITMAP, item_threads=256)) == hp.HP_EINVAL
        assert ctx.try_set_tuning(w.n_events, w.n_digis,
                                  dict(default, label_store=hp.HP_STORE_HASH, item_threads=64)) == hp.HP_EINVAL
        assert ctx.try_set_tuning(w.n_events, w.n_digis,
                                  dict(default, label_store=hp.HP_STORE_HASH, item_threads=256)) == hp.HP_OK


def test_cache_file_round_trip_and_off_switch(torch_cuda, tmp_path, monkeypatch):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    w = synth.workload("batched", n_events=8)
    path = str(tmp_path / "tune.jsonl")
    monkeypatch.setenv("HP_TUNE_CACHE", path)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        _, (d_offs, d_words, d_mods, out) = _run(torch, ctx, w, dev)
        best, _, _ = ctx.autotune(w.n_events, w.n_digis, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                                  out, reps=1)
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and '"tile_slots"' in lines[0]
    entry = json.loads(lines[0])
    assert {k: entry[k] for k in best} == best
    # force a non-default choice into the file so that the reload is visible
    other = {"tile_slots": 4096, "blocks_per_sm": 2, "ticket_items": 8, "warp_max": 64,
             "label_store": hp.HP_STORE_HASH, "item_threads": 256}
    with open(path, "a") as f:
        f.write(json.dumps(dict(entry, **other)) + "\n")
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        assert ctx.get_tuning(w.n_events, w.n_digis) == other
    monkeypatch.setenv("HP_TUNE", "off")
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        off = ctx.get_tuning(w.n_events, w.n_digis)
    assert off != other
    monkeypatch.delenv("HP_TUNE")
    monkeypatch.delenv("HP_TUNE_CACHE")
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:  # nothing tuned: the same size default
        assert ctx.get_tuning(w.n_events, w.n_digis) == off
    os.remove(path)


def test_untuned_buckets_take_the_nearest_tuned_entry(torch_cuda):
    w = synth.workload("batched", n_events=8)
    with hp.Context(w.n_modules, w.gain, w.pedestal) as ctx:
        small = ctx.get_tuning(1, 10)  # one digi per item on average: the plain default
        assert small == DEFAULT
        big = ctx.get_tuning(w.n_events, w.n_digis)  # over a thousand digis per item: single-block tile
        assert big["blocks_per_sm"] == 1 and big["tile_slots"] > 4096
        pick = dict(DEFAULT, ticket_items=8, warp_max=32)
        ctx.set_tuning(w.n_events, w.n_digis, pick)
        assert ctx.get_tuning(2 * w.n_events, 2 * w.n_digis) == pick  # one bucket away
        assert ctx.get_tuning(1, 10) == small  # far away: still the default
