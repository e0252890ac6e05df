"""Autotuner: installing cached choices (host only) and, on the GPU, tuning
small size classes and sorting correctly with the tuned choices."""
import json

import numpy as np
import pytest

import oracle
import paper_1506_01446_gb300 as bt
from paper_1506_01446_gb300 import autotune


def test_install_and_clear_cached_choices(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({"gpu": "TestGPU", "uint32": {"20": {"tile_log2": 13, "keys_per_thread_log2": 5,
                                                                     "global_bits": 0, "ms": 1.0}},
                                 "pairs": {}}))
    base = bt.plan_info(1 << 20)
    assert autotune.load(str(cache), gpu_name="OtherGPU") is None          # other GPU: ignored
    assert autotune.load(str(cache), gpu_name="TestGPU") is not None
    tuned = bt.plan_info(1 << 20)
    assert tuned["hbm_passes"] > base["hbm_passes"]                         # 8K tiles: more passes
    assert bt.plan_info(1 << 21) == bt.plan_info(1 << 21)
    bt.set_class_options(4, 20, None)
    assert bt.plan_info(1 << 20) == base


def test_rejected_choice():
    with pytest.raises(bt.BitonicError):
        bt.set_class_options(4, 20, {"tile_log2": 14, "keys_per_thread_log2": 3})  # no such config


@pytest.mark.gpu
def test_tune_small_classes_and_sort_with_choices(tmp_path):
    torch = pytest.importorskip("torch")
    res = autotune.tune(classes=(16, 18), pair_classes=(16,), reps=3, cache_path=str(tmp_path / "t.json"))
    assert set(res["uint32"]) == {"16", "18"} and set(res["pairs"]) == {"16"}
    import workloads
    for k in (16, 18):
        keys = workloads.uniform_u32((1 << k) - 5, seed=k)
        t = torch.from_numpy(keys.view(np.int32)).cuda()
        bt.sort_(t)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy().view(np.uint32), oracle.merge_sort(keys))
    for k in (16, 18):
        bt.set_class_options(4, k, None)
    bt.set_class_options(8, 16, None)


def test_segmented_option_validation_needs_no_gpu():
    bt.set_segmented_options(False, 16, dict(tile_log2=13, class_floor_gap=8, ctas_per_sm=1))
    bt.set_segmented_options(False, 16, None)
    for bad in (dict(tile_log2=12), dict(class_floor_gap=11), dict(ctas_per_sm=3)):
        with pytest.raises(bt.BitonicError):
            bt.set_segmented_options(False, 16, bad)
    with pytest.raises(bt.BitonicError):
        bt.set_segmented_options(True, 16, dict(tile_log2=14))   # pairs: 8K composites only


@pytest.mark.gpu
@pytest.mark.parametrize("pairs", [False, True])
def test_tune_segmented_and_sort_with_every_candidate(tmp_path, pairs):
    # every packed-tile candidate sorts a batch with segments from 1 key to
    # past one tile exactly like the oracle; the tuner caches a choice for
    # the batch's class of segment count
    torch = pytest.importorskip("torch")
    import workloads
    keys, offs = workloads.segmented_u32(3000, seed=8, max_len=20000)
    if pairs:
        keys = (keys >> np.uint32(25)).astype(np.uint32)   # ties: index order matters
    vals = np.arange(keys.size, dtype=np.uint32)
    cands = autotune.SEG_CANDIDATES_PAIRS if pairs else autotune.SEG_CANDIDATES_KEYS
    to = torch.from_numpy(offs).cuda()
    for cand in cands:
        bt.set_segmented_options(pairs, 12, cand)
        tk = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        if pairs:
            tv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
            bt.sort_segmented_pairs_(tk, tv, to)
            wk, wv = oracle.segmented_sort_pairs(keys, vals, offs)
            torch.cuda.synchronize()
            assert np.array_equal(tk.cpu().numpy().view(np.uint32), wk), cand
            assert np.array_equal(tv.cpu().numpy().view(np.uint32), wv), cand
        else:
            bt.sort_segmented_(tk, to)
            torch.cuda.synchronize()
            assert np.array_equal(tk.cpu().numpy().view(np.uint32), oracle.segmented_sort(keys, offs)), cand
    bt.set_segmented_options(pairs, 12, None)
    res = autotune.tune_segmented(keys, offs, pairs=pairs, reps=2, cache_path=str(tmp_path / "t.json"))
    assert res["class_log2_nseg"] == 12
    saved = json.loads((tmp_path / "t.json").read_text())
    assert "12" in saved["segmented_pairs" if pairs else "segmented_keys"]
    bt.set_segmented_options(pairs, 12, None)
