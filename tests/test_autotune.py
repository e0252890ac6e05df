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
