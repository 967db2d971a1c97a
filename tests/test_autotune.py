"""Host logic of the tile-depth autotuner (size classes and the JSON cache)."""
import importlib

import pytest


def test_size_class_buckets():
    from paper_2601_01787_gb300 import autotune
    assert autotune.size_class((512, 512, 512)) == autotune.size_class((500, 520, 510))
    assert autotune.size_class((64, 64, 64)) != autotune.size_class((512, 512, 512))
    assert autotune.size_class((1, 1, 1)) == "z1_p1"


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("MSZ_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2601_01787_gb300 import autotune
    importlib.reload(autotune)
    try:
        assert autotune.lookup((100, 100, 100), device_key="GB300") == autotune.DEFAULT
        autotune.record((100, 100, 100), 16, {8: 1.0, 16: 0.5, 32: 0.7, 64: 0.9}, "GB300")
        assert autotune.lookup((100, 100, 100), device_key="GB300") == 16
        assert autotune.lookup((101, 99, 100), device_key="GB300") == 16
        assert autotune.lookup((100, 100, 100), device_key="other") == autotune.DEFAULT
    finally:
        monkeypatch.delenv("MSZ_AUTOTUNE_CACHE")
        importlib.reload(autotune)


@pytest.mark.gpu
def test_tile_depth_changes_speed_not_results():
    import numpy as np
    import torch

    from paper_2601_01787_gb300 import api, autotune, synth
    fl = synth.perlin3d_prequant((70, 90, 130), seed=5, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    ref = api.correct(f, fh, fl.xi)
    for tz in autotune.CANDIDATES + (1, 3, 100):
        r = api.correct(f, fh, fl.xi, tile_z=tz)
        assert torch.equal(r.out.view(torch.int32), ref.out.view(torch.int32))
        assert torch.equal(r.edit_idx, ref.edit_idx)
    assert autotune.tune((70, 90, 130), reps=1) in autotune.CANDIDATES
