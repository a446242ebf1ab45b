"""The autotuner: its workload classes and cache on the CPU; on the GPU, every tuning it may pick gives the same
M and O, and the pick is applied and cached."""
import numpy as np
import pytest

from paper_2408_14050_gb300 import autotune


def test_workload_classes():
    assert autotune.size_class([(480, 640)]) == "small"
    assert autotune.size_class([(480, 640), (1080, 1920)]) == "medium"
    assert autotune.size_class([(2160, 4096)]) == "large"
    assert autotune.scan_bucket(117) == "L<=254" and autotune.scan_bucket(740) == "L<=1022"
    assert autotune.angle_class([(0.0, 1), (90.0, 1), (270.0, 1)]) == "axial"
    assert autotune.angle_class([(0.0, 1), (45.0, 1.4), (315.0, 1.4)]) == "octant"
    assert autotune.angle_class([(0.0, 1), (30.0, 1.4)]) == "general"
    k = autotune.workload_key("GB300", [(1080, 1920)], [(0.0, 1.0)], 117, 8)
    assert k == "GB300|medium|L<=254|axial|N8"


def test_candidates_cover_every_mapping():
    c = autotune.candidates(3)
    assert {t["line_max_runs"] for t in c} == {0, 1, 2}
    assert {t["warp_lines_per_block"] for t in c} == {4, 8}
    assert all(1 <= t["line_blocks_per_sm"] <= 3 for t in c)
    assert {t["strip_px"] for t in c} == {0, *autotune.STRIP_SHAPES}
    assert {(t["strip_px"], t["fused"]) for t in c if t["strip_px"]} == {(px, f) for px in autotune.STRIP_SHAPES
                                                                       for f in (0, 1)}
    assert len({autotune.tuning_name(t) for t in c}) == len(c)


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"k": {"tuning": {"line_max_runs": 1}}}, path)
    assert autotune.load_cache(path)["k"]["tuning"]["line_max_runs"] == 1


@pytest.mark.gpu
def test_every_tuning_gives_the_same_result(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_14050_gb300 as occ
    import scenes
    D = torch.from_numpy(scenes.array_3x3(frame=3, H=270, W=480).frames[0]).cuda()
    views = scenes.views_3x3()
    with occ.occ_create(0, max_pixels=270 * 480, max_views=8) as ctx:
        M0, O0 = occ.occ_detect(ctx, D, views)
        _, max_bps = occ.occ_get_tuning(ctx)
        for t in autotune.candidates(max_bps):
            occ.occ_set_tuning(ctx, t)
            M, O = occ.occ_detect(ctx, D, views)
            assert occ.occ_get_status(ctx) == occ.OCC_OK
            assert torch.equal(O, O0) and torch.equal(M, M0), t
        best, ms = autotune.autotune(ctx, [D], views, reps=2, cache_path=str(tmp_path / "t.json"))
        assert best in autotune.candidates(max_bps) and len(ms) == len(autotune.candidates(max_bps))
        assert occ.occ_get_tuning(ctx)[0] == best
        again, _ = autotune.autotune(ctx, [D], views, reps=2, cache_path=str(tmp_path / "t.json"))
        assert again == best
        with pytest.raises(occ.OccError):
            occ.occ_set_tuning(ctx, {"line_max_runs": 3, "line_blocks_per_sm": 1, "warp_lines_per_block": 8})
        for px in (512, 4100, occ.OCC_STRIP_PX_MAX + 64):       # too small, not a multiple of 64, too large
            with pytest.raises(occ.OccError):
                occ.occ_set_tuning(ctx, {"line_max_runs": 2, "line_blocks_per_sm": 1, "warp_lines_per_block": 8,
                                         "strip_px": px})
        with pytest.raises(occ.OccError):
            occ.occ_set_tuning(ctx, {"line_max_runs": 2, "line_blocks_per_sm": 1, "warp_lines_per_block": 8,
                                     "strip_px": 4096, "fused": 2})
