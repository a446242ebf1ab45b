"""Median fusion of the stereo disparity maps (Section 4.2) and the masked backward warp of the peripheral images
(Section 1, Section 4.2) on the GPU, bit for bit against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("W", [301, 304])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 16, 17, 24, 32, 33, 64])
def test_median_matches_oracle(n, W):
    H = 37
    D = scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(40, n))
    maps = scenes.stereo_maps(D, n, seed=scenes.seed_of(41, n))
    got = occ.occ_fuse_median([cuda(m) for m in maps])
    np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), oracle.median(maps).view(np.uint32))


@pytest.mark.parametrize("offset", [4, 5])          # 16-byte aligned and unaligned rows
def test_median_full_size_ties_signed_zeros_and_pitch(offset):
    H, W = 1080, 1920
    D = scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(42, 0))
    maps = scenes.stereo_maps(D, 8, seed=scenes.seed_of(43, 0))
    maps[1][::7] = np.round(maps[1][::7])            # many exact ties between maps
    maps[2][::7] = np.round(maps[2][::7])
    maps[3][:5] = -0.0                               # signed zeros
    maps[4][:5] = 0.0
    big = [torch.zeros((H, W + 40), dtype=torch.float32, device="cuda") for _ in maps]
    views = []
    for b, m in zip(big, maps):
        b[:, offset:offset + W].copy_(cuda(m))
        views.append(b[:, offset:offset + W])        # row stride W + 40
    out = torch.full((H, W + 8), -1.0, device="cuda")
    st = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    occ.occ_fuse_median(views, D=out[:, :W], status=st)
    assert int(st.item()) == occ.OCC_OK
    exp = oracle.median(maps)
    np.testing.assert_array_equal(out[:, :W].cpu().numpy().view(np.uint32), exp.view(np.uint32))
    assert bool((out[:, W:] == -1.0).all())           # nothing written past W


def test_median_reports_nonfinite():
    maps = [np.zeros((20, 30), np.float32) for _ in range(3)]
    maps[2][4, 9] = np.nan
    st = torch.zeros((1,), dtype=torch.int32, device="cuda")
    occ.occ_fuse_median([cuda(m) for m in maps], status=st)
    assert int(st.item()) == occ.OCC_ERR_NONFINITE_INPUT
    maps[2][4, 9] = np.inf
    occ.occ_fuse_median([cuda(m) for m in maps], status=st)
    assert int(st.item()) == occ.OCC_ERR_NONFINITE_INPUT
    maps[2][4, 9] = 1.0
    occ.occ_fuse_median([cuda(m) for m in maps], status=st)
    assert int(st.item()) == occ.OCC_OK
    occ.occ_fuse_median([cuda(m) for m in maps])     # no status word


@pytest.mark.parametrize("H,W", [(1, 1), (3, 200), (97, 131), (270, 480)])
def test_warp_matches_oracle(H, W):
    D = scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(44, H))
    views = scenes.views_3x3()
    imgs = scenes.peripheral_images(H, W, len(views), seed=scenes.seed_of(45, W))
    rng = np.random.default_rng(H * 1000 + W)
    M = (rng.random((len(views), H, W)) < 0.2).astype(np.uint8)
    Dg = cuda(D)
    got = occ.occ_warp_views(Dg, views, [cuda(i) for i in imgs], M=cuda(M)).cpu().numpy()
    got_nomask = occ.occ_warp_views(Dg, views, [cuda(i) for i in imgs]).cpu().numpy()
    for v, (a, r) in enumerate(views):
        np.testing.assert_array_equal(got[v].view(np.uint32), oracle.warp_view(D, a, r, imgs[v], M[v]).view(np.uint32))
        np.testing.assert_array_equal(got_nomask[v].view(np.uint32), oracle.warp_view(D, a, r, imgs[v]).view(np.uint32))


def test_warp_views_of_a_5x5_ring_with_pitch():
    H, W = 200, 333
    D = scenes.make_scene(scenes.spec_stress(H, W), scenes.seed_of(46, 0))
    views = scenes.views_5x5_ring()
    imgs = scenes.peripheral_images(H, W, len(views), seed=scenes.seed_of(47, 0))
    bigD = torch.zeros((H, W + 3), device="cuda")
    bigD[:, :W].copy_(cuda(D))
    big_imgs = []
    for im in imgs:
        b = torch.zeros((H, W + 13), device="cuda")
        b[:, 13:].copy_(cuda(im))
        big_imgs.append(b[:, 13:])
    got = occ.occ_warp_views(bigD[:, :W], views, big_imgs).cpu().numpy()
    for v, (a, r) in enumerate(views):
        np.testing.assert_array_equal(got[v].view(np.uint32), oracle.warp_view(D, a, r, imgs[v]).view(np.uint32))


def test_registration_pipeline_fuse_detect_warp():
    """Eight stereo maps -> median (Section 4.2) -> detection (Section 3) -> masked warp (Section 1): every stage on
    the GPU equals the oracle's stage on the oracle's previous output."""
    H, W = 270, 480
    Dtrue = scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(48, 0))
    maps = scenes.stereo_maps(Dtrue, 8, seed=scenes.seed_of(49, 0))
    views = scenes.views_3x3()
    imgs = scenes.peripheral_images(H, W, len(views), seed=scenes.seed_of(50, 0))
    ctx = occ.occ_create(0, max_pixels=H * W, max_views=len(views))
    try:
        Dg = occ.occ_fuse_median([cuda(m) for m in maps])
        M, O = occ.occ_detect(ctx, Dg, views)
        assert occ.occ_get_status(ctx) == occ.OCC_OK
        out = occ.occ_warp_views(Dg, views, [cuda(i) for i in imgs], M=M).cpu().numpy()
    finally:
        ctx.close()
    Do = oracle.median(maps)
    np.testing.assert_array_equal(Dg.cpu().numpy().view(np.uint32), Do.view(np.uint32))
    _, Mo, _ = oracle.detect(Do, views)
    np.testing.assert_array_equal(M.cpu().numpy(), Mo)
    for v, (a, r) in enumerate(views):
        np.testing.assert_array_equal(out[v].view(np.uint32), oracle.warp_view(Do, a, r, imgs[v], Mo[v]).view(np.uint32))


def test_warp_full_size_matches_oracle():
    H, W = 1080, 1920
    D = scenes.array_3x3(frame=0).frames[0]
    views = scenes.views_3x3()
    imgs = scenes.peripheral_images(H, W, len(views), seed=scenes.seed_of(51, 0))
    got = occ.occ_warp_views(cuda(D), views, [cuda(i) for i in imgs]).cpu().numpy()
    for v, (a, r) in enumerate(views):
        np.testing.assert_array_equal(got[v].view(np.uint32), oracle.warp_view(D, a, r, imgs[v]).view(np.uint32))
