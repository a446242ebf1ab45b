"""occ_detect_batched_tiles: per-tile proposals (the candidates of unproposed tiles are not scanned) and per-tile hit
flags (the plain method's labels for the learned tile proposer), bit for bit against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = occ.occ_create(0, max_pixels=8 * 1024 * 1024, max_views=24)
    yield c
    c.close()


def frames(seed=0, sizes=((96, 128), (100, 77), (33, 65), (192, 256))):
    out = []
    for i, (H, W) in enumerate(sizes):
        spec = scenes.SceneSpec(H=H, W=W, bg_base=(2.0, 6.0), bg_slope=(2.0, 8.0), n_objects=4, obj_disp=(8.0, 24.0),
                                obj_size=(0.1, 0.5), d_max=64.0, sigma=0.25 if i % 2 else 0.0)
        out.append(scenes.make_scene(spec, scenes.seed_of(70 + seed, i)))
    return out


def tables(fs, V, fill):
    return [torch.full((V, *occ.tiles_of(*f.shape)), fill, dtype=torch.uint8, device="cuda") for f in fs]


def test_all_tiles_proposed_equals_plain_and_hits_match_oracle_labels(ctx):
    fs = frames()
    views = scenes.views_3x3()
    V = len(views)
    Ds = [torch.from_numpy(f).cuda() for f in fs]
    M0, O0 = occ.occ_detect_batched(ctx, Ds, views)
    hits = tables(fs, V, 7)
    M1, O1 = occ.occ_detect_batched(ctx, Ds, views, proposals=tables(fs, V, 1), hits=hits)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    for f, a, b, c, d, h in zip(fs, M0, M1, O0, O1, hits):
        assert torch.equal(a, b) and torch.equal(c, d)
        for v, (al, r) in enumerate(views):
            np.testing.assert_array_equal(h[v].cpu().numpy(), oracle.tile_labels(f, al, r))


def test_hits_without_proposals(ctx):
    fs = frames(seed=1)[:2]
    views = scenes.views_3x3()[:3]
    Ds = [torch.from_numpy(f).cuda() for f in fs]
    hits = tables(fs, len(views), 9)
    M, O = occ.occ_detect_batched(ctx, Ds, views, hits=hits)
    for f, h in zip(fs, hits):
        for v, (al, r) in enumerate(views):
            np.testing.assert_array_equal(h[v].cpu().numpy(), oracle.tile_labels(f, al, r))


@pytest.mark.parametrize("density", [0.0, 0.3, 0.7])
def test_random_proposals_match_the_oracle_on_the_proposed_tiles(ctx, density):
    fs = frames(seed=2)
    views = scenes.views_3x3()
    V = len(views)
    rng = np.random.default_rng(int(density * 10))
    props_np = [(rng.random((V, *occ.tiles_of(*f.shape))) < density).astype(np.uint8) for f in fs]
    props = [torch.from_numpy(p).cuda() for p in props_np]
    hits = tables(fs, V, 5)
    Ds = [torch.from_numpy(f).cuda() for f in fs]
    Ms, Os = occ.occ_detect_batched(ctx, Ds, views, proposals=props, hits=hits)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    for f, p, M, O, h in zip(fs, props_np, Ms, Os, hits):
        for v, (al, r) in enumerate(views):
            Oo, Mo = oracle.detect_view_proposed(f, al, r, None, p[v])
            np.testing.assert_array_equal(O[v].cpu().numpy(), Oo)
            np.testing.assert_array_equal(M[v].cpu().numpy(), Mo)
            # A skipped tile reports no hit; a proposed one reports its label.
            exp = oracle.tile_labels(f, al, r) * (p[v] != 0)
            np.testing.assert_array_equal(h[v].cpu().numpy(), exp)


def test_long_lines_take_the_warp_kernels_and_still_flag_hits(ctx):
    """A 5x5-ring view set with long scan lines and N = 16 (the warp kernels only)."""
    H, W = 120, 200
    f = scenes.make_scene(scenes.spec_stress(H, W), scenes.seed_of(72, 0))
    views = scenes.views_5x5_ring()[:6]
    V = len(views)
    p = occ.occ_default_params()
    p.N = 16
    rng = np.random.default_rng(3)
    prop_np = (rng.random((V, *occ.tiles_of(H, W))) < 0.5).astype(np.uint8)
    hits = tables([f], V, 3)
    Ms, Os = occ.occ_detect_batched(ctx, [torch.from_numpy(f).cuda()], views, p,
                                    proposals=[torch.from_numpy(prop_np).cuda()], hits=hits)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    po = oracle.default_params(N=16)
    for v, (al, r) in enumerate(views):
        Oo, Mo = oracle.detect_view_proposed(f, al, r, po, prop_np[v])
        np.testing.assert_array_equal(Os[0][v].cpu().numpy(), Oo)
        np.testing.assert_array_equal(hits[0][v].cpu().numpy(), oracle.tile_labels(f, al, r, po) * prop_np[v])


def test_tile_table_shape_is_checked(ctx):
    D = torch.zeros((40, 40), device="cuda")
    with pytest.raises(ValueError):
        occ.occ_detect_batched(ctx, [D], [(0.0, 1.0)], proposals=[torch.ones((1, 1, 1), dtype=torch.uint8,
                                                                           device="cuda")])
