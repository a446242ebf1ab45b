"""Runs each kernel that sits beside the detection a few times on bench-sized inputs, for profiling (ncu -k ...):
the median fusion of 8 stereo maps and the masked backward warp of 8 views on the 1920x1080 3x3-array frame, then the
learned tile proposer's forward pass on 8 frames of 256x192 and two training steps.

    python -m paper_2408_14050_gb300.probe
"""
from __future__ import annotations


def main():
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_2408_14050_gb300 as occ
    import scenes

    views = scenes.views_3x3()
    f = scenes.array_3x3(frame=0).frames[0]
    H, W = f.shape
    maps = [torch.from_numpy(m).cuda() for m in scenes.stereo_maps(f, 8, seed=3)]
    imgs = [torch.from_numpy(i).cuda() for i in scenes.peripheral_images(H, W, 8, seed=4)]
    D = torch.empty((H, W), device="cuda")
    with occ.occ_create(0, max_pixels=H * W, max_views=8) as ctx:
        M, _ = occ.occ_detect(ctx, torch.from_numpy(f).cuda(), views)
    out = torch.empty((8, H, W), device="cuda")
    for _ in range(3):
        occ.occ_fuse_median(maps, D=D)
    for _ in range(3):
        occ.occ_warp_views(D, views, imgs, M=M, out=out)
    Dn = torch.from_numpy(scenes.proposer_frames(8, 192, 256, seed=5)).cuda()
    net = occ.Net(0, max_pixels=8 * 192 * 256, max_views=8)
    net.set_params(scenes.net_init(1))
    for _ in range(3):
        net.forward(Dn, views)
    labels = torch.ones((8, 8, 6, 8), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        net.loss_grad(Dn, views, labels)
    torch.cuda.synchronize()
    if occ.occ_net_status() != occ.OCC_OK:
        raise RuntimeError("a tensor-core wait of the network expired")
    net.close()
    print("probe ok")


if __name__ == "__main__":
    main()
