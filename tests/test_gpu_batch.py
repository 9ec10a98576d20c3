"""mesh_batch: images meshed concurrently on several streams must give, mesh
for mesh, exactly what one mesh_bitmap call per image gives, and an invalid
image in a batch must fail the whole batch without leaving meshes behind."""
import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import assert_same_mesh, ctx
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def _fetch(c, m):
    out = sb.view_numpy(sb.mesh_query(c, m, -1))  # host copies
    sb.mesh_release(c, m)
    return out


def test_batch_equals_single_calls():
    c = ctx()
    imgs = synth.noise_batch(n=14, lo=40, hi=420, first=14)
    hs = [(2, 1), (4, 1), (8, 1), (2, 3)] * 4
    hn = [a for a, _ in hs[: len(imgs)]]
    hd = [b for _, b in hs[: len(imgs)]]
    ids = sb.mesh_batch(c, imgs, hn, hd)
    batched = [_fetch(c, m) for m in ids]
    for k, img in enumerate(imgs):
        single = _fetch(c, sb.mesh_bitmap(c, img, hn[k], hd[k]))
        for key in ("tri", "label", "code", "xy"):
            assert np.array_equal(batched[k][key], single[key]), (k, key)
    # and the batch against the oracle on two of them
    for k in (0, 5):
        o = oracle.mesh_bitmap(imgs[k], hn[k], hd[k])
        assert_same_mesh(batched[k], o, hn[k] / hd[k], W=imgs[k].shape[1])


def test_batch_with_one_shared_h_and_repeat():
    c = ctx()
    imgs = synth.noise_batch(n=9, lo=30, hi=200, first=9)
    a = [_fetch(c, m) for m in sb.mesh_batch(c, imgs, 4)]
    b = [_fetch(c, m) for m in sb.mesh_batch(c, imgs, 4)]
    for x, y in zip(a, b):
        for key in ("tri", "label", "code", "xy"):
            assert np.array_equal(x[key], y[key])


def test_batch_error_fails_whole_batch():
    c = ctx()
    imgs = synth.noise_batch(n=8, lo=30, hi=120, first=8)
    hn = [2] * 8
    hn[5] = 3  # odd h_num: outside the accepted class
    with pytest.raises(sb.SbmtError):
        sb.mesh_batch(c, imgs, hn, 1)
    # the context stays usable
    ids = sb.mesh_batch(c, imgs[:3], 2)
    assert len(ids) == 3
    for m in ids:
        sb.mesh_release(c, m)


def test_noise512_batch_sampled_images_match_oracle():
    """The 512-bitmap batch (sides 131..2038 px, h = 2) through one
    mesh_batch call from device-resident images, as the bench runs it; 16
    meshes spread over the size range, the largest included, against the
    oracle in full."""
    import torch

    c = ctx()
    specs = synth.noise_batch_specs()
    imgs = [synth.noise_batch_item(sp) for sp in specs]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    ids = sb.mesh_batch(c, dev, 2)
    order = sorted(range(len(imgs)), key=lambda i: imgs[i].size)
    pick = sorted(set([order[(k * (len(order) - 1)) // 15] for k in range(16)]))
    assert order[-1] in pick and len(pick) == 16
    views = {}
    for k, m in enumerate(ids):
        if k in pick:
            views[k] = _fetch(c, m)
        else:
            sb.mesh_release(c, m)
    for k in pick:
        o = oracle.mesh_bitmap(imgs[k], 2, 1)
        assert_same_mesh(views[k], o, 2.0, W=imgs[k].shape[1])
