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


def _meshes(c, imgs, hn):
    return [_fetch(c, m) for m in sb.mesh_batch(c, imgs, hn)]


def test_every_launch_tuning_gives_the_same_meshes():
    """Launch parameters change only launch shapes and stream placement:
    persistent blocks per SM, Tier-G on side streams or not, the emission
    phase replayed as a CUDA graph or not -- the meshes stay identical."""
    c = ctx()
    imgs = synth.noise_batch(n=12, lo=60, hi=700, first=12)
    hn = [2, 4, 8] * 4
    ref = _meshes(c, imgs, hn)
    for cut, tg, fork, graph in ((4, 8, 0, 0), (16, 32, 1, 1), (8, 24, 0, 1), (12, 16, 1, 1)):
        sb.mesh_set_tuning(c, imgs, hn, cut_blocks_per_sm=cut, tierg_blocks_per_sm=tg, fork=fork, graph=graph)
        assert sb.mesh_tuning(c, imgs, hn) == {"cut_blocks_per_sm": cut, "tierg_blocks_per_sm": tg, "fork": fork,
                                              "graph": graph}
        for _ in range(2):  # a graph is updated in place on the second run
            got = _meshes(c, imgs, hn)
            for a, b in zip(ref, got):
                for key in ("tri", "label", "code", "xy"):
                    assert np.array_equal(a[key], b[key]), (cut, tg, fork, graph, key)


def test_autotune_writes_its_choice(tmp_path, monkeypatch):
    monkeypatch.setenv("SBMT_TUNE_FILE", str(tmp_path / "tune.txt"))
    c = sb.mesh_create(0)
    try:
        imgs = synth.noise_batch(n=6, lo=100, hi=400, first=6)
        before = _meshes(c, imgs, 2)
        sb.mesh_autotune(c, imgs, 2, repeats=1)
        t = sb.mesh_tuning(c, imgs, 2)
        lines = (tmp_path / "tune.txt").read_text().split("\n")
        key, vals = lines[0].split()[0], [int(v) for v in lines[0].split()[1:]]
        assert vals == [t["cut_blocks_per_sm"], t["tierg_blocks_per_sm"], t["fork"], t["graph"]]
        assert key.startswith("n2_")  # 6 images: log2 bucket 2
        after = _meshes(c, imgs, 2)
        for a, b in zip(before, after):
            for k in ("tri", "label", "code", "xy"):
                assert np.array_equal(a[k], b[k])
    finally:
        sb.mesh_destroy(c)
    # a new context reads the file
    c2 = sb.mesh_create(0)
    try:
        assert sb.mesh_tuning(c2, imgs, 2) == t
    finally:
        sb.mesh_destroy(c2)


def test_a_device_wait_that_runs_out_is_reported_and_the_context_survives():
    """Every device wait of the path is bounded: here one tile of the
    counting scan withholds its sums (a flag nothing sets), the next tile's
    wait runs out after about a second, and the call returns SBMT_ETIMEDOUT
    with no fault; the same context then meshes normally."""
    c = ctx()
    rng = np.random.default_rng(5)
    img = (rng.random((220, 240)) < 0.5).astype(np.uint8)  # thousands of segments
    with pytest.raises(sb.SbmtError) as e:
        sb.mesh_bitmap(c, img, 2, flags=sb.SBMT_DEBUG_STALL_SCAN)
    assert e.value.code == sb.SBMT_ETIMEDOUT
    with pytest.raises(sb.SbmtError) as e:
        sb.mesh_batch(c, [img, img[:50, :60]], 2, flags=sb.SBMT_DEBUG_STALL_SCAN)
    assert e.value.code == sb.SBMT_ETIMEDOUT
    g = _fetch(c, sb.mesh_bitmap(c, img, 2))
    assert_same_mesh(g, oracle.mesh_bitmap(img, 2, 1), 2.0, W=img.shape[1])
