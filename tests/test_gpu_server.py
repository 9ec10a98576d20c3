"""Serving (include/sbmt.h server_*): requests of different sizes admitted by
device memory and meshed in batches while others are on the GPU.  A
request's mesh is the same alone and in a mix (every cell's patch is
independent of the others, Sec. 3.5's corollary) and equal to the oracle's;
reservations never exceed the budget; faults are injected on the host only
(an admission check that sees no free memory, cancelled requests, malformed
requests)."""
import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import assert_same_mesh
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def _host(v):
    return sb.view_numpy(v)


def _mix(n, lo=64, hi=700, seed=0):
    rng = np.random.default_rng(seed)
    imgs = synth.noise_batch(n=n, lo=lo, hi=hi, first=n)
    hs = [int(rng.choice([2, 4, 8])) for _ in range(n)]
    return imgs, hs


def test_a_request_alone_equals_the_same_request_in_a_mix():
    import torch

    srv = sb.server_create(0)
    try:
        target = synth.ellipses(size=600, n=30, amin=8, amax=80)
        rid = sb.server_submit(srv, target, 4)
        v, info = sb.server_wait(srv, rid, -1)
        alone = _host(v)
        assert info["batch_size"] == 1
        sb.server_release(srv, rid)
        # the same image among 40 others, as a device-resident bitmap
        imgs, hs = _mix(40)
        dev = [torch.from_numpy(im).cuda() for im in imgs]
        tdev = torch.from_numpy(target).cuda()
        ids = []
        for k, (im, h) in enumerate(zip(dev, hs)):
            ids.append(sb.server_submit(srv, im, h))
            if k == 20:
                tid = sb.server_submit(srv, tdev, 4)
        sizes = []
        for rid_ in ids:
            _, inf = sb.server_wait(srv, rid_, -1)
            sizes.append(inf["batch_size"])
        v, info = sb.server_wait(srv, tid, -1)
        mixed = _host(v)
        for key in ("tri", "label", "code", "xy"):
            assert np.array_equal(alone[key], mixed[key]), key
        assert_same_mesh(mixed, oracle.mesh_bitmap(target, 4, 1), 4.0, W=target.shape[1])
        assert max(sizes + [info["batch_size"]]) > 1  # requests did share batches
        # every request of the mix equals the oracle on a sample
        for k in (0, 13, 39):
            v, _ = sb.server_wait(srv, ids[k], -1)
            assert_same_mesh(_host(v), oracle.mesh_bitmap(imgs[k], hs[k], 1), float(hs[k]), W=imgs[k].shape[1])
        for rid_ in ids + [tid]:
            sb.server_release(srv, rid_)
        st = sb.server_stats(srv)
        assert st["completed"] == 42 and st["failed"] == 0 and st["reserved_bytes"] == 0
    finally:
        sb.server_destroy(srv)


def test_admission_never_exceeds_the_budget_and_every_request_completes():
    imgs, hs = _mix(24, lo=200, hi=900, seed=1)
    # a budget of about three of the largest requests' bounds: most requests wait
    budget = 3 * max(_bound_bytes(im, h) for im, h in zip(imgs, hs))
    srv = sb.server_create(0, hbm_budget=budget, max_batch=8)
    try:
        ids = [sb.server_submit(srv, im, h) for im, h in zip(imgs, hs)]
        views = []
        for rid in ids:
            v, info = sb.server_wait(srv, rid, -1)
            views.append(_host(v))
        st = sb.server_stats(srv)
        assert st["peak_reserved_bytes"] <= budget == st["budget_bytes"]
        assert st["completed"] == len(imgs) and st["batches"] > 3
        for k in (2, 11):
            assert_same_mesh(views[k], oracle.mesh_bitmap(imgs[k], hs[k], 1), float(hs[k]), W=imgs[k].shape[1])
        for rid in ids:
            sb.server_release(srv, rid)
        assert sb.server_stats(srv)["reserved_bytes"] == 0
    finally:
        sb.server_destroy(srv)


def _bound_bytes(img, h):
    return sb.mesh_bound(img, h)


def test_injected_out_of_memory_delays_requests_without_changing_them():
    imgs, hs = _mix(12, seed=2)
    srv = sb.server_create(0, oom_every=2, max_batch=4)
    try:
        ids = [sb.server_submit(srv, im, h) for im, h in zip(imgs, hs)]
        for k, rid in enumerate(ids):
            v, _ = sb.server_wait(srv, rid, -1)
            if k in (0, 7):
                assert_same_mesh(_host(v), oracle.mesh_bitmap(imgs[k], hs[k], 1), float(hs[k]), W=imgs[k].shape[1])
            sb.server_release(srv, rid)
        assert sb.server_stats(srv)["completed"] == 12
    finally:
        sb.server_destroy(srv)


def test_over_budget_cancelled_and_malformed_requests():
    img = synth.noise_batch(n=1, lo=300, hi=301, first=1)[0]
    srv = sb.server_create(0, hbm_budget=1 << 20)  # below any request's bound
    try:
        rid = sb.server_submit(srv, img, 2)
        with pytest.raises(sb.SbmtError) as e:
            sb.server_wait(srv, rid, -1)
        assert e.value.code == sb.SBMT_ENOMEM
        sb.server_release(srv, rid)
        with pytest.raises(sb.SbmtError) as e:
            sb.server_submit(srv, img, 3)  # odd h_num: refused at submission
        assert e.value.code == sb.SBMT_EINVAL
        assert sb.server_stats(srv)["submitted"] == 1
    finally:
        sb.server_destroy(srv)
    # cancel: with room for one request at a time, later ones are still queued
    imgs, hs = _mix(8, lo=400, hi=600, seed=3)
    budget = int(1.5 * max(_bound_bytes(im, 2) for im in imgs))
    srv = sb.server_create(0, hbm_budget=budget, workers=1)
    try:
        ids = [sb.server_submit(srv, im, 2) for im in imgs]
        sb.server_cancel(srv, ids[-1])
        with pytest.raises(sb.SbmtError) as e:
            sb.server_wait(srv, ids[-1], -1)
        assert e.value.code == sb.SBMT_ECANCELED
        for k, rid in enumerate(ids[:-1]):
            v, _ = sb.server_wait(srv, rid, -1)
            if k == 3:
                assert_same_mesh(_host(v), oracle.mesh_bitmap(imgs[k], 2, 1), 2.0, W=imgs[k].shape[1])
            sb.server_release(srv, rid)
        sb.server_release(srv, ids[-1])
        st = sb.server_stats(srv)
        assert st["cancelled"] == 1 and st["completed"] == 7 and st["reserved_bytes"] == 0
    finally:
        sb.server_destroy(srv)
