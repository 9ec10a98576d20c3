"""Brute force over tiny inputs on the device: every binary 4 x 4 bitmap
(2^16 of them) at h = 2/3, 2 and 4, meshed in batches of 8192 through
mesh_batch, each mesh equal to the oracle's -- vertex ids, labels and codes
bit-exact, coordinates within 1e-6 h."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import ctx

pytestmark = pytest.mark.gpu

N = 1 << 16
CHUNK = 8192


def _bitmap(b):
    return np.array([(b >> k) & 1 for k in range(16)], np.uint8).reshape(4, 4)


def _oracle_chunk(args):
    hn, hd, lo, hi = args
    out = []
    for b in range(lo, hi):
        o = oracle.mesh_bitmap(_bitmap(b), hn, hd)
        out.append((o["tri"], o["label"], o["code"], o["xy"]))
    return out


def _gpu_chunk(c, hn, hd, lo, hi):
    import torch

    imgs = [_bitmap(b) for b in range(lo, hi)]
    ids = sb.mesh_batch(c, imgs, hn, hd)
    views = [sb.mesh_query(c, m, -1) for m in ids]
    ts = [sb.view_tensors(v) for v in views]
    cat = {k: torch.cat([t[k].reshape(-1) for t in ts]).cpu().numpy() for k in ("tri", "label", "code", "xy")}
    nt = np.array([v.n_triangles for v in views])
    nv = np.array([v.n_vertices for v in views])
    for m in ids:
        sb.mesh_release(c, m)
    return cat, nt, nv


@pytest.mark.parametrize("hn,hd", [(2, 3), (2, 1), (4, 1)])
def test_every_4x4_binary_bitmap_matches_the_oracle(hn, hd):
    oracle.build()
    c = ctx()
    with mp.get_context("spawn").Pool(16) as pool:
        for lo in range(0, N, CHUNK):
            hi = lo + CHUNK
            step = CHUNK // 16
            parts = pool.map(_oracle_chunk, [(hn, hd, a, a + step) for a in range(lo, hi, step)])
            ref = [m for p in parts for m in p]
            cat, nt, nv = _gpu_chunk(c, hn, hd, lo, hi)
            to = np.concatenate([[0], np.cumsum(nt)])
            vo = np.concatenate([[0], np.cumsum(nv)])
            tri = cat["tri"].reshape(-1, 3)
            lab = cat["label"].view(np.uint16)
            code = cat["code"].view(np.uint16)
            xy = cat["xy"].reshape(-1, 2)
            for k, (otri, olab, ocode, oxy) in enumerate(ref):
                b = lo + k
                assert nt[k] == len(otri) and nv[k] == len(oxy), b
                assert np.array_equal(tri[to[k]:to[k + 1]], otri), b
                assert np.array_equal(lab[to[k]:to[k + 1]], olab), b
                assert np.array_equal(code[to[k]:to[k + 1]], ocode), b
                assert np.abs(xy[vo[k]:vo[k + 1]] - oxy).max() <= 1e-6 * hn / hd, b
