"""The SBMT_COMPACT format: uncut cells implicit (a label and a zero code per
base cell), the cut cells' patches listed.  Expanded cell by cell it must
give the explicit mesh of the same image exactly -- the same patch
triangles in the same order, labels, codes and the non-lattice vertices'
coordinates to the bit."""
import numpy as np
import pytest

import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def _fetch(c, m):
    out = sb.view_numpy(sb.mesh_query(c, m, -1))
    sb.mesh_release(c, m)
    return out


def check_compact_expands_to_explicit(e, k):
    assert k["format"] == sb.SBMT_COMPACT and e["format"] == sb.SBMT_EXPLICIT
    for key in ("n_cells", "n_cut_cells", "n_tierG_cells", "n_lattice_vertices", "n_tierG_triangles"):
        assert k[key] == e[key], key
    assert k["n_triangles"] == len(e["tri"]) and k["n_vertices"] == len(e["xy"])
    C, K, NVg = e["n_cells"], e["n_cut_cells"], e["n_lattice_vertices"]
    cell_code, cell_label = k["cell_code"], k["cell_label"]
    patch_cell, patch_off = k["patch_cell"].astype(np.int64), k["patch_off"].astype(np.int64)
    assert len(cell_code) == C and len(patch_cell) == K and len(patch_off) == K + 1
    # the cut cells: increasing ids, exactly those with a nonzero code
    assert (np.diff(patch_cell) > 0).all()
    cut = cell_code != 0
    assert cut.sum() == K and np.array_equal(np.nonzero(cut)[0], patch_cell)
    assert (cell_label[cut] == 0xFFFF).all()
    assert patch_off[0] == 0 and patch_off[-1] == k["n_patch_triangles"] == len(k["tri"])
    per = np.diff(patch_off)
    assert (per >= 2).all()
    # per-cell triangle counts give the explicit mesh's cell ranges
    cnt = np.ones(C, np.int64)
    cnt[patch_cell] = per
    start = np.concatenate([[0], np.cumsum(cnt)])
    assert start[-1] == len(e["tri"]) == (C - K) + k["n_patch_triangles"]
    base = start[:-1][~cut]
    assert (e["code"][base] == 0).all()
    assert np.array_equal(e["label"][base], cell_label[~cut])
    rows = np.concatenate([np.arange(start[c], start[c + 1]) for c in patch_cell]) if K else np.zeros(0, np.int64)
    assert np.array_equal(e["tri"][rows], k["tri"])
    assert np.array_equal(e["label"][rows], k["label"])
    assert np.array_equal(e["code"][rows], k["code"])
    assert np.array_equal(e["code"][start[patch_cell]], cell_code[cut])
    # vertices after the lattice, to the bit
    assert np.array_equal(e["xy"][NVg:].view(np.uint64), k["xy"].view(np.uint64))
    # every patch corner that is a lattice vertex is one of the explicit mesh's
    assert (k["tri"] < k["n_vertices"]).all() and (k["tri"] >= 0).all()


@pytest.mark.parametrize("name,img,hn,hd", [
    ("disk", synth.disk(), 2, 1),
    ("noise_tierg", synth.noise_batch(n=2, lo=300, hi=500, first=2)[1], 8, 1),
    ("voronoi", synth.voronoi_labels(size=700, nseeds=80), 4, 1),
    ("star_third", synth.star(), 2, 3),
])
def test_compact_expands_to_explicit(name, img, hn, hd):
    c = ctx()
    e = _fetch(c, sb.mesh_bitmap(c, img, hn, hd))
    k = _fetch(c, sb.mesh_bitmap(c, img, hn, hd, format=sb.SBMT_COMPACT))
    if name == "noise_tierg":
        assert e["n_tierG_cells"] > 0  # the greedy path writes into the patch list too
    check_compact_expands_to_explicit(e, k)


def test_compact_uniform_image_has_no_patches():
    c = ctx()
    img = np.full((97, 131), 7, np.uint8)
    k = _fetch(c, sb.mesh_bitmap(c, img, 4, 1, format=sb.SBMT_COMPACT))
    e = _fetch(c, sb.mesh_bitmap(c, img, 4, 1))
    # only the image border cuts cells
    check_compact_expands_to_explicit(e, k)
    inside = k["cell_label"][k["cell_code"] == 0]
    assert set(np.unique(inside)) <= {7, 0xFFFF}


def test_compact_batch_and_quality_rejected():
    c = ctx()
    imgs = synth.noise_batch(n=6, lo=40, hi=260, first=6)
    ks = [_fetch(c, m) for m in sb.mesh_batch(c, imgs, 4, format=sb.SBMT_COMPACT)]
    es = [_fetch(c, m) for m in sb.mesh_batch(c, imgs, 4)]
    for e, k in zip(es, ks):
        check_compact_expands_to_explicit(e, k)
    m = sb.mesh_bitmap(c, imgs[0], 4, 1, format=sb.SBMT_COMPACT)
    with pytest.raises(sb.SbmtError):
        sb.mesh_quality(c, m)
    sb.mesh_release(c, m)
