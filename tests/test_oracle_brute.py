"""Brute force over tiny inputs: every binary 4 x 4 bitmap (2^16 of them) at
h = 2/3 (the paper's regime, Lemma 3.1), 2 and 4, meshed by the oracle and
checked against the invariants any correct output has -- counter-clockwise
triangles, closure and consistent orientation, Euler characteristic of a
disk, total area of the base cells (every cell tiled), per-label area equal
to the pixel count, and boundary conformity (label changes only across mesh
edges on pixel lines, adding up to the bitmap's boundary length).  The
bitmaps are split over host processes."""
import multiprocessing as mp

import pytest

import oracle


def _slice(args):
    hn, hd, first, stride = args
    return oracle.brute(4, 4, hn, hd, first, stride)


@pytest.mark.parametrize("hn,hd", [(2, 3), (2, 1), (4, 1)])
def test_every_4x4_binary_bitmap(hn, hd):
    oracle.build()
    k = 8
    with mp.get_context("spawn").Pool(k) as pool:
        done = pool.map(_slice, [(hn, hd, f, k) for f in range(k)])
    assert sum(done) == 1 << 16


def test_planted_mistakes_fail_the_checks():
    import numpy as np

    img = np.array([[0, 1, 1, 0], [1, 1, 0, 0], [0, 1, 0, 1], [1, 0, 0, 1]], np.uint8)
    m = oracle.mesh_bitmap(img, 2, 1)
    assert oracle.check_mesh(img, 2, 1, m) == 0

    def broken(fn):
        c = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
        fn(c)
        return oracle.check_mesh(img, 2, 1, c)

    assert broken(lambda c: c["tri"].__setitem__(0, c["tri"][0][[0, 2, 1]])) != 0  # one triangle clockwise
    cut = int(np.nonzero(m["code"])[0][0])
    lab = m["label"][cut]
    assert broken(lambda c: c["label"].__setitem__(cut, 1 - lab if lab < 2 else 0)) != 0  # a wrong label
    assert broken(lambda c: c.__setitem__("tri", c["tri"][1:])) != 0  # a triangle missing
    assert broken(lambda c: c["xy"].__setitem__((c["tri"][cut][0], 0), c["xy"][c["tri"][cut][0]][0] + 0.01)) != 0
    assert broken(lambda c: c.__setitem__("n_cells", c["n_cells"] + 1)) != 0  # the cell count off by one
    assert oracle.brute(3, 3, 2, 1) == 512
