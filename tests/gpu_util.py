"""Helpers for the GPU tests: run the CUDA path through the C interface and
compare its output with the CPU oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2602_19474_gb300 as sb

_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        sb.build_library()
        _CTX = sb.mesh_create(0)
    return _CTX


def gpu_mesh(img, h_num, h_den=1, stages=False, on_device=False):
    c = ctx()
    src = img
    if on_device:
        import torch

        src = torch.from_numpy(img.astype(np.int16) if img.dtype == np.uint16 else img).cuda()
    m = sb.mesh_bitmap(c, src, h_num, h_den, keep_stages=stages)
    v = sb.mesh_query(c, m, -1)
    out = sb.view_numpy(v)
    if stages:
        out["seg"] = sb.mesh_stage(c, m, 1)
        out["ev"] = sb.mesh_stage(c, m, 2)
        out["cut"] = sb.mesh_stage(c, m, 3)
    sb.mesh_release(c, m)
    return out


def assert_same_mesh(g, o, h, W=None, stages=False):
    """Bit-exact connectivity, labels and codes in the canonical order;
    coordinates within 1e-6 h."""
    assert g["n_cells"] == o["n_cells"]
    assert g["n_cut_cells"] == o["n_cut_cells"]
    assert g["n_tierG_cells"] == o["n_tierG_cells"]
    assert g["tri"].shape == o["tri"].shape, (g["tri"].shape, o["tri"].shape)
    assert g["xy"].shape == o["xy"].shape
    bad = np.nonzero((g["tri"] != o["tri"]).any(axis=1))[0]
    assert len(bad) == 0, "first differing triangle %d: gpu %s oracle %s" % (bad[0], g["tri"][bad[0]], o["tri"][bad[0]])
    assert np.array_equal(g["label"], o["label"])
    assert np.array_equal(g["code"], o["code"])
    err = np.abs(g["xy"] - o["xy"]).max() if len(o["xy"]) else 0.0
    assert err <= 1e-6 * h, err
    if stages:
        # segments: same set (the device emits them in any order)
        og = o["seg"].copy()
        og[:, 4:6][og[:, 4:6] == 0x10000] = 0xFFFF
        a = np.unique(og[:, :7], axis=0)
        b = np.unique(g["seg"][:, :7], axis=0)
        assert np.array_equal(a, b)
        # events: same vertex ids on the same grid edges, crossed by the same segment
        oseg = o["seg"][o["ev"][:, 1]].astype(np.int64)
        corner = oseg[:, 1] * (W + 1) + oseg[:, 0]
        exp = np.stack([o["ev"][:, 0], o["ev"][:, 2], corner, oseg[:, 2]], axis=1)
        assert np.array_equal(exp, g["ev"])
        # cut cells: id, code, triangles, inside vertices, outside-regime flag
        assert np.array_equal(g["cut"], o["cut"])
