"""sbmt_extract_segments_static: boundary extraction for callers that may not
allocate device memory (for example a host application that owns the whole
device budget, or a latency-critical path where an allocation could block or
fail).  Its working memory is a static device array, so this test calls it
twice in a row on different images and compares each result with the
boundary segments of the CPU oracle for the same image."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def _lib():
    sb.build_library()
    lib = sb.load()
    lib.sbmt_extract_segments_static.restype = ctypes.c_int
    lib.sbmt_extract_segments_static.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                                 ctypes.c_void_p]
    lib.sbmt_static_last_error.restype = ctypes.c_char_p
    return lib


def _static_segments(lib, img):
    import torch

    t = torch.from_numpy(img.view(np.int16) if img.dtype == np.uint16 else img).cuda()
    H, W = img.shape
    cap = 2 * (W + 1) * (H + 1)
    out = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    rc = lib.sbmt_extract_segments_static(t.data_ptr(), W, H, t.stride(0) * t.element_size(), img.itemsize,
                                          out.data_ptr(), cap, cnt.data_ptr(), st.cuda_stream)
    assert rc == 0, lib.sbmt_static_last_error()
    st.synchronize()
    n = int(cnt.item())
    r = out[:n].cpu().numpy().view(np.uint32)
    ldr = r[:, 2]
    return np.stack([r[:, 0], r[:, 1], (ldr >> 30) & 1, ldr & 0x3FFFFFFF, r[:, 3] & 0xFFFF, r[:, 3] >> 16, ldr >> 31],
                    axis=1).astype(np.int64)


def _canon(a):
    a = np.asarray(a, dtype=np.int64)
    return a[np.lexsort(a.T[::-1])]


def _oracle_segments(img):
    """The oracle's segments as (x, y, dir, len, label left/below, label
    right/above, reversed), the outside label written as 0xFFFF."""
    seg = oracle.mesh_bitmap(img, 2)["seg"][:, :7].astype(np.int64)
    lab = seg[:, 4:6]
    lab[lab == 0x10000] = 0xFFFF
    return seg


def test_static_extraction_matches_the_oracle_on_consecutive_calls():
    lib = _lib()
    images = [synth.voronoi_labels(size=640, nseeds=90, nlabels=7), synth.disk(),
              synth.noise_batch(n=3, lo=300, hi=900, first=3)[2]]
    for img in images:
        got = _static_segments(lib, img)
        ref = _oracle_segments(img)
        assert len(got) == len(ref)
        assert np.array_equal(_canon(got), _canon(ref))


def test_static_extraction_rejects_a_misaligned_u16_image():
    import torch

    lib = _lib()
    t = torch.zeros((8, 18), dtype=torch.int16, device="cuda")
    out = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    # odd pitch: rejected before any launch
    rc = lib.sbmt_extract_segments_static(t.data_ptr(), 16, 8, 33, 2, out.data_ptr(), 16, cnt.data_ptr(), None)
    assert rc == sb.SBMT_EINVAL
    # odd address: rejected before any launch
    rc = lib.sbmt_extract_segments_static(t.data_ptr() + 1, 16, 8, 36, 2, out.data_ptr(), 16, cnt.data_ptr(), None)
    assert rc == sb.SBMT_EINVAL


def test_static_extraction_rejects_images_above_its_limit():
    import torch

    lib = _lib()
    t = torch.zeros((4097, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.sbmt_extract_segments_static(t.data_ptr(), 16, 4097, 16, 1, out.data_ptr(), 16, cnt.data_ptr(), None)
    assert rc == sb.SBMT_EINVAL
    assert b"4096" in lib.sbmt_static_last_error()
