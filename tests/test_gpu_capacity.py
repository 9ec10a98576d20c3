"""A cell whose local boundary graph has more vertices than the Tier-G rule's
per-cell limit (64) cannot be triangulated; the mesh then reports
SBMT_ECAPACITY, and mesh_stage 4 lists exactly those cells: the Tier-G cells
of the oracle whose local vertex count (triangles + 2 - inside vertices) is
above the limit."""
import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu

LIMIT = 64


@pytest.mark.parametrize("hn,nexp", [(24, 3), (32, 51)])
def test_cells_over_the_limit_are_listed(hn, nexp):
    img = synth.noise_bitmap(synth.rng_for(21), 200, 150, 2.0)
    o = oracle.mesh_bitmap(img, hn, 1)
    cut = o["cut"]
    n_local = cut[:, 2] + 2 - cut[:, 3]
    expected = np.sort(cut[(cut[:, 4] == 1) & (n_local > LIMIT), 0])
    assert len(expected) == nexp
    c = ctx()
    m = sb.mesh_bitmap(c, img, hn, 1)
    with pytest.raises(sb.SbmtError) as e:  # the mesh's status comes back as the error
        sb.mesh_query(c, m, -1)
    assert e.value.code == sb.SBMT_ECAPACITY
    got = sb.mesh_stage(c, m, 4)[:, 0]
    assert np.array_equal(got, expected)
    sb.mesh_release(c, m)


def test_no_cells_over_the_limit_at_h2():
    c = ctx()
    m = sb.mesh_bitmap(c, synth.disk(), 2, 1)
    v = sb.mesh_query(c, m, -1)
    assert v.status == sb.SBMT_OK
    assert len(sb.mesh_stage(c, m, 4)) == 0
    sb.mesh_release(c, m)
