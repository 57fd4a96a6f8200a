"""The exhaustive initialisation on the tensor cores (six-channel descriptor,
squared L2): the coarsest level's fields right after their initialisation
(one visit, no iterations) equal the oracle's brute-force nearest neighbour
(Sec. III-D; exact costs, ties to the smaller target raster index) at every
seed.  The shapes give several seed tiles and centre bands with ragged ends,
odd and even patches, seed strides 1 to 4 (one to sixteen phase images), and
flat images where every cost ties."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1704_03217_gb300 import synth
from pgm_compare import compare_fields, run_both


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api as A
    return A


def _init_only(prm):
    L = prm["levels"]
    return dict(prm, max_visits=1, iters_level=tuple([-1] * (L - 1) + [0]))


@pytest.mark.parametrize("name,prm,size", [
    ("sintel-L5", dict(levels=5, color=1), (1024, 436)),
    ("kitti-L5", dict(levels=5, color=1), (1242, 375)),
    ("stride1", dict(levels=3, color=1, seed_stride=1, patch_fwd=7, patch_bwd=5), (160, 96)),
    ("stride2-even", dict(levels=3, color=1, seed_stride=2, patch_fwd=15, patch_bwd=6), (257, 131)),
    ("stride4", dict(levels=3, color=1, seed_stride=4, patch_fwd=9, patch_bwd=9), (300, 200)),
    ("patch1", dict(levels=2, color=1, patch_fwd=1, patch_bwd=3), (90, 70)),
    ("plain-rgb", dict(levels=3, color=1, cs_sched=1, sobel=3), (211, 99)),
    ("sector", dict(levels=4, color=1, descriptor=2), (384, 164)),
    ("tiny", dict(levels=2, color=1, patch_fwd=5, patch_bwd=5), (24, 17)),
])
def test_init_equals_brute_force(api, name, prm, size):
    f1, f2, _ = synth.sintel_like_pair(7, *size, t_max=min(150.0, size[0] / 6))
    p = _init_only(prm)
    (_, _, ws, _, _), (_, _, M, _, _) = run_both(api, p, f1, f2, stream_id=2)
    compare_fields(ws, M, prm["levels"], name)
    top = ws.field(prm["levels"] - 1, 0)
    assert top["valid"].all().item(), name                   # every seed initialised


def test_init_ties_on_flat_images(api):
    """Constant colour images: every cost is zero, so every seed takes the
    target centre of raster index 0."""
    f1 = np.full((120, 200, 3), 90, np.uint8)
    f2 = np.full((120, 200, 3), 30, np.uint8)
    p = _init_only(dict(levels=3, color=1))
    (_, _, ws, _, _), (_, _, M, _, _) = run_both(api, p, f1, f2)
    compare_fields(ws, M, 3, "flat")
    top = ws.field(2, 0)
    assert (top["cost"].view(torch.int64) == 0).all().item()
