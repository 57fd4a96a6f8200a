"""End-to-end sanity of the GPU path against synthetic ground truth, and the
ablation switches of Table 1 (no refinement of the initial field, propagate
inliers and outliers, no outlier-record propagation)."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import evaluate
    return evaluate


def test_exact_translation_every_variant(ev):
    """A shift by a multiple of 2^(L-1) is recovered exactly by every variant
    away from the borders."""
    from paper_1704_03217_gb300 import api, synth
    f1, f2, fl = synth.translate_pair(3, 320, 240, 16, -8, channels=3)
    for bits in (0, 1, 2, 4):
        for color, desc in ((1, 0), (1, 1), (0, 0), (0, 1)):
            p = api.Params(levels=4, color=color, descriptor=desc, ablation=bits)
            r = ev.run(p, [(f1, f2, fl)])
            assert r["matches"] > 0.5 * 106 * 79
            assert r["epe"] < 0.25 and r["outliers_3px"] < 0.02


def test_sintel_like_accuracy_and_ablations(ev):
    """On Sintel-shaped pairs the complete method exports dense, accurate
    matches; each ablation switch changes the result."""
    from paper_1704_03217_gb300 import api, synth
    pairs = [synth.sintel_like_pair(200 + s, 512, 218, t_max=60.0) for s in range(3)]
    base = api.Params(levels=4, color=1)
    tab = ev.ablation_table(pairs, base)
    full = tab["complete"]
    assert full["density"] > 0.5
    assert full["epe"] < 2.5 and full["outliers_3px"] < 0.06
    for name, r in tab.items():
        if name != "complete":
            assert r["matches"] != full["matches"] or r["epe"] != full["epe"], name
