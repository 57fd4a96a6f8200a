"""The random-search stability experiment (Sec. III-C secret (3), Fig. 4) on
the GPU at full size: different Philox keys give different fields with the
same statistics, and the seeds that move between keys are mostly outliers.
The key reaches the kernels exactly as it reaches the oracle."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api, evaluate, synth
    return api, evaluate, synth


def test_keys_change_fields_not_statistics(mods):
    api, E, synth = mods
    pairs = [synth.sintel_like_pair(300 + s) for s in range(4)]
    r = E.stability(api.Params(levels=5, color=1), pairs)
    t = r["total"]
    assert t["unstable"] > 0 and t["stable_share"] >= 0.8
    epes = [k["epe"] for k in t["per_key"]]
    rates = [k["outliers_3px"] for k in t["per_key"]]
    assert max(rates) - min(rates) <= 0.01
    assert max(epes) - min(epes) <= 0.1 * min(epes)   # outliers dominate the mean
    assert t["outliers_3px_unstable"] > 0.5
    assert t["outliers_3px_unstable"] >= 5 * t["outliers_3px_stable"]


def test_key_parity_with_the_oracle(mods):
    """A non-default key: every level and direction equals the oracle's."""
    api, E, synth = mods
    from pgm_compare import assert_parity
    f1, f2, _ = synth.sintel_like_pair(9, 320, 240, t_max=30.0)
    for key in E.KEYS[1:]:
        assert_parity(api, dict(levels=4, color=1, philox_key=key), f1, f2, stream_id=5,
                      what="key %x" % key)
