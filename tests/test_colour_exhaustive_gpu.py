"""Every 24-bit colour through the CUDA colour conversion.  A 4096 x 4096
RGB image holds each colour once; with one pyramid level and the Table 2
schedule the backward scheme converts level 0 to CIELab, and the converted
planes must equal the oracle's integer CIELab (reading R3: no companding,
exact integer cube root) for all 2^24 colours."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03217_gb300 import build
    build.build()
    from paper_1704_03217_gb300 import api as A
    return A


def test_lab_every_colour(api):
    r, g, b = np.meshgrid(np.arange(256), np.arange(256), np.arange(256), indexing="ij")
    rgb = np.stack([r, g, b], -1).reshape(4096, 4096, 3).astype(np.uint8)
    P = api.build_pyramid(api.Params(levels=1, color=1), torch.from_numpy(rgb).cuda())
    torch.cuda.synchronize()
    got = P.cimage(1, 0).cpu().numpy()                      # (3, 4096, 4096)
    want = O.convert(O.SP_LAB, rgb.reshape(-1, 3)).reshape(4096, 4096, 3).transpose(2, 0, 1)
    bad = np.argwhere(got != want)
    assert bad.size == 0, (len(bad), bad[:5].tolist())
