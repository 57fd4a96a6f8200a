"""Sparse-to-dense interpolation (Sec. III-G) on the GPU against the CPU
oracle: the k-nearest geodesic lists bit-exact, the interpolated flow equal
up to the last bits of exp (double precision, stored as float), at full size
and on the edge cases."""
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
    from paper_1704_03217_gb300 import api
    return api


def gpu_interp(api, prm, img1, rows, ip, count=None):
    P1 = api.build_pyramid(prm, torch.from_numpy(np.ascontiguousarray(img1)).cuda())
    r = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, 4)).cuda()
    if r.shape[0] == 0:
        r = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    n = len(rows) if count is None else count
    c = torch.tensor([n], dtype=torch.int32, device="cuda")
    flow, ws = api.interpolate(prm, P1, r, c, ip)
    torch.cuda.synchronize()
    keys = api.interp_keys(ws, P1.w, P1.h, ip.k).cpu().numpy().view(np.uint64)
    return flow.cpu().numpy(), keys


def oracle_interp(prm_d, img1, rows, ip):
    desc = O.Pyramid(O.make_params(prm_d), img1).desc(0, 0)
    return O.interpolate(desc, rows, K=ip.k, lam=ip.lam, shift=ip.cost_shift, mode=ip.mode,
                         la_permyriad=ip.la_permyriad)


def compare(flow, keys, okeys, oflow, what):
    bad = np.argwhere(keys != okeys)
    assert bad.size == 0, "%s: neighbour lists differ at %s" % (what, bad[:5])
    of = oflow.astype(np.float32)
    assert np.abs(flow - of).max() <= 1e-3, what
    assert (flow == of).mean() >= 0.999, what


def test_full_size_parity_and_accuracy(api):
    from paper_1704_03217_gb300 import synth
    f1, f2, gt = synth.sintel_like_pair(21)
    prm_d = dict(levels=5, color=1)
    _, _, _, rows = O.run_pair(prm_d, f1, f2)
    ip = api.InterpParams()
    flow, keys = gpu_interp(api, api.Params(**prm_d), f1, rows, ip)
    okeys, oflow, la = oracle_interp(prm_d, f1, rows, ip)
    assert la                                  # grid-3 matches are far above 2.2 %
    compare(flow, keys, okeys, oflow, "full size")
    epe = np.hypot(*(flow - gt).transpose(2, 0, 1))
    assert np.median(epe) < 1.0


@pytest.mark.parametrize("mode,k", [(1, 8), (2, 8), (0, 1), (2, 16)])
def test_modes_and_k(api, mode, k):
    from paper_1704_03217_gb300 import synth
    f1, f2, _ = synth.sintel_like_pair(22, 320, 240, t_max=40.0)
    prm_d = dict(levels=4, color=1)
    _, _, _, rows = O.run_pair(prm_d, f1, f2)
    ip = api.InterpParams(k=k, mode=mode, lam=12.0, cost_shift=9)
    flow, keys = gpu_interp(api, api.Params(**prm_d), f1, rows, ip)
    okeys, oflow, _ = oracle_interp(prm_d, f1, rows, ip)
    compare(flow, keys, okeys, oflow, "mode %d k %d" % (mode, k))


def test_edge_cases(api):
    """No match, one match, sparse matches (NW by the paper's rule), two
    matches at one pixel, positions outside the image, and a count above
    the buffer's rows."""
    from paper_1704_03217_gb300 import synth
    f1, _, _ = synth.sintel_like_pair(23, 200, 120, t_max=20.0)
    prm_d = dict(levels=3, color=1)
    prm = api.Params(**prm_d)
    ip = api.InterpParams(k=4)
    flow, keys = gpu_interp(api, prm, f1, np.zeros((0, 4), np.int32), ip)
    assert (flow == 0).all() and (keys == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    one = np.array([[50, 60, 57, 58]], np.int32)
    flow, keys = gpu_interp(api, prm, f1, one, ip)
    assert np.allclose(flow, [7, -2], atol=1e-6)
    rng = np.random.default_rng(3)
    sparse = np.stack([rng.integers(0, 200, 40), rng.integers(0, 120, 40),
                       rng.integers(0, 200, 40), rng.integers(0, 120, 40)], 1).astype(np.int32)
    sparse[5, :2] = sparse[2, :2]               # a shared pixel: index 2 stays
    sparse[7, :2] = (-3, 10)                    # outside
    sparse[9, :2] = (150, 120)                  # outside
    flow, keys = gpu_interp(api, prm, f1, sparse, ip)
    okeys, oflow, la = oracle_interp(prm_d, f1, sparse, ip)
    assert not la
    compare(flow, keys, okeys, oflow, "sparse")
    flow2, keys2 = gpu_interp(api, prm, f1, sparse, ip, count=10 ** 6)   # count capped by the rows
    assert (keys2 == keys).all() and (flow2 == flow).all()
