"""The whole hot path from a plain C program (tests/c_match_pair.c): device
memory from cudaMalloc, the legacy default stream, no Python or PyTorch in the
process, and pyramid buffers and a match workspace filled with 0xff before
use.  Its exported matches equal the CPU oracle's (checkerboard schedule,
same stream id) and the Python binding's, and pgm_sync_status reports no
failure although every buffer started as garbage.  Cases: PGM-C at full size,
and at an odd size gray with the direction descriptor (its bit-planes) and
PGM-C."""
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("w,h,levels,color,descriptor",
                         [(1024, 436, 5, 1, 0), (203, 117, 3, 0, 1), (203, 117, 3, 1, 0)])
def test_c_program_matches_oracle_and_binding(tmp_path, w, h, levels, color, descriptor):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from c_build import compile_c
    from paper_1704_03217_gb300 import api, synth
    exe = str(tmp_path / "c_match_pair")
    ok, log = compile_c("c_match_pair.c", exe, cudart=True)
    if ok is None:
        pytest.skip(log)
    assert ok, log
    f1, f2, _ = synth.sintel_like_pair(41 + levels, w, h, t_max=min(150.0, w / 6))
    p1, p2, out = (str(tmp_path / n) for n in ("a.rgb", "b.rgb", "rows.bin"))
    np.ascontiguousarray(f1).tofile(p1)
    np.ascontiguousarray(f2).tofile(p2)
    r = subprocess.run([exe, str(w), str(h), str(levels), str(color), str(descriptor), p1, p2,
                        out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(out, dtype=np.int32)
    n = int(raw[0])
    rows = raw[1:].reshape(-1, 4)
    assert rows.shape[0] == n and n > 0

    prm = dict(levels=levels, color=color, descriptor=descriptor)  # the defaults otherwise
    _, _, _, orows = O.run_pair(prm, f1, f2, O.SCHED_CHECKERBOARD, 7)
    assert orows.shape == rows.shape and (orows == rows).all()

    p = api.Params(**prm)
    P1 = api.build_pyramid(p, torch.from_numpy(f1).cuda())
    P2 = api.build_pyramid(p, torch.from_numpy(f2).cuda())
    ws = api.match(p, P1, P2, stream_id=7)
    got, _ = api.filter_matches(p, ws)
    assert (got.cpu().numpy() == rows).all()
