"""include/pgm.h from a plain C99 program: the header compiles as strict C
(-std=c99 -pedantic, warnings as errors), the program links against
libpgm.so, and what a C compiler makes of the header's structs and constants
is what the Python binding declares (field offsets and sizes of pgm_params,
pgm_tuning and pgm_interp_params; the workspace and no-allocation constants;
the status codes).  The program makes host-side calls only (defaults, size
queries, argument checks), so it runs without a GPU."""
import ctypes as C
import subprocess

import pytest


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    from c_build import compile_c
    exe = str(tmp_path_factory.mktemp("cabi") / "probe")
    ok, log = compile_c("c_abi_probe.c", exe)
    if ok is None:
        pytest.skip(log)
    assert ok, log
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {}
    for line in r.stdout.splitlines():
        key, _, val = line.partition(" ")
        out[key] = val
    return out


def _layout(struct, out, cname):
    assert int(out["sizeof_" + cname]) == C.sizeof(struct), cname
    for name, _ in struct._fields_:
        cfield = "lambda" if name == "lambda_" else name
        assert int(out["off_%s_%s" % (cname, cfield)]) == getattr(struct, name).offset, name


def test_struct_layouts_match_the_binding(probe):
    from paper_1704_03217_gb300 import _lib
    _layout(_lib.CParams, probe, "pgm_params")
    _layout(_lib.CTuning, probe, "pgm_tuning")
    _layout(_lib.CInterp, probe, "pgm_interp_params")


def test_constants_and_status_codes_match_the_binding(probe):
    from paper_1704_03217_gb300 import _lib
    assert int(probe["const_PGM_NOALLOC_MAX_SEEDS"]) == _lib.NOALLOC_MAX_SEEDS
    assert int(probe["const_PGM_WS_EVALS_OFFSET"]) == _lib.WS_EVALS_OFFSET
    assert int(probe["const_PGM_WS_EVALS_COUNT"]) == _lib.WS_EVALS_COUNT
    assert int(probe["const_PGM_K_COUNT"]) == len(_lib.K_CLASSES)
    assert int(probe["const_PGM_ERR_UNSUPPORTED"]) == 7 and _lib.STATUS[7] == "PGM_ERR_UNSUPPORTED"
    L = _lib.load()
    for code in range(8):
        assert probe["status_%d" % code] == L.pgm_status_string(code).decode()


def test_calls_from_c_agree_with_the_binding(probe):
    from paper_1704_03217_gb300 import _lib
    from paper_1704_03217_gb300.api import Params
    L = _lib.load()
    d = Params()
    assert int(probe["default_levels"]) == d.levels
    assert (int(probe["default_patch_fwd"]), int(probe["default_patch_bwd"])) == (15, 11)
    assert int(probe["default_rs_W"]) == d.rs_W and int(probe["default_iters_level_11"]) == -1
    assert int(probe["default_philox_key"]) == d.philox_key
    cp = d.replace(levels=5).cstruct()
    assert int(probe["pyramid_bytes_1024x436"]) == L.pgm_pyramid_bytes(C.byref(cp), 1024, 436)
    assert int(probe["workspace_bytes_1024x436"]) == \
        L.pgm_match_workspace_bytes(C.byref(cp), 1024, 436, 1024, 436)
    assert int(probe["nominal_evals_1024x436"]) == \
        L.pgm_nominal_evals(C.byref(cp), 1024, 436, 1024, 436)
    assert int(probe["match_null"]) == 1              # PGM_ERR_ARG
    assert int(probe["match_patch17"]) == 7           # PGM_ERR_UNSUPPORTED
    ip = _lib.CInterp()
    L.pgm_interp_default_params(C.byref(ip))
    assert (int(probe["interp_k"]), int(probe["interp_la_permyriad"])) == (ip.k, ip.la_permyriad)
    assert float(probe["interp_lambda"]) == pytest.approx(ip.lambda_)
    assert int(probe["interp_ws_bytes_64x48"]) == L.pgm_interp_workspace_bytes(64, 48, C.byref(ip))
    assert int(probe["get_tuning"]) == 0 and int(probe["tuning_tile_w"]) == 8
    assert int(probe["set_tuning_bad"]) == 1          # tile_w 5 is rejected
    assert int(probe["checked_build"]) == 0


def test_whole_path_program_builds(tmp_path):
    """tests/c_match_pair.c, the whole path from C with cudaMalloc'ed buffers
    (run on a GPU by tests/test_c_pipeline_gpu.py), compiles as strict C99
    and links against libpgm.so and the CUDA runtime."""
    from c_build import compile_c
    ok, log = compile_c("c_match_pair.c", str(tmp_path / "c_match_pair"), cudart=True)
    if ok is None:
        pytest.skip(log)
    assert ok, log
    r = subprocess.run([str(tmp_path / "c_match_pair")], capture_output=True, text=True)
    assert r.returncode == 2 and "usage" in r.stderr      # no arguments: usage, no CUDA call
