"""ctypes declarations of libpgm's C ABI (include/pgm.h).

Loading fails loudly: there is no fallback implementation of any step.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# PGM_CHECKED=1: the build with device index checks (build(checked=True))
LIB_PATH = os.path.join(HERE, "_build", "libpgm_checked.so" if os.environ.get("PGM_CHECKED") == "1"
                        else "libpgm.so")

PARAM_FIELDS = [
    ("levels", 3), ("seed_stride", 3), ("patch_fwd", 15), ("patch_bwd", 11), ("sobel", 5),
    ("color", 1), ("descriptor", 0), ("cs_sched", 0), ("norm", 0), ("iters_coarse", 4),
    ("iters_fine", 6), ("refine_rounds", 2), ("rs_W", 2), ("rs_mode", 0), ("tau2", 1),
    ("min_region", 9), ("region_dmax2", 144), ("max_visits", 0), ("ablation", 0),
    ("rs_grid", 0),
]


class CParams(C.Structure):
    _fields_ = ([(n, C.c_int32) for n, _ in PARAM_FIELDS] + [("philox_key", C.c_uint64)]
                + [("iters_level", C.c_int32 * 12)])


STATUS = {0: "PGM_OK", 1: "PGM_ERR_ARG", 2: "PGM_ERR_SIZE", 3: "PGM_ERR_WORKSPACE",
          4: "PGM_ERR_CUDA", 5: "PGM_ERR_TIMEOUT", 6: "PGM_ERR_DEVICE_BOUNDS",
          7: "PGM_ERR_UNSUPPORTED"}

# every symbol include/pgm.h declares
EXPORTS = [
    "pgm_default_params", "pgm_status_string", "pgm_pyramid_bytes", "pgm_build_pyramid",
    "pgm_pyramid_desc_layout", "pgm_pyramid_image_layout", "pgm_match_workspace_bytes",
    "pgm_match", "pgm_match_batch", "pgm_field_layout", "pgm_filter", "pgm_sync_status",
    "pgm_nominal_evals", "pgm_launch_count", "pgm_profile_enable", "pgm_profile_read",
    "pgm_filter_noalloc", "pgm_build_pyramid_batch", "pgm_filter_batch", "pgm_set_tuning",
    "pgm_get_tuning", "pgm_set_wait_limit", "pgm_error_detail", "pgm_interp_default_params",
    "pgm_interp_workspace_bytes", "pgm_interpolate", "pgm_checked_build",
    "pgm_inject_launch_failure",
]


class CTuning(C.Structure):
    _fields_ = [("window_slack", C.c_int32), ("pairs_per_launch", C.c_int32), ("tile_w", C.c_int32)]


class CInterp(C.Structure):
    _fields_ = [("k", C.c_int32), ("mode", C.c_int32), ("cost_shift", C.c_int32),
                ("la_permyriad", C.c_int32), ("lambda_", C.c_double)]


NOALLOC_MAX_SEEDS = 1 << 20
K_CLASSES = ["pyramid", "init", "cost", "pm", "consist", "transfer", "filter"]
WS_EVALS_OFFSET, WS_EVALS_COUNT = 8, 8   # pm, cost, init, pm-from-global: fwd/bwd each


class PGMError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        msg = "%s failed: %s (%d)" % (where, STATUS.get(code, "?"), code)
        super().__init__(msg + (" [%s]" % detail if detail else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Load libpgm.so (built by paper_1704_03217_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libpgm.so not built (%s); run paper_1704_03217_gb300.build" % path)
    L = C.CDLL(path)
    P = C.POINTER(CParams)
    vp, sz, i32, i64, u64 = C.c_void_p, C.c_size_t, C.c_int, C.c_int64, C.c_uint64
    pi, psz = C.POINTER(C.c_int), C.POINTER(C.c_size_t)
    L.pgm_default_params.argtypes = [P]; L.pgm_default_params.restype = None
    L.pgm_status_string.argtypes = [i32]; L.pgm_status_string.restype = C.c_char_p
    L.pgm_error_detail.argtypes = []; L.pgm_error_detail.restype = C.c_char_p
    L.pgm_pyramid_bytes.argtypes = [P, i32, i32]; L.pgm_pyramid_bytes.restype = sz
    L.pgm_build_pyramid.argtypes = [P, vp, i32, i32, i32, sz, vp, sz, vp]
    L.pgm_pyramid_desc_layout.argtypes = [P, i32, i32, i32, i32, psz, pi, pi, pi, pi, pi, pi]
    L.pgm_pyramid_image_layout.argtypes = [P, i32, i32, i32, i32, psz, pi, pi, pi, pi, psz]
    L.pgm_match_workspace_bytes.argtypes = [P, i32, i32, i32, i32]
    L.pgm_match_workspace_bytes.restype = sz
    L.pgm_match.argtypes = [P, vp, vp, i32, i32, i32, i32, u64, vp, sz, vp]
    L.pgm_match_batch.argtypes = [P, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int32),
                                  C.POINTER(u64), C.POINTER(vp), psz, vp]
    L.pgm_field_layout.argtypes = [P, i32, i32, i32, i32, i32, i32, pi, pi, psz, psz, psz]
    L.pgm_filter.argtypes = [P, i32, i32, i32, i32, vp, sz, vp, i64, vp, vp, vp]
    L.pgm_sync_status.argtypes = [P, i32, i32, i32, i32, vp, sz, vp]
    L.pgm_nominal_evals.argtypes = [P, i32, i32, i32, i32]; L.pgm_nominal_evals.restype = i64
    L.pgm_launch_count.argtypes = []; L.pgm_launch_count.restype = i64
    L.pgm_profile_enable.argtypes = [i32]; L.pgm_profile_enable.restype = C.c_int
    L.pgm_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.pgm_profile_read.restype = C.c_int
    L.pgm_filter_noalloc.argtypes = [P, i32, i32, vp, vp, vp, i64, vp, vp]
    L.pgm_set_tuning.argtypes = [C.POINTER(CTuning)]; L.pgm_set_tuning.restype = C.c_int
    L.pgm_get_tuning.argtypes = [C.POINTER(CTuning)]; L.pgm_get_tuning.restype = C.c_int
    L.pgm_set_wait_limit.argtypes = [C.c_int64]; L.pgm_set_wait_limit.restype = C.c_int
    L.pgm_inject_launch_failure.argtypes = [C.c_int]; L.pgm_inject_launch_failure.restype = C.c_int
    L.pgm_checked_build.argtypes = []; L.pgm_checked_build.restype = C.c_int
    L.pgm_interp_default_params.argtypes = [C.POINTER(CInterp)]; L.pgm_interp_default_params.restype = None
    L.pgm_interp_workspace_bytes.argtypes = [i32, i32, C.POINTER(CInterp)]
    L.pgm_interp_workspace_bytes.restype = C.c_size_t
    L.pgm_interpolate.argtypes = [P, vp, i32, i32, vp, vp, i64, C.POINTER(CInterp), vp, C.c_size_t,
                                  vp, vp]
    L.pgm_interpolate.restype = C.c_int
    L.pgm_build_pyramid_batch.argtypes = [P, i32, C.POINTER(vp), C.POINTER(C.c_int32), psz,
                                          C.POINTER(vp), psz, vp]
    L.pgm_filter_batch.argtypes = [P, i32, C.POINTER(C.c_int32), C.POINTER(vp), psz,
                                   C.POINTER(vp), C.POINTER(C.c_int64), C.POINTER(vp), vp]
    for name in ("pgm_filter_noalloc", "pgm_build_pyramid_batch", "pgm_filter_batch",
                 "pgm_build_pyramid", "pgm_pyramid_desc_layout", "pgm_pyramid_image_layout",
                 "pgm_match", "pgm_match_batch", "pgm_field_layout", "pgm_filter",
                 "pgm_sync_status"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(code, where):
    if code != 0:
        detail = load().pgm_error_detail().decode() if code == 4 else ""
        raise PGMError(code, where, detail)
