"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gs_status|void|const char\s*\*|gs_\w+_opts)\s*(gs_\w+)\s*\(", text,
                                 flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gs_create_scene", "gs_destroy_scene", "gs_render", "gs_render_pose_grad", "gs_render_batch",
                     "gs_render_pose_grad_batch", "gs_refine_pose", "gs_refine_poses_batch", "gs_refine_defaults",
                     "gs_last_error", "gs_pmm_create", "gs_pmm_match", "gs_pmm_destroy", "gs_visibility",
                     "gs_pnp_create", "gs_pnp_solve", "gs_pnp_destroy", "gs_pnp_defaults"):
        assert required in names


def test_library_exports_every_declared_symbol(libgsr_path):
    lib = ctypes.CDLL(libgsr_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.gs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.gs_version()


def test_invalid_arguments_fail_without_a_gpu(libgsr_path):
    lib = ctypes.CDLL(libgsr_path)
    lib.gs_create_scene.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.gs_last_error.restype = ctypes.c_char_p
    assert lib.gs_create_scene(None, None) == 1  # GS_ERR_INVALID_ARG
    assert b"required" in lib.gs_last_error()
    lib.gs_render.argtypes = [ctypes.c_void_p] * 5
    assert lib.gs_render(None, None, None, None, None) == 1
    lib.gs_visibility.argtypes = [ctypes.c_void_p] * 10
    assert lib.gs_visibility(*([None] * 10)) == 1


def test_pmm_create_rejects_bad_sizes_without_a_gpu(libgsr_path):
    lib = ctypes.CDLL(libgsr_path)
    lib.gs_pmm_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.gs_pmm_create(31, 64, 64, ctypes.byref(h)) == 1  # 32 channels only
    assert lib.gs_pmm_create(32, 60, 64, ctypes.byref(h)) == 1  # multiples of 8
    assert not h.value


def test_pnp_create_rejects_bad_sizes_without_a_gpu(libgsr_path):
    lib = ctypes.CDLL(libgsr_path)
    lib.gs_pnp_create.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.gs_pnp_create(0, 16, ctypes.byref(h)) == 1
    assert lib.gs_pnp_create(100, 0, ctypes.byref(h)) == 1
    assert not h.value
    lib.gs_pnp_solve.argtypes = [ctypes.c_void_p] * 12
    assert lib.gs_pnp_solve(*([None] * 12)) == 1
