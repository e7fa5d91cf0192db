"""Thin ctypes binding of libgsr (include/gsr.h).

Functions with the C names (``gs_create_scene``, ``gs_render``, ...) pass
arguments straight through; the helpers below them (``Scene``, ``PoseLoss``)
only marshal torch tensors (device memory, current stream) into those calls.
Every step of rendering and differentiation runs in the CUDA library. Importing
this module loads ``libgsr.so`` and raises ImportError if it has not been built
(``python -m paper_2507_15683_gb300.build``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsr.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_INTERNAL = range(7)
GS_BATCH_GRAPH = 1
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_OOM", 4: "GS_ERR_CAPACITY",
                5: "GS_ERR_TIMEOUT", 6: "GS_ERR_INTERNAL"}


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class gs_scene_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int), ("feat_dim", ctypes.c_int),
                ("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("feats_bf16", ctypes.c_void_p),
                ("n_partitions", ctypes.c_int), ("partition_offsets", ctypes.c_void_p),
                ("device_resident", ctypes.c_int)]


class gs_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class gs_pose(ctypes.Structure):
    _fields_ = [("T_cw", ctypes.c_double * 16)]


class gs_refine_opts(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("lr_rot", ctypes.c_double), ("lr_trans", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("depth_weight", ctypes.c_float)]


class gs_outputs(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("final_T", ctypes.c_void_p), ("feats", ctypes.c_void_p), ("last_idx", ctypes.c_void_p)]


class gs_pmm_result(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("codes_q", ctypes.c_void_p), ("codes_r", ctypes.c_void_p),
                ("lse_row", ctypes.c_void_p), ("lse_col", ctypes.c_void_p), ("row_best", ctypes.c_void_p),
                ("col_best", ctypes.c_void_p), ("n_coarse", ctypes.c_int64), ("coarse", ctypes.c_void_p),
                ("coarse_prob", ctypes.c_void_p), ("n_fine", ctypes.c_int64), ("fine", ctypes.c_void_p),
                ("fine_prob", ctypes.c_void_p)]


class gs_launch(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("grid_mult", ctypes.c_int),
                ("batch", ctypes.c_int), ("min_blocks", ctypes.c_int), ("occupancy", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class gs_tune_result(ctypes.Structure):
    _fields_ = [("best", gs_launch), ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double),
                ("candidates", ctypes.c_int)]


GS_MODE_FORWARD, GS_MODE_FEATURES, GS_MODE_POSE_GRAD = 0, 1, 2
GS_COMPOSITE_VARIANTS = 4


class gs_pnp_opts(ctypes.Structure):
    _fields_ = [("tau_px", ctypes.c_float), ("min_alpha", ctypes.c_float), ("refine_iters", ctypes.c_int)]


class gs_pnp_result(ctypes.Structure):
    _fields_ = [("T_cw", ctypes.c_double * 16), ("n_valid", ctypes.c_int64), ("n_inliers", ctypes.c_int64),
                ("best_hypothesis", ctypes.c_int32), ("best_solution", ctypes.c_int32),
                ("best_count", ctypes.c_int64), ("refine_steps", ctypes.c_int32), ("inlier", ctypes.c_void_p),
                ("valid_index", ctypes.c_void_p), ("points", ctypes.c_void_p), ("hyp_counts", ctypes.c_void_p),
                ("hyp_poses", ctypes.c_void_p)]


GS_LOCALIZE_MAX_ROUNDS = 8


class gs_localize_opts(ctypes.Structure):
    _fields_ = [("n_rounds", ctypes.c_int), ("pmm_tau", ctypes.c_float), ("max_angle_deg", ctypes.c_double),
                ("n_hypotheses", ctypes.c_int), ("pnp", gs_pnp_opts)]


class gs_localize_result(ctypes.Structure):
    _fields_ = [("T_cw", ctypes.c_double * 16), ("reliable", ctypes.c_int), ("n_rounds", ctypes.c_int),
                ("round_T", (ctypes.c_double * 16) * GS_LOCALIZE_MAX_ROUNDS),
                ("angle_deg", ctypes.c_double * GS_LOCALIZE_MAX_ROUNDS),
                ("trans", ctypes.c_double * GS_LOCALIZE_MAX_ROUNDS),
                ("n_matches", ctypes.c_int64 * GS_LOCALIZE_MAX_ROUNDS),
                ("n_inliers", ctypes.c_int64 * GS_LOCALIZE_MAX_ROUNDS)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgsr.so is not built (run: python -m paper_2507_15683_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    sigs = {
        "gs_create_scene": [P(gs_scene_desc), P(vp)],
        "gs_scene_reserve": [vp, i64, i64],
        "gs_render": [vp, P(gs_camera), P(gs_pose), P(gs_outputs), vp],
        "gs_render_async": [vp, P(gs_camera), P(gs_pose), P(gs_outputs), vp],
        "gs_render_pose_grad": [vp, P(gs_camera), P(gs_pose), vp, vp, vp, ctypes.c_float, P(gs_outputs), vp, vp, vp],
        "gs_render_pose_grad_async": [vp, P(gs_camera), P(gs_pose), vp, vp, vp, ctypes.c_float, P(gs_outputs), vp,
                                      vp],
        "gs_render_pose_grad_host": [vp, P(gs_camera), P(gs_pose), vp, vp, vp, ctypes.c_float, P(gs_outputs), vp,
                                     vp, vp],
        "gs_render_batch": [vp, ctypes.c_int, P(gs_camera), P(gs_pose), P(gs_outputs), ctypes.c_uint, vp],
        "gs_render_pose_grad_batch": [vp, ctypes.c_int, P(gs_camera), P(gs_pose), vp, vp, vp, ctypes.c_float,
                                      vp, vp, vp, vp, ctypes.c_uint, vp],
        "gs_scene_status": [vp, vp, vp, vp],
        "gs_get_tile_lists": [vp, ctypes.c_int, vp, vp, vp, i64, vp, vp],
        "gs_get_records": [vp, ctypes.c_int, vp, i64, vp, vp],
        "gs_render_noalloc": [P(gs_scene_desc), P(gs_camera), P(gs_pose), P(gs_outputs), vp],
        "gs_scene_set_timing": [vp, ctypes.c_int],
        "gs_scene_stream_stats": [vp, vp, vp, vp],
        "gs_scene_evict": [vp],
        "gs_scene_kernel_times": [vp, vp, vp],
        "gs_scene_blend_count": [vp, vp, vp],
        "gs_scene_work_counts": [vp, vp, vp, vp],
        "gs_visibility": [vp, P(gs_camera), P(gs_pose), vp, vp, vp, vp, vp, vp, vp],
        "gs_pmm_create": [st, st, st, P(vp)],
        "gs_pmm_match": [vp, vp, vp, ctypes.c_float, P(gs_pmm_result), vp],
        "gs_pnp_create": [i64, st, P(vp)],
        "gs_pose_difference": [P(gs_pose), P(gs_pose), P(ctypes.c_double), P(ctypes.c_double)],
        "gs_pnp_set_timing": [vp, st],
        "gs_pnp_phase_times": [vp, vp, vp],
        "gs_dense_localize": [vp, vp, vp, P(gs_camera), P(gs_pose), vp, vp, P(gs_localize_opts),
                              P(gs_localize_result), vp],
        "gs_scene_shape": [vp, vp, vp, vp],
        "gs_pmm_shape": [vp, vp, vp, vp],
        "gs_pmm_set_wait_limit": [vp, st],
        "gs_scene_set_launch": [vp, st, st, P(gs_camera), P(gs_launch)],
        "gs_scene_get_launch": [vp, st, st, P(gs_camera), P(gs_launch)],
        "gs_autotune": [vp, st, st, P(gs_camera), P(gs_pose), st, P(gs_tune_result), vp],
        "gs_tune_save": [vp, ctypes.c_char_p],
        "gs_tune_load": [vp, ctypes.c_char_p, P(ctypes.c_int)],
        "gs_pnp_solve": [vp, P(gs_camera), P(gs_pose), vp, vp, vp, i64, vp, st, P(gs_pnp_opts), P(gs_pnp_result), vp],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = st
    L.gs_refine_pose.argtypes = [vp, P(gs_camera), P(gs_pose), vp, vp, vp, P(gs_refine_opts), vp, vp]
    L.gs_refine_pose.restype = st
    L.gs_refine_poses_batch.argtypes = [vp, ctypes.c_int, P(gs_camera), P(gs_pose), vp, vp, vp,
                                        P(gs_refine_opts), vp, vp]
    L.gs_refine_poses_batch.restype = st
    L.gs_refine_defaults.argtypes = []
    L.gs_refine_defaults.restype = gs_refine_opts
    L.gs_destroy_scene.argtypes = [vp]
    L.gs_destroy_scene.restype = None
    L.gs_pmm_destroy.argtypes = [vp]
    L.gs_pmm_destroy.restype = None
    L.gs_pnp_destroy.argtypes = [vp]
    L.gs_pnp_destroy.restype = None
    L.gs_pnp_defaults.argtypes = []
    L.gs_pnp_defaults.restype = gs_pnp_opts
    L.gs_localize_defaults.argtypes = []
    L.gs_localize_defaults.restype = gs_localize_opts
    L.gs_last_error.argtypes = []
    L.gs_last_error.restype = ctypes.c_char_p
    L.gs_version.argtypes = []
    L.gs_version.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(status: int):
    if status != GS_OK:
        raise GsError(status, lib.gs_last_error().decode())


# ---- C entry points under their own names -------------------------------------------------------
def gs_create_scene(desc: gs_scene_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib.gs_create_scene(ctypes.byref(desc), ctypes.byref(h)))
    return h


def gs_destroy_scene(h) -> None:
    lib.gs_destroy_scene(h)


def gs_scene_reserve(h, max_records: int, max_pairs: int) -> None:
    _check(lib.gs_scene_reserve(h, int(max_records), int(max_pairs)))


def gs_render(h, cam: gs_camera, pose: gs_pose, out: gs_outputs, stream: int) -> None:
    _check(lib.gs_render(h, ctypes.byref(cam), ctypes.byref(pose), ctypes.byref(out), stream))


def gs_render_async(h, cam: gs_camera, pose: gs_pose, out: gs_outputs, stream: int) -> None:
    _check(lib.gs_render_async(h, ctypes.byref(cam), ctypes.byref(pose), ctypes.byref(out), stream))


def gs_render_pose_grad(h, cam, pose, target_rgb: int, target_depth: int, pixel_weight, depth_weight: float,
                        out, stream: int):
    loss = ctypes.c_double()
    grad = (ctypes.c_double * 6)()
    _check(lib.gs_render_pose_grad(h, ctypes.byref(cam), ctypes.byref(pose), target_rgb, target_depth,
                                   pixel_weight, float(depth_weight), ctypes.byref(out) if out is not None else None,
                                   ctypes.byref(loss), grad, stream))
    return loss.value, np.array(grad[:], np.float64)


def gs_render_pose_grad_host(h, cam, pose, target_rgb: int, target_depth: int, pixel_weight, depth_weight: float,
                             out, stream: int):
    """As gs_render_pose_grad with the targets as host addresses (pinned for overlap)."""
    loss = ctypes.c_double()
    grad = (ctypes.c_double * 6)()
    _check(lib.gs_render_pose_grad_host(h, ctypes.byref(cam), ctypes.byref(pose), target_rgb, target_depth,
                                        pixel_weight, float(depth_weight),
                                        ctypes.byref(out) if out is not None else None, ctypes.byref(loss), grad,
                                        stream))
    return loss.value, np.array(grad[:], np.float64)


def gs_render_pose_grad_async(h, cam, pose, target_rgb, target_depth, pixel_weight, depth_weight, out,
                              result_dev: int, stream: int) -> None:
    _check(lib.gs_render_pose_grad_async(h, ctypes.byref(cam), ctypes.byref(pose), target_rgb, target_depth,
                                         pixel_weight, float(depth_weight),
                                         ctypes.byref(out) if out is not None else None, result_dev, stream))


def gs_render_batch(h, cams, poses, outs, flags: int, stream: int) -> None:
    n = len(cams)
    ca = (gs_camera * n)(*cams)
    pa = (gs_pose * n)(*poses)
    oa = (gs_outputs * n)(*outs)
    _check(lib.gs_render_batch(h, n, ca, pa, oa, int(flags), stream))


def gs_render_pose_grad_batch(h, cams, poses, target_rgb, target_depth, pixel_weight, depth_weight, outs,
                              results_dev: int, flags: int, stream: int):
    """target_rgb / target_depth / pixel_weight: sequences of device pointers
    (pixel_weight may be None). Returns (loss[n], grad[n, 6]) in synchronous
    mode, None in graph mode (results in results_dev)."""
    n = len(cams)
    ca = (gs_camera * n)(*cams)
    pa = (gs_pose * n)(*poses)
    tr = (ctypes.c_void_p * n)(*[int(p) for p in target_rgb])
    td = (ctypes.c_void_p * n)(*[int(p) for p in target_depth])
    pw = None if pixel_weight is None else (ctypes.c_void_p * n)(*[int(p) if p else None for p in pixel_weight])
    oa = None if outs is None else (gs_outputs * n)(*outs)
    loss = np.zeros(n, np.float64)
    grad = np.zeros((n, 6), np.float64)
    graph = bool(flags & GS_BATCH_GRAPH)
    _check(lib.gs_render_pose_grad_batch(h, n, ca, pa, tr, td, pw, float(depth_weight), oa,
                                         None if graph else loss.ctypes.data, None if graph else grad.ctypes.data,
                                         results_dev or None, int(flags), stream))
    return None if graph else (loss, grad)


def gs_refine_defaults() -> gs_refine_opts:
    return lib.gs_refine_defaults()


def gs_refine_pose(h, cam, pose_, target_rgb: int, target_depth: int, pixel_weight, opts, stream: int):
    """Refines pose_ (gs_pose) in place; returns the loss history."""
    hist = np.zeros(max(opts.iterations, 1), np.float64)
    _check(lib.gs_refine_pose(h, ctypes.byref(cam), ctypes.byref(pose_), target_rgb, target_depth,
                              pixel_weight or None, ctypes.byref(opts), hist.ctypes.data, stream))
    return hist[:opts.iterations]


def gs_refine_poses_batch(h, cams, poses, target_rgb, target_depth, pixel_weight, opts, stream: int):
    """Refines the gs_pose list in place; returns the loss history (n, iterations)."""
    n = len(cams)
    ca = (gs_camera * n)(*cams)
    pa = (gs_pose * n)(*poses)
    tr = (ctypes.c_void_p * n)(*[int(p) for p in target_rgb])
    td = (ctypes.c_void_p * n)(*[int(p) for p in target_depth])
    pw = None if pixel_weight is None else (ctypes.c_void_p * n)(*[int(p) if p else None for p in pixel_weight])
    hist = np.zeros((n, max(opts.iterations, 1)), np.float64)
    _check(lib.gs_refine_poses_batch(h, n, ca, pa, tr, td, pw, ctypes.byref(opts), hist.ctypes.data, stream))
    for k in range(n):
        poses[k] = pa[k]
    return hist[:, :opts.iterations]


def pose_matrix(p: gs_pose) -> np.ndarray:
    return np.array(p.T_cw[:], np.float64).reshape(4, 4)


def gs_scene_status(h, stream: int):
    nr, npr = ctypes.c_int64(), ctypes.c_int64()
    s = lib.gs_scene_status(h, stream, ctypes.byref(nr), ctypes.byref(npr))
    return s, nr.value, npr.value


def gs_get_tile_lists(h, view: int, tiles: int, capacity: int, stream: int):
    keys = np.zeros(max(capacity, 1), np.uint64)
    gids = np.zeros(max(capacity, 1), np.uint32)
    ts = np.zeros(tiles + 1, np.int64)
    n = ctypes.c_int64()
    _check(lib.gs_get_tile_lists(h, view, keys.ctypes.data, gids.ctypes.data, ts.ctypes.data, capacity,
                                 ctypes.byref(n), stream))
    return ts, keys[:n.value], gids[:n.value]


def gs_get_records(h, view: int, capacity: int, stream: int) -> np.ndarray:
    rec = np.zeros((max(capacity, 1), 10), np.int32)
    n = ctypes.c_int64()
    _check(lib.gs_get_records(h, view, rec.ctypes.data, capacity, ctypes.byref(n), stream))
    return rec[:n.value]


GS_NOALLOC_MAX_GAUSSIANS = 32768
GS_NOALLOC_MAX_TILES = 16384
GS_NOALLOC_MAX_PAIRS = 524288


def gs_render_noalloc(desc: gs_scene_desc, cam: gs_camera, pose: gs_pose, out: gs_outputs, stream: int) -> None:
    """Forward render using only the library's fixed device scratch array (no
    allocation); desc holds device pointers. See include/gsr.h for the limits."""
    _check(lib.gs_render_noalloc(ctypes.byref(desc), ctypes.byref(cam), ctypes.byref(pose), ctypes.byref(out),
                                 stream))


KERNEL_NAMES = ("project", "shade", "scan_tiles", "scatter", "sort", "composite", "vis_backward", "vis_select")


def gs_scene_set_timing(h, enable: bool) -> None:
    _check(lib.gs_scene_set_timing(h, int(bool(enable))))


def gs_scene_kernel_times(h):
    ms = np.zeros(len(KERNEL_NAMES), np.float64)
    n = np.zeros(len(KERNEL_NAMES), np.int64)
    _check(lib.gs_scene_kernel_times(h, ms.ctypes.data, n.ctypes.data))
    return ms, n


def gs_scene_blend_count(h, stream=None):
    """(pixel, Gaussian) pairs blended by the last pose-gradient call."""
    b = ctypes.c_int64()
    _check(lib.gs_scene_blend_count(h, _stream() if stream is None else stream, ctypes.byref(b)))
    return b.value


def gs_visibility(h, cam: gs_camera, pose_: gs_pose, mask: int, uv, grad_mean, visible_ids, visible_uv,
                  stream: int) -> int:
    """Algorithm 1 visibility check; device pointers (all but mask may be None).
    Returns the number of Gaussians kept."""
    n = ctypes.c_int64()
    _check(lib.gs_visibility(h, ctypes.byref(cam), ctypes.byref(pose_), mask, uv, grad_mean, visible_ids,
                             visible_uv, ctypes.byref(n), stream))
    return n.value


def gs_scene_work_counts(h, stream=None):
    """(blended, evaluated) pairs of the last call's backward walk."""
    b, e = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.gs_scene_work_counts(h, _stream() if stream is None else stream, ctypes.byref(b), ctypes.byref(e)))
    return b.value, e.value


def gs_scene_stream_stats(h):
    """(bytes uploaded, partitions resident, partitions walked by the last call)."""
    b, r, a = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    _check(lib.gs_scene_stream_stats(h, ctypes.byref(b), ctypes.byref(r), ctypes.byref(a)))
    return b.value, r.value, a.value


def gs_scene_evict(h) -> None:
    _check(lib.gs_scene_evict(h))


def gs_version() -> str:
    return lib.gs_version().decode()


# ---- marshalling helpers (torch supplies device memory and the stream) ---------------------------
def camera(c) -> gs_camera:
    return gs_camera(int(c["width"]), int(c["height"]), float(c["fx"]), float(c["fy"]), float(c["cx"]),
                     float(c["cy"]))


def pose(T) -> gs_pose:
    # one copy of the 16 row-major doubles (a 4 x 4 matrix or 16 values)
    return gs_pose.from_buffer_copy(np.ascontiguousarray(T, np.float64).reshape(16))


def _ptr(t):
    """Raw pointer of a dense tensor: the C ABI reads every array in row-major
    order, so a strided view (a transpose, a slice) is refused, not misread."""
    if t is None:
        return 0
    if not t.is_contiguous():
        raise ValueError("arrays passed to the library must be contiguous (got strides %s for shape %s)"
                         % (tuple(t.stride()), tuple(t.shape)))
    return t.data_ptr()


def _f32(t, name):
    """_ptr of a float32 CUDA tensor (None passes through)."""
    if t is None:
        return 0
    import torch
    if not (t.is_cuda and t.dtype == torch.float32):
        raise ValueError("%s must be a float32 CUDA tensor" % name)
    return _ptr(t)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Scene:
    """Owns a gs_scene built from a dict of arrays (numpy or torch).

    Keys: means (n,3), scales (n,3), quats (n,4), opacities (n,), sh (n,K,3),
    sh_degree, optional feats_bf16 (n,32) uint16 and partition_offsets.
    """

    def __init__(self, scene: dict, stream_partitions: bool = False):
        """stream_partitions: pass host arrays and the partition table, so the
        library keeps the scene in pinned host memory and uploads partitions on
        demand (requires scene["partition_offsets"])."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if stream_partitions:
            self._init_host(scene)
            return

        def t(x, dtype):
            if isinstance(x, torch.Tensor):
                return x.to(device=dev, dtype=dtype).contiguous()
            return torch.from_numpy(np.ascontiguousarray(x)).to(device=dev, dtype=dtype).contiguous()

        self.n = int(np.asarray(scene["means"]).reshape(-1, 3).shape[0]) if not isinstance(scene["means"], torch.Tensor) \
            else int(scene["means"].reshape(-1, 3).shape[0])
        self.sh_degree = int(scene["sh_degree"])
        f = scene.get("feats_bf16")
        self.feat_dim = 0 if f is None else 32
        keep = [t(scene["means"], torch.float32), t(scene["scales"], torch.float32), t(scene["quats"], torch.float32),
                t(scene["opacities"], torch.float32), t(scene["sh"], torch.float32)]
        fb = None if f is None else t(np.asarray(f).view(np.int16) if not isinstance(f, torch.Tensor) else f,
                                      torch.int16)
        po = scene.get("partition_offsets")
        po_np = None if po is None else np.ascontiguousarray(po, np.int64)
        self._desc = gs_scene_desc(self.n, self.sh_degree, self.feat_dim, *[_ptr(k) for k in keep], _ptr(fb),
                                   0 if po_np is None else len(po_np) - 1,
                                   None if po_np is None else po_np.ctypes.data, 1)
        torch.cuda.synchronize()
        self.handle = gs_create_scene(self._desc)

    def _init_host(self, scene):
        keep = [np.ascontiguousarray(scene[k], np.float32) for k in ("means", "scales", "quats", "opacities", "sh")]
        f = scene.get("feats_bf16")
        fb = None if f is None else np.ascontiguousarray(f, np.uint16)
        po = np.ascontiguousarray(scene["partition_offsets"], np.int64)
        self.n = int(keep[0].reshape(-1, 3).shape[0])
        self.sh_degree = int(scene["sh_degree"])
        self.feat_dim = 0 if fb is None else 32
        self._desc = gs_scene_desc(self.n, self.sh_degree, self.feat_dim, *[k.ctypes.data for k in keep],
                                   None if fb is None else fb.ctypes.data, len(po) - 1, po.ctypes.data, 0)
        self.handle = gs_create_scene(self._desc)

    def stream_stats(self):
        return gs_scene_stream_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            gs_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def alloc_outputs(cam, feat_dim=0, last_idx=True):
        import torch
        H, W = int(cam["height"]), int(cam["width"])
        o = {"rgb": torch.empty((3, H, W), device="cuda"), "depth": torch.empty((H, W), device="cuda"),
             "alpha": torch.empty((H, W), device="cuda"), "final_T": torch.empty((H, W), device="cuda")}
        if feat_dim:
            o["feats"] = torch.empty((feat_dim, H, W), device="cuda")
        if last_idx:
            o["last_idx"] = torch.empty((H, W), device="cuda", dtype=torch.int32)
        return o

    @staticmethod
    def outputs_struct(o) -> gs_outputs:
        if o is None:
            return gs_outputs()
        return gs_outputs(_ptr(o.get("rgb")), _ptr(o.get("depth")), _ptr(o.get("alpha")), _ptr(o.get("final_T")),
                          _ptr(o.get("feats")), _ptr(o.get("last_idx")))

    def render(self, cam, T, out=None, sync=True):
        out = out if out is not None else self.alloc_outputs(cam, self.feat_dim)
        fn = gs_render if sync else gs_render_async
        fn(self.handle, camera(cam), pose(T), self.outputs_struct(out), _stream())
        return out

    def render_pose_grad(self, cam, T, target_rgb, target_depth, pixel_weight=None, depth_weight=0.1, out=None):
        return gs_render_pose_grad(self.handle, camera(cam), pose(T), _f32(target_rgb, "target_rgb"),
                                   _f32(target_depth, "target_depth"), _f32(pixel_weight, "pixel_weight") or None,
                                   depth_weight,
                                   self.outputs_struct(out) if out is not None else None, _stream())

    def render_pose_grad_host(self, cam, T, target_rgb, target_depth, pixel_weight=None, depth_weight=0.1,
                              out=None):
        """Pose gradient with host-memory targets: contiguous float32 numpy arrays or
        CPU torch tensors (pinned tensors let the upload overlap the projection)."""
        def hptr(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                if a.is_cuda or a.dtype != __import__("torch").float32 or not a.is_contiguous():
                    raise ValueError("host targets must be contiguous float32 CPU tensors")
                return a.data_ptr()
            if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host targets must be contiguous float32 arrays")
            return a.ctypes.data
        return gs_render_pose_grad_host(self.handle, camera(cam), pose(T), hptr(target_rgb), hptr(target_depth),
                                        hptr(pixel_weight), depth_weight,
                                        self.outputs_struct(out) if out is not None else None, _stream())

    def render_pose_grad_batch(self, cams, poses, target_rgb, target_depth, pixel_weight=None, depth_weight=0.1,
                               outs=None, results=None, graph=False):
        """Batched pose gradient; tensors are per-view lists. Returns (loss[n], grad[n,6])
        synchronously, or None in graph mode (results: device float64 tensor (n, 8))."""
        return gs_render_pose_grad_batch(
            self.handle, [camera(c) for c in cams], [pose(T) for T in poses],
            [_f32(t, "target_rgb") for t in target_rgb], [_f32(t, "target_depth") for t in target_depth],
            None if pixel_weight is None else [_f32(t, "pixel_weight") for t in pixel_weight],
            depth_weight, None if outs is None else [self.outputs_struct(o) for o in outs],
            _ptr(results), GS_BATCH_GRAPH if graph else 0, _stream())

    def render_batch(self, cams, poses, outs, graph=False):
        gs_render_batch(self.handle, [camera(c) for c in cams], [pose(T) for T in poses],
                        [self.outputs_struct(o) for o in outs], GS_BATCH_GRAPH if graph else 0, _stream())
        return outs

    def visibility(self, cam, T, grad=True, compact=True):
        """Algorithm 1 from pose T: dict of device tensors mask (n uint8: bit 0 M,
        bit 1 M^r, bit 2 M^i), uv (n, 2), grad (n, 3) or None, ids (K,) and
        uv_visible (K, 2) of the kept Gaussians (compact=True), and n_visible."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        mask = torch.empty(max(self.n, 1), dtype=torch.uint8, device=dev)
        uv = torch.empty((max(self.n, 1), 2), dtype=torch.float32, device=dev)
        g = torch.empty((max(self.n, 1), 3), dtype=torch.float32, device=dev) if grad else None
        ids = torch.empty(max(self.n, 1), dtype=torch.int32, device=dev) if compact else None
        uvv = torch.empty((max(self.n, 1), 2), dtype=torch.float32, device=dev) if compact else None
        k = gs_visibility(self.handle, camera(cam), pose(T), _ptr(mask), _ptr(uv), _ptr(g), _ptr(ids), _ptr(uvv),
                          _stream())
        n = self.n
        return {"mask": mask[:n], "uv": uv[:n], "grad": None if g is None else g[:n],
                "ids": None if ids is None else ids[:k], "uv_visible": None if uvv is None else uvv[:k],
                "n_visible": k}

    def status(self):
        return gs_scene_status(self.handle, _stream())

    def reserve(self, max_records, max_pairs):
        gs_scene_reserve(self.handle, max_records, max_pairs)

    def tile_lists(self, view, cam, capacity):
        tiles = ((int(cam["width"]) + 15) // 16) * ((int(cam["height"]) + 15) // 16)
        return gs_get_tile_lists(self.handle, view, tiles, capacity, _stream())

    def records(self, view, capacity):
        return gs_get_records(self.handle, view, capacity, _stream())


def pose_loss_function():
    """torch.autograd.Function: loss(xi) of the L1 photometric + depth objective
    at the pose tangent xi = 0 of a given pose; backward returns dL/dxi from the
    CUDA adjoint (gs_render_pose_grad). The tangent is re-linearised at every
    call, so callers update the pose (T <- Exp(-step) T) and pass xi = 0."""
    import torch

    class PoseLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xi, scene, cam, T, target_rgb, target_depth, pixel_weight=None, depth_weight=0.1):
            loss, grad = scene.render_pose_grad(cam, T, target_rgb, target_depth, pixel_weight, depth_weight)
            ctx.save_for_backward(torch.as_tensor(grad, dtype=xi.dtype, device=xi.device))
            return torch.as_tensor(loss, dtype=xi.dtype, device=xi.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad, None, None, None, None, None, None, None

    return PoseLoss


# ---- probabilistic mutual matching (Sec. 3.4, Eq. 11) ---------------------------------------------
def gs_pmm_create(channels: int, height: int, width: int):
    h = ctypes.c_void_p()
    _check(lib.gs_pmm_create(int(channels), int(height), int(width), ctypes.byref(h)))
    return h


def gs_pmm_destroy(h) -> None:
    lib.gs_pmm_destroy(h)


def _cams(cams):
    arr = (gs_camera * len(cams))(*[c if isinstance(c, gs_camera) else camera(c) for c in cams])
    return len(cams), arr


def gs_scene_set_launch(h, mode: int, cams, variant: int, ctas_per_sm: int = 0, grid_mult: int = 8) -> None:
    n, arr = _cams(cams)
    cfg = gs_launch(int(variant), int(ctas_per_sm), int(grid_mult), 0, 0, 0)
    _check(lib.gs_scene_set_launch(h, int(mode), n, arr, ctypes.byref(cfg)))


def gs_scene_get_launch(h, mode: int, cams) -> dict:
    n, arr = _cams(cams)
    cfg = gs_launch()
    _check(lib.gs_scene_get_launch(h, int(mode), n, arr, ctypes.byref(cfg)))
    return cfg.as_dict()


def gs_autotune(h, mode: int, cams, poses, reps: int = 5, stream=None) -> dict:
    n, arr = _cams(cams)
    pp = (gs_pose * n)(*[p if isinstance(p, gs_pose) else pose(p) for p in poses])
    r = gs_tune_result()
    _check(lib.gs_autotune(h, int(mode), n, arr, pp, int(reps), ctypes.byref(r), _stream() if stream is None else stream))
    return {"best": r.best.as_dict(), "ms_default": r.ms_default, "ms_best": r.ms_best, "candidates": r.candidates}


def gs_tune_save(h, path: str) -> None:
    _check(lib.gs_tune_save(h, path.encode()))


def gs_tune_load(h, path: str) -> int:
    n = ctypes.c_int()
    _check(lib.gs_tune_load(h, path.encode(), ctypes.byref(n)))
    return n.value


GS_PMM_DEFAULT_WAIT_POLLS = 1 << 22


def gs_pmm_set_wait_limit(h, polls: int) -> None:
    _check(lib.gs_pmm_set_wait_limit(h, int(polls)))


def gs_pmm_match(h, feat_query: int, feat_render: int, tau: float, stream: int) -> gs_pmm_result:
    r = gs_pmm_result()
    _check(lib.gs_pmm_match(h, feat_query, feat_render, float(tau), ctypes.byref(r), stream))
    return r


class _DevView:
    """A device array of the library, seen by torch without a copy."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


class Matcher:
    """PMM of two (32, H, W) fp32 CUDA feature maps; ``match`` returns copies of the results."""

    def __init__(self, height: int, width: int, channels: int = 32):
        self.H, self.W = int(height), int(width)
        self.handle = gs_pmm_create(channels, self.H, self.W)

    def close(self):
        if self.handle:
            gs_pmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def match_raw(self, feat_query, feat_render, tau: float = 0.1):
        """The gs_pmm_match call alone: its result struct, whose device arrays
        belong to the matcher until its next call."""
        import torch
        for f in (feat_query, feat_render):
            if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous() and f.shape[1:] == (self.H, self.W)):
                raise ValueError("feature maps must be contiguous float32 CUDA tensors of shape (32, H, W)")
        return gs_pmm_match(self.handle, feat_query.data_ptr(), feat_render.data_ptr(), tau, _stream())

    def match(self, feat_query, feat_render, tau: float = 0.1) -> dict:
        """match_raw, with copies of the matcher's device outputs."""
        import torch
        r = self.match_raw(feat_query, feat_render, tau)
        n, nc, nf = r.n_cells, r.n_coarse, r.n_fine
        v = lambda p, shape, t: torch.as_tensor(_DevView(p, shape, t), device="cuda").clone()
        return {"codes_q": v(r.codes_q, (n, 64), "<u2"), "codes_r": v(r.codes_r, (n, 64), "<u2"),
                "lse_row": v(r.lse_row, (n,), "<f4"), "lse_col": v(r.lse_col, (n,), "<f4"),
                "row_best": v(r.row_best, (n,), "<i4"), "col_best": v(r.col_best, (n,), "<i4"),
                "coarse": v(r.coarse, (nc, 2), "<i4") if nc else torch.zeros((0, 2), dtype=torch.int32, device="cuda"),
                "coarse_prob": v(r.coarse_prob, (nc,), "<f4") if nc else torch.zeros(0, device="cuda"),
                "fine": v(r.fine, (nf, 3), "<i4") if nf else torch.zeros((0, 3), dtype=torch.int32, device="cuda"),
                "fine_prob": v(r.fine_prob, (nf,), "<f4") if nf else torch.zeros(0, device="cuda")}


# ---- dense PnP + RANSAC (Sec. 3.4, Eq. 10) ------------------------------------------------------
def gs_pnp_defaults() -> gs_pnp_opts:
    return lib.gs_pnp_defaults()


def gs_pnp_create(max_matches: int, max_hypotheses: int):
    h = ctypes.c_void_p()
    _check(lib.gs_pnp_create(max_matches, max_hypotheses, ctypes.byref(h)))
    return h


def gs_pnp_destroy(h) -> None:
    lib.gs_pnp_destroy(h)


def gs_pnp_solve(h, cam: gs_camera, T_render: gs_pose, depth: int, alpha: int, matches: int, n_matches: int,
                 words: int, n_hypotheses: int, opts: gs_pnp_opts, stream: int) -> gs_pnp_result:
    r = gs_pnp_result()
    _check(lib.gs_pnp_solve(h, ctypes.byref(cam), ctypes.byref(T_render), depth, alpha, matches, n_matches, words,
                            n_hypotheses, ctypes.byref(opts), ctypes.byref(r), stream))
    return r


PNP_PHASES = ("lift", "p3p", "score", "best", "refine", "final")


def gs_pnp_set_timing(h, enable: bool) -> None:
    _check(lib.gs_pnp_set_timing(h, int(bool(enable))))


def gs_pnp_phase_times(h):
    ms = np.zeros(len(PNP_PHASES), np.float64)
    n = ctypes.c_int64()
    _check(lib.gs_pnp_phase_times(h, ms.ctypes.data, ctypes.byref(n)))
    return ms, n.value


class PnP:
    """Dense PnP + RANSAC on rendered depth; ``solve`` returns the pose and copies
    of the device results."""

    def __init__(self, max_matches: int, max_hypotheses: int = 256):
        self.handle = gs_pnp_create(max_matches, max_hypotheses)

    def close(self):
        if self.handle:
            gs_pnp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve_raw(self, cam, T_render, depth, alpha, matches, words, tau=2.0, min_alpha=0.5,
                  refine_iters=5) -> "gs_pnp_result":
        """The gs_pnp_solve call alone: its result struct, whose device arrays
        belong to the solver until its next call."""
        import torch
        for t, dt in ((depth, torch.float32), (alpha, torch.float32), (matches, torch.int32)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise ValueError("depth / alpha (float32) and matches (int32) must be contiguous CUDA tensors")
        if not (words.is_cuda and words.is_contiguous() and words.element_size() == 4):
            raise ValueError("words must be a contiguous 32-bit CUDA tensor")
        o = gs_pnp_opts(tau, min_alpha, refine_iters)
        K, nh = int(matches.shape[0]), int(words.shape[0])
        return gs_pnp_solve(self.handle, camera(cam), pose(T_render), depth.data_ptr(), alpha.data_ptr(),
                            matches.data_ptr() if K else None, K, words.data_ptr() if nh else None, nh, o,
                            _stream())

    def solve(self, cam, T_render, depth, alpha, matches, words, tau=2.0, min_alpha=0.5, refine_iters=5) -> dict:
        """depth, alpha: (H, W) float32 CUDA tensors rendered at T_render; matches:
        (K, 3) int32 CUDA tensor (PMM fine layout); words: (n_hyp, 3) int32 or
        uint32-bits CUDA tensor of random words."""
        import torch
        r = self.solve_raw(cam, T_render, depth, alpha, matches, words, tau, min_alpha, refine_iters)
        K, nh = int(matches.shape[0]), int(words.shape[0])
        nv = r.n_valid
        v = lambda p, shape, t: torch.as_tensor(_DevView(p, shape, t), device="cuda").clone()
        empty = lambda shape, dt: torch.zeros(shape, dtype=dt, device="cuda")
        return {"T": np.array(r.T_cw[:], np.float64).reshape(4, 4), "n_valid": nv, "n_inliers": r.n_inliers,
                "best": (r.best_hypothesis, r.best_solution), "best_count": r.best_count,
                "refine_steps": r.refine_steps,
                "inlier": v(r.inlier, (K,), "|u1") if K else empty((0,), torch.uint8),
                "valid_index": v(r.valid_index, (nv,), "<i4") if nv else empty((0,), torch.int32),
                "points": v(r.points, (nv, 3), "<f8") if nv else empty((0, 3), torch.float64),
                "hyp_counts": v(r.hyp_counts, (nh, 4), "<i4") if nh else empty((0, 4), torch.int32),
                "hyp_poses": v(r.hyp_poses, (nh, 4, 12), "<f8") if nh else empty((0, 4, 12), torch.float64)}


# ---- dense stage with Algorithm 2's consistency check ------------------------------------------
def gs_pose_difference(T1, T2):
    """Algorithm 2's Psi: (angle in degrees, translation distance)."""
    a, d = ctypes.c_double(), ctypes.c_double()
    _check(lib.gs_pose_difference(ctypes.byref(pose(T1)), ctypes.byref(pose(T2)), ctypes.byref(a), ctypes.byref(d)))
    return a.value, d.value


def gs_localize_defaults() -> gs_localize_opts:
    return lib.gs_localize_defaults()


def dense_localize(scene, matcher, solver, cam, T_init, feat_query, words, n_rounds=3, n_hypotheses=None,
                   pmm_tau=0.1, max_angle_deg=20.0, tau=2.0, min_alpha=0.5, refine_iters=5) -> dict:
    """Algorithm 2 around n rounds of render -> PMM -> PnP. feat_query: (32, H, W)
    float32 CUDA tensor; words: (n_rounds, n_hypotheses, 3) 32-bit CUDA tensor."""
    import torch
    if not (feat_query.is_cuda and feat_query.dtype == torch.float32 and feat_query.is_contiguous()):
        raise ValueError("feat_query must be a contiguous float32 CUDA tensor")
    if not (words.is_cuda and words.is_contiguous() and words.element_size() == 4 and words.dim() == 3):
        raise ValueError("words must be a contiguous 32-bit CUDA tensor (rounds, hypotheses, 3)")
    nh = int(words.shape[1]) if n_hypotheses is None else int(n_hypotheses)
    o = gs_localize_opts(n_rounds, pmm_tau, max_angle_deg, nh, gs_pnp_opts(tau, min_alpha, refine_iters))
    r = gs_localize_result()
    _check(lib.gs_dense_localize(scene.handle, matcher.handle, solver.handle, ctypes.byref(camera(cam)),
                                 ctypes.byref(pose(T_init)), feat_query.data_ptr(), words.data_ptr(),
                                 ctypes.byref(o), ctypes.byref(r), _stream()))
    n = r.n_rounds
    return {"T": np.array(r.T_cw[:], np.float64).reshape(4, 4), "reliable": bool(r.reliable), "n_rounds": n,
            "round_T": [np.array(r.round_T[i][:], np.float64).reshape(4, 4) for i in range(n)],
            "angle_deg": list(r.angle_deg[:max(0, n - 1)]), "trans": list(r.trans[:max(0, n - 1)]),
            "n_matches": list(r.n_matches[:n]), "n_inliers": list(r.n_inliers[:n])}
