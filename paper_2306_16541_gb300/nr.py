"""Thin ctypes binding of libnr.so (the C ABI declared in include/nr.h).

Argument marshalling only: every step of rendering and training runs in the
library's CUDA kernels.  The functions keep the ABI's names (nr_create_subject,
nr_set_pose, nr_render, nr_query, nr_set_frames, nr_train_step, nr_param,
nr_destroy); `Subject` wraps one handle.  Device buffers are torch CUDA
tensors; streams are torch CUDA streams.  Importing this module raises if
libnr.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnr.so")

NR_OK, NR_EINVAL, NR_ENOMEM, NR_ECUDA, NR_ESTATE, NR_ETIMEOUT, NR_EBUSY, NR_EUNSUPPORTED = range(8)
NR_F32, NR_F16, NR_BF16, NR_FP8E4M3 = range(4)
DTYPES = {"f32": NR_F32, "f16": NR_F16, "bf16": NR_BF16, "fp8": NR_FP8E4M3}
NR_POSE_MATRICES = 1
NR_GRAD_ONLY = 1
NR_FORWARD_ONLY = 2
NR_TRAIN_WVOL, NR_TRAIN_HASH, NR_TRAIN_MLP, NR_TRAIN_RES, NR_TRAIN_REFINER, NR_TRAIN_CNN = 1, 2, 4, 8, 16, 32
NR_TRAIN_ALL = 63
NR_PARAM_WVOL, NR_PARAM_HASH, NR_PARAM_MLP, NR_PARAM_RES, NR_PARAM_REFINER, NR_PARAM_CNN = range(6)
# Per-group learning-rate multipliers (weight volume, hash, canonical MLP, residual MLP):
# Sec. 5.2 uses a 10x smaller rate for the networks other than the NeRF network.
PAPER_LR_SCALE = (0.1, 1.0, 1.0, 0.1)
PAPER_MSE_WEIGHT = 0.2      # lambda_mse of Sec. 5.2
NR_QUERY_STRIDE = 12
NR_RENDER_PROFILE = 1
NR_RENDER_ALL_BONES = 8
NR_RENDER_TCGEN05 = 2
NR_RENDER_MMA2 = 4
NR_RENDER_F32_TC = 16
NR_RENDER_MMA_SYNC = 32
NR_SERVE_SMALLEST_FIRST, NR_SERVE_FIFO, NR_SERVE_EDF = 0, 1, 2
NR_ABI_VERSION = 1

_fp = C.POINTER(C.c_float)
_up = C.POINTER(C.c_uint32)


class nr_subject_desc(C.Structure):
    _fields_ = [("abi_version", C.c_uint32), ("n_bones", C.c_uint32),
                ("parents", C.POINTER(C.c_int32)), ("rest_joints", _fp),
                ("box_min", C.c_float * 3), ("box_max", C.c_float * 3),
                ("wvol_res", C.c_uint32), ("wvol", _fp),
                ("hash_levels", C.c_uint32), ("hash_feats", C.c_uint32), ("log2_T", C.c_uint32),
                ("level_res", _up), ("hash_table", _fp),
                ("mlp_in", C.c_uint32), ("mlp_width", C.c_uint32), ("mlp_hidden_layers", C.c_uint32),
                ("mlp_params", _fp),
                ("res_enabled", C.c_uint32), ("res_pe_freqs", C.c_uint32), ("res_params", _fp),
                ("ellipsoids", _fp), ("occ_grid", C.c_uint32), ("device", C.c_int32)]


class nr_camera(C.Structure):
    _fields_ = [("width", C.c_uint32), ("height", C.c_uint32),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("t_near", C.c_float), ("t_far", C.c_float), ("n_samples", C.c_uint32),
                ("bg", C.c_float * 3)]


class nr_render_opts(C.Structure):
    _fields_ = [("mlp_dtype", C.c_int), ("feat_dtype", C.c_int), ("use_occupancy", C.c_uint32),
                ("t_min", C.c_float), ("hann_alpha", C.c_float), ("flags", C.c_uint32)]


class nr_train_batch(C.Structure):
    _fields_ = [("n_rays", C.c_uint32), ("frame_id", _up), ("px", _up), ("py", _up),
                ("target_rgb", _fp), ("n_samples", C.c_uint32), ("bg", C.c_float * 3),
                ("step_seed", C.c_uint64), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("hann_alpha", C.c_float), ("flags", C.c_uint32),
                ("train_mask", C.c_uint32), ("lr_scale", C.c_float * 4), ("loss_weight", C.c_float),
                ("lr_scale_refiner", C.c_float), ("lr_scale_cnn", C.c_float),
                ("pred_rgb", _fp), ("grad_rgb", _fp)]


class nr_request(C.Structure):
    _fields_ = [("subject", C.c_uint32), ("cam", nr_camera), ("axis_angle", C.c_float * 72),
                ("root_t", C.c_float * 3), ("opts", nr_render_opts), ("out_rgba", C.c_void_p)]


class nr_server_policy(C.Structure):
    _fields_ = [("order", C.c_uint32), ("age_ms", C.c_float), ("deadline_ms", C.c_float),
                ("deadline_ms_per_mpixel", C.c_float), ("priority_streams", C.c_uint32)]


class nr_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("rejected", C.c_uint64), ("active", C.c_uint32), ("queued", C.c_uint32),
                ("slots", C.c_uint32), ("peak_active", C.c_uint32), ("bytes_in_use", C.c_uint64),
                ("rays_done", C.c_double)]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2306_16541_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "nr_create_subject": ([C.POINTER(nr_subject_desc), vp, C.POINTER(vp)], C.c_int),
        "nr_destroy": ([vp], C.c_int),
        "nr_set_pose": ([vp, _fp, _fp, C.c_uint32, vp], C.c_int),
        "nr_render": ([vp, C.POINTER(nr_camera), C.POINTER(nr_render_opts), vp, vp], C.c_int),
        "nr_query": ([vp, C.c_uint32, vp, C.POINTER(nr_render_opts), vp, vp], C.c_int),
        "nr_set_frames": ([vp, C.c_uint32, _fp, _fp, C.POINTER(nr_camera), vp], C.c_int),
        "nr_train_step": ([vp, C.POINTER(nr_train_batch), _fp, vp], C.c_int),
        "nr_param": ([vp, C.c_uint32, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_size_t)], C.c_int),
        "nr_params_changed": ([vp], C.c_int),
        "nr_pose_transforms": ([vp, _fp], C.c_int),
        "nr_occupancy": ([vp, _up], C.c_int),
        "nr_refresh_occupancy": ([vp, C.c_float, C.c_uint32, C.c_float, vp], C.c_int),
        "nr_set_canonical_occupancy": ([vp, _up, C.c_float, vp], C.c_int),
        "nr_canonical_occupancy": ([vp, _up], C.c_int),
        "nr_set_pose_refiner": ([vp, C.c_uint32, C.c_uint32, _fp, vp], C.c_int),
        "nr_set_weight_cnn": ([vp, _up, _fp, _fp, _fp, vp], C.c_int),
        "nr_render_static": ([vp, C.POINTER(nr_camera), C.POINTER(nr_render_opts), vp, vp], C.c_int),
        "nr_stage_times": ([vp, _fp], C.c_int),
        "nr_launch_count": ([], C.c_uint64),
        "nr_field_error_word": ([vp, C.POINTER(vp)], C.c_int),
        "nr_l2_gather_rate": ([C.c_int, C.c_uint64, C.c_uint32, C.POINTER(C.c_double)], C.c_int),
        "nr_server_create": ([C.c_int, C.c_uint64, C.c_uint32, C.POINTER(vp)], C.c_int),
        "nr_server_add_subject": ([vp, vp, C.POINTER(C.c_uint32)], C.c_int),
        "nr_server_set_policy": ([vp, C.POINTER(nr_server_policy)], C.c_int),
        "nr_server_submit": ([vp, C.POINTER(nr_request), C.POINTER(C.c_uint64)], C.c_int),
        "nr_server_poll": ([vp, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_double)], C.c_int),
        "nr_server_wait": ([vp, C.c_uint64, C.c_uint32, C.POINTER(C.c_double)], C.c_int),
        "nr_server_get_stats": ([vp, C.POINTER(nr_server_stats)], C.c_int),
        "nr_server_stop": ([vp, C.c_uint32], C.c_int),
        "nr_server_destroy": ([vp], C.c_int),
        "nr_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


class NRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: status {code}: {lib.nr_last_error().decode()}")


def check(code: int, where: str) -> None:
    if code != NR_OK:
        raise NRError(code, where)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, np.float32))


def _ptr(a: np.ndarray, t=C.c_float):
    return a.ctypes.data_as(C.POINTER(t))


def _stream(stream) -> C.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_camera(cam) -> nr_camera:
    """nr_camera from an object with width, height, fx, fy, cx, cy, R, t, t_near, t_far, n_samples, bg."""
    c = nr_camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.R[:] = [float(v) for v in _f32(cam.R).ravel()]
    c.t[:] = [float(v) for v in _f32(cam.t).ravel()]
    c.t_near, c.t_far, c.n_samples = float(cam.t_near), float(cam.t_far), int(cam.n_samples)
    c.bg[:] = [float(v) for v in _f32(cam.bg).ravel()]
    return c


def make_opts(mlp: str = "f32", feat: str = "f32", occupancy: bool = False, t_min: float = 0.0,
              hann_alpha: float = -1.0, profile: bool = False, tcgen05: bool = False,
              mma2: bool = False, all_bones: bool = False, f32_tc: bool = False,
              mma_sync: bool = False) -> nr_render_opts:
    o = nr_render_opts()
    o.mlp_dtype, o.feat_dtype = DTYPES[mlp], DTYPES[feat]
    o.use_occupancy, o.t_min, o.hann_alpha = int(bool(occupancy)), float(t_min), float(hann_alpha)
    o.flags = ((NR_RENDER_PROFILE if profile else 0) | (NR_RENDER_TCGEN05 if tcgen05 else 0)
               | (NR_RENDER_MMA2 if mma2 else 0) | (NR_RENDER_ALL_BONES if all_bones else 0)
               | (NR_RENDER_F32_TC if f32_tc else 0) | (NR_RENDER_MMA_SYNC if mma_sync else 0))
    return o


def nr_stage_times(h) -> dict:
    """Stage times (ms) and live-sample count of the last profiled nr_render."""
    ms = np.zeros(6, np.float32)
    check(lib.nr_stage_times(h, _ptr(ms)), "nr_stage_times")
    return dict(march_ms=float(ms[0]), field_ms=float(ms[1]), composite_ms=float(ms[2]),
                chunks=int(ms[3]), live_samples=int(ms[4]), bones_read_per_sample=float(ms[5]))


def nr_launch_count() -> int:
    return int(lib.nr_launch_count())


def nr_l2_gather_rate(device: int, table_bytes: int, load_bytes: int) -> float:
    """Bytes per second of random L2-resident gathers of load_bytes (see include/nr.h)."""
    v = C.c_double()
    check(lib.nr_l2_gather_rate(int(device), int(table_bytes), int(load_bytes), C.byref(v)), "nr_l2_gather_rate")
    return float(v.value)


class _DevArray:
    """A float32 device buffer exposed through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3, "strides": None}


def nr_create_subject(subj: dict, device: int = 0, stream=None) -> C.c_void_p:
    keep = {}

    def arr(name, a, t=np.float32):
        keep[name] = np.ascontiguousarray(np.asarray(a, t))
        return keep[name]

    d = nr_subject_desc()
    d.abi_version, d.n_bones = NR_ABI_VERSION, len(subj["parents"])
    d.parents = _ptr(arr("parents", subj["parents"], np.int32), C.c_int32)
    d.rest_joints = _ptr(arr("rest", subj["rest_joints"]))
    d.box_min[:] = [float(v) for v in subj["box_min"]]
    d.box_max[:] = [float(v) for v in subj["box_max"]]
    d.wvol_res = int(subj["wvol_res"])
    d.wvol = _ptr(arr("wvol", subj["wvol"]))
    d.hash_levels, d.hash_feats, d.log2_T = int(subj["hash_levels"]), int(subj["hash_feats"]), int(subj["log2_T"])
    d.level_res = _ptr(arr("levels", subj["level_res"], np.uint32), C.c_uint32)
    d.hash_table = _ptr(arr("table", subj["hash_table"]))
    d.mlp_in, d.mlp_width, d.mlp_hidden_layers = (int(subj["mlp_in"]), int(subj["mlp_width"]),
                                                  int(subj["mlp_hidden_layers"]))
    d.mlp_params = _ptr(arr("mlp", subj["mlp_params"]))
    d.res_enabled, d.res_pe_freqs = int(subj["res_enabled"]), int(subj["res_pe_freqs"])
    d.res_params = _ptr(arr("res", subj["res_params"]))
    if subj.get("ellipsoids") is not None:
        d.ellipsoids = _ptr(arr("ell", subj["ellipsoids"]))
    d.occ_grid = int(subj.get("occ_grid", 128))
    d.device = int(device)
    h = C.c_void_p()
    check(lib.nr_create_subject(C.byref(d), _stream(stream), C.byref(h)), "nr_create_subject")
    return h


def nr_destroy(h) -> None:
    check(lib.nr_destroy(h), "nr_destroy")


def nr_set_pose(h, axis_angle, root_t=None, flags: int = 0, stream=None) -> None:
    aa = _f32(axis_angle)
    rt = _f32(root_t if root_t is not None else np.zeros(3))
    check(lib.nr_set_pose(h, _ptr(aa), _ptr(rt), flags, _stream(stream)), "nr_set_pose")


def nr_render(h, cam: nr_camera, opts: nr_render_opts, out, stream=None) -> None:
    """out: a CUDA tensor or a host numpy/torch buffer of height*width*4 float32."""
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    check(lib.nr_render(h, C.byref(cam), C.byref(opts), C.c_void_p(ptr), _stream(stream)), "nr_render")


def nr_render_static(h, cam: nr_camera, opts: nr_render_opts, out, stream=None) -> None:
    """Allocation-free render into a CUDA tensor (see include/nr.h for its limits)."""
    check(lib.nr_render_static(h, C.byref(cam), C.byref(opts), C.c_void_p(out.data_ptr()), _stream(stream)),
          "nr_render_static")


def nr_query(h, x_obs, opts: nr_render_opts, out, stream=None) -> None:
    check(lib.nr_query(h, int(x_obs.shape[0]), C.c_void_p(x_obs.data_ptr()), C.byref(opts),
                       C.c_void_p(out.data_ptr()), _stream(stream)), "nr_query")


def nr_set_frames(h, axis_angle, root_t, cameras, stream=None) -> None:
    aa = _f32(axis_angle)
    rt = _f32(root_t)
    cams = (nr_camera * len(cameras))(*[make_camera(c) for c in cameras])
    check(lib.nr_set_frames(h, len(cameras), _ptr(aa), _ptr(rt), cams, _stream(stream)), "nr_set_frames")


def nr_train_step(h, batch: nr_train_batch, stream=None) -> float:
    loss = C.c_float(0.0)
    check(lib.nr_train_step(h, C.byref(batch), C.byref(loss), _stream(stream)), "nr_train_step")
    return float(loss.value)


def nr_param(h, which: int):
    """(params, grads) as zero-copy float32 CUDA tensors."""
    import torch
    p, g, n = C.c_void_p(), C.c_void_p(), C.c_size_t()
    check(lib.nr_param(h, which, C.byref(p), C.byref(g), C.byref(n)), "nr_param")
    if n.value == 0 or not p.value:   # a group not in use (no refiner, no CNN_skel)
        return (torch.empty(0, device="cuda"), torch.empty(0, device="cuda"))
    return (torch.as_tensor(_DevArray(p.value, n.value), device="cuda"),
            torch.as_tensor(_DevArray(g.value, n.value), device="cuda"))


def nr_params_changed(h) -> None:
    check(lib.nr_params_changed(h), "nr_params_changed")


def nr_pose_transforms(h) -> np.ndarray:
    G = np.zeros((24, 12), np.float32)
    check(lib.nr_pose_transforms(h, _ptr(G)), "nr_pose_transforms")
    return G


def nr_occupancy(h, grid: int = 128) -> np.ndarray:
    bits = np.zeros(grid ** 3 // 32, np.uint32)
    check(lib.nr_occupancy(h, _ptr(bits, C.c_uint32)), "nr_occupancy")
    return bits


OCC_S_MIN = 1e-3   # default least bone-weight sum of a posed occupancy cell


def nr_refresh_occupancy(h, sigma_threshold: float, dilate: int = 1, s_min: float = OCC_S_MIN,
                         stream=None) -> None:
    check(lib.nr_refresh_occupancy(h, float(sigma_threshold), int(dilate), float(s_min), _stream(stream)),
          "nr_refresh_occupancy")


def nr_set_canonical_occupancy(h, bits, s_min: float = OCC_S_MIN, stream=None) -> None:
    b = np.ascontiguousarray(bits, np.uint32)
    check(lib.nr_set_canonical_occupancy(h, _ptr(b, C.c_uint32), float(s_min), _stream(stream)),
          "nr_set_canonical_occupancy")


def nr_canonical_occupancy(h, grid: int = 128) -> np.ndarray:
    bits = np.zeros(grid ** 3 // 32, np.uint32)
    check(lib.nr_canonical_occupancy(h, _ptr(bits, C.c_uint32)), "nr_canonical_occupancy")
    return bits


def nr_set_pose_refiner(h, layers, stream=None) -> None:
    """layers: MLP_theta as [(W [out][in], b [out]), ...] (hidden layers then the output
    layer), or None to switch the refiner off."""
    if layers is None:
        check(lib.nr_set_pose_refiner(h, 0, 0, None, _stream(stream)), "nr_set_pose_refiner")
        return
    width = int(layers[0][0].shape[0])
    flat = np.ascontiguousarray(np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(),
                                                                np.asarray(b, np.float32).ravel()])
                                                for W, b in layers]), np.float32)
    check(lib.nr_set_pose_refiner(h, width, len(layers) - 1, _ptr(flat), _stream(stream)), "nr_set_pose_refiner")


def nr_set_weight_cnn(h, layers, z=None, log_prior=None, stream=None) -> None:
    """layers: CNN_skel as [(W_fc [C0][256], b_fc), (W_1 [C0][C1][4][4][4], b_1), ...,
    (W_5 [C4][25][4][4][4], b_5)], or None to switch the generator off."""
    if layers is None:
        check(lib.nr_set_weight_cnn(h, None, None, None, None, _stream(stream)), "nr_set_weight_cnn")
        return
    ch = np.array([layers[0][0].shape[0]] + [W.shape[1] for W, _ in layers[1:5]], np.uint32)
    flat = np.ascontiguousarray(np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(),
                                                                np.asarray(b, np.float32).ravel()])
                                                for W, b in layers]), np.float32)
    zz = np.ascontiguousarray(z, np.float32)
    lp = None if log_prior is None else np.ascontiguousarray(log_prior, np.float32)
    check(lib.nr_set_weight_cnn(h, _ptr(ch, C.c_uint32), _ptr(flat), _ptr(zz),
                                None if lp is None else _ptr(lp), _stream(stream)), "nr_set_weight_cnn")


class Subject:
    """One performer resident on the GPU (owns an nr_subject handle)."""

    def __init__(self, subj: dict, device: int = 0, stream=None):
        self.h = nr_create_subject(subj, device, stream)
        self.occ_grid = int(subj.get("occ_grid", 128))

    def set_pose(self, axis_angle, root_t=None, matrices: bool = False, stream=None):
        nr_set_pose(self.h, axis_angle, root_t, NR_POSE_MATRICES if matrices else 0, stream)

    def render(self, cam, opts=None, out=None, stream=None):
        import torch
        c = cam if isinstance(cam, nr_camera) else make_camera(cam)
        if out is None:
            out = torch.empty(c.height, c.width, 4, device="cuda", dtype=torch.float32)
        nr_render(self.h, c, opts if opts is not None else make_opts(), out, stream)
        return out

    def query(self, x_obs, opts=None, stream=None):
        import torch
        out = torch.empty(x_obs.shape[0], NR_QUERY_STRIDE, device="cuda", dtype=torch.float32)
        nr_query(self.h, x_obs.contiguous(), opts if opts is not None else make_opts(), out, stream)
        return out

    def set_frames(self, axis_angle, root_t, cameras, stream=None):
        nr_set_frames(self.h, axis_angle, root_t, cameras, stream)

    def train_step(self, frame_id, px, py, target_rgb, n_samples: int, step_seed: int, lr: float = 1e-2,
                   betas=(0.9, 0.99), eps: float = 1e-8, bg=(0.0, 0.0, 0.0), hann_alpha: float = -1.0,
                   grad_only: bool = False, train_mask: int = 0, lr_scale=(0.0, 0.0, 0.0, 0.0),
                   loss_weight: float = 0.0, lr_scale_refiner: float = 0.0, lr_scale_cnn: float = 0.0,
                   pred_rgb=None, grad_rgb=None, forward_only: bool = False, stream=None) -> float:
        b = nr_train_batch()
        b.n_rays = int(frame_id.shape[0])
        b.frame_id = C.cast(C.c_void_p(frame_id.data_ptr()), _up)
        b.px = C.cast(C.c_void_p(px.data_ptr()), _up)
        b.py = C.cast(C.c_void_p(py.data_ptr()), _up)
        if target_rgb is not None:
            b.target_rgb = C.cast(C.c_void_p(target_rgb.data_ptr()), _fp)
        if pred_rgb is not None:
            b.pred_rgb = C.cast(C.c_void_p(pred_rgb.data_ptr()), _fp)
        if grad_rgb is not None:
            b.grad_rgb = C.cast(C.c_void_p(grad_rgb.data_ptr()), _fp)
        b.n_samples, b.step_seed = int(n_samples), int(step_seed)
        b.bg[:] = [float(v) for v in bg]
        b.lr, b.beta1, b.beta2, b.eps = float(lr), float(betas[0]), float(betas[1]), float(eps)
        b.hann_alpha, b.train_mask = float(hann_alpha), int(train_mask)
        b.flags = (NR_GRAD_ONLY if grad_only else 0) | (NR_FORWARD_ONLY if forward_only else 0)
        b.lr_scale[:] = [float(v) for v in lr_scale]
        b.loss_weight = float(loss_weight)
        b.lr_scale_refiner = float(lr_scale_refiner)
        b.lr_scale_cnn = float(lr_scale_cnn)
        return nr_train_step(self.h, b, stream)

    def param(self, which: int):
        return nr_param(self.h, which)

    def parameter_groups(self):
        """The trainable groups in use: weight volume (or CNN_skel), hash table, canonical
        MLP, residual MLP, and the pose refiner when one is installed."""
        groups = [NR_PARAM_WVOL, NR_PARAM_HASH, NR_PARAM_MLP, NR_PARAM_RES]
        if self.param(NR_PARAM_REFINER)[0].numel():
            groups.append(NR_PARAM_REFINER)
        if self.param(NR_PARAM_CNN)[0].numel():
            groups[0] = NR_PARAM_CNN
        return groups

    def parameters(self):
        """Zero-copy device tensors of the groups in use, marked requires_grad (leaf tensors
        for torch.autograd and torch.optim)."""
        return [self.param(g)[0].requires_grad_(True) for g in self.parameter_groups()]

    def parameter_grads(self):
        return [self.param(g)[1] for g in self.parameter_groups()]

    def params_changed(self):
        nr_params_changed(self.h)

    def pose_transforms(self):
        return nr_pose_transforms(self.h)

    def stage_times(self):
        return nr_stage_times(self.h)

    def occupancy(self):
        return nr_occupancy(self.h, self.occ_grid)

    def refresh_occupancy(self, sigma_threshold: float, dilate: int = 1, s_min: float = OCC_S_MIN, stream=None):
        nr_refresh_occupancy(self.h, sigma_threshold, dilate, s_min, stream)

    def set_canonical_occupancy(self, bits, s_min: float = OCC_S_MIN, stream=None):
        nr_set_canonical_occupancy(self.h, bits, s_min, stream)

    def set_pose_refiner(self, layers, stream=None):
        nr_set_pose_refiner(self.h, layers, stream)

    def set_weight_cnn(self, layers, z=None, log_prior=None, stream=None):
        nr_set_weight_cnn(self.h, layers, z, log_prior, stream)

    def canonical_occupancy(self):
        return nr_canonical_occupancy(self.h, self.occ_grid)

    def close(self):
        if getattr(self, "h", None) is not None:
            nr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderFn:
    """The training render as a torch.autograd.Function: colours of a batch of pixel rays
    (stratified samples, as in nr_train_step), differentiable in the subject's parameter
    groups through the library's hand-written backward.

        params = sub.parameters()               # zero-copy device tensors, requires_grad
        rgb = RenderFn.apply(sub, frame_id, px, py, n_samples, seed, *params)
        loss = any_function(rgb); loss.backward()    # params[i].grad filled by the library
        optimizer.step(); sub.params_changed()       # the library rebuilds its derived layouts

    The backward re-runs the batch's forward (same seed, so the same samples) and feeds
    dL/drgb into the compositing adjoint."""

    @staticmethod
    def apply(sub, frame_id, px, py, n_samples, seed, *params):
        return _render_fn().apply(sub, frame_id, px, py, n_samples, seed, *params)


def _render_fn():
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sub, frame_id, px, py, n_samples, seed, *params):
            pred = torch.empty(frame_id.shape[0], 3, device=frame_id.device, dtype=torch.float32)
            sub.train_step(frame_id, px, py, None, int(n_samples), int(seed), pred_rgb=pred, forward_only=True)
            ctx.sub, ctx.n_samples, ctx.seed, ctx.n_params = sub, int(n_samples), int(seed), len(params)
            ctx.save_for_backward(frame_id, px, py)
            return pred

        @staticmethod
        def backward(ctx, grad_pred):
            frame_id, px, py = ctx.saved_tensors
            sub = ctx.sub
            sub.train_step(frame_id, px, py, None, ctx.n_samples, ctx.seed,
                           grad_rgb=grad_pred.contiguous().float(), grad_only=True)
            grads = [g.clone() for g in sub.parameter_grads()[:ctx.n_params]]
            return (None, None, None, None, None, None) + tuple(grads)

    return _Fn


class Server:
    """The continuous-batching render server (nr_server_*)."""

    def __init__(self, max_bytes: int, max_slots: int, device: int = 0):
        self.h = C.c_void_p()
        check(lib.nr_server_create(device, int(max_bytes), int(max_slots), C.byref(self.h)), "nr_server_create")
        self.subjects = []

    def set_policy(self, order: int = NR_SERVE_EDF, age_ms: float = 40.0, deadline_ms: float = 20.0,
                   deadline_ms_per_mpixel: float = 5.0, priority_streams: bool = False) -> None:
        p = nr_server_policy(int(order), float(age_ms), float(deadline_ms), float(deadline_ms_per_mpixel),
                             int(bool(priority_streams)))
        check(lib.nr_server_set_policy(self.h, C.byref(p)), "nr_server_set_policy")

    def add_subject(self, subject: Subject) -> int:
        idx = C.c_uint32()
        check(lib.nr_server_add_subject(self.h, subject.h, C.byref(idx)), "nr_server_add_subject")
        self.subjects.append(subject)
        return int(idx.value)

    @staticmethod
    def request(subject: int, cam, axis_angle, root_t, opts, out) -> nr_request:
        r = nr_request()
        r.subject = int(subject)
        r.cam = cam if isinstance(cam, nr_camera) else make_camera(cam)
        r.axis_angle[:] = [float(v) for v in np.asarray(axis_angle, np.float32).ravel()]
        r.root_t[:] = [float(v) for v in np.asarray(root_t if root_t is not None else np.zeros(3), np.float32)]
        r.opts = opts
        r.out_rgba = out.data_ptr() if hasattr(out, "data_ptr") else int(out)
        return r

    def submit(self, req: nr_request) -> int:
        rid = C.c_uint64()
        check(lib.nr_server_submit(self.h, C.byref(req), C.byref(rid)), "nr_server_submit")
        return int(rid.value)

    def wait(self, rid: int, timeout_ms: int = 60000) -> float:
        lat = C.c_double()
        check(lib.nr_server_wait(self.h, rid, int(timeout_ms), C.byref(lat)), "nr_server_wait")
        return float(lat.value)

    def poll(self, rid: int):
        state, lat = C.c_int32(), C.c_double()
        check(lib.nr_server_poll(self.h, rid, C.byref(state), C.byref(lat)), "nr_server_poll")
        return int(state.value), float(lat.value)

    def stats(self) -> dict:
        st = nr_server_stats()
        check(lib.nr_server_get_stats(self.h, C.byref(st)), "nr_server_get_stats")
        return {k: getattr(st, k) for k, _ in nr_server_stats._fields_}

    def stop(self, timeout_ms: int = 60000) -> None:
        check(lib.nr_server_stop(self.h, int(timeout_ms)), "nr_server_stop")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            check(lib.nr_server_destroy(self.h), "nr_server_destroy")
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
