"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates inputs*: a 24-joint stick-figure skeleton, per-bone
poses, pinhole cameras, a canonical motion-weight volume, canonical occupancy
ellipsoids, hash-table and MLP initial values, training ray batches and serving
request streams.  It holds none of the rendering method's arithmetic (no
forward kinematics, no warp, no encoding, no compositing); both the CUDA path
and the FP64 oracle consume what it returns.

The paper trains and evaluates on ZJU-MoCap (Sec. 5.1: one performer of about
1.7 m, 1024x1024 frames, 128 samples per ray, Sec. 5.2).  That dataset is not
used; these seeded stand-ins reproduce its shapes: a human-proportioned
skeleton with SMPL topology (24 joints, Sec. 4.1), a 2 m bounding box around
the performer (Sec. 4.4), a 25-channel canonical weight volume (24 bones plus
background, supplementary Fig. S2) and cameras on a 2.5 m sphere.

Every generator takes an explicit seed and splits it per object with
``numpy.random.SeedSequence.spawn`` so that changing one object's draw never
moves another's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_BONES = 24
N_CHANNELS = N_BONES + 1          # 24 bones + background (Fig. S2)

# SMPL kinematic tree (parent of each joint; -1 for the pelvis root).
PARENTS = np.array([-1, 0, 0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 9, 9, 12, 13, 14,
                    16, 17, 18, 19, 20, 21], dtype=np.int32)

# Rest (= canonical) T-pose joint positions in metres, pelvis at the origin,
# y up, the performer facing +z.  About 1.73 m from sole to crown.
_REST_JOINTS = np.array([
    [0.00, 0.00, 0.00],    # 0 pelvis
    [0.09, -0.08, 0.00],   # 1 left hip
    [-0.09, -0.08, 0.00],  # 2 right hip
    [0.00, 0.11, 0.00],    # 3 spine 1
    [0.10, -0.48, 0.00],   # 4 left knee
    [-0.10, -0.48, 0.00],  # 5 right knee
    [0.00, 0.24, 0.00],    # 6 spine 2
    [0.10, -0.88, 0.00],   # 7 left ankle
    [-0.10, -0.88, 0.00],  # 8 right ankle
    [0.00, 0.30, 0.00],    # 9 spine 3
    [0.11, -0.93, 0.12],   # 10 left foot
    [-0.11, -0.93, 0.12],  # 11 right foot
    [0.00, 0.50, 0.00],    # 12 neck
    [0.08, 0.42, 0.00],    # 13 left collar
    [-0.08, 0.42, 0.00],   # 14 right collar
    [0.00, 0.62, 0.03],    # 15 head
    [0.18, 0.45, 0.00],    # 16 left shoulder
    [-0.18, 0.45, 0.00],   # 17 right shoulder
    [0.45, 0.45, 0.00],    # 18 left elbow
    [-0.45, 0.45, 0.00],   # 19 right elbow
    [0.70, 0.45, 0.00],    # 20 left wrist
    [-0.70, 0.45, 0.00],   # 21 right wrist
    [0.79, 0.45, 0.00],    # 22 left hand
    [-0.79, 0.45, 0.00],   # 23 right hand
], dtype=np.float64)

# Direction in which a leaf joint's body part extends (head up, hands out,
# feet forward); used only to place the synthetic blobs and ellipsoids.
_LEAF_EXTENT = {10: (0.0, -0.02, 0.08), 11: (0.0, -0.02, 0.08),
                15: (0.0, 0.16, 0.0), 22: (0.08, 0.0, 0.0), 23: (-0.08, 0.0, 0.0)}

BOX_MIN = np.array([-1.0, -1.0, -1.0])
BOX_MAX = np.array([1.0, 1.0, 1.0])

# Object streams split from one seed (see module docstring).
_STREAMS = ("skeleton", "pose", "volume", "hash", "mlp", "residual", "camera",
            "requests", "ellipsoid", "rays", "frames")


def _rngs(seed: int) -> dict:
    kids = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    return {k: np.random.default_rng(s) for k, s in zip(_STREAMS, kids)}


# --------------------------------------------------------------------------
# Skeleton, bones, poses
# --------------------------------------------------------------------------

def rest_joints(rng: np.random.Generator, jitter: float = 0.02) -> np.ndarray:
    """Seeded stick-figure rest joints: the template above plus U(-jitter, jitter)."""
    j = _REST_JOINTS + rng.uniform(-jitter, jitter, size=_REST_JOINTS.shape)
    j[0] = 0.0                                     # pelvis stays at the origin
    return j


def bone_segments(joints: np.ndarray) -> np.ndarray:
    """Segment [a, b] (2x3) of each bone's body part, in canonical space.

    Bone i spans joint i to the mean of its children, or a fixed extent for
    leaf joints.  Only the synthetic volume and ellipsoids use this.
    """
    seg = np.zeros((N_BONES, 2, 3))
    for i in range(N_BONES):
        kids = np.nonzero(PARENTS == i)[0]
        a = joints[i]
        b = joints[kids].mean(0) if len(kids) else a + np.array(_LEAF_EXTENT[i])
        seg[i, 0], seg[i, 1] = a, b
    return seg


def random_pose(rng: np.random.Generator, max_deg: float = 30.0,
                root_t_scale: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Per-bone axis-angle rotations: random unit axis, angle U(0, max_deg).

    Returns (axis_angle [24][3] float32, root translation [3] float32).
    """
    axis = rng.normal(size=(N_BONES, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(0.0, max_deg, size=(N_BONES, 1)))
    root_t = rng.uniform(-root_t_scale, root_t_scale, size=3)
    return (axis * ang).astype(np.float32), root_t.astype(np.float32)


# --------------------------------------------------------------------------
# Canonical motion-weight volume and occupancy ellipsoids
# --------------------------------------------------------------------------

def _dist_to_segments(pts: np.ndarray, seg: np.ndarray) -> np.ndarray:
    """Euclidean distance of each point to each segment: [n_pts][n_seg]."""
    a = seg[:, 0][None]                 # [1][S][3]
    ab = (seg[:, 1] - seg[:, 0])[None]
    ap = pts[:, None, :] - a
    h = np.clip((ap * ab).sum(-1) / np.maximum((ab * ab).sum(-1), 1e-12), 0, 1)
    return np.linalg.norm(ap - h[..., None] * ab, axis=-1)


def weight_volume(rng: np.random.Generator, joints: np.ndarray, res: int) -> np.ndarray:
    """Softmax of seeded Gaussian blobs around the bones: [25][res][res][res] float32.

    Channel i < 24 has logit -d(x, segment_i)^2 / (2 s_i^2) with s_i ~ U(4, 8) cm;
    the background channel has the constant logit -0.15^2 / (2 * 0.06^2).
    Vertex (ix, iy, iz) sits at box_min + (ix, iy, iz) * 2 m / (res - 1) and the
    array is indexed [channel][iz][iy][ix].
    """
    seg = bone_segments(joints)
    s = rng.uniform(0.04, 0.08, size=N_BONES)
    g = np.linspace(BOX_MIN[0], BOX_MAX[0], res)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], -1)
    out = np.empty((N_CHANNELS, res ** 3), dtype=np.float64)
    chunk = 65536
    bg_logit = -(0.15 ** 2) / (2 * 0.06 ** 2)
    for c0 in range(0, pts.shape[0], chunk):
        d = _dist_to_segments(pts[c0:c0 + chunk], seg)
        logit = np.concatenate([-(d ** 2) / (2 * s ** 2),
                                np.full((d.shape[0], 1), bg_logit)], 1)
        logit -= logit.max(1, keepdims=True)
        e = np.exp(logit)
        out[:, c0:c0 + chunk] = (e / e.sum(1, keepdims=True)).T
    return out.reshape(N_CHANNELS, res, res, res).astype(np.float32)


ELLIPSOID_FLOATS = 15   # centre[3], rotation rows[9] (canonical -> local), radii[3]


def ellipsoids(rng: np.random.Generator, joints: np.ndarray,
               target_frac: float = 0.15, grid: int = 40) -> np.ndarray:
    """One canonical ellipsoid per bone segment, inflated until ~target_frac of
    the box is covered at the rest pose (measured on a coarse grid).

    Layout per bone: centre (3), the 3x3 rotation whose rows are the local
    axes (canonical -> local), radii (3).  float32 [24][15].
    """
    seg = bone_segments(joints)
    cen = seg.mean(1)
    ax = seg[:, 1] - seg[:, 0]
    half = np.linalg.norm(ax, axis=1) / 2
    e0 = ax / np.maximum(2 * half[:, None], 1e-9)
    rot = np.zeros((N_BONES, 3, 3))
    for i in range(N_BONES):
        helper = np.array([0.0, 0.0, 1.0]) if abs(e0[i, 2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        e1 = np.cross(e0[i], helper)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(e0[i], e1)
        rot[i] = np.stack([e0[i], e1, e2])
    thick = rng.uniform(0.8, 1.2, size=N_BONES)
    g = (np.arange(grid) + 0.5) / grid * 2 - 1
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], -1)

    def radii(scale):
        r = np.stack([half + scale * thick, scale * thick, scale * thick], 1)
        return r

    def frac(scale):
        r = radii(scale)
        inside = np.zeros(pts.shape[0], bool)
        for i in range(N_BONES):
            loc = (pts - cen[i]) @ rot[i].T
            inside |= ((loc / r[i]) ** 2).sum(1) <= 1.0
        return inside.mean()

    lo, hi = 0.01, 0.6
    for _ in range(16):                 # bisection on the tube radius
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if frac(mid) < target_frac else (lo, mid)
    r = radii(0.5 * (lo + hi))
    out = np.concatenate([cen, rot.reshape(N_BONES, 9), r], 1)
    return out.astype(np.float32)


# --------------------------------------------------------------------------
# Hash grid and MLP initial values
# --------------------------------------------------------------------------

def level_resolutions(n_levels: int, n_min: int, n_max: int) -> list[int]:
    """Per-level grid resolution N_l = floor(N_min * b^l), b = (N_max/N_min)^(1/(L-1)).

    This is the growth rule of the multiresolution hash encoding (Mueller et
    al. 2022, cited by the paper in Sec. 2.3); it is a configuration value,
    computed once in FP64 and handed to both sides as integers.
    """
    if n_levels == 1:
        return [n_min]
    b = math.exp((math.log(n_max) - math.log(n_min)) / (n_levels - 1))
    return [int(math.floor(n_min * b ** l + 1e-9)) for l in range(n_levels)]


def hash_entries(rng: np.random.Generator, n_levels: int, log2_t: int, n_feat: int = 2,
                 scale: float = 1e-4, dtype=np.float32) -> np.ndarray:
    """Table entries U(-scale, scale): [L][T][F], stored values already in `dtype`."""
    t = rng.uniform(-scale, scale, size=(n_levels, 1 << log2_t, n_feat))
    return t.astype(dtype).astype(np.float32)


def kaiming_layers(rng: np.random.Generator, dims: list[tuple[int, int]],
                   zero_last: bool = False, last_std: float | None = None) -> list[tuple[np.ndarray, np.ndarray]]:
    """Kaiming-normal weights (std sqrt(2 / fan_in)) and zero biases per (in, out) layer."""
    out = []
    for li, (fi, fo) in enumerate(dims):
        std = math.sqrt(2.0 / fi)
        if li == len(dims) - 1 and last_std is not None:
            std = last_std
        w = rng.normal(0.0, std, size=(fo, fi))
        if zero_last and li == len(dims) - 1:
            w[:] = 0.0
        out.append((w.astype(np.float32), np.zeros(fo, np.float32)))
    return out


def pack_layers(layers) -> np.ndarray:
    """Concatenate W (row-major [out][in]) then b for each layer, float32."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers]).astype(np.float32)


def canonical_dims(mlp_in: int, width: int, hidden_layers: int) -> list[tuple[int, int]]:
    """(in, out) of each canonical-MLP layer: in->w, (hidden-1) x w->w, w->4."""
    return [(mlp_in, width)] + [(width, width)] * (hidden_layers - 1) + [(width, 4)]


RES_POSE_DIM = N_BONES * 3


def residual_dims(pe_freqs: int, width: int = 64) -> list[tuple[int, int]]:
    """(in, out) of each residual-MLP layer.

    Layer 1 sees [gamma(x_skel) (3 + 6 * pe_freqs), Omega (72)]; layer 4 sees
    [h3, gamma(x_skel)] (the skip connection of Fig. S3); layer 5 emits x_res.
    """
    g = 3 + 6 * pe_freqs
    return [(g + RES_POSE_DIM, width), (width, width), (width, width),
            (width + g, width), (width, 3)]


# --------------------------------------------------------------------------
# Cameras and rays
# --------------------------------------------------------------------------

@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # [3][3] world -> camera (OpenCV: x right, y down, z forward)
    t: np.ndarray          # [3]
    t_near: float
    t_far: float
    n_samples: int
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """World->camera (R, t) of an OpenCV camera at `eye` looking at `target`."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    dn = np.cross(f, r)
    R = np.stack([r, dn, f])
    return R.astype(np.float32), (-R @ eye).astype(np.float32)


def camera(width: int, height: int, focal: float, eye, n_samples: int,
           t_near: float, t_far: float, bg=(0.0, 0.0, 0.0)) -> Camera:
    R, t = look_at(eye)
    return Camera(width, height, float(focal), float(focal), width / 2.0, height / 2.0,
                  R, t, float(t_near), float(t_far), int(n_samples), np.asarray(bg, np.float32))


def random_eye(rng: np.random.Generator, radius: float = 2.5, max_elev_deg: float = 30.0) -> np.ndarray:
    az = rng.uniform(0, 2 * math.pi)
    el = math.radians(rng.uniform(-max_elev_deg, max_elev_deg))
    return radius * np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])


# --------------------------------------------------------------------------
# Workload configurations (the five workloads: tiny, single frame, training,
# precision sweep, multi-subject serving)
# --------------------------------------------------------------------------

def subject(seed: int, *, vol_res: int = 32, hash_levels: int = 8, log2_t: int = 14,
            n_min: int = 16, n_max: int = 256, table_dtype=np.float32, hash_scale: float = 1e-4,
            hidden_layers: int = 2, mlp_in: int = 32, width: int = 64, res_freqs: int = 6,
            res_last_std: float | None = None, with_ellipsoids: bool = False) -> dict:
    """All per-subject arrays for one seeded synthetic performer."""
    r = _rngs(seed)
    joints = rest_joints(r["skeleton"])
    levels = level_resolutions(hash_levels, n_min, n_max)
    canon = kaiming_layers(r["mlp"], canonical_dims(mlp_in, width, hidden_layers))
    res = kaiming_layers(r["residual"], residual_dims(res_freqs, width),
                         zero_last=res_last_std is None, last_std=res_last_std)
    d = dict(
        parents=PARENTS.copy(), rest_joints=joints.astype(np.float32),
        box_min=BOX_MIN.astype(np.float32), box_max=BOX_MAX.astype(np.float32),
        wvol=weight_volume(r["volume"], joints, vol_res), wvol_res=vol_res,
        hash_levels=hash_levels, hash_feats=2, log2_T=log2_t, level_res=np.array(levels, np.uint32),
        table_dtype=np.dtype(table_dtype).name,
        hash_table=hash_entries(r["hash"], hash_levels, log2_t, 2, hash_scale, table_dtype),
        mlp_in=mlp_in, mlp_width=width, mlp_hidden_layers=hidden_layers,
        mlp_layers=canon, mlp_params=pack_layers(canon),
        res_enabled=1, res_pe_freqs=res_freqs, res_layers=res, res_params=pack_layers(res),
        seed=seed,
    )
    if with_ellipsoids:
        d["ellipsoids"] = ellipsoids(r["ellipsoid"], joints)
    return d


def refiner_dims(width: int = 256, hidden_layers: int = 4) -> list[tuple[int, int]]:
    """(in, out) of each pose-refiner layer: 3(K-1) joint angles -> width x hidden -> 3(K-1)."""
    n = 3 * (N_BONES - 1)
    return [(n, width)] + [(width, width)] * (hidden_layers - 1) + [(width, n)]


def refiner_layers(seed: int, width: int = 256, hidden_layers: int = 4, last_std: float = 1e-5):
    """Seeded MLP_theta weights: Kaiming hidden layers, a near-zero output layer (the
    refined pose starts at the estimate)."""
    rng = np.random.default_rng(seed)
    return kaiming_layers(rng, refiner_dims(width, hidden_layers), last_std=last_std)


def cnn_layers(seed: int, channels=(1024, 512, 256, 128, 64), last_std: float = 1e-2):
    """Seeded CNN_skel weights: the fully-connected layer and five transposed convolutions
    (He-normal over each output's fan-in: 256, and C_in x 8 taps), zero biases; a small last
    layer so that the generated volume starts near softmax(log prior)."""
    rng = np.random.default_rng(seed)
    out = [((rng.normal(0.0, math.sqrt(2.0 / 256), size=(channels[0], 256))).astype(np.float32),
            np.zeros(channels[0], np.float32))]
    ins = list(channels)
    outs = list(channels[1:]) + [N_BONES + 1]
    for k, (ci, co) in enumerate(zip(ins, outs)):
        std = last_std if k == 4 else math.sqrt(2.0 / (ci * 8))
        out.append((rng.normal(0.0, std, size=(ci, co, 4, 4, 4)).astype(np.float32), np.zeros(co, np.float32)))
    return out


def cnn_latent(seed: int) -> np.ndarray:
    """The constant random latent z [256] of CNN_skel."""
    return np.random.default_rng(seed).normal(size=256).astype(np.float32)


def shaped_density(subj: dict, beta: float = 8.0, bias: float = -4.0, keep_ellipsoids: bool = False) -> dict:
    """A copy of `subj` (made with ellipsoids) whose canonical density follows the performer's body.

    The finest dense hash level holds, in feature 0, f(v) = clip(1 - min_i q_i(v), -1, 1) at each
    vertex v, q_i the normalised squared radius of v in canonical ellipsoid i (positive inside
    the body, negative away from it).  The canonical MLP is rewired so that hidden units 0 and 1
    carry relu(f) and relu(-f) through every layer and o_3 = beta (relu(f) - relu(-f)) + bias =
    beta f + bias: sigma = softplus(beta f + bias) is ~softplus(beta + bias) inside the body and
    ~softplus(-beta + bias) away from it.  Colour keeps the random weights on the other units.
    """
    d = dict(subj)
    levels = [int(n) for n in d["level_res"]]
    T = 1 << int(d["log2_T"])
    dense = [l for l, n in enumerate(levels) if (n + 1) ** 3 <= T]
    lv = dense[-1]
    n = levels[lv]
    iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    bmin, bmax = np.asarray(d["box_min"], np.float64), np.asarray(d["box_max"], np.float64)
    v = bmin + np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) / n * (bmax - bmin)
    E = np.asarray(subj["ellipsoids"], np.float64)
    q = np.full(v.shape[0], np.inf)
    for e in E:
        loc = (v - e[:3]) @ e[3:12].reshape(3, 3).T / e[12:15]
        q = np.minimum(q, (loc ** 2).sum(1))
    f = np.clip(1.0 - q, -1.0, 1.0)
    tab = np.array(d["hash_table"], np.float32, copy=True)
    idx = ix.ravel() + iy.ravel() * (n + 1) + iz.ravel() * (n + 1) ** 2
    tab[lv, idx, 0] = f.astype(np.float32)
    d["hash_table"] = tab
    layers = [(np.array(W, np.float32, copy=True), np.array(b, np.float32, copy=True)) for W, b in d["mlp_layers"]]
    k = 2 * lv
    W, b = layers[0]
    W[0:2, :] = 0.0
    W[0, k], W[1, k] = 1.0, -1.0
    b[0:2] = 0.0
    for W, b in layers[1:-1]:
        W[0:2, :] = 0.0
        W[:, 0:2] = 0.0
        W[0, 0] = W[1, 1] = 1.0
        b[0:2] = 0.0
    W, b = layers[-1]
    W[:, 0:2] = 0.0
    W[3, :] = 0.0
    W[3, 0], W[3, 1] = beta, -beta
    b[3] = bias
    d["mlp_layers"] = layers
    d["mlp_params"] = pack_layers(layers)
    if not keep_ellipsoids:
        d.pop("ellipsoids", None)
    return d


def config_tiny(seed: int = 1234) -> dict:
    """64x64 image, fx=fy=80, 32 samples in [1.5, 3.5] m, no occupancy skip,
    32^3x25 volume, 8x2 hash levels of 2^14 entries (N 16..256), MLP 32-64-64-4, FP32."""
    subj = subject(seed)
    r = _rngs(seed)
    pose = random_pose(r["pose"])
    cam = camera(64, 64, 80.0, (0.0, 0.0, 2.5), 32, 1.5, 3.5)
    return dict(name="tiny_64x64_s32_fp32", subject=subj, pose=pose, camera=cam,
                use_occupancy=False)


def config_frame512(seed: int = 1235, structured: bool = False) -> dict:
    """512x512, 128 samples, occupancy 128^3 (~15 % set), 16x2 levels of 2^19 FP16 entries
    (N 16..2048), MLP 32-64-64-64-4 in BF16, 64^3x25 FP32 volume."""
    subj = subject(seed, vol_res=64, hash_levels=16, log2_t=19, n_max=2048, table_dtype=np.float16,
                   hidden_layers=3, hash_scale=(0.5 if structured else 1e-4), with_ellipsoids=True)
    r = _rngs(seed)
    pose = random_pose(r["pose"])
    cam = camera(512, 512, 640.0, (0.0, 0.0, 2.5), 128, 0.5, 4.5)
    return dict(name="frame_512x512_s128_occ_bf16", subject=subj, pose=pose, camera=cam,
                use_occupancy=True)


def config_sweep(seed: int = 1237) -> dict:
    """1920x1080, 192 samples, tiny-config field with 2^20 entries per level."""
    subj = subject(seed, log2_t=20, with_ellipsoids=True)
    r = _rngs(seed)
    pose = random_pose(r["pose"])
    cam = camera(1920, 1080, 1.25 * 1080, (0.0, 0.0, 2.5), 192, 0.5, 4.5)
    return dict(name="sweep_1920x1080_s192", subject=subj, pose=pose, camera=cam,
                use_occupancy=True)


def sweep_variants() -> tuple:
    """The precision sweep's inputs: the 1920x1080 x 192 workload and its two fields, the
    workload's own subject and a textured one (2^20 entries per level), both with hash entries
    rounded to f16 so that the f16 table tier stores them exactly."""
    cfg = config_sweep()
    out = []
    for name, subj in (("as_configured", cfg["subject"]),
                       ("textured", subject(1237, log2_t=20, hash_scale=0.5, res_last_std=0.02))):
        subj = dict(subj)
        subj["hash_table"] = subj["hash_table"].astype(np.float16).astype(np.float32)
        out.append((name, subj))
    return cfg, out


def sweep_pixels(width: int, height: int, n: int = 384, seed: int = 11) -> tuple:
    """The seeded pixels at which the precision sweep compares each tier with the oracle."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, width, n), rng.integers(0, height, n)


def training_frames(seed: int, n_frames: int = 16, res: int = 512) -> dict:
    """Seeded poses (<= 30 deg per bone) and cameras on the 2.5 m sphere for n frames."""
    r = _rngs(seed)
    poses = [random_pose(r["frames"]) for _ in range(n_frames)]
    cams = [camera(res, res, 1.25 * res, random_eye(r["camera"]), 128, 0.5, 4.5)
            for _ in range(n_frames)]
    return dict(axis_angle=np.stack([p[0] for p in poses]),
                root_t=np.stack([p[1] for p in poses]), cameras=cams)


def pixel_batch(seed: int, n_rays: int, n_frames: int, width: int, height: int) -> dict:
    """Uniformly drawn (frame, pixel) pairs for one training batch."""
    rng = np.random.default_rng(seed)
    return dict(frame=rng.integers(0, n_frames, n_rays).astype(np.uint32),
                px=rng.integers(0, width, n_rays).astype(np.uint32),
                py=rng.integers(0, height, n_rays).astype(np.uint32))


def patch_batch(seed: int, frames, n_images: int, n_patches: int = 6, size: int = 20,
                width: int = 512, height: int = 512) -> dict:
    """Patch-based ray batch (Sec. 5.2: 6 patches of 20 x 20 pixels per image): n_images frames
    drawn from `frames` (a count), each contributing n_patches square patches at random positions."""
    rng = np.random.default_rng(seed)
    fr, px, py = [], [], []
    yy, xx = np.meshgrid(np.arange(size), np.arange(size), indexing="ij")
    for f in rng.integers(0, frames, n_images):
        for _ in range(n_patches):
            x0 = int(rng.integers(0, width - size + 1))
            y0 = int(rng.integers(0, height - size + 1))
            fr.append(np.full(size * size, f))
            px.append((x0 + xx).ravel())
            py.append((y0 + yy).ravel())
    return dict(frame=np.concatenate(fr).astype(np.uint32), px=np.concatenate(px).astype(np.uint32),
                py=np.concatenate(py).astype(np.uint32))


def request_stream(seed: int, n_subjects: int, rate_hz: float, duration_s: float,
                   resolutions=(256, 512, 1024), probs=(0.3, 0.5, 0.2)) -> list[dict]:
    """Poisson arrivals with a random subject, camera on the 2.5 m sphere, fresh pose
    (<= 30 deg per bone) and a resolution drawn from `resolutions` with `probs`."""
    r = _rngs(seed)
    g = r["requests"]
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        res = int(g.choice(resolutions, p=probs))
        aa, rt = random_pose(g)
        out.append(dict(t_arrive=t, subject=int(g.integers(n_subjects)),
                        camera=camera(res, res, 1.25 * res, random_eye(g), 128, 0.5, 4.5),
                        axis_angle=aa, root_t=rt))
    return out
