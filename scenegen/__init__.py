"""Seeded synthetic inputs shaped like the paper's neural animals.

This module is shared by the oracle (``oracle/``) and the CUDA path
(``paper_2202_05628_gb300``).  It holds only input generation: a procedural
quadruped (union of capsules), its band voxelisation into the leaf voxels of a
canonical octree, skinning weights from a Gaussian bone falloff, features and
densities, a walk cycle and random poses, orbit cameras and shading-network
weights.  It contains none of the rendering method's arithmetic (no skinning,
no ray/voxel intersection, no compositing, no convolution).

The paper's Dynamic Furry Animal dataset (Sec. 6, "Dynamic Furry Animal
Dataset") and its trained feature tables are not available; these scenes stand
in for them with the same shapes: small quadrupeds with a 24-joint rig, a
feature look-up table of C channels per leaf voxel (Sec. 3.1, "Octree Feature
Indexing"), walk motions and megapixel views.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

__all__ = [
    "Skeleton", "Octree", "Pose", "Camera", "Scene",
    "quadruped_skeleton", "make_octree", "random_pose", "walk_pose",
    "rest_pose", "orbit_camera", "tiny_net_weights", "unet_weights",
    "UNET_CHANNELS", "unet_layer_shapes", "two_branch_weights", "ALPHA_CHANNELS", "preset", "PRESETS",
]

J_JOINTS = 24


@dataclasses.dataclass
class Skeleton:
    """Tree skeleton: ``parent[j] < j`` (root has -1); ``rest[j]`` is the joint
    position in the canonical (rest) pose, in metres.  Canonical joint
    rotations are zero, so M^c_j = [I | rest[j]] (Eq. 4)."""
    parent: np.ndarray  # int32 [J]
    rest: np.ndarray    # float32 [J,3]

    @property
    def J(self) -> int:
        return int(self.parent.shape[0])


@dataclasses.dataclass
class Octree:
    """Leaf voxels of the canonical octree at a uniform depth.

    Voxel i covers the cube origin + (ijk[i] + [0,1]^3) * h with
    h = extent / 2**depth.  ``features`` is the FLUT (Sec. 3.1) in FP32,
    ``density`` the per-voxel sigma in 1/m."""
    depth: int
    origin: np.ndarray      # float32 [3]
    extent: float
    ijk: np.ndarray         # uint16 [N,3]
    joint_idx: np.ndarray   # uint8 [N,4]
    weights: np.ndarray     # float32 [N,4], rows sum to 1
    features: np.ndarray    # float32 [N,C]
    density: np.ndarray     # float32 [N]
    sdf: np.ndarray         # float32 [N] (generator bookkeeping only)

    @property
    def n(self) -> int:
        return int(self.ijk.shape[0])

    @property
    def C(self) -> int:
        return int(self.features.shape[1])

    @property
    def h(self) -> float:
        return float(self.extent) / float(1 << self.depth)

    def centers(self) -> np.ndarray:
        """Canonical voxel centres (FP64), origin + (ijk + 1/2) h."""
        return self.origin.astype(np.float64) + (self.ijk.astype(np.float64) + 0.5) * self.h

    def subset(self, idx: np.ndarray) -> "Octree":
        idx = np.asarray(idx)
        return Octree(self.depth, self.origin.copy(), self.extent, self.ijk[idx].copy(),
                      self.joint_idx[idx].copy(), self.weights[idx].copy(),
                      self.features[idx].copy(), self.density[idx].copy(), self.sdf[idx].copy())


@dataclasses.dataclass
class Pose:
    """Skeleton parameters S = {r, R, T} (Sec. 3.1, "Rigging and
    Deformation"): per-joint axis-angle r [J,3], global axis-angle R [3] and
    global translation T [3]."""
    axis_angle: np.ndarray  # float32 [J,3]
    R: np.ndarray           # float32 [3]
    T: np.ndarray           # float32 [3]


@dataclasses.dataclass
class Camera:
    """Pinhole camera.  Camera frame: +x right, +y down, +z forward.
    ``world_to_cam`` is the 3x4 [R | t] with x_cam = R x_world + t.  Pixel
    (x, y) is sampled at its centre (x + 1/2, y + 1/2).  ``near``/``far`` are
    distances along the unit-length ray."""
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # float32 [3,4]
    near: float
    far: float

    def __post_init__(self):
        # The library takes the intrinsics as FP32: they are kept at their
        # FP32 rounding, so that any consumer (the FP64 oracle included) sees
        # exactly the camera the library renders.  (orbit_camera's matrix is
        # FP32 already; hand-made FP64 matrices stay exact for closed forms.)
        for k in ("fx", "fy", "cx", "cy"):
            setattr(self, k, float(np.float32(getattr(self, k))))


@dataclasses.dataclass
class Scene:
    octree: Octree
    skeleton: Skeleton
    centroid: np.ndarray     # canonical voxel centroid (camera target)
    scale: float             # template scale chosen to hit the voxel count
    bones: np.ndarray        # [J,2,3] bone segments used for skin weights
    capsules: List[Tuple[np.ndarray, np.ndarray, float]]


# ---------------------------------------------------------------------------
# Procedural quadruped
# ---------------------------------------------------------------------------

# 24 joints: root, spine x3, neck x2, head, 4 legs x 4, tail.  Body along +x,
# up +y, lateral +z.  Template units are metres before scaling.
_JOINTS = [
    ("root", -1, (-0.100, 0.200, 0.000)),
    ("spine1", 0, (-0.040, 0.205, 0.000)),
    ("spine2", 1, (0.020, 0.210, 0.000)),
    ("spine3", 2, (0.080, 0.210, 0.000)),
    ("neck1", 3, (0.110, 0.240, 0.000)),
    ("neck2", 4, (0.130, 0.270, 0.000)),
    ("head", 5, (0.160, 0.290, 0.000)),
    ("fl_shoulder", 3, (0.080, 0.180, 0.045)),
    ("fl_elbow", 7, (0.085, 0.110, 0.045)),
    ("fl_wrist", 8, (0.080, 0.040, 0.045)),
    ("fl_paw", 9, (0.095, 0.012, 0.045)),
    ("fr_shoulder", 3, (0.080, 0.180, -0.045)),
    ("fr_elbow", 11, (0.085, 0.110, -0.045)),
    ("fr_wrist", 12, (0.080, 0.040, -0.045)),
    ("fr_paw", 13, (0.095, 0.012, -0.045)),
    ("hl_hip", 0, (-0.100, 0.180, 0.045)),
    ("hl_knee", 15, (-0.085, 0.110, 0.045)),
    ("hl_ankle", 16, (-0.105, 0.045, 0.045)),
    ("hl_paw", 17, (-0.090, 0.012, 0.045)),
    ("hr_hip", 0, (-0.100, 0.180, -0.045)),
    ("hr_knee", 19, (-0.085, 0.110, -0.045)),
    ("hr_ankle", 20, (-0.105, 0.045, -0.045)),
    ("hr_paw", 21, (-0.090, 0.012, -0.045)),
    ("tail", 0, (-0.140, 0.220, 0.000)),
]
_HEAD_TIP = (0.215, 0.280, 0.000)
_TAIL_TIP = (-0.230, 0.265, 0.000)
_PAW_TIP = (0.022, 0.0, 0.0)

# Capsules (joint or tip index pairs, radius in template metres).  The radii
# are thin so that, once the 3 cm band is added around them, the voxel budget
# of each preset yields an animal about 0.3 m long (cat-sized).
_RADIUS_SCALE = 0.3
_CAPSULES = [(a, b, r * _RADIUS_SCALE) for a, b, r in [
    (0, 1, 0.056), (1, 2, 0.060), (2, 3, 0.057),          # torso
    (3, 5, 0.036), (5, 6, 0.031), (6, "head_tip", 0.042),  # neck, head
    (7, 8, 0.024), (8, 9, 0.019), (9, 10, 0.016),          # front left
    (11, 12, 0.024), (12, 13, 0.019), (13, 14, 0.016),     # front right
    (15, 16, 0.026), (16, 17, 0.020), (17, 18, 0.016),     # hind left
    (19, 20, 0.026), (20, 21, 0.020), (21, 22, 0.016),     # hind right
    (0, 23, 0.028), (23, "tail_tip", 0.016),               # tail
    (10, "paw10", 0.014), (14, "paw14", 0.014), (18, "paw18", 0.014), (22, "paw22", 0.014),
]]


def _template() -> Tuple[np.ndarray, np.ndarray, dict]:
    parent = np.array([p for _, p, _ in _JOINTS], dtype=np.int32)
    pos = np.array([q for _, _, q in _JOINTS], dtype=np.float64)
    tips = {"head_tip": np.array(_HEAD_TIP), "tail_tip": np.array(_TAIL_TIP)}
    for paw in (10, 14, 18, 22):
        tips[f"paw{paw}"] = pos[paw] + np.array(_PAW_TIP)
    return parent, pos, tips


def quadruped_skeleton(scale: float = 1.0, center: Optional[np.ndarray] = None) -> Tuple[Skeleton, list, np.ndarray]:
    """Scaled quadruped: returns the skeleton, capsule list and bone segments.

    The template is scaled uniformly about its bounding-box centre and placed
    with that centre at ``center`` (default: the origin)."""
    parent, pos, tips = _template()
    allpts = np.concatenate([pos, np.stack(list(tips.values()))], 0)
    bb_c = 0.5 * (allpts.min(0) + allpts.max(0))
    c = np.zeros(3) if center is None else np.asarray(center, np.float64)

    def tf(p):
        return (np.asarray(p, np.float64) - bb_c) * scale + c

    jpos = tf(pos)
    caps = []
    for a, b, r in _CAPSULES:
        pa = jpos[a] if isinstance(a, int) else tf(tips[a])
        pb = jpos[b] if isinstance(b, int) else tf(tips[b])
        caps.append((pa, pb, r * scale))
    # Bone segment of joint j: from the joint to the mean of its children (or
    # to its tip for leaves).
    bones = np.zeros((len(parent), 2, 3))
    for j in range(len(parent)):
        kids = [k for k in range(len(parent)) if parent[k] == j]
        if kids:
            end = jpos[kids].mean(0)
        elif j == 6:
            end = tf(tips["head_tip"])
        elif j == 23:
            end = tf(tips["tail_tip"])
        else:
            end = tf(tips[f"paw{j}"])
        bones[j, 0] = jpos[j]
        bones[j, 1] = end
    sk = Skeleton(parent=parent.copy(), rest=jpos.astype(np.float32))
    return sk, caps, bones


def _seg_dist(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    ab = b - a
    L2 = float(ab @ ab)
    ap = p - a
    t = np.clip((ap @ ab) / L2, 0.0, 1.0) if L2 > 0 else np.zeros(p.shape[0])
    q = ap - t[:, None] * ab
    return np.sqrt(np.einsum("ij,ij->i", q, q))


def _sdf(p: np.ndarray, caps) -> np.ndarray:
    d = np.full(p.shape[0], np.inf)
    for a, b, r in caps:
        np.minimum(d, _seg_dist(p, a, b) - r, out=d)
    return d


def _band_voxels(caps, depth: int, origin: np.ndarray, extent: float, band: Tuple[float, float]):
    """All voxel indices whose centre sdf lies in [band[0], band[1]].

    Hierarchical: cells of 8^3 voxels are kept when the 1-Lipschitz sdf at the
    cell centre allows a band voxel inside the cell."""
    h = extent / (1 << depth)
    coarse = max(depth - 3, 0)
    f = 1 << (depth - coarse)
    hc = extent / (1 << coarse)
    nc = 1 << coarse
    g = (np.arange(nc) + 0.5) * hc
    cc = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + origin
    d = _sdf(cc, caps)
    half_diag = 0.5 * math.sqrt(3.0) * hc
    keep = (d + half_diag >= band[0]) & (d - half_diag <= band[1])
    cells = np.argwhere(keep.reshape(nc, nc, nc))
    if len(cells) == 0:
        return np.zeros((0, 3), np.int64), np.zeros(0)
    sub = np.stack(np.meshgrid(np.arange(f), np.arange(f), np.arange(f), indexing="ij"), -1).reshape(-1, 3)
    out_ijk, out_sdf = [], []
    chunk = max(1, 400000 // len(sub))
    for s in range(0, len(cells), chunk):
        ijk = (cells[s:s + chunk, None, :] * f + sub[None]).reshape(-1, 3)
        p = origin + (ijk + 0.5) * h
        dd = _sdf(p, caps)
        m = (dd >= band[0]) & (dd <= band[1])
        out_ijk.append(ijk[m])
        out_sdf.append(dd[m])
    ijk = np.concatenate(out_ijk)
    sd = np.concatenate(out_sdf)
    order = np.lexsort((ijk[:, 2], ijk[:, 1], ijk[:, 0]))
    return ijk[order], sd[order]


def _skin_weights(p: np.ndarray, bones: np.ndarray, sigma: float = 0.05, topk: int = 4):
    """Gaussian falloff of the distance to each bone, top-k kept, normalised.

    (Stands in for the paper's mesh-derived weights of Eq. 3, which need a
    skinned CGI mesh that is not available.)"""
    J = bones.shape[0]
    d = np.stack([_seg_dist(p, bones[j, 0], bones[j, 1]) for j in range(J)], 1)
    # Rank by distance (equivalent to ranking the Gaussian weight, without
    # underflow); ties broken by joint index.
    idx = np.argsort(d, axis=1, kind="stable")[:, :topk]
    dk = np.take_along_axis(d, idx, 1)
    w = np.exp(-0.5 * (dk - dk[:, :1]) * (dk + dk[:, :1]) / sigma ** 2)
    w = w / w.sum(1, keepdims=True)
    w32 = w.astype(np.float32)
    # Renormalise in FP32 so that each row sums to 1 within one ulp.
    w32 /= w32.sum(1, keepdims=True)
    return idx.astype(np.uint8), w32


def make_octree(depth: int, target: int, C: int, band: Tuple[float, float], seed: int,
                fur_shell: bool = False, extent: float = 1.0, tol: float = 0.05) -> Scene:
    """Band-voxelise the quadruped at ``depth`` with about ``target`` voxels.

    The template scale is found by a secant search on log(count) vs
    log(scale) (count grows with surface area, i.e. scale^2).  Features are
    N(0, 0.5^2); density is softplus(N(0,1)) * 20 / m, times
    exp(-max(sdf,0)/l) with l = 2 cm / ln 100 for the fur-like outer shell."""
    origin = np.full(3, -0.5 * extent)
    s = 1.0
    # Coarse search at depth <= 8 (count ~ band volume / h^3), then refine at
    # the full depth.
    d0 = min(depth, 8)
    t0 = target / float(8 ** (depth - d0))
    for _ in range(8):
        _, caps, _ = quadruped_skeleton(s)
        n0 = len(_band_voxels(caps, d0, origin, extent, band)[0])
        if n0 == 0 or abs(n0 - t0) <= 0.01 * t0:
            break
        s *= math.sqrt(t0 / n0)
    best = None
    for _ in range(6):
        sk, caps, bones = quadruped_skeleton(s)
        ijk, sd = _band_voxels(caps, depth, origin, extent, band)
        n = len(ijk)
        if best is None or abs(n - target) < abs(best[0] - target):
            best = (n, s, sk, caps, bones, ijk, sd)
        if abs(n - target) <= tol * 0.5 * target or n == 0:
            break
        s *= math.sqrt(target / max(n, 1))
    n, s, sk, caps, bones, ijk, sd = best
    rng = np.random.default_rng(seed)
    h = extent / (1 << depth)
    centers = origin + (ijk + 0.5) * h
    jidx, w = _skin_weights(centers, bones)
    feats = (0.5 * rng.standard_normal((n, C))).astype(np.float32)
    z = rng.standard_normal(n)
    dens = np.logaddexp(0.0, z) * 20.0
    if fur_shell:
        ell = 0.02 / math.log(100.0)
        dens = dens * np.exp(-np.maximum(sd, 0.0) / ell)
    oc = Octree(depth=depth, origin=origin.astype(np.float32), extent=float(extent),
                ijk=ijk.astype(np.uint16), joint_idx=jidx, weights=w, features=feats,
                density=dens.astype(np.float32), sdf=sd.astype(np.float32))
    return Scene(octree=oc, skeleton=sk, centroid=centers.mean(0), scale=s, bones=bones, capsules=caps)


# ---------------------------------------------------------------------------
# Poses and cameras
# ---------------------------------------------------------------------------

def rest_pose(J: int = J_JOINTS) -> Pose:
    return Pose(np.zeros((J, 3), np.float32), np.zeros(3, np.float32), np.zeros(3, np.float32))


def random_pose(seed: int, J: int = J_JOINTS, max_deg: float = 30.0,
                R: Optional[np.ndarray] = None, T: Optional[np.ndarray] = None) -> Pose:
    """Per-joint rotation: axis uniform on the sphere, angle U[0, max_deg]."""
    rng = np.random.default_rng(seed)
    ax = rng.standard_normal((J, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(0.0, max_deg, J))
    aa = (ax * ang[:, None]).astype(np.float32)
    return Pose(aa, np.zeros(3, np.float32) if R is None else np.asarray(R, np.float32),
                np.zeros(3, np.float32) if T is None else np.asarray(T, np.float32))


def walk_pose(frame: int, n_frames: int = 60, J: int = J_JOINTS) -> Pose:
    """Synthetic walk cycle: shoulders/hips swing +-25 deg about the lateral
    axis with diagonal pairs in phase, elbows/knees flex, spine sways +-5 deg,
    neck bobs and the tail wags."""
    ph = 2.0 * math.pi * (frame % n_frames) / n_frames
    aa = np.zeros((J, 3))
    lat = np.array([0.0, 0.0, 1.0])
    up = np.array([0.0, 1.0, 0.0])
    legs = {7: 0.0, 11: math.pi, 15: math.pi, 19: 0.0}  # FL+HR, FR+HL in phase
    for top, off in legs.items():
        a = math.radians(25.0) * math.sin(ph + off)
        aa[top] = lat * a
        bend = math.radians(20.0) * 0.5 * (1.0 - math.cos(ph + off))
        aa[top + 1] = lat * (-bend if top < 15 else bend)
        aa[top + 2] = lat * (0.5 * bend if top < 15 else -0.5 * bend)
    for j in (1, 2, 3):
        aa[j] = up * math.radians(5.0) * math.sin(ph + 0.4 * j)
    aa[4] = lat * math.radians(6.0) * math.sin(2 * ph)
    aa[23] = up * math.radians(15.0) * math.sin(ph)
    return Pose(aa.astype(np.float32), np.zeros(3, np.float32), np.zeros(3, np.float32))


def look_at(eye: np.ndarray, target: np.ndarray, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World-to-camera [R | t] for a camera at ``eye`` looking at ``target``
    (+x right, +y down, +z forward)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    t = -R @ eye
    return np.concatenate([R, t[:, None]], 1)


def orbit_camera(target: np.ndarray, W: int, H: int, az_deg: float = 0.0, elev_deg: float = 15.0,
                 dist: float = 2.0, fov_deg: float = 40.0, near: float = 0.5, far: float = 3.5,
                 shift_x: float = 0.0) -> Camera:
    """Camera on a sphere of radius ``dist`` about ``target`` (vertical fov).
    ``shift_x`` moves it along its own x axis (stereo eyes)."""
    az, el = math.radians(az_deg), math.radians(elev_deg)
    eye = np.asarray(target, np.float64) + dist * np.array(
        [math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    M = look_at(eye, target)
    if shift_x:
        # x_cam' = x_cam - shift along camera x: eye moves by +shift * x_axis.
        M = M.copy()
        M[0, 3] -= shift_x
    fy = 0.5 * H / math.tan(0.5 * math.radians(fov_deg))
    return Camera(W=W, H=H, fx=fy, fy=fy, cx=0.5 * W, cy=0.5 * H,
                  world_to_cam=M.astype(np.float32), near=near, far=far)


# ---------------------------------------------------------------------------
# Shading network weights (He-normal from the seed)
# ---------------------------------------------------------------------------

UNET_CHANNELS = (32, 64, 128, 256)


def _conv_w(rng, cout: int, cin: int, k: int) -> Tuple[np.ndarray, np.ndarray]:
    std = math.sqrt(2.0 / (k * k * cin))
    w = (std * rng.standard_normal((cout, k, k, cin))).astype(np.float32)
    b = (0.05 * rng.standard_normal(cout)).astype(np.float32)
    return w, b


def tiny_net_weights(seed: int, cin: int = 16, mid: int = 32, cout: int = 4):
    """Three 3x3 layers cin->mid->mid->cout; layout [Cout][3][3][Cin]."""
    rng = np.random.default_rng(seed)
    return [_conv_w(rng, mid, cin, 3), _conv_w(rng, mid, mid, 3), _conv_w(rng, cout, mid, 3)]


def unet_layer_shapes(cin: int = 32, ch=UNET_CHANNELS, cout: int = 4):
    """(Cout, Cin, k) of every layer of a len(ch)-level U-Net, in execution
    order: enc0 a/b, ..., enc(L-1) a/b (bottleneck), dec(L-2) a/b, ...,
    dec0 a/b, head (1x1).  A decoder level's first layer takes the upsampled
    level below concatenated with the skip."""
    L = len(ch)
    shapes, prev = [], cin
    for c in ch:
        shapes += [(c, prev, 3), (c, c, 3)]
        prev = c
    for l in range(L - 2, -1, -1):
        shapes += [(ch[l], ch[l + 1] + ch[l], 3), (ch[l], ch[l], 3)]
    return shapes + [(cout, ch[0], 1)]


def unet_weights(seed: int, cin: int = 32, ch=UNET_CHANNELS, cout: int = 4):
    rng = np.random.default_rng(seed)
    return [_conv_w(rng, co, ci, k) for co, ci, k in unet_layer_shapes(cin, ch, cout)]


ALPHA_CHANNELS = (32, 64)  # the paper gives no widths; these fit the tensor-core kernels


def two_branch_weights(seed: int, cin: int = 32, rgb_ch=UNET_CHANNELS, alpha_ch=ALPHA_CHANNELS):
    """The two-branch shading network's weights: an RGB U-Net cin -> 3 with
    len(rgb_ch) levels and an alpha U-Net (1 + 3) -> 1 with len(alpha_ch)
    levels (its input is the coarse opacity and the RGB branch's image)."""
    return unet_weights(seed, cin, rgb_ch, 3), unet_weights(seed + 1, 4, alpha_ch, 1)


# ---------------------------------------------------------------------------
# Presets (the workloads the tests and the bench use)
# ---------------------------------------------------------------------------

PRESETS = {
    # ~20k leaf voxels at depth 8, |sdf| <= 1.5 cm, C=16, 128^2 view.
    "tiny": dict(depth=8, target=20000, C=16, band=(-0.015, 0.015), fur_shell=False, res=(128, 128)),
    # ~1M leaf voxels at depth 10, -1 cm <= sdf <= 2 cm with fur shell, C=32, 1024^2.
    "paper": dict(depth=10, target=1000000, C=32, band=(-0.010, 0.020), fur_shell=True, res=(1024, 1024)),
    # ~200k leaf voxels at depth 9, C=16, 512^2 (gradient workload).
    "diff": dict(depth=9, target=200000, C=16, band=(-0.010, 0.020), fur_shell=True, res=(512, 512)),
    # small scenes for quick parity cases
    "mini": dict(depth=7, target=3000, C=8, band=(-0.02, 0.02), fur_shell=False, res=(64, 64)),
}

_CACHE: dict = {}


def preset(name: str, seed: int = 0, C: Optional[int] = None) -> Scene:
    """Scene for a named workload (memoised per process)."""
    key = (name, seed, C)
    if key not in _CACHE:
        p = PRESETS[name]
        _CACHE[key] = make_octree(p["depth"], p["target"], C or p["C"], p["band"], seed,
                                  fur_shell=p["fur_shell"])
    return _CACHE[key]
