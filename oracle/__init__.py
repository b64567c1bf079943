"""FP64 CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
compiled by :func:`build`) and composes the shading networks from its
convolution primitives.  Every function follows a passage of the paper
(arXiv 2202.05628):

* :func:`fk`, :func:`lbs` - skeleton S = {r, R, T} and linear blend skinning,
  Sec. 3.1 "Rigging and Deformation", Eq. 4.
* :func:`render`, :func:`pixels`, :func:`pixel_brute` - exact ray / warped-voxel
  hits and front-to-back compositing into the feature map F and coarse opacity
  map A, Sec. 3.1 "Dynamic Volume Rendering", Eq. 5-6 and the early-stop rule.
* :func:`tile_pairs` - screen-tile coverage of the warped voxels (the per-frame
  indexing step that replaces the paper's octree rebuild).
* :func:`shade_tiny`, :func:`shade_unet` - the neural shading network,
  Sec. 3.1 "Neural Shading" (single-branch "Light" form, Sec. 6 "Runtime
  Analysis").
* :func:`render_backward`, :func:`lbs_backward` - gradients of Eq. 5-6 and
  Eq. 4 (the paper optimises the feature table end to end).
* :func:`proposal_inputs`, :func:`proposal_mlp`, :func:`proposal_bins`,
  :func:`render_interval`, :func:`tau_hist`, :func:`coarse_bound`,
  :func:`tile_union_bins`, :func:`skip_render` - the learned ray-interval proposal that lets the
  composite skip empty depth (project addition; the paper's nearest passage
  is the early-stop rule of Sec. 3.1).

Pins: each of these is checked in ``tests/test_oracle_pins.py`` against
closed forms, brute force, invariants and library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

TAU_DEFAULT = 1e-4


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, FP64, OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
            _lib.orc_render.restype = ctypes.c_int64
            _lib.orc_tile_pairs.restype = ctypes.c_int64
            _lib.orc_grid_snap.restype = ctypes.c_int64
            _lib.orc_render_grid.restype = ctypes.c_int64
    return _lib


def num_threads() -> int:
    return int(_L().orc_num_threads())


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("C", ctypes.c_int), ("h", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("ijk", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("feat", ctypes.c_void_p), ("sigma", ctypes.c_void_p)]


class _Cam(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("w2c", ctypes.c_double * 12), ("near_", ctypes.c_double), ("far_", ctypes.c_double)]


def _p(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _Bound:
    """Keeps the numpy arrays alive while C holds pointers to them."""

    def __init__(self, octree, A: np.ndarray, features=None, density=None):
        self.ijk = np.ascontiguousarray(octree.ijk, dtype=np.uint16)
        self.A = _f64(A)
        self.feat = _f64(octree.features if features is None else features)
        self.sigma = _f64(octree.density if density is None else density)
        s = _Scene()
        s.n = self.ijk.shape[0]
        s.C = self.feat.shape[1]
        s.h = float(octree.extent) / float(1 << octree.depth)
        for a in range(3):
            s.origin[a] = float(octree.origin[a])
        s.ijk, s.A, s.feat, s.sigma = (self.ijk.ctypes.data, self.A.ctypes.data,
                                       self.feat.ctypes.data, self.sigma.ctypes.data)
        self.s = s


def _cam(c) -> _Cam:
    k = _Cam()
    k.W, k.H = int(c.W), int(c.H)
    k.fx, k.fy, k.cx, k.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    m = np.asarray(c.world_to_cam, np.float64).reshape(12)
    for i in range(12):
        k.w2c[i] = float(m[i])
    k.near_, k.far_ = float(c.near), float(c.far)
    return k


# ---------------------------------------------------------------------------
# Eq. 4: skeleton and LBS
# ---------------------------------------------------------------------------

def rodrigues(r) -> np.ndarray:
    out = np.zeros(9)
    r = _f64(r)  # keep the converted array alive across the call
    _L().orc_rodrigues(_p(r), _p(out))
    return out.reshape(3, 3)


def fk(skeleton, pose) -> np.ndarray:
    """G_j = M^t_j (M^c_j)^-1 for every joint, [J,3,4] FP64."""
    J = skeleton.J
    G = np.zeros((J, 12))
    parent = np.ascontiguousarray(skeleton.parent, dtype=np.int32)
    rest, aa = _f64(skeleton.rest), _f64(pose.axis_angle)
    R, T = _f64(pose.R), _f64(pose.T)
    rc = _L().orc_fk(ctypes.c_int(J), _p(parent), _p(rest), _p(aa), _p(R), _p(T), _p(G))
    if rc != 0:
        raise ValueError(f"orc_fk failed ({rc}): parent[j] must be < j with a single root 0")
    return G.reshape(J, 3, 4)


def lbs(octree, G: np.ndarray, weights=None) -> Tuple[np.ndarray, np.ndarray]:
    """A_i = sum_k w_ik G_{j_ik} ([N,3,4]) and det of its 3x3 block ([N])."""
    n = octree.n
    G = _f64(G).reshape(-1, 12)
    jidx = np.ascontiguousarray(octree.joint_idx, dtype=np.uint8)
    w = _f64(octree.weights if weights is None else weights)
    A = np.zeros((n, 12))
    det = np.zeros(n)
    _L().orc_lbs(ctypes.c_int64(n), ctypes.c_int(G.shape[0]), _p(G), _p(jidx), _p(w), _p(A), _p(det))
    return A.reshape(n, 3, 4), det


def pose_transforms(scene, pose, weights=None):
    G = fk(scene.skeleton, pose)
    A, det = lbs(scene.octree, G, weights)
    return G, A, det


# ---------------------------------------------------------------------------
# Eq. 5-6: rays, hits, compositing
# ---------------------------------------------------------------------------

def pixel_ray(cam, x: int, y: int) -> Tuple[np.ndarray, np.ndarray]:
    o, d = np.zeros(3), np.zeros(3)
    k = _cam(cam)
    _L().orc_pixel_ray(ctypes.byref(k), ctypes.c_int(x), ctypes.c_int(y), _p(o), _p(d))
    return o, d


def render(octree, A: np.ndarray, cam, tau: float = TAU_DEFAULT, hits: bool = False,
           features=None, density=None) -> dict:
    """Feature map F [H,W,C], coarse opacity A [H,W], per-pixel hit counts and,
    with ``hits=True``, the ordered per-pixel hit lists (CSR)."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), features, density)
    k = _cam(cam)
    H, W, C = cam.H, cam.W, b.feat.shape[1]
    F = np.zeros((H, W, C))
    Am = np.zeros((H, W))
    nhit = np.zeros((H, W), np.int32)
    nused = np.zeros((H, W), np.int32)
    L = _L()
    out = dict(F=F, A=Am, nhit=nhit, nused=nused)
    if not hits:
        r = L.orc_render(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau), _p(F), _p(Am),
                         _p(nhit), _p(nused), None, None, None, None, ctypes.c_int64(0))
        if r < 0:
            raise MemoryError("orc_render failed")
        return out
    cap = int(1.5 * 64 * H * W) + 1024
    while True:
        off = np.zeros(H * W + 1, np.int64)
        hid = np.zeros(cap, np.int64)
        t0 = np.zeros(cap)
        t1 = np.zeros(cap)
        r = L.orc_render(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau), _p(F), _p(Am),
                         _p(nhit), _p(nused), _p(off), _p(hid), _p(t0), _p(t1), ctypes.c_int64(cap))
        if r >= 0:
            break
        if r < -(1 << 40):
            raise MemoryError("orc_render failed")
        cap = int(-r) + 16
    out.update(hit_off=off, hit_id=hid[:r], hit_t0=t0[:r], hit_t1=t1[:r])
    return out


def depth(octree, A: np.ndarray, cam, sigma_min: float, density=None) -> dict:
    """Depth buffer (Sec. 3.1 "Hybrid Rendering"): per pixel the entry distance
    of the first hit (compositing order, all hits in [near, far]) whose density
    exceeds ``sigma_min``, +inf where there is none; ``chord`` = t1 - t0 of
    that hit.  [H, W] each."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), None, density)
    k = _cam(cam)
    D = np.zeros((cam.H, cam.W))
    ch = np.zeros((cam.H, cam.W))
    if _L().orc_depth(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(sigma_min), _p(D), _p(ch)) != 0:
        raise MemoryError("orc_depth failed")
    return dict(depth=D, chord=ch)


# ---------------------------------------------------------------------------
# The paper's per-frame index: warped centres snapped to the leaf lattice
# ---------------------------------------------------------------------------

def grid_snap(octree, A: np.ndarray) -> dict:
    """Each voxel's lattice cell floor((A_i p_i^c - origin) / h) [n, 3], the
    survivor of its cell [n] (smallest id; -1 = not placed) and the number of
    occupied cells."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), np.zeros((octree.n, 1)))
    cell = np.zeros((octree.n, 3), np.int64)
    win = np.zeros(octree.n, np.int64)
    nc = _L().orc_grid_snap(ctypes.byref(b.s), _p(cell), _p(win))
    if nc < 0:
        raise MemoryError("orc_grid_snap failed")
    return dict(cell=cell, winner=win, n_cells=int(nc))


def render_grid(octree, A: np.ndarray, cam, tau: float = TAU_DEFAULT, features=None, density=None) -> dict:
    """F [H,W,C], A [H,W], hit counts [H,W] of the snapped index: the occupied
    lattice cells as axis-aligned boxes carrying their survivors' features and
    densities, composited as the voxel path does."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), features, density)
    k = _cam(cam)
    F = np.zeros((cam.H, cam.W, b.feat.shape[1]))
    Am = np.zeros((cam.H, cam.W))
    nhit = np.zeros((cam.H, cam.W), np.int32)
    nc = _L().orc_render_grid(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau), _p(F), _p(Am), _p(nhit))
    if nc < 0:
        raise MemoryError("orc_render_grid failed")
    return dict(F=F, A=Am, nhit=nhit, n_cells=int(nc))


def vrt_loss(octree, A: np.ndarray, features=None, lam: float = 1.0) -> float:
    """The voxel regularisation term (Sec. 3.1, "Training"): lam times the mean
    over the placed voxels of || Q(p_i^t, T^t) - f_i ||_1, Q returning the
    feature of the survivor of the cell that p_i^t falls in."""
    f = _f64(octree.features if features is None else features)
    win = grid_snap(octree, A)["winner"]
    placed = win >= 0
    if not placed.any():
        return 0.0
    return float(lam * np.abs(f[win[placed]] - f[placed]).sum(1).mean())


# ---------------------------------------------------------------------------
# Eq. 2: view-dependent features (spherical harmonics)
# ---------------------------------------------------------------------------

SH_LMAX = 9


def sh_basis(L: int, dirs) -> np.ndarray:
    """Real orthonormal spherical harmonics of degree <= L at unit directions
    ``dirs`` [m, 3]: [m, (L+1)^2], index l^2 + l + m."""
    d = _f64(np.atleast_2d(dirs))
    H = (L + 1) ** 2
    out = np.zeros((d.shape[0], H))
    row = np.zeros(H)
    for k in range(d.shape[0]):
        dk = np.ascontiguousarray(d[k])
        if _L().orc_sh_basis(ctypes.c_int(L), _p(dk), _p(row)) != 0:
            raise ValueError(f"degree {L} out of range [0, {SH_LMAX}]")
        out[k] = row
    return out


def polar_rotation(A) -> np.ndarray:
    """Rotation factor of the polar decomposition of each 3x4 transform's
    linear part: [n, 3, 3]."""
    A = _f64(A).reshape(-1, 12)
    R = np.zeros((A.shape[0], 9))
    for i in range(A.shape[0]):
        a = np.ascontiguousarray(A[i])
        r = np.zeros(9)
        if _L().orc_polar_rotation(_p(a), _p(r)) != 0:
            raise ValueError("polar_rotation: det <= 0")
        R[i] = r
    return R.reshape(-1, 3, 3)


def render_sh(octree, A: np.ndarray, cam, L: int, coef, tau: float = TAU_DEFAULT, density=None) -> dict:
    """F [H,W,C] and A [H,W] with view-dependent features (Eq. 2): hit i's
    feature is sum_h coef[i, h] Y_h(R_i^T d), R_i the rotation factor of its
    transform, d the unit ray direction.  coef: [n, (L+1)^2, C]."""
    coef = _f64(coef)
    n, H, C = coef.shape
    assert n == octree.n and H == (L + 1) ** 2
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), np.zeros((n, C)), density)
    k = _cam(cam)
    F = np.zeros((cam.H, cam.W, C))
    Am = np.zeros((cam.H, cam.W))
    if _L().orc_render_sh(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau), ctypes.c_int(L), _p(coef),
                          _p(F), _p(Am)) != 0:
        raise ValueError("orc_render_sh failed (degree out of range or allocation)")
    return dict(F=F, A=Am)


def render_sh_backward(octree, A: np.ndarray, cam, L: int, gF, tau: float = TAU_DEFAULT, density=None,
                       C: Optional[int] = None) -> np.ndarray:
    """dL/dcoef [n, (L+1)^2, C] of render_sh's feature map for dL/dF = gF [H, W, C]."""
    gF = _f64(gF)
    C = gF.shape[2] if C is None else C
    n, H = octree.n, (L + 1) ** 2
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), np.zeros((n, C)), density)
    k = _cam(cam)
    g = np.zeros((n, H, C))
    if _L().orc_render_sh_backward(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau), ctypes.c_int(L),
                                   _p(gF), _p(g)) != 0:
        raise ValueError("orc_render_sh_backward failed (degree out of range or allocation)")
    return g


def pixels(octree, A: np.ndarray, cam, px: Sequence[int], py: Sequence[int],
           tau: float = TAU_DEFAULT, features=None, density=None, tie_eps: float = 1e-6) -> dict:
    """Sampled pixels, each by brute force over every voxel.  ``tie`` is, per
    pixel, the largest change of a feature channel that swapping two
    consecutive composited hits with entry distances within ``tie_eps`` would
    cause (T_i alpha_i alpha_j |f_i - f_j|; 0 without such a pair): the part
    of F that rounding of the entry distances can decide."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), features, density)
    k = _cam(cam)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    m = px.shape[0]
    F = np.zeros((m, b.feat.shape[1]))
    Am = np.zeros(m)
    nh = np.zeros(m, np.int32)
    tie = np.zeros(m)
    _L().orc_pixels(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_int64(m), _p(px), _p(py),
                    ctypes.c_double(tau), _p(F), _p(Am), _p(nh), ctypes.c_double(tie_eps), _p(tie))
    return dict(F=F, A=Am, nhit=nh, tie=tie)


def pixel_brute(octree, A: np.ndarray, cam, x: int, y: int, tau: float = TAU_DEFAULT,
                features=None, density=None, cap: int = 4096) -> dict:
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), features, density)
    k = _cam(cam)
    F = np.zeros(b.feat.shape[1])
    Am = np.zeros(1)
    ids = np.zeros(cap, np.int64)
    t0 = np.zeros(cap)
    t1 = np.zeros(cap)
    used = ctypes.c_int(0)
    m = _L().orc_pixel_brute(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_int(x), ctypes.c_int(y),
                             ctypes.c_double(tau), _p(F), _p(Am), _p(ids), _p(t0), _p(t1),
                             ctypes.c_int(cap), ctypes.byref(used))
    m2 = min(m, cap)
    return dict(F=F, A=float(Am[0]), ids=ids[:m2], t0=t0[:m2], t1=t1[:m2], nhit=m, nused=used.value)


def tile_pairs(octree, A: np.ndarray, cam, tsx: int = 8, tsy: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray]:
    """(tile id, voxel id) pairs of the screen-tile coverage (tiles of
    tsx x tsy pixels, row-major tile ids), voxel-major."""
    tsy = tsx if tsy is None else tsy
    b = _Bound(octree, np.asarray(A).reshape(-1, 12))
    k = _cam(cam)
    cap = 4 * octree.n + 1024
    while True:
        tile = np.zeros(cap, np.int32)
        vid = np.zeros(cap, np.int64)
        r = _L().orc_tile_pairs(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_int(tsx), ctypes.c_int(tsy), _p(tile),
                                _p(vid), ctypes.c_int64(cap))
        if r >= 0:
            return tile[:r], vid[:r]
        if r < -(1 << 40):
            raise MemoryError("orc_tile_pairs failed")
        cap = int(-r) + 16


def voxel_bounds(octree, A: np.ndarray, cam) -> np.ndarray:
    """Per voxel: ok, umin, umax, vmin, vmax, dmin, dmax (FP64)."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12))
    out = np.zeros((octree.n, 7))
    _L().orc_voxel_bounds(ctypes.byref(b.s), ctypes.byref(_cam(cam)), _p(out))
    return out


# ---------------------------------------------------------------------------
# Gradients (project addition, see module docstring)
# ---------------------------------------------------------------------------

def render_backward(octree, A: np.ndarray, cam, gF: np.ndarray, gA: np.ndarray,
                    tau: float = TAU_DEFAULT, features=None, density=None):
    """dL/df [N,C], dL/dsigma [N], dL/dAinv [N,3,4] for upstream gF, gA."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12), features, density)
    k = _cam(cam)
    n, C = octree.n, b.feat.shape[1]
    gfeat = np.zeros((n, C))
    gsig = np.zeros(n)
    gAi = np.zeros((n, 12))
    gF, gA = _f64(gF), _f64(gA)  # keep the converted arrays alive across the call
    rc = _L().orc_render_backward(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau),
                                  _p(gF), _p(gA), _p(gfeat), _p(gsig), _p(gAi))
    if rc != 0:
        raise MemoryError("orc_render_backward failed")
    return gfeat, gsig, gAi.reshape(n, 3, 4)


def lbs_backward(octree, G: np.ndarray, A: np.ndarray, gAinv: np.ndarray):
    """dL/dA [N,3,4] and dL/dw [N,4] from dL/dAinv."""
    n = octree.n
    G = _f64(G).reshape(-1, 12)
    jidx = np.ascontiguousarray(octree.joint_idx, dtype=np.uint8)
    gA = np.zeros((n, 12))
    gw = np.zeros((n, 4))
    A64 = _f64(A).reshape(-1, 12)
    gAi64 = _f64(gAinv).reshape(-1, 12)
    _L().orc_lbs_backward(ctypes.c_int64(n), ctypes.c_int(G.shape[0]), _p(G), _p(jidx), _p(A64), _p(gAi64), _p(gA),
                          _p(gw))
    return gA.reshape(n, 3, 4), gw


# ---------------------------------------------------------------------------
# Neural shading (Sec. 3.1 "Neural Shading")
# ---------------------------------------------------------------------------

ACT_NONE, ACT_RELU, ACT_SIGMOID = 0, 1, 2


def conv2d(x: np.ndarray, w: np.ndarray, b: Optional[np.ndarray], act: int) -> np.ndarray:
    """x [H,W,Cin], w [Cout,k,k,Cin], zero 'same' padding."""
    x = _f64(x)
    w = _f64(w)
    H, W, Cin = x.shape
    Cout, k = w.shape[0], w.shape[1]
    assert w.shape == (Cout, k, k, Cin)
    out = np.zeros((H, W, Cout))
    bb = None if b is None else _f64(b)
    _L().orc_conv2d(ctypes.c_int(H), ctypes.c_int(W), ctypes.c_int(Cin), ctypes.c_int(Cout),
                    ctypes.c_int(k), _p(x), _p(w), _p(bb), _p(out), ctypes.c_int(act))
    return out


def maxpool2(x: np.ndarray) -> np.ndarray:
    x = _f64(x)
    H, W, C = x.shape
    out = np.zeros((H // 2, W // 2, C))
    _L().orc_maxpool2(ctypes.c_int(H), ctypes.c_int(W), ctypes.c_int(C), _p(x), _p(out))
    return out


def upsample2(x: np.ndarray) -> np.ndarray:
    x = _f64(x)
    H, W, C = x.shape
    out = np.zeros((2 * H, 2 * W, C))
    _L().orc_upsample2(ctypes.c_int(H), ctypes.c_int(W), ctypes.c_int(C), _p(x), _p(out))
    return out


def shade_tiny(F: np.ndarray, layers) -> np.ndarray:
    """conv3x3 + ReLU, conv3x3 + ReLU, conv3x3 + sigmoid -> RGBA [H,W,4]."""
    (w0, b0), (w1, b1), (w2, b2) = layers
    x = conv2d(F, w0, b0, ACT_RELU)
    x = conv2d(x, w1, b1, ACT_RELU)
    return conv2d(x, w2, b2, ACT_SIGMOID)


def unet(x: np.ndarray, layers, levels: int) -> np.ndarray:
    """U-Net of ``levels`` levels: per level two conv3x3 + ReLU; 2x2 max-pool
    down; nearest x2 up, concatenation [upsampled, skip] on channels, two
    conv3x3 + ReLU; 1x1 head + sigmoid.  x [H,W,Cin], H and W divisible by
    2^(levels-1)."""
    it = iter(layers)

    def block(x):
        w, b = next(it)
        x = conv2d(x, w, b, ACT_RELU)
        w, b = next(it)
        return conv2d(x, w, b, ACT_RELU)

    skips = [block(x)]
    for _ in range(levels - 1):
        skips.append(block(maxpool2(skips[-1])))
    d = skips.pop()
    while skips:
        d = block(np.concatenate([upsample2(d), skips.pop()], axis=2))
    w, b = next(it)
    return conv2d(d, w, b, ACT_SIGMOID)


def shade_unet(F: np.ndarray, layers) -> np.ndarray:
    """The 4-level U-Net shading F -> RGBA [H,W,4]."""
    return unet(F, layers, 4)


def shade_two_branch(F: np.ndarray, A: np.ndarray, rgb_layers, alpha_layers, rgb_levels: int = 4,
                     alpha_levels: int = 2) -> np.ndarray:
    """The paper's two-branch shading network G (Sec. 3.1 "Neural Shading",
    Fig. 4): the appearance branch turns the feature map F into the texture
    image I_f [H,W,3]; the opacity branch refines the coarse opacity map A
    from [A, I_f] (4 channels) into alpha [H,W,1].  Returns [I_f, alpha]."""
    I_f = unet(F, rgb_layers, rgb_levels)
    alpha = unet(np.concatenate([_f64(A)[..., None], I_f], axis=2), alpha_layers, alpha_levels)
    return np.concatenate([I_f, alpha], axis=2)


def shade(F: np.ndarray, layers) -> np.ndarray:
    return shade_tiny(F, layers) if len(layers) == 3 else shade_unet(F, layers)


def render_frame(scene, pose, cam, layers=None, tau: float = TAU_DEFAULT) -> dict:
    """Whole path for one view: FK, LBS, F and A maps, RGBA."""
    G, A, det = pose_transforms(scene, pose)
    out = render(scene.octree, A, cam, tau)
    out["G"], out["Ablend"], out["det"] = G, A, det
    if layers is not None:
        out["rgba"] = shade(out["F"], layers)
    return out


# ---------------------------------------------------------------------------
# Learned ray-interval proposal (project addition, see module docstring)
# ---------------------------------------------------------------------------
#
# Definitions followed by both sides:
#   input x (107) = [72 pose axis-angles (J = 24 joints x 3, as given to the
#     pose), 3 unit world ray direction, sin(2^k pi u) k<8, cos(2^k pi u) k<8,
#     sin(2^k pi v) k<8, cos(2^k pi v) k<8], u = (x + 1/2) / W, v = (y + 1/2) / H;
#   MLP 107 -> 64 -> 64 -> 64 -> 64 (ReLU) -> 128 logits; parameters flat as
#     W0 [64][107], b0, W1 [64][64], b1, W2, b2, W3, b3, W4 [128][64], b4
#     (y = W x + b);
#   bins: bn = argmax of logits[0:64], bf = argmax of logits[64:128] (first
#     index on ties); interval [near + bn D, near + (bf + 1) D], D = (far -
#     near) / 64; bf < bn is the empty interval.

PROPOSAL_IN, PROPOSAL_HIDDEN, PROPOSAL_BINS = 107, 64, 64
PROPOSAL_SHAPES = [(64, 107), (64, 64), (64, 64), (64, 64), (128, 64)]
PROPOSAL_PARAMS = sum(o * i + o for o, i in PROPOSAL_SHAPES)
MISSED_MAX = 1e-3   # coarse-check threshold of lost transmittance mass
LABEL_WMIN = 1e-6   # a hit is significant when its weight T_i alpha_i exceeds this


def round_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 (ties to even) via FP32; returns FP64."""
    b = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def ray_dirs(cam) -> np.ndarray:
    """Unit world-space directions of every pixel's ray, [H, W, 3]."""
    d = np.zeros((cam.H, cam.W, 3))
    _L().orc_ray_dirs(ctypes.byref(_cam(cam)), _p(d))
    return d


def proposal_inputs(axis_angle, cam) -> np.ndarray:
    """The 107-dim proposal input of every pixel's ray, [H*W, 107] FP64."""
    H, W = cam.H, cam.W
    pose = _f64(axis_angle).reshape(-1)
    assert pose.size == 72, "the proposal takes the 24 joints' axis-angles"
    d = ray_dirs(cam).reshape(-1, 3)
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    u = ((xs + 0.5) / W).reshape(-1, 1)
    v = ((ys + 0.5) / H).reshape(-1, 1)
    fr = np.pi * (2.0 ** np.arange(8))[None, :]
    four = np.concatenate([np.sin(fr * u), np.cos(fr * u), np.sin(fr * v), np.cos(fr * v)], 1)
    return np.concatenate([np.broadcast_to(pose, (H * W, 72)), d, four], 1)


def proposal_layers(params):
    """Split the flat parameter vector into [(W, b)] of the five layers."""
    p = _f64(params).reshape(-1)
    assert p.size == PROPOSAL_PARAMS, (p.size, PROPOSAL_PARAMS)
    out, o = [], 0
    for n_out, n_in in PROPOSAL_SHAPES:
        W = p[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = p[o:o + n_out]
        o += n_out
        out.append((W, b))
    return out


def proposal_mlp(x, params, bf16: bool = False) -> np.ndarray:
    """Logits [M, 128].  With ``bf16`` the inputs, weights and hidden
    activations are rounded to BF16 where the GPU stores them (biases FP32,
    sums exact): the precision in which the GPU takes the argmax."""
    h = _f64(x)
    layers = proposal_layers(params)
    if bf16:
        h = round_bf16(h)
    for li, (W, b) in enumerate(layers):
        if bf16:
            W, b = round_bf16(W), np.asarray(b, np.float32).astype(np.float64)
        h = h @ W.T + b
        if li < len(layers) - 1:
            h = np.maximum(h, 0.0)
            if bf16:
                h = round_bf16(h)
    return h


def proposal_bins(logits) -> np.ndarray:
    """(bn, bf) per row: first argmax of each half of the logits, [M, 2] int32."""
    lg = np.asarray(logits)
    return np.stack([np.argmax(lg[:, :PROPOSAL_BINS], 1), np.argmax(lg[:, PROPOSAL_BINS:], 1)], 1).astype(np.int32)


def label_bins(labels, hist, cam, tsx: int = 8, tsy: int = 4, nb: int = PROPOSAL_BINS,
               budget: float = 0.4 * MISSED_MAX) -> np.ndarray:
    """Training label (bn, bf) of every ray, [H*W, 2] int32: the interval
    that keeps every significant hit and that the coarse check passes.
    ``labels`` [H, W, 3] = (lo, hi, Ts) of the plain composite (min t1 and
    max t0 over significant hits, transmittance after the last of them);
    ``hist`` the tile histogram of :func:`tau_hist`.
      bn = min(bin(lo), the largest b with 1 - exp(-sum_{b' < b} hist) <= budget)
      bf = the smallest b >= bin(hi) with Ts (1 - exp(-sum_{b' > b} hist)) <= budget
    (bin(t) = floor((t - near) / D) clamped to [0, nb - 1]; no significant
    hit: bin(lo) = nb - 1, bin(hi) = 0, Ts = 1).  With the two budgets at
    0.4 of the threshold the check passes for these bins."""
    H, W = cam.H, cam.W
    lab = np.asarray(labels, np.float64).reshape(-1, 3)
    D = (cam.far - cam.near) / nb
    tw = (W + tsx - 1) // tsx
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    tile = ((ys // tsy) * tw + xs // tsx).reshape(-1)
    Ht = np.asarray(hist, np.float64)[tile]                      # [M, nb]
    before = np.cumsum(Ht, 1) - Ht                               # sum over b' < b
    after = Ht.sum(1, keepdims=True) - np.cumsum(Ht, 1)          # sum over b' > b
    sig = np.isfinite(lab[:, 0])
    b_lo = np.where(sig, np.clip(np.floor((np.where(sig, lab[:, 0], cam.near) - cam.near) / D), 0, nb - 1), nb - 1)
    b_hi = np.where(sig, np.clip(np.floor((np.where(sig, lab[:, 1], cam.near) - cam.near) / D), 0, nb - 1), 0)
    ok_f = (1.0 - np.exp(-before)) <= budget                      # monotone: true up to some b
    front = np.where(ok_f.all(1), nb - 1, np.argmin(ok_f, 1) - 1)
    bn = np.minimum(b_lo, front)
    ok_b = lab[:, 2:3] * (1.0 - np.exp(-after)) <= budget          # monotone: true from some b on
    bidx = np.arange(nb)[None, :]
    cand = ok_b & (bidx >= b_hi[:, None])
    bf = np.argmax(cand, 1)
    return np.stack([bn, bf], 1).astype(np.int32)


def render_interval(octree, A: np.ndarray, cam, bins=None, tau: float = TAU_DEFAULT, nb: int = PROPOSAL_BINS,
                    wmin: float = LABEL_WMIN, eps: float = 1e-5, labels: bool = False) -> dict:
    """Composite restricted to the interval of ``bins`` [H*W, 2] (None: the
    whole [near, far]), its exact lost mass ``missed`` and the ambiguity flag
    ``amb`` (a hit within ``eps`` of an interval end); with ``labels`` also
    the plain composite's (min t1, max t0) over significant hits and the
    transmittance after the last of them, [H, W, 3]."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12))
    k = _cam(cam)
    H, W, C = cam.H, cam.W, b.feat.shape[1]
    F = np.zeros((H, W, C))
    Am = np.zeros((H, W))
    missed = np.zeros((H, W))
    amb = np.zeros((H, W), np.int32)
    lab = np.zeros((H, W, 3)) if labels else None
    bn = None if bins is None else np.ascontiguousarray(np.asarray(bins).reshape(-1, 2), np.int32)
    rc = _L().orc_render_interval(ctypes.byref(b.s), ctypes.byref(k), ctypes.c_double(tau), ctypes.c_int(nb),
                                  _p(bn), ctypes.c_double(wmin), ctypes.c_double(eps), _p(lab), _p(F), _p(Am),
                                  _p(missed), _p(amb))
    if rc != 0:
        raise MemoryError("orc_render_interval failed")
    out = dict(F=F, A=Am, missed=missed, amb=amb)
    if labels:
        out["labels"] = lab
    return out


def tau_hist(octree, A: np.ndarray, cam, tsx: int = 8, tsy: int = 4, nb: int = PROPOSAL_BINS) -> np.ndarray:
    """Coarse optical-depth bound per (screen tile, depth bin), [tiles, nb]."""
    b = _Bound(octree, np.asarray(A).reshape(-1, 12))
    tw, th = (cam.W + tsx - 1) // tsx, (cam.H + tsy - 1) // tsy
    hist = np.zeros((tw * th, nb))
    rc = _L().orc_tau_hist(ctypes.byref(b.s), ctypes.byref(_cam(cam)), ctypes.c_int(tsx), ctypes.c_int(tsy),
                           ctypes.c_int(nb), _p(hist))
    if rc != 0:
        raise MemoryError("orc_tau_hist failed")
    return hist


def coarse_bound(hist, bins, T_end, cam, tsx: int = 8, tsy: int = 4) -> np.ndarray:
    """Per pixel: an upper bound of the lost mass from the tile histogram,
    (1 - exp(-tau_front)) + T_end (1 - exp(-tau_back)), tau_front = the bins
    before bn (all bins for an empty interval), tau_back = the bins after bf."""
    H, W = cam.H, cam.W
    tw = (W + tsx - 1) // tsx
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    tile = ((ys // tsy) * tw + xs // tsx).reshape(-1)
    bins = np.asarray(bins).reshape(-1, 2)
    cs = np.cumsum(hist, 1)[tile]  # inclusive prefix sums of the pixel's tile
    tot = cs[:, -1]
    bn, bf = bins[:, 0], bins[:, 1]
    empty = bf < bn
    rows = np.arange(H * W)
    front = np.where(bn > 0, cs[rows, np.maximum(bn - 1, 0)], 0.0)
    back = tot - cs[rows, np.clip(bf, 0, hist.shape[1] - 1)]
    front = np.where(empty, tot, front)
    back = np.where(empty, 0.0, back)
    T = np.asarray(T_end).reshape(-1)
    return ((1.0 - np.exp(-front)) + T * (1.0 - np.exp(-back))).reshape(H, W)


def tile_union_bins(bins, cam, margin: int = 0, tsx: int = 8, tsy: int = 4, nb: int = PROPOSAL_BINS) -> np.ndarray:
    """Per pixel, the interval its screen tile composites over: the union of
    the tile's non-empty pixel intervals (min bn .. max bf), widened by
    ``margin`` bins and clamped; empty (nb, -1) when every pixel's is empty.
    [H*W, 2] int32."""
    H, W = cam.H, cam.W
    tw, th = (W + tsx - 1) // tsx, (H + tsy - 1) // tsy
    b = np.asarray(bins).reshape(H, W, 2).astype(np.int64)
    ne = b[..., 1] >= b[..., 0]
    lo = np.full((th * tsy, tw * tsx), nb, np.int64)
    hi = np.full((th * tsy, tw * tsx), -1, np.int64)
    lo[:H, :W] = np.where(ne, b[..., 0], nb)
    hi[:H, :W] = np.where(ne, b[..., 1], -1)
    lo_t = lo.reshape(th, tsy, tw, tsx).min((1, 3))
    hi_t = hi.reshape(th, tsy, tw, tsx).max((1, 3))
    empty = hi_t < lo_t
    lo_t = np.where(empty, nb, np.maximum(lo_t - margin, 0))
    hi_t = np.where(empty, -1, np.minimum(hi_t + margin, nb - 1))
    up = lambda t: np.repeat(np.repeat(t, tsy, 0), tsx, 1)[:H, :W]
    return np.stack([up(lo_t), up(hi_t)], -1).reshape(-1, 2).astype(np.int32)


def skip_render(octree, A: np.ndarray, cam, bins, tau: float = TAU_DEFAULT, nb: int = PROPOSAL_BINS,
                max_missed: float = MISSED_MAX, margin: int = 0, tsx: int = 8, tsy: int = 4) -> dict:
    """The learned-skip render: every screen tile composited over the union
    of its pixels' predicted intervals (:func:`tile_union_bins`); a tile in
    which any pixel's coarse bound exceeds ``max_missed`` is rendered again
    with the full traversal (the fallback)."""
    bins = tile_union_bins(bins, cam, margin, tsx, tsy, nb)
    r = render_interval(octree, A, cam, bins, tau, nb)
    full = render_interval(octree, A, cam, None, tau, nb)
    hist = tau_hist(octree, A, cam, tsx, tsy, nb)
    bound = coarse_bound(hist, bins, 1.0 - r["A"], cam, tsx, tsy)
    H, W = cam.H, cam.W
    tw, th = (W + tsx - 1) // tsx, (H + tsy - 1) // tsy
    pad = np.zeros((th * tsy, tw * tsx), bool)
    pad[:H, :W] = bound > max_missed
    fail = pad.reshape(th, tsy, tw, tsx).any((1, 3))
    fb_px = np.repeat(np.repeat(fail, tsy, 0), tsx, 1)[:H, :W]
    F = np.where(fb_px[..., None], full["F"], r["F"])
    Am = np.where(fb_px, full["A"], r["A"])
    return dict(F=F, A=Am, fallback=fail.reshape(-1), bound=bound, missed=r["missed"], amb=r["amb"],
                restricted=r, full=full, hist=hist, bins=bins)
