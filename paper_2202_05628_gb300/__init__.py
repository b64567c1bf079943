"""Python binding of ``libartemis_gb.so``, the GB300 rendering path of ARTEMIS
neural animals (arXiv 2202.05628, Sec. 3.1).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
device memory and streams come from PyTorch.  Importing this package raises
if the compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libartemis_gb.so")

ART_F32, ART_BF16, ART_F16, ART_FP8 = 0, 1, 2, 3
ART_NET_TINY, ART_NET_UNET, ART_NET_TWO_BRANCH = 0, 1, 2
(BUF_JOINT_G, BUF_VOXEL_REC, BUF_VOXEL_GEO, BUF_RECT, BUF_DEPTHKEY, BUF_KEYS, BUF_VALS, BUF_RANGES, BUF_FP8_SCALES,
 BUF_ACTIVATIONS, BUF_BINS, BUF_FALLBACK, BUF_TAU_HIST) = range(13)
SKIP_PLAIN, SKIP_LEARNED = 0, 1
INDEX_BOXES, INDEX_GRID = 0, 1
PROPOSAL_PARAMS = 27712  # 64*107+64 + 3*(64*64+64) + 128*64+128
_STATUS = {0: "ART_OK", 1: "ART_ERR_INVALID_ARG", 2: "ART_ERR_CUDA", 3: "ART_ERR_OOM", 4: "ART_ERR_OVERFLOW",
           5: "ART_ERR_STATE", 6: "ART_ERR_UNSUPPORTED"}
DTYPES = {"f32": ART_F32, "bf16": ART_BF16, "f16": ART_F16, "fp8": ART_FP8}


class ArtemisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class NetDesc(ctypes.Structure):
    _fields_ = [("arch", ctypes.c_int), ("cin", ctypes.c_int), ("ch", ctypes.c_int * 4), ("cout", ctypes.c_int),
                ("ach", ctypes.c_int * 2)]


class Config(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("instance_cap", ctypes.c_int64), ("tile_log2", ctypes.c_int),
                ("profile", ctypes.c_int), ("skip", ctypes.c_int), ("max_missed", ctypes.c_float),
                ("margin", ctypes.c_int), ("segment", ctypes.c_int), ("index", ctypes.c_int),
                ("no_subpixel", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int64), ("degenerate", ctypes.c_int64), ("overflow_inst", ctypes.c_int64),
                ("overflow_order", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("fallback_tiles", ctypes.c_int64), ("exact_tiles", ctypes.c_int64), ("grid_cells", ctypes.c_int64),
                ("forced_tiles", ctypes.c_int64), ("check_fail_tiles", ctypes.c_int64)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2202_05628_gb300.build.build() "
                          "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    sig = {
        "art_create": [ctypes.POINTER(vp), vp],
        "art_set_stream": [vp, vp],
        "art_load_octree": [vp, i64, i32, vp, f32, vp, vp, vp, vp, i32, i32, vp],
        "art_load_skeleton": [vp, i32, vp, vp],
        "art_set_pose": [vp, vp, vp, vp],
        "art_set_camera": [vp, i32, i32, i32, f32, f32, f32, f32, vp, f32, f32],
        "art_render_feature_maps": [vp, i32, vp, i32, vp],
        "art_render_depth": [vp, i32, f32, vp],
        "art_load_sh_features": [vp, i32, vp],
        "art_load_shader": [vp, ctypes.POINTER(NetDesc), vp, i64, i32],
        "art_shade": [vp, i32, vp, i32, vp],
        "art_render_frame": [vp, i32, vp, vp, vp, vp],
        "art_render_frame_async": [vp, i32, vp, vp, vp, vp],
        "art_wait_frames": [vp],
        "art_set_config": [vp, ctypes.POINTER(Config)],
        "art_sync_status": [vp, ctypes.POINTER(Stats)],
        "art_get_kernel_times": [vp, i32, vp, vp, vp, ctypes.POINTER(i32), i32],
        "art_sort_pairs": [vp, vp, vp, i64, i32],
        "art_shade_with_opacity": [vp, i32, vp, i32, vp, vp],
        "art_render_views": [vp, i32, vp, vp, i32, vp],
        "art_sort_pairs_static": [vp, vp, i64, i32, vp],
        "art_update_voxels": [vp, vp, vp, vp],
        "art_render_backward": [vp, i32, vp, vp, vp, vp, vp, vp, vp],
        "art_debug_buffer": [vp, i32, vp, i64, ctypes.POINTER(i64)],
        "art_debug_hits": [vp, i32, i32, vp, vp, vp, vp, vp, vp],
        "art_load_proposal": [vp, vp, i64],
        "art_run_proposal": [vp, i32, vp, vp],
        "art_render_labels": [vp, i32, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.art_destroy.argtypes = [vp]
    lib.art_destroy.restype = None
    lib.art_last_error.argtypes = [vp]
    lib.art_last_error.restype = ctypes.c_char_p
    return lib


_lib = load_library()


def library() -> ctypes.CDLL:
    return _lib


def _ptr(x) -> Optional[int]:
    """Address of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _np(x, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


class Renderer:
    """One library context on one CUDA stream."""

    def __init__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        st = _lib.art_create(ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream))
        if st != 0:
            raise ArtemisError(st, "art_create failed")
        self._h = h
        self._keep = []
        self.C = 0
        self.views = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.art_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, st: int):
        if st != 0:
            raise ArtemisError(st, _lib.art_last_error(self._h).decode())

    # ----------------------------------------------------------------- setup
    def set_config(self, tau: float = 1e-4, instance_cap: int = 0, tile_log2: int = 3, profile: bool = False,
                   skip: int = SKIP_PLAIN, max_missed: float = 1e-3, margin: int = 0, segment: int = 256,
                   index: int = 0, no_subpixel: bool = False):
        c = Config(tau, instance_cap, tile_log2, int(profile), int(skip), float(max_missed), int(margin),
                   int(segment), int(index), int(no_subpixel))
        self._check(_lib.art_set_config(self._h, ctypes.byref(c)))

    def load_octree(self, depth: int, origin, extent: float, ijk, joint_idx, weights, features, density,
                    storage: str = "f32"):
        ijk, jidx = _np(ijk, np.uint16), _np(joint_idx, np.uint8)
        w, f, d = _np(weights, np.float32), _np(features, np.float32), _np(density, np.float32)
        o = _np(origin, np.float32)
        n, C = f.shape
        self._check(_lib.art_load_octree(self._h, n, depth, _ptr(o), float(extent), _ptr(ijk), _ptr(jidx), _ptr(w),
                                         _ptr(f), C, DTYPES[storage], _ptr(d)))
        self.C = C
        self.n = n

    def load_skeleton(self, parent, rest):
        p, r = _np(parent, np.int32), _np(rest, np.float32)
        self._check(_lib.art_load_skeleton(self._h, p.shape[0], _ptr(p), _ptr(r)))

    def set_pose(self, axis_angle, R, T):
        aa = axis_angle if hasattr(axis_angle, "data_ptr") else _np(axis_angle, np.float32)
        R = R if hasattr(R, "data_ptr") else _np(R, np.float32)
        T = T if hasattr(T, "data_ptr") else _np(T, np.float32)
        self._check(_lib.art_set_pose(self._h, _ptr(aa), _ptr(R), _ptr(T)))

    def set_camera(self, view: int, W: int, H: int, fx: float, fy: float, cx: float, cy: float, world_to_cam,
                   near: float, far: float):
        M = _np(world_to_cam, np.float32).reshape(12)
        self._check(_lib.art_set_camera(self._h, view, W, H, fx, fy, cx, cy, _ptr(M), near, far))
        self.views[view] = (W, H)

    def load_shader(self, arch: int, cin: int, ch: Sequence[int], cout: int, params, dtype: str = "f32",
                    ach: Sequence[int] = (0, 0)):
        d = NetDesc(arch, cin, (ctypes.c_int * 4)(*(list(ch) + [0] * (4 - len(ch)))), cout,
                    (ctypes.c_int * 2)(*list(ach)))
        p = _np(params, np.float32).reshape(-1)
        self._check(_lib.art_load_shader(self._h, ctypes.byref(d), _ptr(p), p.size, DTYPES[dtype]))

    # ------------------------------------------------------------- rendering
    def render_feature_maps(self, view: int, F_out, A_out=None, F_dtype: str = "f32"):
        self._check(_lib.art_render_feature_maps(self._h, view, _ptr(F_out), DTYPES[F_dtype], _ptr(A_out)))

    def load_sh_features(self, degree: int, coef=None):
        """View-dependent features: coef [n][(degree+1)^2][C] float32 (degree -1: back to plain)."""
        c = None if coef is None else (coef if hasattr(coef, "data_ptr") else _np(coef, np.float32))
        self._check(_lib.art_load_sh_features(self._h, int(degree), _ptr(c)))

    def render_depth(self, view: int, sigma_min: float, depth_out):
        """Depth buffer: entry distance of the first hit denser than sigma_min (+inf where none)."""
        self._check(_lib.art_render_depth(self._h, view, float(sigma_min), _ptr(depth_out)))

    def shade(self, view: int, F, rgba_out, F_dtype: str = "f32"):
        self._check(_lib.art_shade(self._h, view, _ptr(F), DTYPES[F_dtype], _ptr(rgba_out)))

    def render_views(self, views: Sequence[int], F_outs, A_outs=None, F_dtype: str = "f32"):
        nv = len(views)
        vv = (ctypes.c_int * nv)(*views)
        fp = (ctypes.c_void_p * nv)(*[_ptr(f) for f in F_outs])
        ap = None if A_outs is None else (ctypes.c_void_p * nv)(*[_ptr(a) for a in A_outs])
        self._check(_lib.art_render_views(self._h, nv, vv, fp, DTYPES[F_dtype], ap))

    def shade_with_opacity(self, view: int, F, A, rgba_out, F_dtype: str = "f32"):
        self._check(_lib.art_shade_with_opacity(self._h, view, _ptr(F), DTYPES[F_dtype], _ptr(A), _ptr(rgba_out)))

    def render_frame(self, view: int, axis_angle, R, T, rgba_out):
        aa = axis_angle if hasattr(axis_angle, "data_ptr") else _np(axis_angle, np.float32)
        R = R if hasattr(R, "data_ptr") else _np(R, np.float32)
        T = T if hasattr(T, "data_ptr") else _np(T, np.float32)
        self._check(_lib.art_render_frame(self._h, view, _ptr(aa), _ptr(R), _ptr(T), _ptr(rgba_out)))

    def render_frame_async(self, view: int, axis_angle, R, T, rgba_out):
        """art_render_frame_async: queue a frame whose RGBA is copied into the
        host buffer rgba_out (pinned for an asynchronous copy); rgba_out and
        pinned pose tensors must stay unchanged until wait_frames()."""
        aa = axis_angle if hasattr(axis_angle, "data_ptr") else _np(axis_angle, np.float32)
        R = R if hasattr(R, "data_ptr") else _np(R, np.float32)
        T = T if hasattr(T, "data_ptr") else _np(T, np.float32)
        self._check(_lib.art_render_frame_async(self._h, view, _ptr(aa), _ptr(R), _ptr(T), _ptr(rgba_out)))

    def wait_frames(self):
        self._check(_lib.art_wait_frames(self._h))

    def update_voxels(self, features=None, density=None, weights=None):
        self._check(_lib.art_update_voxels(self._h, _ptr(features), _ptr(density), _ptr(weights)))

    def render_backward(self, view: int, F, A, dF, dA, d_features, d_density, d_weights):
        """Accumulate dL/df, dL/dsigma, dL/dw (device FP32 tensors) for the
        current pose and `view`, given the forward's F, A and dL/dF, dL/dA."""
        self._check(_lib.art_render_backward(self._h, view, _ptr(F), _ptr(A), _ptr(dF), _ptr(dA), _ptr(d_features),
                                             _ptr(d_density), _ptr(d_weights)))

    # ------------------------------------------------ learned interval skip
    def load_proposal(self, params):
        """Load the ray-interval proposal MLP (flat FP32, PROPOSAL_PARAMS values)."""
        p = params if hasattr(params, "data_ptr") else _np(params, np.float32).reshape(-1)
        self._check(_lib.art_load_proposal(self._h, _ptr(p), int(p.numel() if hasattr(p, "numel") else p.size)))

    def run_proposal(self, view: int, bins=None, logits=None):
        """Proposal bins [H,W,2] uint8 and/or logits [H,W,128] float (device tensors)."""
        self._check(_lib.art_run_proposal(self._h, view, _ptr(bins), _ptr(logits)))

    def render_labels(self, view: int, labels=None, bins=None):
        """Plain-render training labels [H,W,3] float and label bins [H,W,2] uint8 (device tensors)."""
        self._check(_lib.art_render_labels(self._h, view, _ptr(labels), _ptr(bins)))

    def sort_pairs(self, keys, vals, key_bits: int = 32):
        _check_pairs(keys, vals)
        self._check(_lib.art_sort_pairs(self._h, _ptr(keys), _ptr(vals), int(keys.numel()), key_bits))

    # ------------------------------------------------------------ inspection
    def sync_status(self, raise_on_overflow: bool = True) -> dict:
        s = Stats()
        st = _lib.art_sync_status(self._h, ctypes.byref(s))
        if st != 0 and (raise_on_overflow or st != 4):
            self._check(st)
        return dict(instances=s.instances, degenerate=s.degenerate, overflow_inst=s.overflow_inst,
                    overflow_order=s.overflow_order, kernel_launches=s.kernel_launches,
                    fallback_tiles=s.fallback_tiles, exact_tiles=s.exact_tiles, grid_cells=s.grid_cells,
                    forced_tiles=s.forced_tiles, check_fail_tiles=s.check_fail_tiles, status=st)

    def kernel_times(self, reset: bool = False) -> dict:
        cap = 64
        names = (ctypes.c_char_p * cap)()
        launches = np.zeros(cap, np.int64)
        ms = np.zeros(cap, np.float64)
        count = ctypes.c_int(0)
        self._check(_lib.art_get_kernel_times(self._h, cap, ctypes.cast(names, ctypes.c_void_p), _ptr(launches),
                                              _ptr(ms), ctypes.byref(count), int(reset)))
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(count.value, cap))}

    def debug_buffer(self, which: int, dtype) -> np.ndarray:
        need = ctypes.c_int64(0)
        self._check(_lib.art_debug_buffer(self._h, which, None, 0, ctypes.byref(need)))
        out = np.zeros(max(need.value, 1) // np.dtype(dtype).itemsize, dtype)
        self._check(_lib.art_debug_buffer(self._h, which, _ptr(out), out.nbytes, ctypes.byref(need)))
        return out

    def debug_hits(self, view: int, cap: int = 64):
        W, H = self.views[view]
        count = np.zeros((H, W), np.int32)
        ids = np.zeros((H, W, cap), np.uint32)
        t0 = np.zeros((H, W, cap), np.float32)
        t1 = np.zeros((H, W, cap), np.float32)
        F = np.zeros((H, W, self.C), np.float32)
        A = np.zeros((H, W), np.float32)
        self._check(_lib.art_debug_hits(self._h, view, cap, _ptr(count), _ptr(ids), _ptr(t0), _ptr(t1), _ptr(F),
                                        _ptr(A)))
        return dict(count=count, ids=ids, t0=t0, t1=t1, F=F, A=A)


def render_features(renderer: "Renderer", view: int, features, density, weights, pose):
    """Differentiable render of one view: (F [H,W,C], A [H,W]) as functions of
    the voxel features [n,C], densities [n] and skinning weights [n,4] (FP32
    CUDA tensors), through art_update_voxels + art_set_pose +
    art_render_feature_maps; the backward calls art_render_backward.
    ``pose`` is (axis_angle [J,3], R [3], T [3])."""
    return _RenderFn.apply(features, density, weights, renderer, view, pose)


def _make_render_fn():
    import torch

    class RenderFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, features, density, weights, renderer, view, pose):
            features, density, weights = features.contiguous(), density.contiguous(), weights.contiguous()
            renderer.update_voxels(features, density, weights)
            renderer.set_pose(*pose)
            W, H = renderer.views[view]
            F = torch.empty((H, W, features.shape[1]), dtype=torch.float32, device=features.device)
            A = torch.empty((H, W), dtype=torch.float32, device=features.device)
            renderer.render_feature_maps(view, F, A, "f32")
            ctx.save_for_backward(F, A)
            ctx.renderer, ctx.view, ctx.shapes = renderer, view, (features.shape, density.shape, weights.shape)
            return F, A

        @staticmethod
        def backward(ctx, dF, dA):
            F, A = ctx.saved_tensors
            sf, sd, sw = ctx.shapes
            gf = torch.zeros(sf, dtype=torch.float32, device=F.device)
            gd = torch.zeros(sd, dtype=torch.float32, device=F.device)
            gw = torch.zeros(sw, dtype=torch.float32, device=F.device)
            dF = torch.zeros_like(F) if dF is None else dF.contiguous().float()
            dA = torch.zeros_like(A) if dA is None else dA.contiguous().float()
            ctx.renderer.render_backward(ctx.view, F, A, dF, dA, gf, gd, gw)
            return gf, gd, gw, None, None, None

    return RenderFn


class _LazyFn:
    fn = None

    def apply(self, *a):
        if _LazyFn.fn is None:
            _LazyFn.fn = _make_render_fn()
        return _LazyFn.fn.apply(*a)


_RenderFn = _LazyFn()

SORT_STATIC_MAX_PAIRS = 1 << 20


def _check_pairs(keys, vals):
    """keys and vals of a device sort: contiguous 4-byte CUDA tensors of the
    same length on the current device."""
    import torch
    for t in (keys, vals):
        if not (t.is_cuda and t.element_size() == 4 and t.is_contiguous()):
            raise ValueError("sort: keys and vals must be contiguous 4-byte CUDA tensors")
        if t.device.index != torch.cuda.current_device():
            raise ValueError("sort: keys and vals must be on the current CUDA device")
    if keys.numel() != vals.numel():
        raise ValueError(f"sort: {keys.numel()} keys but {vals.numel()} values")


def sort_pairs_static(keys, vals, key_bits: int = 32, stream=None) -> int:
    """art_sort_pairs_static: the radix sort without any device allocation
    (scratch in a fixed array inside the library; see include/artemis.h).
    Returns the library status (0 = ART_OK)."""
    import torch
    _check_pairs(keys, vals)
    s = torch.cuda.current_stream() if stream is None else stream
    return int(_lib.art_sort_pairs_static(_ptr(keys), _ptr(vals), int(keys.numel()), key_bits,
                                          ctypes.c_void_p(s.cuda_stream)))


def flat_params(layers) -> np.ndarray:
    """Concatenate [(w [Cout,k,k,Cin], b [Cout]), ...] into the art_load_shader layout."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for w, b in layers])
