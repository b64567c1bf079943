/*
 * artemis.h - C ABI of the GB300 rendering path of ARTEMIS neural animals
 * (arXiv 2202.05628, Sec. 3.1 "Animatable Neural Volumes").
 *
 * The library renders, per frame, the paper's pipeline: skeleton pose ->
 * linear-blend-skinning warp of the canonical octree's leaf voxels (Eq. 4) ->
 * per-pixel indexing of the warped voxels -> front-to-back compositing of the
 * voxel features and densities into the feature map F and coarse opacity map
 * A (Eq. 5-6, early stop) -> neural shading network -> RGBA ("Neural
 * Shading").  The call sequence follows the order stated in Sec. 5
 * ("Implementations Details"): pose, LBS, indexing, tracing, shading.
 *
 * Conventions (all calls):
 *   - Every call returns an art_status; ART_OK is 0.  On failure the context
 *     keeps a message readable with art_last_error().  No C++ exception
 *     crosses this boundary.
 *   - Work is enqueued asynchronously on the context's CUDA stream (borrowed,
 *     never destroyed by the library).  Calls that take HOST output pointers
 *     synchronise the stream before returning; calls with DEVICE outputs do
 *     not.  art_sync_status() synchronises and reports device-side errors.
 *   - Pointer arguments may be host or device memory unless stated; the
 *     library tells them apart with cudaPointerGetAttributes.  Inputs are
 *     copied into library-owned device memory; the caller keeps ownership of
 *     everything it passes.  A pageable host input may be reused as soon as
 *     the call returns; a page-locked (pinned) host input, and any device
 *     input, is read asynchronously and must stay unchanged until the stream
 *     has passed the call.
 *   - All arrays are dense, row-major, with the layouts given per argument.
 *   - A context is not thread-safe; use one per host thread / stream.
 */
#ifndef ARTEMIS_H
#define ARTEMIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct art_ctx art_ctx;

typedef enum {
  ART_OK = 0,
  ART_ERR_INVALID_ARG = 1, /* bad size, null pointer, out-of-range index */
  ART_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  ART_ERR_OOM = 3,         /* device allocation failed */
  ART_ERR_OVERFLOW = 4,    /* a device-side capacity was exceeded (see art_stats) */
  ART_ERR_STATE = 5,       /* call out of order (e.g. render before load) */
  ART_ERR_UNSUPPORTED = 6  /* a configuration this build does not provide */
} art_status;

/* element types */
enum { ART_F32 = 0, ART_BF16 = 1, ART_F16 = 2, ART_FP8 = 3 };

/* shading network architectures (Sec. 3.1 "Neural Shading"; the single-branch
 * "Light" form of Sec. 6 "Runtime Analysis", RGB and alpha from one net) */
enum { ART_NET_TINY = 0, ART_NET_UNET = 1, ART_NET_TWO_BRANCH = 2 };

/* ---------------------------------------------------------------- context */

/* Create a context bound to cuda_stream (a cudaStream_t; NULL = legacy
 * default stream) on the current device.  *out receives the context. */
art_status art_create(art_ctx** out, void* cuda_stream);

/* Release every device buffer of the context.  NULL is ignored. */
void art_destroy(art_ctx* ctx);

/* Message of the last failed call; owned by ctx, valid until the next call. */
const char* art_last_error(const art_ctx* ctx);

/* Rebind the context to another stream (cudaStream_t). */
art_status art_set_stream(art_ctx* ctx, void* cuda_stream);

/* ------------------------------------------------------------------ scene */

/*
 * Load the canonical octree's leaf voxels and their feature look-up table
 * (Sec. 3.1 "Octree Feature Indexing": voxel array P and FLUT F; skinning
 * weights of "Rigging and Deformation").
 *   n            number of leaf voxels (1 .. 2^31-1)
 *   depth        octree depth; voxel side h = extent / 2^depth (depth <= 16)
 *   origin[3]    world position of the octree cube's minimum corner (metres)
 *   extent       side of the octree cube (metres, > 0)
 *   ijk          [n][3] uint16 integer voxel coordinates, each < 2^depth;
 *                voxel i is the cube origin + (ijk_i + [0,1]^3) h
 *   joint_idx    [n][4] uint8 joint of each skinning weight (< J of the skeleton)
 *   weights      [n][4] float skinning weights (used as given: the library
 *                does not renormalise)
 *   features     [n][C] float features (FP32); stored on the device in
 *                storage_dtype (ART_F32, ART_BF16 or ART_F16, rounded to
 *                nearest even)
 *   C            feature channels: 4, 8, 16 or 32
 *   density      [n] float density sigma_i (1/m, >= 0)
 * Replaces any previously loaded octree.
 */
art_status art_load_octree(art_ctx* ctx, int64_t n, int depth, const float origin[3], float extent,
                           const uint16_t* ijk, const uint8_t* joint_idx, const float* weights,
                           const float* features, int C, int storage_dtype, const float* density);

/*
 * Load the skeleton (Sec. 3.1: S = {r, R, T} over J joints).
 *   J         number of joints, 1 .. 64
 *   parent    [J] int32 parent joint, parent[0] = -1 and parent[j] < j
 *   rest_pos  [J][3] float joint positions in the canonical pose (metres);
 *             canonical joint rotations are zero, so M^c_j = [I | rest_j]
 */
art_status art_load_skeleton(art_ctx* ctx, int J, const int32_t* parent, const float* rest_pos);

/*
 * Set the target pose S_t and warp every voxel (Eq. 4): forward kinematics
 * M^t_j = M^t_parent(j) [Rod(r_j) | rest_j - rest_parent(j)], the root
 * premultiplied by [Rod(R) | T]; G_j = M^t_j (M^c_j)^-1; per voxel the blended
 * A_i = sum_k w_ik G_{j_ik}, its inverse, and its warped bounding data.
 *   axis_angle  [J][3] joint rotations r (axis-angle, radians)
 *   R[3], T[3]  global rotation (axis-angle) and translation (metres)
 * Voxels whose blended 3x3 part has det < 1e-3 are dropped from rendering and
 * counted in art_stats.degenerate.
 */
art_status art_set_pose(art_ctx* ctx, const float* axis_angle, const float R[3], const float T[3]);

/*
 * Set camera `view` (0 .. 7): the camera whose pixel rays are cast through
 * the warped volume (Sec. 3.1 "Dynamic Volume Rendering": a ray per pixel,
 * composited front to back, Eq. 5-6).  Pinhole with intrinsics fx, fy, cx, cy
 * in pixels, world_to_cam[12] the 3x4 row-major [R | t] (x_cam = R x + t; +x
 * right, +y down, +z forward), image W x H (1 .. 8192 each).  Pixel (x, y) is
 * sampled at its centre; its ray is o = -R^T t, d = R^T dc / |R^T dc| with
 * dc = ((x+1/2-cx)/fx, (y+1/2-cy)/fy, 1).  znear < zfar are distances along
 * the unit ray.  world_to_cam may be host or device memory (copied); the
 * call is synchronous with respect to the host.  Errors: ART_ERR_INVALID_ARG
 * for a view out of range, sizes out of range, non-positive focal lengths or
 * znear >= zfar; ART_ERR_UNSUPPORTED when the image has too many screen
 * tiles for the 32-bit depth keys.
 */
art_status art_set_camera(art_ctx* ctx, int view, int W, int H, float fx, float fy, float cx, float cy,
                          const float world_to_cam[12], float znear, float zfar);

/* --------------------------------------------------------------- rendering */

/*
 * Render the feature map F and coarse opacity map A of `view` under the
 * current pose (Eq. 5-6): each pixel ray is intersected exactly with every
 * warped voxel (the parallelepiped A_i * cube_i) that the screen-tile index
 * lists for its tile; hits are composited front to back in order of entry
 * distance, F = sum_i T_i (1 - exp(-sigma_i delta_i)) f_i with
 * T_i = prod_{j<i} exp(-sigma_j delta_j), stopping after the hit at which
 * T < tau (art_config.tau, default 1e-4); A = 1 - T.
 *   F_out   [H][W][C] in F_dtype (ART_F32 or ART_BF16); device or host
 *   A_out   [H][W] float; device or host (may be NULL)
 * Background pixels get F = 0, A = 0.
 */
art_status art_render_feature_maps(art_ctx* ctx, int view, void* F_out, int F_dtype, float* A_out);

/*
 * View-dependent features (Eq. 2 and the canonical ray direction of
 * Sec. 3.1): each voxel's feature becomes a set of spherical-harmonics
 * coefficient vectors k_h (h = l^2 + l + m, l <= degree), and a hit's
 * feature S = sum_h k_h Y_h(R_i^T d) with Y_h the real orthonormal harmonics
 * (no Condon-Shortley phase in the real basis), d the unit pixel ray and
 * R_i the rotation factor of voxel i's blended transform (polar
 * decomposition).  Later art_render_feature_maps / art_render_frame calls
 * composite these features (plain traversal only).
 *   degree  0 .. 3; -1 returns to the per-voxel features of art_load_octree
 *   coef    [n][(degree+1)^2][C] float, host or device; copied
 * Errors: ART_ERR_STATE before art_load_octree, ART_ERR_UNSUPPORTED for a
 * degree above 3; art_render_backward and the learned skip then return
 * ART_ERR_UNSUPPORTED.  A new art_load_octree returns to the plain features.
 */
art_status art_load_sh_features(art_ctx* ctx, int degree, const float* coef);

/*
 * Depth buffer of `view` under the current pose (Sec. 3.1 "Hybrid
 * Rendering": each pixel ray is traced to the first voxel whose density is
 * larger than a threshold, whose distance becomes the pixel's depth): the
 * entry distance t0 (from the camera centre along the unit pixel ray,
 * clipped to [znear, zfar]) of the first hit, in order of entry distance,
 * with sigma > sigma_min among all of the ray's hits — not cut by the early
 * stop of the compositing — and +infinity where the ray meets none.
 *   sigma_min  density threshold (>= 0; 1/m)
 *   depth_out  [H][W] float; device or host
 * Errors: ART_ERR_STATE before the camera or the pose is set,
 * ART_ERR_INVALID_ARG for a null output or a negative threshold.
 */
art_status art_render_depth(art_ctx* ctx, int view, float sigma_min, float* depth_out);

/* ---------------------------------------------------------- differentiation */

/*
 * Replace, in place, the voxel features ([n][C] FP32, converted to the storage
 * dtype), densities ([n]) and/or skinning weights ([n][4]) of the loaded
 * octree; NULL keeps an array.  Host or device pointers.  After new densities
 * or weights, call art_set_pose again before rendering (the pose's per-voxel
 * records carry both).
 */
art_status art_update_voxels(art_ctx* ctx, const float* features, const float* density, const float* weights);

/*
 * Gradients of a loss L through art_render_feature_maps of `view` under the
 * current pose, with respect to the voxel features f, densities sigma and
 * skinning weights w (Eq. 4-6; the paper optimises the feature table end to
 * end, Sec. 3.1 "Training").  Each ray is re-traced (per-ray recomputation;
 * no per-sample state is stored): hits, their order and the early-stop index
 * are recomputed exactly as in the forward and held fixed.
 *   F, A        the forward's outputs for this view and pose: F [H][W][C]
 *               FP32, A [H][W]
 *   dF, dA      dL/dF [H][W][C] and dL/dA [H][W] (dA may be NULL = 0); pixels
 *               with zero upstream gradient are skipped
 *   d_features  [n][C], d_density [n], d_weights [n][4]: FP32 outputs that
 *               are ACCUMULATED into (zero them first), so that calls for
 *               several views sum
 * All arrays are DEVICE memory.  Gradients accumulate with atomics, so their
 * last bits depend on the order in which rays finish.
 */
art_status art_render_backward(art_ctx* ctx, int view, const float* F, const float* A, const float* dF,
                               const float* dA, float* d_features, float* d_density, float* d_weights);

/* ----------------------------------------------------------------- shading */

typedef struct {
  int arch;     /* ART_NET_TINY, ART_NET_UNET or ART_NET_TWO_BRANCH */
  int cin;      /* input channels (= C of the feature map) */
  int ch[4];    /* TINY: ch[0] hidden width; UNET, TWO_BRANCH: widths of the 4 levels (appearance branch) */
  int cout;     /* output channels (4 = RGBA; TWO_BRANCH: 4) */
  int ach[2];   /* TWO_BRANCH: widths of the opacity branch's 2 levels */
} art_net_desc;

/*
 * Load the shading network G (Sec. 3.1 "Neural Shading").
 * TINY: conv3x3 cin->ch0, ReLU, conv3x3 ch0->ch0, ReLU, conv3x3 ch0->cout,
 *       sigmoid.
 * UNET: 4 levels; per level two conv3x3 + ReLU; 2x2 max-pool between
 *       levels; decoder: nearest x2 upsample, channel concat [upsampled,
 *       skip], two conv3x3 + ReLU; head conv1x1 -> cout, sigmoid.
 * TWO_BRANCH: the paper's two-branch G (Sec. 3.1 "Neural Shading", Fig. 4):
 *       an appearance UNET (widths ch) from F to the texture image I_f
 *       (3 channels, sigmoid head), then an opacity U-Net of 2 levels
 *       (widths ach) from [A, I_f] (4 channels, the coarse opacity map
 *       first) to alpha (1 channel, sigmoid head); RGBA = [I_f, alpha].
 *       params: the appearance layers, then the opacity layers.  Shaded
 *       with art_shade_with_opacity (it needs A); F32 or BF16 only.
 * params: float array, for every layer in execution order its weights
 *   [Cout][k][k][Cin] followed by its bias [Cout]; n_params must match.
 * compute_dtype: ART_F32 (CUDA-core FP32), ART_BF16 (tensor cores, BF16
 *   operands, FP32 accumulation) or ART_FP8 (U-Net only: E4M3 operands,
 *   FP32 accumulation, per-output-channel weight scales max|w_co| / 448 and
 *   per-tensor activation scales; each art_shade quantises with the scales
 *   measured (max |value| / 448) on the previous call and records its own,
 *   and the first call after loading runs the network twice to calibrate).
 *   BF16 and FP8 networks take a BF16 feature map.
 */
art_status art_load_shader(art_ctx* ctx, const art_net_desc* desc, const float* params, int64_t n_params,
                           int compute_dtype);

/*
 * Shade feature map F ([H][W][cin] in F_dtype, H and W of `view`, both
 * multiples of 8 for UNET) into rgba_out [H][W][cout] float (device or host).
 */
art_status art_shade(art_ctx* ctx, int view, const void* F, int F_dtype, float* rgba_out);

/*
 * Shade with a network that also reads the coarse opacity map A [H][W]
 * float (host or device; Eq. 5's accumulated alpha, as written by
 * art_render_feature_maps): the TWO_BRANCH network (Sec. 3.1 "Neural
 * Shading").  Other networks ignore A.  F and rgba_out as in art_shade.
 */
art_status art_shade_with_opacity(art_ctx* ctx, int view, const void* F, int F_dtype, const float* A, float* rgba_out);

/*
 * Several views of the current pose in one pass (the paper's stereo VR
 * pairs and multi-view rendering, Sec. 5-6): one projection per view into
 * one tile space (the views' screen tiles end to end), one scan, scatter and
 * sort of all their instances, one composite walk over all their tiles.
 *   nv       1 .. 8 distinct views (set with art_set_camera), listed in views
 *   F_out    nv DEVICE arrays [H_k][W_k][C] in F_dtype (F32 or BF16)
 *   A_out    NULL, or nv DEVICE arrays [H_k][W_k] float (entries may be NULL)
 * Each view's maps equal those of art_render_feature_maps up to the
 * regrouping of FP32 sums (the joint tile space has its own depth-key
 * layout, hence other segment cuts).  With the learned skip or SH features
 * configured, the views are rendered one after another instead.
 */
art_status art_render_views(art_ctx* ctx, int nv, const int* views, void* const* F_out, int F_dtype,
                            float* const* A_out);

/* One frame of one view: art_set_pose + art_render_feature_maps into
 * library-owned buffers + art_shade.  rgba_out as in art_shade. */
art_status art_render_frame(art_ctx* ctx, int view, const float* axis_angle, const float R[3], const float T[3],
                            float* rgba_out);

/*
 * The frame of art_render_frame with a HOST rgba_out ([H][W][cout] float),
 * without waiting for it (a frame loop that overlaps frame k's copy to the
 * host and the host's queueing of frame k + 1 with the GPU's work; Sec. 5's
 * per-frame order pose -> LBS -> tracing -> shading is unchanged).  The call
 * queues the pose upload, the render and the network into one of two
 * library-owned device slots, then the slot's copy to rgba_out on a second
 * stream, and returns.  At most two frames are in flight: a third call first
 * waits for the oldest frame's copy.  rgba_out, and the pose arrays when they
 * are pinned host memory (read when their copy runs), must stay valid and
 * unchanged until art_wait_frames returns; rgba_out should be pinned (a
 * pageable buffer makes the copy synchronous).  Errors of the queued work
 * are reported by art_wait_frames (or a later call); ART_ERR_INVALID_ARG for
 * a device rgba_out.
 */
art_status art_render_frame_async(art_ctx* ctx, int view, const float* axis_angle, const float R[3], const float T[3],
                                  float* rgba_out);

/* Waits until every frame queued by art_render_frame_async has reached its
 * host buffer and the library's stream is idle; returns the first error. */
art_status art_wait_frames(art_ctx* ctx);

/* ------------------------------------------- learned ray-interval proposal */

/*
 * A small MLP that predicts, per camera ray, the depth interval in which the
 * ray's composite takes its mass, so that compositing can skip the rest
 * (project addition; the paper's nearest passage is the early-stop rule of
 * Sec. 3.1 "Dynamic Volume Rendering").
 *   input x (107) = [the 72 joint axis-angles of the current pose (J = 24),
 *     the unit world direction of the ray, sin(2^k pi u), k < 8, cos(2^k pi u),
 *     sin(2^k pi v), cos(2^k pi v)], u = (x + 1/2) / W, v = (y + 1/2) / H
 *   layers 107 -> 64 -> 64 -> 64 -> 64 (ReLU) -> 128 logits, BF16 operands,
 *     FP32 accumulation (tensor cores), FP32 biases
 *   bins bn = argmax logits[0:64], bf = argmax logits[64:128] (first index on
 *     ties) over 64 uniform bins of [znear, zfar] of the view: the interval
 *     [znear + bn D, znear + (bf + 1) D], D = (zfar - znear) / 64; bf < bn is
 *     empty.  Each 8 x 4 screen tile takes the union of its rays' non-empty
 *     intervals (bins min bn .. max bf, widened by config.margin; empty when
 *     all are empty), and its rays composite the hits with t1 >= the lower end
 *     and t0 <= the upper end, in the plain order with the plain stop rule.
 * Coarse check: each voxel adds sigma_i 2 r_i (a bound of its optical depth on
 * any ray) to every depth bin its distance range |c_i - o| -+ r_i overlaps, in
 * every screen tile it covers.  A ray's lost mass is bounded by (1 - exp(-sum
 * of its tile's bins before the tile's interval)) + (1 - exp(-sum after it))
 * (empty: the first term over all bins; the transmittance after the interval
 * is bounded by 1).  The check runs with the proposal, before compositing: a
 * tile whose bound exceeds config.max_missed is composited over its whole
 * list instead of the interval, in the same pass (the fallback), and counted
 * in art_stats.check_fail_tiles.
 */

#define ART_PROPOSAL_PARAMS 27712 /* 64*107+64 + 3*(64*64+64) + 128*64+128 */

/* Load the proposal MLP: params (FP32, host or device) = W0 [64][107], b0,
 * W1 [64][64], b1, W2, b2, W3, b3, W4 [128][64], b4 (y = W x + b);
 * n_params must be ART_PROPOSAL_PARAMS.  The skeleton must have 24 joints. */
art_status art_load_proposal(art_ctx* ctx, const float* params, int64_t n_params);

/*
 * Run the proposal for every pixel of `view` under the current pose:
 * bins_out [H][W][2] uint8 (bn, bf) and/or logits_out [H][W][128] float;
 * DEVICE arrays, either may be NULL.
 */
art_status art_run_proposal(art_ctx* ctx, int view, uint8_t* bins_out, float* logits_out);

/*
 * Training labels from the plain renderer, for the current pose and `view`:
 *   labels_out [H][W][3] float: (min t1, max t0) over the composited hits whose
 *     weight T_i alpha_i exceeds 1e-6, and the transmittance just after the
 *     last of them; (+inf, -inf, 1) when there is none
 *   bins_out [H][W][2] uint8: the label interval (bn, bf) with
 *     bn = min(bin(lo), the largest b with 1 - exp(-sum of the tile's bins
 *     before b) <= 0.4 max_missed), bf = the smallest b >= bin(hi) with
 *     Ts (1 - exp(-sum after b)) <= 0.4 max_missed (no significant hit:
 *     bin(lo) = 63, bin(hi) = 0, Ts = 1): it keeps every significant hit and
 *     passes the coarse check
 * DEVICE arrays, either may be NULL.  F and A are not written.
 */
art_status art_render_labels(art_ctx* ctx, int view, float* labels_out, uint8_t* bins_out);

/* ------------------------------------------------------------ configuration */

typedef struct {
  float tau;               /* early-stop transmittance (default 1e-4) */
  int64_t instance_cap;    /* capacity of (tile, voxel) instances; 0 = 4 n + 65536 */
  int tile_log2;           /* log2 of the screen-tile width: 3 (8 x 4 pixel tiles, the only size built) */
  int profile;             /* 1: time every kernel with CUDA events (art_get_kernel_times) */
  int skip;                /* ART_SKIP_PLAIN (default) or ART_SKIP_LEARNED: composite each ray only
                              over the depth interval its proposal predicts (art_load_proposal) */
  float max_missed;        /* learned skip: coarse-check threshold of lost transmittance mass
                              (0 = default 1e-3); a tile above it is traversed in full */
  int margin;              /* learned skip: bins added on both sides of the predicted interval (default 0) */
  int segment;             /* composite: a tile's list is walked in segments of about this many entries by
                              separate warps and merged front to back (0 = default 256; >= 32) */
  int index;               /* ART_INDEX_BOXES (default): every warped voxel is its exact parallelepiped;
                              ART_INDEX_GRID: the paper's per-frame index (Sec. 3.1 "Dynamic Volume
                              Rendering"): each warped centre is snapped to the cell of the leaf lattice
                              (canonical origin, leaf size h) that holds it, the smallest voxel id of a
                              cell survives, and each occupied cell renders as its axis-aligned leaf box
                              with its survivor's feature and density (forward only; no SH features) */
  int no_subpixel;         /* BF16 U-Net: 0 (default) runs each decoder block's first convolution over
                              [up2(d) | e] in its sub-pixel form (per output phase, 9 taps of e and 4 taps
                              of the low-resolution d with summed weights, which are rounded to BF16 once);
                              1 runs it over the 2x2-replicated concatenation (the same function, another
                              rounding of the weights, more work) */
} art_config;

enum { ART_INDEX_BOXES = 0, ART_INDEX_GRID = 1 };

#define ART_SKIP_PLAIN 0
#define ART_SKIP_LEARNED 1

/* Replace the configuration (NULL restores the defaults). */
art_status art_set_config(art_ctx* ctx, const art_config* cfg);

typedef struct {
  int64_t instances;       /* (tile, voxel) instances of the last render */
  int64_t degenerate;      /* voxels dropped at the last pose (det < 1e-3) */
  int64_t overflow_inst;   /* instances that did not fit instance_cap */
  int64_t overflow_order;  /* pixels whose hits could not all be put in order: more than
                              1024 hits on one ray (result may be out of order) */
  int64_t kernel_launches; /* kernels launched by this context so far */
  int64_t fallback_tiles;  /* tiles of the last render walked again by the sequential walk: a pixel's
                              stop (T < tau) fell inside a later segment of the split walk */
  int64_t exact_tiles;     /* tiles of the last render walked again exactly because a pixel
                              had more pending hits than its 16-entry reorder buffer holds */
  int64_t grid_cells;      /* ART_INDEX_GRID: occupied lattice cells of the last pose (the survivors) */
  int64_t forced_tiles;    /* learned skip: tiles of the last render whose coarse bound alone fixes the
                              walk (the whole range, or nothing), rendered without a prediction */
  int64_t check_fail_tiles; /* learned skip: predicted tiles of the last render that failed the coarse
                               check, composited over their whole list instead of the interval */
} art_stats;

/* Synchronise the stream, fill *out (may be NULL) and return
 * ART_ERR_OVERFLOW if a device-side capacity was exceeded since the last
 * call (the flags are then cleared), else ART_OK. */
art_status art_sync_status(art_ctx* ctx, art_stats* out);

/*
 * Per-kernel timing (config.profile = 1): for up to `cap` kernels, names[i]
 * (static strings), launches[i] and total milliseconds[i] accumulated since
 * the last reset.  *count receives the number of distinct kernels.  The
 * stream is synchronised.  reset != 0 clears the accumulators afterwards.
 */
art_status art_get_kernel_times(art_ctx* ctx, int cap, const char** names, int64_t* launches, double* ms,
                                int* count, int reset);


/* ---------------------------------------------------------- building blocks */

/*
 * Stable LSD radix sort of (key, value) pairs by the low key_bits bits of
 * the keys (key_bits in {8, 16, 24, 32}).  Given the screen-tile instances
 * (tile << depth_bits | depth quantum, voxel id) in voxel order it yields the
 * (tile, depth) order that the render computes internally with a
 * most-significant-digit sort (tile buckets, then depth bins per tile).
 * keys, vals: DEVICE arrays of n uint32 each
 * (0 <= n <= 2^31 - 1), sorted in place.  Scratch (2 n pairs plus histograms)
 * is allocated by the context on first use and kept for later calls.
 */
art_status art_sort_pairs(art_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n, int key_bits);

/*
 * The same stable radix sort as art_sort_pairs, for callers that must not
 * allocate device memory while they run: a VR or game-engine frame loop that
 * cannot afford the device-wide synchronisation and the unbounded latency a
 * cudaMalloc/cudaFree may incur in the middle of a frame, and hosts whose
 * device memory is owned by a pool allocator (PyTorch's caching allocator, an
 * engine's arena) with a fixed budget.  It takes no context and allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  (The
 * paper has no counterpart; this is an interface choice of the library.)
 *   keys, vals   DEVICE arrays of n uint32 each, sorted in place by the low
 *                key_bits bits of the keys (key_bits in {8, 16, 24, 32})
 *   n            0 .. ART_SORT_STATIC_MAX_PAIRS; larger n returns
 *                ART_ERR_INVALID_ARG without launching anything
 *   cuda_stream  cudaStream_t the work is enqueued on (asynchronous)
 * Scratch: a fixed device array of about 8.6 MB inside the library (room for
 * ART_SORT_STATIC_MAX_PAIRS pairs plus histograms), held by every GPU that
 * loads the library until the process exits.  Every call rewrites the parts
 * of it that it reads, so no state carries over between calls; but all calls
 * share it, so calls that overlap on the GPU (other streams, other host
 * threads) race: order them on one stream or with events.
 * keys and vals must be device (or managed) memory of the current device,
 * else ART_ERR_INVALID_ARG is returned without launching.
 * The first call on each device (and again after a cudaDeviceReset) looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  If a CUDA error
 * is already pending when the call starts (left by an earlier call), it
 * returns ART_ERR_CUDA without launching and leaves that error pending.
 * Returns ART_ERR_CUDA if the lookup or a launch fails.
 */
#define ART_SORT_STATIC_MAX_PAIRS (1 << 20)
art_status art_sort_pairs_static(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits, void* cuda_stream);

/* ------------------------------------------------------------ inspection */

/* internal buffers readable with art_debug_buffer (layouts as stated) */
enum {
  ART_BUF_JOINT_G = 0,   /* [J][12] float: G_j = M^t_j (M^c_j)^-1 of the last pose */
  ART_BUF_VOXEL_REC = 1, /* [n][16] float: rows of A_lin^-1 / h with cw (3 x 4), then sigma, valid, 0, 0 */
  ART_BUF_VOXEL_GEO = 2, /* [n][16] float: (cw, r), half axes A_lin e_a h/2 (3 x (xyz, 0)) */
  ART_BUF_RECT = 3,      /* [n][4] int16: pixel rectangle x0, y0, x1, y1 of the last render */
  ART_BUF_DEPTHKEY = 4,  /* [n] uint32: depth quantum of the last render */
  ART_BUF_KEYS = 5,      /* [instances] uint32 sorted keys (tile << depth_bits | depth) */
  ART_BUF_VALS = 6,      /* [instances] uint32 voxel ids in key order */
  ART_BUF_RANGES = 7,    /* [tiles][2] uint32 [start, end) of each tile */
  ART_BUF_FP8_SCALES = 8, /* [11] float: FP8 network activation scales used by the next call */
  ART_BUF_ACTIVATIONS = 9, /* bytes of the tensor-core U-Net's activation arena after the last art_shade:
                             NHWC tensors, each padded to 256 bytes.  FP8: E4M3 codes of input, e0a,
                             cat0, p0, e1a, cat1, p1, e2a, cat2, p2, e3a, d2a, d1a, d0a; BF16: the same
                             tensors without the input.  cat = [upsampled decoder | encoder] */
  ART_BUF_BINS = 10,      /* [H][W][2] uint8: proposal bins of the last learned-skip render (tiles
                             without instances are not predicted) */
  ART_BUF_FALLBACK = 11,  /* [check_fail_tiles] uint32: tiles of the last learned-skip render that failed
                             the coarse check */
  ART_BUF_TAU_HIST = 12   /* [tiles][64] float: coarse optical-depth bound per (tile, depth bin) of the
                             last learned-skip or label render */
};

/*
 * Copy an internal buffer of the last pose / render to host memory dst
 * (capacity `bytes`).  *needed receives the byte size (call with dst NULL to
 * query).  Synchronises the stream.
 */
art_status art_debug_buffer(art_ctx* ctx, int which, void* dst, int64_t bytes, int64_t* needed);

/*
 * Re-render `view` recording, per pixel, the composited hits in front-to-back
 * order: count [H][W] int32 (number of composited hits, may exceed cap),
 * ids [H][W][cap] uint32, t0/t1 [H][W][cap] float (ray parameters of entry
 * and exit).  All four are HOST arrays.  Also writes F ([H][W][C] float,
 * host, may be NULL) and A ([H][W] float, host, may be NULL).
 */
art_status art_debug_hits(art_ctx* ctx, int view, int cap, int32_t* count, uint32_t* ids, float* t0, float* t1,
                          float* F, float* A);

#ifdef __cplusplus
}
#endif
#endif /* ARTEMIS_H */
