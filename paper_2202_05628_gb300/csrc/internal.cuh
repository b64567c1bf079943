// Internal declarations of the GB300 ARTEMIS rendering library.
// Not part of the public ABI (include/artemis.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/artemis.h"

namespace art {

constexpr int kMaxJoints = 64;
constexpr int kMaxViews = 8;
constexpr int kOpacityPad = 32;  // two-branch network: channels of the opacity branch's packed input [A, I_f, 0 ...]
constexpr float kDetMin = 1e-3f;   // blended transforms below this are dropped
constexpr float kZMin = 1e-6f;     // corners must lie in front of the camera
constexpr float kBboxPad = 2e-3f;  // conservative pixel-bbox growth (pixels)

// Device status words (uint64 counters).
enum StatusWord {
  kStInstances = 0,     // instances emitted by the last binning
  kStDegenerate = 1,    // voxels dropped at the last pose
  kStOverflowInst = 2,  // instances beyond capacity (cumulative until cleared)
  kStOverflowOrder = 3, // reorder-buffer overflows (cumulative until cleared)
  kStTcError = 4,       // tensor-core convolution CTAs that timed out waiting
  kStFallback = 5,      // tiles queued for the full traversal (last render)
  kStItems = 8,         // composite segments planned (last render)
  kStMulti = 9,         // tiles split into two or more segments
  kStNext = 10,         // next segment to walk (work counter)
  kStNextMerge = 11,    // next split tile to merge (work counter)
  kStRmax = 12,         // largest voxel bounding radius of the last pose (float bits)
  kStReserved13 = 13,   // (reserved)
  kStSortTiles = 14,    // binning: tiles whose bucket needs sorting
  kStSortNext = 15,     // binning: next bucket to sort (work counter)
  kStSortBig = 16,      // binning: buckets sorted by a whole block
  kStSortBigNext = 17,  // binning: next such bucket (work counter)
  kStScanTicket = 18,   // binning: blocks of the tile scan started (their order)
  kStScanError = 19,    // binning: tile-scan blocks that timed out waiting for a predecessor
  kStActiveGroups = 20, // binning: groups of four consecutive tiles with instances (listed in d_agroups)
  kStExactQ = 21,       // composite: tiles queued for the exact re-walk (a pixel's reorder buffer overflowed)
  kStGridCells = 22,    // lattice index: occupied cells of the last pose
  kStPredGroups = 23,   // learned skip: tile groups holding a tile whose interval the proposal predicts
  kStForcedTiles = 24,  // learned skip: tiles walked in full (or not at all) without a prediction
  kStCheckFail = 25,    // learned skip: predicted tiles that failed the coarse check, walked in full (listed in d_fbq2)
  kStWords = 26
};

// Per-view camera, with host-precomputed ray frame.
struct ViewParams {
  int W, H;
  float fx, fy, cx, cy;
  float R[9];      // world_to_cam rotation (row-major)
  float t[3];
  float o[3];      // camera centre -R^T t (FP32 rounding of the FP64 value)
  float o_lo[3];   // its rounding error: o + o_lo is the centre to ~48 bits
  float znear, zfar;
  int tiles_x, tiles_y;
  int tile_w, tile_h;  // screen tile size in pixels (powers of two)
  int tile_wl, tile_hl;  // their log2
  int depth_bits;  // key = tile << depth_bits | depth quantum
  float dscale;    // depth quanta per metre
};

// Several views rendered in one pass (art_render_views): their screen tiles
// laid end to end in one tile space (view k owns global tiles
// [toff[k], toff[k + 1])), each view's parameters with the depth-key layout
// of the joint space (one depth_bits for all), its per-voxel rectangles at
// rect + k * rect_stride, and its output maps.  Held in device memory; a
// kernel finds the view of a global tile with view_of.
struct ViewSet {
  int nv;
  uint32_t toff[kMaxViews + 1];
  int64_t rect_stride;
  ViewParams v[kMaxViews];
  void* F[kMaxViews];
  float* A[kMaxViews];
};

__host__ __device__ inline int view_of(const ViewSet& vs, uint32_t tile) {
  int k = 0;
  while (k + 1 < vs.nv && tile >= vs.toff[k + 1]) ++k;
  return k;
}

// Layer of a convolutional network (device pointers owned by the context).
struct ConvLayer {
  int cout, cin, k;
  int cin_pad;                 // input channels of the BF16 / FP8 weights (cin, or cin zero-padded)
  float* w32 = nullptr;        // [cout][k][k][cin] FP32
  float* b32 = nullptr;        // [cout]
  __nv_bfloat16* wbf = nullptr;  // [cout][k*k*cin] BF16 (K-major)
  // the first decoder convolution of a level-0 U-Net block in its sub-pixel
  // form (launch_sub_conv): BF16 weight blocks of the skip part, then of the
  // low-resolution part; sub_cs / sub_cu = their input channels
  __nv_bfloat16* wsub = nullptr;
  int sub_cs = 0, sub_cu = 0;
  // ... of levels 1 and up (the tap-by-tap kernel, TcConv::sub): per output
  // phase [4][cout][9 cs + 4 cu]
  __nv_bfloat16* wtap = nullptr;
  uint8_t* w8 = nullptr;       // [cout][k*k*cin] E4M3
  float* wscale = nullptr;     // [cout] FP8 per-output-channel scale
};

struct Timer {
  const char* name;
  cudaEvent_t e0, e1;
};

struct KernelStat {
  const char* name;
  int64_t launches;
  double ms;
};

}  // namespace art

struct art_ctx {
  cudaStream_t stream = nullptr;
  // a second stream for work beside the bucket sort (tile classes, proposal,
  // clear of the empty tiles), forked from and joined into `stream` by events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_pose = nullptr;
  // frames in flight of art_render_frame_async: their RGBA in two device
  // slots, copied to the host on copy_stream (ev_ready: the slot is written;
  // ev_done: its copy has landed); frame k of the ring is slot (head + k) % 2
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_ready[2] = {}, ev_done[2] = {};
  float* d_rgba_slot[2] = {};
  size_t d_rgba_slot_bytes[2] = {};
  int fr_head = 0, fr_n = 0;
  bool pose_bias_side = false;  // the proposal's pose bias is being computed on the side stream
  bool f_cleared = false;  // the empty tiles of this frame's F and A are cleared already
  std::string err;
  art_config cfg{};
  int device = 0;
  int num_sms = 0;

  // ---- octree (static)
  int64_t n = 0;
  int depth = 0;
  float origin[3] = {0, 0, 0};
  float extent = 0, h = 0;
  int C = 0;
  int feat_dtype = ART_F32;
  uint2* d_ijk = nullptr;       // packed (i | j << 16, k)
  uint32_t* d_jidx = nullptr;   // 4 x uint8
  float4* d_w = nullptr;
  void* d_feat = nullptr;       // [n][C] in feat_dtype
  float* d_sigma = nullptr;

  // ---- skeleton
  int J = 0;
  int32_t parent[art::kMaxJoints];
  float rest[art::kMaxJoints * 3];
  float* d_skel = nullptr;      // parent (as float bits) + rest, uploaded once
  float* d_pose = nullptr;      // J*3 + 6
  float* d_G = nullptr;         // [J][12]

  // ---- per pose
  float4* d_rec = nullptr;      // [n][4] : Binv rows (3) + (sigma, valid, 0, 0)
  float4* d_geo = nullptr;      // [n][4] : (cw, r), (ax, _), (ay, _), (az, _)
  bool posed = false;
  bool jidx_ok = false;         // joint indices validated against J

  // ---- per view / binning
  art::ViewParams views[art::kMaxViews];
  bool view_set[art::kMaxViews] = {};
  int64_t n_cap = 0;            // voxel capacity of per-voxel buffers
  int64_t inst_cap = 0;
  short4* d_rect = nullptr;     // [n] pixel rect (x0, y0, x1, y1), empty if x0 > x1
  uint32_t* d_q = nullptr;      // [n] depth quantum
  uint32_t* d_cnt = nullptr;    // [n] tile count
  uint32_t* d_keys = nullptr;   // instances in (tile, depth, voxel) order: tile << depth_bits | depth quantum
  uint32_t* d_vals = nullptr;   // ... and their voxel ids
  unsigned long long* d_sort_tmp = nullptr;  // staging of the buckets too long for shared memory
  uint2* d_ranges = nullptr;    // per tile [start, end)
  int64_t ranges_cap = 0;
  uint32_t* d_tcount = nullptr;  // per tile instance count
  uint32_t* d_toff = nullptr;    // per tile bucket cursor
  uint32_t* d_sortlist = nullptr;  // tiles whose bucket needs sorting
  unsigned long long* d_scan_state = nullptr;  // tile scan: per block aggregate and inclusive prefix words
  uint32_t* d_agroups = nullptr;  // groups of four consecutive tiles with instances (unordered)
  uint32_t* d_pgroups = nullptr;  // learned skip: the groups with a tile to predict (unordered)
  uint8_t* d_tclass = nullptr;    // learned skip: per tile 0 = predict, 1 = whole range, 2 = nothing
  unsigned long long* d_status = nullptr;
  unsigned long long* h_status = nullptr;  // pinned
  float* d_sh = nullptr;        // [n][(L+1)^2][C] spherical-harmonics coefficients (view-dependent features)
  float* d_sh_rot = nullptr;    // [n][9] world -> canonical direction map per voxel
  int sh_degree = -1;           // L, or -1: plain features
  bool attr_tile_sort = false;  // large shared-memory attributes set on this context's device
  bool attr_proposal = false;

  // ---- frame buffers (art_render_frame)
  void* d_F = nullptr;
  size_t d_F_bytes = 0;
  float* d_A = nullptr;
  size_t d_A_bytes = 0;
  float* d_rgba = nullptr;
  size_t d_rgba_bytes = 0;

  // ---- shading network
  art_net_desc net{};
  int net_dtype = -1;
  std::vector<art::ConvLayer> layers;
  void* d_act = nullptr;        // activation arena
  size_t d_act_bytes = 0;
  bool conv_rows = true;        // row-blocked kernel for the narrow BF16 convolutions
  float* d_f8_scale = nullptr;  // FP8 network: per-tensor activation scales
  unsigned int* d_f8_amax = nullptr;
  bool f8_calibrated = false;

  // ---- learned ray-interval proposal
  bool prop_loaded = false;
  uint8_t* d_prop_img = nullptr;  // BF16 weights of layers 0 (ray part) .. 4 in the UMMA shared-memory image
  float* d_prop_f32 = nullptr;    // W0 pose columns [64][72] (BF16-rounded), b0, b1, b2, b3, b4
  float* d_pose_bias = nullptr;   // [64] b0 + W0[:, :72] pose of the current pose
  uint8_t* d_bins = nullptr;      // [H][W][2] proposal bins of the last learned-skip render
  size_t d_bins_bytes = 0;
  float* d_thist = nullptr;       // [tiles][64] optical-depth bound per (tile, depth bin)
  size_t d_thist_bytes = 0;
  uint32_t* d_hbin = nullptr;     // [n] per-voxel depth-bin range b0 | b1 << 8 (0xFFFF: none)
  float* d_htau = nullptr;        // [n] per-voxel optical-depth bound sigma 2 r
  int64_t hist_n_cap = 0;
  uint32_t* d_fbq = nullptr;      // [tiles] tiles for the sequential walk (stop inside a later segment)
  size_t d_fbq_bytes = 0;
  uint32_t* d_fbq2 = nullptr;     // [tiles] learned skip: tiles that failed the coarse check
  size_t d_fbq2_bytes = 0;
  // ---- several views in one pass (art_render_views)
  short4* d_rect_v = nullptr;     // [views][n] per-view pixel rects, depth quanta, tile counts
  uint32_t* d_q_v = nullptr;
  uint32_t* d_cnt_v = nullptr;
  int64_t views_cap = 0;          // (views x n) capacity of the three
  art::ViewSet* d_vset = nullptr; // the batch's view table (device)
  art::ViewSet h_vset{};          // ... and its host copy
  // ---- the paper's per-frame lattice index (art_config.index = ART_INDEX_GRID)
  unsigned long long* d_gkeys = nullptr;  // [slots] packed cell of each hash slot (all ones: empty)
  uint32_t* d_gvals = nullptr;            // [slots] smallest voxel id of the slot's cell
  int64_t grid_slots = 0;                 // power of two >= 2 n
  // ---- exact re-walk of tiles whose reorder buffer overflowed
  uint32_t* d_xflag = nullptr;    // [tiles] stamp of the render that queued the tile (zeroed when allocated)
  uint32_t xstamp = 0;            // the last render's stamp
  uint32_t* d_xqueue = nullptr;   // [tiles] the queue (count in status[kStExactQ])
  size_t d_xflag_bytes = 0, d_xqueue_bytes = 0;
  float2* d_xhit = nullptr;       // [blocks][32][kExactCap] per-lane hit lists (t0, chord) ...
  uint32_t* d_xpos = nullptr;     // ... and list positions
  // ---- split composite walk
  int seg_len = 256;              // list entries per segment
  int composite_blocks = 0;       // persistent one-warp blocks of the split walk
  int composite_key = 0;          // (C, feature bytes) composite_blocks was computed for
  uint2* d_seg = nullptr;         // [tiles] (first segment, segment count)
  size_t d_seg_bytes = 0;
  uint32_t* d_items = nullptr;    // [segments] tile of each segment
  size_t d_items_bytes = 0;
  uint32_t* d_multi = nullptr;    // [tiles] tiles with two or more segments
  size_t d_multi_bytes = 0;
  float* d_part = nullptr;        // [segments][C + 1][32] partial sums
  size_t d_part_bytes = 0;
  // ---- backward
  float* d_gN = nullptr;        // [n][12] dL/d(A_i^-1) accumulator
  int64_t gN_cap = 0;

  // ---- art_sort_pairs scratch
  uint32_t* d_sk = nullptr;
  uint32_t* d_sv = nullptr;
  uint32_t* d_shist = nullptr;
  uint32_t* d_sbsum = nullptr;
  int64_t sort_cap = 0;

  // ---- profiling
  std::vector<art::Timer> pending;
  std::vector<cudaEvent_t> free_events;
  std::vector<art::KernelStat> stats;
  int64_t launches = 0;
};

namespace art {

// ---- error helpers (api.cu)
art_status fail(art_ctx* ctx, art_status st, const char* fmt, ...);
art_status cuda_fail(art_ctx* ctx, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
art_status ensure(art_ctx* ctx, void** p, size_t* have, size_t need, const char* what);

// Profiling wrappers (api.cu): bracket a launch with events when enabled.
void prof_begin(art_ctx* ctx, const char* name);
void prof_end(art_ctx* ctx);

// ---- kernels: LBS (lbs.cu)
void launch_fk(art_ctx* ctx);
void launch_lbs(art_ctx* ctx);
// The paper's per-frame index after LBS: snap each placed voxel's warped
// centre to the leaf lattice (hash table of cells, the smallest id wins a
// cell) and rewrite the records so that survivors are their cells'
// axis-aligned leaf boxes and the others are dropped.
void launch_grid_snap(art_ctx* ctx);
// With hbin / htau set, also the per-voxel depth-bin range and optical-depth
// bound of the coarse check (64 bins over [znear, zfar]).  Also counts each
// tile's instances and resets the tile scan: launch_bin follows it.
void launch_project(art_ctx* ctx, const ViewParams& v, uint32_t* hbin = nullptr, float* htau = nullptr);
// Projection of view k of a batch into the joint tile space: its rectangles,
// depth quanta and tile counts at rect / q / cnt (the view's slices), its
// tiles' instance counts at tcount (the view's first global tile); the tile
// scan state is reset by view 0's launch.
void launch_project_view(art_ctx* ctx, const ViewParams& v, short4* rect, uint32_t* q, uint32_t* cnt,
                         uint32_t* tcount, bool first);

// ---- binning and sorting (binsort.cu)
// With thist set (zeroed [tiles][64]), also accumulate the coarse optical-depth
// bound of every instance into its tile's depth bins.
// Binning of the projected voxels (after launch_project, which counts the
// instances of every tile): the scan of the counts (the tile ranges), the
// scatter of every instance into its tile's bucket and the sort of each
// bucket by (depth quantum, voxel id).  With thist set, the
// scatter also adds each voxel's optical-depth bound htau to the depth bins
// hbin of each of its tiles (thist: zeroed [tiles][64]; the coarse check of
// the learned skip).
// With sort false the bucket sort is left to launch_tile_sort (so that work
// which needs only the ranges can run beside it).
void launch_bin(art_ctx* ctx, const ViewParams& v, const uint32_t* hbin = nullptr, const float* htau = nullptr,
                float* thist = nullptr, bool sort = true);
void launch_tile_sort(art_ctx* ctx, const ViewParams& v);
// Binning of a batch of views in one tile space (ntiles in all, joint
// depth_bits): one scan of all tiles' counts, one scatter per view (its
// instances keyed by global tile), one sort of all buckets.
void launch_bin_views(art_ctx* ctx, const ViewSet& vs, int64_t ntiles);
// Radix sort of count (device word) pairs ping-ponging between (k0, v0) and
// (k1, v1); returns the index (0 or 1) of the buffer holding the result.
int launch_sort_bufs(art_ctx* ctx, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t cap,
                     const unsigned long long* count, int key_bits, uint32_t* hist, uint32_t* bsum);
void launch_set_word(art_ctx* ctx, unsigned long long* p, unsigned long long value);
size_t sort_hist_words(int64_t n);
size_t scan_block_words(int64_t n);
size_t tile_scan_state_words(int64_t ntiles);  // look-back words of the tile scan

// ---- depth buffer (depth.cu): after launch_project + launch_bin of the view,
// depth [H][W] = entry distance of the nearest hit denser than sigma_min
// (+inf where none)
void launch_depth(art_ctx* ctx, const ViewParams& v, float sigma_min, float* depth);

// ---- composite (composite.cu)
art_status launch_composite(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A,
                            const void* hit_log = nullptr);
// View-dependent features (Eq. 2): each hit's feature from its SH
// coefficients at the ray direction in its canonical frame (sequential walk).
art_status launch_composite_sh(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A);
// Learned skip: composite over the proposal intervals (ctx->d_bins), coarse
// check against ctx->d_thist, then the full traversal of the queued tiles.
art_status launch_composite_skip(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A);
// Zero F and A of the tiles without instances (needs only the tile ranges);
// a composite that follows on the same frame with ctx->f_cleared set skips
// its own clear.
art_status launch_composite_clear(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A);
// Labels of the plain composite (labels [H][W][3], bins [H][W][2]; either may be null).
art_status launch_composite_labels(art_ctx* ctx, const ViewParams& v, float* labels, uint8_t* bins);
// Plain composite of a batch of views in one split pass over the joint tile
// space (after launch_bin_views); vs is the host copy of *ctx->d_vset.
art_status launch_composite_views(art_ctx* ctx, const ViewSet& vs, int F_dtype);
// One-warp blocks of the composite walk that fit on an SM (C channels of feat_bytes).
int composite_blocks_per_sm(int C, int feat_bytes);
constexpr int kShMaxDegree = 3;  // view-dependent features: spherical harmonics up to this degree
constexpr int kShMaxBases = (kShMaxDegree + 1) * (kShMaxDegree + 1);
constexpr int kPropBins = 64;          // proposal depth bins over [znear, zfar]
constexpr int kExactBlocks = 64;       // one-warp blocks of the exact re-walk
constexpr int kExactCap = 1024;        // hits per pixel the exact re-walk sorts (beyond: overflow_order)
constexpr float kLabelWmin = 1e-6f;    // significant hit: weight above this
constexpr float kLabelBudget = 0.4f;   // label bins keep the coarse bound under this fraction of max_missed
constexpr float kHistPad = 1e-5f;      // metres added to both ends of a voxel's distance range before binning
constexpr float kHistSlack = 1e-4f;    // relative growth of the optical-depth bound: covers FP32 rounding of r and sums
// ---- proposal (proposal.cu)
art_status load_proposal(art_ctx* ctx, const float* params);
void launch_pose_bias(art_ctx* ctx);
// bins [H][W][2] (may be null), logits [H][W][128] (may be null); with
// active_only, only 4-tile groups with a non-empty tile are predicted.
// classified: only the groups the tile classes list (launch_tile_class), and
// only their class-0 tiles' bins written.
art_status launch_proposal(art_ctx* ctx, const ViewParams& v, uint8_t* bins, float* logits, bool active_only,
                           bool classified = false);
// Learned skip, after launch_bin with the tile histogram: per tile with
// instances whether the proposal can change its walk (class 0), else its
// bins set to the whole range (1) or to nothing (2); lists the groups to predict.
void launch_tile_class(art_ctx* ctx, const ViewParams& v, uint8_t* bins);
void* make_hit_log(int32_t* count, uint32_t* ids, float* t0, float* t1, int cap);
void free_hit_log(void* p);

// ---- backward (backward.cu)
art_status launch_backward(art_ctx* ctx, const ViewParams& v, const float* F, const float* A, const float* dF,
                           const float* dA, float* gfeat, float* gsig, float* gw);

// ---- shading (cnn.cu, cnn_tc.cu)
// A: the coarse opacity map (device), used by the two-branch network only.
art_status run_shader(art_ctx* ctx, const ViewParams& v, const void* F, int F_dtype, const float* A, float* rgba);

// One 3x3 convolution on the tensor cores: input [H][W][cin] BF16 (NHWC,
// dense), weights [cout][3][3][cin] BF16, bias FP32; output BF16 written at
// channel offset ch_off of a tensor with ld_out channels per pixel, at the
// same resolution or (up2) replicated 2x2 into a 2H x 2W tensor; or, with
// rgba set, the fused 1x1 head (cout -> 4) + sigmoid into FP32 RGBA.
struct TcConv {
  const void* in;
  int cin, H, W;
  const void* w;
  const float* bias;
  int cout, act;
  void* out;
  int ld_out, ch_off, up2;
  float* rgba;             // fused 1x1 head + sigmoid into head_n (<= 4) FP32 channels of rgba,
  const float* head_w;     // starting at channel head_off of head_ld per pixel
  const float* head_b;
  int head_n = 4, head_ld = 4, head_off = 0;
  // also the 2x2 max pooling of the output, a dense [H/2][W/2][cout] tensor
  // (BF16 or E4M3; fused into the row-blocked kernel's epilogue, else a pass of its own)
  void* pool = nullptr;
  // BF16 output stored x-phase split: row y holds the even pixels, then the
  // odd ones ([H][2][W/2][ld_out]), the layout the sub-pixel decoder
  // convolutions read their skip input in (BF16 only)
  int psplit = 0;
  // sub-pixel decoder convolution over [up2(up) | in] (BF16, tap-by-tap
  // kernel): H x W is the output; `in` = the skip tensor, x-phase split
  // ([H][2][W/2][cs]), `up` = the low-resolution tensor ([H/2][W/2][cu]),
  // w = the layer's wtap blocks, cin = cs + cu; dense [H][W][cout] output
  int sub = 0;
  const void* up = nullptr;
  int cs = 0, cu = 0;
  // FP8 (E4M3) network: operands and output in E4M3; the accumulator is
  // dequantised by in_scale x w_scale[co], the output quantised by out_scale
  // and its max |value| recorded in out_amax (float bits).
  bool f8 = false;
  const float* in_scale = nullptr;
  const float* w_scale = nullptr;
  const float* out_scale = nullptr;
  unsigned int* out_amax = nullptr;
};
bool tc_conv_ok(const TcConv& c);
art_status launch_tc_conv(art_ctx* ctx, const TcConv& c);
// cuTensorMapEncodeTiled from the driver (null when unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Sub-pixel form of conv3x3 + ReLU over the concatenation [up2(u) | s] (the
// first convolution of a U-Net decoder block at level 0): 32 output
// channels at H x W; s = the skip tensor, x-phase split ([H][2][W/2][cs]),
// u = the low-resolution tensor ([H/2][W/2][cu]) that nearest x2
// upsampling would repeat; w = the layer's wsub blocks.
struct SubConv {
  const void* skip;
  int cs;
  const void* up;
  int cu;
  int H, W;
  const void* w;
  const float* bias;
  void* out;  // [H][W][32] BF16
};
bool sub_conv_ok(int cout, int cs, int cu, int H, int W);
size_t sub_weight_elems(int cs, int cu);
// Builds wsub from the layer's FP32 weights [32][3][3][cu + cs] (channels
// of the low-resolution part first, as in the concatenation).
void launch_sub_weights(art_ctx* ctx, const float* w32, int cs, int cu, __nv_bfloat16* wsub);
// The per-phase weights of the tap-by-tap sub-pixel form from the FP32
// weights [cout][3][3][cu + cs]: [4][cout][9 cs + 4 cu], per output phase
// (py, px) the skip part's 9 taps (W[dy][dx][cu + ci]) then the 4 summed
// taps of the low-resolution part ((oy, ox) in {py - 1, py} x {px - 1, px}).
void launch_sub_tap_weights(art_ctx* ctx, const float* w32, int cout, int cs, int cu, __nv_bfloat16* wtap);
art_status launch_sub_conv(art_ctx* ctx, const SubConv& c);
void launch_pool_bf16(art_ctx* ctx, const __nv_bfloat16* in, int ld, int ch_off, __nv_bfloat16* out, int H, int W,
                      int C, int psplit = 0);
void launch_pool_fp8(art_ctx* ctx, const uint8_t* in, int ld, int ch_off, uint8_t* out, int H, int W, int C);
void launch_quantize_weights(art_ctx* ctx, const float* w, int cout, int K, uint8_t* w8, float* scale);
void launch_quantize_input(art_ctx* ctx, const __nv_bfloat16* in, int64_t m, const float* scale, uint8_t* out,
                           unsigned int* amax);
void launch_update_scales(art_ctx* ctx, float* scale, unsigned int* amax, int n, float fixed);
constexpr int kF8Tensors = 11;  // FP8 U-Net activation tensors with their own scale

}  // namespace art

// Launch helper: counts and (optionally) times every kernel launch.
// First statement of a kernel launched with ART_LAUNCH_PDL: wait until the
// previous kernel of the stream has completed (its memory visible), then let
// the next kernel start launching.  Only the launch and the ramp of the grid
// overlap the previous one.
#define ART_PDL_ENTRY()                                        \
  do {                                                         \
    asm volatile("griddepcontrol.wait;" ::: "memory");         \
    asm volatile("griddepcontrol.launch_dependents;" :::);     \
  } while (0)

// A launch that may overlap the tail of the previous kernel of the stream
// (programmatic dependent launch): the kernel itself waits (griddepcontrol)
// before it reads or writes memory the previous kernel touches.
#define ART_LAUNCH_PDL(ctx, name, kernel, grid, block, smem, ...)              \
  do {                                                                         \
    art::prof_begin((ctx), (name));                                            \
    cudaLaunchAttribute pdl_attr_[1];                                          \
    pdl_attr_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;     \
    pdl_attr_[0].val.programmaticStreamSerializationAllowed = 1;               \
    cudaLaunchConfig_t pdl_cfg_ = {};                                          \
    pdl_cfg_.gridDim = dim3(grid);                                             \
    pdl_cfg_.blockDim = dim3(block);                                           \
    pdl_cfg_.dynamicSmemBytes = (smem);                                        \
    pdl_cfg_.stream = (ctx)->stream;                                           \
    pdl_cfg_.attrs = pdl_attr_;                                                \
    pdl_cfg_.numAttrs = 1;                                                     \
    cudaLaunchKernelEx(&pdl_cfg_, kernel, __VA_ARGS__);                        \
    art::prof_end((ctx));                                                      \
    (ctx)->launches++;                                                         \
  } while (0)

#define ART_LAUNCH(ctx, name, kernel, grid, block, smem, ...)                  \
  do {                                                                         \
    art::prof_begin((ctx), (name));                                            \
    kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);           \
    art::prof_end((ctx));                                                      \
    (ctx)->launches++;                                                         \
  } while (0)
