// Learned ray-interval proposal: a per-ray MLP that predicts the depth
// interval in which a ray's composite takes its mass (project addition; the
// paper's nearest passage is the early-stop rule of Sec. 3.1 "Dynamic Volume
// Rendering").
//
// Input (107) = [72 joint axis-angles, unit world ray direction, sin / cos of
// 2^k pi u and 2^k pi v for k < 8], layers 107 -> 64 -> 64 -> 64 -> 64 (ReLU)
// -> 128 logits, BF16 operands with FP32 accumulation.  The 72 pose inputs
// are the same for every ray of a frame, so their product with the first
// layer is folded into that layer's bias once per pose (pose_bias_kernel);
// the tensor-core layer then sees K = 35 ray inputs, padded to one 64-wide
// K chunk.
//
// One CTA of 4 warps runs 128 rays (four 8x4 screen tiles) at a time: each
// thread builds its ray's input row in shared memory (BF16, 128-byte swizzled
// K-major rows), one thread issues tcgen05.mma for M = 128 rays x N = 64 (or
// 128) x K = 64, the accumulator lands in TMEM, and every warp reads its 32
// rows back (tcgen05.ld), adds bias, applies ReLU, rounds to BF16 and writes
// the next layer's input rows in place.  All five layers' weights (48 KB)
// stay in shared memory for the whole persistent loop.  The last layer's
// epilogue takes the two argmaxes and writes the bins.
#include <cuda_bf16.h>

#include <vector>

#include "internal.cuh"
#include "raster.cuh"
#include "tc.cuh"

namespace art {
namespace {

constexpr int kPoseIn = 72;                 // 24 joints x 3
constexpr int kRayIn = 35;                  // direction (3) + Fourier features (32)
constexpr int kMatBytes = 64 * 128;         // 64 rows x 64 BF16 (one swizzled K chunk)
constexpr int kImgBytes = 4 * kMatBytes + 2 * kMatBytes;  // layers 0..3 (N = 64) + layer 4 (N = 128)
constexpr int kABytes = 128 * 128;          // 128 rays x 64 BF16
constexpr int kF32Words = 64 * kPoseIn + 64 * 4 + 128;  // pose columns of W0, b0..b3, b4
constexpr int kSmem = 1024 + kImgBytes + kABytes + 4 * 384 + 64;

// Byte offset of element (n, k) of a [rows][64] BF16 operand stored as
// 128-byte K-major rows with the 128-byte swizzle (16-byte unit k / 8 of row
// n sits at unit (k / 8) ^ (n % 8)).
__host__ __device__ inline int sw128(int n, int k) { return n * 128 + ((((k >> 3) ^ (n & 7))) << 4) + ((k & 7) << 1); }

struct PropParams {
  const uint4* img;        // kImgBytes: weights of the five layers in the shared-memory image
  const float* f32;        // kF32Words
  const float* pose_bias;  // [64]
  ViewParams v;
  const uint2* ranges;     // per tile [start, end)
  int ngroups;             // groups of four screen tiles
  int active_only;         // only the groups listed in agroups (count: *n_active)
  const uint32_t* agroups;
  const unsigned long long* n_active;
  uint8_t* tclass;         // per tile: predict only class 0 (null: every tile); failed checks become class 1
  uint8_t* bins;           // [H][W][2] or null
  // with tclass: the coarse check of each predicted tile (tile depth-bin
  // bounds thist, threshold max_missed, union widened by margin); failing
  // tiles are listed in fail_list (count *fail_count)
  const float* thist;
  float max_missed;
  int margin;
  uint32_t* fail_list;
  unsigned long long* fail_count;
  float* logits;           // [H][W][128] or null
  unsigned long long* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// b0 + W0[:, :72] x, x = the current pose's axis-angles rounded to BF16; FP32.
// 256 threads: the weights and the pose come in with coalesced loads, four
// threads share an output (k = q, q + 4, ...), summed in a fixed order.
__global__ void __launch_bounds__(256) pose_bias_kernel(const float* __restrict__ f32, const float* __restrict__ pose,
                                                        float* __restrict__ out) {
  ART_PDL_ENTRY();
  __shared__ float sx[kPoseIn];
  const int j = threadIdx.x >> 2, q = threadIdx.x & 3;
  float w[kPoseIn / 4];  // this thread's weights, loaded together
#pragma unroll
  for (int i = 0; i < kPoseIn / 4; ++i) w[i] = f32[j * kPoseIn + q + 4 * i];
  if (threadIdx.x < kPoseIn) sx[threadIdx.x] = __bfloat162float(__float2bfloat16_rn(pose[threadIdx.x]));
  __syncthreads();
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < kPoseIn / 4; ++i) acc = fmaf(w[i], sx[q + 4 * i], acc);
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (q == 0) out[j] = f32[64 * kPoseIn + j] + acc;
}

__global__ void __launch_bounds__(128) proposal_kernel(PropParams p) {
  ART_PDL_ENTRY();
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* s_img = sm;
  uint8_t* s_a = sm + kImgBytes;
  float* s_bias = reinterpret_cast<float*>(s_a + kABytes);  // pose bias, b1, b2, b3 (64 each), b4 (128)
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_bias + 384);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_items = p.active_only ? (int)*p.n_active : p.ngroups;
  if ((int)blockIdx.x >= n_items) return;  // no group for this CTA

  // the weight image: all copies in flight at once
  for (int i = tid; i < kImgBytes / 16; i += 128) cp_async16(s_img + 16 * i, p.img + i);
  cp_async_commit();
  if (tid < 64) s_bias[tid] = p.pose_bias[tid];
  for (int i = tid; i < 320; i += 128) s_bias[64 + i] = p.f32[64 * kPoseIn + 64 + i];
  if (tid == 0) {
    mbar_init(bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 128);
  cp_async_wait<0>();
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 TMEM lanes
  const uint32_t a_addr = smem_u32(s_a), w_addr = smem_u32(s_img);
  const ViewParams& v = p.v;
  const int ntiles = v.tiles_x * v.tiles_y;
  uint32_t phase = 0;
  bool failed = false;

  for (int it = blockIdx.x; it < n_items && !failed; it += gridDim.x) {
    const int g = p.active_only ? (int)p.agroups[it] : it;
    const int tile = 4 * g + warp;
    bool act = tile < ntiles;
    if (act && p.active_only) {
      const uint2 rg = p.ranges[tile];
      act = rg.y > rg.x;
    }
    if (!__syncthreads_or(act)) continue;
    const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
    const int px = tx * TSX + (lane & 7), py = ty * TSY + (lane >> 3);
    const bool inside = tile < ntiles && px < v.W && py < v.H;
    {  // input row: direction, Fourier features, zero padding
      float e[40];
#pragma unroll
      for (int k = 0; k < 40; ++k) e[k] = 0.0f;
      if (inside) {
        pixel_dir(v, px, py, e[0], e[1], e[2]);
        const float u = ((float)px + 0.5f) / (float)v.W, w = ((float)py + 0.5f) / (float)v.H;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float sc = (float)(1 << k);
          sincospif(sc * u, &e[3 + k], &e[11 + k]);
          sincospif(sc * w, &e[19 + k], &e[27 + k]);
        }
      }
#pragma unroll
      for (int un = 0; un < 8; ++un) {
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (un < 5)
          q = make_uint4(pack_bf16(e[8 * un], e[8 * un + 1]), pack_bf16(e[8 * un + 2], e[8 * un + 3]),
                         pack_bf16(e[8 * un + 4], e[8 * un + 5]), pack_bf16(e[8 * un + 6], e[8 * un + 7]));
        *reinterpret_cast<uint4*>(s_a + sw128(tid, 8 * un)) = q;
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    for (int L = 0; L < 5; ++L) {
      if (tid == 0) {
        tc_fence_after();
        const uint32_t wb = w_addr + (uint32_t)(L * kMatBytes);
        const uint32_t id = L == 4 ? idesc_bf16(128, 128) : idesc_bf16(128, 64);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          umma<false>(tmem, umma_desc<128>(a_addr + kk * 32), umma_desc<128>(wb + kk * 32), id, kk != 0);
        umma_commit(bar);
      }
      const bool ok = mbar_wait(bar, phase, abort_flag, tid == 0 ? 0u : 64u);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      if (L < 4) {  // bias, ReLU, BF16: the next layer's input row
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t r[32];
          tmem_ld32(t_row + (uint32_t)(32 * h), r);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float o[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              o[j] = fmaxf(__uint_as_float(r[8 * q + j]) + s_bias[64 * L + 32 * h + 8 * q + j], 0.0f);
            *reinterpret_cast<uint4*>(s_a + sw128(tid, 32 * h + 8 * q)) =
                make_uint4(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]), pack_bf16(o[4], o[5]), pack_bf16(o[6], o[7]));
          }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncthreads();
      } else {  // logits: first argmax of each half
        float mn = -3.4e38f, mf = -3.4e38f;
        int bn = 0, bf = 0;
        const size_t pix = (size_t)py * v.W + px;
#pragma unroll 1
        for (int h = 0; h < 4; ++h) {
          uint32_t r[32];
          tmem_ld32(t_row + (uint32_t)(32 * h), r);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = 32 * h + j;
            const float val = __uint_as_float(r[j]) + s_bias[256 + col];
            if (p.logits && inside) p.logits[pix * 128 + col] = val;
            if (col < 64) {
              if (val > mn) {
                mn = val;
                bn = col;
              }
            } else if (val > mf) {
              mf = val;
              bf = col - 64;
            }
          }
        }
        const bool pred = tile < ntiles && (!p.tclass || p.tclass[tile] == 0);  // (uniform over the warp)
        if (p.bins && inside && pred) reinterpret_cast<uchar2*>(p.bins)[pix] = make_uchar2((uint8_t)bn, (uint8_t)bf);
        if (p.bins && p.tclass && pred) {
          // Coarse check of the tile's interval (the union of its pixels'
          // predictions, widened by the margin, as the composite walks it):
          // lost mass <= (1 - e^-front) + (1 - e^-back), front / back = the
          // tile's optical-depth bound in the bins before / after the
          // interval (T_end <= 1 bounds the back part).  A tile that fails is
          // walked in full in the same pass: its pixels get bins (0, 63) and
          // the tile class 1, like the tiles no prediction can change.
          int lo_b = kPropBins, hi_b = -1;
          if (inside && bf >= bn) {
            lo_b = bn;
            hi_b = bf;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            lo_b = min(lo_b, __shfl_xor_sync(0xffffffffu, lo_b, o));
            hi_b = max(hi_b, __shfl_xor_sync(0xffffffffu, hi_b, o));
          }
          const bool empty = hi_b < lo_b;
          const int b_n = empty ? lo_b : max(lo_b - p.margin, 0);
          const int b_f = empty ? hi_b : min(hi_b + p.margin, kPropBins - 1);
          const float* th = p.thist + (size_t)tile * kPropBins;
          float p0 = th[lane], p1 = th[32 + lane];  // inclusive prefix sums over the 64 bins
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float a = __shfl_up_sync(0xffffffffu, p0, o), b = __shfl_up_sync(0xffffffffu, p1, o);
            if (lane >= o) {
              p0 += a;
              p1 += b;
            }
          }
          p1 += __shfl_sync(0xffffffffu, p0, 31);
          const float tot = __shfl_sync(0xffffffffu, p1, 31);
          auto pre = [&](int k) {  // prefix through bin k (k warp-uniform)
            const float x = __shfl_sync(0xffffffffu, k < 32 ? p0 : p1, k & 31);
            return k < 0 ? 0.0f : x;
          };
          const float f_pre = pre(b_n - 1), b_pre = pre(b_f);
          const float front = empty ? tot : f_pre;
          const float back = empty ? 0.0f : tot - b_pre;
          const bool fail = -expm1f(-front) + -expm1f(-back) > p.max_missed;
          if (fail && __any_sync(0xffffffffu, inside)) {
            if (inside) reinterpret_cast<uchar2*>(p.bins)[pix] = make_uchar2(0, kPropBins - 1);
            if (lane == 0) {
              p.tclass[tile] = 1;
              p.fail_list[atomicAdd(p.fail_count, 1ull)] = (uint32_t)tile;
            }
          }
        }
        tc_fence_before();
        __syncthreads();  // TMEM and the input rows are reused by the next group
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 128);
  if (tid == 0 && *abort_flag) atomicAdd(p.err, 1ull);
}

}  // namespace

art_status load_proposal(art_ctx* ctx, const float* params) {
  std::vector<float> P(ART_PROPOSAL_PARAMS);
  cudaError_t e = cudaMemcpy(P.data(), params, sizeof(float) * P.size(), cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy proposal params");
  // offsets of W0, b0, W1, b1, ..., W4, b4 in the flat vector
  const int shapes[5][2] = {{64, 107}, {64, 64}, {64, 64}, {64, 64}, {128, 64}};
  size_t off[5][2], o = 0;
  for (int l = 0; l < 5; ++l) {
    off[l][0] = o;
    o += (size_t)shapes[l][0] * shapes[l][1];
    off[l][1] = o;
    o += shapes[l][0];
  }
  std::vector<__nv_bfloat16> img(kImgBytes / 2, __float2bfloat16_rn(0.0f));
  std::vector<float> f32(kF32Words, 0.0f);
  for (int l = 0; l < 5; ++l) {
    const int N = shapes[l][0], K = shapes[l][1];
    const int base = l * (kMatBytes / 2);
    for (int n = 0; n < N; ++n) {
      if (l == 0) {
        for (int k = 0; k < kPoseIn; ++k)
          f32[n * kPoseIn + k] = __bfloat162float(__float2bfloat16_rn(P[off[0][0] + (size_t)n * K + k]));
        for (int k = 0; k < kRayIn; ++k)
          img[base + sw128(n, k) / 2] = __float2bfloat16_rn(P[off[0][0] + (size_t)n * K + kPoseIn + k]);
      } else {
        for (int k = 0; k < K; ++k) img[base + sw128(n, k) / 2] = __float2bfloat16_rn(P[off[l][0] + (size_t)n * K + k]);
      }
    }
    float* bdst = l < 4 ? &f32[64 * kPoseIn + 64 * l] : &f32[64 * kPoseIn + 256];
    for (int n = 0; n < N; ++n) bdst[n] = P[off[l][1] + n];
  }
  art_status st;
  if (!ctx->d_prop_img) {
    if (cudaMalloc(&ctx->d_prop_img, kImgBytes) != cudaSuccess || cudaMalloc(&ctx->d_prop_f32, 4 * kF32Words) != cudaSuccess ||
        cudaMalloc(&ctx->d_pose_bias, 4 * 64) != cudaSuccess)
      return fail(ctx, ART_ERR_OOM, "proposal buffers");
  }
  if ((e = cudaMemcpy(ctx->d_prop_img, img.data(), kImgBytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_prop_f32, f32.data(), 4 * kF32Words, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(ctx, e, "upload proposal");
  ctx->prop_loaded = true;
  (void)st;
  return ART_OK;
}

void launch_pose_bias(art_ctx* ctx) {
  ART_LAUNCH_PDL(ctx, "proposal_pose_bias", pose_bias_kernel, 1, 256, 0, ctx->d_prop_f32, ctx->d_pose, ctx->d_pose_bias);
}

// Tiles whose walk the proposal cannot change (learned skip).  From a tile's
// coarse optical-depth bound per depth bin (h, total tot, first and last
// occupied bins lo, hi) and the check lost = (1 - e^-front) + (1 - e^-back)
// <= max_missed (front / back: the bins before / after the interval; the
// transmittance after the interval, T_end <= 1, left out):
//   - if 1 - e^-tot <= max_missed, the empty interval passes: the tile
//     composites nothing (class 2);
//   - if 1 - e^-h[lo] > max_missed, no interval may start after bin lo; if
//     e^-tot (1 - e^-h[hi]) > max_missed, none may end before bin hi (this
//     holds even with the check weighted by T_end >= e^-tot, as the bound
//     sums every hit's sigma 2 r); with both, every passing interval covers
//     [lo, hi], which holds all of the tile's hits: the tile is walked in full
//     without a prediction (class 1).
// Other tiles are predicted (class 0); the groups holding one are listed for
// the proposal, whose epilogue applies the check to their intervals.
// Classes 1 and 2 write their pixels' bins (0, 63) and (63, 0): the
// composite reads them as it reads predictions.
__global__ void __launch_bounds__(128) tile_class_kernel(ViewParams v, const uint2* __restrict__ ranges,
                                                        const float* __restrict__ thist,
                                                        const uint32_t* __restrict__ agroups,
                                                        unsigned long long* __restrict__ status, float max_missed,
                                                        uint8_t* __restrict__ tclass, uint32_t* __restrict__ pgroups,
                                                        uint8_t* __restrict__ bins) {
  ART_PDL_ENTRY();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long n_groups = status[kStActiveGroups];
  const int ntiles = v.tiles_x * v.tiles_y;
  for (unsigned long long gi = blockIdx.x; gi < n_groups; gi += gridDim.x) {
    const int g = (int)agroups[gi];
    const int tile = 4 * g + warp;
    int cls = 3;  // no instances: not walked, not predicted
    if (tile < ntiles) {
      const uint2 rg = ranges[tile];
      if (rg.y > rg.x) {
        const float h0 = thist[(size_t)tile * kPropBins + lane], h1 = thist[(size_t)tile * kPropBins + 32 + lane];
        float tot = h0 + h1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        const uint32_t m0 = __ballot_sync(0xffffffffu, h0 > 0.0f), m1 = __ballot_sync(0xffffffffu, h1 > 0.0f);
        const int lo = m0 ? __ffs(m0) - 1 : (m1 ? 32 + __ffs(m1) - 1 : 0);
        const int hi = m1 ? 63 - __clz(m1) : (m0 ? 31 - __clz(m0) : 0);
        const float hlo = __shfl_sync(0xffffffffu, lo < 32 ? h0 : h1, lo & 31);
        const float hhi = __shfl_sync(0xffffffffu, hi < 32 ? h0 : h1, hi & 31);
        if (-expm1f(-tot) <= max_missed) {
          cls = 2;
        } else if (-expm1f(-hlo) > max_missed && expf(-tot) * -expm1f(-hhi) > max_missed) {
          cls = 1;
        } else {
          cls = 0;
        }
        if (cls != 0) {
          const int px = (tile % v.tiles_x) * TSX + (lane & 7), py = (tile / v.tiles_x) * TSY + (lane >> 3);
          if (px < v.W && py < v.H)
            reinterpret_cast<uchar2*>(bins)[(size_t)py * v.W + px] = cls == 1 ? make_uchar2(0, kPropBins - 1)
                                                                               : make_uchar2(kPropBins - 1, 0);
        }
      }
    }
    if (tile < ntiles && lane == 0) tclass[tile] = (uint8_t)cls;
    __shared__ int s_pred[4];
    if (lane == 0) s_pred[warp] = cls == 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_pred[0] | s_pred[1] | s_pred[2] | s_pred[3]) pgroups[atomicAdd(status + kStPredGroups, 1ull)] = (uint32_t)g;
    }
    __syncthreads();
    if (lane == 0 && (cls == 1 || cls == 2)) atomicAdd(status + kStForcedTiles, 1ull);
  }
}

void launch_tile_class(art_ctx* ctx, const ViewParams& v, uint8_t* bins) {
  // (kStPredGroups, kStForcedTiles, kStCheckFail)
  static_assert(kStForcedTiles == kStPredGroups + 1 && kStCheckFail == kStPredGroups + 2, "status words");
  cudaMemsetAsync(ctx->d_status + kStPredGroups, 0, 3 * sizeof(unsigned long long), ctx->stream);
  const int ngroups = (v.tiles_x * v.tiles_y + 3) / 4;
  ART_LAUNCH_PDL(ctx, "tile_class", tile_class_kernel, std::max(1, std::min(ngroups, 8 * ctx->num_sms)), 128, 0, v,
             ctx->d_ranges, ctx->d_thist, ctx->d_agroups, ctx->d_status, ctx->cfg.max_missed, ctx->d_tclass,
             ctx->d_pgroups, bins);
}

art_status launch_proposal(art_ctx* ctx, const ViewParams& v, uint8_t* bins, float* logits, bool active_only,
                           bool classified) {
  if (!ctx->attr_proposal) {  // (a function attribute holds per device: set once per context)
    cudaError_t e = cudaFuncSetAttribute(proposal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "proposal smem attribute");
    ctx->attr_proposal = true;
  }
  PropParams p;
  p.img = reinterpret_cast<const uint4*>(ctx->d_prop_img);
  p.f32 = ctx->d_prop_f32;
  p.pose_bias = ctx->d_pose_bias;
  p.v = v;
  p.ranges = ctx->d_ranges;
  const int ntiles = v.tiles_x * v.tiles_y;
  p.ngroups = (ntiles + 3) / 4;
  p.active_only = active_only ? 1 : 0;
  p.agroups = classified ? ctx->d_pgroups : ctx->d_agroups;
  p.n_active = ctx->d_status + (classified ? kStPredGroups : kStActiveGroups);
  p.tclass = classified ? ctx->d_tclass : nullptr;
  p.bins = bins;
  p.thist = ctx->d_thist;
  p.max_missed = ctx->cfg.max_missed;
  p.margin = ctx->cfg.margin;
  p.fail_list = ctx->d_fbq2;
  p.fail_count = ctx->d_status + kStCheckFail;
  p.logits = logits;
  p.err = ctx->d_status + kStTcError;
  const int grid = std::min(p.ngroups, 3 * ctx->num_sms);
  ART_LAUNCH_PDL(ctx, "proposal_mlp", proposal_kernel, grid, 128, kSmem, p);
  return ART_OK;
}

}  // namespace art
