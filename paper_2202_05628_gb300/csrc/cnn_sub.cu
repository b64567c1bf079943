// Sub-pixel form of the first decoder convolution of the level-0 U-Net
// block on the tensor cores (arXiv 2202.05628, Sec. 3.1 "Neural Shading":
// the U-Net's decoder upsamples and concatenates the encoder's skip tensor).
//
// The layer computes y = ReLU(conv3x3([up2(u) | s]) + b) at H x W, with u the
// low-resolution tensor (h x w = H/2 x W/2) that nearest x2 upsampling
// repeats and s the skip tensor.  Split the output pixels into four phases
// (py, px) = (Y mod 2, X mod 2) and write Y = 2i + py, X = 2j + px:
// - the skip part reads s at row 2i + r, column 2j + c with r = py + dy and
//   c = px + dx in {-1, 0, 1, 2};
// - the upsampled part reads u at row i + oy, column j + ox with
//   oy = floor((py + dy) / 2) in {-1, 0, 1}: each phase sees u through four
//   taps, whose weights are sums of the 3x3 weights that land on the same
//   low-resolution pixel (W'_{py,px}[oy][ox] = sum over dy, dx with
//   floor((py + dy) / 2) = oy, floor((px + dx) / 2) = ox of W[dy][dx]).
// So the low-resolution tensor is read once instead of its 2x2-replicated
// copy, and that part costs 4 instead of 9 taps per output pixel.
//
// GEMM view: M = 128 low-resolution pixels j of one row i, N = the two
// column phases px x 32 output channels of one output row 2i + py (one TMEM
// accumulator of 64 columns), K = taps x channels.  A CTA computes one row
// phase py (blockIdx parity) for all its units, so it keeps only that
// phase's weight blocks resident (68 KB for the 96 -> 32 layer) and two CTAs
// share an SM: two threads issue MMAs there.  A stage is one TMA box of 130
// pixels (j0 - 1 .. j0 + 128) x 32 channels of one input row: of u (rows
// i + oy, oy in {py - 1, py}), or of s (rows 2i + r, r in {py - 1, py,
// py + 1}) stored x-phase split (even pixels of the row, then the odd
// ones), so that the column offsets c = -1, 0, 1, 2 are the odd box from
// row 0, the even box from row 1, the odd box from row 1 and the even box
// from row 2.  For each column shift a box serves, one MMA over the column
// phases it feeds (N = 64 for both, else 32), whose weight blocks sit side
// by side in shared memory.  Zero padding comes from the boxes' out of range
// pixels (TMA fills zeros), which is exact: an upsampled pixel outside the
// image maps to a low-resolution one outside it.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "internal.cuh"
#include "tc.cuh"

namespace art {
namespace {

constexpr int kThreads = 192;   // warp 0 TMA, warp 1 MMA + TMEM, warps 2..5 epilogue
constexpr int kC = 32;          // output channels
constexpr int kKCB = 64;        // bytes per row of a K chunk: 32 BF16 channels (64-B swizzle)
constexpr int kKC = 32;
constexpr int kHalo = 130;      // input pixels of a row box (128 + 2)
constexpr int kBoxBytes = kHalo * kKCB;
constexpr int kStageBytes = (kBoxBytes + 511) / 512 * 512;  // stages on 64-B swizzle atoms (8 rows x 64 B)
constexpr int kBlock = kC * kKCB;  // one weight block: 32 output x 32 input channels
constexpr int kSkipEntries = 18;   // per row phase: (r, c, px) of the skip part
constexpr int kUpEntries = 8;      // per row phase: (oy, ox, px) of the low-resolution part
constexpr int kAccCols = 2 * kC;   // one accumulator: two column phases x 32 channels
constexpr int kMaxWeights = 80 * 1024;
constexpr int kMaxStages = 16;
constexpr int kCtas = 2;           // CTAs per SM (one issuing thread each)

// Column phases a column offset of the skip part feeds: c in {-1, 0, 1, 2}
// reaches px with dx = c - px in {-1, 0, 1} (likewise rows: r and py).
__host__ __device__ constexpr int skip_n(int v) { return (v == -1 || v == 2) ? 1 : 2; }
__host__ __device__ constexpr int skip_min(int v) { return v == 2 ? 1 : 0; }
// ... and of the low-resolution part: ox in {-1, 0, 1} is reached by px = 0
// (ox = -1, 0) and px = 1 (ox = 0, 1).
__host__ __device__ constexpr int up_n(int v) { return v == 0 ? 2 : 1; }
__host__ __device__ constexpr int up_min(int v) { return v == 1 ? 1 : 0; }
// First weight block of (r, c) among row phase py's skip entries, ordered by
// r (py - 1 .. py + 1), c, then px; of (oy, ox) among its low-resolution
// entries, ordered by oy (py - 1, py), ox, then px.
__host__ __device__ constexpr int skip_base(int py, int r, int c) {
  int b = 6 * (r - (py - 1));
  for (int cc = -1; cc < c; ++cc) b += skip_n(cc);
  return b;
}
__host__ __device__ constexpr int up_base(int py, int oy, int ox) {
  int b = 4 * (oy - (py - 1));
  for (int xx = -1; xx < ox; ++xx) b += up_n(xx);
  return b;
}
static_assert(skip_base(0, 1, 2) + 1 == kSkipEntries && up_base(1, 1, 1) + 1 == kUpEntries, "entry tables");

// floor(v / 2) for v in {-1, 0, 1, 2}
__host__ __device__ constexpr int half_floor(int v) { return (v + 2) / 2 - 1; }

struct SubParams {
  int H, W, w;            // output size, low-resolution width
  int cs_ch, cu_ch;       // 32-channel chunks of the skip and the low-resolution input
  int tiles_per_row, n_units;
  int n_stages;
  int w_bytes;
  const float* bias;
  __nv_bfloat16* out;     // [H][W][32]
  unsigned long long* err;
};

// MMA of one column offset whose column phases are px0 .. px0 + nc - 1
// (TMEM columns and weight blocks consecutive).  Two K steps of 16
// channels each.
__device__ __forceinline__ void sub_mma(uint32_t d, uint32_t a, uint32_t wb0, int nc, int px0) {
  const uint32_t idesc = nc == 2 ? idesc_bf16(128, 2 * kC) : idesc_bf16(128, kC);
  const uint32_t dc = d + (uint32_t)(px0 * kC);
#pragma unroll
  for (int kk = 0; kk < kKCB / 32; ++kk)
    umma<false>(dc, umma_desc<kKCB>(a + kk * 32), umma_desc<kKCB>(wb0 + kk * 32), idesc, 1u);
}

__global__ void __launch_bounds__(kThreads, kCtas)
    conv_sub_kernel(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmU,
                    const __grid_constant__ CUtensorMap tmWs, const __grid_constant__ CUtensorMap tmWu, SubParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* wsm = sm;  // row phase py's skip blocks [cs_ch][18], then low-resolution blocks [cu_ch][8], 2 KB each
  uint8_t* stages = sm + p.w_bytes;
  const int S = p.n_stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(stages + (size_t)S * kStageBytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint64_t* wbar = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* s_bias = reinterpret_cast<float*>(tmem_slot + 4);
  // epilogue store staging: 32 output pixels x 4 16-B chunks per warp
  uint4* s_stage = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(s_bias + kC) + 15) & ~(uintptr_t)15);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int py = blockIdx.x & 1;                  // this CTA's output rows 2i + py
  const int u0 = blockIdx.x >> 1, du = gridDim.x >> 1;
  const int n_skip = 6 * p.cs_ch;                 // skip stages: per chunk 3 rows x (even, odd) boxes
  const int n_stage_unit = n_skip + 2 * p.cu_ch;  // + per chunk 2 low-resolution rows
  const int ubase_off = p.cs_ch * kSkipEntries * kBlock;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    mbar_init(wbar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kC; i += kThreads) s_bias[i] = p.bias[i];
  if (warp == 1) tmem_alloc(tmem_slot, 2 * kAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  grid_dep_launch();  // the next layer may start its prologue where this one's CTAs leave SMs
  if (warp == 0) {
    // ------------------------------------------------------------ TMA
    if (lane == 0) {
      mbar_expect_tx(wbar, (uint32_t)p.w_bytes);  // the weights are static: loaded before the wait
      for (int cc = 0; cc < p.cs_ch; ++cc)
        for (int e = 0; e < kSkipEntries; ++e)
          tma_load_2d(wsm + (size_t)(cc * kSkipEntries + e) * kBlock, &tmWs, wbar, cc * kKC,
                      (py * kSkipEntries + e) * kC);
      for (int cc = 0; cc < p.cu_ch; ++cc)
        for (int e = 0; e < kUpEntries; ++e)
          tma_load_2d(wsm + ubase_off + (size_t)(cc * kUpEntries + e) * kBlock, &tmWu, wbar, cc * kKC,
                      (py * kUpEntries + e) * kC);
    }
    grid_dep_wait();  // the previous layers' outputs (this one's inputs) are complete
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      for (int u = u0; u < p.n_units && !*abort_flag; u += du) {
        const int i = u / p.tiles_per_row, j0 = (u % p.tiles_per_row) * 128;
        for (int st = 0; st < n_stage_unit; ++st) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
          uint8_t* dst = stages + (size_t)s * kStageBytes;
          mbar_expect_tx(&full[s], (uint32_t)kBoxBytes);
          if (st < n_skip) {
            const int cc = st / 6, k = st - 6 * cc, r = py - 1 + (k >> 1), q = k & 1;
            tma_load_4d(dst, &tmS, &full[s], cc * kKC, j0 - 1, q, 2 * i + r);
          } else {
            const int t = st - n_skip, cc = t >> 1, oy = py - 1 + (t & 1);
            tma_load_3d(dst, &tmU, &full[s], cc * kKC, j0 - 1, i + oy);
          }
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA
    grid_dep_wait();
    if (lane == 0) {
      int s = 0, buf = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = mbar_wait(wbar, 0u, abort_flag);
      const uint32_t wbase = smem_u32(wsm), ubase = wbase + (uint32_t)ubase_off;
      for (int u = u0; ok && u < p.n_units && !*abort_flag; u += du) {
        // the epilogue clears the accumulators (phase 0 = the initial clear)
        if (!mbar_wait(&acce[buf], aph, abort_flag)) break;
        tc_fence_after();
        const uint32_t d0 = tmem_base + (uint32_t)(buf * kAccCols);
        for (int st = 0; st < n_stage_unit; ++st) {
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stages + (size_t)s * kStageBytes);
          if (st < n_skip) {
            const int cc = st / 6, k = st - 6 * cc, r = py - 1 + (k >> 1), q = k & 1;
            // even box: c = 0 (from row 1), c = 2 (row 2); odd box: c = -1 (row 0), c = 1 (row 1)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              const int c = q == 0 ? 2 * t : 2 * t - 1;
              const int off = q == 0 ? t + 1 : t;
              const uint32_t wb0 = wbase + (uint32_t)((cc * kSkipEntries + skip_base(py, r, c)) * kBlock);
              sub_mma(d0, a0 + (uint32_t)(off * kKCB), wb0, skip_n(c), skip_min(c));
            }
          } else {
            const int t = st - n_skip, cc = t >> 1, oy = py - 1 + (t & 1);
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
              const uint32_t wb0 = ubase + (uint32_t)((cc * kUpEntries + up_base(py, oy, ox)) * kBlock);
              sub_mma(d0, a0 + (uint32_t)((ox + 1) * kKCB), wb0, up_n(ox), up_min(ox));
            }
          }
          umma_commit(&empty[s]);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&accf[buf]);
        if (++buf == 2) {
          buf = 0;
          aph ^= 1u;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    grid_dep_wait();  // the output tensor may still be read by the previous layer
    const int qd = warp & 3;
    const uint32_t tq = tmem_base + ((uint32_t)(qd * 32) << 16);  // this warp's lane quarter
    uint4* stg = s_stage + (warp - 2) * 32 * 4;
    {  // zero both accumulators, then release them to the MMA
      for (int c0 = 0; c0 < 2 * kAccCols; c0 += 32) tmem_zero32(tq + (uint32_t)c0);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&acce[0]);
      mbar_arrive(&acce[1]);
    }
    int buf = 0;
    uint32_t aph = 0;
    for (int u = u0; u < p.n_units; u += du) {
      if (!mbar_wait(&accf[buf], aph, abort_flag, 256)) break;
      tc_fence_after();
      const int i = u / p.tiles_per_row;
      const int jw = (u % p.tiles_per_row) * 128 + qd * 32;  // this warp's first low-resolution pixel
      const uint32_t tb = tq + (uint32_t)(buf * kAccCols);
      // output row 2i + py: per column phase px the warp's 32 pixels 2j + px, staged
      // (chunk k of pixel q at 4 q + (k ^ q % 4)) and stored 8 pixels x 64 B per instruction
      __nv_bfloat16* orow = p.out + (size_t)(2 * i + py) * p.W * kC;
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        uint32_t r[32];
        tmem_ld32(tb + (uint32_t)(px * kC), r);
        uint4 pk[4];
        uint32_t* w = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float t0 = fmaxf(__uint_as_float(r[2 * j]) + s_bias[2 * j], 0.0f);
          const float t1 = fmaxf(__uint_as_float(r[2 * j + 1]) + s_bias[2 * j + 1], 0.0f);
          __nv_bfloat162 b2 = __floats2bfloat162_rn(t0, t1);
          w[j] = *reinterpret_cast<uint32_t*>(&b2);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) stg[lane * 4 + (k ^ (lane & 3))] = pk[k];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int f = t * 32 + lane, q = f >> 2, c4 = f & 3;
          if (jw + q < p.w)
            reinterpret_cast<uint4*>(orow + (size_t)(2 * (jw + q) + px) * kC)[c4] = stg[q * 4 + (c4 ^ (q & 3))];
        }
        __syncwarp();
      }
#pragma unroll
      for (int c0 = 0; c0 < kAccCols; c0 += 32) tmem_zero32(tb + (uint32_t)c0);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      if (++buf == 2) {
        buf = 0;
        aph ^= 1u;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, 2 * kAccCols);
  if (threadIdx.x == 0 && *abort_flag) atomicAdd(p.err, 1ull);
}

// wsub from the FP32 weights w32 [32][3][3][cu + cs] (the low-resolution
// part's channels first), per row phase py: the skip part's blocks
// [2][18][32][cs] (entry (r, c, px): W[r - py][c - px]) and the
// low-resolution part's blocks [2][8][32][cu] (entry (oy, ox, px): the sum
// of W[dy][dx] over the taps with floor((py + dy) / 2) = oy and
// floor((px + dx) / 2) = ox, in FP32, rounded once to BF16).
__global__ void sub_weights_kernel(const float* __restrict__ w32, int cs, int cu, __nv_bfloat16* __restrict__ ws,
                                   __nv_bfloat16* __restrict__ wu) {
  const int64_t n_s = 2LL * kSkipEntries * kC * cs, n_u = 2LL * kUpEntries * kC * cu;
  const int cin = cu + cs;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_s + n_u;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const bool skip = idx < n_s;
    const int64_t t = skip ? idx : idx - n_s;
    const int ci = (int)(t % (skip ? cs : cu));
    const int row = (int)(t / (skip ? cs : cu));
    const int co = row % kC;
    const int ent = row / kC;  // py * entries + e
    const int per = skip ? kSkipEntries : kUpEntries, per_row = skip ? 6 : 4;
    const int py = ent / per, e = ent % per;
    const int ry = py - 1 + e / per_row;  // r, or oy
    int rem = e % per_row, rx = -1, px = 0;  // c (or ox) and px of the entry
    for (int b = -1; b <= (skip ? 2 : 1); ++b) {
      const int nb = skip ? skip_n(b) : up_n(b);
      if (rem < nb) {
        rx = b;
        px = (skip ? skip_min(b) : up_min(b)) + rem;
        break;
      }
      rem -= nb;
    }
    const float* wc = w32 + (size_t)co * 9 * cin;
    if (skip) {
      const int dy = ry - py, dx = rx - px;
      ws[t] = __float2bfloat16_rn(wc[((dy + 1) * 3 + (dx + 1)) * cin + cu + ci]);
    } else {
      float acc = 0.0f;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          if (half_floor(py + dy) == ry && half_floor(px + dx) == rx) acc += wc[((dy + 1) * 3 + (dx + 1)) * cin + ci];
      wu[t] = __float2bfloat16_rn(acc);
    }
  }
}

// Per output phase (py, px) of the tap-by-tap sub-pixel form: row co of
// phase ph holds the skip part's 9 taps (tap = (dy + 1) 3 + dx + 1:
// W[dy][dx][cu + ci]) and then the low-resolution part's 4 taps (tu: oy =
// py - 1 + tu / 2, ox = px - 1 + tu % 2: the FP32 sum of W[dy][dx][ci] over
// the taps with floor((py + dy) / 2) = oy and floor((px + dx) / 2) = ox),
// rounded to BF16.
__global__ void sub_tap_weights_kernel(const float* __restrict__ w32, int cout, int cs, int cu,
                                       __nv_bfloat16* __restrict__ out) {
  const int K = 9 * cs + 4 * cu, cin = cu + cs;
  const int64_t n = 4LL * cout * K;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % K);
    const int row = (int)(idx / K);
    const int co = row % cout, ph = row / cout, py = ph >> 1, px = ph & 1;
    const float* wc = w32 + (size_t)co * 9 * cin;
    if (k < 9 * cs) {
      const int tap = k / cs, ci = k % cs;
      out[idx] = __float2bfloat16_rn(wc[tap * cin + cu + ci]);
    } else {
      const int tu = (k - 9 * cs) / cu, ci = (k - 9 * cs) % cu;
      const int oy = py - 1 + (tu >> 1), ox = px - 1 + (tu & 1);
      float acc = 0.0f;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          if (half_floor(py + dy) == oy && half_floor(px + dx) == ox) acc += wc[((dy + 1) * 3 + (dx + 1)) * cin + ci];
      out[idx] = __float2bfloat16_rn(acc);
    }
  }
}

}  // namespace

size_t sub_weight_elems(int cs, int cu) { return 2 * ((size_t)kSkipEntries * kC * cs + (size_t)kUpEntries * kC * cu); }

bool sub_conv_ok(int cout, int cs, int cu, int H, int W) {
  const int w_bytes = (kSkipEntries * (cs / kKC) + kUpEntries * (cu / kKC)) * kBlock;
  return cout == kC && cs > 0 && cu > 0 && cs % kKC == 0 && cu % kKC == 0 && H % 2 == 0 && W % 2 == 0 && H > 0 &&
         W > 0 && w_bytes <= kMaxWeights && tensor_map_encoder() != nullptr;
}

void launch_sub_weights(art_ctx* ctx, const float* w32, int cs, int cu, __nv_bfloat16* wsub) {
  const int64_t n = (int64_t)sub_weight_elems(cs, cu);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
  ART_LAUNCH(ctx, "sub_weights", sub_weights_kernel, grid, 256, 0, w32, cs, cu, wsub,
             wsub + 2 * (size_t)kSkipEntries * kC * cs);
}

void launch_sub_tap_weights(art_ctx* ctx, const float* w32, int cout, int cs, int cu, __nv_bfloat16* wtap) {
  const int64_t n = 4LL * cout * (9 * cs + 4 * cu);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  ART_LAUNCH(ctx, "sub_weights", sub_tap_weights_kernel, grid, 256, 0, w32, cout, cs, cu, wtap);
}

art_status launch_sub_conv(art_ctx* ctx, const SubConv& c) {
  if (!sub_conv_ok(kC, c.cs, c.cu, c.H, c.W)) return fail(ctx, ART_ERR_UNSUPPORTED, "sub-pixel conv: unsupported shape");
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  const int h = c.H / 2, w = c.W / 2;
  const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_64B;
  CUtensorMap tmS, tmU, tmWs, tmWu;
  {  // skip tensor, x-phase split: (channel, j, phase, Y)
    cuuint64_t dims[4] = {(cuuint64_t)c.cs, (cuuint64_t)w, 2, (cuuint64_t)c.H};
    cuuint64_t strides[3] = {(cuuint64_t)c.cs * 2, (cuuint64_t)w * c.cs * 2, (cuuint64_t)c.W * c.cs * 2};
    cuuint32_t box[4] = {(cuuint32_t)kKC, (cuuint32_t)kHalo, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(&tmS, dt, 4, (void*)c.skip, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (skip) failed: %d", (int)r);
  }
  {  // low-resolution tensor: (channel, j, i)
    cuuint64_t dims[3] = {(cuuint64_t)c.cu, (cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[2] = {(cuuint64_t)c.cu * 2, (cuuint64_t)w * c.cu * 2};
    cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)kHalo, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(&tmU, dt, 3, (void*)c.up, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (low resolution) failed: %d", (int)r);
  }
  const __nv_bfloat16* ws = (const __nv_bfloat16*)c.w;
  const __nv_bfloat16* wu = ws + 2 * (size_t)kSkipEntries * kC * c.cs;
  for (int part = 0; part < 2; ++part) {  // weight blocks: (channel, row phase x entry row)
    const int ci = part == 0 ? c.cs : c.cu, rows = 2 * (part == 0 ? kSkipEntries : kUpEntries) * kC;
    cuuint64_t dims[2] = {(cuuint64_t)ci, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ci * 2};
    cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)kC};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(part == 0 ? &tmWs : &tmWu, dt, 2, (void*)(part == 0 ? ws : wu), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (sub-pixel weights) failed: %d", (int)r);
  }
  SubParams p;
  p.H = c.H;
  p.W = c.W;
  p.w = w;
  p.cs_ch = c.cs / kKC;
  p.cu_ch = c.cu / kKC;
  p.tiles_per_row = (w + 127) / 128;
  p.n_units = p.tiles_per_row * h;
  p.w_bytes = (kSkipEntries * p.cs_ch + kUpEntries * p.cu_ch) * kBlock;
  p.bias = c.bias;
  p.out = (__nv_bfloat16*)c.out;
  p.err = ctx->d_status + kStTcError;
  const int tail = 8 * (2 * kMaxStages + 5) + 16 + 4 * kC + 16 + 4 * 32 * 4 * 16;
  // two CTAs per SM: each within half of the SM's shared memory (less what
  // the runtime reserves per CTA)
  const int avail = 232448 / kCtas - 1024 - 1024 - p.w_bytes - tail;
  p.n_stages = std::min(kMaxStages, avail / kStageBytes);
  if (p.n_stages < 2) return fail(ctx, ART_ERR_UNSUPPORTED, "sub-pixel conv: weights too large");
  const int smem = 1024 + p.w_bytes + p.n_stages * kStageBytes + tail;
  cudaError_t e = cudaFuncSetAttribute(conv_sub_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "conv_sub shared memory attribute");
  // an even grid: CTA b computes row phase b % 2 of the units b / 2, b / 2 + grid / 2, ...
  const int grid = 2 * std::min(p.n_units, kCtas * ctx->num_sms / 2);
  ART_LAUNCH_PDL(ctx, "conv_tc", conv_sub_kernel, grid, kThreads, smem, tmS, tmU, tmWs, tmWu, p);
  return ART_OK;
}

}  // namespace art
