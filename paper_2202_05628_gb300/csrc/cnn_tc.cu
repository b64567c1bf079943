// Tensor-core (tcgen05) implicit-GEMM 3x3 convolution for the BF16 shading
// network (arXiv 2202.05628, Sec. 3.1 "Neural Shading"; half-precision
// network of Sec. 6 "Runtime Analysis").
//
// GEMM view: M = pixels (tiles of 128 consecutive pixels of one image row),
// N = output channels (the whole Cout, <= 256), K = 9 taps x Cin.  For each
// K chunk (one tap, KC channels) a TMA load brings the 128 x KC input box
// shifted by the tap (rows / columns outside the image arrive as zeros, which
// is the convolution's zero padding) and the N x KC weight box into shared
// memory with the swizzle the UMMA descriptors expect.  One thread issues
// tcgen05.mma (BF16 x BF16 -> FP32 in TMEM); a double-buffered accumulator
// lets four epilogue warps drain tile t (tcgen05.ld, bias, ReLU, BF16, store,
// optional x2 nearest upsampling into a concatenation buffer, optional fused
// 1x1 head + sigmoid) while tile t+1 accumulates.  The CTA is persistent over
// the tiles.  Every mbarrier wait is bounded; on time-out the CTA raises an
// error word, stops its loops, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <mutex>

#include "internal.cuh"
#include "tc.cuh"

namespace art {
namespace {

constexpr int kThreads = 192;  // warp 0 TMA, warp 1 MMA + TMEM, warps 2..5 epilogue

__device__ __forceinline__ float* align16(float* p) {
  return reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}

struct TcParams {
  int H, W, cin, cout;
  int tiles_per_row, n_tiles;
  int act;
  const float* bias;
  void* out;             // BF16, or E4M3 for the FP8 network
  const float* in_scale;   // FP8: dequantisation scale of the input tensor (device scalar)
  const float* w_scale;    // FP8: per-output-channel weight scales [cout]
  const float* out_scale;  // FP8: quantisation scale of the output tensor (device scalar)
  unsigned int* out_amax;  // FP8: running max |output| (float bits) for the next call's scale
  int ld_out, ch_off, up2;
  float* rgba;           // fused 1x1 head (cout -> head_n <= 4) + sigmoid when non-null
  const float* head_w;   // [head_n][cout]
  const float* head_b;   // [head_n]
  int head_n, head_ld, head_off;  // head outputs, FP32 values per output pixel, channel of the first
  void* pool;            // row-blocked kernel: fused 2x2 max pooling, dense [H/2][W/2][cout] (BF16 or E4M3)
  int psplit;            // staged BF16 stores: x-phase split rows (even pixels, then odd)
  // sub-pixel decoder convolution (tap-by-tap kernel, BF16): H x W is the
  // low-resolution grid; a tile is (output phase, low-resolution row,
  // 128-pixel segment); its K chunks are 9 taps of the x-phase split skip
  // tensor (tmA, cs_ch chunks each) then 4 taps of the low-resolution tensor
  // (tmU, cu_ch chunks each); output pixel (2y + py, 2x + px)
  int sub, cs_ch, cu_ch;
  unsigned long long* err;
};

// One 32-channel BF16 group (64 B per pixel) of the warp's 32 pixels of
// output row y (this lane: x0 + lane), staged through stage[32 x 4] (chunk k
// of pixel q at 4 q + (k ^ (q % 4))) and stored four lanes per pixel into
// channels [ch_off + c0, + 32) (with up2: the pixel's 2x2 block; with an
// output phase ph >= 0 (sub-pixel tiles): pixel (2y + ph / 2, 2x + ph % 2)
// of the 2H x 2W output; with psplit: x-phase split rows).
__device__ __forceinline__ void store_staged_group(const TcParams& p, int y, int x0, int lane, int c0,
                                                   const uint4 (&pk)[4], uint4* stage, int ph = -1) {
#pragma unroll
  for (int k = 0; k < 4; ++k) stage[lane * 4 + (k ^ (lane & 3))] = pk[k];
  __syncwarp();
  __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(p.out);
  const int nd = p.up2 ? 4 : 1;
  const int Wd = (p.up2 || ph >= 0) ? 2 * p.W : p.W;
  for (int d = 0; d < nd; ++d) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int f = i * 32 + lane, q = f >> 2, c = f & 3;
      const int x = x0 + q;
      if (x < p.W) {
        int X, Y;
        if (ph >= 0) {
          X = 2 * x + (ph & 1);
          Y = 2 * y + (ph >> 1);
        } else {
          X = p.up2 ? 2 * x + (d & 1) : (p.psplit ? (x & 1) * (p.W >> 1) + (x >> 1) : x);
          Y = p.up2 ? 2 * y + (d >> 1) : y;
        }
        uint4* dst = reinterpret_cast<uint4*>(out + ((size_t)Y * Wd + X) * p.ld_out + p.ch_off + c0) + c;
        *dst = stage[q * 4 + (c ^ (q & 3))];
      }
    }
  }
  __syncwarp();
}

// Epilogue of one 128-pixel output row segment: this thread's pixel x of
// row y; the accumulator's N columns start at TMEM address taddr (lane
// quarter included).  Bias, ReLU, then BF16 / E4M3 store (optionally 2x2
// replicated into the upsampled concatenation), or the fused 1x1 head.
template <int N, bool F8>
__device__ __forceinline__ void epi_row(const TcParams& p, uint32_t taddr, int y, int x, const float* s_bias,
                                        const float* s_head, const float* s_wsc, float in_s, float out_inv,
                                        float& amax, uint4* stage = nullptr, int x0 = 0, int lane = 0, int ph = -1) {
  const bool valid = x < p.W;
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += 32) {
    uint32_t r[32];
    tmem_ld32(taddr + (uint32_t)c0, r);
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float acc = F8 ? __uint_as_float(r[j]) * (in_s * s_wsc[c0 + j]) : __uint_as_float(r[j]);
      const float t = acc + s_bias[c0 + j];
      v[j] = p.act == 1 ? fmaxf(t, 0.0f) : t;
    }
    if (!F8 && stage && !p.rgba) {  // BF16 group staged: the warp stores 8 pixels x 64 B per instruction
      uint4 pk[4];
      uint32_t* w = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<uint32_t*>(&b2);
      }
      store_staged_group(p, y, x0, lane, c0, pk, stage, ph);
      continue;
    }
    if (!valid) continue;
    if (p.rgba) {  // fused 1x1 head (N == 32) + sigmoid -> head_n FP32 channels of the output
      float o[4];
      const float4* hw = reinterpret_cast<const float4*>(s_head + c0);  // 16-B aligned rows of N weights
      // two partial sums per output: eight independent FMA chains of 16
      float a0[4], a1[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a0[k] = s_head[4 * N + k];
        a1[k] = 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 w = hw[k * (N / 4) + q];
          a0[k] = fmaf(w.x, v[4 * q], a0[k]);
          a1[k] = fmaf(w.y, v[4 * q + 1], a1[k]);
          a0[k] = fmaf(w.z, v[4 * q + 2], a0[k]);
          a1[k] = fmaf(w.w, v[4 * q + 3], a1[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        o[k] = __frcp_rn(1.0f + __expf(-(a0[k] + a1[k])));  // (fast exponential: relative error ~1e-6 on a [0, 1] output)
      float* dst = p.rgba + (size_t)(y * p.W + x) * p.head_ld + p.head_off;
      if (p.head_n == 4 && p.head_ld == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < p.head_n) dst[k] = o[k];
      }
      continue;
    }
    constexpr int kVec = F8 ? 2 : 4;  // 16-B stores of the 32 channels
    uint4 pk[kVec];
    if constexpr (F8) {
      uint16_t* w = reinterpret_cast<uint16_t*>(pk);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        amax = fmaxf(amax, fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1])));
        w[j] = (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(v[2 * j] * out_inv, v[2 * j + 1] * out_inv),
                                                  __NV_SATFINITE, __NV_E4M3);
      }
    } else {
      uint32_t* w = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<uint32_t*>(&b2);
      }
    }
    constexpr int kEs = F8 ? 1 : 2;
    uint8_t* outb = reinterpret_cast<uint8_t*>(p.out);
    if (!p.up2) {
      uint4* dst = reinterpret_cast<uint4*>(outb + (((size_t)y * p.W + x) * p.ld_out + p.ch_off + c0) * kEs);
#pragma unroll
      for (int k = 0; k < kVec; ++k) dst[k] = pk[k];
    } else {
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const size_t pix = (size_t)(2 * y + dy) * (2 * p.W) + (2 * x + dx);
          uint4* dst = reinterpret_cast<uint4*>(outb + (pix * p.ld_out + p.ch_off + c0) * kEs);
#pragma unroll
          for (int k = 0; k < kVec; ++k) dst[k] = pk[k];
        }
    }
  }
}

// Row-blocked epilogue, stores staged through shared memory.  A lane holds
// its pixel's N output channels (U 16-byte chunks after packing to BF16 or
// E4M3); written as they are, a warp store would put 32 16-byte pieces one
// pixel stride apart (32 cache lines per instruction, four times over with
// the 2x2 upsampling).  Instead the warp's 32 pixels are transposed through
// a 32 x U chunk buffer (chunk k of pixel q at q U + (k ^ (q % U)), so that
// neither the writes nor the reads conflict on banks) and stored U lanes per
// pixel: each store instruction covers 32 / U whole pixel blocks.
template <int N, bool F8>
struct RowOut {
  static constexpr int kEs = F8 ? 1 : 2;
  static constexpr int U = N * kEs / 16;  // 16-byte chunks of one pixel's outputs
};

// Bias, ReLU, rounding (BF16, or E4M3 with the dequantisation and output
// scales) of all N channels of this lane's pixel into pk.
template <int N, bool F8>
__device__ __forceinline__ void epi_pack(const TcParams& p, uint32_t taddr, const float* s_bias, const float* s_wsc,
                                         float in_s, float out_inv, float& amax, bool valid,
                                         uint4 (&pk)[RowOut<N, F8>::U]) {
#pragma unroll
  for (int c0 = 0; c0 < N; c0 += 32) {
    uint32_t r[32];
    tmem_ld32(taddr + (uint32_t)c0, r);
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float acc = F8 ? __uint_as_float(r[j]) * (in_s * s_wsc[c0 + j]) : __uint_as_float(r[j]);
      const float t = acc + s_bias[c0 + j];
      v[j] = p.act == 1 ? fmaxf(t, 0.0f) : t;
    }
    if constexpr (F8) {
      uint16_t* w = reinterpret_cast<uint16_t*>(pk) + c0 / 2;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (valid) amax = fmaxf(amax, fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1])));  // pixels of the image only
        w[j] = (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(v[2 * j] * out_inv, v[2 * j + 1] * out_inv),
                                                  __NV_SATFINITE, __NV_E4M3);
      }
    } else {
      uint32_t* w = reinterpret_cast<uint32_t*>(pk) + c0 / 2;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<uint32_t*>(&b2);
      }
    }
  }
}

// The warp's 32 pixels of output row y, x0 .. x0 + 31 (this lane: x0 + lane),
// through the staging buffer stage[32 U] into channels [ch_off, ch_off + N)
// of the ld_out-channel output (with up2: its 2x2 block of the 2H x 2W
// output).
template <int N, bool F8>
__device__ __forceinline__ void store_staged(const TcParams& p, int y, int x0, int lane,
                                             const uint4 (&pk)[RowOut<N, F8>::U], uint4* stage) {
  constexpr int U = RowOut<N, F8>::U;
  constexpr int kEs = RowOut<N, F8>::kEs;
#pragma unroll
  for (int k = 0; k < U; ++k) stage[lane * U + (k ^ (lane % U))] = pk[k];
  __syncwarp();
  uint8_t* outb = reinterpret_cast<uint8_t*>(p.out);
  const int nd = p.up2 ? 4 : 1;
  const int Wd = p.up2 ? 2 * p.W : p.W;
  for (int d = 0; d < nd; ++d) {
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int f = i * 32 + lane, q = f / U, c = f % U;
      const int x = x0 + q;
      if (x < p.W) {
        const int X = p.up2 ? 2 * x + (d & 1) : (p.psplit ? (x & 1) * (p.W >> 1) + (x >> 1) : x);
        const int Y = p.up2 ? 2 * y + (d >> 1) : y;
        uint4* dst = reinterpret_cast<uint4*>(outb + (((size_t)Y * Wd + X) * p.ld_out + p.ch_off) * kEs) + c;
        *dst = stage[q * U + (c ^ (q % U))];
      }
    }
  }
  __syncwarp();
}

// Epilogue of one output row of the row-blocked kernel with the 2x2 max
// pooling fused: the row's packed values are returned for the staged store
// (BF16, no upsampling), and kept (first row of a pair) or pooled with the kept
// row and the neighbouring pixel's lane (second row), the pooled pixel stored
// by the even lane.  Max and BF16 rounding commute, so this equals pooling
// the stored tensor.
template <int N>
__device__ __forceinline__ void epi_row_pool(const TcParams& p, uint32_t taddr, int y, int x, const float* s_bias,
                                             uint32_t (&keep)[N / 2], bool second, uint4 (&pk_all)[N / 8]) {
#pragma unroll
  for (int c0 = 0; c0 < N; c0 += 32) {
    uint32_t r[32];
    tmem_ld32(taddr + (uint32_t)c0, r);
    uint4 pk[4];
    uint32_t* w = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float t0 = __uint_as_float(r[2 * j]) + s_bias[c0 + 2 * j];
      float t1 = __uint_as_float(r[2 * j + 1]) + s_bias[c0 + 2 * j + 1];
      if (p.act == 1) {
        t0 = fmaxf(t0, 0.0f);
        t1 = fmaxf(t1, 0.0f);
      }
      __nv_bfloat162 b2 = __floats2bfloat162_rn(t0, t1);
      w[j] = *reinterpret_cast<uint32_t*>(&b2);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) pk_all[c0 / 8 + k] = pk[k];  // the row itself: stored staged by the caller
    if (!second) {
#pragma unroll
      for (int j = 0; j < 16; ++j) keep[c0 / 2 + j] = w[j];
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&keep[c0 / 2 + j]);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&w[j]);
        __nv_bfloat162 m = __hmax2(a, b);
        uint32_t mu = *reinterpret_cast<uint32_t*>(&m);
        uint32_t nu = __shfl_xor_sync(0xffffffffu, mu, 1);
        __nv_bfloat162 n = *reinterpret_cast<__nv_bfloat162*>(&nu);
        m = __hmax2(m, n);
        w[j] = *reinterpret_cast<uint32_t*>(&m);
      }
      const int Wp = p.W / 2, Hp = p.H / 2;
      if (!(x & 1) && (x >> 1) < Wp && (y >> 1) < Hp) {
        uint4* dst =
            reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(p.pool) + ((size_t)(y >> 1) * Wp + (x >> 1)) * N + c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = pk[k];
      }
    }
  }
}

// E4M3 epilogue of one output row with the fused 2x2 max pooling: the row
// is stored as epi_row stores it; the first row of a pair keeps its codes,
// the second takes the byte-wise maximum with them and with the neighbouring
// lane's (the codes of one scale order like their values, as the pooling
// pass of its own compares them) and writes the pooled pixel.
template <int N>
__device__ __forceinline__ void epi_row_pool_f8(const TcParams& p, uint32_t taddr, int y, int x, const float* s_bias,
                                                const float* s_wsc, float in_s, float out_inv, float& amax,
                                                uint32_t* keep, bool second) {
  const bool valid = x < p.W;
#pragma unroll
  for (int c0 = 0; c0 < N; c0 += 32) {
    uint32_t r[32];
    tmem_ld32(taddr + (uint32_t)c0, r);
    uint4 pk[2];
    uint16_t* w = reinterpret_cast<uint16_t*>(pk);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float t0 = __uint_as_float(r[2 * j]) * (in_s * s_wsc[c0 + 2 * j]) + s_bias[c0 + 2 * j];
      float t1 = __uint_as_float(r[2 * j + 1]) * (in_s * s_wsc[c0 + 2 * j + 1]) + s_bias[c0 + 2 * j + 1];
      if (p.act == 1) {
        t0 = fmaxf(t0, 0.0f);
        t1 = fmaxf(t1, 0.0f);
      }
      if (valid) amax = fmaxf(amax, fmaxf(fabsf(t0), fabsf(t1)));
      w[j] = (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(t0 * out_inv, t1 * out_inv), __NV_SATFINITE, __NV_E4M3);
    }
    if (valid) {
      uint4* dst = reinterpret_cast<uint4*>(static_cast<uint8_t*>(p.out) + ((size_t)y * p.W + x) * p.ld_out +
                                            p.ch_off + c0);
      dst[0] = pk[0];
      dst[1] = pk[1];
    }
    uint32_t* u = reinterpret_cast<uint32_t*>(pk);
    if (!second) {
#pragma unroll
      for (int k = 0; k < 8; ++k) keep[c0 / 4 + k] = u[k];
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t m = __vmaxu4(keep[c0 / 4 + k], u[k]);
        u[k] = __vmaxu4(m, __shfl_xor_sync(0xffffffffu, m, 1));
      }
      const int Wp = p.W / 2, Hp = p.H / 2;
      if (!(x & 1) && (x >> 1) < Wp && (y >> 1) < Hp) {
        uint4* dst = reinterpret_cast<uint4*>(static_cast<uint8_t*>(p.pool) + ((size_t)(y >> 1) * Wp + (x >> 1)) * N +
                                              c0);
        dst[0] = pk[0];
        dst[1] = pk[1];
      }
    }
  }
}

template <int N, int KCB, bool F8>
struct TcCfg {
  static constexpr int kA = 128 * KCB;
  static constexpr int kB = N * KCB;
  static constexpr int kStage = kA + kB;
  // two CTAs per SM (two issuing threads) where the accumulators fit twice in TMEM
  static constexpr int kCtas = (N <= 128 && !F8) ? 2 : 1;
  static constexpr int kStagesRaw = 196608 / kCtas / kStage;
  static constexpr int kStages = kStagesRaw > 24 ? 24 : kStagesRaw;
  static constexpr int kTmemCols = 2 * N;  // two accumulators; N in {32, 64, 128, 256}
  static constexpr uint32_t kFmt = F8 ? 0u : 1u;  // A/B format: E4M3 (kind::f8f6f4) or BF16 (kind::f16)
  static constexpr uint32_t kIdesc = (1u << 4)                          // D: FP32
                                     | (kFmt << 7) | (kFmt << 10)       // A, B formats
                                     | ((uint32_t)(N >> 3) << 17)       // N / 8
                                     | ((uint32_t)(128 >> 4) << 24);    // M / 16
  static constexpr int kStageBuf = F8 ? 0 : 4 * 32 * 4 * 16;  // BF16 epilogue staging: 4 warps x 32 pixels x 64 B
  static constexpr int kSmem =
      kStages * kStage + 1024 + 8 * (2 * kStages + 4) + 16 + 4 * N + 16 + 4 * (4 * 32 + 4) + 4 * N + 16 + kStageBuf;
};

template <int N, int KCB, bool F8>
__global__ void __launch_bounds__(kThreads, TcCfg<N, KCB, F8>::kCtas)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmU, TcParams p) {
  using Cfg = TcCfg<N, KCB, F8>;
  constexpr int KC = F8 ? KCB : KCB / 2;  // channels per K chunk
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* stages = sm;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + Cfg::kStages * Cfg::kStage);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* accf = empty + Cfg::kStages;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* s_bias = reinterpret_cast<float*>(tmem_slot + 4);
  float* s_head = align16(s_bias + N);  // (read as float4 rows)
  float* s_wsc = s_head + 4 * 32 + 4;  // FP8 per-output-channel weight scales
  uint4* s_stage = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(s_wsc + N) + 15) & ~(uintptr_t)15);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpt = p.cin / KC;  // K chunks per tap
  const int n_skip = 9 * p.cs_ch;  // sub-pixel tiles: the skip part's chunks, then 4 taps x cu_ch
  const int n_chunks = p.sub ? n_skip + 4 * p.cu_ch : 9 * cpt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < N; i += kThreads) s_bias[i] = i < p.cout ? p.bias[i] : 0.0f;
  if (p.rgba)
    for (int i = threadIdx.x; i < 4 * N + 4; i += kThreads)  // rows beyond head_n are zero
      s_head[i] = i < 4 * N ? (i < p.head_n * N ? p.head_w[i] : 0.0f) : (i - 4 * N < p.head_n ? p.head_b[i - 4 * N] : 0.0f);
  if (F8)
    for (int i = threadIdx.x; i < N; i += kThreads) s_wsc[i] = i < p.cout ? p.w_scale[i] : 0.0f;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  float amax = 0.0f;  // FP8 epilogue: max |output| seen by this thread
  grid_dep_launch();  // the next layer may start its prologue where this one's CTAs leave SMs
  grid_dep_wait();    // the previous layer's outputs (this one's input) are complete

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      for (int tile = blockIdx.x; tile < p.n_tiles && !*abort_flag; tile += gridDim.x) {
        const int st = p.sub ? tile >> 2 : tile, oph = tile & 3;  // (sub-pixel: output phase (py, px))
        const int y = st / p.tiles_per_row, x0 = (st % p.tiles_per_row) * 128;
        for (int c = 0; c < n_chunks; ++c) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
          uint8_t* a = stages + s * Cfg::kStage;
          mbar_expect_tx(&full[s], Cfg::kStage);
          if (!p.sub) {
            const int tap = c / cpt, cc = c - tap * cpt;
            const int r = tap / 3, q = tap - 3 * (tap / 3);
            tma_load_3d(a, &tmA, &full[s], cc * KC, x0 + q - 1, y + r - 1);
            tma_load_2d(a + Cfg::kA, &tmB, &full[s], tap * p.cin + cc * KC, 0);
          } else if (c < n_skip) {
            // skip tap (dy, dx): input column 2x + px + dx = 2 (x + jo) + q of the x-phase split rows
            const int tap = c / p.cs_ch, cc = c - tap * p.cs_ch;
            const int dy = tap / 3 - 1, cpos = (oph & 1) + tap % 3 - 1;
            const int q = cpos & 1, jo = (cpos - q) / 2;
            tma_load_4d(a, &tmA, &full[s], cc * KC, x0 + jo, q, 2 * y + (oph >> 1) + dy);
            tma_load_2d(a + Cfg::kA, &tmB, &full[s], tap * p.cs_ch * KC + cc * KC, oph * N);
          } else {
            // low-resolution tap (oy, ox), oy in {py - 1, py}, ox in {px - 1, px}
            const int t = c - n_skip, tu = t / p.cu_ch, cc = t - tu * p.cu_ch;
            const int oy = (oph >> 1) - 1 + (tu >> 1), ox = (oph & 1) - 1 + (tu & 1);
            tma_load_3d(a, &tmU, &full[s], cc * KC, x0 + ox, y + oy);
            tma_load_2d(a + Cfg::kA, &tmB, &full[s], (9 * p.cs_ch + tu * p.cu_ch) * KC + cc * KC, oph * N);
          }
          if (++s == Cfg::kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      int s = 0, buf = 0;
      uint32_t ph = 0, aph = 0;
      for (int tile = blockIdx.x; tile < p.n_tiles && !*abort_flag; tile += gridDim.x) {
        if (!mbar_wait(&acce[buf], aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(buf * N);
        bool ok = true;
        for (int c = 0; c < n_chunks; ++c) {
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(stages + s * Cfg::kStage), b = a + Cfg::kA;
#pragma unroll
          for (int kk = 0; kk < KCB / 32; ++kk)
            umma<F8>(d, umma_desc<KCB>(a + kk * 32), umma_desc<KCB>(b + kk * 32), Cfg::kIdesc, (c | kk) != 0);
          umma_commit(&empty[s]);
          if (++s == Cfg::kStages) {
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
    // ---------------------------------------------------------------- epilogue
    const int qd = warp & 3;           // TMEM lane quarter this warp may access
    const int m = qd * 32 + lane;      // row of the tile = pixel offset
    const float in_s = F8 ? *p.in_scale : 1.0f;
    const float out_inv = (F8 && p.out) ? 1.0f / *p.out_scale : 1.0f;
    int buf = 0;
    uint32_t aph = 0;
    for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
      if (!mbar_wait(&accf[buf], aph, abort_flag, 256)) break;
      tc_fence_after();
      const int st = p.sub ? tile >> 2 : tile;
      const int y = st / p.tiles_per_row, x = (st % p.tiles_per_row) * 128 + m;
      epi_row<N, F8>(p, tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(buf * N), y, x, s_bias, s_head, s_wsc,
                     in_s, out_inv, amax, F8 ? nullptr : s_stage + (warp - 2) * 32 * 4, x - lane, lane,
                     p.sub ? (tile & 3) : -1);
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      if (++buf == 2) {
        buf = 0;
        aph ^= 1u;
      }
    }
  }
  if (F8 && warp >= 2 && p.out_amax) {  // running max |output| for the next call's scale
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) atomicMax(p.out_amax, __float_as_uint(amax));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                              "r"(Cfg::kTmemCols));
  if (threadIdx.x == 0 && *abort_flag) atomicAdd(p.err, 1ull);
}

// Row-blocked variant for the narrow layers (N = 32 or 64 output channels,
// BF16): the weights of all nine taps stay in shared memory for the whole
// persistent loop, and a work unit is R = 4 output rows of one 128-pixel
// segment.  The producer brings each of the R + 2 input rows, per channel
// chunk, as one box of 130 pixels (x - 1 .. x + 128); the three horizontal
// taps read it from row 0, 1 or 2 of the box, and every box serves the up to
// three output rows it neighbours vertically (one MMA per row into that
// row's accumulator).  Per output row that is (R + 2) / R boxes instead of
// 9, and no weight traffic.  Accumulators: R x N TMEM columns per unit, two
// units in flight.
constexpr int kRows = 4;

// The vertical taps are stacked into one operand:
// the accumulators of the unit's R output rows sit in consecutive TMEM
// column slots in reverse row order (slot of output row r = R - 1 - r), so
// that one MMA per input-row box, N x (the taps whose output row lies in
// the unit: 3 inside, 2 or 1 at the unit's edge rows) columns, accumulates into
// every row it touches.  Every MMA accumulates; the epilogue zeroes each
// slot after reading it.
template <int N, int KCB, bool F8 = false>
struct RowCfg {
  static constexpr int KC = F8 ? KCB : KCB / 2;  // channels per chunk (KCB bytes)
  static constexpr int kSlots = kRows;
  static constexpr int kBufCols = kSlots * N;  // columns of one accumulator buffer
  static constexpr int kHalo = 130;                                   // input pixels of a row box (128 + 2)
  // input rows per stage (one box); two measured slower on the 32-channel
  // layers (a deeper box per barrier round trip, half as many stages in flight)
  static constexpr int kStageRows = 1;
  static constexpr int kRowBytes = kHalo * KCB;                       // one input row of the box
  static constexpr int kBoxBytes = kStageRows * kRowBytes;
  static constexpr int kStageBytes = (kBoxBytes + 1023) / 1024 * 1024;  // stages stay on swizzle-atom boundaries
  static_assert((kRows + 2) % kStageRows == 0, "a unit's input rows fill whole stages");
};

struct RowParams {
  TcParams p;
  int cpt;        // channel chunks per tap
  int n_units;    // ceil(H / R) x tiles per row
  int n_stages;   // stages in flight (three boxes each)
  int w_bytes;    // resident weights: 9 x cpt blocks of N x KCB bytes
  int nbuf;       // accumulator buffers (2, or 1 when two CTAs share an SM's TMEM)
};

template <int N, int KCB, bool F8>
__global__ void __launch_bounds__(kThreads, 2)
    conv_rows_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, RowParams rp) {
  using Cfg = RowCfg<N, KCB, F8>;
  const TcParams& p = rp.p;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* wsm = sm;
  uint8_t* stages = sm + rp.w_bytes;
  const int S = rp.n_stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(stages + (size_t)S * Cfg::kStageBytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint64_t* wbar = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* s_bias = reinterpret_cast<float*>(tmem_slot + 4);
  float* s_head = align16(s_bias + N);  // (read as float4 rows)
  float* s_wsc = s_head + 4 * 32 + 4;  // FP8 per-output-channel weight scales
  // epilogue store staging: 32 pixels x U chunks per epilogue warp (16-B aligned)
  uint4* s_stage = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(s_wsc + N) + 15) & ~(uintptr_t)15);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpt = rp.cpt;
  const int n_stage_unit = (kRows + 2) / Cfg::kStageRows * cpt;  // stages per unit
  const int kStage = Cfg::kStageBytes;  // one box of kStageRows rows of 130 pixels: the three shifts are row offsets
  // the swizzle follows the absolute shared-memory address, so a descriptor
  // may start at any row of the box: shift dx is the box from row dx on
  // resident weight block of (dy + 1, dx + 1, chunk): the three vertical
  // taps of one (dx, chunk) are adjacent (one stacked operand of up to 3 N rows)
  auto wblk = [&](int dyi, int dxi, int c) { return (dxi * cpt + c) * 3 + dyi; };

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
  for (int i = threadIdx.x; i < N; i += kThreads) s_bias[i] = i < p.cout ? p.bias[i] : 0.0f;
  if (p.rgba)
    for (int i = threadIdx.x; i < 4 * N + 4; i += kThreads)  // rows beyond head_n are zero
      s_head[i] = i < 4 * N ? (i < p.head_n * N ? p.head_w[i] : 0.0f) : (i - 4 * N < p.head_n ? p.head_b[i - 4 * N] : 0.0f);
  if (F8)
    for (int i = threadIdx.x; i < N; i += kThreads) s_wsc[i] = i < p.cout ? p.w_scale[i] : 0.0f;
  const int nbuf = rp.nbuf;
  const uint32_t tmem_cols = (uint32_t)(nbuf * Cfg::kBufCols);
  if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  float amax = 0.0f;

  // A stage is kStageRows input rows of one channel chunk (one box, one
  // barrier round trip); each row serves the three horizontal shifts.
  grid_dep_launch();  // the next layer may start its prologue where this one's CTAs leave SMs
  if (warp == 0) {
    // ------------------------------------------------------------ TMA
    if (lane == 0) {
      mbar_expect_tx(wbar, (uint32_t)rp.w_bytes);  // the weights are static: loaded before the wait
      for (int tap = 0; tap < 9; ++tap)
        for (int c = 0; c < cpt; ++c)
          tma_load_2d(wsm + (size_t)wblk(tap / 3, tap % 3, c) * N * KCB, &tmB, wbar, tap * p.cin + c * Cfg::KC, 0);
    }
    grid_dep_wait();  // the previous layer's outputs (this one's input) are complete
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      for (int u = blockIdx.x; u < rp.n_units && !*abort_flag; u += gridDim.x) {
        const int y0 = (u / p.tiles_per_row) * kRows, x0 = (u % p.tiles_per_row) * 128;
        for (int st = 0; st < n_stage_unit; ++st) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
          const int jj = st / cpt, c = st - jj * cpt;
          uint8_t* dst = stages + (size_t)s * kStage;
          mbar_expect_tx(&full[s], (uint32_t)Cfg::kBoxBytes);
          tma_load_3d(dst, &tmA, &full[s], c * Cfg::KC, x0 - 1, y0 - 1 + jj * Cfg::kStageRows);
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
      const uint32_t wbase = smem_u32(wsm);
      for (int u = blockIdx.x; ok && u < rp.n_units && !*abort_flag; u += gridDim.x) {
        // the epilogue clears the accumulators (phase 0 = the initial clear)
        if (!mbar_wait(&acce[buf], aph, abort_flag)) break;
        tc_fence_after();
        const uint32_t d0 = tmem_base + (uint32_t)(buf * Cfg::kBufCols);
        for (int st = 0; st < n_stage_unit; ++st) {
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int jj = st / cpt, c = st - jj * cpt;
#pragma unroll
          for (int r = 0; r < Cfg::kStageRows; ++r) {
            const int j = jj * Cfg::kStageRows + r;
            const uint32_t a0 = smem_u32(stages + (size_t)s * kStage) + (uint32_t)(r * Cfg::kRowBytes);
            // input row j feeds output rows j - dyi of the unit for the taps dyi in [lo, hi]
            // (slots R - 1 - j + lo ..., consecutive like the stacked taps' weight blocks)
            const int lo = max(0, j - kRows + 1), hi = min(2, j);
            const uint32_t dj = d0 + (uint32_t)((kRows - 1 - j + lo) * N);
            const uint32_t idesc = F8 ? idesc_e4m3(128, (hi - lo + 1) * N) : idesc_bf16(128, (hi - lo + 1) * N);
#pragma unroll
            for (int dxi = 0; dxi < 3; ++dxi) {
              const uint32_t bw = wbase + (uint32_t)((wblk(0, dxi, c) + lo) * N * KCB);
#pragma unroll
              for (int kk = 0; kk < KCB / 32; ++kk)
                umma<F8>(dj, umma_desc<KCB>(a0 + dxi * KCB + kk * 32), umma_desc<KCB>(bw + kk * 32), idesc, 1u);
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
        if (++buf == nbuf) {
          buf = 0;
          aph ^= 1u;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    grid_dep_wait();  // the output tensors may still be read by the previous layer
    const int qd = warp & 3;
    const int m = qd * 32 + lane;
    const uint32_t tq = tmem_base + ((uint32_t)(qd * 32) << 16);  // this warp's lane quarter
    const float in_s = F8 ? *p.in_scale : 1.0f;
    const float out_inv = (F8 && p.out) ? 1.0f / *p.out_scale : 1.0f;
    uint32_t keep[N / 2];  // fused pooling: the first row of the pair, packed BF16 (or E4M3 codes)
    int buf = 0;
    uint32_t aph = 0;
    {  // zero every slot of both buffers, then release them to the MMA
      for (int c0 = 0; c0 < (int)tmem_cols; c0 += 32) tmem_zero32(tq + (uint32_t)c0);
      tmem_wait_st();
      tc_fence_before();
      for (int b = 0; b < nbuf; ++b) mbar_arrive(&acce[b]);
    }
    for (int u = blockIdx.x; u < rp.n_units; u += gridDim.x) {
      if (!mbar_wait(&accf[buf], aph, abort_flag, 256)) break;
      tc_fence_after();
      const int y0 = (u / p.tiles_per_row) * kRows, x = (u % p.tiles_per_row) * 128 + m;
      for (int r = 0; r < kRows; ++r) {
        const int slot = kRows - 1 - r;
        const uint32_t ta = tq + (uint32_t)(buf * Cfg::kBufCols + slot * N);
        if (y0 + r < p.H) {
          uint4* stg = s_stage + (warp - 2) * 32 * RowOut<N, F8>::U;
          const int xw = (u % p.tiles_per_row) * 128 + qd * 32;  // this warp's first pixel
          if (p.rgba) {
            epi_row<N, F8>(p, ta, y0 + r, x, s_bias, s_head, s_wsc, in_s, out_inv, amax);  // coalesced already
          } else if constexpr (!F8) {
            uint4 pk[RowOut<N, false>::U];
            if (p.pool)
              epi_row_pool<N>(p, ta, y0 + r, x, s_bias, keep, (r & 1) != 0, pk);
            else
              epi_pack<N, false>(p, ta, s_bias, s_wsc, in_s, out_inv, amax, x < p.W, pk);
            store_staged<N, false>(p, y0 + r, xw, lane, pk, stg);
          } else if (p.pool) {  // E4M3 rows are 32 or 64 bytes: stored directly (staging measured slower)
            epi_row_pool_f8<N>(p, ta, y0 + r, x, s_bias, s_wsc, in_s, out_inv, amax, keep, (r & 1) != 0);
          } else {
            epi_row<N, true>(p, ta, y0 + r, x, s_bias, s_head, s_wsc, in_s, out_inv, amax);
          }
        }
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 32) tmem_zero32(ta + (uint32_t)c0);
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      if (++buf == nbuf) {
        buf = 0;
        aph ^= 1u;
      }
    }
  }
  if (F8 && warp >= 2 && p.out_amax) {  // running max |output| for the next call's scale
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) atomicMax(p.out_amax, __float_as_uint(amax));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, tmem_cols);
  if (threadIdx.x == 0 && *abort_flag) atomicAdd(p.err, 1ull);
}

// 2x2 max pooling of a channel slice [ch_off, ch_off + C) of an NHWC tensor
// with ld channels per pixel (rows x-phase split when psplit: even pixels,
// then odd), into a dense [H/2][W/2][C] tensor.
__global__ void maxpool2_bf16_kernel(const __nv_bfloat16* __restrict__ in, int ld, int ch_off,
                                     __nv_bfloat16* __restrict__ out, int H, int W, int C, int psplit) {
  const int C8 = C / 8;
  const int64_t total = (int64_t)(H / 2) * (W / 2) * C8;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C8) * 8;
    const int64_t pp = idx / C8;
    const int x = (int)(pp % (W / 2)), y = (int)(pp / (W / 2));
    // pixel 2x of row 2y and its right neighbour (in the odd half when x-phase split)
    const __nv_bfloat16* q = in + (((size_t)(2 * y) * W) + (psplit ? x : 2 * x)) * ld + ch_off + c;
    const size_t nb = psplit ? (size_t)(W / 2) * ld : (size_t)ld;
    uint4 a = *reinterpret_cast<const uint4*>(q);
    uint4 b = *reinterpret_cast<const uint4*>(q + nb);
    uint4 cc = *reinterpret_cast<const uint4*>(q + (size_t)W * ld);
    uint4 d = *reinterpret_cast<const uint4*>(q + (size_t)W * ld + nb);
    const __nv_bfloat162* pa = reinterpret_cast<const __nv_bfloat162*>(&a);
    const __nv_bfloat162* pb = reinterpret_cast<const __nv_bfloat162*>(&b);
    const __nv_bfloat162* pc = reinterpret_cast<const __nv_bfloat162*>(&cc);
    const __nv_bfloat162* pd = reinterpret_cast<const __nv_bfloat162*>(&d);
    uint4 o;
    __nv_bfloat162* po = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int k = 0; k < 4; ++k) po[k] = __hmax2(__hmax2(pa[k], pb[k]), __hmax2(pc[k], pd[k]));
    *reinterpret_cast<uint4*>(out + (size_t)pp * C + c) = o;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

template <int N, int KCB, bool F8>
art_status launch_typed(art_ctx* ctx, const TcConv& c) {
  using Cfg = TcCfg<N, KCB, F8>;
  constexpr int kEs = F8 ? 1 : 2;
  constexpr int KC = KCB / kEs;
  const CUtensorMapDataType dt = F8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle swz = KCB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                            : (KCB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  CUtensorMap tmA, tmB, tmU;
  const int gh = c.sub ? c.H / 2 : c.H, gw = c.sub ? c.W / 2 : c.W;  // the kernel's pixel grid
  if (!c.sub) {
    cuuint64_t dims[3] = {(cuuint64_t)c.cin, (cuuint64_t)c.W, (cuuint64_t)c.H};
    cuuint64_t strides[2] = {(cuuint64_t)c.cin * kEs, (cuuint64_t)c.W * c.cin * kEs};
    cuuint32_t box[3] = {(cuuint32_t)KC, 128, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(&tmA, dt, 3, (void*)c.in, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (activations) failed: %d", (int)r);
    tmU = tmA;
  } else {
    {  // skip tensor, x-phase split: (channel, x / 2, x % 2, y) at the output resolution
      cuuint64_t dims[4] = {(cuuint64_t)c.cs, (cuuint64_t)gw, 2, (cuuint64_t)c.H};
      cuuint64_t strides[3] = {(cuuint64_t)c.cs * kEs, (cuuint64_t)gw * c.cs * kEs, (cuuint64_t)c.W * c.cs * kEs};
      cuuint32_t box[4] = {(cuuint32_t)KC, 128, 1, 1};
      cuuint32_t es[4] = {1, 1, 1, 1};
      CUresult r = g_encode(&tmA, dt, 4, (void*)c.in, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (skip) failed: %d", (int)r);
    }
    {  // low-resolution tensor: (channel, x, y)
      cuuint64_t dims[3] = {(cuuint64_t)c.cu, (cuuint64_t)gw, (cuuint64_t)gh};
      cuuint64_t strides[2] = {(cuuint64_t)c.cu * kEs, (cuuint64_t)gw * c.cu * kEs};
      cuuint32_t box[3] = {(cuuint32_t)KC, 128, 1};
      cuuint32_t es[3] = {1, 1, 1};
      CUresult r = g_encode(&tmU, dt, 3, (void*)c.up, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (low resolution) failed: %d", (int)r);
    }
  }
  {  // weights: [cout][9 cin] (K-major), or per output phase [4][cout][9 cs + 4 cu]
    const int K = c.sub ? 9 * c.cs + 4 * c.cu : 9 * c.cin;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)(c.sub ? 4 : 1) * c.cout};
    cuuint64_t strides[1] = {(cuuint64_t)K * kEs};
    cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)N};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(&tmB, dt, 2, (void*)c.w, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (weights) failed: %d", (int)r);
  }
  TcParams p;
  p.H = gh;
  p.W = gw;
  p.cin = c.sub ? c.cs + c.cu : c.cin;
  p.cout = c.cout;
  p.tiles_per_row = (gw + 127) / 128;
  p.n_tiles = p.tiles_per_row * gh * (c.sub ? 4 : 1);
  p.sub = c.sub;
  p.cs_ch = c.sub ? c.cs / KC : 0;
  p.cu_ch = c.sub ? c.cu / KC : 0;
  p.act = c.act;
  p.bias = c.bias;
  p.out = c.out;
  p.in_scale = c.in_scale;
  p.w_scale = c.w_scale;
  p.out_scale = c.out_scale;
  p.out_amax = c.out_amax;
  p.ld_out = c.ld_out;
  p.ch_off = c.ch_off;
  p.up2 = c.up2;
  p.rgba = c.rgba;
  p.head_w = c.head_w;
  p.head_b = c.head_b;
  p.head_n = c.head_n;
  p.head_ld = c.head_ld;
  p.head_off = c.head_off;
  p.pool = nullptr;  // pooled by a pass of its own
  p.psplit = c.psplit;
  p.err = ctx->d_status + kStTcError;
  auto kfn = conv_tc_kernel<N, KCB, F8>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "conv_tc shared memory attribute");
  const int grid = std::min(p.n_tiles, Cfg::kCtas * ctx->num_sms);
  ART_LAUNCH_PDL(ctx, F8 ? "conv_tc_fp8" : "conv_tc", kfn, grid, kThreads, Cfg::kSmem, tmA, tmB, tmU, p);
  return ART_OK;
}

// 2x2 max pooling of E4M3 activations (non-negative after ReLU, whose bit
// patterns order like unsigned integers): byte-wise integer maximum.
__global__ void maxpool2_fp8_kernel(const uint8_t* __restrict__ in, int ld, int ch_off, uint8_t* __restrict__ out,
                                    int H, int W, int C) {
  const int C16 = C / 16;
  const int64_t total = (int64_t)(H / 2) * (W / 2) * C16;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C16) * 16;
    const int64_t pp = idx / C16;
    const int x = (int)(pp % (W / 2)), y = (int)(pp / (W / 2));
    const uint8_t* q = in + (((size_t)(2 * y) * W) + 2 * x) * ld + ch_off + c;
    uint4 a = *reinterpret_cast<const uint4*>(q);
    uint4 b = *reinterpret_cast<const uint4*>(q + ld);
    uint4 cc = *reinterpret_cast<const uint4*>(q + (size_t)W * ld);
    uint4 d = *reinterpret_cast<const uint4*>(q + (size_t)W * ld + ld);
    uint4 o;
    o.x = __vmaxu4(__vmaxu4(a.x, b.x), __vmaxu4(cc.x, d.x));
    o.y = __vmaxu4(__vmaxu4(a.y, b.y), __vmaxu4(cc.y, d.y));
    o.z = __vmaxu4(__vmaxu4(a.z, b.z), __vmaxu4(cc.z, d.z));
    o.w = __vmaxu4(__vmaxu4(a.w, b.w), __vmaxu4(cc.w, d.w));
    *reinterpret_cast<uint4*>(out + (size_t)pp * C + c) = o;
  }
}

}  // namespace

namespace {

constexpr int kRowsMaxWeights = 80 * 1024;  // resident weights of the row-blocked kernel
// E4M3: up to the 192 -> 64 layer (110.6 KB, one CTA per SM)
constexpr int kRowsMaxWeightsF8 = 112 * 1024;

template <int N, int KCB, bool F8>
art_status launch_rows(art_ctx* ctx, const TcConv& c) {
  using Cfg = RowCfg<N, KCB, F8>;
  constexpr int kEs = F8 ? 1 : 2;
  const CUtensorMapDataType dt = F8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap tmA, tmB;
  const CUtensorMapSwizzle swz = KCB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                            : (KCB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  {
    cuuint64_t dims[3] = {(cuuint64_t)c.cin, (cuuint64_t)c.W, (cuuint64_t)c.H};
    cuuint64_t strides[2] = {(cuuint64_t)c.cin * kEs, (cuuint64_t)c.W * c.cin * kEs};
    cuuint32_t box[3] = {(cuuint32_t)Cfg::KC, (cuuint32_t)Cfg::kHalo, (cuuint32_t)Cfg::kStageRows};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(&tmA, dt, 3, (void*)c.in, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (activations) failed: %d", (int)r);
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)9 * c.cin, (cuuint64_t)c.cout};
    cuuint64_t strides[1] = {(cuuint64_t)9 * c.cin * kEs};
    cuuint32_t box[2] = {(cuuint32_t)Cfg::KC, (cuuint32_t)N};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(&tmB, dt, 2, (void*)c.w, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, ART_ERR_CUDA, "cuTensorMapEncodeTiled (weights) failed: %d", (int)r);
  }
  RowParams rp;
  TcParams& p = rp.p;
  p = TcParams{};
  p.H = c.H;
  p.W = c.W;
  p.cin = c.cin;
  p.cout = c.cout;
  p.tiles_per_row = (c.W + 127) / 128;
  p.n_tiles = p.tiles_per_row * c.H;
  p.act = c.act;
  p.bias = c.bias;
  p.out = c.out;
  p.ld_out = c.ld_out;
  p.ch_off = c.ch_off;
  p.up2 = c.up2;
  p.rgba = c.rgba;
  p.head_w = c.head_w;
  p.head_b = c.head_b;
  p.head_n = c.head_n;
  p.head_ld = c.head_ld;
  p.head_off = c.head_off;
  p.pool = c.pool;
  p.psplit = c.psplit;
  p.in_scale = c.in_scale;
  p.w_scale = c.w_scale;
  p.out_scale = c.out_scale;
  p.out_amax = c.out_amax;
  p.err = ctx->d_status + kStTcError;
  rp.cpt = c.cin / Cfg::KC;
  rp.n_units = ((c.H + kRows - 1) / kRows) * p.tiles_per_row;
  rp.w_bytes = 9 * rp.cpt * N * KCB;
  const int tail =
      8 * (2 * 24 + 5) + 16 + 4 * N + 16 + 4 * (4 * 32 + 4) + 4 * N + 16 + (F8 ? 0 : 4 * 32 * 16 * RowOut<N, F8>::U);
  // two CTAs per SM (two issuing threads, one accumulator buffer each) when
  // the resident weights and three input rows fit in half the shared memory
  const int half = 232448 / 2 - 1024 - rp.w_bytes - tail;
  auto kfn = conv_rows_kernel<N, KCB, F8>;
  cudaFuncAttributes fa;
  const bool regs2 = cudaFuncGetAttributes(&fa, kfn) == cudaSuccess && 2 * kThreads * fa.numRegs <= 65536;
  // (at least three input rows in flight per CTA) and both CTAs' registers fit
  const int ctas = (half >= (3 + Cfg::kStageRows - 1) / Cfg::kStageRows * Cfg::kStageBytes && regs2) ? 2 : 1;
  const int avail = 232448 / ctas - 1024 - rp.w_bytes - tail;
  rp.nbuf = (ctas == 2 && Cfg::kBufCols > 128) ? 1 : 2;  // 512 TMEM columns per SM
  rp.n_stages = std::min(24, avail / Cfg::kStageBytes);
  if (rp.n_stages < 2) return fail(ctx, ART_ERR_UNSUPPORTED, "row-blocked conv: weights too large");
  const int smem = 1024 + rp.w_bytes + rp.n_stages * Cfg::kStageBytes + tail;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "conv_rows shared memory attribute");
  const int grid = std::min(rp.n_units, ctas * ctx->num_sms);
  ART_LAUNCH_PDL(ctx, F8 ? "conv_tc_fp8" : "conv_tc", kfn, grid, kThreads, smem, tmA, tmB, rp);
  return ART_OK;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn() ? g_encode : nullptr; }

bool tc_conv_ok(const TcConv& c) {
  const bool n_ok = c.cout == 32 || c.cout == 64 || c.cout == 128 || c.cout == 256;
  const int al = c.f8 ? 16 : 8;  // 16-byte aligned output rows and channel offsets
  // x-phase split output: BF16 through the staged stores, even widths
  const bool ps_ok = !c.psplit || (!c.f8 && !c.up2 && !c.rgba && c.W % 2 == 0);
  // sub-pixel decoder convolution: BF16, dense output, 32-channel chunks of both parts
  const bool sub_ok = !c.sub || (!c.f8 && !c.up2 && !c.rgba && !c.pool && !c.psplit && c.ch_off == 0 &&
                                 c.ld_out == c.cout && c.H % 2 == 0 && c.W % 2 == 0 && c.cs % 32 == 0 &&
                                 c.cu % 32 == 0 && c.cs > 0 && c.cu > 0 && c.cin == c.cs + c.cu);
  return n_ok && (c.cin % 32 == 0) && c.cin >= 32 && (c.ld_out % al == 0) && (c.ch_off % al == 0) &&
         (!c.rgba || c.cout == 32) && ps_ok && sub_ok && encode_fn();
}

art_status launch_tc_conv(art_ctx* ctx, const TcConv& c) {
  if (!tc_conv_ok(c)) return fail(ctx, ART_ERR_UNSUPPORTED, "tensor-core conv: unsupported shape");
  if (c.sub) {  // the tap-by-tap kernel over sub-pixel tiles
    const bool k64 = c.cs % 64 == 0 && c.cu % 64 == 0;
    switch (c.cout) {
      case 32: return k64 ? launch_typed<32, 128, false>(ctx, c) : launch_typed<32, 64, false>(ctx, c);
      case 64: return k64 ? launch_typed<64, 128, false>(ctx, c) : launch_typed<64, 64, false>(ctx, c);
      case 128: return k64 ? launch_typed<128, 128, false>(ctx, c) : launch_typed<128, 64, false>(ctx, c);
      default: return k64 ? launch_typed<256, 128, false>(ctx, c) : launch_typed<256, 64, false>(ctx, c);
    }
  }
  if (c.f8) {  // row bytes = channels per K chunk: 128, 64 or 32
    const int kcb = c.cin % 128 == 0 ? 128 : (c.cin % 64 == 0 ? 64 : 32);
    if ((c.cout == 32 || c.cout == 64) && 9 * c.cin * c.cout <= kRowsMaxWeightsF8 && ctx->conv_rows &&
        (!c.pool || (!c.up2 && !c.rgba))) {
      // the narrow layers on the row-blocked kernel: K = 32 per FP8 MMA halves its instruction count
#define ART_F8R(NN)                                                                \
  return kcb == 128 ? launch_rows<NN, 128, true>(ctx, c)                           \
                    : (kcb == 64 ? launch_rows<NN, 64, true>(ctx, c) : launch_rows<NN, 32, true>(ctx, c))
      if (c.cout == 32) {
        ART_F8R(32);
      }
      ART_F8R(64);
#undef ART_F8R
    }
#define ART_F8(NN)                                                             \
  st = kcb == 128 ? launch_typed<NN, 128, true>(ctx, c)                        \
                  : (kcb == 64 ? launch_typed<NN, 64, true>(ctx, c) : launch_typed<NN, 32, true>(ctx, c))
    art_status st;
    switch (c.cout) {
      case 32: ART_F8(32); break;
      case 64: ART_F8(64); break;
      case 128: ART_F8(128); break;
      default: ART_F8(256); break;
    }
#undef ART_F8
    if (st == ART_OK && c.pool)  // (the tap-by-tap kernel pools in a pass of its own)
      launch_pool_fp8(ctx, (const uint8_t*)c.out, c.ld_out, c.ch_off, (uint8_t*)c.pool, c.H, c.W, c.cout);
    return st;
  }
  const bool k64 = c.cin % 64 == 0;  // BF16: 64 channels = 128-B rows, else 32 = 64-B rows
  if ((c.cout == 32 || c.cout == 64) && 9 * c.cin * c.cout * 2 <= kRowsMaxWeights && ctx->conv_rows &&
      (!c.pool || (!c.up2 && !c.rgba))) {
    if (c.cout == 32) return k64 ? launch_rows<32, 128, false>(ctx, c) : launch_rows<32, 64, false>(ctx, c);
    return k64 ? launch_rows<64, 128, false>(ctx, c) : launch_rows<64, 64, false>(ctx, c);
  }
  art_status st;
  switch (c.cout) {
    case 32: st = k64 ? launch_typed<32, 128, false>(ctx, c) : launch_typed<32, 64, false>(ctx, c); break;
    case 64: st = k64 ? launch_typed<64, 128, false>(ctx, c) : launch_typed<64, 64, false>(ctx, c); break;
    case 128: st = k64 ? launch_typed<128, 128, false>(ctx, c) : launch_typed<128, 64, false>(ctx, c); break;
    default: st = k64 ? launch_typed<256, 128, false>(ctx, c) : launch_typed<256, 64, false>(ctx, c); break;
  }
  if (st == ART_OK && c.pool)
    launch_pool_bf16(ctx, (const __nv_bfloat16*)c.out, c.ld_out, c.ch_off, (__nv_bfloat16*)c.pool, c.H, c.W, c.cout,
                     c.psplit);
  return st;
}

void launch_pool_bf16(art_ctx* ctx, const __nv_bfloat16* in, int ld, int ch_off, __nv_bfloat16* out, int H, int W,
                      int C, int psplit) {
  const int64_t total = (int64_t)(H / 2) * (W / 2) * (C / 8);
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8);
  ART_LAUNCH(ctx, "maxpool2_bf16", maxpool2_bf16_kernel, grid, 256, 0, in, ld, ch_off, out, H, W, C, psplit);
}

namespace {

constexpr float kE4M3Max = 448.0f;

// Per-output-channel E4M3 weights: scale_co = max |w_co| / 448, w8 = rn(w / scale_co).
__global__ void quantize_weights_kernel(const float* __restrict__ w, int K, uint8_t* __restrict__ w8,
                                        float* __restrict__ scale) {
  const int co = blockIdx.x;
  const float* row = w + (size_t)co * K;
  float m = 0.0f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmaxf(m, fabsf(row[k]));
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const float s = fmaxf(red[0], 1e-30f) / kE4M3Max;
  if (threadIdx.x == 0) scale[co] = s;
  const float inv = 1.0f / s;
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    w8[(size_t)co * K + k] = (uint8_t)__nv_cvt_float_to_fp8(row[k] * inv, __NV_SATFINITE, __NV_E4M3);
}

// BF16 feature map -> E4M3 with the current input scale; records max |F|.
// Sixteen values per thread and step (two 16-B loads, one 16-B store) when
// both arrays are 16-byte aligned (vec); the rest pair by pair.
__global__ void quantize_input_kernel(const __nv_bfloat16* __restrict__ in, int64_t m, const float* __restrict__ scale,
                                      uint8_t* __restrict__ out, unsigned int* __restrict__ amax, int vec) {
  ART_PDL_ENTRY();
  const float inv = 1.0f / *scale;
  float a = 0.0f;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t m16 = vec ? m / 16 : 0;
  for (int64_t g = tid; g < m16; g += nth) {
    const uint4* src = reinterpret_cast<const uint4*>(in + g * 16);
    const uint4 x0 = src[0], x1 = src[1];
    const uint32_t w[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t u = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t b = w[2 * k + h];
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&b));
        a = fmaxf(a, fmaxf(fabsf(v.x), fabsf(v.y)));
        u |= (uint32_t)(uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(v.x * inv, v.y * inv), __NV_SATFINITE, __NV_E4M3)
             << (16 * h);
      }
      o[k] = u;
    }
    *reinterpret_cast<uint4*>(out + g * 16) = make_uint4(o[0], o[1], o[2], o[3]);
  }
  for (int64_t i = m16 * 16 + tid * 2; i < m; i += nth * 2) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(in + i));
    a = fmaxf(a, fmaxf(fabsf(v.x), fabsf(v.y)));
    *reinterpret_cast<uint16_t*>(out + i) =
        (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(v.x * inv, v.y * inv), __NV_SATFINITE, __NV_E4M3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(a));
}

// Delayed scaling: next call's scale = max |value| of this call / 448; or a
// fixed value (calibration).
__global__ void update_scales_kernel(float* __restrict__ scale, unsigned int* __restrict__ amax, int n, float fixed) {
  ART_PDL_ENTRY();
  const int i = threadIdx.x;
  if (i >= n) return;
  scale[i] = fixed > 0.0f ? fixed : fmaxf(__uint_as_float(amax[i]), 1e-12f) / kE4M3Max;
  amax[i] = 0u;
}

}  // namespace

void launch_quantize_weights(art_ctx* ctx, const float* w, int cout, int K, uint8_t* w8, float* scale) {
  ART_LAUNCH(ctx, "quantize_w_fp8", quantize_weights_kernel, cout, 256, 0, w, K, w8, scale);
}

void launch_quantize_input(art_ctx* ctx, const __nv_bfloat16* in, int64_t m, const float* scale, uint8_t* out,
                           unsigned int* amax) {
  const int vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const int64_t per = vec ? 16 : 2;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m / per + 255) / 256, (int64_t)ctx->num_sms * 8));
  ART_LAUNCH_PDL(ctx, "quantize_f_fp8", quantize_input_kernel, grid, 256, 0, in, m, scale, out, amax, vec);
}

void launch_update_scales(art_ctx* ctx, float* scale, unsigned int* amax, int n, float fixed) {
  ART_LAUNCH_PDL(ctx, "fp8_scales", update_scales_kernel, 1, 32, 0, scale, amax, n, fixed);
}

void launch_pool_fp8(art_ctx* ctx, const uint8_t* in, int ld, int ch_off, uint8_t* out, int H, int W, int C) {
  const int64_t total = (int64_t)(H / 2) * (W / 2) * (C / 16);
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8);
  ART_LAUNCH(ctx, "maxpool2_fp8", maxpool2_fp8_kernel, grid, 256, 0, in, ld, ch_off, out, H, W, C);
}

}  // namespace art
