// Dynamic volume rendering of the warped voxels into the feature map F and
// the coarse opacity map A (arXiv 2202.05628, Sec. 3.1 "Dynamic Volume
// Rendering", Eq. 5-6 and the early-stop rule).
//
// One 64-thread CTA per 8x8 screen tile, one thread per pixel; warp w owns
// the 8x4 pixel strip of rows 4w..4w+3.  The tile's instance list is sorted
// by a lower bound of the distance from the camera centre to the voxel.  It is
// staged through shared memory in chunks of 64 instances (one per thread:
// unit-cube map, density, pixel-rectangle masks and the feature row, all
// gathered with vector loads); feature rows stay in a ring of chunks so that
// late releases still read shared memory.  For each batch of 32 instances a
// warp transposes the 32x32 bit matrix "instance covers pixel" with shuffles,
// so that every lane walks only the instances whose rectangle contains its
// pixel.  A lane intersects its ray exactly with each such voxel, keeps hits
// in a small register reorder buffer sorted by (t0, t1, voxel id), and
// composites a hit front to back once no later list entry can start before it
// (t0 < lower bound of the next candidate).  A block-wide vote ends the walk
// once every pixel of the tile has stopped (T < tau).
#include "internal.cuh"

namespace art {
namespace {

constexpr int kPend = 12;  // reorder-buffer depth per pixel

// Optional per-pixel record of the composited hits (inspection only).
struct HitLog {
  int32_t* count;
  uint32_t* ids;
  float* t0;
  float* t1;
  int cap;
};

// A pending hit: entry and exit ray parameters and its position in the tile's
// list (which locates the staged density, voxel id and feature row).  Exact
// (t0, t1) ties, which only coincident voxels produce, fall back to list order.
struct Pend {
  float t0, t1;
  uint32_t pos;
};

__device__ __forceinline__ bool pless(const Pend& a, const Pend& b) {
  return a.t0 < b.t0 || (a.t0 == b.t0 && (a.t1 < b.t1 || (a.t1 == b.t1 && a.pos < b.pos)));
}

// feature row loads (vectorised) --------------------------------------------
template <int C>
__device__ __forceinline__ void load_feat(const float* __restrict__ p, float* f) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < C / 4; ++k) {
    float4 x = __ldg(q + k);
    f[4 * k] = x.x;
    f[4 * k + 1] = x.y;
    f[4 * k + 2] = x.z;
    f[4 * k + 3] = x.w;
  }
}

__device__ __forceinline__ void unpack2(uint32_t u, float* f, const __nv_bfloat16*) {
  __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u);
  float2 x = __bfloat1622float2(b);
  f[0] = x.x;
  f[1] = x.y;
}
__device__ __forceinline__ void unpack2(uint32_t u, float* f, const __half*) {
  __half2 b = *reinterpret_cast<__half2*>(&u);
  float2 x = __half22float2(b);
  f[0] = x.x;
  f[1] = x.y;
}

template <int C, typename T16>
__device__ __forceinline__ void load_feat16(const T16* __restrict__ p, float* f) {
  if constexpr (C % 8 == 0) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int k = 0; k < C / 8; ++k) {
      uint4 x = __ldg(q + k);
      unpack2(x.x, f + 8 * k, p);
      unpack2(x.y, f + 8 * k + 2, p);
      unpack2(x.z, f + 8 * k + 4, p);
      unpack2(x.w, f + 8 * k + 6, p);
    }
  } else {
    const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
      uint2 x = __ldg(q + k);
      unpack2(x.x, f + 4 * k, p);
      unpack2(x.y, f + 4 * k + 2, p);
    }
  }
}

template <int C>
__device__ __forceinline__ void load_feat(const __nv_bfloat16* __restrict__ p, float* f) {
  load_feat16<C>(p, f);
}
template <int C>
__device__ __forceinline__ void load_feat(const __half* __restrict__ p, float* f) {
  load_feat16<C>(p, f);
}

// output row stores ----------------------------------------------------------
template <int C>
__device__ __forceinline__ void store_row(float* __restrict__ p, const float* f) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < C / 4; ++k) q[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

template <int C>
__device__ __forceinline__ void store_row(__nv_bfloat16* __restrict__ p, const float* f) {
  uint32_t u[C / 2];
#pragma unroll
  for (int k = 0; k < C / 2; ++k) {
    __nv_bfloat162 b = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    u[k] = *reinterpret_cast<uint32_t*>(&b);
  }
  if constexpr (C % 8 == 0) {
    uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int k = 0; k < C / 8; ++k) q[k] = make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
  } else {
    uint2* q = reinterpret_cast<uint2*>(p);
#pragma unroll
    for (int k = 0; k < C / 4; ++k) q[k] = make_uint2(u[2 * k], u[2 * k + 1]);
  }
}

// Transpose of a 32x32 bit matrix held one row per lane: afterwards lane c
// holds column c (bit r of lane c = bit c of the old row r).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int j = 16 >> i;
    uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m[i]) | ((y >> j) & m[i])) : ((x & m[i]) | ((y << j) & ~m[i]));
  }
  return x;
}

constexpr int TSX = 8, TSY = 4;  // tile: 8 x 4 pixels = one warp
constexpr int NT = 32;           // instances per staged chunk

template <int C, typename TF>
struct Ring {
  // chunks of staged feature rows kept in shared memory (<= 32 KB, <= 16)
  static constexpr int kRaw = 32768 / (NT * C * (int)sizeof(TF));
  static constexpr int kChunks = kRaw < 16 ? kRaw : 16;
};

template <int C, typename TF>
__device__ __forceinline__ void copy_row(const TF* __restrict__ src, TF* dst) {
  constexpr int kVec = (C * (int)sizeof(TF)) % 16 == 0 ? 16 : 8;
  constexpr int kN = C * (int)sizeof(TF) / kVec;
  if constexpr (kVec == 16) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int k = 0; k < kN; ++k) d[k] = __ldg(s + k);
  } else {
    const uint2* s = reinterpret_cast<const uint2*>(src);
    uint2* d = reinterpret_cast<uint2*>(dst);
#pragma unroll
    for (int k = 0; k < kN; ++k) d[k] = __ldg(s + k);
  }
}

template <int C>
__device__ __forceinline__ void row_to_float(const float* p, float* f) {
#pragma unroll
  for (int c = 0; c < C; c += 4) {
    float4 x = *reinterpret_cast<const float4*>(p + c);
    f[c] = x.x;
    f[c + 1] = x.y;
    f[c + 2] = x.z;
    f[c + 3] = x.w;
  }
}
template <int C>
__device__ __forceinline__ void row_to_float(const __nv_bfloat16* p, float* f) {
#pragma unroll
  for (int c = 0; c < C; c += 2) {
    float2 x = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p + c));
    f[c] = x.x;
    f[c + 1] = x.y;
  }
}
template <int C>
__device__ __forceinline__ void row_to_float(const __half* p, float* f) {
#pragma unroll
  for (int c = 0; c < C; c += 2) {
    float2 x = __half22float2(*reinterpret_cast<const __half2*>(p + c));
    f[c] = x.x;
    f[c + 1] = x.y;
  }
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One warp per 8x4 tile, lane = pixel (x = lane & 7, y = lane >> 3).
template <int C, typename TF, typename TO, bool DBG>
__global__ void __launch_bounds__(32) composite_kernel(const uint2* __restrict__ ranges,
                                                       const uint32_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ vals,
                                                       const float4* __restrict__ rec,
                                                       const short4* __restrict__ rect,
                                                       const TF* __restrict__ feat, ViewParams v, float tau,
                                                       TO* __restrict__ Fout, float* __restrict__ Aout,
                                                       unsigned long long* __restrict__ status, HitLog dbg) {
  constexpr int RING = Ring<C, TF>::kChunks;
  __shared__ float4 s_b0[NT], s_b1[NT], s_b2[NT];
  __shared__ float s_thr[NT];
  __shared__ uint32_t s_mask[NT];
  __shared__ float s_sig[RING][NT];
  __shared__ uint32_t s_vid[RING][NT];
  __shared__ __align__(16) TF s_feat[RING][NT][C];

  const int lane = threadIdx.x;
  const int tile = blockIdx.x;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int sx = tx * TSX, sy = ty * TSY;
  const int px = sx + (lane & 7), py = sy + (lane >> 3);
  const bool inside = px < v.W && py < v.H;

  float dcx = ((float)px + 0.5f - v.cx) / v.fx, dcy = ((float)py + 0.5f - v.cy) / v.fy;
  float d0 = v.R[0] * dcx + v.R[3] * dcy + v.R[6];
  float d1 = v.R[1] * dcx + v.R[4] * dcy + v.R[7];
  float d2 = v.R[2] * dcx + v.R[5] * dcy + v.R[8];
  float inrm = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  d0 *= inrm;
  d1 *= inrm;
  d2 *= inrm;

  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.0f;
  float T = 1.0f;
  bool done = !inside;
  Pend buf[kPend];
#pragma unroll
  for (int k = 0; k < kPend; ++k) buf[k] = Pend{0.f, 0.f, 0u};
  int nb = 0;
  uint32_t n_over = 0;
  const uint32_t qmask = (1u << v.depth_bits) - 1u;
  const float qinv = 1.0f / v.dscale;
  const size_t pix = (size_t)py * v.W + px;
  int n_used = 0;
  int cur_chunk = 0;
  const uint2 rg = ranges[tile];

  auto release_front = [&]() {
    Pend h = buf[0];
#pragma unroll
    for (int k = 0; k < kPend - 1; ++k) buf[k] = buf[k + 1];
    --nb;
    const int ch = (int)(h.pos / NT), sl = (int)(h.pos % NT);
    float f[C];
    float sig;
    uint32_t vid;
    if (cur_chunk - ch < RING) {
      sig = s_sig[ch % RING][sl];
      vid = s_vid[ch % RING][sl];
      row_to_float<C>(&s_feat[ch % RING][sl][0], f);
    } else {  // staged long ago: read the voxel again
      vid = vals[rg.x + h.pos];
      sig = rec[4 * (size_t)vid + 3].x;
      load_feat<C>(feat + (size_t)vid * C, f);
    }
    if constexpr (DBG) {
      if (n_used < dbg.cap) {
        dbg.ids[pix * dbg.cap + n_used] = vid;
        dbg.t0[pix * dbg.cap + n_used] = h.t0;
        dbg.t1[pix * dbg.cap + n_used] = h.t1;
      }
      ++n_used;
    }
    float e = expf(-sig * (h.t1 - h.t0));
    float w = T * (1.0f - e);
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = fmaf(w, f[c], acc[c]);
    T *= e;
    if (T < tau) done = true;
  };

  for (uint32_t base = rg.x; base < rg.y; base += NT) {
    cur_chunk = (int)((base - rg.x) / NT);
    const int slot = cur_chunk % RING;
    __syncwarp();
    {  // stage one instance per lane
      const uint32_t k = base + lane;
      uint32_t m = 0;
      float thr = 3.4e38f;
      if (k < rg.y) {
        const uint32_t vid = vals[k];
        const uint32_t key = keys[k];
        const float4* rp = rec + 4 * (size_t)vid;
        const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2], r3 = rp[3];
        const short4 rc = rect[vid];
        copy_row<C, TF>(feat + (size_t)vid * C, &s_feat[slot][lane][0]);
        const float ex = v.o[0] - r0.w, ey = v.o[1] - r1.w, ez = v.o[2] - r2.w;
        s_b0[lane] = make_float4(r0.x, r0.y, r0.z, r0.x * ex + r0.y * ey + r0.z * ez);
        s_b1[lane] = make_float4(r1.x, r1.y, r1.z, r1.x * ex + r1.y * ey + r1.z * ez);
        s_b2[lane] = make_float4(r2.x, r2.y, r2.z, r2.x * ex + r2.y * ey + r2.z * ez);
        s_sig[slot][lane] = r3.x;
        s_vid[slot][lane] = vid;
        thr = v.znear + (float)(key & qmask) * qinv;
        const int lx0 = max((int)rc.x - sx, 0), lx1 = min((int)rc.z - sx, TSX - 1);
        const int ly0 = max((int)rc.y - sy, 0), ly1 = min((int)rc.w - sy, TSY - 1);
        if (lx0 <= lx1 && ly0 <= ly1) {
          const uint32_t cm = ((2u << lx1) - 1u) & ~((1u << lx0) - 1u);
          const uint32_t rows = ((2u << ly1) - 1u) & ~((1u << ly0) - 1u);
          // spread row bits r to byte positions 8r, then replicate the column mask
          const uint32_t spread = (rows & 1u) | ((rows & 2u) << 7) | ((rows & 4u) << 14) | ((rows & 8u) << 21);
          m = cm * spread;
        }
      }
      s_mask[lane] = m;
      s_thr[lane] = thr;
    }
    __syncwarp();
    // every instance of this chunk and later enters at t >= the first threshold
    const float thr0 = s_thr[0];
    while (!done && nb > 0 && buf[0].t0 < thr0) release_front();
    uint32_t cand = transpose32(s_mask[lane], lane);
    if (done) cand = 0;
    while (cand) {
      const int idx = __ffs(cand) - 1;
      cand &= cand - 1;
      const float4 b0 = s_b0[idx], b1 = s_b1[idx], b2 = s_b2[idx];
      // ray in the voxel's unit-cube frame: o' = b.w, d' = B d
      const float e0 = b0.x * d0 + b0.y * d1 + b0.z * d2;
      const float e1 = b1.x * d0 + b1.y * d1 + b1.z * d2;
      const float e2 = b2.x * d0 + b2.y * d1 + b2.z * d2;
      const float i0 = rcp_approx(e0), i1 = rcp_approx(e1), i2 = rcp_approx(e2);
      const float a0 = (-0.5f - b0.w) * i0, c0 = (0.5f - b0.w) * i0;
      const float a1 = (-0.5f - b1.w) * i1, c1 = (0.5f - b1.w) * i1;
      const float a2 = (-0.5f - b2.w) * i2, c2 = (0.5f - b2.w) * i2;
      const float t0 = fmaxf(fmaxf(v.znear, fminf(a0, c0)), fmaxf(fminf(a1, c1), fminf(a2, c2)));
      const float t1 = fminf(fminf(v.zfar, fmaxf(a0, c0)), fminf(fmaxf(a1, c1), fmaxf(a2, c2)));
      if (!(t1 > t0)) continue;
      const Pend p{t0, t1, base - rg.x + (uint32_t)idx};
      if (nb == kPend) {
        // buffer full: release what this candidate's own bound allows (still
        // exact), and only if nothing can go, the earliest hit (counted)
        const float thr = s_thr[idx];
        while (!done && nb > 0 && buf[0].t0 < thr) release_front();
        if (!done && nb == kPend) {
          ++n_over;
          release_front();
        }
        if (done) {
          cand = 0;
          break;
        }
      }
#pragma unroll
      for (int q = 0; q < kPend; ++q)
        if (q == nb) buf[q] = p;
#pragma unroll
      for (int q = kPend - 1; q >= 1; --q) {
        if (q <= nb && pless(buf[q], buf[q - 1])) {
          const Pend tmp = buf[q];
          buf[q] = buf[q - 1];
          buf[q - 1] = tmp;
        }
      }
      ++nb;
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  while (nb > 0 && !done) release_front();

  if (inside) {
    if constexpr (DBG) dbg.count[pix] = n_used;
    store_row<C>(Fout + pix * C, acc);
    if (Aout) Aout[pix] = 1.0f - T;
  }
  if (n_over) atomicAdd(status + kStOverflowOrder, (unsigned long long)n_over);
}

template <int C, typename TF, typename TO>
void launch_c(art_ctx* ctx, const ViewParams& v, void* F, float* A, const HitLog* dbg) {
  int ntiles = v.tiles_x * v.tiles_y;
  if (dbg) {
    auto kfn = composite_kernel<C, TF, TO, true>;
    ART_LAUNCH(ctx, "composite_debug", kfn, ntiles, 32, 0, ctx->d_ranges, ctx->d_keys[0], ctx->d_vals[0], ctx->d_rec,
               ctx->d_rect, (const TF*)ctx->d_feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, *dbg);
  } else {
    auto kfn = composite_kernel<C, TF, TO, false>;
    ART_LAUNCH(ctx, "composite", kfn, ntiles, 32, 0, ctx->d_ranges, ctx->d_keys[0], ctx->d_vals[0], ctx->d_rec,
               ctx->d_rect, (const TF*)ctx->d_feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, HitLog{});
  }
}

template <int C>
art_status dispatch_dtypes(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A, const HitLog* dbg) {
  int fd = ctx->feat_dtype;
  if (F_dtype == ART_F32) {
    if (fd == ART_F32) launch_c<C, float, float>(ctx, v, F, A, dbg);
    else if (fd == ART_BF16) launch_c<C, __nv_bfloat16, float>(ctx, v, F, A, dbg);
    else launch_c<C, __half, float>(ctx, v, F, A, dbg);
  } else {
    if (dbg) return fail(ctx, ART_ERR_INVALID_ARG, "hit logging writes FP32 feature maps");
    if (fd == ART_F32) launch_c<C, float, __nv_bfloat16>(ctx, v, F, A, nullptr);
    else if (fd == ART_BF16) launch_c<C, __nv_bfloat16, __nv_bfloat16>(ctx, v, F, A, nullptr);
    else launch_c<C, __half, __nv_bfloat16>(ctx, v, F, A, nullptr);
  }
  return ART_OK;
}

}  // namespace

art_status launch_composite(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A, const void* dbg_log) {
  const HitLog* dbg = (const HitLog*)dbg_log;
  if (v.tile_w != TSX || v.tile_h != TSY) return fail(ctx, ART_ERR_UNSUPPORTED, "composite: tiles must be 8x4");
  switch (ctx->C) {
    case 4: return dispatch_dtypes<4>(ctx, v, F, F_dtype, A, dbg);
    case 8: return dispatch_dtypes<8>(ctx, v, F, F_dtype, A, dbg);
    case 16: return dispatch_dtypes<16>(ctx, v, F, F_dtype, A, dbg);
    case 32: return dispatch_dtypes<32>(ctx, v, F, F_dtype, A, dbg);
    default: return fail(ctx, ART_ERR_UNSUPPORTED, "composite: C=%d not built (4, 8, 16, 32)", ctx->C);
  }
}

// Hit log layout shared with api.cu.
void* make_hit_log(int32_t* count, uint32_t* ids, float* t0, float* t1, int cap) {
  HitLog* h = new HitLog{count, ids, t0, t1, cap};
  return h;
}
void free_hit_log(void* p) { delete (HitLog*)p; }

}  // namespace art
