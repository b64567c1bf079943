// Device helpers shared by the forward composite (composite.cu) and its
// backward (backward.cu): per-pixel reorder buffer, warp bit-matrix
// transpose, staged feature ring, vectorised feature loads and the exact
// ray / warped-voxel slab test.  Both kernels walk a tile's instances with
// the same code so that they see the same hits in the same order.
#pragma once

#include "internal.cuh"

namespace art {

constexpr int kPend = 16;  // reorder-buffer depth per pixel
static_assert((kPend & (kPend - 1)) == 0, "the composite keeps its pending hits in a power-of-two ring");

// Optional per-pixel record of the composited hits (inspection only).
struct HitLog {
  int32_t* count;
  uint32_t* ids;
  float* t0;
  float* t1;
  int cap;
};

// A pending hit: entry distance t0, chord length dl (the exit is t0 + dl)
// and its position in the tile's list (which locates the staged density,
// voxel id and feature row).  Ordered by (t0, exit, position): at equal t0 the
// exit order is the chord order.  Exact ties, which only coincident voxels
// produce, fall back to list order.
struct Pend {
  float t0, dl;
  uint32_t pos;
};

__device__ __forceinline__ bool pless(const Pend& a, const Pend& b) {
  return a.t0 < b.t0 || (a.t0 == b.t0 && (a.dl < b.dl || (a.dl == b.dl && a.pos < b.pos)));
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

// Resident one-warp blocks of the composite walk per SM (its register cap is
// 64K / (32 x this)) and the shared memory of each block's feature ring.
constexpr int kCompositeWarps = 12;
constexpr int kRingBytes = 10240;

template <int C, typename TF>
struct Ring {
  // chunks of staged feature rows kept in shared memory (<= kRingBytes, 1 ..
  // 16): small enough for many resident one-warp blocks; a hit released
  // after its chunk left the ring reads its voxel again from global memory
  static constexpr int kRaw = kRingBytes / (NT * C * (int)sizeof(TF));
  static constexpr int kChunks = kRaw < 1 ? 1 : (kRaw < 16 ? kRaw : 16);
};

// Asynchronous global -> shared copies (cp.async): issued, grouped per
// commit, and waited for by group; a thread sees its own copies after the
// wait, the other lanes after a __syncwarp that follows it.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A feature row into shared memory, asynchronously.
template <int C, typename TF>
__device__ __forceinline__ void copy_row_async(const TF* __restrict__ src, TF* dst) {
  constexpr int kBytes = C * (int)sizeof(TF);
  if constexpr (kBytes % 16 == 0) {
#pragma unroll
    for (int k = 0; k < kBytes / 16; ++k)
      cp_async16(reinterpret_cast<uint8_t*>(dst) + 16 * k, reinterpret_cast<const uint8_t*>(src) + 16 * k);
  } else {
#pragma unroll
    for (int k = 0; k < kBytes / 8; ++k)
      cp_async8(reinterpret_cast<uint8_t*>(dst) + 8 * k, reinterpret_cast<const uint8_t*>(src) + 8 * k);
  }
}

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


// Error-free FP32 transformations (exact results as unevaluated sums).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// (h, l) + (bh, bl) as a double-float (error ~2^-44 relative)
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// The pixel ray's direction D, not normalised, held to ~44 bits as the sum
// of two FP32 vectors (hi + lo), and 1 / |D|.  The hit test works at metre
// scale 2 m from the voxels; there a plain FP32 direction (~1e-7 relative
// error) moves the ray by ~3e-7 m sideways, which misplaces the chord of a
// ray that meets a face at a shallow angle by micrometres.  The ray through
// the pixel centre (Sec. 3.1's camera rays) is R^T ((x + 1/2 - cx) / fx,
// (y + 1/2 - cy) / fy, 1); scaled by fx fy > 0 (the same ray) it needs no
// division: D = R^T ((x + 1/2 - cx) fy, (y + 1/2 - cy) fx, fx fy), formed
// with two-sums and two-products, FP32 only.  |D| enters as a scale of every
// ray parameter of the pixel (FP32, ~1e-7 relative).
struct RayDir {
  float h[3], l[3];
  float inv_n;  // 1 / |D|
};

__device__ __forceinline__ RayDir pixel_ray(const ViewParams& v, int px, int py) {
  float ux, uxl, uy, uyl;  // pixel centre minus principal point, exactly
  two_sum((float)px + 0.5f, -v.cx, ux, uxl);
  two_sum((float)py + 0.5f, -v.cy, uy, uyl);
  float c0, c0l, c1, c1l, c2, c2l;  // the camera-frame direction scaled by fx fy
  two_prod(ux, v.fy, c0, c0l);
  c0l = __fmaf_rn(uxl, v.fy, c0l);
  two_prod(uy, v.fx, c1, c1l);
  c1l = __fmaf_rn(uyl, v.fx, c1l);
  two_prod(v.fx, v.fy, c2, c2l);
  RayDir r;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float h, l, th, tl;
    two_prod(v.R[a], c0, h, l);
    l = __fmaf_rn(v.R[a], c0l, l);
    two_prod(v.R[3 + a], c1, th, tl);
    df_add(h, l, th, __fmaf_rn(v.R[3 + a], c1l, tl));
    two_prod(v.R[6 + a], c2, th, tl);
    df_add(h, l, th, __fmaf_rn(v.R[6 + a], c2l, tl));
    r.h[a] = h;
    r.l[a] = l;
  }
  r.inv_n = rsqrtf(r.h[0] * r.h[0] + r.h[1] * r.h[1] + r.h[2] * r.h[2]);
  return r;
}

// Staged form of a voxel record for the hit test: rows of its unit-cube map
// A_lin^-1 / h in b0..b2 (.xyz) with x = o - cw, the camera centre relative to
// the warped centre, split into hi (b0..b2 .w) and lo (xl.xyz) parts: the hi
// part is the FP32 difference, the lo part its exact rounding error (two-sum)
// plus the low part of the camera centre.
__device__ __forceinline__ void stage_voxel(const float4& r0, const float4& r1, const float4& r2, const ViewParams& v,
                                            float4& b0, float4& b1, float4& b2, float4& xl) {
  const float cw[3] = {r0.w, r1.w, r2.w};
  float xh[3], xo[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = v.o[a], q = -cw[a];
    const float s = __fadd_rn(p, q);
    const float qq = __fsub_rn(s, p);
    const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, qq)), __fsub_rn(q, qq));
    xh[a] = s;
    xo[a] = __fadd_rn(err, v.o_lo[a]);
  }
  b0 = make_float4(r0.x, r0.y, r0.z, xh[0]);
  b1 = make_float4(r1.x, r1.y, r1.z, xh[1]);
  b2 = make_float4(r2.x, r2.y, r2.z, xh[2]);
  xl = make_float4(xo[0], xo[1], xo[2], 0.0f);
}

// Exact hit of the pixel ray P(lambda) = o + lambda D with a staged voxel
// (stage_voxel), anchored at the voxel: s = <cw - o, D> / |D|^2 is the ray
// parameter of the point nearest the warped centre and q = (o - cw) + s D
// that point relative to the centre (millimetres, formed with one rounding
// from the split parts, so ~1e-10 m); u = local ray parameters of the entry /
// exit planes of the unit cube, from A_lin^-1 q / h and the direction
// A_lin^-1 D / h.  The chord delta (Eq. 5's distance travelled through the
// voxel) is |D| times the difference of the small local parameters; the
// entry distance t0 = |D| (s + u_entry) (for ordering).  Both are clipped to
// [near, far] (distances along the unit ray).  ax0 / ax1 are the axes of
// the entry / exit planes (-1 when the near / far bound is the active one)
// and e the unit ray direction in unit-cube coordinates.  Returns
// delta > 0.
__device__ __forceinline__ bool slab_hit(const float4& b0, const float4& b1, const float4& b2, const float4& xl,
                                         const RayDir& d, float znear, float zfar, float& t0, float& delta, int& ax0,
                                         int& ax1, float (&e)[3]) {
  const float n = 1.0f / d.inv_n;
  const float s = -(b0.w * d.h[0] + b1.w * d.h[1] + b2.w * d.h[2]) * (d.inv_n * d.inv_n);
  const float q0 = fmaf(s, d.h[0], b0.w) + fmaf(s, d.l[0], xl.x);
  const float q1 = fmaf(s, d.h[1], b1.w) + fmaf(s, d.l[1], xl.y);
  const float q2 = fmaf(s, d.h[2], b2.w) + fmaf(s, d.l[2], xl.z);
  const float p0 = b0.x * q0 + b0.y * q1 + b0.z * q2;
  const float p1 = b1.x * q0 + b1.y * q1 + b1.z * q2;
  const float p2 = b2.x * q0 + b2.y * q1 + b2.z * q2;
  e[0] = b0.x * d.h[0] + b0.y * d.h[1] + b0.z * d.h[2];
  e[1] = b1.x * d.h[0] + b1.y * d.h[1] + b1.z * d.h[2];
  e[2] = b2.x * d.h[0] + b2.y * d.h[1] + b2.z * d.h[2];
  const float i0 = rcp_approx(e[0]), i1 = rcp_approx(e[1]), i2 = rcp_approx(e[2]);
  const float a0 = (-0.5f - p0) * i0, c0 = (0.5f - p0) * i0;
  const float a1 = (-0.5f - p1) * i1, c1 = (0.5f - p1) * i1;
  const float a2 = (-0.5f - p2) * i2, c2 = (0.5f - p2) * i2;
  const float l0 = fminf(a0, c0), l1 = fminf(a1, c1), l2 = fminf(a2, c2);
  const float h0 = fmaxf(a0, c0), h1 = fmaxf(a1, c1), h2 = fmaxf(a2, c2);
  const float ul = fmaxf(fmaxf(znear * d.inv_n - s, l0), fmaxf(l1, l2));
  const float uh = fminf(fminf(zfar * d.inv_n - s, h0), fminf(h1, h2));
  ax0 = ul == l0 ? 0 : (ul == l1 ? 1 : (ul == l2 ? 2 : -1));
  ax1 = uh == h0 ? 0 : (uh == h1 ? 1 : (uh == h2 ? 2 : -1));
  e[0] *= d.inv_n;
  e[1] *= d.inv_n;
  e[2] *= d.inv_n;
  t0 = (s + ul) * n;
  delta = (uh - ul) * n;
  return uh > ul;
}

// Pixel-rectangle mask of one instance over a TSX x TSY tile at (sx, sy):
// bit (y * 8 + x) set when pixel (sx + x, sy + y) lies in the rectangle.
__device__ __forceinline__ uint32_t rect_mask(short4 rc, int sx, int sy) {
  const int lx0 = max((int)rc.x - sx, 0), lx1 = min((int)rc.z - sx, TSX - 1);
  const int ly0 = max((int)rc.y - sy, 0), ly1 = min((int)rc.w - sy, TSY - 1);
  if (lx0 > lx1 || ly0 > ly1) return 0u;
  const uint32_t cm = ((2u << lx1) - 1u) & ~((1u << lx0) - 1u);
  const uint32_t rows = ((2u << ly1) - 1u) & ~((1u << ly0) - 1u);
  // spread row bits r to byte positions 8r, then replicate the column mask
  const uint32_t spread = (rows & 1u) | ((rows & 2u) << 7) | ((rows & 4u) << 14) | ((rows & 8u) << 21);
  return cm * spread;
}

// Unit-length ray direction through the centre of pixel (px, py).
__device__ __forceinline__ void pixel_dir(const ViewParams& v, int px, int py, float& d0, float& d1, float& d2) {
  const float dcx = ((float)px + 0.5f - v.cx) / v.fx, dcy = ((float)py + 0.5f - v.cy) / v.fy;
  d0 = v.R[0] * dcx + v.R[3] * dcy + v.R[6];
  d1 = v.R[1] * dcx + v.R[4] * dcy + v.R[7];
  d2 = v.R[2] * dcx + v.R[5] * dcy + v.R[8];
  const float inrm = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  d0 *= inrm;
  d1 *= inrm;
  d2 *= inrm;
}


// ------------------------------------------------------------ split walk

// The part of a tile's list one warp walks: list positions [begin, end),
// hits whose entry t0 lies in [t0_lo, t0_hi); with part set, the walk stores
// its partial feature sum and transmittance there instead of the outputs.
struct Seg {
  uint32_t begin, end;
  float t0_lo, t0_hi;
  float* part;  // [C + 1][32]: partial F (per channel), then T
};

constexpr int kMaxSegs = 255;

// Per tile: number of segments and the index of its first one; the segments
// of all tiles in one list, the tiles with two or more in another.
// With tiles_in set, only the tiles listed there (count in status[in_word]).
static __global__ void seg_plan_kernel(int ntiles, const uint2* __restrict__ ranges, int seg_len, uint2* __restrict__ seg,
                                uint32_t* __restrict__ items, uint32_t* __restrict__ multi,
                                unsigned long long* __restrict__ status, const uint32_t* __restrict__ tiles_in,
                                int in_word) {
  ART_PDL_ENTRY();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int t = i;
  if (tiles_in) {
    if ((unsigned long long)i >= status[in_word]) return;
    t = (int)tiles_in[i];
  }
  if (t >= ntiles) return;
  const uint2 rg = ranges[t];
  const uint32_t len = rg.y - rg.x;
  uint32_t S = len == 0 ? 0u : (len + seg_len - 1) / seg_len;
  if (S > kMaxSegs) S = kMaxSegs;
  uint32_t base = 0;
  if (S) {
    base = (uint32_t)atomicAdd(status + kStItems, (unsigned long long)S);
    for (uint32_t k = 0; k < S; ++k) items[base + k] = (uint32_t)t;
    if (S > 1) multi[atomicAdd(status + kStMulti, 1ull)] = (uint32_t)t;
  }
  seg[t] = make_uint2(base, S);
}

// First position in [a, b) whose depth quantum is >= qt (b if none): keys are
// sorted within the tile.  Warp-cooperative: 32 probes per round.
__device__ __forceinline__ uint32_t lower_bound_q(const uint32_t* __restrict__ keys, uint32_t a, uint32_t b,
                                                  uint32_t qmask, uint32_t qt, int lane) {
  while (b - a > 31u) {
    const uint32_t step = (b - a + 31u) / 32u;
    const uint32_t idx = a + (uint32_t)lane * step;
    const bool ge = idx >= b || (keys[idx] & qmask) >= qt;
    const uint32_t m = __ballot_sync(0xffffffffu, ge);
    if (m & 1u) return a;
    const uint32_t f = m ? (uint32_t)(__ffs(m) - 1) : 32u;
    const uint32_t na = a + (f - 1u) * step + 1u;
    const uint32_t nb = f < 32u ? min(b, a + f * step) : b;
    a = na;
    b = nb;
  }
  const uint32_t idx = a + (uint32_t)lane;
  const bool ge = idx >= b || (keys[idx] & qmask) >= qt;
  const uint32_t m = __ballot_sync(0xffffffffu, ge);
  return a + (uint32_t)(__ffs(m) - 1);  // lane b - a (<= 31) is always set
}

// Window of a segment's scan before its first depth bound, in depth quanta:
// 2 r_max + 3 quanta (+ FP32 slack); r_max of the pose is status[kStRmax].
__device__ __forceinline__ uint32_t seg_window(const ViewParams& v, const unsigned long long* status) {
  const float rmax = __uint_as_float((uint32_t)status[kStRmax]);
  return (uint32_t)ceilf((2.0f * rmax + 1e-5f) * v.dscale) + 3u;
}

// Segment k = i - first of a tile with S segments: list positions
// p_k = start + k len / S; it composites the hits with entry t0 in
// [D_k, D_{k+1}) (D_k the depth bound at p_k) and walks from the first entry
// whose bound lies within the window before D_k up to p_{k+1}.
__device__ __forceinline__ Seg make_seg(const ViewParams& v, uint2 rg, uint2 sgt, uint32_t i,
                                        const uint32_t* __restrict__ keys, uint32_t wq, int lane) {
  const uint32_t qmask = (1u << v.depth_bits) - 1u;
  const float qinv = 1.0f / v.dscale;
  const uint32_t k = i - sgt.x, S = sgt.y;
  const uint32_t len = rg.y - rg.x;
  const uint32_t pk = rg.x + (uint32_t)(((unsigned long long)k * len) / S);
  const uint32_t pk1 = rg.x + (uint32_t)(((unsigned long long)(k + 1) * len) / S);
  Seg sg;
  sg.end = pk1;
  if (k == 0) {
    sg.begin = rg.x;
    sg.t0_lo = -3.4e38f;
  } else {
    const uint32_t qk = keys[pk] & qmask;
    sg.t0_lo = v.znear + (float)qk * qinv;
    sg.begin = lower_bound_q(keys, rg.x, pk, qmask, qk > wq ? qk - wq : 0u, lane);
  }
  sg.t0_hi = k + 1 < S ? v.znear + (float)(keys[pk1] & qmask) * qinv : 3.4e38f;
  sg.part = nullptr;
  return sg;
}

}  // namespace art
