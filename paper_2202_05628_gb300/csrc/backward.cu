// Backward of the dynamic volume rendering (arXiv 2202.05628, Eq. 5-6) and
// of the LBS warp (Eq. 4) with respect to the voxel features, densities and
// skinning weights: the gradients the paper's end-to-end optimisation of the
// feature table needs (Sec. 3.1 "Training").
//
// Per-ray recomputation instead of stored sample lists: the backward walks
// each tile's instance list with exactly the forward's code (staging, masks,
// slab test, reorder buffer, release rule, early stop), so every pixel
// revisits the same hits in the same order.  Long lists are split into the
// forward's depth segments, walked by separate warps: a first pass gives each
// segment's own transmittance product and sum of w <f, g>, a prefix over the
// segments the values each is entered with, and the gradient pass walks every
// segment from those (exact stop rule: the true transmittance is carried).  With w_i = T_i a_i,
// a_i = 1 - exp(-sigma_i delta_i), T_{i+1} = T_i (1 - a_i), g = dL/dF and
// g_A = dL/dA at the pixel:
//   dL/df_i      += w_i g
//   dL/d(s_i)     = T_{i+1} <f_i, g> - <F - P_i, g> + T_final g_A,
//                   s_i = sigma_i delta_i, P_i = sum_{k<=i} w_k f_k
//   dL/dsigma_i  += delta_i dL/d(s_i);  dL/ddelta_i = sigma_i dL/d(s_i)
// and delta_i = t1 - t0 where each clipped-by-a-face end t of the chord
// solves row_a(N) [o + t d; 1] = const for N = A_i^-1, so
//   dt/dN[a][0..2] = -(o + t d) / d'_a,  dt/dN[a][3] = -1 / d'_a,
// d'_a = row_a(N_lin) d.  The per-voxel dL/dN is then mapped to dL/dA by
// dA = -N^T dN N^T (4x4 affine forms) and to dL/dw_k = <dL/dA, G_{j_k}>.
// The hit set, the order and the stop index are held fixed (piecewise
// differentiation, as for any ray-marched renderer).
#include "raster.cuh"

namespace art {
namespace {

// Pending hit of the backward: the forward's fields plus what the geometric
// gradient needs (entry / exit axes and the direction component along them).
struct PendG {
  float t0, dl;  // entry distance and chord (the exit is t0 + dl)
  uint32_t pos;
  int axes;  // (ax0 + 1) | (ax1 + 1) << 4
  float e0, e1;
};

__device__ __forceinline__ bool pless(const PendG& a, const PendG& b) {
  return a.t0 < b.t0 || (a.t0 == b.t0 && (a.dl < b.dl || (a.dl == b.dl && a.pos < b.pos)));
}

__device__ __forceinline__ void atomic_add4(float* p, float a, float b, float c, float d) {
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
}

// One segment of a tile's list (the forward's split walk: Seg, make_seg),
// entered with the pixel's transmittance T_in and <P, g>_in of everything
// composited before it.  PASS 0 walks the segment from T = 1, <P, g> = 0 and
// stores its own product of (1 - a) and sum of w <f, g> ([2][32] at out);
// PASS 1 walks it with the true incoming values and accumulates the
// gradients.  One segment per tile is the sequential walk.
template <int C, typename TF, int PASS>
__device__ __forceinline__ void bwd_tile(const int tile, const Seg& sg, float T_in, float pg_in, float* out,
                                         const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                         const float4* __restrict__ rec, const short4* __restrict__ rect,
                                         const TF* __restrict__ feat, const ViewParams& v, float tau, float h,
                                         const float* __restrict__ Ffwd, const float* __restrict__ Afwd,
                                         const float* __restrict__ dF, const float* __restrict__ dA,
                                         float* __restrict__ gfeat, float* __restrict__ gsig, float* __restrict__ gN,
                                         unsigned long long* __restrict__ status) {
  constexpr int RING = Ring<C, TF>::kChunks;
  __shared__ float4 s_b0[NT], s_b1[NT], s_b2[NT], s_xl[NT];
  __shared__ float s_thr[NT];
  __shared__ uint32_t s_mask[NT];
  __shared__ float s_sig[RING][NT];
  __shared__ uint32_t s_vid[RING][NT];
  __shared__ __align__(16) TF s_feat[RING][NT][C];

  const int lane = threadIdx.x & 31;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int sx = tx * TSX, sy = ty * TSY;
  const int px = sx + (lane & 7), py = sy + (lane >> 3);
  const bool inside = px < v.W && py < v.H;
  const size_t pix = inside ? (size_t)py * v.W + px : 0;

  const RayDir rd = pixel_ray(v, px, py);
  const float d0 = rd.h[0] * rd.inv_n, d1 = rd.h[1] * rd.inv_n, d2 = rd.h[2] * rd.inv_n;  // unit direction

  // upstream gradient of this pixel and the forward's outputs
  float g[C];
  float Fg = 0.0f, ga = 0.0f, Tfin = 1.0f;
  bool any = false;
#pragma unroll
  for (int c = 0; c < C; c += 4) {
    float4 gv = inside ? *reinterpret_cast<const float4*>(dF + pix * C + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 fv = inside ? *reinterpret_cast<const float4*>(Ffwd + pix * C + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    g[c] = gv.x;
    g[c + 1] = gv.y;
    g[c + 2] = gv.z;
    g[c + 3] = gv.w;
    Fg += fv.x * gv.x + fv.y * gv.y + fv.z * gv.z + fv.w * gv.w;
    any = any || gv.x != 0.f || gv.y != 0.f || gv.z != 0.f || gv.w != 0.f;
  }
  if (inside) {
    ga = dA ? dA[pix] : 0.0f;
    Tfin = 1.0f - Afwd[pix];
  }
  any = any || ga != 0.0f;

  float T = T_in, pg = pg_in;  // transmittance before the next hit; <P_i, g>
  bool done = !(inside && any) || T < tau;
  PendG buf[kPend];
#pragma unroll
  for (int k = 0; k < kPend; ++k) buf[k] = PendG{0.f, 0.f, 0u, 0, 0.f, 0.f};
  int nb = 0;
  uint32_t n_over = 0;
  const uint32_t qmask = (1u << v.depth_bits) - 1u;
  const float qinv = 1.0f / v.dscale;
  int cur_chunk = 0;
  const uint2 rg = make_uint2(sg.begin, sg.end);

  auto release_front = [&]() {
    const PendG hh = buf[0];
#pragma unroll
    for (int k = 0; k < kPend - 1; ++k) buf[k] = buf[k + 1];
    --nb;
    const int ch = (int)(hh.pos / NT), sl = (int)(hh.pos % NT);
    float f[C];
    float sig;
    uint32_t vid;
    if (cur_chunk - ch < RING) {
      sig = s_sig[ch % RING][sl];
      vid = s_vid[ch % RING][sl];
      row_to_float<C>(&s_feat[ch % RING][sl][0], f);
    } else {
      vid = vals[rg.x + hh.pos];
      sig = rec[4 * (size_t)vid + 3].x;
      load_feat<C>(feat + (size_t)vid * C, f);
    }
    const float delta = hh.dl;
    const float t1 = hh.t0 + hh.dl;
    const float e = expf(-sig * delta);
    const float w = T * (1.0f - e);
    float fg = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) fg = fmaf(f[c], g[c], fg);
    pg = fmaf(w, fg, pg);
    if constexpr (PASS == 0) {  // the segment's own product and sum only
      T *= e;
      if (T < tau) done = true;
      return;
    }
    const float core = T * e * fg - (Fg - pg) + Tfin * ga;
#pragma unroll
    for (int c = 0; c < C; c += 4)
      atomic_add4(gfeat + (size_t)vid * C + c, w * g[c], w * g[c + 1], w * g[c + 2], w * g[c + 3]);
    atomicAdd(gsig + vid, delta * core);
    const float gdelta = sig * core;
    const int a0 = (hh.axes & 15) - 1, a1 = (hh.axes >> 4) - 1;
    if (a0 >= 0) {  // entry end: d(delta)/d(t0) = -1
      const float gt = -gdelta / (h * hh.e0);
      atomic_add4(gN + (size_t)vid * 12 + 4 * a0, -gt * (v.o[0] + hh.t0 * d0), -gt * (v.o[1] + hh.t0 * d1),
                  -gt * (v.o[2] + hh.t0 * d2), -gt);
    }
    if (a1 >= 0) {  // exit end: d(delta)/d(t1) = +1
      const float gt = gdelta / (h * hh.e1);
      atomic_add4(gN + (size_t)vid * 12 + 4 * a1, -gt * (v.o[0] + t1 * d0), -gt * (v.o[1] + t1 * d1),
                  -gt * (v.o[2] + t1 * d2), -gt);
    }
    T *= e;
    if (T < tau) done = true;
  };

  for (uint32_t base = rg.x; base < rg.y; base += NT) {
    cur_chunk = (int)((base - rg.x) / NT);
    const int slot = cur_chunk % RING;
    __syncwarp();
    {
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
        stage_voxel(r0, r1, r2, v, s_b0[lane], s_b1[lane], s_b2[lane], s_xl[lane]);
        s_sig[slot][lane] = r3.x;
        s_vid[slot][lane] = vid;
        thr = v.znear + (float)(key & qmask) * qinv;
        m = rect_mask(rc, sx, sy);
      }
      s_mask[lane] = m;
      s_thr[lane] = thr;
    }
    __syncwarp();
    const float thr0 = s_thr[0];
    while (!done && nb > 0 && buf[0].t0 < thr0) release_front();
    uint32_t cand = transpose32(s_mask[lane], lane);
    if (done) cand = 0;
    while (cand) {
      const int idx = __ffs(cand) - 1;
      cand &= cand - 1;
      float t0, dl, e[3];
      int ax0, ax1;
      if (!slab_hit(s_b0[idx], s_b1[idx], s_b2[idx], s_xl[idx], rd, v.znear, v.zfar, t0, dl, ax0, ax1, e)) continue;
      if (t0 < sg.t0_lo || t0 >= sg.t0_hi) continue;  // another segment's hit
      const PendG p{t0, dl, base - rg.x + (uint32_t)idx, (ax0 + 1) | ((ax1 + 1) << 4),
                    ax0 == 0 ? e[0] : (ax0 == 1 ? e[1] : e[2]), ax1 == 0 ? e[0] : (ax1 == 1 ? e[1] : e[2])};
      if (nb == kPend) {
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
          const PendG tmp = buf[q];
          buf[q] = buf[q - 1];
          buf[q - 1] = tmp;
        }
      }
      ++nb;
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  while (nb > 0 && !done) release_front();
  if constexpr (PASS == 0) {
    out[lane] = T;
    out[32 + lane] = pg;
  }
  if (n_over) atomicAdd(status + kStOverflowOrder, (unsigned long long)n_over);
}

// The segments of every tile, pulled by persistent one-warp blocks.  PASS 0
// runs only the segments of split tiles; PASS 1 every segment.
template <int C, typename TF, int PASS>
__global__ void __launch_bounds__(32) bwd_split_kernel(
    const uint2* __restrict__ ranges, const uint2* __restrict__ seg, const uint32_t* __restrict__ items,
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
    const short4* __restrict__ rect, const TF* __restrict__ feat, ViewParams v, float tau, float h,
    const float* __restrict__ Ffwd, const float* __restrict__ Afwd, const float* __restrict__ dF,
    const float* __restrict__ dA, float* __restrict__ gfeat, float* __restrict__ gsig, float* __restrict__ gN,
    unsigned long long* __restrict__ status, float* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const unsigned long long n_items = status[kStItems];
  const uint32_t wq = seg_window(v, status);
  for (;;) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(status + kStNext, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= n_items) break;
    const int tile = (int)items[i];
    const uint2 sgt = seg[tile];
    if (PASS == 0 && sgt.y < 2) continue;
    const Seg sg = make_seg(v, ranges[tile], sgt, (uint32_t)i, keys, wq, lane);
    float* pp = part + (size_t)i * 64;
    const float T_in = (PASS == 1 && sgt.y > 1) ? pp[lane] : 1.0f;
    const float pg_in = (PASS == 1 && sgt.y > 1) ? pp[32 + lane] : 0.0f;
    bwd_tile<C, TF, PASS>(tile, sg, T_in, pg_in, pp, keys, vals, rec, rect, feat, v, tau, h, Ffwd, Afwd, dF, dA, gfeat,
                          gsig, gN, status);
  }
}

// Per split tile and pixel, in segment order: replace each segment's own
// (product T, sum w <f, g>) by the values it is entered with,
// T_in(s) = prod_{r<s} T_r and <P, g>_in(s) = sum_{r<s} T_in(r) sum_r.
__global__ void __launch_bounds__(32) bwd_prefix_kernel(const uint2* __restrict__ seg,
                                                        const uint32_t* __restrict__ multi,
                                                        unsigned long long* __restrict__ status,
                                                        float* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const unsigned long long n = status[kStMulti];
  for (unsigned long long m = blockIdx.x; m < n; m += gridDim.x) {
    const uint2 sgt = seg[multi[m]];
    float T = 1.0f, pg = 0.0f;
    for (uint32_t k = 0; k < sgt.y; ++k) {
      float* pp = part + (size_t)(sgt.x + k) * 64;
      const float Tk = pp[lane], sk = pp[32 + lane];
      pp[lane] = T;
      pp[32 + lane] = pg;
      pg = fmaf(T, sk, pg);
      T *= Tk;
    }
  }
}

// dL/dA_i = -N^T dL/dN N^T (top 3 rows of the 4x4 affine forms) with
// N = A_i^-1 = [h Binv | c - h Binv cw]; dL/dw_ik += <dL/dA_i, G_{j_ik}>.
__global__ void __launch_bounds__(256) lbs_bwd_kernel(int64_t n, const float* __restrict__ G,
                                                      const uint2* __restrict__ ijk, const uint32_t* __restrict__ jidx,
                                                      const float4* __restrict__ rec, float ox, float oy, float oz,
                                                      float h, const float* __restrict__ gN,
                                                      float* __restrict__ gw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 r3 = rec[4 * i + 3];
  if (r3.y == 0.0f) return;  // dropped voxel (det < 1e-3): no gradient
  const uint2 p = ijk[i];
  const float c[3] = {ox + ((float)(p.x & 0xffffu) + 0.5f) * h, oy + ((float)(p.x >> 16) + 0.5f) * h,
                      oz + ((float)p.y + 0.5f) * h};
  float N[3][4], dN[3][4];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float4 rr = rec[4 * i + r];
    N[r][0] = h * rr.x;
    N[r][1] = h * rr.y;
    N[r][2] = h * rr.z;
    N[r][3] = 0.0f;  // filled below
#pragma unroll
    for (int k = 0; k < 4; ++k) dN[r][k] = gN[12 * i + 4 * r + k];
  }
  const float cw[3] = {rec[4 * i].w, rec[4 * i + 1].w, rec[4 * i + 2].w};
#pragma unroll
  for (int r = 0; r < 3; ++r) N[r][3] = c[r] - (N[r][0] * cw[0] + N[r][1] * cw[1] + N[r][2] * cw[2]);
  // T = N^T dN (4x4; dN's and N's bottom rows are 0 and (0,0,0,1))
  float Tm[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s = 0.0f;
#pragma unroll
      for (int m = 0; m < 3; ++m) s += N[m][r] * dN[m][k];  // bottom row of dN is zero
      Tm[r][k] = s;
    }
  // dA = -T N^T (rows 0..2): column k < 3 pairs T's row with N's row k (all 4
  // entries); column 3 meets N's bottom row (0, 0, 0, 1).
  float dA[3][4];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dA[r][k] = -(Tm[r][0] * N[k][0] + Tm[r][1] * N[k][1] + Tm[r][2] * N[k][2] + Tm[r][3] * N[k][3]);
    dA[r][3] = -Tm[r][3];
  }
  const uint32_t jj = jidx[i];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = (jj >> (8 * q)) & 0xff;
    const float* Gj = G + 12 * j;
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k) s += dA[r][k] * Gj[4 * r + k];
    gw[4 * i + q] += s;
  }
}

template <int C, typename TF>
void launch_bwd_c(art_ctx* ctx, const ViewParams& v, const float* F, const float* A, const float* dF,
                  const float* dA, float* gfeat, float* gsig) {
  const int ntiles = v.tiles_x * v.tiles_y;
  const TF* feat = (const TF*)ctx->d_feat;
  cudaMemsetAsync(ctx->d_status + kStItems, 0, 4 * sizeof(unsigned long long), ctx->stream);  // items .. next merge
  ART_LAUNCH(ctx, "composite_plan", seg_plan_kernel, (ntiles + 255) / 256, 256, 0, ntiles, ctx->d_ranges,
             ctx->seg_len, ctx->d_seg, ctx->d_items, ctx->d_multi, ctx->d_status, (const uint32_t*)nullptr, 0);
  const int grid = ctx->composite_blocks;
  auto k0 = bwd_split_kernel<C, TF, 0>;
  ART_LAUNCH(ctx, "composite_bwd_scan", k0, grid, 32, 0, ctx->d_ranges, ctx->d_seg, ctx->d_items, ctx->d_keys,
             ctx->d_vals, ctx->d_rec, ctx->d_rect, feat, v, ctx->cfg.tau, ctx->h, F, A, dF, dA, gfeat, gsig,
             ctx->d_gN, ctx->d_status, ctx->d_part);
  ART_LAUNCH(ctx, "composite_bwd_prefix", bwd_prefix_kernel, 4 * ctx->num_sms, 32, 0, ctx->d_seg, ctx->d_multi,
             ctx->d_status, ctx->d_part);
  cudaMemsetAsync(ctx->d_status + kStNext, 0, sizeof(unsigned long long), ctx->stream);
  auto k1 = bwd_split_kernel<C, TF, 1>;
  ART_LAUNCH(ctx, "composite_bwd", k1, grid, 32, 0, ctx->d_ranges, ctx->d_seg, ctx->d_items, ctx->d_keys,
             ctx->d_vals, ctx->d_rec, ctx->d_rect, feat, v, ctx->cfg.tau, ctx->h, F, A, dF, dA, gfeat, gsig,
             ctx->d_gN, ctx->d_status, ctx->d_part);
}

template <int C>
void dispatch_bwd(art_ctx* ctx, const ViewParams& v, const float* F, const float* A, const float* dF, const float* dA,
                  float* gfeat, float* gsig) {
  if (ctx->feat_dtype == ART_F32) launch_bwd_c<C, float>(ctx, v, F, A, dF, dA, gfeat, gsig);
  else if (ctx->feat_dtype == ART_BF16) launch_bwd_c<C, __nv_bfloat16>(ctx, v, F, A, dF, dA, gfeat, gsig);
  else launch_bwd_c<C, __half>(ctx, v, F, A, dF, dA, gfeat, gsig);
}

}  // namespace

art_status launch_backward(art_ctx* ctx, const ViewParams& v, const float* F, const float* A, const float* dF,
                           const float* dA, float* gfeat, float* gsig, float* gw) {
  switch (ctx->C) {
    case 4: dispatch_bwd<4>(ctx, v, F, A, dF, dA, gfeat, gsig); break;
    case 8: dispatch_bwd<8>(ctx, v, F, A, dF, dA, gfeat, gsig); break;
    case 16: dispatch_bwd<16>(ctx, v, F, A, dF, dA, gfeat, gsig); break;
    case 32: dispatch_bwd<32>(ctx, v, F, A, dF, dA, gfeat, gsig); break;
    default: return fail(ctx, ART_ERR_UNSUPPORTED, "backward: C=%d not built", ctx->C);
  }
  const int64_t n = ctx->n;
  ART_LAUNCH(ctx, "lbs_bwd", lbs_bwd_kernel, (unsigned)((n + 255) / 256), 256, 0, n, ctx->d_G, ctx->d_ijk,
             ctx->d_jidx, ctx->d_rec, ctx->origin[0], ctx->origin[1], ctx->origin[2], ctx->h, ctx->d_gN, gw);
  return ART_OK;
}

}  // namespace art
