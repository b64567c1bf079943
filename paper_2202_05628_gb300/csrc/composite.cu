// Dynamic volume rendering of the warped voxels into the feature map F and
// the coarse opacity map A (arXiv 2202.05628, Sec. 3.1 "Dynamic Volume
// Rendering", Eq. 5-6 and the early-stop rule).
//
// One warp per 8x4 screen tile, one lane per pixel.  The tile's instance
// list is sorted by a lower bound of the distance from the camera centre to
// the voxel.  It is staged through shared memory in chunks of 32 instances
// (one per lane: unit-cube map, density, pixel-rectangle mask and the feature
// row, all gathered with vector loads); feature rows stay in a ring of chunks
// so that late releases still read shared memory.  Per chunk the warp
// transposes the 32x32 bit matrix "instance covers pixel" with shuffles, so
// that every lane walks only the instances whose rectangle contains its
// pixel.  A lane intersects its ray exactly with each such voxel, keeps hits
// in a small register reorder buffer sorted by (t0, t1, list position), and
// composites a hit front to back once no later list entry can start before it
// (t0 < the distance bound of the next chunk, or of the candidate when the
// buffer is full).  The walk ends once every pixel of the tile has stopped
// (T < tau).
#include "raster.cuh"

namespace art {
namespace {

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

  float d0, d1, d2;
  pixel_dir(v, px, py, d0, d1, d2);

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
        m = rect_mask(rc, sx, sy);
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
      float t0, t1, e[3];
      int ax0, ax1;
      if (!slab_hit(s_b0[idx], s_b1[idx], s_b2[idx], d0, d1, d2, v.znear, v.zfar, t0, t1, ax0, ax1, e)) continue;
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
