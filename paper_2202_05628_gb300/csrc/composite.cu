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
// buffer is full).  The reorder buffer is a per-lane ring in shared memory
// (slot-major, so the lanes of a warp touch 32 different banks): hits arrive
// nearly in order, so an insertion moves at most a few entries and a release
// only advances the ring's head.  The walk ends once every pixel of the tile has stopped
// (T < tau).
#include <algorithm>

#include "raster.cuh"

namespace art {
namespace {

enum Mode { kPlain = 0, kDebug = 1, kLabel = 2, kInterval = 3, kSH = 4 };

// Inputs and outputs of the learned-skip modes.
struct SkipArgs {
  const uchar2* bins;   // kInterval: proposal bins per pixel
  const float* thist;   // kLabel, kInterval: [tiles][kPropBins] optical-depth bounds
  float max_missed;     // coarse-check threshold
  int margin;           // kInterval: bins added on both sides
  uint32_t* queue;      // tiles queued for a later walk (count in status[qword])
  int qword;            // status word counting the queue
  float* labels;        // kLabel: [H][W][3]
  uchar2* lbins;        // kLabel: [H][W]
  const float* sh_coef; // kSH: [n][(L+1)^2][C] spherical-harmonics coefficients
  const float* sh_rot;  // kSH: [n][9] per voxel the map of world directions into its canonical frame
  int sh_degree;        // kSH: L (0 .. kShMaxDegree)
  uint32_t* xflag;      // kPlain, kInterval: per global tile, the stamp of the render that queued it
  uint32_t* xqueue;     // ... for the exact re-walk (count in status[kStExactQ])
  uint32_t xstamp;      // this render's stamp (never 0)
  int gtile;            // the walked tile's index in the (joint) tile space
  const uint8_t* tclass;  // kInterval: tile classes; forced tiles (class != 0) need no coarse check
};

// Real orthonormal spherical harmonics of degree <= L (<= kShMaxDegree) at
// the unit direction (x, y, z) (Eq. 2): Y[l*l + l + m],
//   Y_{l,0} = K_l^0 Q_l^0(z),  Y_{l,+-m} = sqrt(2) K_l^m Q_l^m(z) {Re, Im}((x + i y)^m)  (m > 0),
// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), Q_l^m the associated Legendre
// function without the Condon-Shortley phase divided by sin(theta)^m:
// Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) z Q_m^m,
// Q_l^m = ((2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m) / (l-m).
__device__ __forceinline__ void sh_basis(int L, float x, float y, float z, float (&Y)[kShMaxBases]) {
  float cr = 1.0f, ci = 0.0f;  // (x + i y)^m
  float qmm = 1.0f;            // (2m-1)!!
#pragma unroll
  for (int m = 0; m <= kShMaxDegree; ++m) {
    if (m > 0) {
      const float r = cr * x - ci * y, i = cr * y + ci * x;
      cr = r;
      ci = i;
      qmm *= (float)(2 * m - 1);
    }
    float q2 = 0.0f, q1 = qmm;  // Q_{l-2}^m, Q_{l-1}^m
#pragma unroll
    for (int l = m; l <= kShMaxDegree; ++l) {
      float q;
      if (l == m) {
        q = qmm;
      } else if (l == m + 1) {
        q = (float)(2 * m + 1) * z * qmm;
      } else {
        q = ((float)(2 * l - 1) * z * q1 - (float)(l + m - 1) * q2) / (float)(l - m);
      }
      if (l > m) {
        q2 = q1;
        q1 = q;
      }
      float ratio = 1.0f;  // (l-m)! / (l+m)!
#pragma unroll
      for (int k = l - m + 1; k <= l + m; ++k) ratio /= (float)k;
      const float K = sqrtf((float)(2 * l + 1) * 0.0795774715459476678f * ratio);  // 1 / (4 pi)
      if (l <= L) {
        if (m == 0) {
          Y[l * l + l] = K * q;
        } else {
          Y[l * l + l + m] = 1.41421356237309505f * K * q * cr;
          Y[l * l + l - m] = 1.41421356237309505f * K * q * ci;
        }
      }
    }
  }
}

// The view-dependent feature of voxel vid along the unit ray d (Eq. 2):
// S = sum_h k_h Y_h(P d), P the voxel's map of world directions into its
// canonical frame.
template <int C>
__device__ __forceinline__ void sh_feature(const SkipArgs& sk, uint32_t vid, float d0, float d1, float d2, float* f) {
  const float* P = sk.sh_rot + 9 * (size_t)vid;
  const float x = P[0] * d0 + P[1] * d1 + P[2] * d2;
  const float y = P[3] * d0 + P[4] * d1 + P[5] * d2;
  const float z = P[6] * d0 + P[7] * d1 + P[8] * d2;
  float Y[kShMaxBases];
#pragma unroll
  for (int h = 0; h < kShMaxBases; ++h) Y[h] = 0.0f;
  sh_basis(sk.sh_degree, x, y, z, Y);
  const int H = (sk.sh_degree + 1) * (sk.sh_degree + 1);
  const float* k = sk.sh_coef + (size_t)vid * H * C;
#pragma unroll
  for (int c = 0; c < C; ++c) f[c] = 0.0f;
#pragma unroll
  for (int h = 0; h < kShMaxBases; ++h) {
    if (h < H) {
      if constexpr (C % 4 == 0) {  // 16-byte loads (the rows of [n][H][C] stay 16-byte aligned)
        const float4* k4 = reinterpret_cast<const float4*>(k + h * C);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
          const float4 w = __ldg(k4 + q);
          f[4 * q] = fmaf(w.x, Y[h], f[4 * q]);
          f[4 * q + 1] = fmaf(w.y, Y[h], f[4 * q + 1]);
          f[4 * q + 2] = fmaf(w.z, Y[h], f[4 * q + 2]);
          f[4 * q + 3] = fmaf(w.w, Y[h], f[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) f[c] = fmaf(__ldg(k + h * C + c), Y[h], f[c]);
      }
    }
  }
}

// Inclusive prefix sums of the tile's depth-bin histogram into pre[64];
// returns the total.
__device__ __forceinline__ float tile_hist_prefix(const float* __restrict__ th, float* pre, int lane) {
  float p0 = th[lane], p1 = th[32 + lane];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float a = __shfl_up_sync(0xffffffffu, p0, o), b = __shfl_up_sync(0xffffffffu, p1, o);
    if (lane >= o) {
      p0 += a;
      p1 += b;
    }
  }
  const float t0 = __shfl_sync(0xffffffffu, p0, 31);
  pre[lane] = p0;
  pre[32 + lane] = p1 + t0;
  __syncwarp();
  return pre[63];
}

// A pixel whose reorder buffer was full released a hit that a later list
// entry may still precede.  With an exact re-walk queue (the composite of F
// and A) the tile is queued once for the exact walk, which rewrites it; else
// the releases are counted (overflow_order).
__device__ __forceinline__ void report_overflow(uint32_t n_over, const SkipArgs& sk,
                                                unsigned long long* __restrict__ status, int lane) {
  const bool any = __any_sync(0xffffffffu, n_over != 0);
  if (!any) return;
  if (sk.xqueue) {
    if (lane == 0 && atomicExch(sk.xflag + sk.gtile, sk.xstamp) != sk.xstamp)
      sk.xqueue[atomicAdd(status + kStExactQ, 1ull)] = (uint32_t)sk.gtile;
  } else if (n_over) {
    atomicAdd(status + kStOverflowOrder, (unsigned long long)n_over);
  }
}

// One warp per 8x4 tile, lane = pixel (x = lane & 7, y = lane >> 3).
template <int C, typename TF, typename TO, int MODE>
__device__ __forceinline__ void composite_tile(const int tile, const Seg& sg,
                                               const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                               const float4* __restrict__ rec, const short4* __restrict__ rect,
                                               const TF* __restrict__ feat, const ViewParams& v, float tau,
                                               TO* __restrict__ Fout, float* __restrict__ Aout,
                                               unsigned long long* __restrict__ status, const HitLog& dbg,
                                               const SkipArgs& sk) {
  constexpr bool DBG = MODE == kDebug;
  constexpr bool SH = MODE == kSH;                 // features evaluated per hit from SH coefficients
  constexpr bool FEAT = MODE != kLabel && !SH;  // staged feature rows (labels need densities only)
  constexpr int RING = Ring<C, TF>::kChunks;
  __shared__ float s_thr[NT];
  __shared__ uint32_t s_mask[NT];
  __shared__ float s_sig[RING][NT];
  __shared__ uint32_t s_vid[RING][NT];
  __shared__ __align__(16) TF s_feat[RING][NT][C];
  // raw voxel records of this chunk and the next; once a chunk is staged its
  // slots hold the instance's slab frame (b0, b1, b2, xl of stage_voxel)
  __shared__ __align__(16) float4 s_rec[2][NT][4];
  __shared__ short4 s_rc[2][NT];
  __shared__ float s_pt0[kPend][NT], s_pdl[kPend][NT];  // pending hits: ring of kPend per lane
  __shared__ uint32_t s_ppos[kPend][NT];

  const int lane = threadIdx.x & 31;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int sx = tx * TSX, sy = ty * TSY;
  const int px = sx + (lane & 7), py = sy + (lane >> 3);
  const bool inside = px < v.W && py < v.H;

  const RayDir rd = pixel_ray(v, px, py);

  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.0f;
  float T = 1.0f;
  bool done = !inside;
  int nb = 0, hd = 0;      // pending hits and the ring slot of the earliest
  Pend head{0.f, 0.f, 0u};  // the earliest pending hit (while nb > 0), kept in registers
  float t_back = 0.0f;      // t0 of the latest pending hit (while nb > 0)
  uint32_t n_over = 0;
  const uint32_t qmask = (1u << v.depth_bits) - 1u;
  const float qinv = 1.0f / v.dscale;
  const size_t pix = (size_t)py * v.W + px;
  int n_used = 0;
  int cur_chunk = 0;
  const uint2 rg = make_uint2(sg.begin, sg.end);
  // learned skip: this pixel's interval [t_lo, t_hi] and the deepest end over the warp
  float t_lo = 0.0f, t_hi = 3.4e38f, hi_w = 3.4e38f;
  int bn = 0, bf = kPropBins - 1;
  bool empty = false;
  if constexpr (MODE == kInterval) {
    // the tile composites over the union of its pixels' predicted intervals
    // (empty predictions contribute nothing), widened by the margin
    int lo_b = kPropBins, hi_b = -1;
    if (inside) {
      const uchar2 b = sk.bins[pix];
      if (b.y >= b.x) {
        lo_b = b.x;
        hi_b = b.y;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo_b = min(lo_b, __shfl_xor_sync(0xffffffffu, lo_b, o));
      hi_b = max(hi_b, __shfl_xor_sync(0xffffffffu, hi_b, o));
    }
    empty = hi_b < lo_b;
    bn = empty ? lo_b : max(lo_b - sk.margin, 0);
    bf = empty ? hi_b : min(hi_b + sk.margin, kPropBins - 1);
    const float D = (v.zfar - v.znear) / (float)kPropBins;
    t_lo = v.znear + (float)bn * D;
    t_hi = v.znear + (float)(bf + 1) * D;
    if (empty) done = true;
    hi_w = empty ? -3.4e38f : t_hi;
  }
  // labels: span of the significant hits and the transmittance after the last
  float lab_lo = 3.4e38f, lab_hi = -3.4e38f, lab_T = 1.0f;

  auto release_front = [&]() {
    const Pend h = head;
    hd = (hd + 1) & (kPend - 1);
    if (--nb > 0) head = Pend{s_pt0[hd][lane], s_pdl[hd][lane], s_ppos[hd][lane]};  // (used at the next release)
    const int ch = (int)(h.pos / NT), sl = (int)(h.pos % NT);
    float f[C];
    float sig;
    uint32_t vid;
    if (cur_chunk - ch < RING - 1) {  // (the ring's last slot takes the next chunk's rows)
      sig = s_sig[ch % RING][sl];
      vid = s_vid[ch % RING][sl];
      if constexpr (FEAT) row_to_float<C>(&s_feat[ch % RING][sl][0], f);
      if constexpr (SH) sh_feature<C>(sk, vid, rd.h[0] * rd.inv_n, rd.h[1] * rd.inv_n, rd.h[2] * rd.inv_n, f);
    } else {  // staged long ago: read the voxel again
      vid = vals[rg.x + h.pos];
      sig = rec[4 * (size_t)vid + 3].x;
      if constexpr (FEAT) load_feat<C>(feat + (size_t)vid * C, f);
      if constexpr (SH) sh_feature<C>(sk, vid, rd.h[0] * rd.inv_n, rd.h[1] * rd.inv_n, rd.h[2] * rd.inv_n, f);
    }
    if constexpr (DBG) {
      if (n_used < dbg.cap) {
        dbg.ids[pix * dbg.cap + n_used] = vid;
        dbg.t0[pix * dbg.cap + n_used] = h.t0;
        dbg.t1[pix * dbg.cap + n_used] = h.t0 + h.dl;
      }
      ++n_used;
    }
    float e = expf(-sig * h.dl);
    float w = T * (1.0f - e);
    if constexpr (FEAT || SH) {
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaf(w, f[c], acc[c]);
    }
    T *= e;
    if constexpr (MODE == kLabel) {
      if (w > kLabelWmin) {
        lab_lo = fminf(lab_lo, h.t0 + h.dl);
        lab_hi = fmaxf(lab_hi, h.t0);
        lab_T = T;
      }
    }
    if (T < tau) done = true;
  };

  // Staging pipeline: the records and feature rows of chunk i + 1 are copied
  // asynchronously while chunk i is walked, and the list entries of chunk
  // i + 2 are loaded into registers meanwhile.
  auto issue = [&](uint32_t cbase, int cslot, int b, uint32_t vid) {
    if (cbase + lane < rg.y) {
      const float4* rp = rec + 4 * (size_t)vid;
#pragma unroll
      for (int q = 0; q < 4; ++q) cp_async16(&s_rec[b][lane][q], rp + q);
      cp_async8(&s_rc[b][lane], rect + vid);
      if constexpr (FEAT) copy_row_async<C, TF>(feat + (size_t)vid * C, &s_feat[cslot][lane][0]);
    }
    cp_async_commit();
  };
  uint32_t vid_c = 0, key_c = 0, vid_n = 0, key_n = 0;  // list entries of the current and the next chunk
  if (rg.x + lane < rg.y) {
    vid_c = vals[rg.x + lane];
    key_c = keys[rg.x + lane];
  }
  issue(rg.x, 0, 0, vid_c);
  if (rg.x + NT + lane < rg.y) {
    vid_n = vals[rg.x + NT + lane];
    key_n = keys[rg.x + NT + lane];
  }

  for (uint32_t base = rg.x; base < rg.y; base += NT) {
    cur_chunk = (int)((base - rg.x) / NT);
    const int slot = cur_chunk % RING;
    const int b = cur_chunk & 1;
    __syncwarp();
    issue(base + NT, (cur_chunk + 1) % RING, b ^ 1, vid_n);
    const uint32_t vid = vid_c, key = key_c;
    vid_c = vid_n;
    key_c = key_n;
    if (base + 2 * NT + lane < rg.y) {
      vid_n = vals[base + 2 * NT + lane];
      key_n = keys[base + 2 * NT + lane];
    }
    cp_async_wait<1>();  // this chunk's copies (the next chunk's may be in flight)
    {  // stage one instance per lane
      const uint32_t k = base + lane;
      uint32_t m = 0;
      float thr = 3.4e38f;
      if (k < rg.y) {
        const float4 r0 = s_rec[b][lane][0], r1 = s_rec[b][lane][1], r2 = s_rec[b][lane][2],
                     r3 = s_rec[b][lane][3];
        const short4 rc = s_rc[b][lane];
        stage_voxel(r0, r1, r2, v, s_rec[b][lane][0], s_rec[b][lane][1], s_rec[b][lane][2], s_rec[b][lane][3]);
        s_sig[slot][lane] = r3.x;
        s_vid[slot][lane] = vid;
        thr = v.znear + (float)(key & qmask) * qinv;
        m = rect_mask(rc, sx, sy);
        if constexpr (MODE == kInterval) {
          if (thr > hi_w) m = 0;  // enters beyond every pixel's interval
        }
      }
      s_mask[lane] = m;
      s_thr[lane] = thr;
    }
    __syncwarp();
    if constexpr (MODE == kInterval) {
      if (s_thr[0] > hi_w) break;  // the list is sorted: nothing later can enter an interval
    }
    // every instance of this chunk and later enters at t >= the first threshold
    const float thr0 = s_thr[0];
    while (!done && nb > 0 && head.t0 < thr0) release_front();
    uint32_t cand = transpose32(s_mask[lane], lane);
    if (done) cand = 0;
    // the slab frame of the next candidate is read while the current one is tested
    int nidx = cand ? __ffs(cand) - 1 : 0;
    float4 f0 = s_rec[b][nidx][0], f1 = s_rec[b][nidx][1], f2 = s_rec[b][nidx][2], f3 = s_rec[b][nidx][3];
    while (cand) {
      const int idx = nidx;
      cand &= cand - 1;
      const float4 g0 = f0, g1 = f1, g2 = f2, g3 = f3;
      if (cand) {
        nidx = __ffs(cand) - 1;
        f0 = s_rec[b][nidx][0];
        f1 = s_rec[b][nidx][1];
        f2 = s_rec[b][nidx][2];
        f3 = s_rec[b][nidx][3];
      }
      float t0, dl, e[3];
      int ax0, ax1;
      if (!slab_hit(g0, g1, g2, g3, rd, v.znear, v.zfar, t0, dl, ax0, ax1, e)) continue;
      if (t0 < sg.t0_lo || t0 >= sg.t0_hi) continue;  // another segment's hit
      if constexpr (MODE == kInterval) {
        if (t0 + dl < t_lo || t0 > t_hi) continue;  // outside this pixel's interval
      }
      const Pend p{t0, dl, base - rg.x + (uint32_t)idx};
      if (nb == kPend) {
        // buffer full: release what this candidate's own bound allows (still
        // exact), and only if nothing can go, the earliest hit (counted)
        const float thr = s_thr[idx];
        while (!done && nb > 0 && head.t0 < thr) release_front();
        if (!done && nb == kPend) {
          ++n_over;
          release_front();
        }
        if (done) {
          cand = 0;
          break;
        }
      }
      int q = nb;
      if (nb > 0 && p.t0 <= t_back) {  // out of order: move the later pending hits up one slot
        while (q > 0) {
          const int j = (hd + q - 1) & (kPend - 1);
          const float bt = s_pt0[j][lane];
          if (p.t0 > bt) break;
          const Pend o{bt, s_pdl[j][lane], s_ppos[j][lane]};
          if (!pless(p, o)) break;
          const int k = (j + 1) & (kPend - 1);
          s_pt0[k][lane] = o.t0;
          s_pdl[k][lane] = o.dl;
          s_ppos[k][lane] = o.pos;
          --q;
        }
      } else {
        t_back = p.t0;  // appended: the latest pending hit
      }
      const int k = (hd + q) & (kPend - 1);
      s_pt0[k][lane] = p.t0;
      s_pdl[k][lane] = p.dl;
      s_ppos[k][lane] = p.pos;
      if (q == 0) head = p;
      ++nb;
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  while (nb > 0 && !done) release_front();
  cp_async_wait<0>();  // no copy may land in a later segment's staging
  __syncwarp();

  if (sg.part) {  // a segment of a split tile: partial sums for the merge
#pragma unroll
    for (int c = 0; c < C; ++c) sg.part[c * 32 + lane] = acc[c];
    sg.part[C * 32 + lane] = T;
    report_overflow(n_over, sk, status, lane);
    return;
  }
  // (the learned skip's coarse check ran with the proposal: a tile walked
  // here over its predicted interval passed it, the others over their
  // whole list)
  if constexpr (MODE == kLabel) {
    {
      __shared__ float s_pre[kPropBins];
      const float tot = tile_hist_prefix(sk.thist + (size_t)tile * kPropBins, s_pre, lane);
      {  // label bins: keep the significant hits and pass the check
        const float budget = kLabelBudget * sk.max_missed;
        const float tau_b = -log1pf(-budget);
        const bool c0 = (lane == 0 ? 0.0f : s_pre[lane - 1]) <= tau_b;
        const bool c1 = s_pre[31 + lane] <= tau_b;
        const int front = __popc(__ballot_sync(0xffffffffu, c0)) + __popc(__ballot_sync(0xffffffffu, c1)) - 1;
        if (inside) {
          const bool sig = lab_lo < 3.0e38f;
          const float bs = (float)kPropBins / (v.zfar - v.znear);
          const int blo = sig ? min(max((int)floorf((lab_lo - v.znear) * bs), 0), kPropBins - 1) : kPropBins - 1;
          const int bhi = sig ? min(max((int)floorf((lab_hi - v.znear) * bs), 0), kPropBins - 1) : 0;
          const float Ts = sig ? lab_T : 1.0f;
          int lbf = kPropBins - 1;
          for (int b = bhi; b < kPropBins; ++b)
            if (Ts * -expm1f(-(tot - s_pre[b])) <= budget) {
              lbf = b;
              break;
            }
          if (sk.labels) {
            sk.labels[3 * pix] = sig ? lab_lo : __int_as_float(0x7f800000);
            sk.labels[3 * pix + 1] = sig ? lab_hi : __int_as_float(0xff800000);
            sk.labels[3 * pix + 2] = Ts;
          }
          if (sk.lbins) sk.lbins[pix] = make_uchar2((uint8_t)min(blo, front), (uint8_t)lbf);
        }
      }
    }
  }
  if (inside && MODE != kLabel) {
    if constexpr (DBG) dbg.count[pix] = n_used;
    store_row<C>(Fout + pix * C, acc);
    if (Aout) Aout[pix] = 1.0f - T;
  }
  report_overflow(n_over, sk, status, lane);
}

template <int C, typename TF, typename TO, int MODE>
__global__ void __launch_bounds__(32) composite_kernel(const uint2* __restrict__ ranges,
                                                       const uint32_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ vals,
                                                       const float4* __restrict__ rec,
                                                       const short4* __restrict__ rect,
                                                       const TF* __restrict__ feat, ViewParams v, float tau,
                                                       TO* __restrict__ Fout, float* __restrict__ Aout,
                                                       unsigned long long* __restrict__ status, HitLog dbg,
                                                       SkipArgs sk) {
  const uint2 rg = ranges[blockIdx.x];
  const Seg sg{rg.x, rg.y, -3.4e38f, 3.4e38f, nullptr};
  composite_tile<C, TF, TO, MODE>(blockIdx.x, sg, keys, vals, rec, rect, feat, v, tau, Fout, Aout, status, dbg, sk);
}

// ------------------------------------------------------------ split walk
//
// A tile's list is cut at list positions p_k = start + k len / S into S
// segments of about seg_len entries.  Segment k composites the hits whose
// entry t0 lies in [D_k, D_{k+1}), D_k = the depth bound of the entry at p_k,
// front to back from T = 1.  It walks positions [p'_k, p_{k+1}): an entry can
// hold such a hit only if its distance range reaches D_k, i.e. its depth bound
// is at least D_k - (2 r_max + 3 quanta), and p'_k is the first such position.
// The merge combines the segments in order, F = F_0 + T_0 F_1 + T_0 T_1 F_2 ...,
// which is the front-to-back sum regrouped.  The stop rule holds exactly in
// the first segment that a pixel's transmittance enters below tau if that
// pixel entered it with T = 1; otherwise its tile is queued for the plain walk.


// Zero F and A of the tiles without instances (the segments cover the rest).
template <int C, typename TO>
__global__ void __launch_bounds__(256) composite_clear_kernel(const uint2* __restrict__ ranges, ViewParams v,
                                                              TO* __restrict__ Fout, float* __restrict__ Aout) {
  ART_PDL_ENTRY();
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= v.tiles_x * v.tiles_y) return;
  const uint2 rg = ranges[tile];
  if (rg.y > rg.x) return;
  const int sx = (tile % v.tiles_x) * TSX, sy = (tile / v.tiles_x) * TSY;
  const int px = sx + (lane & 7), py = sy + (lane >> 3);
  if constexpr ((C * sizeof(TO)) % 16 == 0) {  // each tile row is one contiguous run: 16-B chunks across the lanes
    const int npx = min(TSX, v.W - sx);
    const int chunks = npx * C * (int)sizeof(TO) / 16;
    for (int r = 0; r < TSY && sy + r < v.H; ++r) {
      uint4* row = reinterpret_cast<uint4*>(Fout + ((size_t)(sy + r) * v.W + sx) * C);
      for (int k = lane; k < chunks; k += 32) row[k] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (Aout && px < v.W && py < v.H) Aout[(size_t)py * v.W + px] = 0.0f;
  } else {
    if (px >= v.W || py >= v.H) return;
    const size_t pix = (size_t)py * v.W + px;
    float z[C];
#pragma unroll
    for (int c = 0; c < C; ++c) z[c] = 0.0f;
    store_row<C>(Fout + pix * C, z);
    if (Aout) Aout[pix] = 0.0f;
  }
}

template <int C, typename TF, typename TO, int MODE>
__global__ void __launch_bounds__(32, kCompositeWarps) composite_split_kernel(
    const uint2* __restrict__ ranges, const uint2* __restrict__ seg, const uint32_t* __restrict__ items,
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
    const short4* __restrict__ rect, const TF* __restrict__ feat, ViewParams v, float tau, TO* __restrict__ Fout,
    float* __restrict__ Aout, unsigned long long* __restrict__ status, float* __restrict__ part, SkipArgs sk) {
  ART_PDL_ENTRY();
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
    Seg sg = make_seg(v, ranges[tile], sgt, (uint32_t)i, keys, wq, lane);
    sg.part = sgt.y > 1 ? part + (size_t)i * (C + 1) * 32 : nullptr;
    SkipArgs skt = sk;
    skt.gtile = tile;
    composite_tile<C, TF, TO, MODE>(tile, sg, keys, vals, rec, rect, feat, v, tau, Fout, Aout, status, HitLog{},
                                    skt);
  }
}

// The split walk over a batch of views in one tile space: a segment's global
// tile names its view (vs->toff), whose parameters, rectangles and output
// maps it composites with.
template <int C, typename TF, typename TO>
__global__ void __launch_bounds__(32, kCompositeWarps) composite_split_views_kernel(
    const ViewSet* __restrict__ vs, const uint2* __restrict__ ranges, const uint2* __restrict__ seg,
    const uint32_t* __restrict__ items, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
    const float4* __restrict__ rec, const short4* __restrict__ rect, const TF* __restrict__ feat, float tau,
    unsigned long long* __restrict__ status, float* __restrict__ part, uint32_t* __restrict__ xflag,
    uint32_t* __restrict__ xqueue, uint32_t xstamp) {
  ART_PDL_ENTRY();
  const int lane = threadIdx.x & 31;
  const unsigned long long n_items = status[kStItems];
  for (;;) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(status + kStNext, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= n_items) break;
    const uint32_t tile = items[i];
    const int k = view_of(*vs, tile);
    const ViewParams v = vs->v[k];
    const uint2 sgt = seg[tile];
    Seg sg = make_seg(v, ranges[tile], sgt, (uint32_t)i, keys, seg_window(v, status), lane);
    sg.part = sgt.y > 1 ? part + (size_t)i * (C + 1) * 32 : nullptr;
    SkipArgs sk{};
    sk.xflag = xflag;
    sk.xqueue = xqueue;
    sk.xstamp = xstamp;
    sk.gtile = (int)tile;
    composite_tile<C, TF, TO, kPlain>((int)(tile - vs->toff[k]), sg, keys, vals, rec, rect + k * vs->rect_stride, feat,
                                      v, tau, (TO*)vs->F[k], vs->A[k], status, HitLog{}, sk);
  }
}

// Merge of the segments of the tiles with two or more: outputs, and the
// queue of the tiles whose stop falls inside a later segment.
// Channels merged by one warp: a split tile is merged by C / kMergeCh warps,
// each owning a channel group (the transmittance and the flags are computed
// by all of them; group 0 writes A and queues the tile).
constexpr int kMergeCh = 8;

template <int C, typename TO>
__device__ __forceinline__ void store_group(TO* __restrict__ p, const float* f) {
  store_row<(C >= kMergeCh ? kMergeCh : C)>(p, f);
}

template <int C, typename TO, int MODE>
__device__ __forceinline__ void merge_tile(int tile, int tl, int grp, int lane, const uint2* __restrict__ seg,
                                           const ViewParams& v, float tau, TO* __restrict__ Fout,
                                           float* __restrict__ Aout, unsigned long long* __restrict__ status,
                                           const float* __restrict__ part, const SkipArgs& sk) {
  constexpr int G = C >= kMergeCh ? C / kMergeCh : 1;  // channel groups
  constexpr int CG = C / G;
  const uint2 sgt = seg[tile];
  const int tx = tl % v.tiles_x, ty = tl / v.tiles_x;
  const int px = tx * TSX + (lane & 7), py = ty * TSY + (lane >> 3);
  const bool inside = px < v.W && py < v.H;
  const float* pbase = part + (size_t)sgt.x * (C + 1) * 32;
  // the segments this pixel composites (front to back until the stop) and the stop check
  float T = 1.0f;
  uint32_t kend = sgt.y;
  bool redo = false, stopped = false;
  for (uint32_t k0 = 0; k0 < sgt.y && !stopped; k0 += 8) {  // eight segments' loads in flight
    float tk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) tk[j] = k0 + j < sgt.y ? pbase[(size_t)(k0 + j) * (C + 1) * 32 + C * 32 + lane] : 1.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (stopped || k0 + j >= sgt.y) continue;
      if (T < 1.0f && T * tk[j] < tau) redo = true;  // the stop falls inside a later segment
      T *= tk[j];
      if (T < tau) {
        kend = k0 + j + 1;
        stopped = true;
      }
    }
  }
  // F = sum_k (T_0 ... T_{k-1}) F_k over this warp's channels; loads of two
  // segments in flight together
  float acc[CG];
#pragma unroll
  for (int c = 0; c < CG; ++c) acc[c] = 0.0f;
  float P = 1.0f;
  for (uint32_t k0 = 0; k0 < kend; k0 += 4) {  // four segments' loads in flight
    float f[4][CG], tq[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = k0 + j < kend;
      const float* pj = pbase + (size_t)(k0 + j) * (C + 1) * 32;
#pragma unroll
      for (int c = 0; c < CG; ++c) f[j][c] = in ? pj[(grp * CG + c) * 32 + lane] : 0.0f;
      tq[j] = in ? pj[C * 32 + lane] : 1.0f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int c = 0; c < CG; ++c) acc[c] = fmaf(P, f[j][c], acc[c]);
      P *= tq[j];
    }
  }
  if (inside) {
    const size_t pix = (size_t)py * v.W + px;
    store_group<C, TO>(Fout + pix * C + grp * CG, acc);
    if (grp == 0 && Aout) Aout[pix] = 1.0f - T;
  }
  if (grp == 0 && __any_sync(0xffffffffu, redo && inside) && lane == 0)
    sk.queue[atomicAdd(status + sk.qword, 1ull)] = (uint32_t)tile;
}

template <int C, typename TO, int MODE>
__global__ void __launch_bounds__(32) composite_merge_kernel(const uint2* __restrict__ seg,
                                                             const uint32_t* __restrict__ multi, ViewParams v,
                                                             float tau, TO* __restrict__ Fout,
                                                             float* __restrict__ Aout,
                                                             unsigned long long* __restrict__ status,
                                                             const float* __restrict__ part, SkipArgs sk) {
  ART_PDL_ENTRY();
  constexpr int G = C >= kMergeCh ? C / kMergeCh : 1;  // channel groups
  const int lane = threadIdx.x & 31;
  const unsigned long long n_items = status[kStMulti] * G;
  for (;;) {
    unsigned long long m = 0;
    if (lane == 0) m = atomicAdd(status + kStNextMerge, 1ull);
    m = __shfl_sync(0xffffffffu, m, 0);
    if (m >= n_items) break;
    const int tile = (int)multi[m / G];
    merge_tile<C, TO, MODE>(tile, tile, (int)(m % G), lane, seg, v, tau, Fout, Aout, status, part, sk);
    __syncwarp();
  }
}

// The merge over a batch of views (plain traversal): each split tile's view
// from its global tile.
template <int C, typename TO>
__global__ void __launch_bounds__(32) composite_merge_views_kernel(const ViewSet* __restrict__ vs,
                                                                   const uint2* __restrict__ seg,
                                                                   const uint32_t* __restrict__ multi, float tau,
                                                                   unsigned long long* __restrict__ status,
                                                                   const float* __restrict__ part, SkipArgs sk) {
  ART_PDL_ENTRY();
  constexpr int G = C >= kMergeCh ? C / kMergeCh : 1;
  const int lane = threadIdx.x & 31;
  const unsigned long long n_items = status[kStMulti] * G;
  for (;;) {
    unsigned long long m = 0;
    if (lane == 0) m = atomicAdd(status + kStNextMerge, 1ull);
    m = __shfl_sync(0xffffffffu, m, 0);
    if (m >= n_items) break;
    const uint32_t tile = multi[m / G];
    const int k = view_of(*vs, tile);
    const ViewParams v = vs->v[k];
    merge_tile<C, TO, kPlain>((int)tile, (int)(tile - vs->toff[k]), (int)(m % G), lane, seg, v, tau, (TO*)vs->F[k],
                              vs->A[k], status, part, sk);
    __syncwarp();
  }
}

// The sequential walk over queued tiles (plain, or with SH features).
template <int C, typename TF, typename TO, int MODE>
__global__ void __launch_bounds__(32) composite_queue_kernel(const uint2* __restrict__ ranges,
                                                             const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ vals,
                                                             const float4* __restrict__ rec,
                                                             const short4* __restrict__ rect,
                                                             const TF* __restrict__ feat, ViewParams v, float tau,
                                                             TO* __restrict__ Fout, float* __restrict__ Aout,
                                                             unsigned long long* __restrict__ status,
                                                             const uint32_t* __restrict__ queue, int qword,
                                                             SkipArgs sk_in) {
  ART_PDL_ENTRY();
  const unsigned long long n = status[qword];
  for (unsigned long long i = blockIdx.x; i < n; i += gridDim.x) {
    const int tile = (int)queue[i];
    const uint2 rg = ranges[tile];
    const Seg sg{rg.x, rg.y, -3.4e38f, 3.4e38f, nullptr};
    SkipArgs sk = sk_in;
    sk.gtile = tile;
    composite_tile<C, TF, TO, MODE>(tile, sg, keys, vals, rec, rect, feat, v, tau, Fout, Aout, status, HitLog{}, sk);
  }
}

// The sequential walk of a batch's queued tiles (global tile ids).
template <int C, typename TF, typename TO>
__global__ void __launch_bounds__(32) composite_queue_views_kernel(const ViewSet* __restrict__ vs,
                                                                   const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ keys,
                                                                   const uint32_t* __restrict__ vals,
                                                                   const float4* __restrict__ rec,
                                                                   const short4* __restrict__ rect,
                                                                   const TF* __restrict__ feat, float tau,
                                                                   unsigned long long* __restrict__ status,
                                                                   const uint32_t* __restrict__ queue, int qword,
                                                                   uint32_t* __restrict__ xflag,
                                                                   uint32_t* __restrict__ xqueue, uint32_t xstamp) {
  ART_PDL_ENTRY();
  const unsigned long long n = status[qword];
  for (unsigned long long i = blockIdx.x; i < n; i += gridDim.x) {
    const uint32_t tile = queue[i];
    const int k = view_of(*vs, tile);
    const ViewParams v = vs->v[k];
    const uint2 rg = ranges[tile];
    const Seg sg{rg.x, rg.y, -3.4e38f, 3.4e38f, nullptr};
    SkipArgs sk{};
    sk.xflag = xflag;
    sk.xqueue = xqueue;
    sk.xstamp = xstamp;
    sk.gtile = (int)tile;
    composite_tile<C, TF, TO, kPlain>((int)(tile - vs->toff[k]), sg, keys, vals, rec, rect + k * vs->rect_stride,
                                      feat, v, tau, (TO*)vs->F[k], vs->A[k], status, HitLog{}, sk);
  }
}

// Exact walk of the tiles queued because a pixel's reorder buffer
// overflowed: each lane collects every hit of its pixel's ray over the
// tile's whole list (entry distance, chord, list position) into its own
// scratch list, sorts it by (t0, chord, position) -- the order of the
// reorder buffer, Eq. 5-6's front to back -- and composites it with the
// stop rule, rewriting the tile's F and A.  A ray with more than kExactCap
// hits keeps its first kExactCap in list order and is counted in
// overflow_order.  With VIEWS the queue holds global tiles of a batch.
template <int C, typename TF, typename TO, bool VIEWS>
__global__ void __launch_bounds__(32) composite_exact_kernel(
    const ViewSet* __restrict__ vs, ViewParams v1, TO* __restrict__ F1, float* __restrict__ A1,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
    const float4* __restrict__ rec, const short4* __restrict__ rect, const TF* __restrict__ feat, float tau,
    unsigned long long* __restrict__ status, const uint32_t* __restrict__ xqueue, float2* __restrict__ xhit,
    uint32_t* __restrict__ xpos) {
  ART_PDL_ENTRY();
  __shared__ float4 s_b0[NT], s_b1[NT], s_b2[NT], s_xl[NT];
  __shared__ uint32_t s_mask[NT];
  const int lane = threadIdx.x & 31;
  float2* myh = xhit + ((size_t)blockIdx.x * 32 + lane) * kExactCap;
  uint32_t* myp = xpos + ((size_t)blockIdx.x * 32 + lane) * kExactCap;
  const unsigned long long n = status[kStExactQ];
  for (unsigned long long i = blockIdx.x; i < n; i += gridDim.x) {
    const uint32_t gt = xqueue[i];
    int k = 0;
    if constexpr (VIEWS) k = view_of(*vs, gt);
    const ViewParams v = VIEWS ? vs->v[k] : v1;
    const int tile = VIEWS ? (int)(gt - vs->toff[k]) : (int)gt;
    const short4* rc = VIEWS ? rect + k * vs->rect_stride : rect;
    TO* Fout = VIEWS ? (TO*)vs->F[k] : F1;
    float* Aout = VIEWS ? vs->A[k] : A1;
    const int sx = (tile % v.tiles_x) * TSX, sy = (tile / v.tiles_x) * TSY;
    const int px = sx + (lane & 7), py = sy + (lane >> 3);
    const bool inside = px < v.W && py < v.H;
    const RayDir rd = pixel_ray(v, px, py);
    const uint2 rg = ranges[gt];
    int m = 0;
    bool over = false;
    for (uint32_t base = rg.x; base < rg.y; base += NT) {  // collect
      __syncwarp();
      uint32_t msk = 0;
      if (base + lane < rg.y) {
        const uint32_t vid = vals[base + lane];
        const float4* rp = rec + 4 * (size_t)vid;
        stage_voxel(rp[0], rp[1], rp[2], v, s_b0[lane], s_b1[lane], s_b2[lane], s_xl[lane]);
        msk = rect_mask(rc[vid], sx, sy);
      }
      s_mask[lane] = msk;
      __syncwarp();
      uint32_t cand = transpose32(s_mask[lane], lane);
      if (!inside) cand = 0;
      while (cand) {
        const int idx = __ffs(cand) - 1;
        cand &= cand - 1;
        float t0, dl, e[3];
        int ax0, ax1;
        if (!slab_hit(s_b0[idx], s_b1[idx], s_b2[idx], s_xl[idx], rd, v.znear, v.zfar, t0, dl, ax0, ax1, e)) continue;
        if (m < kExactCap) {
          myh[m] = make_float2(t0, dl);
          myp[m] = base - rg.x + (uint32_t)idx;
          ++m;
        } else {
          over = true;
        }
      }
    }
    for (int a = 1; a < m; ++a) {  // sort by (t0, chord, list position)
      const float2 h = myh[a];
      const uint32_t q = myp[a];
      int b = a;
      while (b > 0) {
        const float2 g = myh[b - 1];
        const uint32_t r = myp[b - 1];
        if (!(h.x < g.x || (h.x == g.x && (h.y < g.y || (h.y == g.y && q < r))))) break;
        myh[b] = g;
        myp[b] = r;
        --b;
      }
      myh[b] = h;
      myp[b] = q;
    }
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.0f;
    float T = 1.0f;
    for (int a = 0; a < m; ++a) {  // composite front to back, stop once T < tau
      const uint32_t vid = vals[rg.x + myp[a]];
      const float sig = rec[4 * (size_t)vid + 3].x;
      float f[C];
      load_feat<C>(feat + (size_t)vid * C, f);
      const float e = expf(-sig * myh[a].y);
      const float w = T * (1.0f - e);
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaf(w, f[c], acc[c]);
      T *= e;
      if (T < tau) break;
    }
    if (inside) {
      const size_t pix = (size_t)py * v.W + px;
      store_row<C>(Fout + pix * C, acc);
      if (Aout) Aout[pix] = 1.0f - T;
    }
    if (over) atomicAdd(status + kStOverflowOrder, 1ull);
  }
}

// Zeroes the status words whose bits are set in mask, in the stream's chain
// of kernels (a memset node between two kernels would end their overlap).
__global__ void __launch_bounds__(32) zero_words_kernel(unsigned long long* __restrict__ status, uint32_t mask) {
  ART_PDL_ENTRY();
  if ((mask >> threadIdx.x) & 1u) status[threadIdx.x] = 0ull;
}
static_assert(kStWords <= 32, "zero_words_kernel covers the status words with one warp");

constexpr uint32_t bit(int w) { return 1u << w; }
// the counters of one split pass: segments, split tiles, both work counters
constexpr uint32_t kPassWords = bit(kStItems) | bit(kStMulti) | bit(kStNext) | bit(kStNextMerge);

void zero_words(art_ctx* ctx, uint32_t mask) {
  ART_LAUNCH_PDL(ctx, "composite_zero", zero_words_kernel, 1, 32, 0, ctx->d_status, mask);
}

// This render's stamp for the exact re-walk flags (a tile is queued once per
// stamp); the flags are zeroed when the stamps wrap.
uint32_t next_xstamp(art_ctx* ctx, size_t ntiles) {
  if (++ctx->xstamp == 0u) {
    cudaMemsetAsync(ctx->d_xflag, 0, sizeof(uint32_t) * ntiles, ctx->stream);
    ctx->xstamp = 1u;
  }
  return ctx->xstamp;
}

// The plain split walk of a batch of views: plan all segments, clear each
// view's empty tiles, walk all segments with persistent warps, merge the
// split tiles, then walk the tiles whose stop fell inside a later segment.
template <int C, typename TF, typename TO>
void views_walk(art_ctx* ctx, const ViewSet& vs) {
  const int ntiles = (int)vs.toff[vs.nv];
  const TF* feat = (const TF*)ctx->d_feat;
  const uint32_t xstamp = next_xstamp(ctx, (size_t)ntiles);
  zero_words(ctx, kPassWords | bit(kStFallback) | bit(kStExactQ));
  ART_LAUNCH_PDL(ctx, "composite_plan", seg_plan_kernel, (ntiles + 255) / 256, 256, 0, ntiles, ctx->d_ranges, ctx->seg_len,
             ctx->d_seg, ctx->d_items, ctx->d_multi, ctx->d_status, (const uint32_t*)nullptr, 0);
  for (int k = 0; k < vs.nv; ++k) {
    const ViewParams& v = vs.v[k];
    auto cfn = composite_clear_kernel<C, TO>;
    ART_LAUNCH_PDL(ctx, "composite_clear", cfn, (v.tiles_x * v.tiles_y + 7) / 8, 256, 0, ctx->d_ranges + vs.toff[k], v,
               (TO*)vs.F[k], vs.A[k]);
  }
  auto kfn = composite_split_views_kernel<C, TF, TO>;
  ART_LAUNCH_PDL(ctx, "composite", kfn, ctx->composite_blocks, 32, 0, ctx->d_vset, ctx->d_ranges, ctx->d_seg, ctx->d_items,
             ctx->d_keys, ctx->d_vals, ctx->d_rec, ctx->d_rect_v, feat, ctx->cfg.tau, ctx->d_status, ctx->d_part,
             ctx->d_xflag, ctx->d_xqueue, xstamp);
  SkipArgs sk{};
  sk.queue = ctx->d_fbq;
  sk.qword = kStFallback;
  auto mfn = composite_merge_views_kernel<C, TO>;
  ART_LAUNCH_PDL(ctx, "composite_merge", mfn, 32 * ctx->num_sms, 32, 0, ctx->d_vset, ctx->d_seg, ctx->d_multi,
             ctx->cfg.tau, ctx->d_status, ctx->d_part, sk);
  auto qfn = composite_queue_views_kernel<C, TF, TO>;
  ART_LAUNCH_PDL(ctx, "composite_fallback", qfn, std::min(ntiles, 16 * ctx->num_sms), 32, 0, ctx->d_vset, ctx->d_ranges,
             ctx->d_keys, ctx->d_vals, ctx->d_rec, ctx->d_rect_v, feat, ctx->cfg.tau, ctx->d_status, ctx->d_fbq,
             kStFallback, ctx->d_xflag, ctx->d_xqueue, xstamp);
  auto xfn = composite_exact_kernel<C, TF, TO, true>;
  ART_LAUNCH_PDL(ctx, "composite_exact", xfn, kExactBlocks, 32, 0, (const ViewSet*)ctx->d_vset, vs.v[0], (TO*)nullptr,
             (float*)nullptr, ctx->d_ranges, ctx->d_keys, ctx->d_vals, ctx->d_rec, ctx->d_rect_v, feat, ctx->cfg.tau,
             ctx->d_status, ctx->d_xqueue, ctx->d_xhit, ctx->d_xpos);
}

template <int C>
void views_dtypes(art_ctx* ctx, const ViewSet& vs, int F_dtype) {
  const int fd = ctx->feat_dtype;
  if (F_dtype == ART_F32) {
    if (fd == ART_F32) views_walk<C, float, float>(ctx, vs);
    else if (fd == ART_BF16) views_walk<C, __nv_bfloat16, float>(ctx, vs);
    else views_walk<C, __half, float>(ctx, vs);
  } else {
    if (fd == ART_F32) views_walk<C, float, __nv_bfloat16>(ctx, vs);
    else if (fd == ART_BF16) views_walk<C, __nv_bfloat16, __nv_bfloat16>(ctx, vs);
    else views_walk<C, __half, __nv_bfloat16>(ctx, vs);
  }
}

// One split pass, plain, learned-skip or SH: plan the segments, walk them
// with persistent warps, merge the split tiles; tiles that need the
// sequential walk go to sk.queue (count in status[sk.qword]).
template <int C, typename TF, typename TO>
void split_pass(art_ctx* ctx, const ViewParams& v, void* F, float* A, int mode, const SkipArgs& sk_in) {
  const int ntiles = v.tiles_x * v.tiles_y;
  const TF* feat = (const TF*)ctx->d_feat;
  SkipArgs sk = sk_in;
  if (mode != kSH) {  // the exact re-walk composites stored feature rows: not for SH features
    sk.xflag = ctx->d_xflag;
    sk.xqueue = ctx->d_xqueue;
  }
  ART_LAUNCH_PDL(ctx, "composite_plan", seg_plan_kernel, (ntiles + 255) / 256, 256, 0, ntiles, ctx->d_ranges,
                 ctx->seg_len, ctx->d_seg, ctx->d_items, ctx->d_multi, ctx->d_status, (const uint32_t*)nullptr, 0);
  if (!ctx->f_cleared) {
    auto cfn = composite_clear_kernel<C, TO>;
    ART_LAUNCH_PDL(ctx, "composite_clear", cfn, (ntiles + 7) / 8, 256, 0, ctx->d_ranges, v, (TO*)F, A);
  }
  const int grid = ctx->composite_blocks;
  const int mgrid = 32 * ctx->num_sms;
  if (mode == kInterval) {
    auto kfn = composite_split_kernel<C, TF, TO, kInterval>;
    ART_LAUNCH_PDL(ctx, "composite_skip", kfn, grid, 32, 0, ctx->d_ranges, ctx->d_seg, ctx->d_items, ctx->d_keys,
               ctx->d_vals, ctx->d_rec, ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, ctx->d_part,
               sk);
    auto mfn = composite_merge_kernel<C, TO, kInterval>;
    ART_LAUNCH_PDL(ctx, "composite_merge", mfn, mgrid, 32, 0, ctx->d_seg, ctx->d_multi, v, ctx->cfg.tau, (TO*)F,
               A, ctx->d_status, ctx->d_part, sk);
  } else if (mode == kSH) {
    auto kfn = composite_split_kernel<C, TF, TO, kSH>;
    ART_LAUNCH_PDL(ctx, "composite_sh", kfn, grid, 32, 0, ctx->d_ranges, ctx->d_seg, ctx->d_items, ctx->d_keys,
                   ctx->d_vals, ctx->d_rec, ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, ctx->d_part,
                   sk);
    auto mfn = composite_merge_kernel<C, TO, kPlain>;
    ART_LAUNCH_PDL(ctx, "composite_merge", mfn, mgrid, 32, 0, ctx->d_seg, ctx->d_multi, v, ctx->cfg.tau,
                   (TO*)F, A, ctx->d_status, ctx->d_part, sk);
  } else {
    auto kfn = composite_split_kernel<C, TF, TO, kPlain>;
    ART_LAUNCH_PDL(ctx, "composite", kfn, grid, 32, 0, ctx->d_ranges, ctx->d_seg, ctx->d_items,
               ctx->d_keys, ctx->d_vals, ctx->d_rec, ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A,
               ctx->d_status, ctx->d_part, sk);
    auto mfn = composite_merge_kernel<C, TO, kPlain>;
    ART_LAUNCH_PDL(ctx, "composite_merge", mfn, mgrid, 32, 0, ctx->d_seg, ctx->d_multi, v, ctx->cfg.tau, (TO*)F,
               A, ctx->d_status, ctx->d_part, sk);
  }
}

// One split pass (plain, learned-skip intervals or SH features), then the
// sequential walk of the tiles whose stop fell inside a later segment.
// With the learned skip, the tiles that failed the coarse check (run with
// the proposal) are walked in full by the same pass.
template <int C, typename TF, typename TO>
void split_walk(art_ctx* ctx, const ViewParams& v, void* F, float* A, int mode, const SkipArgs& sk_in) {
  const int ntiles = v.tiles_x * v.tiles_y;
  const TF* feat = (const TF*)ctx->d_feat;
  SkipArgs sk = sk_in;
  sk.queue = ctx->d_fbq;
  sk.qword = kStFallback;
  sk.xstamp = next_xstamp(ctx, (size_t)ntiles);
  zero_words(ctx, kPassWords | bit(kStFallback) | bit(kStExactQ));
  split_pass<C, TF, TO>(ctx, v, F, A, mode, sk);
  const uint32_t* seq = ctx->d_fbq;
  const int seq_word = kStFallback;
  const int qgrid = std::min(ntiles, 16 * ctx->num_sms);
  SkipArgs sq{};
  if (mode == kSH) {  // the stop cases of SH features: their sequential walk evaluates the harmonics
    sq = sk_in;
    auto qfn = composite_queue_kernel<C, TF, TO, kSH>;
    ART_LAUNCH_PDL(ctx, "composite_fallback", qfn, qgrid, 32, 0, ctx->d_ranges, ctx->d_keys, ctx->d_vals, ctx->d_rec,
                   ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, seq, seq_word, sq);
    return;
  }
  sq.xflag = ctx->d_xflag;
  sq.xqueue = ctx->d_xqueue;
  sq.xstamp = sk.xstamp;
  auto qfn = composite_queue_kernel<C, TF, TO, kPlain>;
  ART_LAUNCH_PDL(ctx, "composite_fallback", qfn, qgrid, 32, 0, ctx->d_ranges, ctx->d_keys, ctx->d_vals, ctx->d_rec,
             ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, seq, seq_word, sq);
  auto xfn = composite_exact_kernel<C, TF, TO, false>;
  ART_LAUNCH_PDL(ctx, "composite_exact", xfn, kExactBlocks, 32, 0, (const ViewSet*)nullptr, v, (TO*)F, A, ctx->d_ranges,
             ctx->d_keys, ctx->d_vals, ctx->d_rec, ctx->d_rect, feat, ctx->cfg.tau, ctx->d_status, ctx->d_xqueue,
             ctx->d_xhit, ctx->d_xpos);
}

template <int C, typename TF, typename TO>
void launch_c(art_ctx* ctx, const ViewParams& v, void* F, float* A, const HitLog* dbg, int mode, const SkipArgs& sk) {
  const int ntiles = v.tiles_x * v.tiles_y;
  const TF* feat = (const TF*)ctx->d_feat;
  if (mode == kDebug) {
    auto kfn = composite_kernel<C, TF, TO, kDebug>;
    ART_LAUNCH(ctx, "composite_debug", kfn, ntiles, 32, 0, ctx->d_ranges, ctx->d_keys, ctx->d_vals, ctx->d_rec,
               ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, *dbg, sk);
  } else if (mode == kLabel) {
    auto kfn = composite_kernel<C, TF, TO, kLabel>;
    ART_LAUNCH(ctx, "composite_labels", kfn, ntiles, 32, 0, ctx->d_ranges, ctx->d_keys, ctx->d_vals, ctx->d_rec,
               ctx->d_rect, feat, v, ctx->cfg.tau, (TO*)F, A, ctx->d_status, HitLog{}, sk);
  } else {
    split_walk<C, TF, TO>(ctx, v, F, A, mode, sk);
  }
}

template <int C>
art_status dispatch_dtypes(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A, const HitLog* dbg,
                           int mode, const SkipArgs& sk) {
  int fd = ctx->feat_dtype;
  if (F_dtype == ART_F32) {
    if (fd == ART_F32) launch_c<C, float, float>(ctx, v, F, A, dbg, mode, sk);
    else if (fd == ART_BF16) launch_c<C, __nv_bfloat16, float>(ctx, v, F, A, dbg, mode, sk);
    else launch_c<C, __half, float>(ctx, v, F, A, dbg, mode, sk);
  } else {
    if (dbg) return fail(ctx, ART_ERR_INVALID_ARG, "hit logging writes FP32 feature maps");
    if (fd == ART_F32) launch_c<C, float, __nv_bfloat16>(ctx, v, F, A, nullptr, mode, sk);
    else if (fd == ART_BF16) launch_c<C, __nv_bfloat16, __nv_bfloat16>(ctx, v, F, A, nullptr, mode, sk);
    else launch_c<C, __half, __nv_bfloat16>(ctx, v, F, A, nullptr, mode, sk);
  }
  return ART_OK;
}

art_status dispatch(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A, const HitLog* dbg, int mode,
                    const SkipArgs& sk) {
  if (v.tile_w != TSX || v.tile_h != TSY) return fail(ctx, ART_ERR_UNSUPPORTED, "composite: tiles must be 8x4");
  switch (ctx->C) {
    case 4: return dispatch_dtypes<4>(ctx, v, F, F_dtype, A, dbg, mode, sk);
    case 8: return dispatch_dtypes<8>(ctx, v, F, F_dtype, A, dbg, mode, sk);
    case 16: return dispatch_dtypes<16>(ctx, v, F, F_dtype, A, dbg, mode, sk);
    case 32: return dispatch_dtypes<32>(ctx, v, F, F_dtype, A, dbg, mode, sk);
    default: return fail(ctx, ART_ERR_UNSUPPORTED, "composite: C=%d not built (4, 8, 16, 32)", ctx->C);
  }
}

}  // namespace

art_status launch_composite(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A, const void* dbg_log) {
  const HitLog* dbg = (const HitLog*)dbg_log;
  return dispatch(ctx, v, F, F_dtype, A, dbg, dbg ? kDebug : kPlain, SkipArgs{});
}

art_status launch_composite_views(art_ctx* ctx, const ViewSet& vs, int F_dtype) {
  switch (ctx->C) {
    case 4: views_dtypes<4>(ctx, vs, F_dtype); return ART_OK;
    case 8: views_dtypes<8>(ctx, vs, F_dtype); return ART_OK;
    case 16: views_dtypes<16>(ctx, vs, F_dtype); return ART_OK;
    case 32: views_dtypes<32>(ctx, vs, F_dtype); return ART_OK;
    default: return fail(ctx, ART_ERR_UNSUPPORTED, "composite: C=%d not built (4, 8, 16, 32)", ctx->C);
  }
}

// Per voxel, the rotation that maps world directions into its canonical
// frame: the orthogonal polar factor of its unit-cube map A_lin^-1 / h
// (A_lin = R S gives A_lin^-1 = S^-1 R^T, whose orthogonal factor is R^T),
// by scaled Newton steps X <- (g X + (g X)^-T) / 2, g = |det X|^(-1/3).
__global__ void __launch_bounds__(256) sh_rot_kernel(int64_t n, const float4* __restrict__ rec, float* __restrict__ rot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 r0 = rec[4 * i], r1 = rec[4 * i + 1], r2 = rec[4 * i + 2], r3 = rec[4 * i + 3];
  float X[9] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
  if (r3.y == 0.0f) {  // dropped voxel: never listed
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = (k % 4 == 0) ? 1.0f : 0.0f;
  } else {
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
      const float cof[9] = {X[4] * X[8] - X[5] * X[7], X[5] * X[6] - X[3] * X[8], X[3] * X[7] - X[4] * X[6],
                            X[2] * X[7] - X[1] * X[8], X[0] * X[8] - X[2] * X[6], X[1] * X[6] - X[0] * X[7],
                            X[1] * X[5] - X[2] * X[4], X[2] * X[3] - X[0] * X[5], X[0] * X[4] - X[1] * X[3]};
      const float det = X[0] * cof[0] + X[1] * cof[1] + X[2] * cof[2];
      const float g = it < 6 ? 1.0f / cbrtf(fabsf(det)) : 1.0f;  // scaling speeds the first steps
#pragma unroll
      for (int k = 0; k < 9; ++k) X[k] = 0.5f * (g * X[k] + cof[k] / (g * det));
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) rot[9 * i + k] = X[k];
}

art_status launch_composite_sh(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A) {
  ART_LAUNCH(ctx, "sh_rot", sh_rot_kernel, (unsigned)((ctx->n + 255) / 256), 256, 0, ctx->n,
             (const float4*)ctx->d_rec, ctx->d_sh_rot);
  SkipArgs sk{};
  sk.sh_coef = ctx->d_sh;
  sk.sh_rot = ctx->d_sh_rot;
  sk.sh_degree = ctx->sh_degree;
  return dispatch(ctx, v, F, F_dtype, A, nullptr, kSH, sk);
}

art_status launch_composite_skip(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A) {
  SkipArgs sk{};
  sk.bins = reinterpret_cast<const uchar2*>(ctx->d_bins);
  sk.thist = ctx->d_thist;
  sk.max_missed = ctx->cfg.max_missed;
  sk.margin = ctx->cfg.margin;
  sk.tclass = ctx->d_tclass;  // (launch_tile_class ran for this view)
  return dispatch(ctx, v, F, F_dtype, A, nullptr, kInterval, sk);
}

namespace {
// Resident one-warp blocks per SM of the interval walk (the largest shared
// memory of the split walk's modes): its feature ring, pending-hit rings and
// staged records bound it, and so do its registers (kCompositeWarps).
template <int C, typename TF>
int split_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, composite_split_kernel<C, TF, __nv_bfloat16, kInterval>, 32,
                                                    0) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  return std::max(1, std::min(kCompositeWarps, n));
}

template <int C>
int split_blocks_c(int feat_bytes) {
  return feat_bytes == 4 ? split_blocks_per_sm<C, float>() : split_blocks_per_sm<C, __nv_bfloat16>();
}
}  // namespace

int composite_blocks_per_sm(int C, int feat_bytes) {
  switch (C) {
    case 4: return split_blocks_c<4>(feat_bytes);
    case 8: return split_blocks_c<8>(feat_bytes);
    case 16: return split_blocks_c<16>(feat_bytes);
    default: return split_blocks_c<32>(feat_bytes);
  }
}

namespace {
template <int C>
void clear_c(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A) {
  const int ntiles = v.tiles_x * v.tiles_y;
  if (F_dtype == ART_F32) {
    ART_LAUNCH_PDL(ctx, "composite_clear", (composite_clear_kernel<C, float>), (ntiles + 7) / 8, 256, 0, ctx->d_ranges,
                   v, (float*)F, A);
  } else {
    ART_LAUNCH_PDL(ctx, "composite_clear", (composite_clear_kernel<C, __nv_bfloat16>), (ntiles + 7) / 8, 256, 0,
                   ctx->d_ranges, v, (__nv_bfloat16*)F, A);
  }
}
}  // namespace

art_status launch_composite_clear(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A) {
  if (v.tile_w != TSX || v.tile_h != TSY) return fail(ctx, ART_ERR_UNSUPPORTED, "composite: tiles must be 8x4");
  switch (ctx->C) {
    case 4: clear_c<4>(ctx, v, F, F_dtype, A); break;
    case 8: clear_c<8>(ctx, v, F, F_dtype, A); break;
    case 16: clear_c<16>(ctx, v, F, F_dtype, A); break;
    case 32: clear_c<32>(ctx, v, F, F_dtype, A); break;
    default: return fail(ctx, ART_ERR_UNSUPPORTED, "composite: C=%d not built (4, 8, 16, 32)", ctx->C);
  }
  return ART_OK;
}

art_status launch_composite_labels(art_ctx* ctx, const ViewParams& v, float* labels, uint8_t* bins) {
  SkipArgs sk{};
  sk.thist = ctx->d_thist;
  sk.max_missed = ctx->cfg.max_missed;
  sk.labels = labels;
  sk.lbins = reinterpret_cast<uchar2*>(bins);
  return dispatch(ctx, v, nullptr, ART_F32, nullptr, nullptr, kLabel, sk);
}

// Hit log layout shared with api.cu.
void* make_hit_log(int32_t* count, uint32_t* ids, float* t0, float* t1, int cap) {
  HitLog* h = new HitLog{count, ids, t0, t1, cap};
  return h;
}
void free_hit_log(void* p) { delete (HitLog*)p; }

}  // namespace art
