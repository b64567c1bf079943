// Forward kinematics, linear blend skinning and per-view projection of the
// warped voxels (arXiv 2202.05628, Sec. 3.1 "Rigging and Deformation", Eq. 4).
#include "internal.cuh"

namespace art {
namespace {

// R = I + a K + b K^2 with K = [r]_x, a = sin(th)/th, b = (1 - cos th)/th^2
// (Rodrigues' formula with an unnormalised axis).
__device__ void rodrigues(const float* r, float* R) {
  float th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  float th = sqrtf(th2);
  float a, b;
  if (th < 1e-6f) {
    a = 1.0f;
    b = 0.5f;
  } else {
    a = sinf(th) / th;
    float sh = sinf(0.5f * th) / th;
    b = 2.0f * sh * sh;
  }
  float K[9] = {0.f, -r[2], r[1], r[2], 0.f, -r[0], -r[1], r[0], 0.f};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float k2 = K[i * 3 + 0] * K[0 * 3 + j] + K[i * 3 + 1] * K[1 * 3 + j] + K[i * 3 + 2] * K[2 * 3 + j];
      R[i * 3 + j] = (i == j ? 1.0f : 0.0f) + a * K[i * 3 + j] + b * k2;
    }
}

// One thread per joint forms its local transform L_j = [R(r_j) | rest_j -
// rest_parent] (the root's premultiplied by the global [R | T]); one thread
// then walks the tree (parents precede children), M_j = M_parent L_j, and
// every joint writes G_j = M_j [I | -rest_j].
// skel: J parent indices stored as floats, then rest[J][3]; pose: r[J][3], R[3], T[3].
__global__ void __launch_bounds__(kMaxJoints) fk_kernel(int J, const float* __restrict__ skel,
                                                        const float* __restrict__ pose, float* __restrict__ G,
                                                        unsigned long long* __restrict__ status) {
  ART_PDL_ENTRY();
  if (threadIdx.x == 0) {  // the pose's counters, accumulated by the skinning that follows
    status[kStDegenerate] = 0ull;
    status[kStRmax] = 0ull;
  }
  __shared__ float sL[kMaxJoints][12];
  __shared__ float sM[kMaxJoints][12];
  __shared__ int sp[kMaxJoints];
  __shared__ float srest[kMaxJoints][3];
  const int j = threadIdx.x;
  const bool on = j < J;
  int p = -1;
  float r[3] = {0.f, 0.f, 0.f}, rg[3], Tg[3];
  if (on) {
    p = (int)skel[j];
    sp[j] = p;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      srest[j][a] = skel[J + 3 * j + a];
      r[a] = pose[3 * j + a];
      rg[a] = pose[3 * J + a];
      Tg[a] = pose[3 * J + 3 + a];
    }
  }
  __syncthreads();
  if (on) {
    float Rl[9];
    rodrigues(r, Rl);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) sL[j][a * 4 + b] = Rl[a * 3 + b];
      sL[j][a * 4 + 3] = srest[j][a] - (p >= 0 ? srest[p][a] : 0.0f);
    }
    if (p < 0) {  // the global transform stands in as the root's parent
      float Rg[9];
      rodrigues(rg, Rg);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) sM[j][a * 4 + b] = Rg[a * 3 + b];
        sM[j][a * 4 + 3] = Tg[a];
      }
    }
  }
  __syncthreads();
  if (j == 0) {
    for (int k = 0; k < J; ++k) {
      const int q = sp[k];
      float P[12];
#pragma unroll
      for (int m = 0; m < 12; ++m) P[m] = sM[q >= 0 ? q : k][m];
      const float* L = sL[k];
      float* Mk = sM[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
          Mk[a * 4 + b] = P[a * 4 + 0] * L[0 * 4 + b] + P[a * 4 + 1] * L[1 * 4 + b] + P[a * 4 + 2] * L[2 * 4 + b];
        Mk[a * 4 + 3] = P[a * 4 + 0] * L[3] + P[a * 4 + 1] * L[7] + P[a * 4 + 2] * L[11] + P[a * 4 + 3];
      }
    }
  }
  __syncthreads();
  if (on) {
    const float* M = sM[j];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) G[12 * j + a * 4 + b] = M[a * 4 + b];
      G[12 * j + a * 4 + 3] =
          M[a * 4 + 3] - (M[a * 4 + 0] * srest[j][0] + M[a * 4 + 1] * srest[j][1] + M[a * 4 + 2] * srest[j][2]);
    }
  }
}

// Per voxel: A = sum_k w_k G_{j_k}; det check; record the unit-cube map
// u = Binv (x - cw), Binv = (A_lin)^-1 / h, and the bounding data of the
// warped parallelepiped (centre cw, half axes, bounding radius r).
__global__ void __launch_bounds__(256) lbs_kernel(int64_t n, int J, const float* __restrict__ G,
                                                  const uint2* __restrict__ ijk, const uint32_t* __restrict__ jidx,
                                                  const float4* __restrict__ wts, const float* __restrict__ sigma,
                                                  float ox, float oy, float oz, float h, float4* __restrict__ rec,
                                                  float4* __restrict__ geo, unsigned long long* __restrict__ status) {
  ART_PDL_ENTRY();
  __shared__ float4 sG[kMaxJoints * 3];  // G_j as three float4 rows
  __shared__ float4 s_out[2][8][32 * 4];  // per warp: the 32 voxels' records and bounds
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < J * 3; k += blockDim.x)
    sG[k] = make_float4(G[4 * k], G[4 * k + 1], G[4 * k + 2], G[4 * k + 3]);
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool degenerate = false;
  float rmax = 0.0f;
  if (i < n) {
    uint2 p = ijk[i];
    float c[3] = {ox + ((float)(p.x & 0xffffu) + 0.5f) * h, oy + ((float)(p.x >> 16) + 0.5f) * h,
                  oz + ((float)p.y + 0.5f) * h};
    uint32_t jj = jidx[i];
    float4 w = wts[i];
    float wk[4] = {w.x, w.y, w.z, w.w};
    float A[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) A[m] = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = (jj >> (8 * k)) & 0xff;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float4 g = sG[3 * j + m];
        A[4 * m] = fmaf(wk[k], g.x, A[4 * m]);
        A[4 * m + 1] = fmaf(wk[k], g.y, A[4 * m + 1]);
        A[4 * m + 2] = fmaf(wk[k], g.z, A[4 * m + 2]);
        A[4 * m + 3] = fmaf(wk[k], g.w, A[4 * m + 3]);
      }
    }
    float a = A[0], b = A[1], cc = A[2], d = A[4], e = A[5], f = A[6], g = A[8], hh = A[9], k2 = A[10];
    float c00 = e * k2 - f * hh, c01 = f * g - d * k2, c02 = d * hh - e * g;
    float det = a * c00 + b * c01 + cc * c02;
    float cw[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) cw[r] = A[r * 4] * c[0] + A[r * 4 + 1] * c[1] + A[r * 4 + 2] * c[2] + A[r * 4 + 3];
    float4 out_rec[4];
    float4 out_geo[4];
    if (!(det >= kDetMin)) {
      degenerate = true;
      out_rec[0] = out_rec[1] = out_rec[2] = make_float4(0.f, 0.f, 0.f, 0.f);
      out_rec[3] = make_float4(sigma[i], 0.f, 0.f, 0.f);
      out_geo[0] = make_float4(cw[0], cw[1], cw[2], -1.0f);
      out_geo[1] = out_geo[2] = out_geo[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      // inverse of the 3x3 block via its adjugate, scaled by 1/h
      float s = 1.0f / (det * h);
      float inv[9] = {c00 * s, (cc * hh - b * k2) * s, (b * f - cc * e) * s,
                      c01 * s, (a * k2 - cc * g) * s, (cc * d - a * f) * s,
                      c02 * s, (b * g - a * hh) * s, (a * e - b * d) * s};
      out_rec[0] = make_float4(inv[0], inv[1], inv[2], cw[0]);
      out_rec[1] = make_float4(inv[3], inv[4], inv[5], cw[1]);
      out_rec[2] = make_float4(inv[6], inv[7], inv[8], cw[2]);
      out_rec[3] = make_float4(sigma[i], 1.0f, 0.f, 0.f);
      float hh2 = 0.5f * h;
      float ax[3] = {A[0] * hh2, A[4] * hh2, A[8] * hh2};
      float ay[3] = {A[1] * hh2, A[5] * hh2, A[9] * hh2};
      float az[3] = {A[2] * hh2, A[6] * hh2, A[10] * hh2};
      float r2 = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float sy = (q & 1) ? -1.0f : 1.0f, sz = (q & 2) ? -1.0f : 1.0f;
        float vx = ax[0] + sy * ay[0] + sz * az[0];
        float vy = ax[1] + sy * ay[1] + sz * az[1];
        float vz = ax[2] + sy * ay[2] + sz * az[2];
        r2 = fmaxf(r2, vx * vx + vy * vy + vz * vz);
      }
      // slight growth keeps the radius a bound under FP32 rounding
      float r = sqrtf(r2) * (1.0f + 1e-6f) + 1e-9f;
      rmax = fmaxf(rmax, r);
      out_geo[0] = make_float4(cw[0], cw[1], cw[2], r);
      out_geo[1] = make_float4(ax[0], ax[1], ax[2], 0.f);
      out_geo[2] = make_float4(ay[0], ay[1], ay[2], 0.f);
      out_geo[3] = make_float4(az[0], az[1], az[2], 0.f);
    }
    // (written below through shared memory, coalesced per warp)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      s_out[0][warp][lane * 4 + (m ^ ((lane >> 1) & 3))] = out_rec[m];
      s_out[1][warp][lane * 4 + (m ^ ((lane >> 1) & 3))] = out_geo[m];
    }
  }
  __syncwarp();
  {  // float4 o of the warp's 32 records: voxel o / 4, row o % 4 (rows stored XOR-swizzled)
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + warp * 32;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int o = m * 32 + lane, vv = o >> 2, slot = vv * 4 + ((o & 3) ^ ((vv >> 1) & 3));
      if (w0 + vv < n) {
        rec[4 * w0 + o] = s_out[0][warp][slot];
        geo[4 * w0 + o] = s_out[1][warp][slot];
      }
    }
  }
  // block totals: degenerate voxels and the largest bounding radius of the
  // pose (positive floats order as their bits), one atomic each per block
  __shared__ unsigned s_deg;
  __shared__ unsigned s_rmax;
  if (threadIdx.x == 0) {
    s_deg = 0;
    s_rmax = 0;
  }
  __syncthreads();
  const unsigned bal = __ballot_sync(0xffffffffu, degenerate);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) {
    if (bal) atomicAdd(&s_deg, (unsigned)__popc(bal));
    if (rmax > 0.0f) atomicMax(&s_rmax, __float_as_uint(rmax));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_deg) atomicAdd(status + kStDegenerate, (unsigned long long)s_deg);
    if (s_rmax) atomicMax(status + kStRmax, (unsigned long long)s_rmax);
  }
}

// Per voxel and view: projected-corner pixel rectangle (grown by kBboxPad),
// screen-tile count, and the depth key: a floor-quantised lower bound of the
// distance from the camera centre to any point of the voxel (|cw - o| - r),
// which bounds the ray parameter t of any entry point from below.
//
// Each voxel then adds one to the instance count of every tile its rectangle
// covers (lanes of a warp that hit the same tile in the same step add
// together), the first step of the binning; block 0 also clears the tile
// scan's look-back words and its block ticket and the active-group count.
__device__ __forceinline__ void project_voxel(int64_t i, const float4* __restrict__ geo, const ViewParams& v,
                                              short4* __restrict__ rect, uint32_t* __restrict__ q,
                                              uint32_t* __restrict__ cnt, const float* __restrict__ sigma,
                                              uint32_t* __restrict__ hbin, float* __restrict__ htau, short4& rc,
                                              uint32_t& c) {
  float4 g0 = geo[4 * i], g1 = geo[4 * i + 1], g2 = geo[4 * i + 2], g3 = geo[4 * i + 3];
  short4 empty = make_short4(1, 1, 0, 0);
  if (!(g0.w >= 0.0f)) {
    rect[i] = empty;
    cnt[i] = 0;
    q[i] = 0;
    return;
  }
  float dx = g0.x - v.o[0], dy = g0.y - v.o[1], dz = g0.z - v.o[2];
  float dc = sqrtf(dx * dx + dy * dy + dz * dz);
  float dmin = dc - g0.w, dmax = dc + g0.w;
  // camera-frame centre and half axes
  float cc[3], ca[3], cb[3], cd[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    cc[r] = v.R[r * 3] * g0.x + v.R[r * 3 + 1] * g0.y + v.R[r * 3 + 2] * g0.z + v.t[r];
    ca[r] = v.R[r * 3] * g1.x + v.R[r * 3 + 1] * g1.y + v.R[r * 3 + 2] * g1.z;
    cb[r] = v.R[r * 3] * g2.x + v.R[r * 3 + 1] * g2.y + v.R[r * 3 + 2] * g2.z;
    cd[r] = v.R[r * 3] * g3.x + v.R[r * 3 + 1] * g3.y + v.R[r * 3 + 2] * g3.z;
  }
  float umin = 3.4e38f, umax = -3.4e38f, vmin = 3.4e38f, vmax = -3.4e38f;
  bool front = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float sa = (k & 1) ? 1.0f : -1.0f, sb = (k & 2) ? 1.0f : -1.0f, sd = (k & 4) ? 1.0f : -1.0f;
    float X = cc[0] + sa * ca[0] + sb * cb[0] + sd * cd[0];
    float Y = cc[1] + sa * ca[1] + sb * cb[1] + sd * cd[1];
    float Z = cc[2] + sa * ca[2] + sb * cb[2] + sd * cd[2];
    front = front && (Z > kZMin);
    float iz = 1.0f / Z;
    float u = v.fx * X * iz + v.cx, w = v.fy * Y * iz + v.cy;
    umin = fminf(umin, u);
    umax = fmaxf(umax, u);
    vmin = fminf(vmin, w);
    vmax = fmaxf(vmax, w);
  }
  int x0 = (int)ceilf(umin - 0.5f - kBboxPad), x1 = (int)floorf(umax - 0.5f + kBboxPad);
  int y0 = (int)ceilf(vmin - 0.5f - kBboxPad), y1 = (int)floorf(vmax - 0.5f + kBboxPad);
  x0 = max(x0, 0);
  y0 = max(y0, 0);
  x1 = min(x1, v.W - 1);
  y1 = min(y1, v.H - 1);
  if (!front || dmin > v.zfar || dmax < v.znear || x0 > x1 || y0 > y1) {
    rect[i] = empty;
    cnt[i] = 0;
    q[i] = 0;
    return;
  }
  rc = make_short4((short)x0, (short)y0, (short)x1, (short)y1);
  c = (uint32_t)(((x1 >> v.tile_wl) - (x0 >> v.tile_wl) + 1) * ((y1 >> v.tile_hl) - (y0 >> v.tile_hl) + 1));
  rect[i] = rc;
  cnt[i] = c;
  float rel = (fmaxf(dmin, v.znear) - v.znear) * v.dscale;
  float qmax = (float)((1u << v.depth_bits) - 1u);
  float qq = fminf(fmaxf(floorf(rel) - 1.0f, 0.0f), qmax);
  q[i] = (uint32_t)qq;
  if (hbin) {  // coarse check: depth bins [b0, b1] of [dmin, dmax] and the bound sigma (dmax - dmin)
    // (the range grown by kHistPad so that FP32 rounding never moves a voxel out of a bin it overlaps)
    const float bs = (float)kPropBins / (v.zfar - v.znear);
    const int b0 = min(max((int)floorf((dmin - kHistPad - v.znear) * bs), 0), kPropBins - 1);
    const int b1 = min(max((int)floorf((dmax + kHistPad - v.znear) * bs), 0), kPropBins - 1);
    hbin[i] = (uint32_t)b0 | ((uint32_t)b1 << 8);
    htau[i] = sigma[i] * (dmax - dmin) * (1.0f + kHistSlack);
  }
}

__global__ void __launch_bounds__(256) project_kernel(int64_t n, const float4* __restrict__ geo, ViewParams v,
                                                      short4* __restrict__ rect, uint32_t* __restrict__ q,
                                                      uint32_t* __restrict__ cnt, const float* __restrict__ sigma,
                                                      uint32_t* __restrict__ hbin, float* __restrict__ htau,
                                                      uint32_t* __restrict__ tcount,
                                                      unsigned long long* __restrict__ scan_state, int scan_words,
                                                      unsigned long long* __restrict__ status) {
  ART_PDL_ENTRY();
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < scan_words; k += blockDim.x) scan_state[k] = 0ull;
    if (threadIdx.x == 0) {
      status[kStScanTicket] = 0ull;
      status[kStActiveGroups] = 0ull;
    }
  }
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  short4 rc = make_short4(1, 1, 0, 0);
  uint32_t c = 0;
  if (i < n) project_voxel(i, geo, v, rect, q, cnt, sigma, hbin, htau, rc, c);
  const int lane = threadIdx.x & 31;
  const int tx0 = rc.x >> v.tile_wl, ty0 = rc.y >> v.tile_hl, w = (rc.z >> v.tile_wl) - tx0 + 1;
  const uint32_t steps = __reduce_max_sync(0xFFFFFFFFu, c);
  for (uint32_t k = 0; k < steps; ++k) {
    const uint32_t tile =
        k < c ? (uint32_t)((ty0 + (int)(k / (uint32_t)w)) * v.tiles_x + tx0 + (int)(k % (uint32_t)w)) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, tile);
    if (tile != 0xFFFFFFFFu && lane == __ffs(grp) - 1) atomicAdd(tcount + tile, (uint32_t)__popc(grp));
  }
}

}  // namespace

// ---------------------------------------------------- the lattice index
//
// The paper rebuilds an index over the warped voxels every frame (Sec. 3.1
// "Dynamic Volume Rendering") and lets voxels that land on one grid location
// collide.  Here the grid is the lattice of the canonical octree's leaves
// (origin, leaf size h): voxel i goes to the cell floor((cw_i - origin) / h)
// of its warped centre, the cells of a pose are keys of an open-addressing
// hash table (linear probing, load <= 1/2) holding the smallest voxel id
// that landed there, and that voxel survives.  Cells more than 2^20 from the
// origin along an axis are not placed.

constexpr unsigned long long kGridEmpty = ~0ull;
constexpr int kGridBits = 21;  // per axis, two's complement

__device__ __forceinline__ bool grid_cell(const float4& r0, const float4& r1, const float4& r2, float ox, float oy,
                                          float oz, float inv_h, unsigned long long& key) {
  const float c[3] = {floorf((r0.w - ox) * inv_h), floorf((r1.w - oy) * inv_h), floorf((r2.w - oz) * inv_h)};
  key = 0ull;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(fabsf(c[a]) < (float)(1 << (kGridBits - 1)))) return false;
    key |= ((unsigned long long)((int)c[a]) & ((1ull << kGridBits) - 1ull)) << (kGridBits * a);
  }
  return true;
}

__device__ __forceinline__ uint64_t grid_hash(unsigned long long key) {
  key ^= key >> 33;
  key *= 0xff51afd7ed558ccdull;
  key ^= key >> 33;
  key *= 0xc4ceb9fe1a85ec53ull;
  key ^= key >> 33;
  return key;
}

// Probe for the cell's slot; insert the key when it is absent.  Returns the
// slot, or -1 when the table is full (never with load <= 1/2).
__device__ __forceinline__ int64_t grid_slot(unsigned long long* keys, int64_t mask, unsigned long long key,
                                             bool insert) {
  int64_t s = (int64_t)(grid_hash(key) & (uint64_t)mask);
  for (int64_t probe = 0; probe <= mask; ++probe) {
    unsigned long long k = keys[s];
    if (k == key) return s;
    if (k == kGridEmpty) {
      if (!insert) return -1;
      k = atomicCAS(keys + s, kGridEmpty, key);
      if (k == kGridEmpty || k == key) return s;
    }
    s = (s + 1) & mask;
  }
  return -1;
}

__global__ void __launch_bounds__(256) grid_insert_kernel(int64_t n, const float4* __restrict__ rec, float ox, float oy,
                                                         float oz, float inv_h, unsigned long long* __restrict__ keys,
                                                         uint32_t* __restrict__ vals, int64_t mask) {
  ART_PDL_ENTRY();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4* r = rec + 4 * i;
  if (r[3].y == 0.0f) return;  // dropped (degenerate blend)
  unsigned long long key;
  if (!grid_cell(r[0], r[1], r[2], ox, oy, oz, inv_h, key)) return;
  const int64_t s = grid_slot(keys, mask, key, true);
  if (s >= 0) atomicMin(vals + s, (uint32_t)i);
}

// Survivors become their cell's axis-aligned leaf box (unit-cube map I / h,
// centre origin + (cell + 1/2) h, bounding radius sqrt(3) h / 2, half axes
// h / 2 along x, y, z); every other voxel is dropped like a degenerate one.
__global__ void __launch_bounds__(256) grid_rewrite_kernel(int64_t n, float4* __restrict__ rec, float4* __restrict__ geo,
                                                          float ox, float oy, float oz, float h,
                                                          const unsigned long long* __restrict__ keys,
                                                          const uint32_t* __restrict__ vals, int64_t mask,
                                                          unsigned long long* __restrict__ status) {
  ART_PDL_ENTRY();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool survive = false;
  if (i < n) {
    float4* r = rec + 4 * i;
    float4* g = geo + 4 * i;
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3];
    unsigned long long key;
    int64_t s = -1;
    if (r3.y != 0.0f && grid_cell(r0, r1, r2, ox, oy, oz, 1.0f / h, key))
      s = grid_slot(const_cast<unsigned long long*>(keys), mask, key, false);
    survive = s >= 0 && vals[s] == (uint32_t)i;
    if (survive) {
      const float ih = 1.0f / h, hh = 0.5f * h;
      const float cx = ox + (floorf((r0.w - ox) * ih) + 0.5f) * h;
      const float cy = oy + (floorf((r1.w - oy) * ih) + 0.5f) * h;
      const float cz = oz + (floorf((r2.w - oz) * ih) + 0.5f) * h;
      r[0] = make_float4(ih, 0.0f, 0.0f, cx);
      r[1] = make_float4(0.0f, ih, 0.0f, cy);
      r[2] = make_float4(0.0f, 0.0f, ih, cz);
      g[0] = make_float4(cx, cy, cz, 0.8660254f * h * (1.0f + 1e-6f) + 1e-9f);
      g[1] = make_float4(hh, 0.0f, 0.0f, 0.0f);
      g[2] = make_float4(0.0f, hh, 0.0f, 0.0f);
      g[3] = make_float4(0.0f, 0.0f, hh, 0.0f);
    } else if (r3.y != 0.0f) {
      r[0] = r[1] = r[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      r[3] = make_float4(r3.x, 0.0f, 0.0f, 0.0f);
      g[0] = make_float4(g[0].x, g[0].y, g[0].z, -1.0f);
    }
  }
  const unsigned cnt = __popc(__ballot_sync(0xffffffffu, survive));
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(status + kStGridCells, (unsigned long long)cnt);
}

void launch_grid_snap(art_ctx* ctx) {
  const int64_t n = ctx->n;
  const unsigned grid = (unsigned)((n + 255) / 256);
  const int64_t mask = ctx->grid_slots - 1;
  cudaMemsetAsync(ctx->d_gkeys, 0xFF, sizeof(unsigned long long) * (size_t)ctx->grid_slots, ctx->stream);
  cudaMemsetAsync(ctx->d_gvals, 0xFF, sizeof(uint32_t) * (size_t)ctx->grid_slots, ctx->stream);
  cudaMemsetAsync(ctx->d_status + kStGridCells, 0, sizeof(unsigned long long), ctx->stream);
  ART_LAUNCH_PDL(ctx, "grid_insert", grid_insert_kernel, grid, 256, 0, n, ctx->d_rec, ctx->origin[0], ctx->origin[1],
             ctx->origin[2], 1.0f / ctx->h, ctx->d_gkeys, ctx->d_gvals, mask);
  ART_LAUNCH_PDL(ctx, "grid_rewrite", grid_rewrite_kernel, grid, 256, 0, n, ctx->d_rec, ctx->d_geo, ctx->origin[0],
             ctx->origin[1], ctx->origin[2], ctx->h, ctx->d_gkeys, ctx->d_gvals, mask, ctx->d_status);
}

void launch_fk(art_ctx* ctx) {
  ART_LAUNCH_PDL(ctx, "fk", fk_kernel, 1, kMaxJoints, 0, ctx->J, ctx->d_skel, ctx->d_pose, ctx->d_G, ctx->d_status);
}

void launch_lbs(art_ctx* ctx) {
  int64_t n = ctx->n;
  unsigned grid = (unsigned)((n + 255) / 256);
  ART_LAUNCH_PDL(ctx, "lbs", lbs_kernel, grid, 256, 0, n, ctx->J, ctx->d_G, ctx->d_ijk, ctx->d_jidx, ctx->d_w,
             ctx->d_sigma, ctx->origin[0], ctx->origin[1], ctx->origin[2], ctx->h, ctx->d_rec, ctx->d_geo,
             ctx->d_status);
}

void launch_project_view(art_ctx* ctx, const ViewParams& v, short4* rect, uint32_t* q, uint32_t* cnt,
                         uint32_t* tcount, bool first) {
  const int64_t n = ctx->n;
  const unsigned grid = (unsigned)((n + 255) / 256);
  const int words = first ? (int)tile_scan_state_words(ctx->ranges_cap) : 0;
  ART_LAUNCH_PDL(ctx, "project", project_kernel, grid, 256, 0, n, ctx->d_geo, v, rect, q, cnt, ctx->d_sigma,
             (uint32_t*)nullptr, (float*)nullptr, tcount, ctx->d_scan_state, words, ctx->d_status);
}

void launch_project(art_ctx* ctx, const ViewParams& v, uint32_t* hbin, float* htau) {
  int64_t n = ctx->n;
  unsigned grid = (unsigned)((n + 255) / 256);
  const int ntiles = v.tiles_x * v.tiles_y;  // (the counts are zero: the last tile scan cleared them)
  ART_LAUNCH_PDL(ctx, "project", project_kernel, grid, 256, 0, n, ctx->d_geo, v, ctx->d_rect, ctx->d_q, ctx->d_cnt,
             ctx->d_sigma, hbin, htau, ctx->d_tcount, ctx->d_scan_state, (int)tile_scan_state_words(ntiles),
             ctx->d_status);
}

}  // namespace art
