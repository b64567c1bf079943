// Screen-tile binning of the warped voxels into (tile, depth)-ordered lists,
// and a device LSD radix sort of key/value pairs.  The per-frame binning
// plays the role of the paper's per-frame octree rebuild before the ray-voxel
// test (arXiv 2202.05628, Sec. 3.1 "Dynamic Volume Rendering").
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace art {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                       // per thread
constexpr int kScanBlock = kScanThreads * kScanItems;  // 2048
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortBlock = kSortThreads * kSortRounds;  // 4096 keys per block
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  uint32_t base = wid > 0 ? warp_sums[wid - 1] : 0u;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

// Sum of each block of kScanBlock elements.
__global__ void __launch_bounds__(kScanThreads) block_sum_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                 const unsigned long long* __restrict__ n_dev,
                                                                 uint32_t* __restrict__ bsum) {
  if (n_dev) n = (int64_t)min((unsigned long long)n, *n_dev);
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ uint32_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of nb block sums in one block of 1024 threads (nb <= 1024 *
// 16); writes the grand total to *total (64-bit) when non-null.
__global__ void __launch_bounds__(1024) scan_bsum_kernel(uint32_t* __restrict__ bsum, int nb,
                                                         unsigned long long* __restrict__ total) {
  constexpr int kPer = 16;
  __shared__ uint32_t warp_sums[32];
  uint32_t v[kPer];
  uint32_t s = 0;
  int base = threadIdx.x * kPer;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    v[k] = (base + k < nb) ? bsum[base + k] : 0u;
    s += v[k];
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  uint32_t run = (wid > 0 ? warp_sums[wid - 1] : 0u) + x - s;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (base + k < nb) bsum[base + k] = run;
    run += v[k];
  }
  if (total && threadIdx.x == 1023) *total = (unsigned long long)run;
}

// Exclusive scan of `in` into `out` given scanned block sums.
// (in and out may alias: each thread reads its own items before writing them)
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t* in, uint32_t* out, int64_t n,
                                                                  const uint32_t* __restrict__ bsum) {
  int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_exclusive_scan(s, nullptr) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

// ---------------------------------------------------------------- radix sort

// number of keys: the device count word, clamped to the capacity
__device__ __forceinline__ int64_t num_keys(const unsigned long long* st, int64_t cap) {
  unsigned long long m = *st;
  return (int64_t)(m < (unsigned long long)cap ? m : (unsigned long long)cap);
}

// Digit histogram of each 4096-key block; layout hist[digit * nb + block].
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t cap,
                                                                  const unsigned long long* __restrict__ st,
                                                                  int shift, int nb, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t n = num_keys(st, cap);
  int64_t base = (int64_t)blockIdx.x * kSortBlock;
  if (base < n) {
#pragma unroll 4
    for (int r = 0; r < kSortRounds; ++r) {
      int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
      if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of each block's keys by digit, using the scanned histogram.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t cap, const unsigned long long* __restrict__ st, int shift, int nb,
    const uint32_t* __restrict__ hist) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t run[kRadix];        // running position of each digit
  __shared__ uint32_t wh[kWarps][kRadix];  // per-warp digit counts -> offsets
  __shared__ uint32_t rt[kRadix];         // round totals
  int64_t n = num_keys(st, cap);
  int64_t base = (int64_t)blockIdx.x * kSortBlock;
  if (base >= n) return;
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  run[t] = hist[(int64_t)t * nb + blockIdx.x];
  unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
    for (int k = 0; k < kWarps; ++k) wh[k][t] = 0;
    __syncthreads();
    int64_t i = base + (int64_t)r * kSortThreads + t;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    uint32_t val = valid ? vin[i] : 0u;
    uint32_t d = valid ? ((key >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) wh[w][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t s = 0;
#pragma unroll
      for (int k = 0; k < kWarps; ++k) {
        uint32_t c = wh[k][t];
        wh[k][t] = s;
        s += c;
      }
      rt[t] = s;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = run[d] + wh[w][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    run[t] += rt[t];
  }
}

// ---------------------------------------------------- binning by tile buckets
//
// The frame's (tile, depth) order as a most-significant-digit radix sort:
// the first digit is the tile (a counting sort: count the instances of
// every tile, scan the counts into the tile ranges, scatter every instance
// into its tile's bucket), the second a depth bin within the tile (a
// counting sort in shared memory), finished by comparisons of (depth
// quantum, voxel id).  That is the order of a stable sort of the keys
// emitted in voxel order, so the result does not depend on the order in
// which the atomics land.

constexpr int kTileScanThreads = 256;
constexpr int kTileScanItems = 4;        // tiles per thread
constexpr int kTileScanBlock = kTileScanThreads * kTileScanItems;  // tiles per block
constexpr long long kScanSpin = 1 << 22;  // look-back polls before a block gives up
constexpr int kTileSortThreads = 512;
constexpr int kTileSortWarps = kTileSortThreads / 32;
constexpr int kSortPer = 16;             // bucket entries per thread held in registers
constexpr int kSortRegs = kTileSortThreads * kSortPer;  // buckets held in registers (8192)
constexpr int kTileSortSmem = kSortRegs;                 // ... and staged in shared memory (64 KB)
constexpr int kWarpSortCap = 256;        // buckets up to this size: one warp each
constexpr int kSortBins = 4096;          // depth bins of a block-sorted bucket
constexpr int kRankMax = 64;             // bins up to this size: entries ranked by counting

// The tiles x0..x1 by y0..y1 of a pixel rectangle, the k-th in row-major order.
__device__ __forceinline__ uint32_t rect_tile(const ViewParams& v, int tx0, int ty0, int w, uint32_t k) {
  return (uint32_t)((ty0 + (int)(k / (uint32_t)w)) * v.tiles_x + tx0 + (int)(k % (uint32_t)w));
}

// Single-pass tile scan with decoupled look-back.  Blocks take consecutive
// runs of kTileScanBlock tiles in the order they start (a ticket), so every
// predecessor of a block is already running.  A block publishes its totals
// (instances; list entries small | big << 31) as soon as it has them, then
// its warp 0 looks back over up to 32 predecessors per round: the nearest one
// that published its inclusive prefix ends the walk, the others contribute
// their totals.  Words carry their value shifted left by one with bit 0 set
// once written (zeroed by the projection kernel).  A poll that does not end within
// kScanSpin tries counts the block in kStScanError and reads zero.
//
// Outputs: bucket cursors and tile ranges (clamped to the capacity), the
// total into kStInstances, and the tiles whose bucket needs sorting: those of
// 2..kWarpSortCap instances from the front of sort_list, longer ones from its
// end (kStSortTiles and kStSortBig of them, written by the last block, which
// also resets both work counters).  The counts it reads are zeroed for the
// next projection, and with thist the 64 depth bins of every tile with
// instances are zeroed for the scatter that adds into them (rows of tiles
// without instances are not read).
struct ScanWords {  // per block: aggregate and inclusive prefix, each (instances, lists)
  unsigned long long agg_i, agg_l, inc_i, inc_l;
};

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long x) {
  *reinterpret_cast<volatile unsigned long long*>(p) = x;
}

__global__ void __launch_bounds__(kTileScanThreads) tile_scan_kernel(int ntiles, uint32_t* __restrict__ tcount,
                                                                     int64_t cap, uint32_t* __restrict__ toff,
                                                                     uint2* __restrict__ ranges,
                                                                     uint32_t* __restrict__ sort_list,
                                                                     ScanWords* __restrict__ sw,
                                                                     uint32_t* __restrict__ agroups,
                                                                     unsigned long long* __restrict__ status,
                                                                     float* __restrict__ thist) {
  ART_PDL_ENTRY();
  __shared__ unsigned long long s_b, s_pi, s_pl;
  if (threadIdx.x == 0) s_b = atomicAdd(status + kStScanTicket, 1ull);
  __syncthreads();
  const int b = (int)s_b;
  const int nblocks = (ntiles + kTileScanBlock - 1) / kTileScanBlock;
  const int base = b * kTileScanBlock + (int)threadIdx.x * kTileScanItems;
  uint32_t c[kTileScanItems];
  if (base + kTileScanItems <= ntiles) {
    const uint4 x = *reinterpret_cast<const uint4*>(tcount + base);
    c[0] = x.x;
    c[1] = x.y;
    c[2] = x.z;
    c[3] = x.w;
  } else {
#pragma unroll
    for (int k = 0; k < kTileScanItems; ++k) c[k] = base + k < ntiles ? tcount[base + k] : 0u;
  }
  // the counts are read: zero them for the next projection, and the depth
  // histograms of the tiles that will receive instances for this scatter
#pragma unroll
  for (int k = 0; k < kTileScanItems; ++k) {
    if (base + k < ntiles && c[k]) {
      tcount[base + k] = 0u;
      if (thist) {
        float4* row = reinterpret_cast<float4*>(thist + (size_t)(base + k) * kPropBins);
#pragma unroll
        for (int j = 0; j < kPropBins / 4; ++j) row[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  uint32_t s = 0, lists = 0;  // lists: small | big << 16 (per block < 2^16 each)
#pragma unroll
  for (int k = 0; k < kTileScanItems; ++k) {
    s += c[k];
    lists += c[k] > (uint32_t)kWarpSortCap ? 0x10000u : (c[k] > 1u ? 1u : 0u);
  }
  {  // this thread's four tiles are one group: listed when any has instances
    static_assert(kTileScanItems == 4, "one group of four tiles per thread");
    const bool act = s > 0;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    unsigned long long g0 = 0;
    if ((threadIdx.x & 31) == 0 && am) g0 = atomicAdd(status + kStActiveGroups, (unsigned long long)__popc(am));
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    if (act) agroups[g0 + __popc(am & ((1u << (threadIdx.x & 31)) - 1u))] = (uint32_t)(base / 4);
  }
  uint32_t tot = 0, lt = 0;
  const uint32_t ps = block_exclusive_scan(s, &tot);
  const uint32_t lp = block_exclusive_scan(lists, &lt);
  const unsigned long long agg_l = (unsigned long long)(lt & 0xFFFFu) | ((unsigned long long)(lt >> 16) << 31);
  if (threadIdx.x == 0) {
    if (b == 0) {
      st_volatile(&sw[0].inc_i, ((unsigned long long)tot << 1) | 1ull);
      st_volatile(&sw[0].inc_l, (agg_l << 1) | 1ull);
    } else {
      st_volatile(&sw[b].agg_i, ((unsigned long long)tot << 1) | 1ull);
      st_volatile(&sw[b].agg_l, (agg_l << 1) | 1ull);
    }
  }
  if (threadIdx.x < 32) {  // look back
    const int lane = threadIdx.x;
    unsigned long long pi = 0, pl = 0;
    for (int p = b - 1; p >= 0; p -= 32) {
      const int q = p - lane;
      unsigned long long vi = 0, vl = 0;
      bool inc = q < 0;
      if (q >= 0) {
        long long spin = 0;
        for (;;) {
          const unsigned long long ii = ld_volatile(&sw[q].inc_i), il = ld_volatile(&sw[q].inc_l);
          if ((ii & 1ull) && (il & 1ull)) {
            vi = ii >> 1;
            vl = il >> 1;
            inc = true;
            break;
          }
          const unsigned long long ai = ld_volatile(&sw[q].agg_i), al = ld_volatile(&sw[q].agg_l);
          if ((ai & 1ull) && (al & 1ull)) {
            vi = ai >> 1;
            vl = al >> 1;
            break;
          }
          if (++spin > kScanSpin) {
            atomicAdd(status + kStScanError, 1ull);
            break;
          }
          __nanosleep(64);
        }
      }
      const unsigned incm = __ballot_sync(0xffffffffu, inc);
      const int stop = incm ? __ffs(incm) - 1 : 32;  // nearest predecessor with its inclusive prefix
      if (lane > stop) {
        vi = 0;
        vl = 0;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
        vl += __shfl_xor_sync(0xffffffffu, vl, o);
      }
      pi += vi;
      pl += vl;
      if (stop < 32) break;
    }
    if (lane == 0) {
      s_pi = pi;
      s_pl = pl;
      if (b > 0) {
        st_volatile(&sw[b].inc_i, ((pi + tot) << 1) | 1ull);
        st_volatile(&sw[b].inc_l, ((pl + agg_l) << 1) | 1ull);
      }
    }
  }
  __syncthreads();
  const unsigned long long pi = s_pi, pl = s_pl;
  uint64_t off = pi + ps;
  uint32_t nsm = (uint32_t)(pl & 0x7FFFFFFFull) + (lp & 0xFFFFu), nbg = (uint32_t)(pl >> 31) + (lp >> 16);
  uint32_t a4[kTileScanItems];
  uint2 r4[kTileScanItems];
#pragma unroll
  for (int k = 0; k < kTileScanItems; ++k) {
    const uint64_t a = min(off, (uint64_t)cap), e = min(off + c[k], (uint64_t)cap);
    a4[k] = (uint32_t)a;
    r4[k] = make_uint2((uint32_t)a, (uint32_t)e);
    if (c[k] > (uint32_t)kWarpSortCap)
      sort_list[ntiles - 1 - (int)nbg++] = (uint32_t)(base + k);
    else if (c[k] > 1u)
      sort_list[nsm++] = (uint32_t)(base + k);
    off += c[k];
  }
  if (base + kTileScanItems <= ntiles) {
    *reinterpret_cast<uint4*>(toff + base) = make_uint4(a4[0], a4[1], a4[2], a4[3]);
    *reinterpret_cast<uint4*>(ranges + base) = make_uint4(r4[0].x, r4[0].y, r4[1].x, r4[1].y);
    *reinterpret_cast<uint4*>(ranges + base + 2) = make_uint4(r4[2].x, r4[2].y, r4[3].x, r4[3].y);
  } else {
#pragma unroll
    for (int k = 0; k < kTileScanItems; ++k)
      if (base + k < ntiles) {
        toff[base + k] = a4[k];
        ranges[base + k] = r4[k];
      }
  }
  if (b == nblocks - 1 && threadIdx.x == 0) {
    status[kStInstances] = pi + tot;
    status[kStSortTiles] = (pl & 0x7FFFFFFFull) + (lt & 0xFFFFu);
    status[kStSortBig] = (pl >> 31) + (lt >> 16);
    status[kStSortNext] = 0;
    status[kStSortBigNext] = 0;
  }
}

// Per voxel: its instances, each at the next free place of its tile's bucket
// (toff: the buckets' starts on entry, their ends on exit); and with thist,
// the coarse optical-depth bound of every instance in its tile's depth bins.
// Lanes of a warp that hit the same tile in the same step take one atomic.
__global__ void __launch_bounds__(256) bucket_emit_kernel(int64_t n, const uint32_t* __restrict__ cnt,
                                                          const short4* __restrict__ rect,
                                                          const uint32_t* __restrict__ q, ViewParams v, int64_t cap,
                                                          uint32_t tile_base,
                                                          uint32_t* __restrict__ toff, uint32_t* __restrict__ keys,
                                                          uint32_t* __restrict__ vals,
                                                          unsigned long long* __restrict__ status,
                                                          const uint32_t* __restrict__ hbin,
                                                          const float* __restrict__ htau, float* __restrict__ thist) {
  ART_PDL_ENTRY();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t c = 0, qq = 0;
  int tx0 = 0, ty0 = 0, w = 1, hb0 = 1, hb1 = 0;
  float ht = 0.0f;
  if (i < n && (c = cnt[i]) != 0) {
    const short4 r = rect[i];
    tx0 = r.x >> v.tile_wl;
    ty0 = r.y >> v.tile_hl;
    w = (r.z >> v.tile_wl) - tx0 + 1;
    qq = q[i];
    if (thist) {
      const uint32_t hb = hbin[i];
      hb0 = (int)(hb & 0xFFu);
      hb1 = (int)(hb >> 8);
      ht = htau[i];
    }
  }
  uint32_t over = 0;
  const uint32_t steps = __reduce_max_sync(0xFFFFFFFFu, c);
  for (uint32_t k = 0; k < steps; ++k) {
    const uint32_t tile = k < c ? tile_base + rect_tile(v, tx0, ty0, w, k) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, tile);
    const int leader = __ffs(grp) - 1;
    uint32_t pos = 0;
    if (tile != 0xFFFFFFFFu && lane == leader) pos = atomicAdd(toff + tile, (uint32_t)__popc(grp));
    pos = __shfl_sync(0xFFFFFFFFu, pos, leader) + (uint32_t)__popc(grp & ((1u << lane) - 1u));
    const unsigned valid = __ballot_sync(0xFFFFFFFFu, tile != 0xFFFFFFFFu);
    if (tile == 0xFFFFFFFFu) continue;
    if (pos < (uint64_t)cap) {
      keys[pos] = (tile << v.depth_bits) | qq;
      vals[pos] = (uint32_t)i;
    } else {
      ++over;
    }
    if (thist) {
      // a voxel almost always spans one depth bin: lanes adding to the same
      // (tile, bin) sum their bounds first and one of them adds the sum
      const uint32_t hk = hb0 == hb1 ? tile * kPropBins + (uint32_t)hb0 : 0xFFFFFFFFu - (uint32_t)lane;
      const unsigned g2 = __match_any_sync(valid, hk);
      if (hb0 == hb1) {
        float sum = 0.0f;
        for (unsigned m = g2; m; m &= m - 1) sum += __shfl_sync(g2, ht, __ffs(m) - 1);
        if (lane == __ffs(g2) - 1) atomicAdd(thist + hk, sum);
      } else {
        for (int b = hb0; b <= hb1; ++b) atomicAdd(thist + (size_t)tile * kPropBins + b, ht);
      }
    }
  }
  if (over) atomicAdd(status + kStOverflowInst, (unsigned long long)over);
}

// Bitonic sorting network with every comparator ascending (the first step of
// each merge compares mirrored positions): entries at positions >= n act as
// +infinity and are never touched, so any n works.  Lanes t0, t0 + 32, ...
// of one warp share the comparators of s[0, n).
__device__ void warp_bitonic(unsigned long long* s, uint32_t n, uint32_t t0) {
  uint32_t P = 1;
  while (P < n) P <<= 1;
  for (uint32_t k = 2; k <= P; k <<= 1) {
    const uint32_t half = k >> 1;
    for (uint32_t i = t0; i < P / 2; i += 32) {  // merge: mirrored pairs
      const uint32_t a = (i / half) * k + i % half, b = (i / half) * k + k - 1 - i % half;
      if (b < n) {
        const unsigned long long x = s[a], y = s[b];
        if (y < x) {
          s[a] = y;
          s[b] = x;
        }
      }
    }
    __syncwarp();
    for (uint32_t j = k >> 2; j > 0; j >>= 1) {  // half-cleaners
      for (uint32_t i = t0; i < P / 2; i += 32) {
        const uint32_t a = (i / j) * 2 * j + i % j, b = a + j;
        if (b < n) {
          const unsigned long long x = s[a], y = s[b];
          if (y < x) {
            s[a] = y;
            s[b] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ unsigned long long bucket_entry(uint32_t key, uint32_t val, uint32_t qmask) {
  return ((unsigned long long)(key & qmask) << 32) | val;
}

// Block-wide sort of one bucket of n >= 2 entries (keys, vals: the bucket)
// by (depth quantum, voxel id) through the staging array S (shared memory
// for n <= kTileSortSmem, else the bucket's own stretch of a global scratch;
// the entries are held in registers for n <= kSortRegs).  A counting sort on the depth
// bin (q - lo) >> shift, with kSortBins bins over the bucket's quanta
// [lo, hi], stages the entries bin by bin; an entry of a bin of up to
// kRankMax entries then goes straight to its place, the number of smaller
// (quantum, voxel id) pairs in its bin; larger bins are sorted by one warp.
__device__ void block_sort_bucket(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t n,
                                  uint32_t qmask, uint32_t thi, unsigned long long* S) {
  __shared__ uint32_t s_start[kSortBins], s_cur[kSortBins];
  __shared__ uint32_t s_lo[kTileSortWarps], s_hi[kTileSortWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool regs = n <= (uint32_t)kSortRegs;
  uint32_t kq[kSortPer], kv[kSortPer];
  uint32_t lo = 0xFFFFFFFFu, hi = 0;
  if (regs) {
#pragma unroll
    for (int e = 0; e < kSortPer; ++e) {
      const uint32_t k = (uint32_t)e * kTileSortThreads + threadIdx.x;
      kq[e] = 0;
      kv[e] = 0;
      if (k < n) {
        kq[e] = keys[k] & qmask;
        kv[e] = vals[k];
        lo = min(lo, kq[e]);
        hi = max(hi, kq[e]);
      }
    }
  } else {
    for (uint32_t k = threadIdx.x; k < n; k += kTileSortThreads) {
      const uint32_t q = keys[k] & qmask;
      lo = min(lo, q);
      hi = max(hi, q);
    }
  }
  lo = __reduce_min_sync(0xFFFFFFFFu, lo);
  hi = __reduce_max_sync(0xFFFFFFFFu, hi);
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  for (int b = threadIdx.x; b < kSortBins; b += kTileSortThreads) s_cur[b] = 0;
  __syncthreads();
  lo = s_lo[0];
  hi = s_hi[0];
#pragma unroll
  for (int w = 1; w < kTileSortWarps; ++w) {
    lo = min(lo, s_lo[w]);
    hi = max(hi, s_hi[w]);
  }
  uint32_t shift = 0;
  while (((hi - lo) >> shift) >= (uint32_t)kSortBins) ++shift;
  // histogram of the bins
  if (regs) {
#pragma unroll
    for (int e = 0; e < kSortPer; ++e)
      if ((uint32_t)e * kTileSortThreads + threadIdx.x < n) atomicAdd(&s_cur[(kq[e] - lo) >> shift], 1u);
  } else {
    for (uint32_t k = threadIdx.x; k < n; k += kTileSortThreads)
      atomicAdd(&s_cur[((keys[k] & qmask) - lo) >> shift], 1u);
  }
  __syncthreads();
  {  // exclusive scan of the bin counts
    constexpr int kPer = kSortBins / kTileSortThreads;
    uint32_t c[kPer], t = 0;
    const int b0 = threadIdx.x * kPer;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      c[e] = s_cur[b0 + e];
      t += c[e];
    }
    uint32_t run = block_exclusive_scan(t, nullptr);
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      s_start[b0 + e] = run;
      s_cur[b0 + e] = run;
      run += c[e];
    }
  }
  __syncthreads();
  // stage bin by bin (s_cur: each bin's end afterwards)
  if (regs) {
#pragma unroll
    for (int e = 0; e < kSortPer; ++e)
      if ((uint32_t)e * kTileSortThreads + threadIdx.x < n)
        S[atomicAdd(&s_cur[(kq[e] - lo) >> shift], 1u)] = ((unsigned long long)kq[e] << 32) | kv[e];
  } else {
    for (uint32_t k = threadIdx.x; k < n; k += kTileSortThreads) {
      const uint32_t key = keys[k];
      S[atomicAdd(&s_cur[((key & qmask) - lo) >> shift], 1u)] = bucket_entry(key, vals[k], qmask);
    }
  }
  __syncthreads();
  // entries of small bins: rank within the bin
  for (uint32_t p = threadIdx.x; p < n; p += kTileSortThreads) {
    const unsigned long long x = S[p];
    const uint32_t q = (uint32_t)(x >> 32), b = (q - lo) >> shift;
    const uint32_t a = s_start[b], m = s_cur[b] - a;
    if (m > (uint32_t)kRankMax) continue;
    uint32_t r = 0;
    for (uint32_t j = 0; j < m; ++j) r += S[a + j] < x ? 1u : 0u;
    keys[a + r] = thi | q;
    vals[a + r] = (uint32_t)x;
  }
  // large bins: one warp each
  for (int b0 = warp * 32; b0 < kSortBins; b0 += kTileSortThreads) {
    unsigned big = __ballot_sync(0xFFFFFFFFu, s_cur[b0 + lane] - s_start[b0 + lane] > (uint32_t)kRankMax);
    while (big) {
      const int b = b0 + __ffs(big) - 1;
      big &= big - 1;
      const uint32_t a = s_start[b], m = s_cur[b] - a;
      warp_bitonic(S + a, m, lane);
      for (uint32_t k = lane; k < m; k += 32) {
        const unsigned long long x = S[a + k];
        keys[a + k] = thi | (uint32_t)(x >> 32);
        vals[a + k] = (uint32_t)x;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// Sort each listed tile's bucket by (depth quantum, voxel id).  Persistent
// blocks take the buckets of more than kWarpSortCap entries first, one block
// each, then the others, one warp each.
__global__ void __launch_bounds__(kTileSortThreads) tile_sort_kernel(const uint2* __restrict__ ranges,
                                                                     const uint32_t* __restrict__ sort_list,
                                                                     int ntiles, int depth_bits,
                                                                     uint32_t* __restrict__ keys,
                                                                     uint32_t* __restrict__ vals,
                                                                     unsigned long long* __restrict__ scratch,
                                                                     unsigned long long* __restrict__ status) {
  ART_PDL_ENTRY();
  extern __shared__ unsigned long long sk[];
  __shared__ unsigned long long s_item;
  const uint32_t qmask = (1u << depth_bits) - 1u;
  const unsigned long long n_big = status[kStSortBig], n_small = status[kStSortTiles];
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(status + kStSortBigNext, 1ull);
    __syncthreads();
    const unsigned long long it = s_item;
    __syncthreads();
    if (it >= n_big) break;
    const uint32_t tile = sort_list[ntiles - 1 - (int)it];
    const uint2 rg = ranges[tile];
    const uint32_t n = rg.y - rg.x;
    if (n > 1)
      block_sort_bucket(keys + rg.x, vals + rg.x, n, qmask, tile << depth_bits,
                        n <= (uint32_t)kTileSortSmem ? sk : scratch + rg.x);
  }
  const uint32_t lane = threadIdx.x & 31u;
  unsigned long long* ws = sk + (threadIdx.x >> 5) * kWarpSortCap;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(status + kStSortNext, 1ull);
    it = __shfl_sync(0xFFFFFFFFu, it, 0);
    if (it >= n_small) break;
    const uint32_t tile = sort_list[it];
    const uint2 rg = ranges[tile];
    const uint32_t n = rg.y - rg.x;
    uint32_t* kp = keys + rg.x;
    uint32_t* vp = vals + rg.x;
    for (uint32_t k = lane; k < n; k += 32) ws[k] = bucket_entry(kp[k], vp[k], qmask);
    __syncwarp();
    warp_bitonic(ws, n, lane);
    for (uint32_t k = lane; k < n; k += 32) {
      kp[k] = (tile << depth_bits) | (uint32_t)(ws[k] >> 32);
      vp[k] = (uint32_t)ws[k];
    }
    __syncwarp();
  }
}

}  // namespace

size_t scan_block_words(int64_t n) { return (size_t)((n + kScanBlock - 1) / kScanBlock) + 1; }

size_t tile_scan_state_words(int64_t ntiles) { return 4 * (size_t)((ntiles + kTileScanBlock - 1) / kTileScanBlock); }

size_t sort_hist_words(int64_t inst_cap) {
  int64_t nb = (inst_cap + kSortBlock - 1) / kSortBlock;
  return (size_t)(nb * kRadix);
}

void launch_bin(art_ctx* ctx, const ViewParams& v, const uint32_t* hbin, const float* htau, float* thist, bool sort) {
  const int64_t n = ctx->n;
  const int ntiles = v.tiles_x * v.tiles_y;
  const unsigned vb = (unsigned)((n + 255) / 256);
  if (!ctx->attr_tile_sort) {  // (a function attribute holds per device: set once per context)
    cudaFuncSetAttribute(tile_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSortSmem * 8);
    ctx->attr_tile_sort = true;
  }
  const int nsb = (ntiles + kTileScanBlock - 1) / kTileScanBlock;
  ART_LAUNCH_PDL(ctx, "bin_scan", tile_scan_kernel, nsb, kTileScanThreads, 0, ntiles, ctx->d_tcount, ctx->inst_cap,
             ctx->d_toff, ctx->d_ranges, ctx->d_sortlist, reinterpret_cast<ScanWords*>(ctx->d_scan_state),
             ctx->d_agroups, ctx->d_status, thist);
  ART_LAUNCH_PDL(ctx, "bin_emit", bucket_emit_kernel, vb, 256, 0, n, ctx->d_cnt, ctx->d_rect, ctx->d_q, v, ctx->inst_cap,
             0u, ctx->d_toff, ctx->d_keys, ctx->d_vals, ctx->d_status, hbin, htau, thist);
  if (sort) launch_tile_sort(ctx, v);
}

void launch_tile_sort(art_ctx* ctx, const ViewParams& v) {
  const int ntiles = v.tiles_x * v.tiles_y;
  ART_LAUNCH_PDL(ctx, "tile_sort", tile_sort_kernel, 2 * ctx->num_sms, kTileSortThreads, kTileSortSmem * 8, ctx->d_ranges,
             ctx->d_sortlist, ntiles, v.depth_bits, ctx->d_keys, ctx->d_vals, ctx->d_sort_tmp, ctx->d_status);
}

void launch_bin_views(art_ctx* ctx, const ViewSet& vs, int64_t ntiles) {
  const int64_t n = ctx->n;
  const unsigned vb = (unsigned)((n + 255) / 256);
  if (!ctx->attr_tile_sort) {
    cudaFuncSetAttribute(tile_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSortSmem * 8);
    ctx->attr_tile_sort = true;
  }
  const int nt = (int)ntiles;
  const int nsb = (nt + kTileScanBlock - 1) / kTileScanBlock;
  ART_LAUNCH_PDL(ctx, "bin_scan", tile_scan_kernel, nsb, kTileScanThreads, 0, nt, ctx->d_tcount, ctx->inst_cap,
             ctx->d_toff, ctx->d_ranges, ctx->d_sortlist, reinterpret_cast<ScanWords*>(ctx->d_scan_state),
             ctx->d_agroups, ctx->d_status, (float*)nullptr);
  for (int k = 0; k < vs.nv; ++k) {
    const int64_t o = (int64_t)k * vs.rect_stride;
    ART_LAUNCH_PDL(ctx, "bin_emit", bucket_emit_kernel, vb, 256, 0, n, ctx->d_cnt_v + o, ctx->d_rect_v + o,
               ctx->d_q_v + o, vs.v[k], ctx->inst_cap, vs.toff[k], ctx->d_toff, ctx->d_keys, ctx->d_vals,
               ctx->d_status, (const uint32_t*)nullptr, (const float*)nullptr, (float*)nullptr);
  }
  ART_LAUNCH_PDL(ctx, "tile_sort", tile_sort_kernel, 2 * ctx->num_sms, kTileSortThreads, kTileSortSmem * 8, ctx->d_ranges,
             ctx->d_sortlist, nt, vs.v[0].depth_bits, ctx->d_keys, ctx->d_vals, ctx->d_sort_tmp, ctx->d_status);
}

int launch_sort_bufs(art_ctx* ctx, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t cap,
                     const unsigned long long* count, int key_bits, uint32_t* hist, uint32_t* bsum) {
  int nb = (int)((cap + kSortBlock - 1) / kSortBlock);
  if (nb < 1) nb = 1;
  int64_t hn = (int64_t)nb * kRadix;
  int hb = (int)((hn + kScanBlock - 1) / kScanBlock);
  uint32_t* K[2] = {k0, k1};
  uint32_t* V[2] = {v0, v1};
  int src = 0;
  for (int shift = 0; shift < key_bits; shift += kRadixBits) {
    ART_LAUNCH(ctx, "sort_hist", radix_hist_kernel, nb, kSortThreads, 0, K[src], cap, count, shift, nb, hist);
    ART_LAUNCH(ctx, "sort_blocksum", block_sum_kernel, hb, kScanThreads, 0, hist, hn,
               (const unsigned long long*)nullptr, bsum);
    ART_LAUNCH(ctx, "sort_scan", scan_bsum_kernel, 1, 1024, 0, bsum, hb, (unsigned long long*)nullptr);
    ART_LAUNCH(ctx, "sort_scanapply", scan_apply_kernel, hb, kScanThreads, 0, hist, hist, hn, bsum);
    ART_LAUNCH(ctx, "sort_scatter", radix_scatter_kernel, nb, kSortThreads, 0, K[src], V[src], K[src ^ 1],
               V[src ^ 1], cap, count, shift, nb, hist);
    src ^= 1;
  }
  return src;
}

namespace {
__global__ void set_word_kernel(unsigned long long* p, unsigned long long value) { *p = value; }
}  // namespace

void launch_set_word(art_ctx* ctx, unsigned long long* p, unsigned long long value) {
  ART_LAUNCH(ctx, "set_word", set_word_kernel, 1, 1, 0, p, value);
}

// ------------------------------------------------ sort without allocation
//
// art_sort_pairs_static keeps all of its scratch in the fixed device array
// below instead of memory it allocates: the ping-pong copy of the pairs, the
// digit histograms, the scan block sums and the key count.  Every kernel of a
// call rewrites the parts it reads, so nothing carries over from an earlier
// call and nothing needs clearing.  Calls that overlap on the GPU share the
// array and race.

namespace {

constexpr int64_t kStaticPairs = ART_SORT_STATIC_MAX_PAIRS;
constexpr int64_t kStaticBlocks = (kStaticPairs + kSortBlock - 1) / kSortBlock;
constexpr int64_t kStaticHist = kStaticBlocks * kRadix;
constexpr int64_t kStaticBsum = (kStaticHist + kScanBlock - 1) / kScanBlock + 1;
// byte offsets inside the array (each 256-byte aligned)
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + 4 * (size_t)kStaticPairs;
constexpr size_t kOffHist = kOffVals + 4 * (size_t)kStaticPairs;
constexpr size_t kOffBsum = kOffHist + 4 * (size_t)kStaticHist;
constexpr size_t kOffCount = (kOffBsum + 4 * (size_t)kStaticBsum + 255) & ~(size_t)255;
constexpr size_t kStaticBytes = kOffCount + 256;
constexpr int kMaxDevices = 64;

}  // namespace

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

namespace {

std::mutex g_scratch_mu;
struct ScratchAddr {
  unsigned long long ctx_id;  // the context the address belongs to (unique per process, never reused)
  void* addr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device.  In host code the
// symbol itself is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress, once per device and context: after a
// cudaDeviceReset the device gets a new primary context (a new id), and the
// next call looks the address up again.
cudaError_t static_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaError_t e = cudaFree(nullptr);  // makes the device's primary context current (frees nothing)
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  // the driver's context calls, found through the runtime (the library does
  // not link the driver library, so that it loads on machines without one)
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 4000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      get_current = nullptr;
      get_id = nullptr;
      return cudaErrorNotSupported;
    }
  }
  CUcontext cu = nullptr;
  unsigned long long id = 0;
  if (get_current(&cu) != CUDA_SUCCESS || !cu || get_id(cu, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (!g_scratch_addr[dev].addr || g_scratch_addr[dev].ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ScratchAddr{id, p};
  }
  *out = g_scratch_addr[dev].addr;
  return cudaSuccess;
}

// keys / vals must be device (or managed) memory of the device the scratch
// belongs to.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // the query's own error on a pointer CUDA does not know
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

}  // namespace art

extern "C" art_status art_sort_pairs_static(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                            void* cuda_stream) {
  using namespace art;
  if (n < 0 || n > kStaticPairs) return ART_ERR_INVALID_ARG;
  if (key_bits != 8 && key_bits != 16 && key_bits != 24 && key_bits != 32) return ART_ERR_INVALID_ARG;
  if (n == 0) return ART_OK;
  if (!keys || !vals) return ART_ERR_INVALID_ARG;
  // an error left pending by an earlier, unrelated call is neither cleared
  // nor reported as this call's: the call refuses to run instead
  if (cudaPeekAtLastError() != cudaSuccess) return ART_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ART_ERR_CUDA;
  if (!on_device(keys, dev) || !on_device(vals, dev)) return ART_ERR_INVALID_ARG;
  void* base = nullptr;
  if (static_scratch(dev, &base) != cudaSuccess) {
    cudaGetLastError();
    return ART_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char* b = (unsigned char*)base;
  uint32_t* sk = (uint32_t*)(b + kOffKeys);
  uint32_t* sv = (uint32_t*)(b + kOffVals);
  uint32_t* hist = (uint32_t*)(b + kOffHist);
  uint32_t* bsum = (uint32_t*)(b + kOffBsum);
  unsigned long long* count = (unsigned long long*)(b + kOffCount);
  const int nb = (int)((n + kSortBlock - 1) / kSortBlock);
  const int64_t hn = (int64_t)nb * kRadix;
  const int hb = (int)((hn + kScanBlock - 1) / kScanBlock);
  uint32_t* K[2] = {keys, sk};
  uint32_t* V[2] = {vals, sv};
  set_word_kernel<<<1, 1, 0, s>>>(count, (unsigned long long)n);
  if (cudaPeekAtLastError() != cudaSuccess) return (cudaGetLastError(), ART_ERR_CUDA);
  int src = 0;
  for (int shift = 0; shift < key_bits; shift += kRadixBits) {
    radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(K[src], n, count, shift, nb, hist);
    block_sum_kernel<<<hb, kScanThreads, 0, s>>>(hist, hn, nullptr, bsum);
    scan_bsum_kernel<<<1, 1024, 0, s>>>(bsum, hb, nullptr);
    scan_apply_kernel<<<hb, kScanThreads, 0, s>>>(hist, hist, hn, bsum);
    radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(K[src], V[src], K[src ^ 1], V[src ^ 1], n, count, shift, nb,
                                                     hist);
    if (cudaPeekAtLastError() != cudaSuccess) return (cudaGetLastError(), ART_ERR_CUDA);
    src ^= 1;
  }
  if (src == 1) {
    if (cudaMemcpyAsync(keys, sk, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(vals, sv, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return (cudaGetLastError(), ART_ERR_CUDA);
  }
  return ART_OK;
}
