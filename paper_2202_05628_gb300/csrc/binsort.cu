// Screen-tile binning of the warped voxels and a device LSD radix sort of the
// (tile, depth) keys.  This per-frame indexing step plays the role of the
// paper's per-frame octree rebuild before the ray-voxel test (arXiv
// 2202.05628, Sec. 3.1 "Dynamic Volume Rendering").
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

// Scan the per-voxel tile counts and emit (key, voxel) instances:
// key = tile << depth_bits | depth quantum.
__global__ void __launch_bounds__(kScanThreads) emit_kernel(int64_t n, const uint32_t* __restrict__ cnt,
                                                            const uint32_t* __restrict__ bsum,
                                                            const short4* __restrict__ rect,
                                                            const uint32_t* __restrict__ q, ViewParams v,
                                                            int64_t cap, uint32_t* __restrict__ keys,
                                                            uint32_t* __restrict__ vals,
                                                            unsigned long long* __restrict__ status,
                                                            const uint32_t* __restrict__ hbin,
                                                            const float* __restrict__ htau,
                                                            float* __restrict__ thist) {
  int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  uint32_t c[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    c[k] = (base + k < n) ? cnt[base + k] : 0u;
    s += c[k];
  }
  uint64_t off = (uint64_t)block_exclusive_scan(s, nullptr) + bsum[blockIdx.x];
  uint32_t over = 0;
  for (int k = 0; k < kScanItems; ++k) {
    if (c[k] == 0) continue;
    int64_t i = base + k;
    short4 r = rect[i];
    uint32_t qq = q[i];
    int tx0 = r.x >> v.tile_wl, tx1 = r.z >> v.tile_wl, ty0 = r.y >> v.tile_hl, ty1 = r.w >> v.tile_hl;
    int hb0 = 1, hb1 = 0;
    float ht = 0.0f;
    if (thist) {
      const uint32_t hb = hbin[i];
      hb0 = (int)(hb & 0xFFu);
      hb1 = (int)(hb >> 8);
      ht = htau[i];
    }
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        uint32_t tile = (uint32_t)(ty * v.tiles_x + tx);
        if (off < (uint64_t)cap) {
          keys[off] = (tile << v.depth_bits) | qq;
          vals[off] = (uint32_t)i;
        } else {
          ++over;
        }
        ++off;
        for (int b = hb0; b <= hb1; ++b) atomicAdd(thist + (size_t)tile * kPropBins + b, ht);
      }
  }
  if (over) atomicAdd(status + kStOverflowInst, (unsigned long long)over);
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

// Tile ranges [start, end) in the sorted instance list.
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, int64_t cap, const unsigned long long* __restrict__ st,
                              int depth_bits, uint2* __restrict__ ranges) {
  int64_t n = num_keys(st, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t tile = keys[i] >> depth_bits;
    if (i == 0 || (keys[i - 1] >> depth_bits) != tile) ranges[tile].x = (uint32_t)i;
    if (i == n - 1 || (keys[i + 1] >> depth_bits) != tile) ranges[tile].y = (uint32_t)(i + 1);
  }
}

}  // namespace

size_t scan_block_words(int64_t n) { return (size_t)((n + kScanBlock - 1) / kScanBlock) + 1; }

size_t sort_hist_words(int64_t inst_cap) {
  int64_t nb = (inst_cap + kSortBlock - 1) / kSortBlock;
  return (size_t)(nb * kRadix);
}

void launch_scan_emit(art_ctx* ctx, const ViewParams& v, const uint32_t* hbin, const float* htau, float* thist) {
  int64_t n = ctx->n;
  int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  ART_LAUNCH(ctx, "bin_blocksum", block_sum_kernel, nb, kScanThreads, 0, ctx->d_cnt, n,
             (const unsigned long long*)nullptr, ctx->d_bsum);
  ART_LAUNCH(ctx, "bin_scan", scan_bsum_kernel, 1, 1024, 0, ctx->d_bsum, nb, ctx->d_status + kStInstances);
  ART_LAUNCH(ctx, "bin_emit", emit_kernel, nb, kScanThreads, 0, n, ctx->d_cnt, ctx->d_bsum, ctx->d_rect, ctx->d_q, v,
             ctx->inst_cap, ctx->d_keys[0], ctx->d_vals[0], ctx->d_status, hbin, htau, thist);
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

void launch_sort(art_ctx* ctx, int key_bits) {
  launch_sort_bufs(ctx, ctx->d_keys[0], ctx->d_vals[0], ctx->d_keys[1], ctx->d_vals[1], ctx->inst_cap,
                   ctx->d_status + kStInstances, key_bits, ctx->d_hist, ctx->d_bsum);
}

namespace {
__global__ void set_word_kernel(unsigned long long* p, unsigned long long value) { *p = value; }
}  // namespace

void launch_set_word(art_ctx* ctx, unsigned long long* p, unsigned long long value) {
  ART_LAUNCH(ctx, "set_word", set_word_kernel, 1, 1, 0, p, value);
}

void launch_ranges(art_ctx* ctx, const ViewParams& v) {
  int64_t ntiles = (int64_t)v.tiles_x * v.tiles_y;
  cudaMemsetAsync(ctx->d_ranges, 0, sizeof(uint2) * (size_t)ntiles, ctx->stream);
  int grid = ctx->num_sms * 4;
  ART_LAUNCH(ctx, "tile_ranges", ranges_kernel, grid, 256, 0, ctx->d_keys[0], ctx->inst_cap,
             ctx->d_status + kStInstances, v.depth_bits, ctx->d_ranges);
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
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once per
// device; in host code the symbol itself is only a host-side stand-in).
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
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
  void* base = nullptr;
  if (static_scratch(&base) != cudaSuccess) {
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
  int src = 0;
  for (int shift = 0; shift < key_bits; shift += kRadixBits) {
    radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(K[src], n, count, shift, nb, hist);
    block_sum_kernel<<<hb, kScanThreads, 0, s>>>(hist, hn, nullptr, bsum);
    scan_bsum_kernel<<<1, 1024, 0, s>>>(bsum, hb, nullptr);
    scan_apply_kernel<<<hb, kScanThreads, 0, s>>>(hist, hist, hn, bsum);
    radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(K[src], V[src], K[src ^ 1], V[src ^ 1], n, count, shift, nb,
                                                     hist);
    src ^= 1;
  }
  if (src == 1) {
    cudaMemcpyAsync(keys, sk, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vals, sv, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError() == cudaSuccess ? ART_OK : ART_ERR_CUDA;
}
