// C ABI of the GB300 ARTEMIS rendering library (include/artemis.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "internal.cuh"

namespace art {

art_status fail(art_ctx* ctx, art_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return st;
}

art_status cuda_fail(art_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? ART_ERR_OOM : ART_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

art_status ensure(art_ctx* ctx, void** p, size_t* have, size_t need, const char* what) {
  if (*p && *have >= need) return ART_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, need > 0 ? need : 256);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(ctx, e, what);
  }
  *have = need;
  return ART_OK;
}

template <typename T>
static art_status alloc(art_ctx* ctx, T** p, size_t count, const char* what) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(ctx, e, what);
  }
  return ART_OK;
}

void prof_begin(art_ctx* ctx, const char* name) {
  if (!ctx->cfg.profile) return;
  Timer t;
  t.name = name;
  for (int k = 0; k < 2; ++k) {
    cudaEvent_t e;
    if (!ctx->free_events.empty()) {
      e = ctx->free_events.back();
      ctx->free_events.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    (k == 0 ? t.e0 : t.e1) = e;
  }
  cudaEventRecord(t.e0, ctx->stream);
  ctx->pending.push_back(t);
}

void prof_end(art_ctx* ctx) {
  if (!ctx->cfg.profile || ctx->pending.empty()) return;
  cudaEventRecord(ctx->pending.back().e1, ctx->stream);
}

static void prof_collect(art_ctx* ctx) {
  for (auto& t : ctx->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.e0, t.e1);
    bool found = false;
    for (auto& s : ctx->stats)
      if (strcmp(s.name, t.name) == 0) {
        s.launches++;
        s.ms += ms;
        found = true;
        break;
      }
    if (!found) ctx->stats.push_back(KernelStat{t.name, 1, (double)ms});
    ctx->free_events.push_back(t.e0);
    ctx->free_events.push_back(t.e1);
  }
  ctx->pending.clear();
}

namespace {

__global__ void pack_ijk_kernel(int64_t n, const uint16_t* __restrict__ ijk, uint2* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_uint2((uint32_t)ijk[3 * i] | ((uint32_t)ijk[3 * i + 1] << 16), (uint32_t)ijk[3 * i + 2]);
}

__global__ void check_octree_kernel(int64_t n, const uint2* __restrict__ ijk, const uint32_t* __restrict__ jidx,
                                    int depth, unsigned long long* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t lim = 1u << depth;
  uint2 p = ijk[i];
  bool b = (p.x & 0xffffu) >= lim || (p.x >> 16) >= lim || p.y >= lim;
  if (b) atomicAdd(bad, 1ull);
  (void)jidx;
}

__global__ void check_jidx_kernel(int64_t n, const uint32_t* __restrict__ jidx, int J, unsigned long long* bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v = jidx[i];
  bool b = false;
  for (int k = 0; k < 4; ++k) b |= (int)((v >> (8 * k)) & 0xff) >= J;
  if (b) atomicAdd(bad, 1ull);
}

template <typename T>
__global__ void convert_kernel(int64_t m, const float* __restrict__ in, T* __restrict__ out);
template <>
__global__ void convert_kernel<__nv_bfloat16>(int64_t m, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = __float2bfloat16_rn(in[i]);
}
template <>
__global__ void convert_kernel<__half>(int64_t m, const float* __restrict__ in, __half* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = __float2half_rn(in[i]);
}

// BF16 copy wb [..][cin_pad] of the FP32 weights w [..][cin] (input channels
// innermost; channels cin .. cin_pad - 1 zero); w is rounded in place so
// that its FP32 values are the BF16 ones.
__global__ void round_bf16_kernel(int64_t m, int cin, int cin_pad, float* __restrict__ w,
                                  __nv_bfloat16* __restrict__ wb) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    const int ci = (int)(i % cin_pad);
    if (ci >= cin) {
      wb[i] = __float2bfloat16_rn(0.0f);
      return;
    }
    const int64_t j = (i / cin_pad) * cin + ci;
    __nv_bfloat16 b = __float2bfloat16_rn(w[j]);
    wb[i] = b;
    w[j] = __bfloat162float(b);
  }
}

art_status sync_check(art_ctx* ctx, const char* what) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return ART_OK;
}

art_status launch_check(art_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return ART_OK;
}

void free_all(art_ctx* ctx) {
  void* ptrs[] = {ctx->d_ijk, ctx->d_jidx, ctx->d_w, ctx->d_feat, ctx->d_sigma, ctx->d_skel, ctx->d_pose, ctx->d_G,
                  ctx->d_rec, ctx->d_geo, ctx->d_rect, ctx->d_q, ctx->d_cnt, ctx->d_keys,
                  ctx->d_vals, ctx->d_sort_tmp, ctx->d_ranges,
                  ctx->d_status, ctx->d_F, ctx->d_A, ctx->d_rgba, ctx->d_act, ctx->d_sk, ctx->d_sv,
                  ctx->d_shist, ctx->d_sbsum, ctx->d_gN, ctx->d_f8_scale, ctx->d_f8_amax, ctx->d_prop_img,
                  ctx->d_prop_f32, ctx->d_pose_bias, ctx->d_bins, ctx->d_thist, ctx->d_hbin, ctx->d_htau, ctx->d_fbq,
                  ctx->d_seg, ctx->d_items, ctx->d_multi, ctx->d_part, ctx->d_fbq2, ctx->d_tcount, ctx->d_toff,
                  ctx->d_sortlist, ctx->d_scan_state, ctx->d_agroups, ctx->d_sh, ctx->d_sh_rot, ctx->d_rect_v,
                  ctx->d_q_v, ctx->d_cnt_v, ctx->d_vset, ctx->d_xflag, ctx->d_xqueue, ctx->d_xhit, ctx->d_xpos,
                  ctx->d_gkeys, ctx->d_gvals, ctx->d_pgroups, ctx->d_tclass};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& L : ctx->layers) {
    if (L.w32) cudaFree(L.w32);
    if (L.b32) cudaFree(L.b32);
    if (L.wbf) cudaFree(L.wbf);
    if (L.wsub) cudaFree(L.wsub);
    if (L.wtap) cudaFree(L.wtap);
    if (L.w8) cudaFree(L.w8);
    if (L.wscale) cudaFree(L.wscale);
  }
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_pose) cudaEventDestroy(ctx->ev_pose);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  for (int k = 0; k < 2; ++k) {
    if (ctx->d_rgba_slot[k]) cudaFree(ctx->d_rgba_slot[k]);
    if (ctx->ev_ready[k]) cudaEventDestroy(ctx->ev_ready[k]);
    if (ctx->ev_done[k]) cudaEventDestroy(ctx->ev_done[k]);
  }
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
}

art_config default_config() {
  art_config c;
  c.tau = 1e-4f;
  c.instance_cap = 0;
  c.tile_log2 = 3;
  c.profile = 0;
  c.skip = ART_SKIP_PLAIN;
  c.max_missed = 1e-3f;
  c.margin = 0;
  c.segment = 256;
  c.index = ART_INDEX_BOXES;
  c.no_subpixel = 0;
  return c;
}

// Binning buffers sized for the loaded octree and the configured capacity.
art_status ensure_bin_buffers(art_ctx* ctx, int64_t ntiles) {
  int64_t cap = ctx->cfg.instance_cap > 0 ? ctx->cfg.instance_cap : 4 * ctx->n + 65536;
  if (cap > (int64_t)0xFFFFFFF0LL) cap = (int64_t)0xFFFFFFF0LL;
  const bool new_cap = cap != ctx->inst_cap, more_tiles = ntiles > ctx->ranges_cap;
  art_status st;
  if (new_cap) {
    if ((st = alloc(ctx, &ctx->d_keys, (size_t)cap, "instance keys")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_vals, (size_t)cap, "instance values")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_sort_tmp, (size_t)cap, "bucket staging")) != ART_OK) return st;
    ctx->inst_cap = cap;
  }
  if (more_tiles) {
    if ((st = alloc(ctx, &ctx->d_ranges, (size_t)ntiles, "tile ranges")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_tcount, (size_t)ntiles, "tile counts")) != ART_OK) return st;
    // zero once: from then on every tile scan zeroes the counts it read
    cudaMemsetAsync(ctx->d_tcount, 0, sizeof(uint32_t) * (size_t)ntiles, ctx->stream);
    if ((st = alloc(ctx, &ctx->d_toff, (size_t)ntiles, "tile offsets")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_sortlist, (size_t)ntiles, "tile sort list")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_scan_state, tile_scan_state_words(ntiles), "tile scan state")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_agroups, (size_t)(ntiles + 3) / 4, "active tile groups")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_pgroups, (size_t)(ntiles + 3) / 4, "predicted tile groups")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_tclass, (size_t)ntiles, "tile classes")) != ART_OK) return st;
    ctx->ranges_cap = ntiles;
  }
  return ART_OK;
}

// Buffers of the coarse check (per-voxel bins and bounds, per-tile histogram,
// the queue of tiles for the sequential walk) and of the proposal bins, for
// `view`; the histogram is zeroed on the stream.
art_status ensure_skip_buffers(art_ctx* ctx, const ViewParams& v) {
  art_status st;
  if (ctx->hist_n_cap < ctx->n) {
    if ((st = alloc(ctx, &ctx->d_hbin, (size_t)ctx->n, "voxel depth bins")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_htau, (size_t)ctx->n, "voxel optical-depth bounds")) != ART_OK) return st;
    ctx->hist_n_cap = ctx->n;
  }
  const size_t ntiles = (size_t)v.tiles_x * v.tiles_y;
  const float* thist_was = ctx->d_thist;
  if ((st = ensure(ctx, (void**)&ctx->d_thist, &ctx->d_thist_bytes, ntiles * kPropBins * 4, "tile histogram")) != ART_OK)
    return st;
  // zeroed once; the tile scan zeroes the rows of the tiles it gives instances
  if (ctx->d_thist != thist_was) cudaMemsetAsync(ctx->d_thist, 0, ctx->d_thist_bytes, ctx->stream);
  if ((st = ensure(ctx, (void**)&ctx->d_fbq, &ctx->d_fbq_bytes, ntiles * 4, "fallback queue")) != ART_OK) return st;
  if ((st = ensure(ctx, (void**)&ctx->d_bins, &ctx->d_bins_bytes, (size_t)v.W * v.H * 2, "proposal bins")) != ART_OK)
    return st;
  return ART_OK;
}

// Buffers of the split composite walk for `view`: per-tile plan, segment
// lists and partial sums (segments <= instances / seg_len + tiles).
art_status ensure_split_buffers(art_ctx* ctx, size_t ntiles) {
  art_status st;
  // a tile of len entries is cut into ceil(len / seg_len) <= len / seg_len + 1 segments
  const size_t items = (size_t)(ctx->inst_cap / std::max(32, ctx->seg_len)) + ntiles + 1;
  if ((st = ensure(ctx, (void**)&ctx->d_seg, &ctx->d_seg_bytes, ntiles * sizeof(uint2), "segment plan")) != ART_OK)
    return st;
  if ((st = ensure(ctx, (void**)&ctx->d_multi, &ctx->d_multi_bytes, ntiles * 4, "split tiles")) != ART_OK) return st;
  if ((st = ensure(ctx, (void**)&ctx->d_items, &ctx->d_items_bytes, items * 4, "segments")) != ART_OK) return st;
  if ((st = ensure(ctx, (void**)&ctx->d_part, &ctx->d_part_bytes, items * (ctx->C + 1) * 32 * sizeof(float),
                   "segment partial sums")) != ART_OK)
    return st;
  if ((st = ensure(ctx, (void**)&ctx->d_fbq, &ctx->d_fbq_bytes, ntiles * 4, "fallback queue")) != ART_OK) return st;
  if ((st = ensure(ctx, (void**)&ctx->d_fbq2, &ctx->d_fbq2_bytes, ntiles * 4, "coarse-check failures")) != ART_OK)
    return st;
  const uint32_t* xflag_was = ctx->d_xflag;
  if ((st = ensure(ctx, (void**)&ctx->d_xflag, &ctx->d_xflag_bytes, ntiles * 4, "exact re-walk flags")) != ART_OK)
    return st;
  if (ctx->d_xflag != xflag_was) {  // stamps start over on a new array
    cudaMemsetAsync(ctx->d_xflag, 0, ctx->d_xflag_bytes, ctx->stream);
    ctx->xstamp = 0;
  }
  if ((st = ensure(ctx, (void**)&ctx->d_xqueue, &ctx->d_xqueue_bytes, ntiles * 4, "exact re-walk queue")) != ART_OK)
    return st;
  if (!ctx->d_xhit) {
    const size_t m = (size_t)kExactBlocks * 32 * kExactCap;
    if ((st = alloc(ctx, &ctx->d_xhit, m, "exact re-walk hit lists")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_xpos, m, "exact re-walk list positions")) != ART_OK) return st;
  }
  const int fb = ctx->feat_dtype == ART_F32 ? 4 : 2;
  if (ctx->composite_key != ctx->C * 8 + fb) {  // resident walk blocks for this channel count and storage
    ctx->composite_blocks = ctx->num_sms * composite_blocks_per_sm(ctx->C, fb);
    ctx->composite_key = ctx->C * 8 + fb;
  }
  return ART_OK;
}

art_status copy_in(art_ctx* ctx, void* dst, const void* src, size_t bytes, const char* what) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return ART_OK;
}

}  // namespace
}  // namespace art

using namespace art;

extern "C" {

art_status art_create(art_ctx** out, void* cuda_stream) {
  if (!out) return ART_ERR_INVALID_ARG;
  *out = nullptr;
  art_ctx* ctx = new (std::nothrow) art_ctx();
  if (!ctx) return ART_ERR_OOM;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->cfg = default_config();
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_status, sizeof(unsigned long long) * kStWords);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned long long) * kStWords);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_status, sizeof(unsigned long long) * kStWords);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? ART_ERR_OOM : ART_ERR_CUDA;
  }
  *out = ctx;
  return ART_OK;
}

void art_destroy(art_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  free_all(ctx);
  delete ctx;
}

const char* art_last_error(const art_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

art_status art_set_stream(art_ctx* ctx, void* cuda_stream) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)cuda_stream;
  return ART_OK;
}

art_status art_set_config(art_ctx* ctx, const art_config* cfg) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  art_config c = cfg ? *cfg : default_config();
  if (!(c.tau >= 0.0f && c.tau < 1.0f)) return fail(ctx, ART_ERR_INVALID_ARG, "tau must be in [0, 1)");
  if (c.tile_log2 == 0) c.tile_log2 = 3;
  if (c.tile_log2 != 3) return fail(ctx, ART_ERR_UNSUPPORTED, "tile_log2 must be 3 (8x4 tiles)");
  if (c.instance_cap < 0) return fail(ctx, ART_ERR_INVALID_ARG, "instance_cap must be >= 0");
  if (c.skip != ART_SKIP_PLAIN && c.skip != ART_SKIP_LEARNED) return fail(ctx, ART_ERR_INVALID_ARG, "skip mode %d", c.skip);
  if (c.max_missed == 0.0f) c.max_missed = 1e-3f;
  if (!(c.max_missed > 0.0f && c.max_missed < 1.0f)) return fail(ctx, ART_ERR_INVALID_ARG, "max_missed must be in (0, 1)");
  if (c.margin < 0 || c.margin > 63) return fail(ctx, ART_ERR_INVALID_ARG, "margin must be in [0, 63]");
  if (c.segment == 0) c.segment = 256;
  if (c.segment < 32 || c.segment > (1 << 24)) return fail(ctx, ART_ERR_INVALID_ARG, "segment must be in [32, 2^24]");
  if (c.index != ART_INDEX_BOXES && c.index != ART_INDEX_GRID) return fail(ctx, ART_ERR_INVALID_ARG, "index %d", c.index);
  if (c.no_subpixel != 0 && c.no_subpixel != 1) return fail(ctx, ART_ERR_INVALID_ARG, "no_subpixel must be 0 or 1");
  if (c.index != ctx->cfg.index) ctx->posed = false;  // the records of the last pose follow the other index
  ctx->cfg = c;
  ctx->seg_len = c.segment;
  return ART_OK;
}

art_status art_load_octree(art_ctx* ctx, int64_t n, int depth, const float origin[3], float extent,
                           const uint16_t* ijk, const uint8_t* joint_idx, const float* weights,
                           const float* features, int C, int storage_dtype, const float* density) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  ctx->sh_degree = -1;  // coefficients belong to the previous octree
  if (n <= 0 || n > (int64_t)1 << 25) return fail(ctx, ART_ERR_INVALID_ARG, "n=%lld out of range [1, 2^25]", (long long)n);
  if (depth < 1 || depth > 16) return fail(ctx, ART_ERR_INVALID_ARG, "depth=%d out of range [1, 16]", depth);
  if (!origin || !(extent > 0.0f)) return fail(ctx, ART_ERR_INVALID_ARG, "origin/extent invalid");
  if (!ijk || !joint_idx || !weights || !features || !density) return fail(ctx, ART_ERR_INVALID_ARG, "null array");
  if (C != 4 && C != 8 && C != 16 && C != 32) return fail(ctx, ART_ERR_INVALID_ARG, "C=%d not in {4,8,16,32}", C);
  if (storage_dtype != ART_F32 && storage_dtype != ART_BF16 && storage_dtype != ART_F16)
    return fail(ctx, ART_ERR_INVALID_ARG, "storage_dtype %d invalid", storage_dtype);
  art_status st;
  size_t un = (size_t)n;
  if ((st = alloc(ctx, &ctx->d_ijk, un, "ijk")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_jidx, un, "joint idx")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_w, un, "weights")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_sigma, un, "density")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_rec, 4 * un, "voxel records")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_geo, 4 * un, "voxel bounds")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_rect, un, "voxel rects")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_q, un, "depth keys")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_cnt, un, "tile counts")) != ART_OK) return st;
  size_t fbytes = un * (size_t)C * (storage_dtype == ART_F32 ? 4 : 2);
  if (ctx->d_feat) cudaFree(ctx->d_feat);
  ctx->d_feat = nullptr;
  cudaError_t e = cudaMalloc(&ctx->d_feat, fbytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "features");
  // staging for u16 ijk and FP32 features to convert
  uint16_t* t_ijk = nullptr;
  float* t_feat = nullptr;
  if ((st = alloc(ctx, &t_ijk, 3 * un, "ijk staging")) != ART_OK) return st;
  if ((st = copy_in(ctx, t_ijk, ijk, 3 * un * sizeof(uint16_t), "copy ijk")) != ART_OK) return st;
  unsigned grid = (unsigned)((n + 255) / 256);
  pack_ijk_kernel<<<grid, 256, 0, ctx->stream>>>(n, t_ijk, ctx->d_ijk);
  if ((st = copy_in(ctx, ctx->d_jidx, joint_idx, un * 4, "copy joint idx")) != ART_OK) return st;
  if ((st = copy_in(ctx, ctx->d_w, weights, un * 16, "copy weights")) != ART_OK) return st;
  if ((st = copy_in(ctx, ctx->d_sigma, density, un * 4, "copy density")) != ART_OK) return st;
  if (storage_dtype == ART_F32) {
    if ((st = copy_in(ctx, ctx->d_feat, features, fbytes, "copy features")) != ART_OK) return st;
  } else {
    if ((st = alloc(ctx, &t_feat, un * C, "feature staging")) != ART_OK) return st;
    if ((st = copy_in(ctx, t_feat, features, un * C * 4, "copy features")) != ART_OK) return st;
    int64_t m = n * C;
    unsigned g2 = (unsigned)((m + 255) / 256);
    if (storage_dtype == ART_BF16)
      convert_kernel<__nv_bfloat16><<<g2, 256, 0, ctx->stream>>>(m, t_feat, (__nv_bfloat16*)ctx->d_feat);
    else
      convert_kernel<__half><<<g2, 256, 0, ctx->stream>>>(m, t_feat, (__half*)ctx->d_feat);
  }
  // validate coordinates
  cudaMemsetAsync(ctx->d_status + 7, 0, sizeof(unsigned long long), ctx->stream);
  check_octree_kernel<<<grid, 256, 0, ctx->stream>>>(n, ctx->d_ijk, ctx->d_jidx, depth, ctx->d_status + 7);
  cudaMemcpyAsync(ctx->h_status + 7, ctx->d_status + 7, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                  ctx->stream);
  st = sync_check(ctx, "load_octree");
  cudaFree(t_ijk);
  if (t_feat) cudaFree(t_feat);
  if (st != ART_OK) return st;
  if (ctx->h_status[7] != 0) {
    ctx->n = 0;
    return fail(ctx, ART_ERR_INVALID_ARG, "%llu voxels have ijk >= 2^depth", ctx->h_status[7]);
  }
  ctx->n = n;
  ctx->depth = depth;
  for (int a = 0; a < 3; ++a) ctx->origin[a] = origin[a];
  ctx->extent = extent;
  ctx->h = (float)((double)extent / (double)(1 << depth));
  ctx->C = C;
  ctx->feat_dtype = storage_dtype;
  ctx->posed = false;
  ctx->jidx_ok = false;
  ctx->inst_cap = 0;  // force re-sizing of binning buffers
  return ART_OK;
}

art_status art_load_skeleton(art_ctx* ctx, int J, const int32_t* parent, const float* rest_pos) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (J < 1 || J > kMaxJoints) return fail(ctx, ART_ERR_INVALID_ARG, "J=%d out of range [1, %d]", J, kMaxJoints);
  if (!parent || !rest_pos) return fail(ctx, ART_ERR_INVALID_ARG, "null array");
  int32_t par[kMaxJoints];
  float rest[kMaxJoints * 3];
  cudaError_t e = cudaMemcpy(par, parent, sizeof(int32_t) * J, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(rest, rest_pos, sizeof(float) * 3 * J, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy skeleton");
  if (par[0] != -1) return fail(ctx, ART_ERR_INVALID_ARG, "parent[0] must be -1");
  for (int j = 1; j < J; ++j)
    if (par[j] < 0 || par[j] >= j) return fail(ctx, ART_ERR_INVALID_ARG, "parent[%d]=%d must be in [0, %d)", j, par[j], j);
  art_status st;
  if ((st = alloc(ctx, &ctx->d_skel, (size_t)4 * J, "skeleton")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_pose, (size_t)3 * J + 6, "pose")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_G, (size_t)12 * J, "joint transforms")) != ART_OK) return st;
  float host[4 * kMaxJoints];
  for (int j = 0; j < J; ++j) host[j] = (float)par[j];
  memcpy(host + J, rest, sizeof(float) * 3 * J);
  e = cudaMemcpy(ctx->d_skel, host, sizeof(float) * 4 * J, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload skeleton");
  ctx->J = J;
  memcpy(ctx->parent, par, sizeof(int32_t) * J);
  memcpy(ctx->rest, rest, sizeof(float) * 3 * J);
  ctx->posed = false;
  ctx->jidx_ok = false;
  return ART_OK;
}

// The side stream and its events, made on first use.
static art_status ensure_side(art_ctx* ctx) {
  if (ctx->side) return ART_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_pose, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "side stream");
  return ART_OK;
}

// The proposal's per-pose bias runs on the side stream beside FK and LBS;
// work on the main stream that reads the bias or the proposal's weights
// waits for it first (pose_bias_join).
static art_status pose_bias_beside(art_ctx* ctx) {
  art_status st = ensure_side(ctx);
  if (st != ART_OK) return st;
  cudaStream_t main_stream = ctx->stream;
  cudaEventRecord(ctx->ev_fork, main_stream);
  cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
  ctx->stream = ctx->side;
  launch_pose_bias(ctx);
  cudaEventRecord(ctx->ev_pose, ctx->side);
  ctx->stream = main_stream;
  ctx->pose_bias_side = true;
  return ART_OK;
}

static void pose_bias_join(art_ctx* ctx) {
  if (!ctx->pose_bias_side) return;
  cudaStreamWaitEvent(ctx->stream, ctx->ev_pose, 0);
  ctx->pose_bias_side = false;
}

art_status art_set_pose(art_ctx* ctx, const float* axis_angle, const float R[3], const float T[3]) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (ctx->n == 0 || ctx->J == 0) return fail(ctx, ART_ERR_STATE, "set_pose before load_octree/load_skeleton");
  if (!axis_angle || !R || !T) return fail(ctx, ART_ERR_INVALID_ARG, "null pose array");
  int J = ctx->J;
  art_status st;
  if ((st = copy_in(ctx, ctx->d_pose, axis_angle, sizeof(float) * 3 * J, "copy pose")) != ART_OK) return st;
  if ((st = copy_in(ctx, ctx->d_pose + 3 * J, R, sizeof(float) * 3, "copy pose R")) != ART_OK) return st;
  if ((st = copy_in(ctx, ctx->d_pose + 3 * J + 3, T, sizeof(float) * 3, "copy pose T")) != ART_OK) return st;
  if (!ctx->jidx_ok) {  // joint indices against J: once per octree/skeleton pair
    cudaMemsetAsync(ctx->d_status + 7, 0, sizeof(unsigned long long), ctx->stream);
    check_jidx_kernel<<<(unsigned)((ctx->n + 255) / 256), 256, 0, ctx->stream>>>(ctx->n, ctx->d_jidx, J, ctx->d_status + 7);
    cudaMemcpyAsync(ctx->h_status + 7, ctx->d_status + 7, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream);
    if ((st = sync_check(ctx, "set_pose (validate joint indices)")) != ART_OK) return st;
    if (ctx->h_status[7] != 0)
      return fail(ctx, ART_ERR_INVALID_ARG, "%llu voxels reference joints >= J=%d", ctx->h_status[7], J);
    ctx->jidx_ok = true;
  }
  launch_fk(ctx);  // (zeroes the pose's counters, kStDegenerate and kStRmax)
  launch_lbs(ctx);
  if (ctx->cfg.index == ART_INDEX_GRID) {
    if (ctx->grid_slots < 2 * ctx->n) {
      int64_t slots = 1024;
      while (slots < 2 * ctx->n) slots <<= 1;
      if ((st = alloc(ctx, &ctx->d_gkeys, (size_t)slots, "lattice index keys")) != ART_OK) return st;
      if ((st = alloc(ctx, &ctx->d_gvals, (size_t)slots, "lattice index voxels")) != ART_OK) return st;
      ctx->grid_slots = slots;
    }
    launch_grid_snap(ctx);
  }
  if (ctx->prop_loaded && (st = pose_bias_beside(ctx)) != ART_OK) return st;
  if ((st = launch_check(ctx, "set_pose")) != ART_OK) return st;
  ctx->posed = true;
  return ART_OK;
}

art_status art_load_proposal(art_ctx* ctx, const float* params, int64_t n_params) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (!params) return fail(ctx, ART_ERR_INVALID_ARG, "null proposal params");
  if (n_params != ART_PROPOSAL_PARAMS)
    return fail(ctx, ART_ERR_INVALID_ARG, "proposal params: %lld given, %d expected", (long long)n_params,
                ART_PROPOSAL_PARAMS);
  if (ctx->J != 24) return fail(ctx, ART_ERR_STATE, "the proposal takes a 24-joint pose (load_skeleton first)");
  pose_bias_join(ctx);  // (a bias still being computed reads the weights about to be replaced)
  art_status st = load_proposal(ctx, params);
  if (st != ART_OK) return st;
  if (ctx->posed) launch_pose_bias(ctx);
  return launch_check(ctx, "load_proposal");
}

art_status art_run_proposal(art_ctx* ctx, int view, uint8_t* bins_out, float* logits_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "run_proposal before set_pose");
  if (!ctx->prop_loaded) return fail(ctx, ART_ERR_STATE, "run_proposal before load_proposal");
  if ((bins_out && !is_device_ptr(bins_out)) || (logits_out && !is_device_ptr(logits_out)))
    return fail(ctx, ART_ERR_INVALID_ARG, "run_proposal writes device arrays");
  pose_bias_join(ctx);
  art_status st = launch_proposal(ctx, ctx->views[view], bins_out, logits_out, false);
  if (st != ART_OK) return st;
  return launch_check(ctx, "run_proposal");
}

art_status art_render_labels(art_ctx* ctx, int view, float* labels_out, uint8_t* bins_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "render_labels before set_pose");
  if ((labels_out && !is_device_ptr(labels_out)) || (bins_out && !is_device_ptr(bins_out)))
    return fail(ctx, ART_ERR_INVALID_ARG, "render_labels writes device arrays");
  const ViewParams& v = ctx->views[view];
  art_status st = ensure_bin_buffers(ctx, (int64_t)v.tiles_x * v.tiles_y);
  if (st != ART_OK) return st;
  if ((st = ensure_skip_buffers(ctx, v)) != ART_OK) return st;
  launch_project(ctx, v, ctx->d_hbin, ctx->d_htau);
  launch_bin(ctx, v, ctx->d_hbin, ctx->d_htau, ctx->d_thist);
  if ((st = launch_composite_labels(ctx, v, labels_out, bins_out)) != ART_OK) return st;
  return launch_check(ctx, "render_labels");
}

art_status art_set_camera(art_ctx* ctx, int view, int W, int H, float fx, float fy, float cx, float cy,
                          const float world_to_cam[12], float znear, float zfar) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews) return fail(ctx, ART_ERR_INVALID_ARG, "view %d out of range", view);
  if (W < 1 || H < 1 || W > 8192 || H > 8192) return fail(ctx, ART_ERR_INVALID_ARG, "image size %dx%d", W, H);
  if (!(fx > 0 && fy > 0) || !world_to_cam) return fail(ctx, ART_ERR_INVALID_ARG, "bad intrinsics");
  if (!(znear > 0 && zfar > znear)) return fail(ctx, ART_ERR_INVALID_ARG, "need 0 < znear < zfar");
  float M[12];
  cudaError_t e = cudaMemcpy(M, world_to_cam, sizeof(M), cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy camera");
  ViewParams& v = ctx->views[view];
  v.W = W;
  v.H = H;
  v.fx = fx;
  v.fy = fy;
  v.cx = cx;
  v.cy = cy;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) v.R[r * 3 + c] = M[r * 4 + c];
    v.t[r] = M[r * 4 + 3];
  }
  for (int a = 0; a < 3; ++a) {
    double s = 0;
    for (int r = 0; r < 3; ++r) s -= (double)M[r * 4 + a] * (double)M[r * 4 + 3];
    v.o[a] = (float)s;
    v.o_lo[a] = (float)(s - (double)v.o[a]);
  }
  v.znear = znear;
  v.zfar = zfar;
  v.tile_wl = 3;  // 8 x 4 pixel tiles: one warp per tile in the composite
  v.tile_hl = 2;
  v.tile_w = 1 << v.tile_wl;
  v.tile_h = 1 << v.tile_hl;
  v.tiles_x = (W + v.tile_w - 1) / v.tile_w;
  v.tiles_y = (H + v.tile_h - 1) / v.tile_h;
  int64_t ntiles = (int64_t)v.tiles_x * v.tiles_y;
  int tb = 1;
  while (((int64_t)1 << tb) < ntiles) ++tb;
  // at most 20 depth bits: one quantum (>= (zfar - znear) / 2^20) stays far
  // above the FP32 rounding of distances, which keeps the key a lower bound
  v.depth_bits = std::min(32 - tb, 20);
  if (v.depth_bits < 12) return fail(ctx, ART_ERR_UNSUPPORTED, "too many tiles for 32-bit keys");
  v.dscale = (float)((double)(1u << v.depth_bits) / ((double)zfar - (double)znear));
  ctx->view_set[view] = true;
  return ART_OK;
}

// After the scan and scatter of a view: the work that needs only the tile
// ranges and the coarse bound (tile classes and proposal for the learned
// skip, the clear of the empty tiles) runs on the side stream while the
// bucket sort runs on the main one; the main stream then waits for both.
static art_status sort_beside(art_ctx* ctx, const ViewParams& v, void* F, int F_dtype, float* A, bool skip) {
  art_status st = ensure_side(ctx);
  if (st != ART_OK) return st;
  cudaStream_t main_stream = ctx->stream;
  cudaEventRecord(ctx->ev_fork, main_stream);
  cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
  ctx->stream = ctx->side;
  if (skip) {
    launch_tile_class(ctx, v, ctx->d_bins);
    st = launch_proposal(ctx, v, ctx->d_bins, nullptr, true, true);
  }
  if (st == ART_OK) st = launch_composite_clear(ctx, v, F, F_dtype, A);
  cudaEventRecord(ctx->ev_join, ctx->side);
  ctx->stream = main_stream;
  launch_tile_sort(ctx, v);
  cudaStreamWaitEvent(main_stream, ctx->ev_join, 0);
  ctx->pose_bias_side = false;  // (the join follows the side stream's pose bias too)
  ctx->f_cleared = st == ART_OK;
  return st;
}

static art_status render_to_device(art_ctx* ctx, int view, void* F, int F_dtype, float* A) {
  const ViewParams& v = ctx->views[view];
  art_status st = ensure_bin_buffers(ctx, (int64_t)v.tiles_x * v.tiles_y);
  if (st != ART_OK) return st;
  if ((st = ensure_split_buffers(ctx, (size_t)v.tiles_x * v.tiles_y)) != ART_OK) return st;
  if (ctx->cfg.skip == ART_SKIP_LEARNED) {  // proposal intervals + coarse check + fallback
    if (ctx->sh_degree >= 0)
      return fail(ctx, ART_ERR_UNSUPPORTED, "view-dependent (SH) features use the plain traversal (skip = 0)");
    if (!ctx->prop_loaded) return fail(ctx, ART_ERR_STATE, "learned skip without a proposal (art_load_proposal)");
    if ((st = ensure_skip_buffers(ctx, v)) != ART_OK) return st;
    launch_project(ctx, v, ctx->d_hbin, ctx->d_htau);
    launch_bin(ctx, v, ctx->d_hbin, ctx->d_htau, ctx->d_thist, false);
    st = sort_beside(ctx, v, F, F_dtype, A, true);
    if (st == ART_OK) st = launch_composite_skip(ctx, v, F, F_dtype, A);
    ctx->f_cleared = false;
    if (st != ART_OK) return st;
    return launch_check(ctx, "render_feature_maps");
  }
  if (ctx->sh_degree >= 0 && ctx->cfg.index == ART_INDEX_GRID)
    return fail(ctx, ART_ERR_UNSUPPORTED, "view-dependent (SH) features need the exact boxes (index 0)");
  launch_project(ctx, v);
  launch_bin(ctx, v, nullptr, nullptr, nullptr, false);
  st = sort_beside(ctx, v, F, F_dtype, A, false);
  if (st == ART_OK) {
    if (ctx->sh_degree >= 0)  // view-dependent features (Eq. 2)
      st = launch_composite_sh(ctx, v, F, F_dtype, A);
    else
      st = launch_composite(ctx, v, F, F_dtype, A);
  }
  ctx->f_cleared = false;
  if (st != ART_OK) return st;
  return launch_check(ctx, ctx->sh_degree >= 0 ? "render_feature_maps (SH)" : "render_feature_maps");
}

art_status art_render_views(art_ctx* ctx, int nv, const int* views, void* const* F_out, int F_dtype,
                            float* const* A_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (nv < 1 || nv > kMaxViews || !views || !F_out) return fail(ctx, ART_ERR_INVALID_ARG, "need 1..%d views", kMaxViews);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "render before set_pose");
  if (F_dtype != ART_F32 && F_dtype != ART_BF16) return fail(ctx, ART_ERR_INVALID_ARG, "F_dtype must be F32 or BF16");
  for (int k = 0; k < nv; ++k) {
    const int vk = views[k];
    if (vk < 0 || vk >= kMaxViews || !ctx->view_set[vk]) return fail(ctx, ART_ERR_STATE, "view %d not set", vk);
    for (int j = 0; j < k; ++j)
      if (views[j] == vk) return fail(ctx, ART_ERR_INVALID_ARG, "view %d listed twice", vk);
    if (!F_out[k] || !is_device_ptr(F_out[k]) || (A_out && A_out[k] && !is_device_ptr(A_out[k])))
      return fail(ctx, ART_ERR_INVALID_ARG, "render_views writes device arrays (view %d)", vk);
  }
  art_status st;
  if (ctx->cfg.skip == ART_SKIP_LEARNED || ctx->sh_degree >= 0) {  // per-view passes
    for (int k = 0; k < nv; ++k)
      if ((st = render_to_device(ctx, views[k], F_out[k], F_dtype, A_out ? A_out[k] : nullptr)) != ART_OK) return st;
    return ART_OK;
  }
  // one tile space: view k's tiles after the first k views'; one depth-key layout
  ViewSet& vs = ctx->h_vset;
  vs = ViewSet{};
  vs.nv = nv;
  int64_t total = 0;
  for (int k = 0; k < nv; ++k) {
    const ViewParams& v = ctx->views[views[k]];
    vs.toff[k] = (uint32_t)total;
    total += (int64_t)v.tiles_x * v.tiles_y;
  }
  vs.toff[nv] = (uint32_t)total;
  int tb = 1;
  while (((int64_t)1 << tb) < total) ++tb;
  const int depth_bits = std::min(32 - tb, 20);
  if (depth_bits < 12) return fail(ctx, ART_ERR_UNSUPPORTED, "too many tiles over the views for 32-bit keys");
  for (int k = 0; k < nv; ++k) {
    ViewParams v = ctx->views[views[k]];
    v.depth_bits = depth_bits;
    v.dscale = (float)((double)(1u << depth_bits) / ((double)v.zfar - (double)v.znear));
    vs.v[k] = v;
    vs.F[k] = F_out[k];
    vs.A[k] = A_out ? A_out[k] : nullptr;
  }
  if ((st = ensure_bin_buffers(ctx, total)) != ART_OK) return st;
  if ((st = ensure_split_buffers(ctx, (size_t)total)) != ART_OK) return st;
  const int64_t need = (int64_t)nv * ctx->n;
  if (ctx->views_cap < need) {
    if ((st = alloc(ctx, &ctx->d_rect_v, (size_t)need, "batch voxel rects")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_q_v, (size_t)need, "batch depth keys")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_cnt_v, (size_t)need, "batch tile counts")) != ART_OK) return st;
    ctx->views_cap = need;
  }
  if (!ctx->d_vset && (st = alloc(ctx, &ctx->d_vset, 1, "view table")) != ART_OK) return st;
  vs.rect_stride = ctx->n;
  if ((st = copy_in(ctx, ctx->d_vset, &vs, sizeof(ViewSet), "copy view table")) != ART_OK) return st;
  for (int k = 0; k < nv; ++k) {  // (the counts are zero: the last tile scan cleared them)
    const int64_t o = (int64_t)k * ctx->n;
    launch_project_view(ctx, vs.v[k], ctx->d_rect_v + o, ctx->d_q_v + o, ctx->d_cnt_v + o, ctx->d_tcount + vs.toff[k],
                        k == 0);
  }
  launch_bin_views(ctx, vs, total);
  if ((st = launch_composite_views(ctx, vs, F_dtype)) != ART_OK) return st;
  return launch_check(ctx, "render_views");
}

art_status art_render_feature_maps(art_ctx* ctx, int view, void* F_out, int F_dtype, float* A_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "render before set_pose");
  if (!F_out) return fail(ctx, ART_ERR_INVALID_ARG, "F_out is null");
  if (F_dtype != ART_F32 && F_dtype != ART_BF16) return fail(ctx, ART_ERR_INVALID_ARG, "F_dtype must be F32 or BF16");
  const ViewParams& v = ctx->views[view];
  size_t npx = (size_t)v.W * v.H;
  size_t fbytes = npx * ctx->C * (F_dtype == ART_F32 ? 4 : 2);
  bool f_dev = is_device_ptr(F_out);
  bool a_dev = A_out ? is_device_ptr(A_out) : true;
  void* F = F_out;
  float* A = A_out;
  art_status st;
  if (!f_dev) {
    if ((st = ensure(ctx, &ctx->d_F, &ctx->d_F_bytes, fbytes, "F buffer")) != ART_OK) return st;
    F = ctx->d_F;
  }
  if (A_out && !a_dev) {
    if ((st = ensure(ctx, (void**)&ctx->d_A, &ctx->d_A_bytes, npx * 4, "A buffer")) != ART_OK) return st;
    A = ctx->d_A;
  }
  if ((st = render_to_device(ctx, view, F, F_dtype, A)) != ART_OK) return st;
  if (!f_dev || (A_out && !a_dev)) {
    if (!f_dev) cudaMemcpyAsync(F_out, F, fbytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (A_out && !a_dev) cudaMemcpyAsync(A_out, A, npx * 4, cudaMemcpyDeviceToHost, ctx->stream);
    return sync_check(ctx, "render_feature_maps (copy out)");
  }
  return ART_OK;
}

art_status art_load_sh_features(art_ctx* ctx, int degree, const float* coef) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (ctx->n == 0) return fail(ctx, ART_ERR_STATE, "load_sh_features before load_octree");
  if (degree < 0) {  // back to the plain per-voxel features
    ctx->sh_degree = -1;
    return ART_OK;
  }
  if (degree > kShMaxDegree)
    return fail(ctx, ART_ERR_UNSUPPORTED, "SH degree %d: degrees 0 .. %d are built", degree, kShMaxDegree);
  if (!coef) return fail(ctx, ART_ERR_INVALID_ARG, "coef is null");
  const size_t count = (size_t)ctx->n * (size_t)((degree + 1) * (degree + 1)) * (size_t)ctx->C;
  art_status st;
  if ((st = alloc(ctx, &ctx->d_sh, count, "SH coefficients")) != ART_OK) return st;
  if ((st = alloc(ctx, &ctx->d_sh_rot, 9 * (size_t)ctx->n, "SH rotations")) != ART_OK) return st;
  cudaError_t e = cudaMemcpyAsync(ctx->d_sh, coef, sizeof(float) * count, cudaMemcpyDefault, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy SH coefficients");
  if ((st = sync_check(ctx, "load_sh_features")) != ART_OK) return st;
  ctx->sh_degree = degree;
  return ART_OK;
}

art_status art_render_depth(art_ctx* ctx, int view, float sigma_min, float* depth_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "render_depth before set_pose");
  if (!depth_out) return fail(ctx, ART_ERR_INVALID_ARG, "depth_out is null");
  if (!(sigma_min >= 0.0f)) return fail(ctx, ART_ERR_INVALID_ARG, "sigma_min must be >= 0");
  const ViewParams& v = ctx->views[view];
  const size_t npx = (size_t)v.W * v.H;
  const bool dev = is_device_ptr(depth_out);
  float* D = depth_out;
  art_status st;
  if (!dev) {
    if ((st = ensure(ctx, (void**)&ctx->d_A, &ctx->d_A_bytes, npx * 4, "depth buffer")) != ART_OK) return st;
    D = ctx->d_A;
  }
  if ((st = ensure_bin_buffers(ctx, (int64_t)v.tiles_x * v.tiles_y)) != ART_OK) return st;
  launch_project(ctx, v);
  launch_bin(ctx, v);
  launch_depth(ctx, v, sigma_min, D);
  if ((st = launch_check(ctx, "render_depth")) != ART_OK) return st;
  if (!dev) {
    cudaMemcpyAsync(depth_out, D, npx * 4, cudaMemcpyDeviceToHost, ctx->stream);
    return sync_check(ctx, "render_depth (copy out)");
  }
  return ART_OK;
}

art_status art_load_shader(art_ctx* ctx, const art_net_desc* desc, const float* params, int64_t n_params,
                           int compute_dtype) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (!desc || !params) return fail(ctx, ART_ERR_INVALID_ARG, "null descriptor or params");
  if (compute_dtype != ART_F32 && compute_dtype != ART_BF16 && compute_dtype != ART_FP8)
    return fail(ctx, ART_ERR_UNSUPPORTED, "compute dtype %d not available", compute_dtype);
  std::vector<int> shapes;  // cout, cin, k
  const art_net_desc& d = *desc;
  // (cout, cin, k) of a U-Net's layers in execution order: enc0 a/b, ...,
  // bottleneck a/b, dec(levels-2) a/b, ..., dec0 a/b, 1x1 head
  auto unet_shapes = [&](int cin, int levels, const int* ch, int cout) {
    int prev = cin;
    for (int l = 0; l < levels; ++l) {
      shapes.insert(shapes.end(), {ch[l], prev, 3, ch[l], ch[l], 3});
      prev = ch[l];
    }
    for (int l = levels - 2; l >= 0; --l) shapes.insert(shapes.end(), {ch[l], ch[l + 1] + ch[l], 3, ch[l], ch[l], 3});
    shapes.insert(shapes.end(), {cout, ch[0], 1});
  };
  if (d.cin < 1 || d.cout < 1 || d.cin > 256 || d.cout > 256) return fail(ctx, ART_ERR_INVALID_ARG, "cin/cout range");
  if (d.arch == ART_NET_TINY) {
    int c = d.ch[0];
    if (c < 1 || c > 256) return fail(ctx, ART_ERR_INVALID_ARG, "hidden width range");
    shapes = {c, d.cin, 3, c, c, 3, d.cout, c, 3};
  } else if (d.arch == ART_NET_UNET || d.arch == ART_NET_TWO_BRANCH) {
    for (int k = 0; k < 4; ++k)
      if (d.ch[k] < 1 || d.ch[k] > 512) return fail(ctx, ART_ERR_INVALID_ARG, "channel range");
    if (d.arch == ART_NET_UNET) {
      unet_shapes(d.cin, 4, d.ch, d.cout);
    } else {
      if (d.cout != 4) return fail(ctx, ART_ERR_INVALID_ARG, "two-branch network: cout must be 4 (RGB + alpha)");
      if (compute_dtype == ART_FP8) return fail(ctx, ART_ERR_UNSUPPORTED, "two-branch network: F32 or BF16 only");
      for (int k = 0; k < 2; ++k)
        if (d.ach[k] < 1 || d.ach[k] > 512) return fail(ctx, ART_ERR_INVALID_ARG, "opacity channel range");
      unet_shapes(d.cin, 4, d.ch, 3);  // appearance: F -> I_f
      unet_shapes(4, 2, d.ach, 1);     // opacity: [A, I_f] -> alpha
    }
  } else {
    return fail(ctx, ART_ERR_INVALID_ARG, "unknown arch %d", d.arch);
  }
  int nl = (int)shapes.size() / 3;
  int64_t need = 0;
  for (int l = 0; l < nl; ++l) need += (int64_t)shapes[3 * l] * shapes[3 * l + 2] * shapes[3 * l + 2] * shapes[3 * l + 1] + shapes[3 * l];
  if (need != n_params)
    return fail(ctx, ART_ERR_INVALID_ARG, "n_params=%lld, network needs %lld", (long long)n_params, (long long)need);
  for (auto& L : ctx->layers) {
    if (L.w32) cudaFree(L.w32);
    if (L.b32) cudaFree(L.b32);
    if (L.wbf) cudaFree(L.wbf);
    if (L.wsub) cudaFree(L.wsub);
    if (L.wtap) cudaFree(L.wtap);
    if (L.w8) cudaFree(L.w8);
    if (L.wscale) cudaFree(L.wscale);
  }
  ctx->layers.clear();
  int64_t off = 0;
  art_status st = ART_OK;
  for (int l = 0; l < nl; ++l) {
    ConvLayer L;
    L.cout = shapes[3 * l];
    L.cin = shapes[3 * l + 1];
    L.k = shapes[3 * l + 2];
    // the opacity branch's first layer reads the packed [A, I_f, 0 ...] tensor on the tensor cores
    const bool padded = d.arch == ART_NET_TWO_BRANCH && l == 15 && compute_dtype == ART_BF16;
    L.cin_pad = padded ? kOpacityPad : L.cin;
    size_t nw = (size_t)L.cout * L.k * L.k * L.cin;
    if ((st = alloc(ctx, &L.w32, nw, "weights")) != ART_OK) break;
    if ((st = alloc(ctx, &L.b32, (size_t)L.cout, "bias")) != ART_OK) break;
    if ((st = copy_in(ctx, L.w32, params + off, nw * 4, "copy weights")) != ART_OK) break;
    off += (int64_t)nw;
    if ((st = copy_in(ctx, L.b32, params + off, (size_t)L.cout * 4, "copy bias")) != ART_OK) break;
    off += L.cout;
    if (compute_dtype == ART_BF16 || compute_dtype == ART_FP8) {
      const size_t nwp = (size_t)L.cout * L.k * L.k * L.cin_pad;
      if ((st = alloc(ctx, &L.wbf, nwp, "bf16 weights")) != ART_OK) break;
      round_bf16_kernel<<<(unsigned)((nwp + 255) / 256), 256, 0, ctx->stream>>>((int64_t)nwp, L.cin, L.cin_pad,
                                                                                 L.w32, L.wbf);
    }
    if (compute_dtype == ART_FP8 && L.k == 3) {  // 1x1 head stays FP32 (fused epilogue)
      if ((st = alloc(ctx, &L.w8, nw, "fp8 weights")) != ART_OK) break;
      if ((st = alloc(ctx, &L.wscale, (size_t)L.cout, "fp8 weight scales")) != ART_OK) break;
      launch_quantize_weights(ctx, L.w32, L.cout, L.k * L.k * L.cin, L.w8, L.wscale);
    }
    ctx->layers.push_back(L);
  }
  if (st != ART_OK) return st;
  // level 0's decoder convolution (after the concatenation with the
  // upsampled level-1 output) in its sub-pixel form: its weight blocks
  auto sub_blocks = [&](int li, int cs, int cu) -> art_status {
    if (li >= (int)ctx->layers.size()) return ART_OK;
    ConvLayer& L = ctx->layers[li];
    if (L.k != 3 || L.cin != cs + cu || L.cin_pad != L.cin || !sub_conv_ok(L.cout, cs, cu, 2, 2)) return ART_OK;
    art_status s2 = alloc(ctx, &L.wsub, sub_weight_elems(cs, cu), "sub-pixel weights");
    if (s2 != ART_OK) return s2;
    launch_sub_weights(ctx, L.w32, cs, cu, L.wsub);
    L.sub_cs = cs;
    L.sub_cu = cu;
    return ART_OK;
  };
  // ... and those of levels 1 and 2 (the tap-by-tap kernel's per-phase weights)
  auto tap_blocks = [&](int li, int cs, int cu) -> art_status {
    if (li >= (int)ctx->layers.size()) return ART_OK;
    ConvLayer& L = ctx->layers[li];
    if (L.k != 3 || L.cin != cs + cu || L.cin_pad != L.cin || cs % 32 || cu % 32) return ART_OK;
    art_status s2 = alloc(ctx, &L.wtap, (size_t)4 * L.cout * (9 * cs + 4 * cu), "sub-pixel weights");
    if (s2 != ART_OK) return s2;
    launch_sub_tap_weights(ctx, L.w32, L.cout, cs, cu, L.wtap);
    L.sub_cs = cs;
    L.sub_cu = cu;
    return ART_OK;
  };
  if (compute_dtype == ART_BF16 && (d.arch == ART_NET_UNET || d.arch == ART_NET_TWO_BRANCH)) {
    st = sub_blocks(12, d.ch[0], d.ch[1]);                  // decoder of level 0
    if (st == ART_OK) st = tap_blocks(10, d.ch[1], d.ch[2]);  // level 1
    if (st == ART_OK) st = tap_blocks(8, d.ch[2], d.ch[3]);   // level 2
    if (st == ART_OK && d.arch == ART_NET_TWO_BRANCH) st = sub_blocks(19, d.ach[0], d.ach[1]);
  }
  if (st != ART_OK) return st;
  ctx->net = d;
  ctx->net_dtype = compute_dtype;
  if (compute_dtype == ART_FP8) {
    if ((st = alloc(ctx, &ctx->d_f8_scale, (size_t)kF8Tensors, "fp8 scales")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_f8_amax, (size_t)kF8Tensors, "fp8 amax")) != ART_OK) return st;
    cudaMemsetAsync(ctx->d_f8_amax, 0, sizeof(unsigned int) * kF8Tensors, ctx->stream);
    ctx->f8_calibrated = false;
  }
  return sync_check(ctx, "load_shader");
}

namespace art {
namespace {

art_status shade_impl(art_ctx* ctx, int view, const void* F, int F_dtype, const float* A, float* rgba_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (ctx->layers.empty()) return fail(ctx, ART_ERR_STATE, "shade before load_shader");
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!F || !rgba_out) return fail(ctx, ART_ERR_INVALID_ARG, "null pointer");
  const ViewParams& v = ctx->views[view];
  const bool two = ctx->net.arch == ART_NET_TWO_BRANCH;
  if (two && !A) return fail(ctx, ART_ERR_INVALID_ARG, "the two-branch network needs A: art_shade_with_opacity");
  if (ctx->net.arch != ART_NET_TINY && ((v.W % 8) || (v.H % 8)))
    return fail(ctx, ART_ERR_INVALID_ARG, "U-Net needs W and H multiples of 8");
  size_t npx = (size_t)v.W * v.H;
  size_t fbytes = npx * ctx->net.cin * (F_dtype == ART_F32 ? 4 : 2);
  const void* Fd = F;
  art_status st;
  if (!is_device_ptr(F)) {
    if ((st = ensure(ctx, &ctx->d_F, &ctx->d_F_bytes, fbytes, "F buffer")) != ART_OK) return st;
    if ((st = copy_in(ctx, ctx->d_F, F, fbytes, "copy F")) != ART_OK) return st;
    Fd = ctx->d_F;
  }
  const float* Ad = two ? A : nullptr;
  if (two && !is_device_ptr(A)) {
    if ((st = ensure(ctx, (void**)&ctx->d_A, &ctx->d_A_bytes, npx * 4, "A buffer")) != ART_OK) return st;
    if ((st = copy_in(ctx, ctx->d_A, A, npx * 4, "copy A")) != ART_OK) return st;
    Ad = ctx->d_A;
  }
  bool out_dev = is_device_ptr(rgba_out);
  float* out = rgba_out;
  size_t obytes = npx * ctx->net.cout * 4;
  if (!out_dev) {
    if ((st = ensure(ctx, (void**)&ctx->d_rgba, &ctx->d_rgba_bytes, obytes, "rgba buffer")) != ART_OK) return st;
    out = ctx->d_rgba;
  }
  if ((st = run_shader(ctx, v, Fd, F_dtype, Ad, out)) != ART_OK) return st;
  if ((st = launch_check(ctx, "shade")) != ART_OK) return st;
  if (!out_dev) {
    cudaMemcpyAsync(rgba_out, out, obytes, cudaMemcpyDeviceToHost, ctx->stream);
    return sync_check(ctx, "shade (copy out)");
  }
  return ART_OK;
}

}  // namespace
}  // namespace art

art_status art_shade(art_ctx* ctx, int view, const void* F, int F_dtype, float* rgba_out) {
  return shade_impl(ctx, view, F, F_dtype, nullptr, rgba_out);
}

art_status art_shade_with_opacity(art_ctx* ctx, int view, const void* F, int F_dtype, const float* A, float* rgba_out) {
  if (ctx && !A) return fail(ctx, ART_ERR_INVALID_ARG, "null A");
  return shade_impl(ctx, view, F, F_dtype, A, rgba_out);
}

art_status art_render_frame(art_ctx* ctx, int view, const float* axis_angle, const float R[3], const float T[3],
                            float* rgba_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (ctx->layers.empty()) return fail(ctx, ART_ERR_STATE, "render_frame before load_shader");
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (ctx->net.cin != ctx->C) return fail(ctx, ART_ERR_INVALID_ARG, "network cin %d != feature C %d", ctx->net.cin, ctx->C);
  art_status st = art_set_pose(ctx, axis_angle, R, T);
  if (st != ART_OK) return st;
  const ViewParams& v = ctx->views[view];
  int fdt = ctx->net_dtype == ART_F32 ? ART_F32 : ART_BF16;  // BF16 F feeds the BF16 and FP8 networks
  size_t fbytes = (size_t)v.W * v.H * ctx->C * (fdt == ART_F32 ? 4 : 2);
  if ((st = ensure(ctx, &ctx->d_F, &ctx->d_F_bytes, fbytes, "F buffer")) != ART_OK) return st;
  if ((st = ensure(ctx, (void**)&ctx->d_A, &ctx->d_A_bytes, (size_t)v.W * v.H * 4, "A buffer")) != ART_OK) return st;
  if ((st = render_to_device(ctx, view, ctx->d_F, fdt, ctx->d_A)) != ART_OK) return st;
  return shade_impl(ctx, view, ctx->d_F, fdt, ctx->d_A, rgba_out);
}

namespace {
// Waits for the oldest frame in flight of art_render_frame_async (its RGBA
// has reached the host) and drops it from the ring.
art_status wait_oldest_frame(art_ctx* ctx) {
  const int s = ctx->fr_head;
  const cudaError_t e = cudaEventSynchronize(ctx->ev_done[s]);
  ctx->fr_head = (ctx->fr_head + 1) % 2;
  --ctx->fr_n;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "render_frame_async (copy out)");
  return ART_OK;
}
}  // namespace

art_status art_render_frame_async(art_ctx* ctx, int view, const float* axis_angle, const float R[3], const float T[3],
                                  float* rgba_out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (!rgba_out) return fail(ctx, ART_ERR_INVALID_ARG, "rgba_out is null");
  if (is_device_ptr(rgba_out))
    return fail(ctx, ART_ERR_INVALID_ARG, "render_frame_async copies to a host buffer (art_render_frame takes device buffers)");
  if (ctx->layers.empty()) return fail(ctx, ART_ERR_STATE, "render_frame_async before load_shader");
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  art_status st;
  if (!ctx->copy_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&ctx->ev_ready[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_done[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
  }
  // two frames in flight at most: a third waits for the oldest's copy
  if (ctx->fr_n == 2 && (st = wait_oldest_frame(ctx)) != ART_OK) return st;
  const int slot = (ctx->fr_head + ctx->fr_n) % 2;  // (its last copy has landed)
  const ViewParams& v = ctx->views[view];
  const size_t obytes = (size_t)v.W * v.H * ctx->net.cout * 4;
  if ((st = ensure(ctx, (void**)&ctx->d_rgba_slot[slot], &ctx->d_rgba_slot_bytes[slot], obytes, "rgba slot")) != ART_OK)
    return st;
  // the frame into the device slot (no synchronisation), then its copy on the copy stream
  if ((st = art_render_frame(ctx, view, axis_angle, R, T, ctx->d_rgba_slot[slot])) != ART_OK) return st;
  cudaError_t e = cudaEventRecord(ctx->ev_ready[slot], ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_ready[slot], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rgba_out, ctx->d_rgba_slot[slot], obytes, cudaMemcpyDeviceToHost, ctx->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_done[slot], ctx->copy_stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "render_frame_async (copy out)");
  ++ctx->fr_n;
  return ART_OK;
}

art_status art_wait_frames(art_ctx* ctx) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  art_status st = ART_OK;
  while (ctx->fr_n > 0) {
    const art_status s2 = wait_oldest_frame(ctx);
    if (st == ART_OK) st = s2;
  }
  if (st != ART_OK) return st;
  return sync_check(ctx, "wait_frames");
}

art_status art_sync_status(art_ctx* ctx, art_stats* out) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(unsigned long long) * kStWords, cudaMemcpyDeviceToHost,
                  ctx->stream);
  art_status st = sync_check(ctx, "sync_status");
  if (st != ART_OK) return st;
  unsigned long long* h = ctx->h_status;
  if (out) {
    out->instances = (int64_t)h[kStInstances];
    out->degenerate = (int64_t)h[kStDegenerate];
    out->overflow_inst = (int64_t)h[kStOverflowInst];
    out->overflow_order = (int64_t)h[kStOverflowOrder];
    out->kernel_launches = ctx->launches;
    out->fallback_tiles = (int64_t)h[kStFallback];
    out->exact_tiles = (int64_t)h[kStExactQ];
    out->grid_cells = ctx->cfg.index == ART_INDEX_GRID ? (int64_t)h[kStGridCells] : 0;
    out->forced_tiles = (int64_t)h[kStForcedTiles];
    out->check_fail_tiles = (int64_t)h[kStCheckFail];
  }
  if (h[kStTcError]) {
    art_status r = fail(ctx, ART_ERR_CUDA, "tensor-core convolution: %llu CTAs timed out waiting on their pipeline",
                        h[kStTcError]);
    cudaMemsetAsync(ctx->d_status + kStTcError, 0, sizeof(unsigned long long), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return r;
  }
  if (h[kStScanError]) {
    art_status r = fail(ctx, ART_ERR_CUDA, "binning: %llu tile-scan blocks timed out waiting for a predecessor",
                        h[kStScanError]);
    cudaMemsetAsync(ctx->d_status + kStScanError, 0, sizeof(unsigned long long), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return r;
  }
  if (h[kStOverflowInst] || h[kStOverflowOrder]) {
    art_status r = fail(ctx, ART_ERR_OVERFLOW, "overflow: %llu instances beyond capacity %lld, %llu reorder-buffer releases",
                        h[kStOverflowInst], (long long)ctx->inst_cap, h[kStOverflowOrder]);
    cudaMemsetAsync(ctx->d_status + kStOverflowInst, 0, 2 * sizeof(unsigned long long), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return r;
  }
  return ART_OK;
}

art_status art_get_kernel_times(art_ctx* ctx, int cap, const char** names, int64_t* launches, double* ms, int* count,
                                int reset) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  art_status st = sync_check(ctx, "get_kernel_times");
  if (st != ART_OK) return st;
  prof_collect(ctx);
  int m = (int)ctx->stats.size();
  if (count) *count = m;
  for (int i = 0; i < m && i < cap; ++i) {
    if (names) names[i] = ctx->stats[i].name;
    if (launches) launches[i] = ctx->stats[i].launches;
    if (ms) ms[i] = ctx->stats[i].ms;
  }
  if (reset) ctx->stats.clear();
  return ART_OK;
}

art_status art_sort_pairs(art_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n, int key_bits) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (n < 0 || n > (int64_t)0x7FFFFFFF) return fail(ctx, ART_ERR_INVALID_ARG, "n=%lld out of range", (long long)n);
  if (key_bits != 8 && key_bits != 16 && key_bits != 24 && key_bits != 32)
    return fail(ctx, ART_ERR_INVALID_ARG, "key_bits=%d must be 8, 16, 24 or 32", key_bits);
  if (n == 0) return ART_OK;
  if (!keys || !vals) return fail(ctx, ART_ERR_INVALID_ARG, "null keys/vals");
  if (!is_device_ptr(keys) || !is_device_ptr(vals)) return fail(ctx, ART_ERR_INVALID_ARG, "keys/vals must be device memory");
  art_status st;
  if (n > ctx->sort_cap) {
    if ((st = alloc(ctx, &ctx->d_sk, (size_t)n, "sort scratch keys")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_sv, (size_t)n, "sort scratch values")) != ART_OK) return st;
    size_t hw = sort_hist_words(n);
    if ((st = alloc(ctx, &ctx->d_shist, hw, "sort histogram")) != ART_OK) return st;
    if ((st = alloc(ctx, &ctx->d_sbsum, scan_block_words((int64_t)hw), "sort block sums")) != ART_OK) return st;
    ctx->sort_cap = n;
  }
  unsigned long long* cnt = ctx->d_status + 6;
  launch_set_word(ctx, cnt, (unsigned long long)n);
  int where = launch_sort_bufs(ctx, keys, vals, ctx->d_sk, ctx->d_sv, n, cnt, key_bits, ctx->d_shist, ctx->d_sbsum);
  if (where == 1) {
    cudaMemcpyAsync(keys, ctx->d_sk, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(vals, ctx->d_sv, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream);
  }
  return launch_check(ctx, "sort_pairs");
}

art_status art_update_voxels(art_ctx* ctx, const float* features, const float* density, const float* weights) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (ctx->n == 0) return fail(ctx, ART_ERR_STATE, "update_voxels before load_octree");
  const size_t n = (size_t)ctx->n;
  art_status st;
  if (density && (st = copy_in(ctx, ctx->d_sigma, density, n * 4, "copy density")) != ART_OK) return st;
  if (weights && (st = copy_in(ctx, ctx->d_w, weights, n * 16, "copy weights")) != ART_OK) return st;
  if (features) {
    if (ctx->feat_dtype == ART_F32) {
      if ((st = copy_in(ctx, ctx->d_feat, features, n * ctx->C * 4, "copy features")) != ART_OK) return st;
    } else {
      float* t = nullptr;
      if ((st = alloc(ctx, &t, n * ctx->C, "feature staging")) != ART_OK) return st;
      if ((st = copy_in(ctx, t, features, n * ctx->C * 4, "copy features")) != ART_OK) return st;
      const int64_t m = (int64_t)n * ctx->C;
      const unsigned g = (unsigned)((m + 255) / 256);
      if (ctx->feat_dtype == ART_BF16)
        convert_kernel<__nv_bfloat16><<<g, 256, 0, ctx->stream>>>(m, t, (__nv_bfloat16*)ctx->d_feat);
      else
        convert_kernel<__half><<<g, 256, 0, ctx->stream>>>(m, t, (__half*)ctx->d_feat);
      st = sync_check(ctx, "update_voxels");
      cudaFree(t);
      if (st != ART_OK) return st;
    }
  }
  ctx->posed = ctx->posed && !weights && !density;  // the pose records hold sigma and the blend
  return launch_check(ctx, "update_voxels");
}

art_status art_render_backward(art_ctx* ctx, int view, const float* F, const float* A, const float* dF,
                               const float* dA, float* d_features, float* d_density, float* d_weights) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "render_backward before set_pose");
  if (ctx->sh_degree >= 0) return fail(ctx, ART_ERR_UNSUPPORTED, "render_backward: view-dependent (SH) features");
  if (ctx->cfg.index == ART_INDEX_GRID) return fail(ctx, ART_ERR_UNSUPPORTED, "render_backward: the lattice index");
  if (!F || !A || !dF || !d_features || !d_density || !d_weights)
    return fail(ctx, ART_ERR_INVALID_ARG, "null pointer");
  const void* dev[] = {F, A, dF, d_features, d_density, d_weights};
  for (const void* p : dev)
    if (!is_device_ptr(p)) return fail(ctx, ART_ERR_INVALID_ARG, "render_backward takes device arrays");
  if (dA && !is_device_ptr(dA)) return fail(ctx, ART_ERR_INVALID_ARG, "render_backward takes device arrays");
  const ViewParams& v = ctx->views[view];
  art_status st = ensure_bin_buffers(ctx, (int64_t)v.tiles_x * v.tiles_y);
  if (st != ART_OK) return st;
  if ((st = ensure_split_buffers(ctx, (size_t)v.tiles_x * v.tiles_y)) != ART_OK) return st;
  if (ctx->gN_cap < ctx->n) {
    if ((st = alloc(ctx, &ctx->d_gN, (size_t)ctx->n * 12, "geometry gradient")) != ART_OK) return st;
    ctx->gN_cap = ctx->n;
  }
  cudaMemsetAsync(ctx->d_gN, 0, sizeof(float) * 12 * (size_t)ctx->n, ctx->stream);
  launch_project(ctx, v);
  launch_bin(ctx, v);
  if ((st = launch_backward(ctx, v, F, A, dF, dA, d_features, d_density, d_weights)) != ART_OK) return st;
  return launch_check(ctx, "render_backward");
}

art_status art_debug_buffer(art_ctx* ctx, int which, void* dst, int64_t bytes, int64_t* needed) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  art_status st = sync_check(ctx, "debug_buffer");
  if (st != ART_OK) return st;
  const void* src = nullptr;
  int64_t sz = 0;
  unsigned long long ninst = 0;
  cudaMemcpy(&ninst, ctx->d_status + kStInstances, sizeof(ninst), cudaMemcpyDeviceToHost);
  if ((int64_t)ninst > ctx->inst_cap) ninst = (unsigned long long)ctx->inst_cap;
  switch (which) {
    case ART_BUF_JOINT_G: src = ctx->d_G; sz = (int64_t)ctx->J * 12 * 4; break;
    case ART_BUF_VOXEL_REC: src = ctx->d_rec; sz = ctx->n * 64; break;
    case ART_BUF_VOXEL_GEO: src = ctx->d_geo; sz = ctx->n * 64; break;
    case ART_BUF_RECT: src = ctx->d_rect; sz = ctx->n * 8; break;
    case ART_BUF_DEPTHKEY: src = ctx->d_q; sz = ctx->n * 4; break;
    case ART_BUF_KEYS: src = ctx->d_keys; sz = (int64_t)ninst * 4; break;
    case ART_BUF_VALS: src = ctx->d_vals; sz = (int64_t)ninst * 4; break;
    case ART_BUF_RANGES: src = ctx->d_ranges; sz = ctx->ranges_cap * 8; break;
    case ART_BUF_FP8_SCALES: src = ctx->d_f8_scale; sz = ctx->d_f8_scale ? kF8Tensors * 4 : 0; break;
    case ART_BUF_ACTIVATIONS: src = ctx->d_act; sz = ctx->d_act ? (int64_t)ctx->d_act_bytes : 0; break;
    case ART_BUF_BINS: src = ctx->d_bins; sz = ctx->d_bins ? (int64_t)ctx->d_bins_bytes : 0; break;
    case ART_BUF_FALLBACK: {
      unsigned long long nf = 0;
      cudaMemcpy(&nf, ctx->d_status + kStCheckFail, sizeof(nf), cudaMemcpyDeviceToHost);
      src = ctx->d_fbq2;
      sz = ctx->d_fbq2 ? (int64_t)std::min<unsigned long long>(nf, ctx->d_fbq2_bytes / 4) * 4 : 0;
      break;
    }
    case ART_BUF_TAU_HIST: src = ctx->d_thist; sz = ctx->d_thist ? (int64_t)ctx->d_thist_bytes : 0; break;
    default: return fail(ctx, ART_ERR_INVALID_ARG, "unknown buffer %d", which);
  }
  if (needed) *needed = sz;
  if (!dst) return ART_OK;
  if (!src && sz > 0) return fail(ctx, ART_ERR_STATE, "buffer %d not allocated yet", which);
  if (bytes < sz) return fail(ctx, ART_ERR_INVALID_ARG, "buffer needs %lld bytes", (long long)sz);
  if (sz > 0) {
    cudaError_t e = cudaMemcpy(dst, src, (size_t)sz, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "debug_buffer copy");
  }
  return ART_OK;
}

art_status art_debug_hits(art_ctx* ctx, int view, int cap, int32_t* count, uint32_t* ids, float* t0, float* t1,
                          float* F, float* A) {
  if (!ctx) return ART_ERR_INVALID_ARG;
  if (view < 0 || view >= kMaxViews || !ctx->view_set[view]) return fail(ctx, ART_ERR_STATE, "view %d not set", view);
  if (!ctx->posed) return fail(ctx, ART_ERR_STATE, "debug_hits before set_pose");
  if (cap < 1 || !count || !ids || !t0 || !t1) return fail(ctx, ART_ERR_INVALID_ARG, "bad hit-log arguments");
  const ViewParams& v = ctx->views[view];
  size_t npx = (size_t)v.W * v.H;
  int32_t* dc = nullptr;
  uint32_t* di = nullptr;
  float *d0 = nullptr, *d1 = nullptr, *dF = nullptr, *dA = nullptr;
  art_status st = ART_OK;
  if ((st = alloc(ctx, &dc, npx, "hit counts")) == ART_OK && (st = alloc(ctx, &di, npx * cap, "hit ids")) == ART_OK &&
      (st = alloc(ctx, &d0, npx * cap, "hit t0")) == ART_OK && (st = alloc(ctx, &d1, npx * cap, "hit t1")) == ART_OK &&
      (st = alloc(ctx, &dF, npx * ctx->C, "F")) == ART_OK && (st = alloc(ctx, &dA, npx, "A")) == ART_OK) {
    st = ensure_bin_buffers(ctx, (int64_t)v.tiles_x * v.tiles_y);
    if (st == ART_OK) {
      void* log = make_hit_log(dc, di, d0, d1, cap);
      launch_project(ctx, v);
      launch_bin(ctx, v);
      st = launch_composite(ctx, v, dF, ART_F32, dA, log);
      free_hit_log(log);
    }
    if (st == ART_OK) st = sync_check(ctx, "debug_hits");
    if (st == ART_OK) {
      cudaMemcpy(count, dc, npx * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(ids, di, npx * cap * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(t0, d0, npx * cap * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(t1, d1, npx * cap * 4, cudaMemcpyDeviceToHost);
      if (F) cudaMemcpy(F, dF, npx * ctx->C * 4, cudaMemcpyDeviceToHost);
      if (A) cudaMemcpy(A, dA, npx * 4, cudaMemcpyDeviceToHost);
    }
  }
  void* ptrs[] = {dc, di, d0, d1, dF, dA};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  return st;
}

}  // extern "C"
