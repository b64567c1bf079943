// Depth buffer of the rendered animal (arXiv 2202.05628, Sec. 3.1 "Hybrid
// Rendering": a pixel's depth is how far along its ray the nearest voxel
// denser than a set threshold lies).  Here:
// the entry distance t0 (from the camera centre along the unit ray, inside
// [near, far]) of the nearest hit with sigma > sigma_min among all of the
// ray's hits, +inf where there is none.
#include "raster.cuh"

namespace art {
namespace {

// One warp per 8x4 tile, lane = pixel, over the tile's (tile, depth)-ordered
// list in chunks of 32 entries staged in shared memory (dense voxels only);
// each lane tests exactly the voxels whose rectangle covers its pixel
// (transposed coverage masks) and keeps its nearest entry.  The list is
// ordered by a lower bound of each voxel's distance from the camera centre,
// so the walk ends once a chunk's first bound reaches every pixel's nearest
// hit so far.
__global__ void __launch_bounds__(32) depth_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                                                   const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                                                   const short4* __restrict__ rect, ViewParams v, float sigma_min,
                                                   float* __restrict__ depth) {
  __shared__ float4 s_b0[NT], s_b1[NT], s_b2[NT], s_xl[NT];
  __shared__ uint32_t s_mask[NT];
  __shared__ float s_bound;
  const int tile = blockIdx.x, lane = threadIdx.x & 31;
  const int sx = (tile % v.tiles_x) * TSX, sy = (tile / v.tiles_x) * TSY;
  const int px = sx + (lane & 7), py = sy + (lane >> 3);
  const bool inside = px < v.W && py < v.H;
  const RayDir rd = pixel_ray(v, px, py);
  float best = __int_as_float(0x7f800000);  // +inf
  const uint2 rg = ranges[tile];
  const uint32_t qmask = (1u << v.depth_bits) - 1u;
  const float qinv = 1.0f / v.dscale;
  for (uint32_t base = rg.x; base < rg.y; base += NT) {
    __syncwarp();
    const uint32_t k = base + lane;
    uint32_t m = 0;
    if (k < rg.y) {
      const uint32_t vid = vals[k];
      const float4* rp = rec + 4 * (size_t)vid;
      const float4 r3 = rp[3];
      if (r3.x > sigma_min) {
        const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2];
        stage_voxel(r0, r1, r2, v, s_b0[lane], s_b1[lane], s_b2[lane], s_xl[lane]);
        m = rect_mask(rect[vid], sx, sy);
      }
    }
    s_mask[lane] = m;
    if (lane == 0) s_bound = v.znear + (float)(keys[base] & qmask) * qinv;
    __syncwarp();
    // every entry of this chunk and of the later ones enters at t >= its first bound
    if (__all_sync(0xffffffffu, !inside || best <= s_bound)) break;
    uint32_t cand = transpose32(s_mask[lane], lane);
    while (cand) {
      const int idx = __ffs(cand) - 1;
      cand &= cand - 1;
      float t0, dl, e[3];
      int ax0, ax1;
      if (slab_hit(s_b0[idx], s_b1[idx], s_b2[idx], s_xl[idx], rd, v.znear, v.zfar, t0, dl, ax0, ax1, e))
        best = fminf(best, t0);
    }
  }
  if (inside) depth[(size_t)py * v.W + px] = best;
}

}  // namespace

void launch_depth(art_ctx* ctx, const ViewParams& v, float sigma_min, float* depth) {
  const int ntiles = v.tiles_x * v.tiles_y;
  ART_LAUNCH(ctx, "depth", depth_kernel, ntiles, 32, 0, ctx->d_ranges, ctx->d_keys, ctx->d_vals, ctx->d_rec,
             ctx->d_rect, v, sigma_min, depth);
}

}  // namespace art
