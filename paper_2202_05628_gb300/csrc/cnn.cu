// Neural shading network (arXiv 2202.05628, Sec. 3.1 "Neural Shading"):
// layer orchestration and the CUDA-core implicit-GEMM convolution used for the
// FP32 form.  The BF16 form runs its 3x3 layers on the tensor cores
// (cnn_tc.cu).
#include <type_traits>

#include "internal.cuh"

namespace art {

// Convolution arguments shared by the CUDA-core and tensor-core kernels.
// The input is the channel concatenation [src0, src1] (NHWC); src0 may be
// read through a nearest x2 upsample (its tensor is H/2 x W/2).
struct ConvArgs {
  const void* src0;
  int c0, up0;
  const void* src1;
  int c1;
  int H, W;
  int cout, k, act;
  const float* w;  // [cout][k][k][cin] FP32
  const float* b;  // [cout]
  void* out;       // [H][W][out_ld], channels [out_off, out_off + cout)
  int out_f32;     // output element type FP32 (else the activation type)
  int out_ld, out_off;
};

namespace {

__device__ __forceinline__ float ld_act(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_act(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }
__device__ __forceinline__ void st_act(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_act(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float activate(float v, int act) {
  if (act == 1) return fmaxf(v, 0.0f);
  if (act == 2) return 1.0f / (1.0f + expf(-v));
  return v;
}

// Implicit GEMM on CUDA cores: a CTA computes 64 consecutive pixels of one
// row x 64 output channels; K runs over taps x 16-channel chunks.
template <typename TI>
__global__ void __launch_bounds__(256) conv_simt_kernel(ConvArgs a) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tpr = (a.W + BM - 1) / BM;
  const int y = blockIdx.x / tpr;
  const int x0 = (blockIdx.x % tpr) * BM;
  const int co0 = blockIdx.y * BN;
  const int tm = tid & 15, tn = tid >> 4;
  const int cin = a.c0 + a.c1;
  const int pad = a.k / 2;
  const TI* s0 = (const TI*)a.src0;
  const TI* s1 = (const TI*)a.src1;
  const int H0 = a.up0 ? a.H / 2 : a.H, W0 = a.up0 ? a.W / 2 : a.W;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  for (int tap = 0; tap < a.k * a.k; ++tap) {
    const int r = tap / a.k, s = tap % a.k;
    const int yy = y + r - pad;
    for (int cb = 0; cb < cin; cb += BK) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int idx = tid + 256 * e;
        int c = idx & 15, i = idx >> 4;
        int xx = x0 + i + s - pad, ch = cb + c;
        float val = 0.0f;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && ch < cin) {
          if (ch < a.c0) {
            int y0 = a.up0 ? yy >> 1 : yy, xs = a.up0 ? xx >> 1 : xx;
            val = ld_act(s0 + ((size_t)y0 * W0 + xs) * a.c0 + ch);
          } else {
            val = ld_act(s1 + ((size_t)yy * a.W + xx) * a.c1 + (ch - a.c0));
          }
        }
        As[c][i] = val;
        int j = idx >> 4, co = co0 + j;
        Bs[c][j] = (co < a.cout && ch < cin) ? __ldg(a.w + (((size_t)co * a.k + r) * a.k + s) * cin + ch) : 0.0f;
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < BK; ++c) {
        float av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[c][tm + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[c][tn + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  (void)H0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int x = x0 + tm + 16 * i;
    if (x >= a.W) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int co = co0 + tn + 16 * j;
      if (co >= a.cout) continue;
      float v = activate(acc[i][j] + a.b[co], a.act);
      size_t o = ((size_t)y * a.W + x) * a.out_ld + a.out_off + co;
      if (a.out_f32)
        ((float*)a.out)[o] = v;
      else
        st_act((TI*)a.out + o, v);
    }
  }
}

// FP32 implicit GEMM on CUDA cores for the FP32 network: a CTA computes BM
// consecutive pixels of one row x BN output channels (128 x 64, or 256 x 32
// for the 32-channel layers), a thread 8 pixels (4 t .. 4 t + 3 and the same
// BM / 2 further, so that a warp's 16-byte reads of a K row are contiguous)
// x 4 channels: 32 FMAs per three 16-byte shared-memory reads; K runs over
// taps x 16-channel chunks,
// double-buffered in shared memory (one barrier per chunk) with the next
// chunk's global loads (16 B: four channels of one pixel) in flight while the
// current one is multiplied.  Needs channel counts and output offsets that
// are multiples of 4 (16-byte rows); the layer's zero padding is the
// out-of-image pixels loading as zeros.
template <int BM, int BN>
__global__ void __launch_bounds__(256) conv_f32_kernel(ConvArgs a) {
  constexpr int BK = 16, TM = 8, TN = 4, NT = 256;
  constexpr int NTM = BM / TM;  // threads along the pixels
  static_assert(NTM * (BN / TN) == NT, "256 threads tile BM x BN");
  constexpr int A_F4 = BM * BK / 4 / NT;        // 16-byte A loads per thread and chunk
  constexpr int B_F4 = BN * BK / 4;             // 16-byte B loads per chunk (threads below it)
  static_assert(B_F4 <= NT, "one B load per thread");
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tm = tid % NTM, tn = tid / NTM;
  const int tpr = (a.W + BM - 1) / BM;
  const int y = blockIdx.x / tpr;
  const int x0 = (blockIdx.x % tpr) * BM;
  const int co0 = blockIdx.y * BN;
  const int cin = a.c0 + a.c1;
  const int pad = a.k / 2;
  const float* s0 = (const float*)a.src0;
  const float* s1 = (const float*)a.src1;
  const int W0 = a.up0 ? a.W / 2 : a.W;
  const int nch = (cin + BK - 1) / BK;
  const int nk = a.k * a.k * nch;

  float4 ra[A_F4], rb;
  auto load = [&](int kk) {
    const int tap = kk / nch, cb = (kk - tap * nch) * BK;
    const int r = tap / a.k, sx = tap - r * a.k;
    const int yy = y + r - pad;
#pragma unroll
    for (int e = 0; e < A_F4; ++e) {
      const int f = tid + NT * e, i = f >> 2, ch = cb + 4 * (f & 3);
      const int xx = x0 + i + sx - pad;
      float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && ch < cin) {
        if (ch < a.c0) {
          const int ys = a.up0 ? yy >> 1 : yy, xs = a.up0 ? xx >> 1 : xx;
          v = __ldg(reinterpret_cast<const float4*>(s0 + ((size_t)ys * W0 + xs) * a.c0 + ch));
        } else {
          v = __ldg(reinterpret_cast<const float4*>(s1 + ((size_t)yy * a.W + xx) * a.c1 + (ch - a.c0)));
        }
      }
      ra[e] = v;
    }
    rb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (tid < B_F4) {
      const int co = co0 + (tid >> 2), ch = cb + 4 * (tid & 3);
      if (co < a.cout && ch < cin)
        rb = __ldg(reinterpret_cast<const float4*>(a.w + (((size_t)co * a.k + r) * a.k + sx) * cin + ch));
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < A_F4; ++e) {
      const int f = tid + NT * e, i = f >> 2, c = 4 * (f & 3);
      As[buf][c][i] = ra[e].x;
      As[buf][c + 1][i] = ra[e].y;
      As[buf][c + 2][i] = ra[e].z;
      As[buf][c + 3][i] = ra[e].w;
    }
    if (tid < B_F4) {
      const int j = tid >> 2, c = 4 * (tid & 3);
      Bs[buf][c][j] = rb.x;
      Bs[buf][c + 1][j] = rb.y;
      Bs[buf][c + 2][j] = rb.z;
      Bs[buf][c + 3][j] = rb.w;
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;
  load(0);
  store(0);
  __syncthreads();
  for (int kk = 0; kk < nk; ++kk) {
    const int buf = kk & 1;
    if (kk + 1 < nk) load(kk + 1);  // in flight while this chunk is multiplied
#pragma unroll
    for (int c = 0; c < BK; ++c) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][c][4 * tm]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][c][BM / 2 + 4 * tm]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][c][tn * TN]);
      const float av[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[TN] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kk + 1 < nk) store(buf ^ 1);  // (the other buffer was last read before the previous barrier)
    __syncthreads();
  }
  const int cb0 = co0 + tn * TN;
  float bias[TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) bias[j] = cb0 + j < a.cout ? a.b[cb0 + j] : 0.0f;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int x = x0 + (i < 4 ? 4 * tm + i : BM / 2 + 4 * tm + i - 4);
    if (x >= a.W) continue;
    float v[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) v[j] = activate(acc[i][j] + bias[j], a.act);
    float* o = (float*)a.out + ((size_t)y * a.W + x) * a.out_ld + a.out_off + cb0;
    if (cb0 + TN <= a.cout) {
      *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int j = 0; j < TN; ++j)
        if (cb0 + j < a.cout) o[j] = v[j];
    }
  }
}

template <typename T>
__global__ void maxpool2_kernel(const T* __restrict__ in, T* __restrict__ out, int H, int W, int C) {
  int64_t total = (int64_t)(H / 2) * (W / 2) * C;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(idx % C);
    int64_t p = idx / C;
    int x = (int)(p % (W / 2)), y = (int)(p / (W / 2));
    const T* q = in + (((size_t)(2 * y) * W) + 2 * x) * C + c;
    float m = fmaxf(fmaxf(ld_act(q), ld_act(q + C)), fmaxf(ld_act(q + (size_t)W * C), ld_act(q + (size_t)W * C + C)));
    st_act(out + idx, m);
  }
}

template <typename TI>
void conv(art_ctx* ctx, const ConvArgs& a, const ConvLayer& L) {
  (void)L;
  // FP32 activations in and out, 16-byte channel rows: the register-blocked kernel
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool f32_ok = std::is_same<TI, float>::value && a.c0 % 4 == 0 && a.c1 % 4 == 0 && a.out_ld % 4 == 0 &&
                      a.out_off % 4 == 0 && al16(a.out) && al16(a.src0) && al16(a.src1) && al16(a.w) &&
                      (a.up0 == 0 || (a.W % 2 == 0 && a.H % 2 == 0));
  if (f32_ok) {
    if (a.cout <= 32) {
      dim3 grid(((a.W + 255) / 256) * a.H, (a.cout + 31) / 32);
      auto kfn = conv_f32_kernel<256, 32>;
      ART_LAUNCH(ctx, "conv_simt", kfn, grid, 256, 0, a);
    } else {
      dim3 grid(((a.W + 127) / 128) * a.H, (a.cout + 63) / 64);
      auto kfn = conv_f32_kernel<128, 64>;
      ART_LAUNCH(ctx, "conv_simt", kfn, grid, 256, 0, a);
    }
    return;
  }
  int tpr = (a.W + 63) / 64;
  dim3 grid(tpr * a.H, (a.cout + 63) / 64);
  auto kfn = conv_simt_kernel<TI>;
  ART_LAUNCH(ctx, "conv_simt", kfn, grid, 256, 0, a);
}

template <typename TI>
void pool(art_ctx* ctx, const void* in, void* out, int H, int W, int C) {
  int64_t total = (int64_t)(H / 2) * (W / 2) * C;
  int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 16);
  auto kfn = maxpool2_kernel<TI>;
  ART_LAUNCH(ctx, "maxpool2", kfn, grid, 256, 0, (const TI*)in, (TI*)out, H, W, C);
}

template <typename TI>
ConvArgs conv_args(const void* s0, int c0, int up0, const void* s1, int c1, int h, int w, const ConvLayer& l,
                   void* out, int act, int out_f32, int out_ld = -1, int out_off = 0) {
  ConvArgs a;
  a.src0 = s0;
  a.c0 = c0;
  a.up0 = up0;
  a.src1 = s1;
  a.c1 = c1;
  a.H = h;
  a.W = w;
  a.cout = l.cout;
  a.k = l.k;
  a.act = act;
  a.w = l.w32;
  a.b = l.b32;
  a.out = out;
  a.out_f32 = out_f32;
  a.out_ld = out_ld < 0 ? l.cout : out_ld;
  a.out_off = out_off;
  return a;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of the CUDA-core U-Net's activations: per level two block outputs
// and the pooled copy, per decoder level two block outputs.
size_t unet_simt_bytes(int H, int W, int levels, const int* ch, size_t es) {
  size_t t = 0;
  for (int l = 0; l < levels; ++l) {
    const size_t px = (size_t)(H >> l) * (W >> l);
    t += 2 * align256(px * ch[l] * es);
    if (l + 1 < levels) t += align256(px / 4 * ch[l] * es) + 2 * align256(px * ch[l] * es);
  }
  return t;
}

// U-Net of `levels` levels on the CUDA cores, layers[lb ...] in the order
// enc0 a/b, ..., bottleneck a/b, dec(levels-2) a/b, ..., dec0 a/b, 1x1 head
// (Sec. 3.1 "Neural Shading"; per level two conv3x3 + ReLU, 2x2 max pooling
// down, nearest x2 up with the concatenation [upsampled, skip], sigmoid
// head).  The head writes its cout channels at out_off of out_ld FP32 values
// per pixel.  Activations live in the arena from byte arena_off on.
template <typename TI>
art_status unet_simt(art_ctx* ctx, int H, int W, const void* in, int cin, int lb, int levels, const int* ch,
                     float* out, int out_ld, int out_off, size_t arena_off) {
  const size_t es = sizeof(TI);
  const size_t need = arena_off + unet_simt_bytes(H, W, levels, ch, es);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, need, "activations") != ART_OK) return ART_ERR_OOM;
  size_t off = arena_off;
  auto take = [&](int l, int c, int shift) {
    void* p = (char*)ctx->d_act + off;
    off += align256((size_t)(H >> (l + shift)) * (W >> (l + shift)) * c * es);
    return p;
  };
  auto L = [&](int i) -> const ConvLayer& { return ctx->layers[lb + i]; };
  void* skip[4] = {};
  const void* x = in;
  int xc = cin;
  int li = 0;
  for (int l = 0; l < levels; ++l) {  // encoder
    const int h = H >> l, w = W >> l;
    void* a = take(l, ch[l], 0);
    void* b = take(l, ch[l], 0);
    conv<TI>(ctx, conv_args<TI>(x, xc, 0, nullptr, 0, h, w, L(li), a, 1, 0), L(li));
    conv<TI>(ctx, conv_args<TI>(a, ch[l], 0, nullptr, 0, h, w, L(li + 1), b, 1, 0), L(li + 1));
    li += 2;
    skip[l] = b;
    if (l + 1 < levels) {
      void* pooled = take(l, ch[l], 1);
      pool<TI>(ctx, b, pooled, h, w, ch[l]);
      x = pooled;
      xc = ch[l];
    }
  }
  const void* d = skip[levels - 1];
  for (int l = levels - 2; l >= 0; --l) {  // decoder: [up(d), skip_l]
    const int h = H >> l, w = W >> l;
    void* a = take(l, ch[l], 0);
    void* b = take(l, ch[l], 0);
    conv<TI>(ctx, conv_args<TI>(d, ch[l + 1], 1, skip[l], ch[l], h, w, L(li), a, 1, 0), L(li));
    conv<TI>(ctx, conv_args<TI>(a, ch[l], 0, nullptr, 0, h, w, L(li + 1), b, 1, 0), L(li + 1));
    li += 2;
    d = b;
  }
  conv<TI>(ctx, conv_args<TI>(d, ch[0], 0, nullptr, 0, H, W, L(li), out, 2, 1, out_ld, out_off), L(li));
  return ART_OK;
}

// The opacity branch's input [A, I_f] of the two-branch network: channel 0
// the coarse opacity A, channels 1..3 the appearance branch's image (FP32
// RGB of rgba [H][W][4]), channels 4 .. C-1 zero (padding for the tensor
// cores' K granularity).
template <typename TI, int C>
__global__ void __launch_bounds__(256) pack_opacity_input_kernel(int64_t npx, const float* __restrict__ A,
                                                                 const float* __restrict__ rgba, TI* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npx) return;
  const float4 c = reinterpret_cast<const float4*>(rgba)[i];
  float v[C];
#pragma unroll
  for (int k = 0; k < C; ++k) v[k] = 0.0f;
  v[0] = A[i];
  v[1] = c.x;
  v[2] = c.y;
  v[3] = c.z;
  TI* o = x + i * C;
#pragma unroll
  for (int k = 0; k < C; ++k) st_act(o + k, v[k]);
}

template <typename TI, int C>
void pack_opacity_input(art_ctx* ctx, int64_t npx, const float* A, const float* rgba, TI* x) {
  auto kfn = pack_opacity_input_kernel<TI, C>;
  ART_LAUNCH(ctx, "pack_opacity_input", kfn, (unsigned)((npx + 255) / 256), 256, 0, npx, A, rgba, x);
}

template <typename TI>
art_status run_typed(art_ctx* ctx, const ViewParams& v, const void* F, const float* A, float* rgba) {
  const int H = v.H, W = v.W;
  const art_net_desc& nd = ctx->net;
  auto L = [&](int i) -> const ConvLayer& { return ctx->layers[i]; };
  const size_t es = sizeof(TI);
  if (nd.arch == ART_NET_TINY) {
    int c = nd.ch[0];
    size_t need = 2 * (size_t)H * W * c * es;
    if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, need, "activations") != ART_OK) return ART_ERR_OOM;
    char* b0 = (char*)ctx->d_act;
    char* b1 = b0 + (size_t)H * W * c * es;
    conv<TI>(ctx, conv_args<TI>(F, nd.cin, 0, nullptr, 0, H, W, L(0), b0, 1, 0), L(0));
    conv<TI>(ctx, conv_args<TI>(b0, c, 0, nullptr, 0, H, W, L(1), b1, 1, 0), L(1));
    conv<TI>(ctx, conv_args<TI>(b1, c, 0, nullptr, 0, H, W, L(2), rgba, 2, 1), L(2));
    return ART_OK;
  }
  if (nd.arch == ART_NET_UNET) return unet_simt<TI>(ctx, H, W, F, nd.cin, 0, 4, nd.ch, rgba, nd.cout, 0, 0);
  // two branches: appearance F -> I_f (rgba channels 0..2), opacity [A, I_f] -> alpha (channel 3)
  art_status st = unet_simt<TI>(ctx, H, W, F, nd.cin, 0, 4, nd.ch, rgba, 4, 0, 0);
  if (st != ART_OK) return st;
  const int64_t npx = (int64_t)H * W;
  const size_t xb = align256((size_t)npx * 4 * es);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, xb + unet_simt_bytes(H, W, 2, nd.ach, es), "activations") != ART_OK)
    return ART_ERR_OOM;
  pack_opacity_input<TI, 4>(ctx, npx, A, rgba, (TI*)ctx->d_act);
  return unet_simt<TI>(ctx, H, W, ctx->d_act, 4, 15, 2, nd.ach, rgba, 4, 3, xb);
}

// Bytes of the tensor-core U-Net's activations (unet_tc's tensors).
size_t unet_tc_bytes(int H, int W, int levels, const int* ch) {
  size_t t = 0;
  for (int l = 0; l + 1 < levels; ++l) {
    const size_t px = (size_t)(H >> l) * (W >> l);
    t += align256(px * ch[l] * 2) + align256(px * (ch[l + 1] + ch[l]) * 2) + align256(px / 4 * ch[l] * 2);
  }
  t += align256((size_t)(H >> (levels - 1)) * (W >> (levels - 1)) * ch[levels - 1] * 2);
  for (int l = levels - 2; l >= 0; --l) t += align256((size_t)(H >> l) * (W >> l) * ch[l] * 2);
  return t;
}

// BF16 U-Net of `levels` levels on the tensor cores, layers[lb ...] in the
// order of unet_simt.  Skip connections and upsampled decoder inputs are
// written straight into per-level concatenation buffers
// cat_l = [up(decoder below) | encoder skip] by the producing convolutions'
// epilogues, so every decoder convolution reads one dense tensor; the last
// convolution carries the 1x1 head + sigmoid in its epilogue, into head_n
// FP32 channels at head_off of head_ld per pixel.  A decoder convolution
// runs in its sub-pixel form when its layer has the blocks (level 0:
// launch_sub_conv; levels 1 and 2: the tap-by-tap kernel): cat_l's space then
// holds the skip tensor, x-phase split, and the block output of level l + 1
// at its own resolution (no 2x2-replicated copy).  Arena order (from arena_off): e0a, cat0, p0, e1a,
// cat1, p1, ..., bottleneck a, then the decoders' first outputs from the
// deepest level up.
art_status unet_tc(art_ctx* ctx, int H, int W, const __nv_bfloat16* in, int cin, int lb, int levels, const int* ch,
                   float* out, int head_n, int head_ld, int head_off, size_t arena_off) {
  const size_t need = arena_off + unet_tc_bytes(H, W, levels, ch);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, need, "activations") != ART_OK) return ART_ERR_OOM;
  size_t off = arena_off;
  auto take = [&](int l, int c, int shift) {
    __nv_bfloat16* p = (__nv_bfloat16*)((char*)ctx->d_act + off);
    off += align256((size_t)(H >> (l + shift)) * (W >> (l + shift)) * c * 2);
    return p;
  };
  __nv_bfloat16 *ea[4] = {}, *cat[4] = {}, *pl[4] = {}, *da[4] = {};
  for (int l = 0; l + 1 < levels; ++l) {
    ea[l] = take(l, ch[l], 0);
    cat[l] = take(l, ch[l + 1] + ch[l], 0);
    pl[l] = take(l, ch[l], 1);
  }
  ea[levels - 1] = take(levels - 1, ch[levels - 1], 0);
  for (int l = levels - 2; l >= 0; --l) da[l] = take(l, ch[l], 0);
  const auto& Ls = ctx->layers;
  const int head = lb + 4 * levels - 2;
  // decoder convolutions in the sub-pixel form (level 0: conv_sub_kernel;
  // levels >= 1: the tap-by-tap kernel): their skip input (x-phase split) and
  // their low-resolution input, both in cat_l's space
  bool sub[4] = {};
  __nv_bfloat16 *sk[4] = {}, *ul[4] = {};
  for (int l = 0; l + 1 < levels && !ctx->cfg.no_subpixel; ++l) {
    const ConvLayer& L = Ls[lb + 2 * levels + 2 * (levels - 2 - l)];
    const int h = H >> l, w = W >> l;
    if (l == 0) {
      sub[0] = L.wsub && L.sub_cs == ch[0] && L.sub_cu == ch[1] && ctx->conv_rows &&
               sub_conv_ok(L.cout, ch[0], ch[1], h, w);
    } else {
      TcConv t{};
      t.sub = 1;
      t.cs = ch[l];
      t.cu = ch[l + 1];
      t.cin = ch[l] + ch[l + 1];
      t.cout = L.cout;
      t.H = h;
      t.W = w;
      t.ld_out = L.cout;
      sub[l] = L.wtap && L.sub_cs == ch[l] && L.sub_cu == ch[l + 1] && tc_conv_ok(t);
    }
  }
  for (int l = 0; l + 1 < levels; ++l) {
    sk[l] = cat[l];
    ul[l] = (__nv_bfloat16*)((char*)cat[l] + align256((size_t)(H >> l) * (W >> l) * ch[l] * 2));
  }
  int psplit = 0;
  auto conv = [&](const __nv_bfloat16* x, int xc, int l, int li, __nv_bfloat16* o, int ld, int o_off, int up2,
                  bool to_head, __nv_bfloat16* pooled) {
    TcConv c;
    c.in = x;
    c.cin = xc;
    c.H = H >> l;
    c.W = W >> l;
    c.w = Ls[lb + li].wbf;
    c.bias = Ls[lb + li].b32;
    c.cout = Ls[lb + li].cout;
    c.act = 1;
    c.out = o;
    c.ld_out = ld;
    c.ch_off = o_off;
    c.up2 = up2;
    c.rgba = to_head ? out : nullptr;
    c.head_w = to_head ? Ls[head].w32 : nullptr;
    c.head_b = to_head ? Ls[head].b32 : nullptr;
    c.head_n = head_n;
    c.head_ld = head_ld;
    c.head_off = head_off;
    c.pool = pooled;
    c.psplit = psplit;
    return launch_tc_conv(ctx, c);
  };
  // the block output of level l + 1 that level l's decoder reads upsampled
  auto up_into = [&](const __nv_bfloat16* x, int l, int li) {
    if (sub[l]) return conv(x, ch[l + 1], l + 1, li, ul[l], ch[l + 1], 0, 0, false, nullptr);
    return conv(x, ch[l + 1], l + 1, li, cat[l], ch[l + 1] + ch[l], 0, 1, false, nullptr);
  };
  art_status st = ART_OK;
#define ART_TRY(x)                  \
  if ((st = (x)) != ART_OK) return st
  const __nv_bfloat16* x = in;
  int xc = cin;
  for (int l = 0; l + 1 < levels; ++l) {  // encoder: the block output goes into cat_l as the skip, + 2x2 pooling
    ART_TRY(conv(x, xc, l, 2 * l, ea[l], ch[l], 0, 0, false, nullptr));
    if (sub[l]) {  // dense and x-phase split for the sub-pixel decoder convolution
      psplit = 1;
      st = conv(ea[l], ch[l], l, 2 * l + 1, sk[l], ch[l], 0, 0, false, pl[l]);
      psplit = 0;
      if (st != ART_OK) return st;
    } else {
      ART_TRY(conv(ea[l], ch[l], l, 2 * l + 1, cat[l], ch[l + 1] + ch[l], ch[l + 1], 0, false, pl[l]));
    }
    x = pl[l];
    xc = ch[l];
  }
  const int lL = levels - 1;  // bottleneck: its block output goes up x2 into cat of the level above
  ART_TRY(conv(x, xc, lL, 2 * lL, ea[lL], ch[lL], 0, 0, false, nullptr));
  ART_TRY(up_into(ea[lL], lL - 1, 2 * lL + 1));
  int li = 2 * levels;
  for (int l = levels - 2; l >= 0; --l, li += 2) {
    const ConvLayer& L = Ls[lb + li];
    if (l == 0 && sub[0]) {
      SubConv sc;
      sc.skip = sk[0];
      sc.cs = ch[0];
      sc.up = ul[0];
      sc.cu = ch[1];
      sc.H = H;
      sc.W = W;
      sc.w = L.wsub;
      sc.bias = L.b32;
      sc.out = da[0];
      ART_TRY(launch_sub_conv(ctx, sc));
    } else if (sub[l]) {
      TcConv c{};
      c.sub = 1;
      c.in = sk[l];
      c.cs = ch[l];
      c.up = ul[l];
      c.cu = ch[l + 1];
      c.cin = ch[l] + ch[l + 1];
      c.H = H >> l;
      c.W = W >> l;
      c.w = L.wtap;
      c.bias = L.b32;
      c.cout = L.cout;
      c.act = 1;
      c.out = da[l];
      c.ld_out = L.cout;
      ART_TRY(launch_tc_conv(ctx, c));
    } else {
      ART_TRY(conv(cat[l], ch[l + 1] + ch[l], l, li, da[l], ch[l], 0, 0, false, nullptr));
    }
    if (l > 0) {
      ART_TRY(up_into(da[l], l - 1, li + 1));  // up x2
    } else {
      ART_TRY(conv(da[0], ch[0], 0, li + 1, nullptr, 0, 0, 0, true, nullptr));  // + fused 1x1 head, sigmoid
    }
  }
#undef ART_TRY
  return ART_OK;
}

// Both branches of the two-branch network on the tensor cores; the
// opacity branch's first layer carries BF16 weights padded to 32 input
// channels (the packed [A, I_f, 0 ...] tensor).
art_status run_two_branch_tc(art_ctx* ctx, const ViewParams& v, const __nv_bfloat16* F, const float* A, float* rgba) {
  const int H = v.H, W = v.W;
  const art_net_desc& nd = ctx->net;
  art_status st = unet_tc(ctx, H, W, F, nd.cin, 0, 4, nd.ch, rgba, 3, 4, 0, 0);
  if (st != ART_OK) return st;
  const int64_t npx = (int64_t)H * W;
  const size_t xb = align256((size_t)npx * kOpacityPad * 2);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, xb + unet_tc_bytes(H, W, 2, nd.ach), "activations") != ART_OK)
    return ART_ERR_OOM;
  pack_opacity_input<__nv_bfloat16, kOpacityPad>(ctx, npx, A, rgba, (__nv_bfloat16*)ctx->d_act);
  return unet_tc(ctx, H, W, (const __nv_bfloat16*)ctx->d_act, kOpacityPad, 15, 2, nd.ach, rgba, 1, 4, 3, xb);
}

// FP8 (E4M3) U-Net on the tensor cores (kind::f8f6f4), same dataflow as
// unet_tc.  Activation tensors carry one scale each (a concatenation
// buffer and its pooled copy share one); every call quantises with the scales
// measured on the previous call (delayed per-tensor scaling from max |value|)
// and records this call's maxima.  The first call after loading calibrates:
// it runs once with unit scales to measure the maxima, then again.
art_status run_unet_f8(art_ctx* ctx, const ViewParams& v, const __nv_bfloat16* F, float* rgba) {
  const int H = v.H, W = v.W;
  const art_net_desc& nd = ctx->net;
  const int c0 = nd.ch[0], c1 = nd.ch[1], c2 = nd.ch[2], c3 = nd.ch[3];
  struct Buf {
    int h, w, c;
    size_t off;
  };
  std::vector<Buf> bufs;
  size_t total = 0;
  auto add = [&](int h, int w, int c) {
    bufs.push_back(Buf{h, w, c, total});
    total += ((size_t)h * w * c + 255) & ~(size_t)255;
    return (int)bufs.size() - 1;
  };
  const int fin = add(H, W, nd.cin);
  const int e0a = add(H, W, c0), cat0 = add(H, W, c1 + c0), p0 = add(H / 2, W / 2, c0);
  const int e1a = add(H / 2, W / 2, c1), cat1 = add(H / 2, W / 2, c2 + c1), p1 = add(H / 4, W / 4, c1);
  const int e2a = add(H / 4, W / 4, c2), cat2 = add(H / 4, W / 4, c3 + c2), p2 = add(H / 8, W / 8, c2);
  const int e3a = add(H / 8, W / 8, c3);
  const int d2a = add(H / 4, W / 4, c2), d1a = add(H / 2, W / 2, c1), d0a = add(H, W, c0);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, total, "activations") != ART_OK) return ART_ERR_OOM;
  auto P = [&](int i) { return (uint8_t*)ctx->d_act + bufs[i].off; };
  // scale slots: 0 input, 1 e0a, 2 cat0/p0, 3 e1a, 4 cat1/p1, 5 e2a, 6 cat2/p2, 7 e3a, 8 d2a, 9 d1a, 10 d0a
  float* sc = ctx->d_f8_scale;
  unsigned int* am = ctx->d_f8_amax;
  const auto& L = ctx->layers;
  auto conv = [&](int in, int sin, int cin, int h, int w, int li, int out, int sout, int ld, int off, int up2,
                  float* head_out, int pooled = -1) {
    TcConv c;
    c.in = P(in);
    c.cin = cin;
    c.H = h;
    c.W = w;
    c.w = L[li].w8;
    c.bias = L[li].b32;
    c.cout = L[li].cout;
    c.act = 1;
    c.out = out >= 0 ? P(out) : nullptr;
    c.ld_out = ld;
    c.ch_off = off;
    c.up2 = up2;
    c.rgba = head_out;
    c.head_w = head_out ? L[14].w32 : nullptr;
    c.head_b = head_out ? L[14].b32 : nullptr;
    c.f8 = true;
    c.in_scale = sc + sin;
    c.w_scale = L[li].wscale;
    c.out_scale = out >= 0 ? sc + sout : nullptr;
    c.out_amax = out >= 0 ? am + sout : nullptr;
    c.pool = pooled >= 0 ? P(pooled) : nullptr;  // (shares the output's scale)
    return launch_tc_conv(ctx, c);
  };
  auto network = [&]() -> art_status {
    art_status st = ART_OK;
#define ART_TRY(x)                  \
  if ((st = (x)) != ART_OK) return st
    launch_quantize_input(ctx, F, (int64_t)H * W * nd.cin, sc + 0, P(fin), am + 0);
    ART_TRY(conv(fin, 0, nd.cin, H, W, 0, e0a, 1, c0, 0, 0, nullptr));
    ART_TRY(conv(e0a, 1, c0, H, W, 1, cat0, 2, c1 + c0, c1, 0, nullptr, p0));
    ART_TRY(conv(p0, 2, c0, H / 2, W / 2, 2, e1a, 3, c1, 0, 0, nullptr));
    ART_TRY(conv(e1a, 3, c1, H / 2, W / 2, 3, cat1, 4, c2 + c1, c2, 0, nullptr, p1));
    ART_TRY(conv(p1, 4, c1, H / 4, W / 4, 4, e2a, 5, c2, 0, 0, nullptr));
    ART_TRY(conv(e2a, 5, c2, H / 4, W / 4, 5, cat2, 6, c3 + c2, c3, 0, nullptr, p2));
    ART_TRY(conv(p2, 6, c2, H / 8, W / 8, 6, e3a, 7, c3, 0, 0, nullptr));
    ART_TRY(conv(e3a, 7, c3, H / 8, W / 8, 7, cat2, 6, c3 + c2, 0, 1, nullptr));
    ART_TRY(conv(cat2, 6, c3 + c2, H / 4, W / 4, 8, d2a, 8, c2, 0, 0, nullptr));
    ART_TRY(conv(d2a, 8, c2, H / 4, W / 4, 9, cat1, 4, c2 + c1, 0, 1, nullptr));
    ART_TRY(conv(cat1, 4, c2 + c1, H / 2, W / 2, 10, d1a, 9, c1, 0, 0, nullptr));
    ART_TRY(conv(d1a, 9, c1, H / 2, W / 2, 11, cat0, 2, c1 + c0, 0, 1, nullptr));
    ART_TRY(conv(cat0, 2, c1 + c0, H, W, 12, d0a, 10, c0, 0, 0, nullptr));
    ART_TRY(conv(d0a, 10, c0, H, W, 13, -1, 0, 0, 0, 0, rgba));
#undef ART_TRY
    return ART_OK;
  };
  art_status st;
  if (!ctx->f8_calibrated) {  // measure the maxima once with unit scales
    launch_update_scales(ctx, sc, am, kF8Tensors, 1.0f);
    if ((st = network()) != ART_OK) return st;
    launch_update_scales(ctx, sc, am, kF8Tensors, 0.0f);
    ctx->f8_calibrated = true;
  }
  if ((st = network()) != ART_OK) return st;
  launch_update_scales(ctx, sc, am, kF8Tensors, 0.0f);  // scales of the next call
  return ART_OK;
}

// FP8 input quantisation reads BF16 pairs: the input channel count must be even
// (it is a multiple of 32 whenever unet_tc_ok holds).
bool f8_input_unusable(art_ctx* ctx) { return (ctx->net.cin % 2) != 0; }

// The tensor-core path covers a U-Net (levels levels, layers[lb ...]) when
// every layer fits its shapes (a padded first layer counts with its padded
// input channels) and the head is a 1x1 layer of at most 4 outputs fused
// into a last convolution of 32 channels.
bool unet_layers_tc_ok(art_ctx* ctx, int lb, int levels) {
  const int nl = 4 * levels - 1;
  if ((int)ctx->layers.size() < lb + nl) return false;
  for (int i = 0; i < nl - 1; ++i) {
    const ConvLayer& l = ctx->layers[lb + i];
    TcConv c{};
    c.cin = l.cin_pad;
    c.cout = l.cout;
    c.ld_out = 16;
    c.rgba = i == nl - 2 ? (float*)1 : nullptr;
    if (l.k != 3 || !l.wbf || !tc_conv_ok(c)) return false;
  }
  const ConvLayer& hd = ctx->layers[lb + nl - 1];
  return hd.k == 1 && hd.cout <= 4;
}

bool unet_tc_ok(art_ctx* ctx, const ViewParams& v) {
  const art_net_desc& nd = ctx->net;
  if (nd.arch != ART_NET_UNET || nd.cout != 4 || v.W % 8 || v.H % 8) return false;
  return unet_layers_tc_ok(ctx, 0, 4);
}

bool two_branch_tc_ok(art_ctx* ctx, const ViewParams& v) {
  if (ctx->net.arch != ART_NET_TWO_BRANCH || v.W % 8 || v.H % 8) return false;
  return unet_layers_tc_ok(ctx, 0, 4) && unet_layers_tc_ok(ctx, 15, 2);
}

}  // namespace

art_status run_shader(art_ctx* ctx, const ViewParams& v, const void* F, int F_dtype, const float* A, float* rgba) {
  if (ctx->net.arch == ART_NET_TWO_BRANCH && !A)
    return fail(ctx, ART_ERR_INVALID_ARG, "the two-branch network needs the coarse opacity map A");
  if (ctx->net_dtype == ART_F32) {
    if (F_dtype != ART_F32) return fail(ctx, ART_ERR_INVALID_ARG, "shade: FP32 network needs an FP32 feature map");
    return run_typed<float>(ctx, v, F, A, rgba);
  }
  if (F_dtype != ART_BF16) return fail(ctx, ART_ERR_INVALID_ARG, "shade: BF16/FP8 network needs a BF16 feature map");
  if (ctx->net_dtype == ART_FP8) {
    if (!unet_tc_ok(ctx, v) || f8_input_unusable(ctx))
      return fail(ctx, ART_ERR_UNSUPPORTED, "FP8 network: U-Net with tensor-core shapes and W, H multiples of 8 only");
    return run_unet_f8(ctx, v, (const __nv_bfloat16*)F, rgba);
  }
  const __nv_bfloat16* Fb = (const __nv_bfloat16*)F;
  if (unet_tc_ok(ctx, v)) return unet_tc(ctx, v.H, v.W, Fb, ctx->net.cin, 0, 4, ctx->net.ch, rgba, 4, 4, 0, 0);
  if (two_branch_tc_ok(ctx, v)) return run_two_branch_tc(ctx, v, Fb, A, rgba);
  return run_typed<__nv_bfloat16>(ctx, v, F, A, rgba);
}

}  // namespace art
