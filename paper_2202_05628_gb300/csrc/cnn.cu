// Neural shading network (arXiv 2202.05628, Sec. 3.1 "Neural Shading"):
// layer orchestration and the CUDA-core implicit-GEMM convolution used for the
// FP32 form.  The BF16 form runs its 3x3 layers on the tensor cores
// (cnn_tc.cu).
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
  void* out;       // [H][W][cout]
  int out_f32;     // output element type FP32 (else the activation type)
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
      size_t o = ((size_t)y * a.W + x) * a.cout + co;
      if (a.out_f32)
        ((float*)a.out)[o] = v;
      else
        st_act((TI*)a.out + o, v);
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
art_status run_typed(art_ctx* ctx, const ViewParams& v, const void* F, float* rgba) {
  const int H = v.H, W = v.W;
  const art_net_desc& nd = ctx->net;
  auto L = [&](int i) -> const ConvLayer& { return ctx->layers[i]; };
  auto mk = [&](const void* s0, int c0, int up0, const void* s1, int c1, int h, int w, const ConvLayer& l, void* out,
                int act, int out_f32) {
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
    return a;
  };
  const size_t es = sizeof(TI);
  if (nd.arch == ART_NET_TINY) {
    int c = nd.ch[0];
    size_t need = 2 * (size_t)H * W * c * es;
    if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, need, "activations") != ART_OK) return ART_ERR_OOM;
    char* b0 = (char*)ctx->d_act;
    char* b1 = b0 + (size_t)H * W * c * es;
    conv<TI>(ctx, mk(F, nd.cin, 0, nullptr, 0, H, W, L(0), b0, 1, 0), L(0));
    conv<TI>(ctx, mk(b0, c, 0, nullptr, 0, H, W, L(1), b1, 1, 0), L(1));
    conv<TI>(ctx, mk(b1, c, 0, nullptr, 0, H, W, L(2), rgba, 2, 1), L(2));
    return ART_OK;
  }
  // U-Net
  const int c0 = nd.ch[0], c1 = nd.ch[1], c2 = nd.ch[2], c3 = nd.ch[3];
  struct Buf {
    int h, w, c;
    size_t off;
  };
  std::vector<Buf> bufs;
  size_t total = 0;
  auto add = [&](int h, int w, int c) {
    bufs.push_back(Buf{h, w, c, total});
    total += ((size_t)h * w * c * es + 255) & ~(size_t)255;
    return (int)bufs.size() - 1;
  };
  int e0a = add(H, W, c0), e0 = add(H, W, c0), p0 = add(H / 2, W / 2, c0);
  int e1a = add(H / 2, W / 2, c1), e1 = add(H / 2, W / 2, c1), p1 = add(H / 4, W / 4, c1);
  int e2a = add(H / 4, W / 4, c2), e2 = add(H / 4, W / 4, c2), p2 = add(H / 8, W / 8, c2);
  int e3a = add(H / 8, W / 8, c3), e3 = add(H / 8, W / 8, c3);
  int d2a = add(H / 4, W / 4, c2), d2 = add(H / 4, W / 4, c2);
  int d1a = add(H / 2, W / 2, c1), d1 = add(H / 2, W / 2, c1);
  int d0a = add(H, W, c0), d0 = add(H, W, c0);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, total, "activations") != ART_OK) return ART_ERR_OOM;
  auto P = [&](int i) { return (void*)((char*)ctx->d_act + bufs[i].off); };
  conv<TI>(ctx, mk(F, nd.cin, 0, nullptr, 0, H, W, L(0), P(e0a), 1, 0), L(0));
  conv<TI>(ctx, mk(P(e0a), c0, 0, nullptr, 0, H, W, L(1), P(e0), 1, 0), L(1));
  pool<TI>(ctx, P(e0), P(p0), H, W, c0);
  conv<TI>(ctx, mk(P(p0), c0, 0, nullptr, 0, H / 2, W / 2, L(2), P(e1a), 1, 0), L(2));
  conv<TI>(ctx, mk(P(e1a), c1, 0, nullptr, 0, H / 2, W / 2, L(3), P(e1), 1, 0), L(3));
  pool<TI>(ctx, P(e1), P(p1), H / 2, W / 2, c1);
  conv<TI>(ctx, mk(P(p1), c1, 0, nullptr, 0, H / 4, W / 4, L(4), P(e2a), 1, 0), L(4));
  conv<TI>(ctx, mk(P(e2a), c2, 0, nullptr, 0, H / 4, W / 4, L(5), P(e2), 1, 0), L(5));
  pool<TI>(ctx, P(e2), P(p2), H / 4, W / 4, c2);
  conv<TI>(ctx, mk(P(p2), c2, 0, nullptr, 0, H / 8, W / 8, L(6), P(e3a), 1, 0), L(6));
  conv<TI>(ctx, mk(P(e3a), c3, 0, nullptr, 0, H / 8, W / 8, L(7), P(e3), 1, 0), L(7));
  conv<TI>(ctx, mk(P(e3), c3, 1, P(e2), c2, H / 4, W / 4, L(8), P(d2a), 1, 0), L(8));
  conv<TI>(ctx, mk(P(d2a), c2, 0, nullptr, 0, H / 4, W / 4, L(9), P(d2), 1, 0), L(9));
  conv<TI>(ctx, mk(P(d2), c2, 1, P(e1), c1, H / 2, W / 2, L(10), P(d1a), 1, 0), L(10));
  conv<TI>(ctx, mk(P(d1a), c1, 0, nullptr, 0, H / 2, W / 2, L(11), P(d1), 1, 0), L(11));
  conv<TI>(ctx, mk(P(d1), c1, 1, P(e0), c0, H, W, L(12), P(d0a), 1, 0), L(12));
  conv<TI>(ctx, mk(P(d0a), c0, 0, nullptr, 0, H, W, L(13), P(d0), 1, 0), L(13));
  conv<TI>(ctx, mk(P(d0), c0, 0, nullptr, 0, H, W, L(14), rgba, 2, 1), L(14));
  return ART_OK;
}

// BF16 U-Net on the tensor cores.  Skip connections and upsampled decoder
// inputs are written straight into per-level concatenation buffers
// cat_l = [up(decoder below) | encoder skip] by the producing convolutions'
// epilogues, so every decoder convolution reads one dense tensor; the last
// convolution carries the 1x1 head + sigmoid in its epilogue.
art_status run_unet_tc(art_ctx* ctx, const ViewParams& v, const __nv_bfloat16* F, float* rgba) {
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
    total += ((size_t)h * w * c * 2 + 255) & ~(size_t)255;
    return (int)bufs.size() - 1;
  };
  const int e0a = add(H, W, c0), cat0 = add(H, W, c1 + c0), p0 = add(H / 2, W / 2, c0);
  const int e1a = add(H / 2, W / 2, c1), cat1 = add(H / 2, W / 2, c2 + c1), p1 = add(H / 4, W / 4, c1);
  const int e2a = add(H / 4, W / 4, c2), cat2 = add(H / 4, W / 4, c3 + c2), p2 = add(H / 8, W / 8, c2);
  const int e3a = add(H / 8, W / 8, c3);
  const int d2a = add(H / 4, W / 4, c2), d1a = add(H / 2, W / 2, c1), d0a = add(H, W, c0);
  if (ensure(ctx, &ctx->d_act, &ctx->d_act_bytes, total, "activations") != ART_OK) return ART_ERR_OOM;
  auto P = [&](int i) { return (__nv_bfloat16*)((char*)ctx->d_act + bufs[i].off); };
  const auto& L = ctx->layers;
  auto conv = [&](const __nv_bfloat16* in, int cin, int h, int w, int li, __nv_bfloat16* out, int ld, int off,
                  int up2, float* head_out, __nv_bfloat16* pooled = nullptr) {
    TcConv c;
    c.in = in;
    c.cin = cin;
    c.H = h;
    c.W = w;
    c.w = L[li].wbf;
    c.bias = L[li].b32;
    c.cout = L[li].cout;
    c.act = 1;
    c.out = out;
    c.ld_out = ld;
    c.ch_off = off;
    c.up2 = up2;
    c.rgba = head_out;
    c.head_w = head_out ? L[14].w32 : nullptr;
    c.head_b = head_out ? L[14].b32 : nullptr;
    c.pool = pooled;
    return launch_tc_conv(ctx, c);
  };
  art_status st = ART_OK;
#define ART_TRY(x)                  \
  if ((st = (x)) != ART_OK) return st
  ART_TRY(conv(F, nd.cin, H, W, 0, P(e0a), c0, 0, 0, nullptr));
  ART_TRY(conv(P(e0a), c0, H, W, 1, P(cat0), c1 + c0, c1, 0, nullptr, P(p0)));  // + 2x2 max pooling
  ART_TRY(conv(P(p0), c0, H / 2, W / 2, 2, P(e1a), c1, 0, 0, nullptr));
  ART_TRY(conv(P(e1a), c1, H / 2, W / 2, 3, P(cat1), c2 + c1, c2, 0, nullptr, P(p1)));
  ART_TRY(conv(P(p1), c1, H / 4, W / 4, 4, P(e2a), c2, 0, 0, nullptr));
  ART_TRY(conv(P(e2a), c2, H / 4, W / 4, 5, P(cat2), c3 + c2, c3, 0, nullptr, P(p2)));
  ART_TRY(conv(P(p2), c2, H / 8, W / 8, 6, P(e3a), c3, 0, 0, nullptr));
  ART_TRY(conv(P(e3a), c3, H / 8, W / 8, 7, P(cat2), c3 + c2, 0, 1, nullptr));  // up x2 into cat2
  ART_TRY(conv(P(cat2), c3 + c2, H / 4, W / 4, 8, P(d2a), c2, 0, 0, nullptr));
  ART_TRY(conv(P(d2a), c2, H / 4, W / 4, 9, P(cat1), c2 + c1, 0, 1, nullptr));  // up x2 into cat1
  ART_TRY(conv(P(cat1), c2 + c1, H / 2, W / 2, 10, P(d1a), c1, 0, 0, nullptr));
  ART_TRY(conv(P(d1a), c1, H / 2, W / 2, 11, P(cat0), c1 + c0, 0, 1, nullptr));  // up x2 into cat0
  ART_TRY(conv(P(cat0), c1 + c0, H, W, 12, P(d0a), c0, 0, 0, nullptr));
  ART_TRY(conv(P(d0a), c0, H, W, 13, nullptr, 0, 0, 0, rgba));  // + fused 1x1 head, sigmoid
#undef ART_TRY
  return ART_OK;
}

// FP8 (E4M3) U-Net on the tensor cores (kind::f8f6f4), same dataflow as
// run_unet_tc.  Activation tensors carry one scale each (a concatenation
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
                  float* head_out) {
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
    return launch_tc_conv(ctx, c);
  };
  auto network = [&]() -> art_status {
    art_status st = ART_OK;
#define ART_TRY(x)                  \
  if ((st = (x)) != ART_OK) return st
    launch_quantize_input(ctx, F, (int64_t)H * W * nd.cin, sc + 0, P(fin), am + 0);
    ART_TRY(conv(fin, 0, nd.cin, H, W, 0, e0a, 1, c0, 0, 0, nullptr));
    ART_TRY(conv(e0a, 1, c0, H, W, 1, cat0, 2, c1 + c0, c1, 0, nullptr));
    launch_pool_fp8(ctx, P(cat0), c1 + c0, c1, P(p0), H, W, c0);
    ART_TRY(conv(p0, 2, c0, H / 2, W / 2, 2, e1a, 3, c1, 0, 0, nullptr));
    ART_TRY(conv(e1a, 3, c1, H / 2, W / 2, 3, cat1, 4, c2 + c1, c2, 0, nullptr));
    launch_pool_fp8(ctx, P(cat1), c2 + c1, c2, P(p1), H / 2, W / 2, c1);
    ART_TRY(conv(p1, 4, c1, H / 4, W / 4, 4, e2a, 5, c2, 0, 0, nullptr));
    ART_TRY(conv(e2a, 5, c2, H / 4, W / 4, 5, cat2, 6, c3 + c2, c3, 0, nullptr));
    launch_pool_fp8(ctx, P(cat2), c3 + c2, c3, P(p2), H / 4, W / 4, c2);
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

// The tensor-core path covers the U-Net when every layer fits its shapes.
bool unet_tc_ok(art_ctx* ctx, const ViewParams& v) {
  const art_net_desc& nd = ctx->net;
  if (nd.arch != ART_NET_UNET || nd.cout != 4 || v.W % 8 || v.H % 8) return false;
  for (int i = 0; i < 14; ++i) {
    TcConv c{};
    c.cin = ctx->layers[i].cin;
    c.cout = ctx->layers[i].cout;
    c.ld_out = 16;
    c.rgba = i == 13 ? (float*)1 : nullptr;
    if (ctx->layers[i].k != 3 || !ctx->layers[i].wbf || !tc_conv_ok(c)) return false;
  }
  return ctx->layers[14].k == 1;
}

}  // namespace

art_status run_shader(art_ctx* ctx, const ViewParams& v, const void* F, int F_dtype, float* rgba) {
  if (ctx->net_dtype == ART_F32) {
    if (F_dtype != ART_F32) return fail(ctx, ART_ERR_INVALID_ARG, "shade: FP32 network needs an FP32 feature map");
    return run_typed<float>(ctx, v, F, rgba);
  }
  if (F_dtype != ART_BF16) return fail(ctx, ART_ERR_INVALID_ARG, "shade: BF16/FP8 network needs a BF16 feature map");
  if (ctx->net_dtype == ART_FP8) {
    if (!unet_tc_ok(ctx, v) || f8_input_unusable(ctx))
      return fail(ctx, ART_ERR_UNSUPPORTED, "FP8 network: U-Net with tensor-core shapes and W, H multiples of 8 only");
    return run_unet_f8(ctx, v, (const __nv_bfloat16*)F, rgba);
  }
  if (unet_tc_ok(ctx, v)) return run_unet_tc(ctx, v, (const __nv_bfloat16*)F, rgba);
  return run_typed<__nv_bfloat16>(ctx, v, F, rgba);
}

}  // namespace art
