// The paper's own U-Net variant (Sec. 3.1, Tab. 2) as a second network kind of the preconditioner.
//
// Tab. 2: 5 inputs, 2 outputs, PReLU, depth 4, 32 channels per layer and state, kernel 8 / stride 2 /
// padding 3, batch normalisation, biases.  Wiring read for this project (Fig. 2 is missing):
//   inputs  (Re v, Im v, c / 1500 m/s, Re sigma_c, Im sigma_c), sigma_c = s_x(i) s_y(j) - 1 (eq. 2);
//   encoder e_l = PReLU(conv_{8,2,3}(e_{l-1})), l = 1..4 (5 -> 32 -> 32 -> 32 -> 32 channels);
//   decoder d_3 = PReLU(convT_{8,2,3}(e_4)), d_l = PReLU(convT_{8,2,3}(cat[d_{l+1}, e_{l+1}])), l = 2..0;
//   output  1x1 conv 32 -> 2; batch normalisation folded into the convolutions (inference form).
// The image is zero-padded to multiples of 16 (four halvings) and cropped back.
//
// Both strided layers become stride-1 5x5 convolutions, so they run on the tcgen05 implicit-GEMM
// kernels of conv_tc.cu (KS = 5):
//   conv_{8,2,3}(x)  = conv5x5(S2D(x)): S2D puts the 2 x 2 phases of x as 4 C_in channels at half
//                      resolution; output pixel i sees input 2i + t - 3, t = 0..7, i.e. phase p of
//                      half-resolution offset d with t = 2 d + p + 3 (25 x 4 C_in taps, 36 % zero);
//   convT_{8,2,3}(x) = D2S(conv5x5(x)) with 4 C_out output columns: output 2y + q receives input
//                      y + d through tap t = q + 3 - 2 d; the kernel's epilogue writes column block q to
//                      output phase q (no separate depth-to-space pass).
// Mixed path: BF16 activations, tcgen05 GEMMs with FP32 accumulation, PReLU in the epilogue.  Plain
// path: FP64 on CUDA cores with the same reformulated weights.  Training of this kind is not built.
#include <math.h>

#include <algorithm>

#include "helm_internal.cuh"
#include "unet.cuh"

namespace helm {

helm_status conv_tc_generic(const __nv_bfloat16* w_tc, const float* bias, int* err, int ks, int mode, int N,
                            int chunk, const void* in0, int C0, const void* in1, int C1, void* out, int B, int H,
                            int W, int act, float slope, cudaStream_t st);

enum PaperKind { P_DOWN = 0, P_UP = 1, P_OUT = 2 };
struct PaperLayer {
  int kind, cin, cout;
  int K, N, chunk;  // GEMM of the reformulated layer: K input channels per tap, N output columns
};
// enc1 enc2 enc3 enc4 dec3 dec2 dec1 dec0 out
static const PaperLayer kP[PAPER_LAYERS] = {
    {P_DOWN, 5, 32, 32, 32, 32},  {P_DOWN, 32, 32, 128, 32, 64}, {P_DOWN, 32, 32, 128, 32, 64},
    {P_DOWN, 32, 32, 128, 32, 64}, {P_UP, 32, 32, 32, 128, 32},  {P_UP, 64, 32, 64, 128, 32},
    {P_UP, 64, 32, 64, 128, 32},   {P_UP, 64, 32, 64, 128, 32},  {P_OUT, 32, 2, 32, 2, 0},
};
constexpr int P_X0_CH = 8;  // network input: 5 channels padded to 8 (16-byte pixels)

int64_t paper_param_count() {
  int64_t t = 0;
  for (const auto& L : kP) t += (int64_t)L.cin * L.cout * (L.kind == P_OUT ? 1 : 64) + L.cout + (L.kind == P_OUT ? 0 : 1);
  return t;
}

// ------------------------------------------------------------------ weight preparation

// Reformulated FP64 weights w5[tap][k][n] (tap = (dy + 2) * 5 + dx + 2) and per-column bias.
// Down layer: k = phase * cpad + c, n = co, master [co][ci][8][8].  Up layer: k = c, n = q * cout + co,
// master [ci][co][8][8].  Output layer: w5[k][n], master [co][ci].
__global__ void k_paper_reform(const double* __restrict__ master, int64_t m_w, int64_t m_b, int kind, int cin,
                               int cpad, int cout, int K, int N, double* __restrict__ w5, double* __restrict__ b5) {
  const int taps = kind == P_OUT ? 1 : 25;
  const int64_t total = (int64_t)taps * K * N;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < N) b5[e] = master[m_b + (e % cout)];
  if (e >= total) return;
  const int n = (int)(e % N);
  const int k = (int)((e / N) % K);
  const int tap = (int)(e / ((int64_t)N * K));
  double v = 0.0;
  if (kind == P_OUT) {
    v = master[m_w + (int64_t)n * cin + k];
  } else {
    const int dy = tap / 5 - 2, dx = tap % 5 - 2;
    if (kind == P_DOWN) {
      const int ph = k / cpad, c = k % cpad;
      const int ty = 2 * dy + (ph >> 1) + 3, tx = 2 * dx + (ph & 1) + 3;
      if (c < cin && ty >= 0 && ty < 8 && tx >= 0 && tx < 8)
        v = master[m_w + (((int64_t)n * cin + c) * 8 + ty) * 8 + tx];
    } else {
      const int q = n / cout, co = n % cout;
      const int ty = (q >> 1) + 3 - 2 * dy, tx = (q & 1) + 3 - 2 * dx;
      if (ty >= 0 && ty < 8 && tx >= 0 && tx < 8) v = master[m_w + (((int64_t)k * cout + co) * 8 + ty) * 8 + tx];
    }
  }
  w5[e] = v;
}

// tcgen05 layout [tap][kc][n][c] in BF16 from w5[tap][k][n]; bias in FP32.
__global__ void k_paper_tc(const double* __restrict__ w5, const double* __restrict__ b5, int K, int N, int chunk,
                           __nv_bfloat16* __restrict__ wtc, float* __restrict__ b32) {
  const int64_t total = (int64_t)25 * K * N;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < N) b32[e] = (float)b5[e];
  if (e >= total) return;
  const int c = (int)(e % chunk);
  const int n = (int)((e / chunk) % N);
  const int kc = (int)((e / ((int64_t)chunk * N)) % (K / chunk));
  const int tap = (int)(e / ((int64_t)chunk * N * (K / chunk)));
  wtc[e] = __float2bfloat16_rn((float)w5[((int64_t)tap * K + kc * chunk + c) * N + n]);
}

// Output layer for the BF16 path: 32 x 2 weights rounded to BF16 (held in FP32), then 2 biases.
__global__ void k_paper_out32(const double* __restrict__ w5, const double* __restrict__ b5, float* __restrict__ o) {
  const int e = threadIdx.x;
  if (e < 64) o[e] = __bfloat162float(__float2bfloat16_rn((float)w5[e]));
  if (e < 2) o[64 + e] = (float)b5[e];
}

helm_status paper_prepare(helm_unet* net, cudaStream_t st) {
  PaperNet& P = *net->pn;
  int64_t off = 0;
  for (int l = 0; l < PAPER_LAYERS; ++l) {
    const PaperLayer& L = kP[l];
    const int64_t nw = (int64_t)L.cin * L.cout * (L.kind == P_OUT ? 1 : 64);
    P.m_w[l] = off;
    P.m_b[l] = off + nw;
    off += nw + L.cout;
    P.m_s[l] = L.kind == P_OUT ? -1 : off;
    off += L.kind == P_OUT ? 0 : 1;
    const int taps = L.kind == P_OUT ? 1 : 25;
    const int64_t n5 = (int64_t)taps * L.K * L.N;
    if (!P.w5[l]) {
      HELM_CK(cudaMalloc(&P.w5[l], sizeof(double) * n5));
      HELM_CK(cudaMalloc(&P.b5[l], sizeof(double) * L.N));
      if (L.kind != P_OUT) {
        HELM_CK(cudaMalloc(&P.wtc[l], sizeof(__nv_bfloat16) * n5));
        HELM_CK(cudaMalloc(&P.b32[l], sizeof(float) * L.N));
      }
    }
    const int cpad = l == 0 ? P_X0_CH : L.cin;
    launch(k_paper_reform, cdiv(std::max<int64_t>(n5, L.N), 256), 256, 0, st, (const double*)net->master, P.m_w[l],
           P.m_b[l], L.kind, L.cin, cpad, L.cout, L.K, L.N, P.w5[l], P.b5[l]);
    if (L.kind != P_OUT)
      launch(k_paper_tc, cdiv(std::max<int64_t>(n5, L.N), 256), 256, 0, st, (const double*)P.w5[l],
             (const double*)P.b5[l], L.K, L.N, L.chunk, P.wtc[l], P.b32[l]);
  }
  if (!P.wout32) HELM_CK(cudaMalloc(&P.wout32, sizeof(float) * 66));
  launch(k_paper_out32, 1, 64, 0, st, (const double*)P.w5[PAPER_LAYERS - 1], (const double*)P.b5[PAPER_LAYERS - 1],
         P.wout32);
  HELM_CK_LAUNCH();
  // PReLU slopes to the host (one per layer, read at launch time)
  std::vector<double> sl(PAPER_LAYERS, 0.0);
  for (int l = 0; l < PAPER_LAYERS - 1; ++l)
    HELM_CK(cudaMemcpyAsync(&sl[l], net->master + P.m_s[l], sizeof(double), cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  for (int l = 0; l < PAPER_LAYERS; ++l) P.slope[l] = sl[l];
  if (!P.err) {
    HELM_CK(cudaMalloc(&P.err, sizeof(int)));
    HELM_CK(cudaMemset(P.err, 0, sizeof(int)));
  }
  return HELM_OK;
}

void paper_release(helm_unet* net) {
  if (!net->pn) return;
  PaperNet& P = *net->pn;
  for (int l = 0; l < PAPER_LAYERS; ++l) {
    cudaFree(P.w5[l]);
    cudaFree(P.b5[l]);
    cudaFree(P.wtc[l]);
    cudaFree(P.b32[l]);
  }
  cudaFree(P.wout32);
  cudaFree(P.err);
  for (auto& s : P.act)
    if (s.base) cudaFree(s.base);
  delete net->pn;
  net->pn = nullptr;
}

// ------------------------------------------------------------------ kernels of the forward pass

// Input channels (Re s v, Im s v, c / 1500, Re sigma_c, Im sigma_c, 0, 0, 0) on the 16-padded grid.
template <typename T, typename R>
__global__ void k_paper_pack(const C<R>* __restrict__ v, int64_t col_stride, const double* __restrict__ in_scale,
                             const double* __restrict__ chat, const double2* __restrict__ px,
                             const double2* __restrict__ py, int Nx, int Ny, int Hp, int Wp, int B,
                             T* __restrict__ x0) {
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)B * Hp * Wp) return;
  const int x = (int)(pix % Wp);
  const int y = (int)((pix / Wp) % Hp);
  const int b = (int)(pix / ((int64_t)Wp * Hp));
  double ch[P_X0_CH] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (x < Nx && y < Ny) {
    const int64_t q = (int64_t)y * Nx + x;
    const C<R> val = v[b * col_stride + q];
    const double s = in_scale[b];
    ch[0] = (double)val.x * s;
    ch[1] = (double)val.y * s;
    ch[2] = chat[q];
    const double2 sx = px[x], sy = py[y];
    ch[3] = sx.x * sy.x - sx.y * sy.y - 1.0;
    ch[4] = sx.x * sy.y + sx.y * sy.x;
  }
  T* o = x0 + pix * P_X0_CH;
#pragma unroll
  for (int k = 0; k < P_X0_CH; ++k) store_act(o + k, (typename Acc<T>::A)ch[k]);
}

// Space-to-depth: out[b][Y][X][(py * 2 + px) C + c] = in[b][2Y + py][2X + px][c]  (Ho = H / 2).
template <typename T>
__global__ void k_s2d(const T* __restrict__ in, T* __restrict__ out, int C, int B, int Ho, int Wo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)B * Ho * Wo * 4 * C;
  if (e >= total) return;
  const int k = (int)(e % (4 * C));
  const int64_t pix = e / (4 * C);
  const int X = (int)(pix % Wo);
  const int Y = (int)((pix / Wo) % Ho);
  const int64_t b = pix / ((int64_t)Wo * Ho);
  const int ph = k / C, c = k % C;
  out[e] = in[((b * 2 * Ho + 2 * Y + (ph >> 1)) * (2 * Wo) + 2 * X + (ph & 1)) * C + c];
}

// FP64 5x5 conv on CUDA cores (plain path): out = act(bias + sum w5[tap][k][n] in[tap-shifted][k]),
// in = concat(in0 (C0 channels), in1 (C1)); up = 1 writes column block q = n / cout to output phase q of
// the 2H x 2W grid (depth-to-space).  One thread per (pixel, 16 output columns).
constexpr int PC_THREADS = 128;
__global__ void __launch_bounds__(PC_THREADS) k_pconv_f64(const double* __restrict__ in0, int C0,
                                                          const double* __restrict__ in1, int C1,
                                                          const double* __restrict__ w5,
                                                          const double* __restrict__ b5, double* __restrict__ out,
                                                          int N, int cout, int up, int B, int H, int W, double slope) {
  const int64_t pix = blockIdx.x * (int64_t)PC_THREADS + threadIdx.x;
  if (pix >= (int64_t)B * H * W) return;
  const int n0 = blockIdx.y * 16;
  const int x = (int)(pix % W);
  const int y = (int)((pix / W) % H);
  const int64_t b = pix / ((int64_t)W * H);
  const int K = C0 + C1;
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = b5[n0 + k];
  for (int tap = 0; tap < 25; ++tap) {
    const int yy = y + tap / 5 - 2, xx = x + tap % 5 - 2;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    const int64_t q = (b * H + yy) * W + xx;
    const double* wt = w5 + (int64_t)tap * K * N + n0;
    for (int c = 0; c < K; ++c) {
      const double v = c < C0 ? in0[q * C0 + c] : in1[q * C1 + (c - C0)];
      const double* wr = wt + (int64_t)c * N;
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[k] += v * wr[k];
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const double f = acc[k] > 0 ? acc[k] : slope * acc[k];
    const int n = n0 + k;
    if (!up) {
      out[pix * N + n] = f;
    } else {
      const int q = n / cout, co = n % cout;
      out[((b * 2 * H + 2 * y + (q >> 1)) * (2 * W) + 2 * x + (q & 1)) * cout + co] = f;
    }
  }
}

// Output layer 32 -> 2, crop to the physical grid and scale: z = out_scale (y0 + i y1).
template <typename T, typename R>
__global__ void k_paper_final(const T* __restrict__ in, const typename Acc<T>::A* __restrict__ w,
                              const typename Acc<T>::A* __restrict__ bias, const double* __restrict__ out_scale,
                              int Nx, int Ny, int Hp, int Wp, int B, C<R>* __restrict__ z, int64_t col_stride) {
  using A = typename Acc<T>::A;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * Ny * Nx) return;
  const int x = (int)(e % Nx);
  const int y = (int)((e / Nx) % Ny);
  const int b = (int)(e / ((int64_t)Nx * Ny));
  const T* ip = in + (((int64_t)b * Hp + y) * Wp + x) * 32;
  A y0 = bias[0], y1 = bias[1];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const A v = to_acc(ip[c]);
    y0 += v * w[c * 2 + 0];
    y1 += v * w[c * 2 + 1];
  }
  const double s = out_scale[b];
  z[b * col_stride + (int64_t)y * Nx + x] = mk<R>((R)(y0 * s), (R)(y1 * s));
}

// ------------------------------------------------------------------ driver

enum PaperAct { PA_X0 = 0, PA_S0, PA_E1, PA_S1, PA_E2, PA_S2, PA_E3, PA_S3, PA_E4, PA_D3, PA_D2, PA_D1, PA_D0 };

static helm_status paper_buffers(PaperNet& P, int B, int Hp, int Wp, bool fp64, void** a) {
  const size_t es = fp64 ? 8 : 2;
  const size_t full = (size_t)Hp * Wp;
  // channels x pixels of each activation, in PaperAct order
  const size_t el[13] = {P_X0_CH * full, 32 * full / 4, 32 * full / 4, 128 * full / 16, 32 * full / 16,
                         128 * full / 64, 32 * full / 64, 128 * full / 256, 32 * full / 256, 32 * full / 64,
                         32 * full / 16, 32 * full / 4, 32 * full};
  size_t need = 0;
  for (size_t v : el) need += (v * B * es + 255) / 256 * 256;
  PaperNet::Set& S = P.act[fp64 ? 1 : 0];
  if (need > S.cap) {
    if (S.base) cudaFree(S.base);
    S.base = nullptr;
    S.cap = 0;
    HELM_CK(cudaMalloc(&S.base, need));
    S.cap = need;
  }
  size_t off = 0;
  for (int k = 0; k < 13; ++k) {
    a[k] = (char*)S.base + off;
    off += (el[k] * B * es + 255) / 256 * 256;
  }
  return HELM_OK;
}

template <typename R>
helm_status paper_precondition(helm_ctx* ctx, const helm_unet* net, int sys, const C<R>* v, C<R>* z, int B,
                               const double* in_scale, const double* out_scale, cudaStream_t st) {
  using T = typename std::conditional<sizeof(R) == 8, double, __nv_bfloat16>::type;
  constexpr bool fp64 = sizeof(R) == 8;
  PaperNet& P = *net->pn;
  const SysHost& s = ctx->sys[sys];
  const int Hp = (s.Ny + 15) / 16 * 16, Wp = (s.Nx + 15) / 16 * 16;
  void* a[13];
  HELM_TRY(paper_buffers(P, B, Hp, Wp, fp64, a));
  const int64_t npix = (int64_t)B * Hp * Wp;
  launch(k_paper_pack<T, R>, cdiv(npix, 256), 256, 0, st, v, s.n, in_scale, (const double*)(ctx->chat64 + s.off),
         (const double2*)(ctx->prof_d + s.prof_x), (const double2*)(ctx->prof_d + s.prof_y), s.Nx, s.Ny, Hp, Wp, B,
         (T*)a[PA_X0]);
  HELM_CK_LAUNCH();
  auto s2d = [&](int src, int dst, int C, int H, int W) -> helm_status {  // H, W: source grid
    const int64_t n = (int64_t)B * (H / 2) * (W / 2) * 4 * C;
    launch(k_s2d<T>, cdiv(n, 256), 256, 0, st, (const T*)a[src], (T*)a[dst], C, B, H / 2, W / 2);
    HELM_CK_LAUNCH();
    return HELM_OK;
  };
  // one reformulated layer on the grid H x W (the GEMM's pixel grid)
  auto layer = [&](int l, int src0, int C0, int src1, int C1, int dst, int H, int W) -> helm_status {
    const PaperLayer& L = kP[l];
    if constexpr (fp64) {
      dim3 grid(cdiv((int64_t)B * H * W, PC_THREADS), L.N / 16);
      launch(k_pconv_f64, grid, PC_THREADS, 0, st, (const double*)a[src0], C0,
             (const double*)(src1 >= 0 ? a[src1] : nullptr), C1, (const double*)P.w5[l], (const double*)P.b5[l],
             (double*)a[dst], L.N, L.cout, L.kind == P_UP ? 1 : 0, B, H, W, P.slope[l]);
      HELM_CK_LAUNCH();
      return HELM_OK;
    } else {
      return conv_tc_generic(P.wtc[l], P.b32[l], P.err, 5, L.kind == P_UP ? 2 : 0, L.N, L.chunk, a[src0], C0,
                             src1 >= 0 ? a[src1] : nullptr, C1, a[dst], B, H, W, 2, (float)P.slope[l], st);
    }
  };
  int H = Hp, W = Wp;
  HELM_TRY(s2d(PA_X0, PA_S0, P_X0_CH, H, W));
  HELM_TRY(layer(0, PA_S0, 4 * P_X0_CH, -1, 0, PA_E1, H / 2, W / 2));
  HELM_TRY(s2d(PA_E1, PA_S1, 32, H / 2, W / 2));
  HELM_TRY(layer(1, PA_S1, 128, -1, 0, PA_E2, H / 4, W / 4));
  HELM_TRY(s2d(PA_E2, PA_S2, 32, H / 4, W / 4));
  HELM_TRY(layer(2, PA_S2, 128, -1, 0, PA_E3, H / 8, W / 8));
  HELM_TRY(s2d(PA_E3, PA_S3, 32, H / 8, W / 8));
  HELM_TRY(layer(3, PA_S3, 128, -1, 0, PA_E4, H / 16, W / 16));
  HELM_TRY(layer(4, PA_E4, 32, -1, 0, PA_D3, H / 16, W / 16));      // -> H/8
  HELM_TRY(layer(5, PA_D3, 32, PA_E3, 32, PA_D2, H / 8, W / 8));    // -> H/4
  HELM_TRY(layer(6, PA_D2, 32, PA_E2, 32, PA_D1, H / 4, W / 4));    // -> H/2
  HELM_TRY(layer(7, PA_D1, 32, PA_E1, 32, PA_D0, H / 2, W / 2));    // -> H
  const int64_t nout = (int64_t)B * s.Ny * s.Nx;
  const typename Acc<T>::A* wf;
  const typename Acc<T>::A* bf;
  if constexpr (fp64) {
    wf = P.w5[PAPER_LAYERS - 1];
    bf = P.b5[PAPER_LAYERS - 1];
  } else {
    wf = P.wout32;
    bf = P.wout32 + 64;
  }
  launch(k_paper_final<T, R>, cdiv(nout, 256), 256, 0, st, (const T*)a[PA_D0], wf, bf, out_scale, s.Nx, s.Ny, Hp, Wp, B,
         z, s.n);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

template helm_status paper_precondition<float>(helm_ctx*, const helm_unet*, int, const float2*, float2*, int,
                                               const double*, const double*, cudaStream_t);
template helm_status paper_precondition<double>(helm_ctx*, const helm_unet*, int, const double2*, double2*, int,
                                                const double*, const double*, cudaStream_t);

helm_status paper_check(const helm_unet* net, cudaStream_t st) {
  if (!net->pn || !net->pn->err) return HELM_OK;
  int e = 0;
  HELM_CK(cudaMemcpyAsync(&e, net->pn->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  if (e) {
    cudaMemsetAsync(net->pn->err, 0, sizeof(int), st);
    return fail(HELM_TIMEOUT, "tcgen05 conv kernel: a pipeline wait ran out of its budget (code " + std::to_string(e) + ")");
  }
  return HELM_OK;
}

}  // namespace helm
