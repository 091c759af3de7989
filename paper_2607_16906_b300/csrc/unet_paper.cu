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
// Mixed path: BF16 activations, tcgen05 GEMMs with FP32 accumulation, PReLU in the epilogue; there the
// first three strided layers take a second form with 4x wider GEMM rows (conv_tc_phase):
//   conv_{8,2,3}(x)  = D2S(conv3x3(S2D_4(x))): a GEMM pixel is a 4 x 4 block of x (16 C_in channels,
//                      read through a strided tensor-map view), its 128 columns the 2 x 2 output pixels
//                      of that block (4 x 32); output 2h + p sees input 4 (h + e) + o, e = -1..1, through
//                      kernel tap t = 4 e + o - 2 p + 3 (5/9 zero).  The N = 128 MMAs need a quarter of the
//                      N = 32 MMAs' instructions per product.
// Plain path: FP64 on CUDA cores with the 5x5 weights.  Training (the end of this file): FP32
// on CUDA cores, forward with the pre-activations kept, backward through the same reformulation.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "helm_internal.cuh"
#include "unet.cuh"

namespace helm {

helm_status conv_tc_generic(const __nv_bfloat16* w_tc, const float* bias, int* err, int ks, int mode, int N,
                            int chunk, const void* in0, int C0, const void* in1, int C1, void* out, int B, int H,
                            int W, int act, float slope, cudaStream_t st, bool s2d0, const RowFinal* fin,
                            const double* img_scale, void* pre_out = nullptr);
helm_status conv_tc_phase(const __nv_bfloat16* wq, const float* bias, int* err, int f, const void* in, void* out,
                          int B, int H, int W, float slope, cudaStream_t st, const double* img_scale,
                          void* pre_out = nullptr);

bool tc_available();

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

// A down layer as a 3x3 convolution of the phase view of its input (the BF16 encoder, conv_tc.cu): GEMM
// pixel (h, w) produces output pixels (2h + py, 2w + px) in column n = (2 py + px) 32 + co; output row
// 2h + py reads input rows 2 (2h + py) + t - 3, t = 0..7, which lie in the 4-row blocks h - 1, h, h + 1:
// input row 4 (h + ey) + oy is kernel row t = 4 ey + oy - 2 py + 3 (zero outside 0..7; 5/9 of the
// products are structural zeros).  Chunk kc = (sy, sx) of a tap holds, for f = 4, the 32 channels of
// input pixel (4 (h + ey) + sy, 4 (w + ex) + sx); for f = 2 (the first layer, whose input arrives
// space-to-depth packed: channel c = (2 ry + rx) 8 + ci of packed pixel (Y, X) is input pixel
// (2Y + ry, 2X + rx)) the packed pixel (2 (h + ey) + sy, 2 (w + ex) + sx), i.e. oy = 2 sy + ry.
// Layout [tap][kc][n][c] BF16 (rounded through FP32 like the other layouts); bias per column.
__global__ void k_paper_phase(const double* __restrict__ master, int64_t m_w, int64_t m_b, int cin, int f,
                              __nv_bfloat16* __restrict__ wq, float* __restrict__ bq) {
  const int nk = f * f;
  const int64_t total = (int64_t)9 * nk * 128 * 32;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < 128) bq[e] = (float)master[m_b + e % 32];
  if (e >= total) return;
  const int c = (int)(e % 32);
  const int n = (int)((e / 32) % 128);
  const int kc = (int)((e / 4096) % nk);
  const int tap = (int)(e / (4096 * (int64_t)nk));
  const int ey = tap / 3 - 1, ex = tap % 3 - 1;
  const int py = n / 64, px = (n / 32) % 2, co = n % 32;
  const int sy = kc / f, sx = kc % f;
  int oy = sy, ox = sx, ci = c;
  if (f == 2) {
    oy = 2 * sy + c / 16;
    ox = 2 * sx + (c / 8) % 2;
    ci = c % 8;
  }
  const int ty = 4 * ey + oy - 2 * py + 3, tx = 4 * ex + ox - 2 * px + 3;
  double v = 0.0;
  if (ci < cin && ty >= 0 && ty < 8 && tx >= 0 && tx < 8) v = master[m_w + (((int64_t)co * cin + ci) * 8 + ty) * 8 + tx];
  wq[e] = __float2bfloat16_rn((float)v);
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

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
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
      HELM_CK(cudaMalloc(&P.w5f[l], sizeof(float) * n5));
      HELM_CK(cudaMalloc(&P.b5[l], sizeof(double) * L.N));
      if (L.kind != P_OUT) {
        HELM_CK(cudaMalloc(&P.wtc[l], sizeof(__nv_bfloat16) * n5));
        HELM_CK(cudaMalloc(&P.b32[l], sizeof(float) * L.N));
      }
    }
    const int cpad = l == 0 ? P_X0_CH : L.cin;
    launch(k_paper_reform, cdiv(std::max<int64_t>(n5, L.N), 256), 256, 0, st, (const double*)net->master, P.m_w[l],
           P.m_b[l], L.kind, L.cin, cpad, L.cout, L.K, L.N, P.w5[l], P.b5[l]);
    launch(k_to_f32, cdiv(n5, 256), 256, 0, st, (const double*)P.w5[l], P.w5f[l], n5);
    if (L.kind != P_OUT)
      launch(k_paper_tc, cdiv(std::max<int64_t>(n5, L.N), 256), 256, 0, st, (const double*)P.w5[l],
             (const double*)P.b5[l], L.K, L.N, L.chunk, P.wtc[l], P.b32[l]);
    if (L.kind == P_DOWN && l < 3) {
      const int f = l == 0 ? 2 : 4;
      const int64_t nq = (int64_t)9 * f * f * 128 * 32;
      if (!P.wq[l]) {
        HELM_CK(cudaMalloc(&P.wq[l], sizeof(__nv_bfloat16) * nq));
        HELM_CK(cudaMalloc(&P.bq[l], sizeof(float) * 128));
      }
      launch(k_paper_phase, cdiv(nq, 256), 256, 0, st, (const double*)net->master, P.m_w[l], P.m_b[l], L.cin, f,
             P.wq[l], P.bq[l]);
    }
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
    cudaFree(P.w5f[l]);
    cudaFree(P.b5[l]);
    cudaFree(P.wtc[l]);
    cudaFree(P.b32[l]);
  }
  for (int l = 0; l < 3; ++l) {
    cudaFree(P.wq[l]);
    cudaFree(P.bq[l]);
  }
  cudaFree(P.wout32);
  cudaFree(P.err);
  for (auto& s : P.act)
    if (s.base) cudaFree(s.base);
  delete net->pn;
  net->pn = nullptr;
}

// ------------------------------------------------------------------ kernels of the forward pass

// Input channels (Re s v, Im s v, c / 1500, Re sigma_c, Im sigma_c, 0, 0, 0) on the 16-padded grid,
// written straight into the space-to-depth layout of the first layer: pixel (y, x) is phase
// (y % 2) * 2 + x % 2 of pixel (y / 2, x / 2), 8 channels per phase.  One thread per pixel of the
// grid (Wp / PACK_THREADS, Hp), looping over the B images: the PML channels (FP64) are formed once per
// pixel, c / 1500 once unless it differs per image (c_stride > 0); the BF16 path scales v in FP32
// (its result is rounded to BF16) and stores each pixel's 8 channels as one 16-byte vector.
constexpr int PACK_THREADS = 128;
template <typename T, typename R>
__global__ void __launch_bounds__(PACK_THREADS) k_paper_pack(const C<R>* __restrict__ v, int64_t col_stride,
                                                             const double* __restrict__ in_scale,
                                                             const double* __restrict__ chat, int64_t c_stride,
                                                             const double2* __restrict__ px,
                                                             const double2* __restrict__ py, int Nx, int Ny, int Hp,
                                                             int Wp, int B, T* __restrict__ x0) {
  constexpr bool bf16 = std::is_same<T, __nv_bfloat16>::value;
  const int x = blockIdx.x * PACK_THREADS + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= Wp) return;
  const bool in = x < Nx && y < Ny;
  const int64_t q = (int64_t)y * Nx + x;
  double sig_re = 0, sig_im = 0, c0 = 0;
  if (in) {
    const double2 sx = px[x], sy = py[y];
    sig_re = sx.x * sy.x - sx.y * sy.y - 1.0;
    sig_im = sx.x * sy.y + sx.y * sy.x;
    c0 = chat[q];
  }
  const int64_t plane = (int64_t)(Hp / 2) * (Wp / 2) * 4 * P_X0_CH;  // elements of one image
  T* o = x0 + (((int64_t)(y / 2) * (Wp / 2) + x / 2) * 4 + (y & 1) * 2 + (x & 1)) * P_X0_CH;
  for (int b = 0; b < B; ++b, o += plane) {
    double ch[P_X0_CH] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (in) {
      const C<R> val = v[b * col_stride + q];
      if constexpr (bf16) {
        const float s = (float)in_scale[b];
        ch[0] = (float)val.x * s;
        ch[1] = (float)val.y * s;
      } else {
        const double s = in_scale[b];
        ch[0] = (double)val.x * s;
        ch[1] = (double)val.y * s;
      }
      ch[2] = c_stride ? chat[b * c_stride + q] : c0;
      ch[3] = sig_re;
      ch[4] = sig_im;
    }
    if constexpr (bf16) {
      __align__(16) __nv_bfloat16 hv[P_X0_CH];
#pragma unroll
      for (int k = 0; k < P_X0_CH; ++k) hv[k] = __float2bfloat16_rn((float)ch[k]);
      *(uint4*)o = *(const uint4*)hv;
    } else {
#pragma unroll
      for (int k = 0; k < P_X0_CH; ++k) store_act(o + k, (typename Acc<T>::A)ch[k]);
    }
  }
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
  // channels x pixels of each activation, in PaperAct order; the input is packed straight into S0, and
  // the BF16 path reads S1..S3 through space-to-depth views and fuses the output layer (no D0)
  const size_t el[13] = {0, 32 * full / 4, 32 * full / 4, fp64 ? 128 * full / 16 : 0, 32 * full / 16,
                         fp64 ? 128 * full / 64 : 0, 32 * full / 64, fp64 ? 128 * full / 256 : 0, 32 * full / 256,
                         32 * full / 64, 32 * full / 16, 32 * full / 4, fp64 ? 32 * full : 0};
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
  launch(k_paper_pack<T, R>, dim3(cdiv(Wp, PACK_THREADS), Hp), PACK_THREADS, 0, st, v, s.n, in_scale, (const double*)(ctx->chat64 + s.off),
         (int64_t)0, (const double2*)(ctx->prof_d + s.prof_x), (const double2*)(ctx->prof_d + s.prof_y), s.Nx, s.Ny,
         Hp, Wp, B, (T*)a[PA_S0]);
  HELM_CK_LAUNCH();
  auto s2d = [&](int src, int dst, int C, int H, int W) -> helm_status {  // H, W: source grid
    const int64_t n = (int64_t)B * (H / 2) * (W / 2) * 4 * C;
    launch(k_s2d<T>, cdiv(n, 256), 256, 0, st, (const T*)a[src], (T*)a[dst], C, B, H / 2, W / 2);
    HELM_CK_LAUNCH();
    return HELM_OK;
  };
  // one reformulated layer on the grid H x W (the GEMM's pixel grid); s2d0: source 0 is the 2H x 2W
  // activation read through its space-to-depth view (BF16 path); fin: the output layer fused in
  auto layer = [&](int l, int src0, int C0, int src1, int C1, int dst, int H, int W, bool s2d0 = false,
                   const RowFinal* fin = nullptr) -> helm_status {
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
                             src1 >= 0 ? a[src1] : nullptr, C1, dst >= 0 ? a[dst] : nullptr, B, H, W, 2,
                             (float)P.slope[l], st, s2d0, fin, in_scale);
    }
  };
  int H = Hp, W = Wp;
  if constexpr (!fp64) {
    // the first three encoder layers as 3x3 convolutions of phase views (N = 128; their output grids
    // have even sides, Hp and Wp being multiples of 16); the last in the 5x5 form, whose 8 x 16 tiles
    // fit its small grid better (a quarter of the pixels per GEMM row of the phase form)
    HELM_TRY(conv_tc_phase(P.wq[0], P.bq[0], P.err, 2, a[PA_S0], a[PA_E1], B, H / 4, W / 4, (float)P.slope[0], st,
                           in_scale));
    HELM_TRY(conv_tc_phase(P.wq[1], P.bq[1], P.err, 4, a[PA_E1], a[PA_E2], B, H / 8, W / 8, (float)P.slope[1], st,
                           in_scale));
    HELM_TRY(conv_tc_phase(P.wq[2], P.bq[2], P.err, 4, a[PA_E2], a[PA_E3], B, H / 16, W / 16, (float)P.slope[2], st,
                           in_scale));
    HELM_TRY(layer(3, PA_E3, 128, -1, 0, PA_E4, H / 16, W / 16, true));
  } else {
    HELM_TRY(layer(0, PA_S0, 4 * P_X0_CH, -1, 0, PA_E1, H / 2, W / 2));
    HELM_TRY(s2d(PA_E1, PA_S1, 32, H / 2, W / 2));
    HELM_TRY(layer(1, PA_S1, 128, -1, 0, PA_E2, H / 4, W / 4));
    HELM_TRY(s2d(PA_E2, PA_S2, 32, H / 4, W / 4));
    HELM_TRY(layer(2, PA_S2, 128, -1, 0, PA_E3, H / 8, W / 8));
    HELM_TRY(s2d(PA_E3, PA_S3, 32, H / 8, W / 8));
    HELM_TRY(layer(3, PA_S3, 128, -1, 0, PA_E4, H / 16, W / 16));
  }
  HELM_TRY(layer(4, PA_E4, 32, -1, 0, PA_D3, H / 16, W / 16));      // -> H/8
  HELM_TRY(layer(5, PA_D3, 32, PA_E3, 32, PA_D2, H / 8, W / 8));    // -> H/4
  HELM_TRY(layer(6, PA_D2, 32, PA_E2, 32, PA_D1, H / 4, W / 4));    // -> H/2
  if constexpr (!fp64) {
    // the last transposed conv with the output layer in its epilogue (no full-resolution activation)
    RowFinal f;
    f.wf = P.wout32;
    f.out_scale = out_scale;
    f.z = (float2*)z;
    f.Nx = s.Nx;
    f.Ny = s.Ny;
    f.zstride = s.n;
    f.io = nullptr;
    return layer(7, PA_D1, 32, PA_E1, 32, -1, H / 2, W / 2, false, &f);
  } else {
    HELM_TRY(layer(7, PA_D1, 32, PA_E1, 32, PA_D0, H / 2, W / 2));  // -> H
  }
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


// ================================================================== training (eqs. 8-9) of kind 1
//
// Forward keeping every layer's input and pre-activation: on the mixed path (R = FP32) the tcgen05
// layers of the preconditioner in BF16 with FP32 accumulation (activations and pre-activations
// stored in BF16, the encoder inputs rearranged space-to-depth for the weight gradients), on the
// FP64 path (gradient checks) CUDA cores in FP64.  Backward on CUDA cores, gradients in E = R,
// in reverse through the same reformulated layers:
//   PReLU:  g_pre = g_post (pre > 0 ? 1 : a),  dL/da = sum g_post (pre > 0 ? 0 : pre);
//   up layer: the pre-activation gradient on the 2H x 2W grid is rearranged space-to-depth into the
//     GEMM's 4 C_out columns (column q C_out + co = output phase q), the inverse of the forward's
//     depth-to-space;
//   5x5 GEMM layer: dW[tap][k][n] = sum_px in[px + tap][k] g[px][n] (split over pixels, FP64
//     partials summed in a fixed order), db[n] = sum_px g[px][n], d in[q][k] = sum_{tap,n}
//     W[tap][k][n] g[q - tap][n];
//   down layer: the input gradient is on the space-to-depth tensor; depth-to-space returns it to the
//     previous activation.  Concatenated inputs split into the decoder and skip gradients.
// Each master weight of an 8x8 layer appears exactly once among the 5x5 taps, so its gradient is read
// back from there (the structural zeros' gradients are dropped).

constexpr int PW_THREADS = 256;  // weight-gradient block: 16 x 16 threads

// Forward GEMM layer on CUDA cores with the pre-activation kept (up: both written depth-to-space).
template <typename E>
__global__ void __launch_bounds__(PC_THREADS) k_pconv_keep(const E* __restrict__ in0, int C0, const E* __restrict__ in1,
                                                           int C1, const E* __restrict__ w5,
                                                           const double* __restrict__ b5, E* __restrict__ pre,
                                                           E* __restrict__ post, int N, int cout, int up, int B,
                                                           int H, int W, int ks, double slope) {
  const int64_t pix = blockIdx.x * (int64_t)PC_THREADS + threadIdx.x;
  if (pix >= (int64_t)B * H * W) return;
  const int n0 = blockIdx.y * 16;
  const int x = (int)(pix % W);
  const int y = (int)((pix / W) % H);
  const int64_t b = pix / ((int64_t)W * H);
  const int K = C0 + C1, r = ks / 2;
  E acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = (E)b5[n0 + k];
  for (int tap = 0; tap < ks * ks; ++tap) {
    const int yy = y + tap / ks - r, xx = x + tap % ks - r;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    const int64_t q = (b * H + yy) * W + xx;
    const E* wt = w5 + (int64_t)tap * K * N + n0;
    for (int c = 0; c < K; ++c) {
      const E v = c < C0 ? in0[q * C0 + c] : in1[q * C1 + (c - C0)];
      const E* wr = wt + (int64_t)c * N;
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[k] += v * wr[k];
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int n = n0 + k;
    int64_t o;
    if (!up) {
      o = pix * N + n;
    } else {
      const int q = n / cout, co = n % cout;
      o = ((b * 2 * H + 2 * y + (q >> 1)) * (2 * W) + 2 * x + (q & 1)) * cout + co;
    }
    if (pre) pre[o] = acc[k];
    if (post) post[o] = acc[k] > E(0) ? acc[k] : (E)slope * acc[k];
  }
}

// Depth-to-space (inverse of k_s2d): out[b][2Y + py][2X + px][c] = in[b][Y][X][(py * 2 + px) C + c].
template <typename E>
__global__ void k_d2s(const E* __restrict__ in, E* __restrict__ out, int C, int B, int Hi, int Wi, int accumulate) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)B * Hi * Wi * 4 * C;
  if (e >= total) return;
  const int k = (int)(e % (4 * C));
  const int64_t pix = e / (4 * C);
  const int X = (int)(pix % Wi);
  const int Y = (int)((pix / Wi) % Hi);
  const int64_t b = pix / ((int64_t)Wi * Hi);
  const int ph = k / C, c = k % C;
  const int64_t o = ((b * 2 * Hi + 2 * Y + (ph >> 1)) * (2 * Wi) + 2 * X + (ph & 1)) * C + c;
  out[o] = accumulate ? out[o] + in[e] : in[e];
}

// PReLU backward in place on g (g_post -> g_pre); per-block partial sums of dL/da.  pre: the kept
// pre-activation (E, or BF16 on the mixed path).
template <typename E, typename T>
__global__ void k_prelu_bwd(E* __restrict__ g, const T* __restrict__ pre, int64_t n, double slope,
                            double* __restrict__ partial) {
  __shared__ double red[256 / 32];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const E p = (E)to_acc(pre[i]), gv = g[i];
    if (p > E(0)) {
      g[i] = gv;
    } else {
      s += (double)gv * (double)p;
      g[i] = gv * (E)slope;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// Weight gradient of a KS x KS GEMM layer: partial[split][tap][k][n] = sum over the split's pixels of
// in[px + tap][k] g[px][n]; one block per (split, 64 x 64 (k, n) tile, tap), each thread a 4 x 4
// register tile of outer-product sums over 32-pixel chunks staged in shared memory.  With
// tap == ks * ks (an extra grid slice) the block sums g for the bias instead (k tile 0 only).  Each
// block accumulates its split in E (FP32 on the training path); the splits are summed in FP64.  The
// activations are of type T (E, or BF16 on the mixed path).
constexpr int PW_TK = 64, PW_TN = 64, PW_PX = 32;
template <typename E, typename T>
__global__ void __launch_bounds__(PW_THREADS) k_pwgrad(const T* __restrict__ in0, int C0, int S0,
                                                       const T* __restrict__ in1, int C1, int S1,
                                                       const E* __restrict__ g, int N, int B, int H, int W, int ks,
                                                       int nsplit, double* __restrict__ partial,
                                                       double* __restrict__ bpartial) {
  const int K = C0 + C1, r = ks / 2;
  const int split = blockIdx.x, tap = blockIdx.z;
  const int nkt = (K + PW_TK - 1) / PW_TK;
  const int k0 = (blockIdx.y % nkt) * PW_TK, n0 = (blockIdx.y / nkt) * PW_TN;
  const int tk = threadIdx.x & 15, tn = threadIdx.x >> 4;  // this thread: k0 + 4 tk + i, n0 + 4 tn + j
  const int64_t P = (int64_t)B * H * W;
  const int64_t pb = P * split / nsplit, pe = P * (split + 1) / nsplit;
  __shared__ __align__(16) E xs[PW_PX][PW_TK];
  __shared__ __align__(16) E gs[PW_PX][PW_TN];
  __shared__ int64_t sq[PW_PX];  // the tap's input pixel of each chunk pixel (-1: outside / past the split)
  __shared__ int64_t sp[PW_PX];  // the chunk pixel itself (-1: past the split)
  const bool bias = tap == ks * ks;
  if (bias && k0 != 0) return;
  const int dy = bias ? 0 : tap / ks - r, dx = bias ? 0 : tap % ks - r;
  E acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int64_t p0 = pb; p0 < pe; p0 += PW_PX) {
    if (threadIdx.x < PW_PX) {
      const int64_t px = p0 + threadIdx.x;
      int64_t q = -1, pp = -1;
      if (px < pe) {
        pp = px;
        const int x = (int)(px % W);
        const int y = (int)((px / W) % H);
        const int64_t b = px / ((int64_t)W * H);
        const int yy = y + dy, xx = x + dx;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) q = (b * H + yy) * W + xx;
      }
      sq[threadIdx.x] = q;
      sp[threadIdx.x] = pp;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < PW_PX * PW_TK; e += PW_THREADS) {
      const int p = e / PW_TK, c = e % PW_TK;
      const int k = k0 + c, n = n0 + c;
      E xv = 0, gv = 0;
      if (bias) {
        xv = (c == 0 && sp[p] >= 0) ? E(1) : E(0);
      } else if (k < K && sq[p] >= 0) {
        const int64_t q = sq[p];
        xv = (E)to_acc(k < C0 ? in0[q * S0 + k] : in1[q * S1 + (k - C0)]);
      }
      if (n < N && sp[p] >= 0) gv = g[sp[p] * N + n];
      xs[p][c] = xv;
      gs[p][c] = gv;
    }
    __syncthreads();
#pragma unroll 4
    for (int p = 0; p < PW_PX; ++p) {
      E xv[4], gv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xv[i] = xs[p][4 * tk + i];
        gv[i] = gs[p][4 * tn + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += xv[i] * gv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + 4 * tk + i, n = n0 + 4 * tn + j;
      if (n >= N) continue;
      if (bias) {
        if (k == 0) bpartial[(int64_t)split * N + n] = (double)acc[i][j];
      } else if (k < K) {
        partial[(((int64_t)split * ks * ks + tap) * K + k) * N + n] = (double)acc[i][j];
      }
    }
}

// Sum the split partials in a fixed order: gw[tap][k][n], gb[n].
__global__ void k_pwgrad_reduce(const double* __restrict__ partial, const double* __restrict__ bpartial, int nsplit,
                                int64_t nw, int N, double* __restrict__ gw, double* __restrict__ gb) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nw) {
    double s = 0;
    for (int sp = 0; sp < nsplit; ++sp) s += partial[(int64_t)sp * nw + e];
    gw[e] = s;
  }
  if (e < N) {
    double s = 0;
    for (int sp = 0; sp < nsplit; ++sp) s += bpartial[(int64_t)sp * N + e];
    gb[e] = s;
  }
}

// Input gradient of a KS x KS GEMM layer: gin[q][k] = sum_{tap, n} W[tap][k][n] g[q - tap][n]; channels
// k < C0 go to gin0 (C0 per pixel), the rest to gin1.  One block per (64 pixels, 64 channels), each
// thread a 4 x 4 register tile; per tap, 32-column chunks of g (rows of the tap-shifted pixels) and
// of the tap's weights are staged in shared memory.
constexpr int PD_PX = 64, PD_TK = 64, PD_NC = 32;
template <typename E>
__global__ void __launch_bounds__(256) k_pdgrad(const E* __restrict__ g, int N, const E* __restrict__ w5,
                                                E* __restrict__ gin0, int C0, E* __restrict__ gin1, int C1, int B,
                                                int H, int W, int ks) {
  const int K = C0 + C1, r = ks / 2;
  const int64_t P = (int64_t)B * H * W;
  const int64_t q0 = (int64_t)blockIdx.x * PD_PX;
  const int k0 = blockIdx.y * PD_TK;
  const int tq = threadIdx.x >> 4, tk = threadIdx.x & 15;  // pixels q0 + 4 tq + i, channels k0 + 4 tk + j
  __shared__ __align__(16) E gs[PD_PX][PD_NC + 1];
  __shared__ __align__(16) E ws[PD_NC][PD_TK];
  __shared__ int sy[PD_PX], sx[PD_PX];
  __shared__ int64_t sb[PD_PX], ssrc[PD_PX];
  if (threadIdx.x < PD_PX) {
    const int64_t q = q0 + threadIdx.x;
    if (q < P) {
      sx[threadIdx.x] = (int)(q % W);
      sy[threadIdx.x] = (int)((q / W) % H);
      sb[threadIdx.x] = q / ((int64_t)W * H);
    } else {
      sb[threadIdx.x] = -1;
    }
  }
  E acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int tap = 0; tap < ks * ks; ++tap) {
    __syncthreads();
    if (threadIdx.x < PD_PX) {  // the output pixel that read this one at `tap`
      int64_t src = -1;
      if (sb[threadIdx.x] >= 0) {
        const int yy = sy[threadIdx.x] - (tap / ks - r), xx = sx[threadIdx.x] - (tap % ks - r);
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) src = (sb[threadIdx.x] * H + yy) * W + xx;
      }
      ssrc[threadIdx.x] = src;
    }
    const E* wt = w5 + (int64_t)tap * K * N;
    for (int nc = 0; nc < N; nc += PD_NC) {
      __syncthreads();
      for (int e = threadIdx.x; e < PD_PX * PD_NC; e += 256) {
        const int p = e / PD_NC, c = e % PD_NC;
        const int64_t src = ssrc[p];
        gs[p][c] = (src >= 0 && nc + c < N) ? g[src * N + nc + c] : E(0);
      }
      for (int e = threadIdx.x; e < PD_NC * PD_TK; e += 256) {
        const int c = e / PD_TK, kk = e % PD_TK;
        const int k = k0 + kk, n = nc + c;
        ws[c][kk] = (k < K && n < N) ? wt[(int64_t)k * N + n] : E(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int c = 0; c < PD_NC; ++c) {
        E gv[4], wv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) gv[i] = gs[4 * tq + i][c];
#pragma unroll
        for (int j = 0; j < 4; ++j) wv[j] = ws[c][4 * tk + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += gv[i] * wv[j];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t q = q0 + 4 * tq + i;
    if (q >= P) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int kk = k0 + 4 * tk + j;
      if (kk < C0)
        gin0[q * C0 + kk] = acc[i][j];
      else if (kk < K)
        gin1[q * C1 + (kk - C0)] = acc[i][j];
    }
  }
}

// Gradient of the network output from the loss: g[b][y][x][0..1] = coef[b] (Re, Im)(A^H r) on the
// physical grid, 0 on the padding; coef = -2 out_scale / (B ||b||^2).
template <typename R, typename E>
__global__ void k_ploss_out(const C<R>* __restrict__ ahr, const double* __restrict__ sums,
                            const double* __restrict__ out_scale, int Nx, int Ny, int Hp, int Wp, int B,
                            E* __restrict__ gy) {
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)B * Hp * Wp) return;
  const int x = (int)(pix % Wp);
  const int y = (int)((pix / Wp) % Hp);
  const int b = (int)(pix / ((int64_t)Wp * Hp));
  E g0 = 0, g1 = 0;
  if (x < Nx && y < Ny) {
    const double bb = sums[2 * b + 1];
    const double c = bb > 0 ? -2.0 * out_scale[b] / (B * bb) : 0.0;
    const C<R> a = ahr[(int64_t)b * Nx * Ny + (int64_t)y * Nx + x];
    g0 = (E)(c * a.x);
    g1 = (E)(c * a.y);
  }
  gy[pix * 2] = g0;
  gy[pix * 2 + 1] = g1;
}

__global__ void k_palpha(const double* __restrict__ nb2, int B, int64_t n, double h2, double* __restrict__ in_s,
                         double* __restrict__ out_s) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double nv = sqrt(nb2[b]);
  const double a = nv > 0 ? sqrt((double)n) / nv : 0.0;
  in_s[b] = a;
  out_s[b] = a > 0 ? h2 / a : 0.0;
}

// Master-layout gradient of one layer from its reformulated weight gradient (see k_paper_reform).
__global__ void k_pgather(const double* __restrict__ gw5, const double* __restrict__ gb5,
                          const double* __restrict__ slope_parts, int nparts, int kind, int cin, int cpad, int cout,
                          int K, int N, int64_t m_w, int64_t m_b, int64_t m_s, double* __restrict__ grad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nw = (int64_t)cin * cout * (kind == P_OUT ? 1 : 64);
  if (e < nw) {
    double v;
    if (kind == P_OUT) {
      const int co = (int)(e / cin), ci = (int)(e % cin);
      v = gw5[(int64_t)ci * N + co];
    } else {
      const int tx = (int)(e % 8), ty = (int)((e / 8) % 8);
      const int a = (int)((e / 64) % (kind == P_DOWN ? cin : cout));
      const int z = (int)(e / (64 * (int64_t)(kind == P_DOWN ? cin : cout)));
      if (kind == P_DOWN) {  // master [co = z][ci = a][ty][tx]
        const int py = (ty - 3) & 1, px = (tx - 3) & 1;
        const int dy = (ty - 3 - py) / 2, dx = (tx - 3 - px) / 2;
        const int tap = (dy + 2) * 5 + dx + 2, k = (py * 2 + px) * cpad + a;
        v = gw5[((int64_t)tap * K + k) * N + z];
      } else {  // master [ci = z][co = a][ty][tx]
        const int qy = (ty - 3) & 1, qx = (tx - 3) & 1;
        const int dy = (qy - (ty - 3)) / 2, dx = (qx - (tx - 3)) / 2;
        const int tap = (dy + 2) * 5 + dx + 2, n = (qy * 2 + qx) * cout + a;
        v = gw5[((int64_t)tap * K + z) * N + n];
      }
    }
    grad[m_w + e] = v;
  }
  if (e < cout) {
    double v = gb5[e];
    if (kind == P_UP) v = gb5[e] + gb5[cout + e] + gb5[2 * cout + e] + gb5[3 * cout + e];
    grad[m_b + e] = v;
  }
  if (e == 0 && kind != P_OUT) {
    double t = 0;
    for (int i = 0; i < nparts; ++i) t += slope_parts[i];  // fixed order
    grad[m_s] = t;
  }
}

template <typename E, typename T>
static helm_status pwgrad(const T* in0, int C0, const T* in1, int C1, const E* g, int N, int B, int H, int W, int ks,
                          double* partial, double* bpartial, int nsplit, double* gw, double* gb, cudaStream_t st) {
  const int K = C0 + C1;
  dim3 grid(nsplit, ((K + PW_TK - 1) / PW_TK) * ((N + PW_TN - 1) / PW_TN), ks * ks + 1);
  launch(k_pwgrad<E, T>, grid, PW_THREADS, 0, st, in0, C0, C0, in1, C1, C1, g, N, B, H, W, ks, nsplit, partial,
         bpartial);
  const int64_t nw = (int64_t)ks * ks * K * N;
  launch(k_pwgrad_reduce, cdiv(std::max<int64_t>(nw, N), 256), 256, 0, st, (const double*)partial,
         (const double*)bpartial, nsplit, nw, N, gw, gb);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

// The tiled gradient kernels for the 3x3 layers of network kind 0 (train.cu): weight-gradient split
// partials [split][tap][C0 + C1][N] (in0 / in1 with channel strides S0 / S1; no bias slice) and the
// input gradient of a ks x ks conv with weights [tap][K][N].
template <typename E, typename T>
helm_status conv_wgrad_tiled(const T* in0, int C0, int S0, const T* in1, int C1, int S1, const E* g, int N, int B,
                             int H, int W, int ks, int nsplit, double* partial, cudaStream_t st) {
  const int K = C0 + C1;
  dim3 grid(nsplit, ((K + PW_TK - 1) / PW_TK) * ((N + PW_TN - 1) / PW_TN), ks * ks);
  launch(k_pwgrad<E, T>, grid, PW_THREADS, 0, st, in0, C0, S0, in1, C1, S1, g, N, B, H, W, ks, nsplit, partial,
         (double*)nullptr);
  HELM_CK_LAUNCH();
  return HELM_OK;
}
template helm_status conv_wgrad_tiled<float, __nv_bfloat16>(const __nv_bfloat16*, int, int, const __nv_bfloat16*, int,
                                                            int, const float*, int, int, int, int, int, int, double*,
                                                            cudaStream_t);
template helm_status conv_wgrad_tiled<double, double>(const double*, int, int, const double*, int, int, const double*,
                                                      int, int, int, int, int, int, double*, cudaStream_t);

template <typename E>
helm_status conv_dgrad_tiled(const E* g, int N, const E* w, E* gin0, int C0, E* gin1, int C1, int B, int H, int W,
                             int ks, cudaStream_t st) {
  dim3 grid(cdiv((int64_t)B * H * W, PD_PX), cdiv(C0 + C1, PD_TK));
  launch(k_pdgrad<E>, grid, 256, 0, st, g, N, w, gin0, C0, gin1, C1, B, H, W, ks);
  HELM_CK_LAUNCH();
  return HELM_OK;
}
template helm_status conv_dgrad_tiled<float>(const float*, int, const float*, float*, int, float*, int, int, int, int,
                                             int, cudaStream_t);
template helm_status conv_dgrad_tiled<double>(const double*, int, const double*, double*, int, double*, int, int, int,
                                              int, int, cudaStream_t);

// Output layer for training: z = out_scale (y0 + i y1), y = D0 Wout + bout with unrounded weights.
template <typename E, typename R>
__global__ void k_pfinal(const E* __restrict__ in, const double* __restrict__ w5, const double* __restrict__ b5,
                         const double* __restrict__ out_scale, int Nx, int Ny, int Hp, int Wp, int B,
                         C<R>* __restrict__ z, int64_t col_stride) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * Ny * Nx) return;
  const int x = (int)(e % Nx);
  const int y = (int)((e / Nx) % Ny);
  const int b = (int)(e / ((int64_t)Nx * Ny));
  const E* ip = in + (((int64_t)b * Hp + y) * Wp + x) * 32;
  E y0 = (E)b5[0], y1 = (E)b5[1];
  for (int c = 0; c < 32; ++c) {
    y0 += ip[c] * (E)w5[c * 2 + 0];
    y1 += ip[c] * (E)w5[c * 2 + 1];
  }
  const double sc = out_scale[b];
  z[b * col_stride + (int64_t)y * Nx + x] = mk<R>((R)(y0 * sc), (R)(y1 * sc));
}

template <typename R>
helm_status paper_loss_grad(helm_ctx* ctx, helm_unet* net, const C<R>* bvec, double* loss_host, cudaStream_t st) {
  using E = R;  // gradients: FP32 (training) or FP64 (checks)
  constexpr bool mixed = sizeof(R) == 4;
  using T = typename std::conditional<mixed, __nv_bfloat16, double>::type;  // activations
  PaperNet& P = *net->pn;
  const SysHost& s0 = ctx->sys[0];
  for (auto& s : ctx->sys)
    if (s.Nx != s0.Nx || s.Ny != s0.Ny || s.h != s0.h || s.p != s0.p)
      return fail(HELM_ERR_INVALID_ARG, "training batches need systems of one grid size, spacing and PML");
  const int B = ctx->nsys;
  const int Hp = (s0.Ny + 15) / 16 * 16, Wp = (s0.Nx + 15) / 16 * 16;
  const int64_t full = (int64_t)Hp * Wp, npx = B * full;
  HELM_TRY(ensure_cols(ctx, 1));
  if (!net->grad) HELM_CK(cudaMalloc(&net->grad, sizeof(double) * net->L.total));
  auto wts = [&](int l) -> const E* {  // reformulated weights in the arithmetic type
    if constexpr (sizeof(E) == 8)
      return P.w5[l];
    else
      return P.w5f[l];
  };
  // ---- workspace: activations and pre-activations (E), gradients (E), FP64 partials
  const int64_t el_act[13] = {8 * full, 32 * full / 4, 32 * full / 4, 128 * full / 16, 32 * full / 16,
                              128 * full / 64, 32 * full / 64, 128 * full / 256, 32 * full / 256, 32 * full / 64,
                              32 * full / 16, 32 * full / 4, 32 * full};
  const int64_t el_pre[8] = {32 * full / 4, 32 * full / 16, 32 * full / 64, 32 * full / 256,
                             32 * full / 64, 32 * full / 16, 32 * full / 4, 32 * full};
  constexpr int NSPLIT = 64, NPP = 1024;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  size_t o_act[13], o_pre[8];
  for (int k = 0; k < 13; ++k) o_act[k] = take(sizeof(T) * el_act[k] * B);
  for (int k = 0; k < 8; ++k) o_pre[k] = take(sizeof(T) * el_pre[k] * B);
  const size_t o_z = take(sizeof(C<R>) * ctx->npts), o_r = take(sizeof(C<R>) * ctx->npts),
               o_ahr = take(sizeof(C<R>) * ctx->npts);
  const size_t o_gy = take(sizeof(E) * 2 * npx);
  const size_t o_ga = take(sizeof(E) * 32 * npx), o_gb = take(sizeof(E) * 32 * npx), o_gc = take(sizeof(E) * 8 * npx);
  const size_t o_ge[4] = {take(sizeof(E) * 32 * npx / 4), take(sizeof(E) * 32 * npx / 16),
                          take(sizeof(E) * 32 * npx / 64), take(sizeof(E) * 32 * npx / 256)};
  const size_t o_part = take(sizeof(double) * (size_t)NSPLIT * 25 * 64 * 128),
               o_bpart = take(sizeof(double) * NSPLIT * 128), o_gw = take(sizeof(double) * 25 * 64 * 128),
               o_gbias = take(sizeof(double) * 128), o_pp = take(sizeof(double) * NPP),
               o_sc = take(sizeof(double) * 5 * B);
  HELM_TRY(ctx->ws_train.reserve(off));
  char* base = (char*)ctx->ws_train.ptr;
  T* a[13];
  T* pre[8];
  for (int k = 0; k < 13; ++k) a[k] = (T*)(base + o_act[k]);
  for (int k = 0; k < 8; ++k) pre[k] = (T*)(base + o_pre[k]);
  C<R>* z = (C<R>*)(base + o_z);
  C<R>* rres = (C<R>*)(base + o_r);
  C<R>* ahr = (C<R>*)(base + o_ahr);
  E* gy = (E*)(base + o_gy);
  E* gA = (E*)(base + o_ga);
  E* gB = (E*)(base + o_gb);
  E* gC = (E*)(base + o_gc);
  E* gE[4];
  for (int k = 0; k < 4; ++k) gE[k] = (E*)(base + o_ge[k]);
  double* part = (double*)(base + o_part);
  double* bpart = (double*)(base + o_bpart);
  double* gw = (double*)(base + o_gw);
  double* gbias = (double*)(base + o_gbias);
  double* pp = (double*)(base + o_pp);
  double* nb2 = (double*)(base + o_sc);
  double* in_s = nb2 + B;
  double* out_s = in_s + B;
  double* sums = out_s + B;  // 2 B entries: ||r||^2, ||b||^2 per sample
  const int H = Hp, W = Wp;

  // ---- forward, keeping every layer's input and pre-activation
  HELM_TRY(col_norm2<R>(ctx, bvec, 1, nb2, st));
  launch(k_palpha, cdiv(B, 64), 64, 0, st, (const double*)nb2, B, s0.n, s0.h * s0.h, in_s, out_s);
  launch(k_paper_pack<T, R>, dim3(cdiv(Wp, PACK_THREADS), Hp), PACK_THREADS, 0, st, bvec, s0.n, (const double*)in_s,
         (const double*)(ctx->chat64), s0.n, (const double2*)(ctx->prof_d + s0.prof_x),
         (const double2*)(ctx->prof_d + s0.prof_y), s0.Nx, s0.Ny, Hp, Wp, B, a[PA_S0]);
  auto s2d_act = [&](const T* src, T* dst, int C, int h, int w) {  // h, w: source grid
    const int64_t n = (int64_t)B * (h / 2) * (w / 2) * 4 * C;
    launch(k_s2d<T>, cdiv(n, 256), 256, 0, st, src, dst, C, B, h / 2, w / 2);
  };
  auto s2d = [&](const E* src, E* dst, int C, int h, int w) {  // h, w: source grid
    const int64_t n = (int64_t)B * (h / 2) * (w / 2) * 4 * C;
    launch(k_s2d<E>, cdiv(n, 256), 256, 0, st, src, dst, C, B, h / 2, w / 2);
  };
  helm_status fst = HELM_OK;
  auto fwd = [&](int l, const T* i0, int C0, const T* i1, int C1, int h, int w) {
    const PaperLayer& L = kP[l];
    T* post = a[l < 4 ? PA_E1 + 2 * l : PA_D3 + (l - 4)];
    if constexpr (mixed) {
      if (fst == HELM_OK)
        fst = conv_tc_generic(P.wtc[l], P.b32[l], P.err, 5, L.kind == P_UP ? 2 : 0, L.N, L.chunk, i0, C0, i1, C1, post,
                              B, h, w, 2, (float)P.slope[l], st, false, nullptr, nullptr, pre[l]);
    } else {
      dim3 grid(cdiv((int64_t)B * h * w, PC_THREADS), L.N / 16);
      launch(k_pconv_keep<T>, grid, PC_THREADS, 0, st, i0, C0, i1, C1, wts(l), (const double*)P.b5[l], pre[l], post,
             L.N, L.cout, L.kind == P_UP ? 1 : 0, B, h, w, 5, P.slope[l]);
    }
  };
  fwd(0, a[PA_S0], 32, nullptr, 0, H / 2, W / 2);
  s2d_act(a[PA_E1], a[PA_S1], 32, H / 2, W / 2);
  fwd(1, a[PA_S1], 128, nullptr, 0, H / 4, W / 4);
  s2d_act(a[PA_E2], a[PA_S2], 32, H / 4, W / 4);
  fwd(2, a[PA_S2], 128, nullptr, 0, H / 8, W / 8);
  s2d_act(a[PA_E3], a[PA_S3], 32, H / 8, W / 8);
  fwd(3, a[PA_S3], 128, nullptr, 0, H / 16, W / 16);
  fwd(4, a[PA_E4], 32, nullptr, 0, H / 16, W / 16);
  fwd(5, a[PA_D3], 32, a[PA_E3], 32, H / 8, W / 8);
  fwd(6, a[PA_D2], 32, a[PA_E2], 32, H / 4, W / 4);
  fwd(7, a[PA_D1], 32, a[PA_E1], 32, H / 2, W / 2);
  HELM_TRY(fst);
  if constexpr (mixed)  // the output layer with the BF16-rounded weights of the preconditioner
    launch(k_paper_final<T, R>, cdiv((int64_t)B * s0.n, 256), 256, 0, st, (const T*)a[PA_D0], P.wout32,
           P.wout32 + 64, (const double*)out_s, s0.Nx, s0.Ny, Hp, Wp, B, z, s0.n);
  else
    launch(k_pfinal<T, R>, cdiv((int64_t)B * s0.n, 256), 256, 0, st, (const T*)a[PA_D0],
           (const double*)P.w5[PAPER_LAYERS - 1], (const double*)P.b5[PAPER_LAYERS - 1], (const double*)out_s,
           s0.Nx, s0.Ny, Hp, Wp, B, z, s0.n);
  HELM_CK_LAUNCH();
  // ---- loss (eq. 9) and the gradient of the network output
  HELM_TRY(residual_op<R>(ctx, z, bvec, rres, 1, sums, st));
  HELM_TRY(apply_op<R>(ctx, rres, ahr, 1, true, st));
  launch(k_ploss_out<R, E>, cdiv(npx, 256), 256, 0, st, (const C<R>*)ahr, (const double*)sums, (const double*)out_s,
         s0.Nx, s0.Ny, Hp, Wp, B, gy);
  HELM_CK_LAUNCH();

  // ---- backward
  auto gather = [&](int l, int nparts) {
    const PaperLayer& L = kP[l];
    const int64_t nw = (int64_t)L.cin * L.cout * (L.kind == P_OUT ? 1 : 64);
    launch(k_pgather, cdiv(std::max<int64_t>(nw, L.cout), 256), 256, 0, st, (const double*)gw, (const double*)gbias,
           (const double*)pp, nparts, L.kind, L.cin, l == 0 ? P_X0_CH : L.cin, L.cout, L.K, L.N, P.m_w[l], P.m_b[l],
           P.m_s[l], net->grad);
  };
  auto prelu_bwd = [&](int l, E* g, int64_t n) {
    const int nb = (int)std::min<int64_t>(NPP, cdiv(n, 256));
    launch(k_prelu_bwd<E, T>, nb, 256, 0, st, g, (const T*)pre[l], n, P.slope[l], pp);
    return nb;
  };
  auto dgrad = [&](const E* g, int N, int l, E* gin0, int C0, E* gin1, int C1, int h, int w, int ks) {
    dim3 grid(cdiv((int64_t)B * h * w, PD_PX), cdiv(C0 + C1, PD_TK));
    launch(k_pdgrad<E>, grid, 256, 0, st, g, N, wts(l), gin0, C0, gin1, C1, B, h, w, ks);
  };
  auto d2s_acc = [&](const E* gs, E* gprev, int C, int hi, int wi) {  // gs on the half grid hi x wi
    const int64_t n = (int64_t)B * hi * wi * 4 * C;
    launch(k_d2s<E>, cdiv(n, 256), 256, 0, st, gs, gprev, C, B, hi, wi, 1);
  };
  // output layer (1 x 1, N = 2): weights, bias, input gradient
  HELM_TRY((pwgrad<E, T>(a[PA_D0], 32, (const T*)nullptr, 0, gy, 2, B, H, W, 1, part, bpart, NSPLIT, gw, gbias, st)));
  gather(PAPER_LAYERS - 1, 0);
  dgrad(gy, 2, PAPER_LAYERS - 1, gA, 32, nullptr, 0, H, W, 1);  // gD0 -> gA
  // decoder: l = 7 (d0) .. 4 (d3); the post-activation gradient in gA is on the layer's output grid
  const int dec_h[4] = {H / 2, H / 4, H / 8, H / 16};  // GEMM grids of l = 7, 6, 5, 4
  for (int i = 0; i < 4; ++i) {
    const int l = 7 - i, h = dec_h[i], w = W * h / H;
    const int64_t nout = (int64_t)B * (2 * h) * (2 * w) * 32;
    const int nparts = prelu_bwd(l, gA, nout);                       // gA: g_pre on the 2h x 2w grid
    s2d(gA, gB, 32, 2 * h, 2 * w);                                   // gB: GEMM columns on h x w (128)
    const T* in0 = a[l == 4 ? PA_E4 : PA_D3 + (l - 4) - 1];          // decoder input of this layer
    const T* in1 = l == 4 ? nullptr : a[PA_E4 - 2 * (l - 4)];        // skip (e_3, e_2, e_1 for l = 5, 6, 7)
    const int C1 = l == 4 ? 0 : 32;
    HELM_TRY((pwgrad<E, T>(in0, 32, in1, C1, gB, 128, B, h, w, 5, part, bpart, NSPLIT, gw, gbias, st)));
    gather(l, nparts);
    E* ge = gE[7 - l];                                               // e_1 (l = 7) .. e_4 (l = 4) grad
    if (l == 4)
      dgrad(gB, 128, l, ge, 32, nullptr, 0, h, w, 5);                // g e_4
    else
      dgrad(gB, 128, l, gA, 32, ge, 32, h, w, 5);                    // g d_{next} -> gA, g skip -> ge
  }
  // encoder: l = 3 (e4) .. 0 (e1); gE[l] holds the post-activation gradient of e_{l+1}
  for (int l = 3; l >= 0; --l) {
    const int h = H >> (l + 1), w = W >> (l + 1);
    const int64_t nout = (int64_t)B * h * w * 32;
    const int nparts = prelu_bwd(l, gE[l], nout);
    const T* in = a[PA_S0 + 2 * l];                                   // S0, S1, S2, S3
    const int K = l == 0 ? 32 : 128;
    HELM_TRY((pwgrad<E, T>(in, K, (const T*)nullptr, 0, gE[l], 32, B, h, w, 5, part, bpart, NSPLIT, gw, gbias, st)));
    gather(l, nparts);
    if (l > 0) {
      dgrad(gE[l], 32, l, gC, 128, nullptr, 0, h, w, 5);             // gradient on S_l (128 channels)
      d2s_acc(gC, gE[l - 1], 32, h, w);                              // back to e_l, added to its skip part
    }
  }
  HELM_CK_LAUNCH();
  if (loss_host) {
    std::vector<double> hs(2 * B);
    HELM_CK(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, st));
    HELM_CK(cudaStreamSynchronize(st));
    double L = 0;
    for (int k = 0; k < B; ++k) L += hs[2 * k + 1] > 0 ? hs[2 * k] / hs[2 * k + 1] : 0.0;
    *loss_host = L / B;
  }
  return HELM_OK;
}

template helm_status paper_loss_grad<float>(helm_ctx*, helm_unet*, const float2*, double*, cudaStream_t);
template helm_status paper_loss_grad<double>(helm_ctx*, helm_unet*, const double2*, double*, cudaStream_t);

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_paper_layer_forward(const helm_unet* net, int layer, const void* in0, const void* in1,
                                                void* out, int B, int H, int W, void* stream) {
  if (!net || !in0 || !out) return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: NULL argument");
  if (net->kind != 1 || !net->pn) return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: network kind 1 only");
  if (layer < 0 || layer > HELM_PAPER_LAYER_DEC0_FINAL)
    return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: layer out of range");
  if (B < 1 || H < 1 || W < 1 || (int64_t)B * H * W > ((int64_t)1 << 29))
    return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: bad image size");
  if (((uintptr_t)in0 | (uintptr_t)in1 | (uintptr_t)out) & 15)
    return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: pointers must be 16-byte aligned");
  const bool fused = layer == HELM_PAPER_LAYER_DEC0_FINAL;
  const int l = fused ? 7 : layer;
  if ((l >= 5) != (in1 != nullptr))
    return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: in1 is required exactly for layers 5..7");
  if (!tc_available())
    return fail(HELM_ERR_INVALID_ARG, "helm_paper_layer_forward: the tcgen05 path is not available on this device");
  const PaperNet& P = *net->pn;
  const PaperLayer& L = kP[l];
  RowFinal f;
  if (fused) {
    f.wf = P.wout32;
    f.out_scale = nullptr;
    f.z = (float2*)out;
    f.Nx = 2 * W;
    f.Ny = 2 * H;
    f.zstride = (int64_t)4 * H * W;
    f.io = nullptr;
  }
  if (l <= 2 && H % 2 == 0 && W % 2 == 0)  // the phase form of enc1..enc3 (output grid with even sides)
    return conv_tc_phase(P.wq[l], P.bq[l], P.err, l == 0 ? 2 : 4, in0, out, B, H / 2, W / 2, (float)P.slope[l],
                         (cudaStream_t)stream, nullptr);
  const int C0 = l == 0 ? 4 * P_X0_CH : (l <= 3 ? 128 : 32), C1 = l >= 5 ? 32 : 0;
  return conv_tc_generic(P.wtc[l], P.b32[l], P.err, 5, L.kind == P_UP ? 2 : 0, L.N, L.chunk, in0, C0, in1, C1,
                         fused ? nullptr : out, B, H, W, 2, (float)P.slope[l], (cudaStream_t)stream,
                         l >= 1 && l <= 3, fused ? &f : nullptr, nullptr);
}
