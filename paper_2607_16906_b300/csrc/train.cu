// Physics-informed training (a9): the loss of eq. 9 averaged over a batch (eq. 8), its gradient by
// the adjoint stencil and backward kernels through the U-Net, global-norm clipping and AdamW.
//
// Batch = the context's systems (all of one grid size), one source each.  Per sample
//   u = (h^2 / alpha) N(alpha b, c),  alpha = sqrt(n) / ||b||,   L = ||b - A u||^2 / ||b||^2,
//   dL/du (Re + i Im) = -2 A^H (b - A u) / (B ||b||^2),   dL/dy = (h^2 / alpha) dL/du.
// Backward through the network follows the forward in reverse: final 1x1 conv, then per decoder
// level conv(ReLU) x2 with the concat gradient split into skip and up-conv parts, transposed conv,
// bottleneck, encoder levels with the max-pool gradient routed to the first maximum of each window
// (row-major order) and added to the skip gradient.
// Two arithmetic paths, like the forward: BF16 activations with FP32 gradients and accumulation
// (training), FP64 throughout (gradient checks).  Weight gradients are split-K reductions over
// pixels with FP64 partials combined in a fixed order (deterministic).
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "unet.cuh"

namespace helm {

constexpr int BW_THREADS = 128;
constexpr int BW_CT = 16;  // channels per thread in the up-conv input-gradient kernel

// ------------------------------------------------------------------ elementwise / small kernels

template <typename T, typename G>
__global__ void k_relu_mask(G* __restrict__ g, const T* __restrict__ act, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !(to_acc(act[i]) > 0)) g[i] = G(0);
}

// coef[b] = -2 out_scale[b] / (B ||b||^2)  (sums[2b+1] = ||b||^2)
__global__ void k_loss_coef(const double* __restrict__ sums, const double* __restrict__ out_scale, int B,
                            double* __restrict__ coef) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double bb = sums[2 * b + 1];
  coef[b] = bb > 0 ? -2.0 * out_scale[b] / (B * bb) : 0.0;
}

// gy[b][y][x][0..1] = coef[b] (Re, Im)(A^H r)[b][y][x] on the physical grid, 0 on the padding.
template <typename R, typename G>
__global__ void k_grad_out(const C<R>* __restrict__ ahr, const double* __restrict__ coef, int Nx, int Ny, int Hp,
                           int Wp, int B, G* __restrict__ gy) {
  int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)B * Hp * Wp) return;
  int x = (int)(pix % Wp);
  int y = (int)((pix / Wp) % Hp);
  int b = (int)(pix / ((int64_t)Wp * Hp));
  G g0 = 0, g1 = 0;
  if (x < Nx && y < Ny) {
    C<R> a = ahr[(int64_t)b * Nx * Ny + (int64_t)y * Nx + x];
    double c = coef[b];
    g0 = (G)(c * a.x);
    g1 = (G)(c * a.y);
  }
  gy[pix * 2] = g0;
  gy[pix * 2 + 1] = g1;
}

// Final 1x1 conv backward to its input: g_in[pix][ci] = sum_co W[ci][co] gy[pix][co].
template <typename G, typename A>
__global__ void k_final_dgrad(const G* __restrict__ gy, const A* __restrict__ W, G* __restrict__ gin, int64_t npix) {
  int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  A g0 = gy[pix * 2], g1 = gy[pix * 2 + 1];
#pragma unroll
  for (int ci = 0; ci < 16; ++ci) gin[pix * 16 + ci] = (G)(W[ci * 2] * g0 + W[ci * 2 + 1] * g1);
}

// 2x2 stride-2 transposed conv backward to its input:
// g_in[b,i,j,ci] = sum_{dy,dx,co} W[dy*2+dx][ci][co] g_out[b,2i+dy,2j+dx,co].
template <typename G, typename A>
__global__ void __launch_bounds__(BW_THREADS) k_up_dgrad(const G* __restrict__ gout, const A* __restrict__ W,
                                                         G* __restrict__ gin, int Cin, int Cout, int B, int Hi,
                                                         int Wi) {
  int64_t pix = blockIdx.x * (int64_t)BW_THREADS + threadIdx.x;
  if (pix >= (int64_t)B * Hi * Wi) return;
  int ci0 = blockIdx.y * BW_CT;
  int j = (int)(pix % Wi);
  int i = (int)((pix / Wi) % Hi);
  int64_t b = pix / ((int64_t)Wi * Hi);
  A acc[BW_CT];
#pragma unroll
  for (int k = 0; k < BW_CT; ++k) acc[k] = 0;
  for (int t = 0; t < 4; ++t) {
    int yo = 2 * i + (t >> 1), xo = 2 * j + (t & 1);
    const G* gp = gout + ((b * 2 * Hi + yo) * (2 * Wi) + xo) * Cout;
    const A* wt = W + ((int64_t)t * Cin + ci0) * Cout;
    for (int co = 0; co < Cout; ++co) {
      A gv = gp[co];
#pragma unroll
      for (int k = 0; k < BW_CT; ++k) acc[k] += wt[(int64_t)k * Cout + co] * gv;
    }
  }
#pragma unroll
  for (int k = 0; k < BW_CT; ++k) gin[pix * Cin + ci0 + k] = (G)acc[k];
}

// Max-pool backward: route g_p to the first maximum (row-major) of each 2x2 window of s; add to g_s.
template <typename T, typename G>
__global__ void k_pool_bwd(const G* __restrict__ gp, const T* __restrict__ s, G* __restrict__ gs, int C, int B, int Ho,
                           int Wo) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * Ho * Wo * C) return;
  int c = (int)(e % C);
  int64_t pix = e / C;
  int x = (int)(pix % Wo);
  int y = (int)((pix / Wo) % Ho);
  int64_t b = pix / ((int64_t)Wo * Ho);
  int Wi = 2 * Wo;
  int64_t base = ((b * 2 * Ho + 2 * y) * Wi + 2 * x) * C + c;
  int64_t off[4] = {0, C, (int64_t)Wi * C, (int64_t)Wi * C + C};
  int best = 0;
  auto m = to_acc(s[base]);
  for (int k = 1; k < 4; ++k) {
    auto v = to_acc(s[base + off[k]]);
    if (v > m) {
      m = v;
      best = k;
    }
  }
  gs[base + off[best]] += gp[e];
}

// ------------------------------------------------------------------ weight gradients (split-K)

// partial[((split * taps + tap) * Cin + ci) * Cout + co] = sum over the split's GEMM rows of
// in(row, ci, tap) * g(row, co, tap).  Rows: output pixels (3x3, 1x1) or input pixels (2x2 up-conv).
template <typename T, typename G, int KIND>
__global__ void __launch_bounds__(256) k_wgrad(const T* __restrict__ in0, int C0, int S0, const T* __restrict__ in1,
                                               int C1, int S1, const G* __restrict__ g, int Cout, int B, int H,
                                               int Wd, int nsplit, int taps, double* __restrict__ partial) {
  using A = typename Acc<T>::A;
  const int Cin = C0 + C1;
  const int split = blockIdx.x, tile = blockIdx.y, tap = blockIdx.z;
  const int nco = (Cout + 15) / 16;
  const int ci0 = (tile / nco) * 16, co0 = (tile % nco) * 16;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t K = (int64_t)B * H * Wd;
  const int64_t kb = K * split / nsplit, ke = K * (split + 1) / nsplit;
  __shared__ A xs[32][17];
  __shared__ A gs[32][17];
  const int ky = KIND == CONV3 ? tap / 3 : 0, kx = KIND == CONV3 ? tap % 3 : 0;
  const int dy = KIND == UP2 ? tap >> 1 : 0, dx = KIND == UP2 ? tap & 1 : 0;
  A acc = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += 32) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      int p = e >> 4, c = e & 15;
      int64_t row = k0 + p;
      A xv = 0, gv = 0;
      if (row < ke) {
        int x = (int)(row % Wd);
        int y = (int)((row / Wd) % H);
        int64_t b = row / ((int64_t)Wd * H);
        int ci = ci0 + c;
        if (ci < Cin) {
          int64_t q = -1;
          if (KIND == CONV3) {
            int yy = y + ky - 1, xx = x + kx - 1;
            if (yy >= 0 && yy < H && xx >= 0 && xx < Wd) q = (b * H + yy) * Wd + xx;
          } else {
            q = row;
          }
          if (q >= 0) xv = ci < C0 ? to_acc(in0[q * S0 + ci]) : to_acc(in1[q * S1 + ci - C0]);
        }
        int co = co0 + c;
        if (co < Cout) {
          int64_t gq = KIND == UP2 ? ((b * 2 * H + 2 * y + dy) * (2 * Wd) + 2 * x + dx) : row;
          gv = (A)g[gq * Cout + co];
        }
      }
      xs[p][c] = xv;
      gs[p][c] = gv;
    }
    __syncthreads();
#pragma unroll 8
    for (int p = 0; p < 32; ++p) acc += xs[p][ty] * gs[p][tx];
    __syncthreads();
  }
  int ci = ci0 + ty, co = co0 + tx;
  if (ci < Cin && co < Cout) partial[(((int64_t)split * taps + tap) * Cin + ci) * Cout + co] = (double)acc;
}

// partial[split * Cout + co] = sum over the split's pixels of g[pix][co]
template <typename G>
__global__ void __launch_bounds__(256) k_bias_grad(const G* __restrict__ g, int Cout, int64_t npix, int nsplit,
                                                   double* __restrict__ partial) {
  const int lanes = 256 / Cout;
  const int t = threadIdx.x;
  const int lane = t / Cout, co = t % Cout;
  const int64_t kb = npix * blockIdx.x / nsplit, ke = npix * (blockIdx.x + 1) / nsplit;
  double acc = 0;
  if (lane < lanes)
    for (int64_t p = kb + lane; p < ke; p += lanes) acc += (double)g[p * Cout + co];
  __shared__ double red[256];
  red[t] = lane < lanes ? acc : 0.0;
  __syncthreads();
  if (t < Cout) {
    double s = 0;
    for (int l = 0; l < lanes; ++l) s += red[l * Cout + t];
    partial[(int64_t)blockIdx.x * Cout + t] = s;
  }
}

// Sum the split partials (fixed order) and scatter into the master (PyTorch) layout.
__global__ void k_wgrad_reduce(const double* __restrict__ partial, int nsplit, int kind, int taps, int cin, int cout,
                               int64_t m_w, double* __restrict__ grad) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t nw = (int64_t)taps * cin * cout;
  if (q >= nw) return;
  double s = 0;
  for (int sp = 0; sp < nsplit; ++sp) s += partial[(int64_t)sp * nw + q];
  int tap = (int)(q / ((int64_t)cin * cout));
  int rem = (int)(q % ((int64_t)cin * cout));
  int ci = rem / cout, co = rem % cout;
  int64_t dst;
  if (kind == CONV3)
    dst = m_w + ((int64_t)(co * cin + ci) * 3 + tap / 3) * 3 + tap % 3;
  else if (kind == UP2)
    dst = m_w + ((int64_t)(ci * cout + co) * 2 + tap / 2) * 2 + tap % 2;
  else
    dst = m_w + (int64_t)co * cin + ci;
  grad[dst] = s;
}

__global__ void k_bias_reduce(const double* __restrict__ partial, int nsplit, int cout, int64_t m_b,
                              double* __restrict__ grad) {
  int co = threadIdx.x;
  if (co >= cout) return;
  double s = 0;
  for (int sp = 0; sp < nsplit; ++sp) s += partial[(int64_t)sp * cout + co];
  grad[m_b + co] = s;
}

// ------------------------------------------------------------------ optimiser

__global__ void k_sumsq(const double* __restrict__ v, int64_t n, double* __restrict__ partial) {
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += v[i] * v[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// AdamW (decoupled weight decay): p <- p (1 - lr wd); m, v moments of g * gscale; bias-corrected step.
__global__ void k_adamw(double* __restrict__ p, const double* __restrict__ grad, double* __restrict__ m,
                        double* __restrict__ v, int64_t n, double lr, double wd, double b1, double b2, double eps,
                        double c1, double c2, double gscale) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g = grad[i] * gscale;
  double pi = p[i] * (1.0 - lr * wd);
  double mi = b1 * m[i] + (1.0 - b1) * g;
  double vi = b2 * v[i] + (1.0 - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  p[i] = pi - lr * (mi / c1) / (sqrt(vi / c2) + eps);
}

// ------------------------------------------------------------------ backward driver

// Per-slot channel counts and resolution level (0 full, 1 half, 2 quarter, 3 eighth).
static const int kSlotCh[NUM_ACTS] = {X0_CH, 16, 16, 16, 32, 32, 32, 64, 64, 64, 128, 128, 64, 64, 64, 32, 32, 32, 16, 16, 16};
static const int kSlotLv[NUM_ACTS] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};

struct GradSet {
  void* g[NUM_ACTS] = {};
  void* gy = nullptr;
  double* wpart = nullptr;  // split-K partials (largest layer)
  size_t wpart_doubles = 0;
  double* misc = nullptr;   // small per-sample vectors
};

constexpr int MAX_SPLIT = 64;

static helm_status grad_buffers(helm_ctx* ctx, int B, int Hp, int Wp, size_t es, GradSet& G) {
  size_t off = 0;
  size_t offs[NUM_ACTS + 3];
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  int64_t f = (int64_t)Hp * Wp;
  for (int a = 1; a < NUM_ACTS; ++a) offs[a] = take((size_t)B * (f >> (2 * kSlotLv[a])) * kSlotCh[a] * es);
  offs[NUM_ACTS] = take((size_t)B * f * 2 * es);
  size_t wp = (size_t)MAX_SPLIT * 9 * 128 * 128;
  offs[NUM_ACTS + 1] = take(wp * sizeof(double));
  offs[NUM_ACTS + 2] = take(sizeof(double) * 64 * 1024);
  HELM_TRY(ctx->ws_train.reserve(off));
  char* base = (char*)ctx->ws_train.ptr;
  for (int a = 1; a < NUM_ACTS; ++a) G.g[a] = base + offs[a];
  G.gy = base + offs[NUM_ACTS];
  G.wpart = (double*)(base + offs[NUM_ACTS + 1]);
  G.wpart_doubles = wp;
  G.misc = (double*)(base + offs[NUM_ACTS + 2]);
  return HELM_OK;
}

template <typename E, typename T>
helm_status conv_wgrad_tiled(const T* in0, int C0, int S0, const T* in1, int C1, int S1, const E* g, int N, int B,
                             int H, int W, int ks, int nsplit, double* partial, cudaStream_t st);
template <typename E>
helm_status conv_dgrad_tiled(const E* g, int N, const E* w, E* gin0, int C0, E* gin1, int C1, int B, int H, int W,
                             int ks, cudaStream_t st);

static int pick_split(int64_t K, int tiles, int taps) {
  int s = (int)std::max<int64_t>(1, 2048 / std::max(1, tiles * taps));
  s = (int)std::min<int64_t>(s, std::max<int64_t>(1, K / 256));
  return std::min(s, MAX_SPLIT);
}

template <typename T, typename G>
struct Backward {
  using A = typename Acc<T>::A;
  helm_unet* net;
  UnetBuffers::Set& S;
  GradSet& GS;
  int B, H, W;
  cudaStream_t st;

  T* act(int a) const { return (T*)S.a[a]; }
  G* grd(int a) const { return (G*)GS.g[a]; }
  const A* weights() const { return cc_weights<T>(net); }

  helm_status mask(int a, int lv) {
    int64_t n = (int64_t)B * (H >> lv) * (W >> lv) * kSlotCh[a];
    launch(k_relu_mask<T, G>, cdiv(n, 256), 256, 0, st, grd(a), (const T*)act(a), n);
    return HELM_OK;
  }

  // weight + bias gradients of layer l given its output gradient g (pre-activation) at the given grid
  helm_status wgrad(int l, const T* in0, int C0, int S0, const T* in1, int C1, int S1, const G* g, int h, int w) {
    const LayerDesc& d = kLayers[l];
    int taps = taps_of(d.kind);
    // 3x3 layers: 64 x 64 register-tiled blocks (unet_paper.cu); up-convs and the 1x1 layer: 16 x 16
    int tiles = d.kind == CONV3 ? ((d.cin + 63) / 64) * ((d.cout + 63) / 64) : ((d.cin + 15) / 16) * ((d.cout + 15) / 16);
    int64_t K = (int64_t)B * h * w;
    int ns = pick_split(K, tiles, taps);
    if ((size_t)ns * taps * d.cin * d.cout > GS.wpart_doubles) return fail(HELM_ERR_INVALID_ARG, "wgrad scratch too small");
    dim3 grid(ns, tiles, taps);
    if (d.kind == CONV3)
      HELM_TRY((conv_wgrad_tiled<G, T>(in0, C0, S0, in1, C1, S1, g, d.cout, B, h, w, 3, ns, GS.wpart, st)));
    else if (d.kind == UP2)
      launch(k_wgrad<T, G, UP2>, grid, 256, 0, st, in0, C0, S0, in1, C1, S1, g, d.cout, B, h, w, ns, taps, GS.wpart);
    else
      launch(k_wgrad<T, G, CONV1>, grid, 256, 0, st, in0, C0, S0, in1, C1, S1, g, d.cout, B, h, w, ns, taps, GS.wpart);
    int64_t nw = (int64_t)taps * d.cin * d.cout;
    launch(k_wgrad_reduce, cdiv(nw, 256), 256, 0, st, (const double*)GS.wpart, ns, d.kind, taps, d.cin, d.cout,
           net->L.m_w[l], net->grad);
    // bias: the rows of the bias gradient are the output pixels (2x2 up-conv: the output grid)
    int64_t npix = d.kind == UP2 ? (int64_t)B * 2 * h * 2 * w : K;
    int nsb = (int)std::min<int64_t>(MAX_SPLIT * 8, std::max<int64_t>(1, npix / 4096));
    double* bp = GS.misc;
    launch(k_bias_grad<G>, nsb, 256, 0, st, g, d.cout, npix, nsb, bp);
    launch(k_bias_reduce, 1, 128, 0, st, (const double*)bp, nsb, d.cout, net->L.m_b[l], net->grad);
    HELM_CK_LAUNCH();
    return HELM_OK;
  }

  helm_status dgrad3(int l, const G* gpre, G* out0, int C0, G* out1, int C1, int h, int w) {
    const LayerDesc& d = kLayers[l];
    static_assert(std::is_same<A, G>::value, "the tiled input gradient reads weights in the gradient type");
    return conv_dgrad_tiled<G>(gpre, d.cout, weights() + net->L.c_w[l], out0, C0, out1, C1, B, h, w, 3, st);
  }

  helm_status up_dgrad(int l, const G* gout, G* gin, int hi, int wi) {
    const LayerDesc& d = kLayers[l];
    dim3 grid(cdiv((int64_t)B * hi * wi, BW_THREADS), d.cin / BW_CT);
    launch(k_up_dgrad<G, A>, grid, BW_THREADS, 0, st, gout, weights() + net->L.c_w[l], gin, d.cin, d.cout, B, hi, wi);
    return HELM_OK;
  }

  helm_status pool_bwd(int gp, int s, int C, int lv_out) {
    int ho = H >> lv_out, wo = W >> lv_out;
    int64_t n = (int64_t)B * ho * wo * C;
    launch(k_pool_bwd<T, G>, cdiv(n, 256), 256, 0, st, (const G*)grd(gp), (const T*)act(s), grd(s), C, B, ho, wo);
    return HELM_OK;
  }

  // a conv3 layer with ReLU output slot `o`, whose input was (in0: C0 ch, in1: C1 ch) at level lv;
  // dgrad targets (d0, d1) may be null for the first layer.
  helm_status conv_layer(int l, int o, int lv, int in0, int C0, int S0, int in1, int C1, G* d0, G* d1) {
    int h = H >> lv, w = W >> lv;
    HELM_TRY(mask(o, lv));
    HELM_TRY(wgrad(l, act(in0), C0, S0, in1 >= 0 ? act(in1) : nullptr, C1, C1, grd(o), h, w));
    if (d0) HELM_TRY(dgrad3(l, grd(o), d0, C0, d1, C1, h, w));
    return HELM_OK;
  }

  helm_status run() {
    G* gy = (G*)GS.gy;
    const A* wf = weights() + net->L.c_w[L_FINAL];
    int64_t npix = (int64_t)B * H * W;
    // final 1x1 conv
    HELM_TRY(wgrad(L_FINAL, act(A_D1B), 16, 16, nullptr, 0, 0, gy, H, W));
    launch(k_final_dgrad<G, A>, cdiv(npix, 256), 256, 0, st, (const G*)gy, wf, grd(A_D1B), npix);
    // decoder level 1
    HELM_TRY(conv_layer(L_DEC1B, A_D1B, 0, A_D1A, 16, 16, -1, 0, grd(A_D1A), nullptr));
    HELM_TRY(conv_layer(L_DEC1A, A_D1A, 0, A_S1, 16, 16, A_U1, 16, grd(A_S1), grd(A_U1)));
    HELM_TRY(wgrad(L_UP1, act(A_D2B), 32, 32, nullptr, 0, 0, grd(A_U1), H >> 1, W >> 1));
    HELM_TRY(up_dgrad(L_UP1, grd(A_U1), grd(A_D2B), H >> 1, W >> 1));
    // decoder level 2
    HELM_TRY(conv_layer(L_DEC2B, A_D2B, 1, A_D2A, 32, 32, -1, 0, grd(A_D2A), nullptr));
    HELM_TRY(conv_layer(L_DEC2A, A_D2A, 1, A_S2, 32, 32, A_U2, 32, grd(A_S2), grd(A_U2)));
    HELM_TRY(wgrad(L_UP2, act(A_D3B), 64, 64, nullptr, 0, 0, grd(A_U2), H >> 2, W >> 2));
    HELM_TRY(up_dgrad(L_UP2, grd(A_U2), grd(A_D3B), H >> 2, W >> 2));
    // decoder level 3
    HELM_TRY(conv_layer(L_DEC3B, A_D3B, 2, A_D3A, 64, 64, -1, 0, grd(A_D3A), nullptr));
    HELM_TRY(conv_layer(L_DEC3A, A_D3A, 2, A_S3, 64, 64, A_U3, 64, grd(A_S3), grd(A_U3)));
    HELM_TRY(wgrad(L_UP3, act(A_BB), 128, 128, nullptr, 0, 0, grd(A_U3), H >> 3, W >> 3));
    HELM_TRY(up_dgrad(L_UP3, grd(A_U3), grd(A_BB), H >> 3, W >> 3));
    // bottleneck
    HELM_TRY(conv_layer(L_BOTB, A_BB, 3, A_BA, 128, 128, -1, 0, grd(A_BA), nullptr));
    HELM_TRY(conv_layer(L_BOTA, A_BA, 3, A_P3, 64, 64, -1, 0, grd(A_P3), nullptr));
    HELM_TRY(pool_bwd(A_P3, A_S3, 64, 3));
    // encoder level 3
    HELM_TRY(conv_layer(L_ENC3B, A_S3, 2, A_E3A, 64, 64, -1, 0, grd(A_E3A), nullptr));
    HELM_TRY(conv_layer(L_ENC3A, A_E3A, 2, A_P2, 32, 32, -1, 0, grd(A_P2), nullptr));
    HELM_TRY(pool_bwd(A_P2, A_S2, 32, 2));
    // encoder level 2
    HELM_TRY(conv_layer(L_ENC2B, A_S2, 1, A_E2A, 32, 32, -1, 0, grd(A_E2A), nullptr));
    HELM_TRY(conv_layer(L_ENC2A, A_E2A, 1, A_P1, 16, 16, -1, 0, grd(A_P1), nullptr));
    HELM_TRY(pool_bwd(A_P1, A_S1, 16, 1));
    // encoder level 1 (no input gradient needed for the first layer)
    HELM_TRY(conv_layer(L_ENC1B, A_S1, 0, A_E1A, 16, 16, -1, 0, grd(A_E1A), nullptr));
    HELM_TRY(conv_layer(L_ENC1A, A_E1A, 0, A_X0, 3, X0_CH, -1, 0, nullptr, nullptr));
    HELM_CK_LAUNCH();
    return HELM_OK;
  }
};

__global__ void k_alpha_b(const double* __restrict__ norm2, int B, int64_t n, double h2, double* __restrict__ in_scale,
                          double* __restrict__ out_scale) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= B) return;
  double nv = sqrt(norm2[c]);
  double a = nv > 0 ? sqrt((double)n) / nv : 0.0;
  in_scale[c] = a;
  out_scale[c] = a > 0 ? h2 / a : 0.0;
}

// Loss (eq. 8-9) and its gradient into net->grad (FP64, master layout).  R = float: BF16 network;
// R = double: FP64 network.
template <typename R>
static helm_status loss_grad_impl(helm_ctx* ctx, helm_unet* net, const C<R>* b, double* loss_host, cudaStream_t st) {
  if (net->kind == 1) return paper_loss_grad<R>(ctx, net, b, loss_host, st);
  using T = typename std::conditional<sizeof(R) == 8, double, __nv_bfloat16>::type;
  using G = typename std::conditional<sizeof(R) == 8, double, float>::type;
  const SysHost& s0 = ctx->sys[0];
  for (auto& s : ctx->sys)
    if (s.Nx != s0.Nx || s.Ny != s0.Ny || s.h != s0.h)
      return fail(HELM_ERR_INVALID_ARG, "training batches need systems of one grid size and spacing");
  const int B = ctx->nsys;
  const int Hp = (s0.Ny + 7) / 8 * 8, Wp = (s0.Nx + 7) / 8 * 8;
  HELM_TRY(ensure_cols(ctx, 1));
  if (!net->grad) HELM_CK(cudaMalloc(&net->grad, sizeof(double) * net->L.total));
  // vectors: u, r, A^H r (C<R>, npts each) in ws_vec; small per-sample arrays after them
  size_t vb = sizeof(C<R>) * ctx->npts;
  size_t vbr = (vb + 255) / 256 * 256;
  HELM_TRY(ctx->ws_vec.reserve(3 * vbr + sizeof(double) * 8 * B + 256));
  char* vbase = (char*)ctx->ws_vec.ptr;
  C<R>* u = (C<R>*)vbase;
  C<R>* r = (C<R>*)(vbase + vbr);
  C<R>* ahr = (C<R>*)(vbase + 2 * vbr);
  double* nb2 = (double*)(vbase + 3 * vbr);
  double* in_s = nb2 + B;
  double* out_s = in_s + B;
  double* sums = out_s + B;  // 2B
  double* coef = sums + 2 * B;
  HELM_TRY(col_norm2<R>(ctx, b, 1, nb2, st));
  launch(k_alpha_b, cdiv(B, 64), 64, 0, st, (const double*)nb2, B, s0.n, s0.h * s0.h, in_s, out_s);
  HELM_TRY(unet_precondition<R>(ctx, net, 0, b, u, B, in_s, out_s, st, s0.n, /*keep_acts=*/true));
  HELM_TRY(residual_op<R>(ctx, u, b, r, 1, sums, st));
  HELM_TRY(apply_op<R>(ctx, r, ahr, 1, true, st));
  launch(k_loss_coef, cdiv(B, 64), 64, 0, st, (const double*)sums, (const double*)out_s, B, coef);
  UnetBuffers* ub;
  HELM_TRY(ensure_buffers(ctx, B, Hp, Wp, sizeof(R) == 8, &ub));
  UnetBuffers::Set& S = ub->set[sizeof(R) == 8 ? 1 : 0];
  GradSet GS;
  HELM_TRY(grad_buffers(ctx, B, Hp, Wp, sizeof(G), GS));
  int64_t npix = (int64_t)B * Hp * Wp;
  launch(k_grad_out<R, G>, cdiv(npix, 256), 256, 0, st, (const C<R>*)ahr, (const double*)coef, s0.Nx, s0.Ny, Hp, Wp,
         B, (G*)GS.gy);
  HELM_CK_LAUNCH();
  Backward<T, G> bw{net, S, GS, B, Hp, Wp, st};
  HELM_TRY(bw.run());
  if (loss_host) {
    std::vector<double> h(2 * B);
    HELM_CK(cudaMemcpyAsync(h.data(), sums, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, st));
    HELM_CK(cudaStreamSynchronize(st));
    double L = 0;
    for (int k = 0; k < B; ++k) L += h[2 * k + 1] > 0 ? h[2 * k] / h[2 * k + 1] : 0.0;
    *loss_host = L / B;
  }
  return HELM_OK;
}

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_loss_grad(helm_ctx* ctx, const helm_unet* net, const void* b, helm_dtype dtype,
                                      double* loss_host, double* grad_dev, void* stream) {
  if (!ctx || !net || !b) return fail(HELM_ERR_INVALID_ARG, "helm_loss_grad: NULL argument");
  if ((uintptr_t)b & 15) return fail(HELM_ERR_INVALID_ARG, "helm_loss_grad: b must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  helm_unet* n = const_cast<helm_unet*>(net);
  if (dtype == HELM_C64)
    HELM_TRY(loss_grad_impl<float>(ctx, n, (const float2*)b, loss_host, st));
  else if (dtype == HELM_C128)
    HELM_TRY(loss_grad_impl<double>(ctx, n, (const double2*)b, loss_host, st));
  else
    return fail(HELM_ERR_INVALID_ARG, "helm_loss_grad: unknown dtype");
  if (grad_dev)
    HELM_CK(cudaMemcpyAsync(grad_dev, n->grad, sizeof(double) * n->L.total, cudaMemcpyDeviceToDevice, st));
  return HELM_OK;
}

extern "C" helm_status helm_train_step(helm_ctx* ctx, helm_unet* net, const void* b, double lr, double wd,
                                       double clip, double* loss_host, double* grad_norm_host, void* stream) {
  if (!ctx || !net || !b) return fail(HELM_ERR_INVALID_ARG, "helm_train_step: NULL argument");
  if (!(lr >= 0) || !(wd >= 0)) return fail(HELM_ERR_INVALID_ARG, "helm_train_step: lr and wd must be >= 0");
  if ((uintptr_t)b & 15) return fail(HELM_ERR_INVALID_ARG, "helm_train_step: b must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  double loss = 0;
  HELM_TRY(loss_grad_impl<float>(ctx, net, (const float2*)b, &loss, st));
  const int64_t P = net->L.total;
  if (!net->adam_m) {
    HELM_CK(cudaMalloc(&net->adam_m, sizeof(double) * P));
    HELM_CK(cudaMalloc(&net->adam_v, sizeof(double) * P));
    HELM_CK(cudaMemsetAsync(net->adam_m, 0, sizeof(double) * P, st));
    HELM_CK(cudaMemsetAsync(net->adam_v, 0, sizeof(double) * P, st));
    net->step = 0;
  }
  // global gradient norm (fixed-order two-stage reduction)
  const int nb = 256;
  HELM_TRY(ctx->ws_red.reserve(sizeof(double) * nb));
  double* part = (double*)ctx->ws_red.ptr;
  launch(k_sumsq, nb, 256, 0, st, (const double*)net->grad, P, part);
  std::vector<double> h(nb);
  HELM_CK(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  double ss = 0;
  for (double v : h) ss += v;
  double gn = sqrt(ss);
  HELM_TRY(conv_tc_check(net, st));  // a forward convolution gave up: no update from that gradient
  if (!std::isfinite(gn) || !std::isfinite(loss)) return fail(HELM_NAN, "helm_train_step: non-finite loss or gradient");
  double scale = (clip > 0 && gn > clip) ? clip / (gn + 1e-6) : 1.0;
  net->step += 1;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  double c1 = 1.0 - pow(b1, (double)net->step), c2 = 1.0 - pow(b2, (double)net->step);
  launch(k_adamw, cdiv(P, 256), 256, 0, st, net->master, (const double*)net->grad, net->adam_m, net->adam_v, P, lr,
         wd, b1, b2, eps, c1, c2, scale);
  HELM_CK_LAUNCH();
  HELM_TRY(net->kind == 1 ? paper_prepare(net, st) : unet_prepare(net, st));
  if (loss_host) *loss_host = loss;
  if (grad_norm_host) *grad_norm_host = gn;
  return HELM_OK;
}

extern "C" helm_status helm_unet_get_adam(const helm_unet* net, double* m_host, double* v_host, int64_t* step_host) {
  if (!net || !m_host || !v_host || !step_host) return fail(HELM_ERR_INVALID_ARG, "helm_unet_get_adam: NULL argument");
  const int64_t P = net->L.total;
  if (!net->adam_m) {  // no step taken yet: zero moments
    for (int64_t i = 0; i < P; ++i) m_host[i] = v_host[i] = 0.0;
    *step_host = 0;
    return HELM_OK;
  }
  HELM_CK(cudaDeviceSynchronize());
  HELM_CK(cudaMemcpy(m_host, net->adam_m, sizeof(double) * P, cudaMemcpyDeviceToHost));
  HELM_CK(cudaMemcpy(v_host, net->adam_v, sizeof(double) * P, cudaMemcpyDeviceToHost));
  *step_host = net->step;
  return HELM_OK;
}

extern "C" helm_status helm_unet_set_adam(helm_unet* net, const double* m_host, const double* v_host, int64_t step) {
  if (!net || !m_host || !v_host || step < 0) return fail(HELM_ERR_INVALID_ARG, "helm_unet_set_adam: bad argument");
  const int64_t P = net->L.total;
  if (!net->adam_m) {
    HELM_CK(cudaMalloc(&net->adam_m, sizeof(double) * P));
    HELM_CK(cudaMalloc(&net->adam_v, sizeof(double) * P));
  }
  HELM_CK(cudaDeviceSynchronize());
  HELM_CK(cudaMemcpy(net->adam_m, m_host, sizeof(double) * P, cudaMemcpyHostToDevice));
  HELM_CK(cudaMemcpy(net->adam_v, v_host, sizeof(double) * P, cudaMemcpyHostToDevice));
  net->step = step;
  return HELM_OK;
}
