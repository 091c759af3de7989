// Fourier-differentiation Helmholtz operator with PML (the paper's discretisation, Sec. 2.1, Tab. 1):
//
//   y = A_F u = -[ (1/s_x) D_x((1/s_x) D_x u) + (1/s_y) D_y((1/s_y) D_y u) ] - k^2 u,
//   D u = IDFT( i kappa DFT(u) ) along one axis, kappa_q = 2 pi q / (N h), the Nyquist mode zeroed,
//
// on the periodic N_x x N_y grid that includes the PML, with the node stretch factors s = 1 + i sigma /
// omega of eq. 2 (the same nodes the 5-point operator uses).  Grid sides are powers of two, 16..1024.
//
// Two passes, each one read of its inputs and one write:
//   x pass: DIF forward FFT of a grid row (natural order in, bit-reversed out), multiply by
//           i kappa / N at the bit-reversed position, DIT inverse FFT (bit-reversed in, natural out),
//           scale by 1/s_x, the same again -> t_x, written to y;
//   y pass: the same derivative pair along the columns -> t_y; then y = -(t_x + t_y) - k^2 u.
// FP32 with sides of 32 or more: one warp transforms one line held in registers (lane l, register r
// hold element l + 32 r): an in-register E-point FFT over r (E = N / 32), the twiddles of the
// N = 32 E split, and a 32-point FFT across the lanes by shuffles (for 1024-point lines a transpose
// of the 32 x 32 split through a per-warp shared-memory tile instead, so the second factor is also an
// in-register FFT); the x pass reads its rows straight into registers, the y pass stages 8 columns of
// the whole height in shared memory (64-byte row segments, a padded pitch so the column reads are
// free of bank conflicts), each thread keeping 8 loads in flight.  FP64 and sides of 16:
// block-wide radix-2 FFTs in shared memory (one block per row; 16 (FP32) or 8 (FP64) columns).
// Twiddle tables exp(-2 pi i t / N), t < N/2, are computed once per grid side on the host in FP64
// and staged into shared memory by every block.  HBM traffic per point: x pass 16 B (FP32), y pass
// 8 (u) + 8 (t_x) + 8 (u again) + 4 (k^2) + 8 (y) = 36 B: 52 B per point and right-hand side.
#include <math.h>

#include <map>
#include <mutex>
#include <vector>

#include "helm_internal.cuh"

namespace helm {

constexpr int FX_THREADS = 256;
constexpr int FY_THREADS = 256;
template <typename R> struct FyCols;
template <> struct FyCols<float> { static constexpr int v = 16; };
template <> struct FyCols<double> { static constexpr int v = 8; };

__device__ __forceinline__ int brev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// In-place radix-2 transforms of `ncols` interleaved columns of length N (element (i, c) at
// a[i * ncols + c]).  tw[t] = exp(-2 pi i t / N), t < N/2.
// DIF forward: natural order in, bit-reversed order out.
template <typename R>
__device__ void fft_dif(C<R>* a, int N, int ncols, const C<R>* tw, int tid, int nt) {
  for (int half = N >> 1, step = 1; half >= 1; half >>= 1, step <<= 1) {
    const int nb = (N >> 1) * ncols;
    for (int b = tid; b < nb; b += nt) {
      const int c = b % ncols, bb = b / ncols;
      const int k = bb & (half - 1), g = bb / half;
      const int i0 = g * 2 * half + k, i1 = i0 + half;
      const C<R> x0 = a[i0 * ncols + c], x1 = a[i1 * ncols + c];
      a[i0 * ncols + c] = cadd(x0, x1);
      a[i1 * ncols + c] = cmul(csub(x0, x1), tw[k * step]);
    }
    __syncthreads();
  }
}
// DIT inverse (conjugate twiddles, no 1/N): bit-reversed order in, natural order out.
template <typename R>
__device__ void ifft_dit(C<R>* a, int N, int ncols, const C<R>* tw, int tid, int nt) {
  for (int half = 1, step = N >> 1; half < N; half <<= 1, step >>= 1) {
    const int nb = (N >> 1) * ncols;
    for (int b = tid; b < nb; b += nt) {
      const int c = b % ncols, bb = b / ncols;
      const int k = bb & (half - 1), g = bb / half;
      const int i0 = g * 2 * half + k, i1 = i0 + half;
      const C<R> x0 = a[i0 * ncols + c], x1 = cmul(a[i1 * ncols + c], cconj(tw[k * step]));
      a[i0 * ncols + c] = cadd(x0, x1);
      a[i1 * ncols + c] = csub(x0, x1);
    }
    __syncthreads();
  }
}

// i kappa_q / N for the spectrum entry at bit-reversed position `pos` (q = brev(pos)).
template <typename R>
__device__ __forceinline__ C<R> ikappa(int pos, int N, int logn, R two_pi_over_L) {
  const int q = brev(pos, logn);
  if (q == (N >> 1)) return mk<R>(0, 0);
  const int qs = q < (N >> 1) ? q : q - N;
  return mk<R>(0, (R)qs * two_pi_over_L / (R)N);
}

// t = (1/s) D((1/s) D t) along the column direction of a (spectral derivative pair), in place.
// inv_s[i]: 1/s at node i.
template <typename R>
__device__ void derivative_pair(C<R>* a, int N, int logn, int ncols, const C<R>* tw, const C<R>* inv_s,
                                R two_pi_over_L, int tid, int nt) {
  for (int rep = 0; rep < 2; ++rep) {
    fft_dif<R>(a, N, ncols, tw, tid, nt);
    for (int e = tid; e < N * ncols; e += nt) a[e] = cmul(a[e], ikappa<R>(e / ncols, N, logn, two_pi_over_L));
    __syncthreads();
    ifft_dit<R>(a, N, ncols, tw, tid, nt);
    for (int e = tid; e < N * ncols; e += nt) a[e] = cmul(a[e], inv_s[e / ncols]);
    __syncthreads();
  }
}

// x pass: one block per (row, rhs).  prof: the system's x profile (s at the Nx nodes first).
template <typename R>
__global__ void __launch_bounds__(FX_THREADS) k_fourier_x(const C<R>* __restrict__ u, C<R>* __restrict__ tx,
                                                          const C<R>* __restrict__ prof, const C<R>* __restrict__ tw_g,
                                                          int Nx, int logn, int Ny, int64_t rhs_stride,
                                                          R two_pi_over_L) {
  extern __shared__ __align__(16) unsigned char fx_smem[];
  C<R>* a = (C<R>*)fx_smem;
  C<R>* tw = a + Nx;
  C<R>* inv_s = tw + Nx / 2;
  const int row = blockIdx.x, rhs = blockIdx.y;
  const int64_t base = rhs * rhs_stride + (int64_t)row * Nx;
  for (int i = threadIdx.x; i < Nx; i += blockDim.x) {
    a[i] = u[base + i];
    const C<R> s = prof[i];
    const R d = s.x * s.x + s.y * s.y;
    inv_s[i] = mk<R>(s.x / d, -s.y / d);
  }
  for (int t = threadIdx.x; t < Nx / 2; t += blockDim.x) tw[t] = tw_g[t];
  __syncthreads();
  derivative_pair<R>(a, Nx, logn, 1, tw, inv_s, two_pi_over_L, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < Nx; i += blockDim.x) tx[base + i] = a[i];
}

// y pass: one block per (column tile, rhs); y holds t_x on entry and A_F u on exit.
template <typename R>
__global__ void __launch_bounds__(FY_THREADS) k_fourier_y(const C<R>* __restrict__ u, C<R>* __restrict__ y,
                                                          const R* __restrict__ k2, const C<R>* __restrict__ prof,
                                                          const C<R>* __restrict__ tw_g, int Nx, int Ny, int logn,
                                                          int64_t rhs_stride, R two_pi_over_L) {
  constexpr int TC = FyCols<R>::v;
  extern __shared__ __align__(16) unsigned char fy_smem[];
  C<R>* a = (C<R>*)fy_smem;
  C<R>* tw = a + (size_t)Ny * TC;
  C<R>* inv_s = tw + Ny / 2;
  const int x0 = blockIdx.x * TC, rhs = blockIdx.y;
  const int64_t base = rhs * rhs_stride + x0;
  for (int e = threadIdx.x; e < Ny * TC; e += blockDim.x) a[e] = u[base + (int64_t)(e / TC) * Nx + (e % TC)];
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) {
    const C<R> s = prof[j];
    const R d = s.x * s.x + s.y * s.y;
    inv_s[j] = mk<R>(s.x / d, -s.y / d);
  }
  for (int t = threadIdx.x; t < Ny / 2; t += blockDim.x) tw[t] = tw_g[t];
  __syncthreads();
  derivative_pair<R>(a, Ny, logn, TC, tw, inv_s, two_pi_over_L, threadIdx.x, blockDim.x);
  for (int e = threadIdx.x; e < Ny * TC; e += blockDim.x) {
    const int64_t q = base + (int64_t)(e / TC) * Nx + (e % TC);
    const int64_t pt = (int64_t)(e / TC) * Nx + x0 + (e % TC);
    const C<R> uv = u[q];
    const R kk = k2[pt];
    const C<R> t = cadd(y[q], a[e]);
    y[q] = mk<R>(-t.x - kk * uv.x, -t.y - kk * uv.y);
  }
}

// ------------------------------------------------------------------ warp-register FFTs (FP32)

// W_N^t for 0 <= t < N from the half table tw (W_N^(t + N/2) = -W_N^t).
template <int N>
__device__ __forceinline__ float2 tw_full(const float2* tw, int t) {
  const float2 w = tw[t & (N / 2 - 1)];
  return t & (N / 2) ? make_float2(-w.x, -w.y) : w;
}

template <int E>
__device__ __forceinline__ int brev_e(int r) {
  int o = 0;
#pragma unroll
  for (int b = 1, c = E >> 1; b < E; b <<= 1, c >>= 1)
    if (r & b) o |= c;
  return o;
}

__device__ __forceinline__ float2 shfl_x(float2 v, int h) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, h), __shfl_xor_sync(0xffffffffu, v.y, h));
}

// Forward DFT of the N = 32 E points a (lane l, register r: point l + 32 r) without scaling; on exit
// position n holds X[brev_L(n)], L = log2 N.  tw: W_N^t, t < N/2.
template <int E>
__device__ __forceinline__ void warp_fft_fwd(float2 (&a)[E], const float2* tw, int lane) {
  constexpr int N = 32 * E;
  // E-point DIF over the registers (W_E^m = W_N^(32 m)): register r ends with frequency brev_e(r)
#pragma unroll
  for (int half = E / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      const int k = i % half, i0 = (i / half) * 2 * half + k, i1 = i0 + half;
      const float2 x0 = a[i0], x1 = a[i1];
      a[i0] = cadd(x0, x1);
      a[i1] = k == 0 ? csub(x0, x1) : cmul(csub(x0, x1), tw[32 * k * (E / (2 * half))]);
    }
  }
  // twiddles of the split: W_N^(lane k1)
#pragma unroll
  for (int r = 1; r < E; ++r) a[r] = cmul(a[r], tw_full<N>(tw, lane * brev_e<E>(r)));
  // 32-point DIF across the lanes (W_32^m = W_N^(E m)): lane l ends with frequency brev_5(l); the
  // stage loop stays rolled (its body takes any h) to keep the kernel's code small
#pragma unroll 1
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = lane & h;
    const float2 w = tw[(lane & (h - 1)) * (16 / h) * E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const float2 p = shfl_x(a[r], h);
      a[r] = upper ? cmul(csub(p, a[r]), w) : cadd(a[r], p);
    }
  }
}

// Inverse of warp_fft_fwd (conjugate twiddles, no 1/N): position n holds the spectrum at brev_L(n) on
// entry, point n in natural order on exit.
template <int E>
__device__ __forceinline__ void warp_fft_inv(float2 (&a)[E], const float2* tw, int lane) {
  constexpr int N = 32 * E;
#pragma unroll 1
  for (int h = 1; h <= 16; h <<= 1) {
    const bool upper = lane & h;
    const float2 w = cconj(tw[(lane & (h - 1)) * (16 / h) * E]);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const float2 t = upper ? cmul(a[r], w) : a[r];
      const float2 p = shfl_x(t, h);
      a[r] = upper ? csub(p, t) : cadd(t, p);
    }
  }
#pragma unroll
  for (int r = 1; r < E; ++r) a[r] = cmul(a[r], cconj(tw_full<N>(tw, lane * brev_e<E>(r))));
#pragma unroll
  for (int half = 1; half < E; half <<= 1) {
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      const int k = i % half, i0 = (i / half) * 2 * half + k, i1 = i0 + half;
      const float2 x0 = a[i0];
      const float2 x1 = k == 0 ? a[i1] : cmul(a[i1], cconj(tw[32 * k * (E / (2 * half))]));
      a[i0] = cadd(x0, x1);
      a[i1] = csub(x0, x1);
    }
  }
}

// 32-point transforms of the 32 registers of a lane (W_32^m = W_1024^(32 m)): DIF, natural order in,
// bit-reversed out; DIT with conjugate twiddles, bit-reversed in, natural out.
__device__ __forceinline__ void reg_dif32(float2 (&a)[32], const float2* tw) {
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = i % half, i0 = (i / half) * 2 * half + k, i1 = i0 + half;
      const float2 x0 = a[i0], x1 = a[i1];
      a[i0] = cadd(x0, x1);
      a[i1] = k == 0 ? csub(x0, x1) : cmul(csub(x0, x1), tw[32 * k * (16 / half)]);
    }
  }
}
__device__ __forceinline__ void reg_dit32_inv(float2 (&a)[32], const float2* tw) {
#pragma unroll
  for (int half = 1; half < 32; half <<= 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = i % half, i0 = (i / half) * 2 * half + k, i1 = i0 + half;
      const float2 x0 = a[i0];
      const float2 x1 = k == 0 ? a[i1] : cmul(a[i1], cconj(tw[32 * k * (16 / half)]));
      a[i0] = cadd(x0, x1);
      a[i1] = csub(x0, x1);
    }
  }
}

// N = 1024 = 32 x 32 with the transpose through shared memory instead of lane shuffles: forward,
// in-register DIF over r (register r: frequency k1 = brev_5(r)), twiddles W^(n2 k1), transpose
// (lane = k1, register = n2), in-register DIF over n2; position (lane, r) then holds X[lane + 32
// brev_5(r)].  ts: the warp's 32 x 33 scratch (padded pitch: conflict-free in both directions).
__device__ __forceinline__ void warp_fft1024_fwd(float2 (&a)[32], const float2* tw, float2* ts, int lane) {
  reg_dif32(a, tw);
#pragma unroll
  for (int r = 1; r < 32; ++r) a[r] = cmul(a[r], tw_full<1024>(tw, lane * brev_e<32>(r)));
#pragma unroll
  for (int r = 0; r < 32; ++r) ts[brev_e<32>(r) * 33 + lane] = a[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) a[r] = ts[lane * 33 + r];
  __syncwarp();
  reg_dif32(a, tw);
}
// Inverse (no 1/N): position (lane, r) holds the spectrum at lane + 32 brev_5(r) on entry, point
// lane + 32 r on exit.
__device__ __forceinline__ void warp_fft1024_inv(float2 (&a)[32], const float2* tw, float2* ts, int lane) {
  reg_dit32_inv(a, tw);
#pragma unroll
  for (int r = 1; r < 32; ++r) a[r] = cmul(a[r], cconj(tw_full<1024>(tw, r * lane)));
#pragma unroll
  for (int r = 0; r < 32; ++r) ts[lane * 33 + r] = a[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) a[r] = ts[brev_e<32>(r) * 33 + lane];
  __syncwarp();
  reg_dit32_inv(a, tw);
}

// t = (1/s) D((1/s) D t) on one line held by the warp; inv_s[n] = 1/s at point n; ts: the warp's
// transpose scratch (N = 1024 only).
template <int E>
__device__ __forceinline__ void warp_derivative_pair(float2 (&a)[E], const float2* tw, const float2* inv_s,
                                                     float two_pi_over_L, int lane, float2* ts) {
  constexpr int N = 32 * E;
  constexpr int LOGN = 5 + (E >= 2) + (E >= 4) + (E >= 8) + (E >= 16) + (E >= 32);
  if constexpr (E == 32) {
#pragma unroll 1
    for (int rep = 0; rep < 2; ++rep) {
      warp_fft1024_fwd(a, tw, ts, lane);
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int q = lane + 32 * brev_e<32>(r);
        const float c = q == N / 2 ? 0.0f : (float)(q < N / 2 ? q : q - N) * two_pi_over_L / (float)N;
        a[r] = make_float2(-c * a[r].y, c * a[r].x);
      }
      warp_fft1024_inv(a, tw, ts, lane);
#pragma unroll
      for (int r = 0; r < 32; ++r) a[r] = cmul(a[r], inv_s[lane + 32 * r]);
    }
  } else {
#pragma unroll 1
    for (int rep = 0; rep < 2; ++rep) {
      warp_fft_fwd<E>(a, tw, lane);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int q = (int)(__brev((unsigned)(lane + 32 * r)) >> (32 - LOGN));
        const float c = q == N / 2 ? 0.0f : (float)(q < N / 2 ? q : q - N) * two_pi_over_L / (float)N;
        a[r] = make_float2(-c * a[r].y, c * a[r].x);
      }
      warp_fft_inv<E>(a, tw, lane);
#pragma unroll
      for (int r = 0; r < E; ++r) a[r] = cmul(a[r], inv_s[lane + 32 * r]);
    }
  }
}

constexpr int FW_WARPS = 8;  // lines per block

// x pass, FP32, Nx = 32 E: warp w of block b transforms line b * 8 + w of the (rhs, row) lines.
template <int E>
__global__ void __launch_bounds__(FW_WARPS * 32) k_fourier_xw(const float2* __restrict__ u, float2* __restrict__ tx,
                                                             const float2* __restrict__ prof,
                                                             const float2* __restrict__ tw_g, int Ny, int nlines,
                                                             int64_t rhs_stride, float two_pi_over_L) {
  constexpr int N = 32 * E;
  __shared__ float2 tw[N / 2];
  __shared__ float2 inv_s[N];
  extern __shared__ __align__(16) unsigned char fxw_smem[];  // N = 1024: 33 x 32 scratch per warp
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float2 s = prof[i];
    const float d = s.x * s.x + s.y * s.y;
    inv_s[i] = make_float2(s.x / d, -s.y / d);
    if (i < N / 2) tw[i] = tw_g[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float2* ts = (float2*)fxw_smem + (threadIdx.x >> 5) * (32 * 33);
  const int line = blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
  if (line >= nlines) return;  // whole warps leave; no block-wide barrier follows
  const int rhs = line / Ny, row = line % Ny;
  const int64_t base = rhs * rhs_stride + (int64_t)row * N;
  float2 a[E];
#pragma unroll
  for (int r = 0; r < E; ++r) a[r] = u[base + lane + 32 * r];
  warp_derivative_pair<E>(a, tw, inv_s, two_pi_over_L, lane, ts);
#pragma unroll
  for (int r = 0; r < E; ++r) tx[base + lane + 32 * r] = a[r];
}

constexpr int FYW_COLS = 8;                 // columns per block (one warp each)
constexpr int FYW_PITCH = FYW_COLS + 1;     // padded row pitch of the shared column slab

// y pass, FP32, Ny = 32 E: one block per (8 columns, rhs); y holds t_x on entry and A_F u on exit.
template <int E>
__global__ void __launch_bounds__(FYW_COLS * 32, E >= 32 ? 1 : 2) k_fourier_yw(const float2* __restrict__ u, float2* __restrict__ y,
                                                                const float* __restrict__ k2,
                                                                const float2* __restrict__ prof,
                                                                const float2* __restrict__ tw_g, int Nx,
                                                                int64_t rhs_stride, float two_pi_over_L) {
  constexpr int N = 32 * E;
  extern __shared__ __align__(16) unsigned char fyw_smem[];
  float2* slab = (float2*)fyw_smem;       // [N][FYW_PITCH]
  float2* tw = slab + N * FYW_PITCH;       // [N / 2]
  float2* inv_s = tw + N / 2;              // [N]
  float2* tsb = inv_s + N;                 // N = 1024: 33 x 32 transpose scratch per warp
  const int x0 = blockIdx.x * FYW_COLS, rhs = blockIdx.y;
  const int64_t base = rhs * rhs_stride + x0;
  const int cols = min(FYW_COLS, Nx - x0);
  // The slab's global traffic: thread t serves column t % FYW_COLS and rows t / FYW_COLS + JSTEP k
  // (the 8 columns of a row are 64 contiguous bytes); its loads are issued BATCH at a time before
  // any of them is used, so that a thread keeps BATCH DRAM requests in flight instead of one.
  constexpr int NT = FYW_COLS * 32, JSTEP = NT / FYW_COLS, PER = N / JSTEP, BATCH = PER < 8 ? PER : 8;
  const int ct = threadIdx.x % FYW_COLS, jt = threadIdx.x / FYW_COLS;
  if (ct < cols)
    for (int k0 = 0; k0 < PER; k0 += BATCH) {
      float2 v[BATCH];
#pragma unroll
      for (int k = 0; k < BATCH; ++k) v[k] = u[base + (int64_t)(jt + (k0 + k) * JSTEP) * Nx + ct];
#pragma unroll
      for (int k = 0; k < BATCH; ++k) slab[(jt + (k0 + k) * JSTEP) * FYW_PITCH + ct] = v[k];
    }
  {
    constexpr int PI = (N + NT - 1) / NT;
    float2 sp[PI], tg[PI];
#pragma unroll
    for (int k = 0; k < PI; ++k) {
      const int i = threadIdx.x + k * NT;
      if (i < N) sp[k] = prof[i];
      if (i < N / 2) tg[k] = tw_g[i];
    }
#pragma unroll
    for (int k = 0; k < PI; ++k) {
      const int i = threadIdx.x + k * NT;
      if (i < N) {
        const float d = sp[k].x * sp[k].x + sp[k].y * sp[k].y;
        inv_s[i] = make_float2(sp[k].x / d, -sp[k].y / d);
      }
      if (i < N / 2) tw[i] = tg[k];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  if (c < cols) {
    float2 a[E];
#pragma unroll
    for (int r = 0; r < E; ++r) a[r] = slab[(lane + 32 * r) * FYW_PITCH + c];
    warp_derivative_pair<E>(a, tw, inv_s, two_pi_over_L, lane, tsb + c * (32 * 33));
#pragma unroll
    for (int r = 0; r < E; ++r) slab[(lane + 32 * r) * FYW_PITCH + c] = a[r];
  }
  __syncthreads();
  if (ct < cols)
    for (int k0 = 0; k0 < PER; k0 += BATCH) {
      float2 uv[BATCH], tv[BATCH];
      float kk[BATCH];
#pragma unroll
      for (int k = 0; k < BATCH; ++k) {
        const int64_t j = jt + (k0 + k) * JSTEP;
        uv[k] = u[base + j * Nx + ct];
        tv[k] = y[base + j * Nx + ct];
        kk[k] = k2[j * Nx + x0 + ct];
      }
#pragma unroll
      for (int k = 0; k < BATCH; ++k) {
        const int j = jt + (k0 + k) * JSTEP;
        const float2 t = cadd(tv[k], slab[j * FYW_PITCH + ct]);
        y[base + (int64_t)j * Nx + ct] = make_float2(-t.x - kk[k] * uv[k].x, -t.y - kk[k] * uv[k].y);
      }
    }
}

template <int E>
static void launch_fourier_w(int axis, const float2* x, float2* y, const float* k2, const float2* pr,
                             const float2* tw, int Nx, int Ny, int nrhs, int64_t n, float tpl, cudaStream_t st) {
  constexpr int N = 32 * E;
  const size_t scratch = E == 32 ? sizeof(float2) * 32 * 33 : 0;  // transpose scratch per warp
  if (axis == 0) {
    const int nlines = Ny * nrhs;
    const size_t sm = FW_WARPS * scratch;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_fourier_xw<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    launch(k_fourier_xw<E>, (nlines + FW_WARPS - 1) / FW_WARPS, FW_WARPS * 32, sm, st, x, y, pr, tw, Ny, nlines, n,
           tpl);
  } else {
    const size_t sm = sizeof(float2) * ((size_t)N * FYW_PITCH + N / 2 + N) + FYW_COLS * scratch;
    cudaFuncSetAttribute(k_fourier_yw<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    launch(k_fourier_yw<E>, dim3((Nx + FYW_COLS - 1) / FYW_COLS, nrhs), FYW_COLS * 32, sm, st, x, y, k2, pr, tw, Nx,
           n, tpl);
  }
}

// FP32 warp-register pass along one axis (0: x, 1: y) for a side of 32..1024; false if the side is
// outside that range (the block-wide kernels serve it).
static bool fourier_warp_pass(int axis, int side, const float2* x, float2* y, const float* k2, const float2* pr,
                              const float2* tw, int Nx, int Ny, int nrhs, int64_t n, float tpl, cudaStream_t st) {
  switch (side) {
    case 32: launch_fourier_w<1>(axis, x, y, k2, pr, tw, Nx, Ny, nrhs, n, tpl, st); return true;
    case 64: launch_fourier_w<2>(axis, x, y, k2, pr, tw, Nx, Ny, nrhs, n, tpl, st); return true;
    case 128: launch_fourier_w<4>(axis, x, y, k2, pr, tw, Nx, Ny, nrhs, n, tpl, st); return true;
    case 256: launch_fourier_w<8>(axis, x, y, k2, pr, tw, Nx, Ny, nrhs, n, tpl, st); return true;
    case 512: launch_fourier_w<16>(axis, x, y, k2, pr, tw, Nx, Ny, nrhs, n, tpl, st); return true;
    case 1024: launch_fourier_w<32>(axis, x, y, k2, pr, tw, Nx, Ny, nrhs, n, tpl, st); return true;
    default: return false;
  }
}

// ------------------------------------------------------------------ host side

static int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}

bool fourier_supported(int Nx, int Ny) {
  const int lx = log2_exact(Nx), ly = log2_exact(Ny);
  return lx >= 4 && lx <= 10 && ly >= 4 && ly <= 10;
}

// Twiddle tables of one grid side, FP64 and FP32, cached per process and device.
struct TwTables {
  double2* d = nullptr;
  float2* f = nullptr;
};
static std::map<std::pair<int, int>, TwTables> g_tw;
static std::mutex g_tw_mu;

static helm_status twiddles(int N, const double2** d, const float2** f) {
  int dev = 0;
  HELM_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto key = std::make_pair(dev, N);
  auto it = g_tw.find(key);
  if (it == g_tw.end()) {
    std::vector<double2> hd(N / 2);
    std::vector<float2> hf(N / 2);
    for (int t = 0; t < N / 2; ++t) {
      const double ang = -2.0 * M_PI * (double)t / (double)N;
      hd[t] = make_double2(cos(ang), sin(ang));
      hf[t] = make_float2((float)hd[t].x, (float)hd[t].y);
    }
    TwTables T;
    HELM_CK(cudaMalloc(&T.d, sizeof(double2) * N / 2));
    HELM_CK(cudaMalloc(&T.f, sizeof(float2) * N / 2));
    HELM_CK(cudaMemcpy(T.d, hd.data(), sizeof(double2) * N / 2, cudaMemcpyHostToDevice));
    HELM_CK(cudaMemcpy(T.f, hf.data(), sizeof(float2) * N / 2, cudaMemcpyHostToDevice));
    it = g_tw.emplace(key, T).first;
  }
  *d = it->second.d;
  *f = it->second.f;
  return HELM_OK;
}

template <typename R> struct fp64_t { static constexpr bool v = sizeof(R) == 8; };

template <typename R>
static helm_status fourier_op(helm_ctx* ctx, const C<R>* x, C<R>* y, int nrhs, cudaStream_t st) {
  constexpr int TC = FyCols<R>::v;
  for (auto& s : ctx->sys)
    if (!fourier_supported(s.Nx, s.Ny))
      return fail(HELM_ERR_INVALID_ARG, "helm_apply_fourier: grid sides (with the PML) must be powers of two in "
                                        "[16, 1024]; got " + std::to_string(s.Nx) + " x " + std::to_string(s.Ny));
  const bool fp64 = sizeof(R) == 8;
  for (auto& s : ctx->sys) {
    const double2* twd[2];
    const float2* twf[2];
    HELM_TRY(twiddles(s.Nx, &twd[0], &twf[0]));
    HELM_TRY(twiddles(s.Ny, &twd[1], &twf[1]));
    const C<R>* tw_x = fp64 ? (const C<R>*)twd[0] : (const C<R>*)twf[0];
    const C<R>* tw_y = fp64 ? (const C<R>*)twd[1] : (const C<R>*)twf[1];
    const C<R>* pr = fp64 ? (const C<R>*)ctx->prof_d : (const C<R>*)ctx->prof_f;
    const R* k2 = fp64 ? (const R*)(ctx->k2d + s.off) : (const R*)(ctx->k2f + s.off);
    const C<R>* xs = x + s.off * nrhs;
    C<R>* ys = y + s.off * nrhs;
    const size_t smx = sizeof(C<R>) * ((size_t)s.Nx + s.Nx / 2 + s.Nx);
    const size_t smy = sizeof(C<R>) * ((size_t)s.Ny * TC + s.Ny / 2 + s.Ny);
    if (smy > 48 * 1024) HELM_CK(cudaFuncSetAttribute(k_fourier_y<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy));
    const R tpl_x = (R)(2.0 * M_PI / (s.Nx * s.h)), tpl_y = (R)(2.0 * M_PI / (s.Ny * s.h));
    bool wx = false, wy = false;
    if constexpr (!fp64_t<R>::v) {
      wx = fourier_warp_pass(0, s.Nx, xs, ys, k2, pr + s.prof_x, tw_x, s.Nx, s.Ny, nrhs, (int64_t)s.n, tpl_x, st);
    }
    if (!wx)
      launch(k_fourier_x<R>, dim3(s.Ny, nrhs), std::min(FX_THREADS, s.Nx / 2), smx, st, xs, ys, pr + s.prof_x, tw_x,
             s.Nx, log2_exact(s.Nx), s.Ny, (int64_t)s.n, tpl_x);
    if constexpr (!fp64_t<R>::v) {
      wy = fourier_warp_pass(1, s.Ny, xs, ys, k2, pr + s.prof_y, tw_y, s.Nx, s.Ny, nrhs, (int64_t)s.n, tpl_y, st);
    }
    if (!wy)
      launch(k_fourier_y<R>, dim3(s.Nx / TC, nrhs), FY_THREADS, smy, st, xs, ys, k2, pr + s.prof_y, tw_y, s.Nx, s.Ny,
             log2_exact(s.Ny), (int64_t)s.n, tpl_y);
  }
  HELM_CK_LAUNCH();
  return HELM_OK;
}

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_apply_fourier(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs,
                                          void* stream) {
  if (!ctx || !x || !y) return fail(HELM_ERR_INVALID_ARG, "helm_apply_fourier: NULL argument");
  HELM_TRY(check_columns(ctx, nrhs, "helm_apply_fourier"));
  if (x == y) return fail(HELM_ERR_INVALID_ARG, "helm_apply_fourier: x and y must not alias");
  if (((uintptr_t)x | (uintptr_t)y) & 15)
    return fail(HELM_ERR_INVALID_ARG, "helm_apply_fourier: pointers must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == HELM_C64) return fourier_op<float>(ctx, (const float2*)x, (float2*)y, nrhs, st);
  if (dtype == HELM_C128) return fourier_op<double>(ctx, (const double2*)x, (double2*)y, nrhs, st);
  return fail(HELM_ERR_INVALID_ARG, "helm_apply_fourier: unknown dtype");
}
