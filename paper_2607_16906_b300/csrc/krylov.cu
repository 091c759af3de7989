// Flexible GMRES (Alg. 1, eq. 4) with CGS2 orthogonalisation, FP64 Givens least squares and an
// FP64 true-residual / iterative-refinement outer loop (a4-a8).
//
// Vectors are batch vectors (all columns = (system, rhs) pairs back to back).  Per iteration j:
//   z_j = N_theta(v_j)                      (unet.cu; z_j = v_j without a network)
//   w   = A z_j                             (stencil.cu)
//   CGS2: h1 = V_j^H w; w -= V_j h1; h2 = V_j^H w; w -= V_j h2  (k_mdot / k_hreduce / k_maxpy)
//   h_{j+1,j} = ||w||, stored unnormalised as V[j+1] with scale 1/||w|| (deferred normalisation)
//   Givens rotation of the new Hessenberg column, residual estimate |g_{j+1}|  (k_givens, FP64)
// End of cycle: y = R^{-1} g (k_backsolve, FP64), x += beta Z y (k_xupdate, FP64 accumulation).
//
// The inner vectors are complex FP32 (mixed path) or FP64 (plain path); reductions accumulate
// per thread in the vector precision and across threads and blocks in FP64, in a fixed order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "helm_internal.cuh"
#include "unet.cuh"

namespace helm {

constexpr int RED_THREADS = 256;
constexpr int CHECK_EVERY = 8;  // iterations between two host reads of the active-column count

// ------------------------------------------------------------------ reductions

struct ColState {
  int active;   // still iterating in this cycle
  int k;        // iterations done in this cycle
  int status;   // helm_status of the cycle
  int pad;
  double target;  // stop when |g_{j+1}| <= target (relative to beta = 1)
  double est;     // last |g_{j+1}|
  double beta;    // ||r|| of the cycle's starting residual (FP64)
  double hscale;  // largest |h| seen (breakdown reference)
};


template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* __restrict__ out) {
  __shared__ double red[RED_THREADS / 32][NV];
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0;
    for (int q = 0; q < RED_THREADS / 32; ++q) s += red[q][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void chunk_range(int64_t len, int nch, int chunk, int64_t& a, int64_t& b) {
  a = len * chunk / nch;
  b = len * (chunk + 1) / nch;
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_colnorm2(const C<R>* __restrict__ v, const ColDesc* __restrict__ cols,
                                                          int nch, double* __restrict__ partial) {
  int col = blockIdx.y, chunk = blockIdx.x;
  ColDesc cd = cols[col];
  int64_t a, b;
  chunk_range(cd.len, nch, chunk, a, b);
  double s[1] = {0.0};
  for (int64_t p = a + threadIdx.x; p < b; p += RED_THREADS) {
    C<R> x = v[cd.off + p];
    s[0] += (double)x.x * x.x + (double)x.y * x.y;
  }
  block_reduce_store<1>(s, partial + (int64_t)col * nch + chunk);
}

// Multi-dot: partial[(col * ndc + chunk) * ldp + i] = sum over points [chunk P, chunk P + P) of
// conj(V_i) w, i < nv.  The chunk of w sits in shared memory; warp k takes basis vectors
// i = k, k + 8, ...: each lane reads every 32nd point (coalesced 256-byte loads, four in flight),
// then one warp reduction in FP64 per vector and chunk.
constexpr int MD_THREADS = 256;
template <typename R>
__global__ void __launch_bounds__(MD_THREADS) k_mdot(const C<R>* __restrict__ V, int64_t vstride, int nv,
                                                     const C<R>* __restrict__ w, const ColDesc* __restrict__ cols,
                                                     const ColState* __restrict__ st, int P, int ndc,
                                                     double2* __restrict__ partial, int ldp) {
  int col = blockIdx.y, chunk = blockIdx.x;
  if (!st[col].active) return;
  ColDesc cd = cols[col];
  double2* outp = partial + ((int64_t)col * ndc + chunk) * ldp;
  int64_t a = (int64_t)chunk * P;
  if (a >= cd.len) {
    for (int i = threadIdx.x; i < nv; i += MD_THREADS) outp[i] = make_double2(0, 0);
    return;
  }
  const int np = (int)min((int64_t)P, cd.len - a);
  extern __shared__ unsigned char md_smem[];
  C<R>* ws = (C<R>*)md_smem;
  for (int p = threadIdx.x; p < np; p += MD_THREADS) ws[p] = w[cd.off + a + p];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nv; i += MD_THREADS / 32) {
    const C<R>* vi = V + (int64_t)i * vstride + cd.off + a;
    C<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
    int p = lane;
    for (; p + 96 < np; p += 128) {
      C<R> v0 = vi[p], v1 = vi[p + 32], v2 = vi[p + 64], v3 = vi[p + 96];
      s0 = cadd(s0, cdotc(v0, ws[p]));
      s1 = cadd(s1, cdotc(v1, ws[p + 32]));
      s0 = cadd(s0, cdotc(v2, ws[p + 64]));
      s1 = cadd(s1, cdotc(v3, ws[p + 96]));
    }
    for (; p < np; p += 32) s0 = cadd(s0, cdotc(vi[p], ws[p]));
    double dx = (double)s0.x + (double)s1.x, dy = (double)s0.y + (double)s1.y;
    for (int o = 16; o > 0; o >>= 1) {
      dx += __shfl_down_sync(0xffffffffu, dx, o);
      dy += __shfl_down_sync(0xffffffffu, dy, o);
    }
    if (lane == 0) outp[i] = make_double2(dx, dy);
  }
}

// h_i = vscale_i * sum_chunks partial;  hbuf (+)= h;  coef_i = h_i * vscale_i (vector precision).
template <typename R>
__global__ void k_hreduce(const double2* __restrict__ partial, int nch, int ldp, int nv,
                          const double* __restrict__ vscale, int ldv, const ColState* __restrict__ st,
                          double2* __restrict__ hbuf, C<R>* __restrict__ coef, int accumulate) {
  int col = blockIdx.x;
  if (!st[col].active) return;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int c = 0; c < nch; ++c) s = cadd(s, partial[((int64_t)col * nch + c) * ldp + i]);
    double sc = vscale[(int64_t)col * ldv + i];
    s = cscale(s, sc);
    double2* hb = hbuf + (int64_t)col * ldp + i;
    *hb = accumulate ? cadd(*hb, s) : s;
    coef[(int64_t)col * ldp + i] = mk<R>((R)(s.x * sc), (R)(s.y * sc));
  }
}

// w -= sum_i V_i coef_i;  optionally write the result to dst and per-chunk |w|^2 partials.
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy(const C<R>* __restrict__ V, int64_t vstride, int nv,
                                                       C<R>* __restrict__ w, const C<R>* __restrict__ coef, int ldc,
                                                       const ColDesc* __restrict__ cols,
                                                       const ColState* __restrict__ st, int nch, C<R>* __restrict__ dst,
                                                       double* __restrict__ npartial) {
  int col = blockIdx.y, chunk = blockIdx.x;
  if (!st[col].active) return;
  extern __shared__ unsigned char smem_raw[];
  C<R>* cf = (C<R>*)smem_raw;
  for (int i = threadIdx.x; i < nv; i += RED_THREADS) cf[i] = coef[(int64_t)col * ldc + i];
  __syncthreads();
  ColDesc cd = cols[col];
  int64_t a, b;
  chunk_range(cd.len, nch, chunk, a, b);
  double s[1] = {0.0};
  for (int64_t p = a + threadIdx.x; p < b; p += RED_THREADS) {
    int64_t q = cd.off + p;
    // eight independent loads in flight per step, two accumulation chains
    C<R> acc = w[q], acc2 = mk<R>(0, 0);
    int i = 0;
    for (; i + 8 <= nv; i += 8) {
      C<R> v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V[(int64_t)(i + u) * vstride + q];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        acc = csub(acc, cmul(v[u], cf[i + u]));
        acc2 = csub(acc2, cmul(v[u + 1], cf[i + u + 1]));
      }
    }
    for (; i < nv; ++i) acc = csub(acc, cmul(V[(int64_t)i * vstride + q], cf[i]));
    acc = cadd(acc, acc2);
    if (dst) {
      dst[q] = acc;
      s[0] += (double)acc.x * acc.x + (double)acc.y * acc.y;
    } else {
      w[q] = acc;
    }
  }
  if (npartial) block_reduce_store<1>(s, npartial + (int64_t)col * nch + chunk);
}

// ------------------------------------------------------------------ per-column scalar kernels

// Rotate Hessenberg column j (entries 0..j in Rc, subdiagonal hn real >= 0) by the previous
// rotations, form the new one, update g and the column state (estimate, k, status, active).
// colmax2 = max_{i <= j} |Rc[i]|^2 of the unrotated column (computed by the caller, in parallel where
// it can).  The rotations form a chain through the entry carried from row i to row i + 1, which
// stays in a register.
__device__ void givens_update(int j, int m, double2* __restrict__ Rc, double hn, double colmax2,
                              double* __restrict__ csc, double2* __restrict__ snc, double2* __restrict__ gc,
                              ColState& S, double breakdown_eps) {
  double hmax = fmax(fmax(S.hscale, sqrt(colmax2)), hn);
  S.hscale = hmax;
  double2 a = Rc[0];
  for (int i = 0; i < j; ++i) {
    const double2 b = Rc[i + 1];
    const double c = csc[i];
    const double2 s = snc[i];
    Rc[i] = cadd(cscale(a, c), cmul(s, b));
    a = csub(cscale(b, c), cmul(cconj(s), a));
  }
  // new rotation zeroing (Rc[j], hn): c = |a| / t, s = (a / |a|) conj(b) / t, b real here
  double aa = hypot(a.x, a.y);
  double c, t = hypot(aa, hn);
  double2 s;
  if (hn == 0.0) {
    c = 1.0;
    s = make_double2(0, 0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1, 0);
  } else {
    c = aa / t;
    s = cscale(a, hn / (aa * t));  // (a/|a|) * conj(hn) / t with hn real
  }
  csc[j] = c;
  snc[j] = s;
  Rc[j] = cadd(cscale(a, c), cscale(s, hn));
  double2 gj = gc[j];
  gc[j + 1] = cscale(cmul(cconj(s), gj), -1.0);
  gc[j] = cscale(gj, c);
  double est = hypot(gc[j + 1].x, gc[j + 1].y);
  S.est = est;
  S.k = j + 1;
  bool bad = !isfinite(hn) || !isfinite(est) || !isfinite(Rc[j].x) || !isfinite(Rc[j].y);
  double rjj = hypot(Rc[j].x, Rc[j].y);
  if (bad) {
    S.status = HELM_NAN;
    S.active = 0;
    S.k = j;  // drop the poisoned column
  } else if (est <= S.target) {
    S.status = HELM_OK;
    S.active = 0;
  } else if (hn <= breakdown_eps * hmax || rjj <= breakdown_eps * hmax) {
    S.status = HELM_BREAKDOWN;
    S.active = 0;
    if (rjj <= breakdown_eps * hmax) S.k = j;
  } else if (j + 1 >= m) {
    S.status = HELM_NOT_CONVERGED;
    S.active = 0;
  }
}

// One thread per column (CGS2): finish ||w||, rotate the new Hessenberg column, update g.
template <typename R>
__global__ void k_givens(int j, int ncol, int m, const double* __restrict__ npartial, int nch,
                         const double2* __restrict__ hbuf, int ldp, double* __restrict__ vscale,
                         double2* __restrict__ Rm, double* __restrict__ cs, double2* __restrict__ sn,
                         double2* __restrict__ g, ColState* __restrict__ st, int* __restrict__ nactive,
                         double* __restrict__ in_scale, const ColDesc* __restrict__ cols, double breakdown_eps,
                         double* __restrict__ hist0) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  ColState& S = st[col];
  if (!S.active) {
    in_scale[col] = 0.0;
    return;
  }
  double nn = 0;
  for (int c = 0; c < nch; ++c) nn += npartial[(int64_t)col * nch + c];
  double hn = sqrt(nn);
  const double2* h = hbuf + (int64_t)col * ldp;
  double2* Rc = Rm + ((int64_t)col * m + j) * (m + 1);  // column j of R
  double colmax2 = 0.0;
  for (int i = 0; i <= j; ++i) {
    const double2 v = h[i];
    Rc[i] = v;
    colmax2 = fmax(colmax2, v.x * v.x + v.y * v.y);
  }
  givens_update(j, m, Rc, hn, colmax2, cs + (int64_t)col * m, sn + (int64_t)col * m, g + (int64_t)col * (m + 1), S,
                breakdown_eps);
  if (col == 0 && S.k == j + 1) hist0[j] = S.est;  // residual-estimate history of column 0
  double inv = hn > 0 ? 1.0 / hn : 0.0;
  vscale[(int64_t)col * (m + 1) + j + 1] = inv;
  in_scale[col] = S.active ? sqrt((double)cols[col].len) * inv : 0.0;
  if (S.active) atomicAdd(nactive, 1);
}

// ------------------------------------------------------------------ CGS2 with delayed reorthogonalisation
//
// Iteration j holds the basis v_0..v_{nv-1} (final, orthonormal) and the pending vector u_j (one CGS
// pass done, not yet normalised; none at j = 0, where v_0 is final and nv = 1).  z_j = N(u_j) is
// admissible in FGMRES: the flexible relation A Z = V Hbar only needs w_j = A z_j orthogonalised
// against the final basis, and u_j equals v_j up to its reorthogonalisation correction.
//   sweep A (one read of the basis):  a = V^H u_j, b = V^H w, alpha = u_j^H u_j, beta = u_j^H w
//   column j-1 final:  h[:, j-1] += a,  h[j, j-1] = rho = sqrt(alpha - |a|^2);  Givens on column j-1
//   v_j = (u_j - V a) / rho,  d = v_j^H w = (beta - a^H b) / rho,  partial column j = (b, d)
//   sweep B (one read of the basis):  v_j -> slot j,  u_{j+1} = w - V b - v_j d -> slot j+1
// The second Gram-Schmidt pass of every vector is thus the first half of the next sweep A:
// 16 nv + 48 bytes per point and iteration instead of 32 nv + 48.

// conj(v) * u and conj(v) * w accumulated for the two points packed in v, u, w (float4 = 2 complex).
__device__ __forceinline__ void dot2_acc(float* acc, float4 v, float4 u, float4 w) {
  acc[0] += v.x * u.x + v.y * u.y + v.z * u.z + v.w * u.w;
  acc[1] += v.x * u.y - v.y * u.x + v.z * u.w - v.w * u.z;
  acc[2] += v.x * w.x + v.y * w.y + v.z * w.z + v.w * w.w;
  acc[3] += v.x * w.y - v.y * w.x + v.z * w.w - v.w * w.z;
}

// Sweep-A dots of the chunk [base, base + np) for basis vectors (2 warp + 16 k, +1): pu[i] = v_i^H u,
// pw[i] = v_i^H w.  V + i vstride + base is 16-byte aligned for every i.
__device__ __forceinline__ void dsweepA_pairs(const float2* __restrict__ V, int64_t vstride, int nv, int64_t base,
                                              int np, const float4* __restrict__ us4,
                                              const float4* __restrict__ ws4, int warp, int lane,
                                              double2* __restrict__ pu, double2* __restrict__ pw) {
  const int n2 = np >> 1;
  for (int i0 = 2 * warp; i0 < nv; i0 += 2 * (MD_THREADS / 32)) {
    const bool has1 = i0 + 1 < nv;
    const float4* v0 = (const float4*)(V + (int64_t)i0 * vstride + base);
    const float4* v1 = has1 ? (const float4*)(V + (int64_t)(i0 + 1) * vstride + base) : v0;
    float a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0}, b0[4] = {0, 0, 0, 0}, b1[4] = {0, 0, 0, 0};
    int q = lane;
    for (; q + 32 < n2; q += 64) {
      const float4 x0 = __ldcg(v0 + q), x1 = __ldcg(v0 + q + 32);
      const float4 y0 = __ldcg(v1 + q), y1 = __ldcg(v1 + q + 32);
      const float4 u0 = us4[q], u1 = us4[q + 32], w0 = ws4[q], w1 = ws4[q + 32];
      dot2_acc(a0, x0, u0, w0);
      dot2_acc(a1, x1, u1, w1);
      dot2_acc(b0, y0, u0, w0);
      dot2_acc(b1, y1, u1, w1);
    }
    for (; q < n2; q += 32) {
      const float4 x0 = __ldcg(v0 + q), y0 = __ldcg(v1 + q);
      const float4 u0 = us4[q], w0 = ws4[q];
      dot2_acc(a0, x0, u0, w0);
      dot2_acc(b0, y0, u0, w0);
    }
    if ((np & 1) && lane == 0) {  // odd chunk length: the last point alone
      const float2 x = ((const float2*)v0)[np - 1], y = ((const float2*)v1)[np - 1];
      const float2 u = ((const float2*)us4)[np - 1], w = ((const float2*)ws4)[np - 1];
      const float4 xv = make_float4(x.x, x.y, 0.f, 0.f), yv = make_float4(y.x, y.y, 0.f, 0.f);
      const float4 uv = make_float4(u.x, u.y, 0.f, 0.f), wv = make_float4(w.x, w.y, 0.f, 0.f);
      dot2_acc(a0, xv, uv, wv);
      dot2_acc(b0, yv, uv, wv);
    }
    double d[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      d[k] = (double)a0[k] + a1[k];
      d[4 + k] = (double)b0[k] + b1[k];
    }
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 8; ++k) d[k] += __shfl_down_sync(0xffffffffu, d[k], o);
    if (lane == 0) {
      pu[i0] = make_double2(d[0], d[1]);
      pw[i0] = make_double2(d[2], d[3]);
      if (has1) {
        pu[i0 + 1] = make_double2(d[4], d[5]);
        pw[i0 + 1] = make_double2(d[6], d[7]);
      }
    }
  }
}

// partial[((col * ndc + chunk) * 2 + t) * ldq + i]: t = 0 dots with u (i < nv; i = nv: u^H u),
// t = 1 dots with w (i < nv; i = nv: u^H w).  u or w may be null.
template <typename R>
__global__ void __launch_bounds__(MD_THREADS) k_dsweepA(const C<R>* __restrict__ V, int64_t vstride, int nv,
                                                        const C<R>* __restrict__ u, const C<R>* __restrict__ w,
                                                        const ColDesc* __restrict__ cols,
                                                        const ColState* __restrict__ st, int P, int ndc,
                                                        double2* __restrict__ partial, int ldq) {
  int col = blockIdx.y, chunk = blockIdx.x;
  if (!st[col].active) return;
  ColDesc cd = cols[col];
  double2* pu = partial + ((int64_t)(col * ndc + chunk) * 2) * ldq;
  double2* pw = pu + ldq;
  int64_t a = (int64_t)chunk * P;
  if (a >= cd.len) {
    for (int i = threadIdx.x; i <= nv; i += MD_THREADS) {
      pu[i] = make_double2(0, 0);
      pw[i] = make_double2(0, 0);
    }
    return;
  }
  const int np = (int)min((int64_t)P, cd.len - a);
  extern __shared__ __align__(16) unsigned char ds_smem[];
  C<R>* us = (C<R>*)ds_smem;
  C<R>* ws = us + P;
  double uu = 0, uwx = 0, uwy = 0;
  for (int p = threadIdx.x; p < np; p += MD_THREADS) {
    C<R> uv = u ? u[cd.off + a + p] : mk<R>(0, 0);
    C<R> wv = w ? w[cd.off + a + p] : mk<R>(0, 0);
    us[p] = uv;
    ws[p] = wv;
    uu += (double)uv.x * uv.x + (double)uv.y * uv.y;
    C<R> t = cdotc(uv, wv);
    uwx += t.x;
    uwy += t.y;
  }
  double sc[3] = {uu, uwx, uwy};
  __shared__ double red3[3];
  block_reduce_store<3>(sc, red3);  // ends with __syncthreads: the chunk tiles are complete
  if (threadIdx.x == 0) {
    pu[nv] = make_double2(red3[0], 0.0);
    pw[nv] = make_double2(red3[1], red3[2]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (sizeof(R) == 4) {
    // 16-byte loads (two points) when every basis column of this chunk starts 16-byte aligned; each
    // warp takes two basis vectors so that the staged u/w values are read once for both
    if ((vstride & 1) == 0 && ((cd.off + a) & 1) == 0 && ((uintptr_t)V & 15) == 0) {
      dsweepA_pairs(V, vstride, nv, cd.off + a, np, (const float4*)us, (const float4*)ws, warp, lane, pu, pw);
      return;
    }
  }
  for (int i = warp; i < nv; i += MD_THREADS / 32) {
    const C<R>* vi = V + (int64_t)i * vstride + cd.off + a;
    C<R> su = mk<R>(0, 0), sw = mk<R>(0, 0), su2 = mk<R>(0, 0), sw2 = mk<R>(0, 0);
    int p = lane;
    for (; p + 32 < np; p += 64) {
      C<R> v0 = vi[p], v1 = vi[p + 32];
      su = cadd(su, cdotc(v0, us[p]));
      sw = cadd(sw, cdotc(v0, ws[p]));
      su2 = cadd(su2, cdotc(v1, us[p + 32]));
      sw2 = cadd(sw2, cdotc(v1, ws[p + 32]));
    }
    for (; p < np; p += 32) {
      C<R> v0 = vi[p];
      su = cadd(su, cdotc(v0, us[p]));
      sw = cadd(sw, cdotc(v0, ws[p]));
    }
    double d[4] = {(double)su.x + su2.x, (double)su.y + su2.y, (double)sw.x + sw2.x, (double)sw.y + sw2.y};
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 4; ++k) d[k] += __shfl_down_sync(0xffffffffu, d[k], o);
    if (lane == 0) {
      pu[i] = make_double2(d[0], d[1]);
      pw[i] = make_double2(d[2], d[3]);
    }
  }
}

// Sum sweep-A partials over chunks: red[(col * 2 + t) * ldq + i], i <= nv.  Grid
// (ceil(2 (nv + 1) / 32), ncol), DR_WARPS warps per block: lane l of every warp serves value
// 32 blockIdx.x + l (consecutive values: coalesced loads), warp w sums chunks w, w + DR_WARPS, ...
// in four independent partial sums, and warp 0 adds the warps' sums in warp order — a fixed order,
// so the result is deterministic, with ndc / DR_WARPS loads per thread on the critical path.
constexpr int DR_WARPS = 8;
__global__ void __launch_bounds__(DR_WARPS * 32) k_dreduce(const double2* __restrict__ partial, int ndc, int ldq,
                                                           int nv, const ColState* __restrict__ st,
                                                           double2* __restrict__ red) {
  const int col = blockIdx.y;
  if (!st[col].active) return;  // whole block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const bool valid = e < 2 * (nv + 1);
  const int t = e / (nv + 1), i = e % (nv + 1);
  double2 s0 = make_double2(0, 0), s1 = s0, s2 = s0, s3 = s0;
  if (valid) {
    const double2* p = partial + ((int64_t)col * ndc * 2 + t) * ldq + i;
    const int64_t step = (int64_t)2 * ldq;
    int c = warp;
    for (; c + 3 * DR_WARPS < ndc; c += 4 * DR_WARPS) {
      s0 = cadd(s0, p[(c + 0 * DR_WARPS) * step]);
      s1 = cadd(s1, p[(c + 1 * DR_WARPS) * step]);
      s2 = cadd(s2, p[(c + 2 * DR_WARPS) * step]);
      s3 = cadd(s3, p[(c + 3 * DR_WARPS) * step]);
    }
    for (; c < ndc; c += DR_WARPS) s0 = cadd(s0, p[c * step]);
  }
  __shared__ double2 sw[DR_WARPS][32];
  sw[warp][lane] = cadd(cadd(s0, s1), cadd(s2, s3));
  __syncthreads();
  if (warp == 0 && valid) {
    double2 r = sw[0][lane];
#pragma unroll
    for (int w = 1; w < DR_WARPS; ++w) r = cadd(r, sw[w][lane]);
    red[((int64_t)col * 2 + t) * ldq + i] = r;
  }
}

// One block per column: finalise column j-1 (when a pending vector exists), Givens on it, build the
// partial column j and the sweep-B coefficients ca = a, cb = b (vector precision) and
// sc = (1 / rho, d).  The reductions run across the block; the sequential rotation of column j-1
// runs on one thread with the column and the previous rotations staged in shared memory.
constexpr int DC_THREADS = 256;
template <typename R>
__global__ void __launch_bounds__(DC_THREADS) k_dcoef(int j, int nv, int has_u, int has_w, int ncol, int m,
                                                      const double2* __restrict__ red, int ldq,
                                                      double2* __restrict__ Rm, double* __restrict__ cs,
                                                      double2* __restrict__ sn, double2* __restrict__ g,
                                                      ColState* __restrict__ st, C<R>* __restrict__ ca,
                                                      C<R>* __restrict__ cb, double2* __restrict__ sc,
                                                      int* __restrict__ nactive, double breakdown_eps,
                                                      double* __restrict__ hist0) {
  const int col = blockIdx.x;
  ColState& S = st[col];
  if (!S.active) return;
  extern __shared__ unsigned char dc_smem[];
  double2* sR = (double2*)dc_smem;     // column j-1, nv + 1 entries
  double2* sS = sR + (nv + 1);         // previous sines, nv entries
  double* sC = (double*)(sS + nv);     // previous cosines, nv entries
  __shared__ double s_rho, s_inv;
  __shared__ double2 s_d;
  __shared__ int s_active;
  const double2* ra = red + (int64_t)col * 2 * ldq;  // a_i, i < nv; ra[nv] = (u^H u, 0)
  const double2* rb = ra + ldq;                      // b_i, i < nv; rb[nv] = u^H w
  // |a|^2 and a^H b across the block
  double v[3] = {0.0, 0.0, 0.0};
  if (has_u)
    for (int i = threadIdx.x; i < nv; i += DC_THREADS) {
      double2 ai = ra[i], bi = rb[i];
      v[0] += ai.x * ai.x + ai.y * ai.y;
      double2 t = cdotc(ai, bi);
      v[1] += t.x;
      v[2] += t.y;
    }
  __shared__ double red3[3];
  block_reduce_store<3>(v, red3);
  if (has_u) {
    double2* Rc = Rm + ((int64_t)col * m + (j - 1)) * (m + 1);  // column j-1: partial (b, d) so far
    double mx = 0.0;
    for (int i = threadIdx.x; i < nv; i += DC_THREADS) {
      const double2 v = cadd(Rc[i], ra[i]);
      sR[i] = v;
      mx = fmax(mx, v.x * v.x + v.y * v.y);
      if (i < j - 1) {
        sC[i] = cs[(int64_t)col * m + i];
        sS[i] = sn[(int64_t)col * m + i];
      }
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    __shared__ double s_mx[DC_THREADS / 32];
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double colmax2 = 0.0;
      for (int w = 0; w < DC_THREADS / 32; ++w) colmax2 = fmax(colmax2, s_mx[w]);
      double r2 = ra[nv].x - red3[0];
      double rho = r2 > 0 ? sqrt(r2) : 0.0;
      s_rho = rho;
      givens_update(j - 1, m, sR, rho, colmax2, sC, sS, g + (int64_t)col * (m + 1), S, breakdown_eps);
      if (col == 0 && S.k == j) hist0[j - 1] = S.est;  // residual-estimate history of column 0
      cs[(int64_t)col * m + j - 1] = sC[j - 1];
      sn[(int64_t)col * m + j - 1] = sS[j - 1];
      if (S.active && !has_w) {  // finalisation pass at the end of a cycle of m iterations
        S.status = HELM_NOT_CONVERGED;
        S.active = 0;
      }
      s_active = S.active;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += DC_THREADS) Rc[i] = sR[i];
    if (!s_active) return;
  } else if (threadIdx.x == 0) {
    s_rho = 1.0;
  }
  if (!has_w) return;
  if (threadIdx.x == 0) {
    double inv = 1.0;
    double2 d = make_double2(0, 0);
    if (has_u) {
      inv = s_rho > 0 ? 1.0 / s_rho : 0.0;
      double2 t = csub(rb[nv], make_double2(red3[1], red3[2]));  // u^H w - a^H b
      d = cscale(t, inv);
    }
    s_inv = inv;
    s_d = d;
    sc[col * 2] = make_double2(inv, 0.0);
    sc[col * 2 + 1] = d;
    atomicAdd(nactive, 1);
  }
  __syncthreads();
  double2* Rj = Rm + ((int64_t)col * m + j) * (m + 1);  // partial column j
  C<R>* cac = ca + (int64_t)col * ldq;
  C<R>* cbc = cb + (int64_t)col * ldq;
  for (int i = threadIdx.x; i < nv; i += DC_THREADS) {
    double2 ai = ra[i], bi = rb[i];
    Rj[i] = bi;
    cac[i] = mk<R>((R)ai.x, (R)ai.y);
    cbc[i] = mk<R>((R)bi.x, (R)bi.y);
  }
  if (has_u && threadIdx.x == 0) Rj[nv] = s_d;
}

// Sweep B: v_j = (u_j - V a) / rho written over u_j (slot j), u_{j+1} = w - V b - v_j d (slot j+1),
// and per-chunk |u_{j+1}|^2 partials.
// v -= x * c for the two complex values packed in v and x.
__device__ __forceinline__ float4 cmsub2(float4 v, float4 x, float2 c) {
  v.x -= x.x * c.x - x.y * c.y;
  v.y -= x.x * c.y + x.y * c.x;
  v.z -= x.z * c.x - x.w * c.y;
  v.w -= x.z * c.y + x.w * c.x;
  return v;
}

// Sweep-B update over point pairs (16-byte loads) of one column chunk; returns the chunk's ||w'||^2.
// Each thread takes two pairs RED_THREADS apart, so that one coefficient load serves two basis
// loads, and keeps 8 basis loads in flight.  Requires V + cd.off and every basis column 16-byte
// aligned.  An odd last point is taken by thread 0 of the last chunk.
#ifndef DB_NP
#define DB_NP 2  // point pairs per thread in sweep B
#endif
#ifndef DB_VB
#define DB_VB 4  // basis vectors per batch of loads in sweep B
#endif
__device__ __forceinline__ void cmsub2_ab(float4& au, float4& aw, float4 x, float4 ab) {
  au = cmsub2(au, x, make_float2(ab.x, ab.y));
  aw = cmsub2(aw, x, make_float2(ab.z, ab.w));
}

template <int NP, int VB>
__device__ __forceinline__ double dsweepB_pairs(const float2* __restrict__ V, int64_t vstride, int nv,
                                                float2* __restrict__ u, const float2* __restrict__ w,
                                                float2* __restrict__ wout, const float4* sab, float inv, float2 d,
                                                const ColDesc& cd, int nch, int chunk) {
  const int64_t npair = cd.len >> 1, vs4 = vstride >> 1;
  int64_t qa, qb;
  chunk_range(npair, nch, chunk, qa, qb);
  const float4* V4 = (const float4*)(V + cd.off);
  float4* u4 = u ? (float4*)(u + cd.off) : nullptr;
  const float4* w4 = (const float4*)(w + cd.off);
  float4* o4 = (float4*)(wout + cd.off);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  double s = 0.0;
  for (int64_t q0 = qa + threadIdx.x; q0 < qb; q0 += NP * RED_THREADS) {
    int64_t q[NP];
    bool ok[NP];
    float4 au[NP], aw[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int64_t qp = q0 + p * RED_THREADS;
      ok[p] = qp < qb;
      q[p] = ok[p] ? qp : q0;  // idle slots repeat pair q0 and are not stored
      au[p] = u4 ? u4[q[p]] : zero;
      aw[p] = w4[q[p]];
    }
    int i = 0;
    for (; i + VB <= nv; i += VB) {
      float4 x[VB][NP];
#pragma unroll
      for (int k = 0; k < VB; ++k)
#pragma unroll
        for (int p = 0; p < NP; ++p) x[k][p] = __ldcg(V4 + (int64_t)(i + k) * vs4 + q[p]);
#pragma unroll
      for (int k = 0; k < VB; ++k) {
        const float4 ab = sab[i + k];
#pragma unroll
        for (int p = 0; p < NP; ++p) cmsub2_ab(au[p], aw[p], x[k][p], ab);
      }
    }
    for (; i < nv; ++i) {
      const float4 ab = sab[i];
#pragma unroll
      for (int p = 0; p < NP; ++p) cmsub2_ab(au[p], aw[p], __ldcg(V4 + (int64_t)i * vs4 + q[p]), ab);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      if (!ok[p]) continue;
      if (u4) {
        const float4 vj = make_float4(au[p].x * inv, au[p].y * inv, au[p].z * inv, au[p].w * inv);
        u4[q[p]] = vj;
        aw[p] = cmsub2(aw[p], vj, d);
      }
      o4[q[p]] = aw[p];
      s += (double)aw[p].x * aw[p].x + (double)aw[p].y * aw[p].y + (double)aw[p].z * aw[p].z +
           (double)aw[p].w * aw[p].w;
    }
  }
  if ((cd.len & 1) && chunk == nch - 1 && threadIdx.x == 0) {
    const int64_t p = cd.len - 1;
    float2 au1 = u ? u[cd.off + p] : make_float2(0.f, 0.f), aw1 = w[cd.off + p];
    for (int i = 0; i < nv; ++i) {
      const float2 x = V[(int64_t)i * vstride + cd.off + p];
      const float4 ab = sab[i];
      au1 = csub(au1, cmul(x, make_float2(ab.x, ab.y)));
      aw1 = csub(aw1, cmul(x, make_float2(ab.z, ab.w)));
    }
    if (u) {
      const float2 vj = cscale(au1, inv);
      u[cd.off + p] = vj;
      aw1 = csub(aw1, cmul(vj, d));
    }
    wout[cd.off + p] = aw1;
    s += (double)aw1.x * aw1.x + (double)aw1.y * aw1.y;
  }
  return s;
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_dsweepB(const C<R>* __restrict__ V, int64_t vstride, int nv,
                                                         C<R>* __restrict__ u, const C<R>* __restrict__ w,
                                                         C<R>* __restrict__ wout, const C<R>* __restrict__ ca,
                                                         const C<R>* __restrict__ cb, const double2* __restrict__ sc,
                                                         int ldq, const ColDesc* __restrict__ cols,
                                                         const ColState* __restrict__ st, int nch,
                                                         double* __restrict__ npartial) {
  int col = blockIdx.y, chunk = blockIdx.x;
  if (!st[col].active) return;
  extern __shared__ __align__(16) unsigned char db_smem[];
  const R inv = (R)sc[col * 2].x;
  const C<R> d = mk<R>((R)sc[col * 2 + 1].x, (R)sc[col * 2 + 1].y);
  ColDesc cd = cols[col];
  int64_t a, b;
  double s[1] = {0.0};
  if constexpr (sizeof(R) == 4) {
    if ((vstride & 1) == 0 && (cd.off & 1) == 0 && ((uintptr_t)V & 15) == 0) {
      // coefficients interleaved (a_i, b_i): one 16-byte shared load per basis vector
      float4* sab = (float4*)db_smem;
      for (int i = threadIdx.x; i < nv; i += RED_THREADS) {
        const float2 ai = ca[(int64_t)col * ldq + i], bi = cb[(int64_t)col * ldq + i];
        sab[i] = make_float4(ai.x, ai.y, bi.x, bi.y);
      }
      __syncthreads();
      s[0] = dsweepB_pairs<DB_NP, DB_VB>(V, vstride, nv, u, w, wout, sab, inv, d, cd, nch, chunk);
      block_reduce_store<1>(s, npartial + (int64_t)col * nch + chunk);
      return;
    }
  }
  C<R>* sa = (C<R>*)db_smem;
  C<R>* sb = sa + nv;
  for (int i = threadIdx.x; i < nv; i += RED_THREADS) {
    sa[i] = ca[(int64_t)col * ldq + i];
    sb[i] = cb[(int64_t)col * ldq + i];
  }
  __syncthreads();
  chunk_range(cd.len, nch, chunk, a, b);
  // two points per thread per pass: two independent load streams over the basis
  for (int64_t p0 = a + threadIdx.x; p0 < b; p0 += 2 * RED_THREADS) {
    const int64_t p1 = p0 + RED_THREADS;
    const bool two = p1 < b;
    const int64_t q0 = cd.off + p0, q1 = cd.off + (two ? p1 : p0);
    C<R> au0 = u ? u[q0] : mk<R>(0, 0), aw0 = w[q0];
    C<R> au1 = u ? u[q1] : mk<R>(0, 0), aw1 = w[q1];
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      C<R> v0[4], v1[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v0[k] = V[(int64_t)(i + k) * vstride + q0];
        v1[k] = V[(int64_t)(i + k) * vstride + q1];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        au0 = csub(au0, cmul(v0[k], sa[i + k]));
        aw0 = csub(aw0, cmul(v0[k], sb[i + k]));
        au1 = csub(au1, cmul(v1[k], sa[i + k]));
        aw1 = csub(aw1, cmul(v1[k], sb[i + k]));
      }
    }
    for (; i < nv; ++i) {
      C<R> x0 = V[(int64_t)i * vstride + q0], x1 = V[(int64_t)i * vstride + q1];
      au0 = csub(au0, cmul(x0, sa[i]));
      aw0 = csub(aw0, cmul(x0, sb[i]));
      au1 = csub(au1, cmul(x1, sa[i]));
      aw1 = csub(aw1, cmul(x1, sb[i]));
    }
    if (u) {
      C<R> vj0 = cscale(au0, inv);
      u[q0] = vj0;
      aw0 = csub(aw0, cmul(vj0, d));
      if (two) {
        C<R> vj1 = cscale(au1, inv);
        u[q1] = vj1;
        aw1 = csub(aw1, cmul(vj1, d));
      }
    }
    wout[q0] = aw0;
    s[0] += (double)aw0.x * aw0.x + (double)aw0.y * aw0.y;
    if (two) {
      wout[q1] = aw1;
      s[0] += (double)aw1.x * aw1.x + (double)aw1.y * aw1.y;
    }
  }
  block_reduce_store<1>(s, npartial + (int64_t)col * nch + chunk);
}

// Network input scale for the pending vector: in_scale = sqrt(n) / ||u_{j+1}||.  One warp per column
// (blocks of NS_WARPS warps): lane l sums the chunk partials l, l + 32, ..., then a shuffle tree in a
// fixed order.
constexpr int NS_WARPS = 4;
__global__ void __launch_bounds__(NS_WARPS * 32) k_nscale(int ncol, const double* __restrict__ npartial, int nch,
                                                          const ColState* __restrict__ st,
                                                          const ColDesc* __restrict__ cols,
                                                          double* __restrict__ in_scale) {
  const int col = blockIdx.x * NS_WARPS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (col >= ncol) return;  // whole warps; no block-wide barrier follows
  if (!st[col].active) {
    if (lane == 0) in_scale[col] = 0.0;
    return;
  }
  double nn = 0;
  for (int c = lane; c < nch; c += 32) nn += npartial[(int64_t)col * nch + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
  if (lane == 0) in_scale[col] = nn > 0 ? sqrt((double)cols[col].len / nn) : 0.0;
}

// y = R^{-1} g (k x k upper triangular), ycoef_i = beta * y_i.
__global__ void k_backsolve(int ncol, int m, const double2* __restrict__ Rm, const double2* __restrict__ g,
                            const ColState* __restrict__ st, double2* __restrict__ y) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const ColState& S = st[col];
  int k = S.k;
  double2* yc = y + (int64_t)col * m;
  const double2* gc = g + (int64_t)col * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double2 s = gc[i];
    for (int jj = i + 1; jj < k; ++jj) s = csub(s, cmul(Rm[((int64_t)col * m + jj) * (m + 1) + i], yc[jj]));
    double2 d = Rm[((int64_t)col * m + i) * (m + 1) + i];
    double den = d.x * d.x + d.y * d.y;
    yc[i] = den > 0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den) : make_double2(0, 0);
  }
  for (int i = 0; i < k; ++i) yc[i] = cscale(yc[i], S.beta);
}

// x += sum_{i<k} Z_i y_i (FP64 accumulation).  Z_i is v_i scaled by zscale_i when Z aliases V.
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_xupdate(const C<R>* __restrict__ Z, int64_t zstride,
                                                         const double2* __restrict__ y, int m,
                                                         const double* __restrict__ zscale,
                                                         const ColState* __restrict__ st,
                                                         const ColDesc* __restrict__ cols, int nch,
                                                         double2* __restrict__ x) {
  int col = blockIdx.y, chunk = blockIdx.x;
  int k = st[col].k;
  if (k == 0) return;
  constexpr int YC = 1024;  // coefficients staged in shared memory per pass
  __shared__ double2 yc[YC];
  ColDesc cd = cols[col];
  int64_t a, b;
  chunk_range(cd.len, nch, chunk, a, b);
  for (int i0 = 0; i0 < k; i0 += YC) {
    int kk = min(YC, k - i0);
    __syncthreads();
    for (int i = threadIdx.x; i < kk; i += RED_THREADS) {
      double2 yv = y[(int64_t)col * m + i0 + i];
      yc[i] = zscale ? cscale(yv, zscale[(int64_t)col * (m + 1) + i0 + i]) : yv;
    }
    __syncthreads();
    for (int64_t p = a + threadIdx.x; p < b; p += RED_THREADS) {
      int64_t q = cd.off + p;
      if constexpr (sizeof(R) == 4) {
        // mixed path: the correction d = Z y in FP32 (four independent chains), added to x in FP64
        float2 s0 = make_float2(0, 0), s1 = s0, s2 = s0, s3 = s0;
        int i = 0;
        for (; i + 4 <= kk; i += 4) {
          float2 z0 = Z[(int64_t)(i0 + i) * zstride + q], z1 = Z[(int64_t)(i0 + i + 1) * zstride + q];
          float2 z2 = Z[(int64_t)(i0 + i + 2) * zstride + q], z3 = Z[(int64_t)(i0 + i + 3) * zstride + q];
          s0 = cadd(s0, cmul(z0, make_float2((float)yc[i].x, (float)yc[i].y)));
          s1 = cadd(s1, cmul(z1, make_float2((float)yc[i + 1].x, (float)yc[i + 1].y)));
          s2 = cadd(s2, cmul(z2, make_float2((float)yc[i + 2].x, (float)yc[i + 2].y)));
          s3 = cadd(s3, cmul(z3, make_float2((float)yc[i + 3].x, (float)yc[i + 3].y)));
        }
        for (; i < kk; ++i)
          s0 = cadd(s0, cmul(Z[(int64_t)(i0 + i) * zstride + q], make_float2((float)yc[i].x, (float)yc[i].y)));
        double2 acc = x[q];
        acc.x += (double)s0.x + (double)s1.x + (double)s2.x + (double)s3.x;
        acc.y += (double)s0.y + (double)s1.y + (double)s2.y + (double)s3.y;
        x[q] = acc;
      } else {
        double2 acc = x[q];
        for (int i = 0; i < kk; ++i) {
          C<R> z = Z[(int64_t)(i0 + i) * zstride + q];
          acc.x += (double)z.x * yc[i].x - (double)z.y * yc[i].y;
          acc.y += (double)z.x * yc[i].y + (double)z.y * yc[i].x;
        }
        x[q] = acc;
      }
    }
  }
}

// V0 = r / beta in the vector precision for active columns.
template <typename R>
__global__ void k_v0(const double2* __restrict__ r, C<R>* __restrict__ V0, const ColState* __restrict__ st,
                     const ColDesc* __restrict__ cols, int nch) {
  int col = blockIdx.y, chunk = blockIdx.x;
  const ColState& S = st[col];
  ColDesc cd = cols[col];
  int64_t a, b;
  chunk_range(cd.len, nch, chunk, a, b);
  double inv = S.active && S.beta > 0 ? 1.0 / S.beta : 0.0;
  for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) {
    double2 v = r[cd.off + p];
    V0[cd.off + p] = mk<R>((R)(v.x * inv), (R)(v.y * inv));
  }
}

// z = s * v per column (identity preconditioner applied to the deferred-scaled basis vector).
template <typename R>
__global__ void k_scale_copy(const C<R>* __restrict__ v, C<R>* __restrict__ z, const double* __restrict__ s,
                             const ColDesc* __restrict__ cols, int nch, const double* __restrict__ in_scale) {
  int col = blockIdx.y, chunk = blockIdx.x;
  ColDesc cd = cols[col];
  int64_t a, b;
  chunk_range(cd.len, nch, chunk, a, b);
  R sc = (R)(in_scale[col] / sqrt((double)cd.len));
  for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) z[cd.off + p] = cscale(v[cd.off + p], sc);
}

// ------------------------------------------------------------------ host helpers

template <typename R>
helm_status col_norm2(helm_ctx* ctx, const C<R>* v, int nrhs, double* out, cudaStream_t st) {
  HELM_TRY(ensure_cols(ctx, nrhs));
  int ncol = num_cols(ctx, nrhs);
  int nch = std::max(1, std::min(64, (int)(2048 / std::max(1, ncol))));
  HELM_TRY(ctx->ws_red.reserve(sizeof(double) * ncol * nch + sizeof(int) * ncol + 64));
  double* partial = (double*)ctx->ws_red.ptr;
  int* np = (int*)(partial + ncol * nch);
  std::vector<int> nph(ncol, nch);
  HELM_CK(cudaMemcpyAsync(np, nph.data(), sizeof(int) * ncol, cudaMemcpyHostToDevice, st));
  launch(k_colnorm2<R>, dim3(nch, ncol), RED_THREADS, 0, st, v, ctx->cols_dev, nch, partial);
  HELM_CK_LAUNCH();
  launch(k_finalize, ncol, 256, 0, st, partial, np, 1, out);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

template helm_status col_norm2<float>(helm_ctx*, const float2*, int, double*, cudaStream_t);
template helm_status col_norm2<double>(helm_ctx*, const double2*, int, double*, cudaStream_t);

// Solver workspace layout (one allocation, 256-byte aligned pieces).
template <typename R>
struct SolverWs {
  C<R>* V;       // (m+1) vectors
  C<R>* Z;       // m vectors (aliases V without a network)
  C<R>* w;       // 1 vector
  double2* r;    // FP64 residual
  double2* partial;
  double* npartial;
  double2* hbuf;
  C<R>* coef;
  double* vscale;
  double2* Rm;
  double* cs;
  double2* sn;
  double2* g;
  double2* y;
  ColState* st;
  double* sums;
  double* in_scale;
  double* out_scale;
  int* nactive;
  double* hist0;  // Givens estimate of column 0 after each iteration of the cycle (m entries)
  // delayed-reorthogonalisation buffers
  double2* red;  // [ncol][2][ldq]
  C<R>* ca;      // [ncol][ldq]
  C<R>* cb;      // [ncol][ldq]
  double2* sc;   // [ncol][2]
};

template <typename R>
static helm_status solver_ws(helm_ctx* ctx, int m, int ncol, int nch, int ndc, bool separate_z, int64_t nvec,
                             int64_t vst, SolverWs<R>& W) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  size_t vb = sizeof(C<R>) * nvec;
  size_t sb = sizeof(C<R>) * vst;  // basis slot stride
  size_t oV = take(sb * (m + 1));
  size_t oZ = separate_z ? take(sb * m) : oV;
  size_t ow = take(vb);
  size_t orr = take(sizeof(double2) * nvec);
  int ldp = m + 1;
  const int ldq = m + 2;
  size_t op = take(sizeof(double2) * ncol * std::max(nch, ndc) * 2 * ldq);
  size_t ored = take(sizeof(double2) * ncol * 2 * ldq);
  size_t oca = take(sizeof(C<R>) * ncol * ldq);
  size_t ocb = take(sizeof(C<R>) * ncol * ldq);
  size_t osc = take(sizeof(double2) * ncol * 2);
  size_t onp = take(sizeof(double) * ncol * nch);
  size_t oh = take(sizeof(double2) * ncol * ldp);
  size_t oc = take(sizeof(C<R>) * ncol * ldp);
  size_t ovs = take(sizeof(double) * ncol * ldp);
  size_t oR = take(sizeof(double2) * ncol * m * (m + 1));
  size_t ocs = take(sizeof(double) * ncol * m);
  size_t osn = take(sizeof(double2) * ncol * m);
  size_t og = take(sizeof(double2) * ncol * (m + 1));
  size_t oy = take(sizeof(double2) * ncol * m);
  size_t ost = take(sizeof(ColState) * ncol);
  size_t osu = take(sizeof(double) * 2 * ncol);
  size_t ois = take(sizeof(double) * ncol);
  size_t oos = take(sizeof(double) * ncol);
  size_t ona = take(sizeof(int) * 4);
  size_t oh0 = take(sizeof(double) * (m + 1));
  HELM_TRY(ctx->ws_solver.reserve(off));
  char* b = (char*)ctx->ws_solver.ptr;
  W.V = (C<R>*)(b + oV);
  W.Z = (C<R>*)(b + oZ);
  W.w = (C<R>*)(b + ow);
  W.r = (double2*)(b + orr);
  W.partial = (double2*)(b + op);
  W.npartial = (double*)(b + onp);
  W.hbuf = (double2*)(b + oh);
  W.coef = (C<R>*)(b + oc);
  W.vscale = (double*)(b + ovs);
  W.Rm = (double2*)(b + oR);
  W.cs = (double*)(b + ocs);
  W.sn = (double2*)(b + osn);
  W.g = (double2*)(b + og);
  W.y = (double2*)(b + oy);
  W.st = (ColState*)(b + ost);
  W.sums = (double*)(b + osu);
  W.in_scale = (double*)(b + ois);
  W.out_scale = (double*)(b + oos);
  W.nactive = (int*)(b + ona);
  W.hist0 = (double*)(b + oh0);
  W.red = (double2*)(b + ored);
  W.ca = (C<R>*)(b + oca);
  W.cb = (C<R>*)(b + ocb);
  W.sc = (double2*)(b + osc);
  return HELM_OK;
}

// Start of a cycle: g = e1, vscale = 1, network input/output scales for a unit-norm v1
// (alpha = sqrt(n), output h^2 / alpha).
__global__ void k_cycle_setup(int ncol, int m, const ColDesc* __restrict__ cols, double2* __restrict__ g,
                              double* __restrict__ vscale, double* __restrict__ in_scale,
                              double* __restrict__ out_scale) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  for (int i = 0; i <= m; ++i) {
    g[(int64_t)col * (m + 1) + i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
    vscale[(int64_t)col * (m + 1) + i] = 1.0;
  }
  double a = sqrt((double)cols[col].len);
  in_scale[col] = a;
  out_scale[col] = cols[col].h2 / a;
}

template <typename R>
helm_status fgmres_solve(helm_ctx* ctx, const helm_unet* net, const double2* b, double2* x, int nrhs,
                         const helm_solve_opts& o, helm_solve_info* info, cudaStream_t stream) {
  HELM_TRY(ensure_cols(ctx, nrhs));
  const int ncol = num_cols(ctx, nrhs);
  const int m = o.m;
  const int64_t nvec = ctx->npts * nrhs;
  // basis slots are vst elements apart: nvec rounded to 1 KB plus 768 B, so that the same point of
  // successive basis vectors does not fall on addresses a large power of two apart
  const int64_t vst = (nvec + 127) / 128 * 128 + 96;
  int64_t maxlen = 0;
  for (auto& c : ctx->cols_host) maxlen = std::max(maxlen, c.len);
  // point-sweep chunking: about 8 blocks of 256 threads per SM in all, at least 256 points per block
  const int nch = (int)std::max<int64_t>(1, std::min<int64_t>((8 * 148 + ncol - 1) / ncol, (maxlen + 255) / 256));
  SolverWs<R> W;
  // dot-product chunking: P points per block (multiple of 256, 256..2048), about 600 blocks in all
  int P = (int)std::max<int64_t>(256, std::min<int64_t>(2048, (maxlen * ncol / 600) / 256 * 256));
  const int ndc = (int)((maxlen + P - 1) / P);
  const dim3 dgrid(ndc, ncol);
  const size_t md_smem = sizeof(C<R>) * P;
  const bool dcgs2 = o.orth == HELM_ORTH_DCGS2;
  HELM_TRY(solver_ws<R>(ctx, m, ncol, nch, ndc, net != nullptr || dcgs2, nvec, vst, W));
  const int ldq = m + 2;
  const size_t ds_smem = 2 * sizeof(C<R>) * P;
  const size_t db_smem = 2 * sizeof(C<R>) * m;
  auto dc_smem = [](int nv) { return (size_t)(nv + 1) * 16 + (size_t)nv * 24; };
  if (dcgs2) {
    if (dc_smem(m) > 48 * 1024)
      HELM_CK(cudaFuncSetAttribute(k_dcoef<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dc_smem(m)));
    if (ds_smem > 48 * 1024)
      HELM_CK(cudaFuncSetAttribute(k_dsweepA<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ds_smem));
    if (db_smem > 48 * 1024)
      HELM_CK(cudaFuncSetAttribute(k_dsweepB<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)db_smem));
  }
  HELM_TRY(ensure_pinned(ctx, sizeof(double) * (2 * ncol + m) + sizeof(ColState) * ncol + 64 + 64));
  double* h_sums = (double*)ctx->pinned;
  double* h_hist = h_sums + 2 * ncol;                 // column 0's estimates of one cycle
  ColState* h_st = (ColState*)(h_hist + m);
  int* h_nact = (int*)(h_st + ncol);
  ctx->history.clear();
  const bool mixed = sizeof(R) == 4;
  const int max_cycles = mixed ? std::max(1, o.max_outer) : std::max(1, o.max_restarts);
  const double breakdown_eps = mixed ? 1e-6 : 1e-14;
  const int ldp = m + 1;
  const size_t maxpy_smem = sizeof(C<R>) * ldp;
  if (maxpy_smem > 48 * 1024)
    HELM_CK(cudaFuncSetAttribute(k_maxpy<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxpy_smem));
  std::vector<helm_solve_info> inf(ncol);
  for (auto& v : inf) {
    v = helm_solve_info{};
    v.status = HELM_NOT_CONVERGED;
  }
  std::vector<double> bnorm(ncol, 0.0), rel(ncol, 0.0);
  std::vector<int> done(ncol, 0);
  dim3 vgrid(nch, ncol);
  for (int cyc = 0; cyc <= max_cycles; ++cyc) {
    // true residual in FP64 (eq. 10)
    prof_begin(ctx, PH_RESIDUAL, stream);
    HELM_TRY(residual_fp64(ctx, x, b, W.r, nrhs, W.sums, stream));
    HELM_CK(cudaMemcpyAsync(h_sums, W.sums, sizeof(double) * 2 * ncol, cudaMemcpyDeviceToHost, stream));
    HELM_CK(cudaStreamSynchronize(stream));
    int nact = 0;
    for (int c = 0; c < ncol; ++c) {
      double rr = sqrt(h_sums[2 * c]), bb = sqrt(h_sums[2 * c + 1]);
      bnorm[c] = bb;
      rel[c] = bb > 0 ? rr / bb : rr;
      inf[c].relres_true = rel[c];
      if (!std::isfinite(rel[c])) {
        inf[c].status = HELM_NAN;
        done[c] = 1;
      } else if (rel[c] <= o.tol) {
        inf[c].status = HELM_OK;
        done[c] = 1;
      }
      ColState s{};
      s.active = !done[c] && cyc < max_cycles;
      s.beta = rr;
      s.target = mixed ? std::max(o.inner_tol, o.tol * bb / std::max(rr, 1e-300))
                       : o.tol * bb / std::max(rr, 1e-300) * 0.5;
      s.status = HELM_NOT_CONVERGED;
      h_st[c] = s;
      nact += s.active;
    }
    if (nact == 0) {
      prof_end(ctx, PH_RESIDUAL, stream);
      break;
    }
    HELM_CK(cudaMemcpyAsync(W.st, h_st, sizeof(ColState) * ncol, cudaMemcpyHostToDevice, stream));
    // The stopping test stays on the device: every kernel of an iteration skips the columns whose
    // ColState is inactive, and k_givens / k_dcoef count the active ones.  The host reads that count
    // only every `check` iterations, so most iterations are queued without a round trip; a batch whose
    // columns all stopped runs at most check - 1 more iterations of early-exiting launches.
    const int check = std::min(CHECK_EVERY, m);
    bool stop = false;
    auto poll = [&](int j) -> helm_status {
      if ((j + 1) % check != 0 && j + 1 != m) return HELM_OK;
      HELM_CK(cudaMemcpyAsync(h_nact, W.nactive, sizeof(int), cudaMemcpyDeviceToHost, stream));
      HELM_CK(cudaStreamSynchronize(stream));
      prof_collect(ctx);
      nact = *h_nact;
      stop = nact == 0;
      return HELM_OK;
    };
    // g = e1 (the cycle runs on r / ||r||), vscale = 1, network scales for a unit-norm v1
    launch(k_cycle_setup, cdiv(ncol, 64), 64, 0, stream, ncol, m, ctx->cols_dev, W.g, W.vscale, W.in_scale,
           W.out_scale);
    launch(k_v0<R>, vgrid, RED_THREADS, 0, stream, W.r, W.V, W.st, ctx->cols_dev, nch);
    HELM_CK_LAUNCH();
    prof_end(ctx, PH_RESIDUAL, stream);
    if (!dcgs2) {
      for (int j = 0; j < m; ++j) {
        C<R>* Vj = W.V + (int64_t)j * vst;
        C<R>* Zj = net ? W.Z + (int64_t)j * vst : Vj;
        // z_j = N_theta(v_j)
        prof_begin(ctx, PH_PRECOND, stream);
        if (ctx->prof_on) {
          ctx->prof_work[PH_PRECOND] += net ? unet_flop_per_point(net->kind) * ctx->npts * nrhs : 0.0;
          ctx->prof_work[PH_STENCIL] += 16.0 * ctx->npts * nrhs + 4.0 * ctx->npts;
          ctx->prof_work[PH_ORTH] += (32.0 * (j + 1) + 48.0) * ctx->npts * nrhs * (double)nact / ncol;
        }
        if (net) {
          for (int s = 0; s < ctx->nsys; ++s) {
            int64_t off = ctx->sys[s].off * nrhs;
            HELM_TRY(unet_precondition<R>(ctx, net, s, Vj + off, Zj + off, nrhs, W.in_scale + s * nrhs,
                                          W.out_scale + s * nrhs, stream, 0));
          }
        } else {
          // z_j = v_j = vscale_j Vraw_j into the FP64 residual buffer, free after k_v0
          launch(k_scale_copy<R>, vgrid, RED_THREADS, 0, stream, Vj, (C<R>*)W.r, nullptr, ctx->cols_dev, nch,
                 W.in_scale);
          HELM_CK_LAUNCH();
        }
        prof_end(ctx, PH_PRECOND, stream);
        // w = A z_j
        prof_begin(ctx, PH_STENCIL, stream);
        HELM_TRY(apply_op<R>(ctx, net ? Zj : (C<R>*)W.r, W.w, nrhs, false, stream));
        prof_end(ctx, PH_STENCIL, stream);
        const int nv = j + 1;
        // CGS2, two passes; the second writes the unnormalised v_{j+1} and its norm partials
        prof_begin(ctx, PH_ORTH, stream);
        for (int pass = 0; pass < 2; ++pass) {
          launch(k_mdot<R>, dgrid, MD_THREADS, md_smem, stream, W.V, vst, nv, W.w, ctx->cols_dev, W.st, P, ndc,
                 W.partial, ldp);
          launch(k_hreduce<R>, ncol, 256, 0, stream, W.partial, ndc, ldp, nv, W.vscale, ldp, W.st, W.hbuf, W.coef,
                 pass);
          C<R>* dst = pass == 1 ? W.V + (int64_t)(j + 1) * vst : nullptr;
          launch(k_maxpy<R>, vgrid, RED_THREADS, maxpy_smem, stream, W.V, vst, nv, W.w, W.coef, ldp, ctx->cols_dev,
                 W.st, nch, dst, pass == 1 ? W.npartial : nullptr);
          HELM_CK_LAUNCH();
        }
        prof_end(ctx, PH_ORTH, stream);
        prof_begin(ctx, PH_LSQ, stream);
        HELM_CK(cudaMemsetAsync(W.nactive, 0, sizeof(int), stream));
        launch(k_givens<R>, cdiv(ncol, 64), 64, 0, stream, j, ncol, m, W.npartial, nch, W.hbuf, ldp, W.vscale, W.Rm,
               W.cs, W.sn, W.g, W.st, W.nactive, W.in_scale, ctx->cols_dev, breakdown_eps, W.hist0);
        HELM_CK_LAUNCH();
        prof_end(ctx, PH_LSQ, stream);
        HELM_TRY(poll(j));
        if (stop) break;
      }
    } else {
      // CGS2 with delayed reorthogonalisation (kernels k_dsweepA / k_dcoef / k_dsweepB above)
      for (int j = 0; j < m; ++j) {
        C<R>* Uj = W.V + (int64_t)j * vst;  // v_0 at j = 0, else the pending u_j
        C<R>* Zj = W.Z + (int64_t)j * vst;
        prof_begin(ctx, PH_PRECOND, stream);
        if (ctx->prof_on) {
          ctx->prof_work[PH_PRECOND] += net ? unet_flop_per_point(net->kind) * ctx->npts * nrhs : 0.0;
          ctx->prof_work[PH_STENCIL] += 16.0 * ctx->npts * nrhs + 4.0 * ctx->npts;
          ctx->prof_work[PH_ORTH] += (16.0 * (j > 0 ? j : 1) + 48.0) * ctx->npts * nrhs * (double)nact / ncol;
        }
        if (net) {
          for (int s = 0; s < ctx->nsys; ++s) {
            int64_t off = ctx->sys[s].off * nrhs;
            HELM_TRY(unet_precondition<R>(ctx, net, s, Uj + off, Zj + off, nrhs, W.in_scale + s * nrhs,
                                          W.out_scale + s * nrhs, stream, 0));
          }
        } else {
          launch(k_scale_copy<R>, vgrid, RED_THREADS, 0, stream, (const C<R>*)Uj, Zj, nullptr, ctx->cols_dev, nch,
                 W.in_scale);
        }
        HELM_CK_LAUNCH();
        prof_end(ctx, PH_PRECOND, stream);
        prof_begin(ctx, PH_STENCIL, stream);
        HELM_TRY(apply_op<R>(ctx, Zj, W.w, nrhs, false, stream));
        prof_end(ctx, PH_STENCIL, stream);
        const int has_u = j > 0;
        const int nv = j > 0 ? j : 1;
        prof_begin(ctx, PH_ORTH, stream);
        HELM_CK(cudaMemsetAsync(W.nactive, 0, sizeof(int), stream));
        launch(k_dsweepA<R>, dgrid, MD_THREADS, ds_smem, stream, (const C<R>*)W.V, vst, nv,
               (const C<R>*)(has_u ? Uj : nullptr), (const C<R>*)W.w, ctx->cols_dev, W.st, P, ndc, W.partial, ldq);
        launch(k_dreduce, dim3(cdiv(2 * (nv + 1), 32), ncol), DR_WARPS * 32, 0, stream, (const double2*)W.partial,
               ndc, ldq, nv, W.st, W.red);
        launch(k_dcoef<R>, ncol, DC_THREADS, dc_smem(nv), stream, j, nv, has_u, 1, ncol, m, (const double2*)W.red, ldq,
               W.Rm, W.cs, W.sn, W.g, W.st, W.ca, W.cb, W.sc, W.nactive, breakdown_eps, W.hist0);
        launch(k_dsweepB<R>, vgrid, RED_THREADS, 2 * sizeof(C<R>) * nv, stream, (const C<R>*)W.V, vst, nv,
               has_u ? Uj : nullptr, (const C<R>*)W.w, W.V + (int64_t)(j + 1) * vst, (const C<R>*)W.ca,
               (const C<R>*)W.cb, (const double2*)W.sc, ldq, ctx->cols_dev, W.st, nch, W.npartial);
        launch(k_nscale, cdiv(ncol, NS_WARPS), NS_WARPS * 32, 0, stream, ncol, (const double*)W.npartial, nch, W.st,
               ctx->cols_dev, W.in_scale);
        HELM_CK_LAUNCH();
        prof_end(ctx, PH_ORTH, stream);
        HELM_TRY(poll(j));
        if (stop) break;
      }
      // columns that ran all m iterations: finalise column m-1 (reorthogonalise the pending u_m)
      prof_begin(ctx, PH_ORTH, stream);
      launch(k_dsweepA<R>, dgrid, MD_THREADS, ds_smem, stream, (const C<R>*)W.V, vst, m,
             (const C<R>*)(W.V + (int64_t)m * vst), (const C<R>*)nullptr, ctx->cols_dev, W.st, P, ndc, W.partial,
             ldq);
      launch(k_dreduce, dim3(cdiv(2 * (m + 1), 32), ncol), DR_WARPS * 32, 0, stream, (const double2*)W.partial, ndc,
             ldq, m, W.st, W.red);
      launch(k_dcoef<R>, ncol, DC_THREADS, dc_smem(m), stream, m, m, 1, 0, ncol, m, (const double2*)W.red, ldq, W.Rm,
             W.cs, W.sn, W.g, W.st, W.ca, W.cb, W.sc, W.nactive, breakdown_eps, W.hist0);
      HELM_CK_LAUNCH();
      prof_end(ctx, PH_ORTH, stream);
    }
    // a pipeline wait that ran out left some z_j or w incomplete: keep x at the last completed
    // cycle's iterate (its true residual is the one reported) and return HELM_TIMEOUT
    {
      helm_status chk = net ? conv_tc_check(net, stream) : HELM_OK;
      if (chk == HELM_OK) chk = stencil_check(ctx, stream);
      if (chk != HELM_OK) {
        const std::string msg = helm_last_error();
        for (int c = 0; c < ncol; ++c) {
          if (!done[c]) inf[c].status = chk;
          if (info) info[c] = inf[c];
        }
        return fail(chk, msg);
      }
    }
    prof_begin(ctx, PH_UPDATE, stream);
    launch(k_backsolve, cdiv(ncol, 64), 64, 0, stream, ncol, m, W.Rm, W.g, W.st, W.y);
    launch(k_xupdate<R>, vgrid, RED_THREADS, 0, stream, W.Z, vst, W.y, m, (net || dcgs2) ? nullptr : W.vscale,
           W.st, ctx->cols_dev, nch, x);
    HELM_CK_LAUNCH();
    HELM_CK(cudaMemcpyAsync(h_st, W.st, sizeof(ColState) * ncol, cudaMemcpyDeviceToHost, stream));
    HELM_CK(cudaMemcpyAsync(h_hist, W.hist0, sizeof(double) * m, cudaMemcpyDeviceToHost, stream));
    prof_end(ctx, PH_UPDATE, stream);
    HELM_CK(cudaStreamSynchronize(stream));
    prof_collect(ctx);
    if (!done[0])  // column 0's estimate after each of its iterations in this cycle
      for (int i = 0; i < h_st[0].k; ++i) ctx->history.push_back(h_hist[i] * rel[0]);
    for (int c = 0; c < ncol; ++c) {
      if (done[c]) continue;
      inf[c].iters += h_st[c].k;
      inf[c].restarts += 1;
      inf[c].outer += mixed ? 1 : 0;
      inf[c].relres_est = h_st[c].est * rel[c];
      if (h_st[c].status == HELM_NAN) {
        inf[c].status = HELM_NAN;
        done[c] = 1;
      } else if (h_st[c].status == HELM_BREAKDOWN && h_st[c].k == 0) {
        inf[c].status = HELM_BREAKDOWN;
        done[c] = 1;
      }
    }
  }
  helm_status worst = HELM_OK;
  for (int c = 0; c < ncol; ++c) {
    if (inf[c].status == HELM_OK && !(inf[c].relres_true <= o.tol)) inf[c].status = HELM_NOT_CONVERGED;
    if (inf[c].status != HELM_OK && worst == HELM_OK) worst = (helm_status)inf[c].status;
    if (info) info[c] = inf[c];
  }
  if (worst != HELM_OK) set_error("helm_fgmres_solve: at least one column did not reach the tolerance");
  return worst;
}

}  // namespace helm

using namespace helm;

extern "C" int helm_solve_history(const helm_ctx* ctx, double* est_host, int max_entries) {
  if (!ctx) return 0;
  int n = (int)ctx->history.size();
  if (est_host)
    for (int i = 0; i < n && i < max_entries; ++i) est_host[i] = ctx->history[i];
  return n;
}

extern "C" helm_status helm_fgmres_solve(helm_ctx* ctx, const helm_unet* net, const void* b, void* x, int nrhs,
                                         const helm_solve_opts* opts, helm_solve_info* info, void* stream) {
  if (!ctx || !b || !x || !opts) return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: NULL argument");
  HELM_TRY(check_columns(ctx, nrhs, "helm_fgmres_solve"));
  if (b == x) return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: b and x must not alias");
  if (((uintptr_t)b | (uintptr_t)x) & 15) return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: pointers must be 16-byte aligned");
  helm_solve_opts o = *opts;
  if (o.m < 1 || o.m > HELM_MAX_M) return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: m out of range");
  if (!(o.tol > 0) || o.max_restarts < 1 || (o.mixed && o.max_outer < 1))
    return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: tol must be > 0 and iteration budgets >= 1");
  if (o.mixed && !(o.inner_tol > 0 && o.inner_tol < 1))
    return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: inner_tol must be in (0, 1)");
  if (o.orth != HELM_ORTH_CGS2 && o.orth != HELM_ORTH_DCGS2)
    return fail(HELM_ERR_INVALID_ARG, "helm_fgmres_solve: unknown orthogonalisation");
  cudaStream_t st = (cudaStream_t)stream;
  if (o.mixed) return fgmres_solve<float>(ctx, net, (const double2*)b, (double2*)x, nrhs, o, info, st);
  return fgmres_solve<double>(ctx, net, (const double2*)b, (double2*)x, nrhs, o, info, st);
}
