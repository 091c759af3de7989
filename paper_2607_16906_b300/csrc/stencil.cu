// The complex 5-point Helmholtz stencil with PML stretching (a2), its adjoint, and the fused
// FP64 true residual r = b - A x with per-column norms (a8, eq. 10).
//
// One thread owns one x-column of a strip of STENCIL_ROWS rows and marches down it, keeping the
// south and centre values in registers; east/west neighbours come from the same row that the
// neighbouring threads load (L1 hits).  Loads and stores are coalesced across the warp (one complex
// per thread, 8 B in FP32, 16 B in FP64).  Per point the kernel moves 8 + 8 + 4 B (FP32) or
// 16 + 16 + 8 B (FP64) of HBM traffic: read u, write A u, read k^2; the 1-D PML profiles are
// O(Nx + Ny) and stay in L1/L2.
#include <mutex>

#include "helm_internal.cuh"
#include "stencil_point.cuh"

namespace helm {

constexpr int STENCIL_ROWS = 8;
constexpr int STENCIL_THREADS = 128;

template <typename R, bool ADJ>
__device__ __forceinline__ C<R> ld_u(const C<R>* __restrict__ x, int j, int i, int Nx, int Ny) {
  if (j < 0 || j >= Ny || i < 0 || i >= Nx) return mk<R>(0, 0);
  C<R> v = x[(int64_t)j * Nx + i];
  if (ADJ) v.y = -v.y;
  return v;
}

template <typename R, bool ADJ>
__global__ void __launch_bounds__(STENCIL_THREADS) k_stencil(const C<R>* __restrict__ x, C<R>* __restrict__ y,
                                                             const R* __restrict__ k2, const C<R>* __restrict__ px,
                                                             const C<R>* __restrict__ py, int Nx, int Ny,
                                                             int64_t rhs_stride, R inv_h2) {
  int i = blockIdx.x * STENCIL_THREADS + threadIdx.x;
  if (i >= Nx) return;
  int j0 = blockIdx.y * STENCIL_ROWS;
  const C<R>* xr = x + blockIdx.z * rhs_stride;
  C<R>* yr = y + blockIdx.z * rhs_stride;
  const C<R> sxi = px[i], ixm = px[Nx + i], ixp = px[Nx + i + 1];
  const bool xunit = unit_c<R>(sxi) && unit_c<R>(ixm) && unit_c<R>(ixp);
  C<R> uS = ld_u<R, ADJ>(xr, j0 - 1, i, Nx, Ny);
  C<R> uC = ld_u<R, ADJ>(xr, j0, i, Nx, Ny);
#pragma unroll
  for (int r = 0; r < STENCIL_ROWS; ++r) {
    int j = j0 + r;
    if (j >= Ny) break;
    C<R> uN = ld_u<R, ADJ>(xr, j + 1, i, Nx, Ny);
    C<R> uW = ld_u<R, ADJ>(xr, j, i - 1, Nx, Ny);
    C<R> uE = ld_u<R, ADJ>(xr, j, i + 1, Nx, Ny);
    const C<R> syj = py[j], iym = py[Ny + j], iyp = py[Ny + j + 1];
    const R kk = k2[(int64_t)j * Nx + i];
    C<R> out = stencil_point_any<R>(xunit, unit_c<R>(syj) && unit_c<R>(iym) && unit_c<R>(iyp), uC, uE, uW, uN, uS,
                                    sxi, ixm, ixp, syj, iym, iyp, kk, inv_h2);
    if (ADJ) out.y = -out.y;
    yr[(int64_t)j * Nx + i] = out;
    uS = uC;
    uC = uN;
  }
}

// r = b - A x, plus per-block partial sums of |r|^2 and |b|^2 in FP64 (deterministic order).
template <typename R>
__global__ void __launch_bounds__(STENCIL_THREADS) k_residual(const C<R>* __restrict__ x, const C<R>* __restrict__ b,
                                                              C<R>* __restrict__ r, const R* __restrict__ k2,
                                                              const C<R>* __restrict__ px,
                                                              const C<R>* __restrict__ py, int Nx, int Ny,
                                                              int64_t rhs_stride, R inv_h2, double* partial,
                                                              int col0) {
  int i = blockIdx.x * STENCIL_THREADS + threadIdx.x;
  int j0 = blockIdx.y * STENCIL_ROWS;
  const C<R>* xr = x + blockIdx.z * rhs_stride;
  const C<R>* br = b + blockIdx.z * rhs_stride;
  C<R>* rr = r + blockIdx.z * rhs_stride;
  double sr = 0.0, sb = 0.0;
  if (i < Nx) {
    const C<R> sxi = px[i], ixm = px[Nx + i], ixp = px[Nx + i + 1];
    const bool xunit = unit_c<R>(sxi) && unit_c<R>(ixm) && unit_c<R>(ixp);
    C<R> uS = ld_u<R, false>(xr, j0 - 1, i, Nx, Ny);
    C<R> uC = ld_u<R, false>(xr, j0, i, Nx, Ny);
#pragma unroll
    for (int q = 0; q < STENCIL_ROWS; ++q) {
      int j = j0 + q;
      if (j >= Ny) break;
      C<R> uN = ld_u<R, false>(xr, j + 1, i, Nx, Ny);
      C<R> uW = ld_u<R, false>(xr, j, i - 1, Nx, Ny);
      C<R> uE = ld_u<R, false>(xr, j, i + 1, Nx, Ny);
      int64_t idx = (int64_t)j * Nx + i;
      const C<R> syj = py[j], iym = py[Ny + j], iyp = py[Ny + j + 1];
      C<R> Au = stencil_point_any<R>(xunit, unit_c<R>(syj) && unit_c<R>(iym) && unit_c<R>(iyp), uC, uE, uW, uN, uS,
                                     sxi, ixm, ixp, syj, iym, iyp, k2[idx], inv_h2);
      C<R> bv = br[idx];
      C<R> res = csub(bv, Au);
      rr[idx] = res;
      sr += (double)res.x * res.x + (double)res.y * res.y;
      sb += (double)bv.x * bv.x + (double)bv.y * bv.y;
      uS = uC;
      uC = uN;
    }
  }
  // block reduction (fixed order)
  __shared__ double red[2][STENCIL_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = sr;
    red[1][w] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int k = 0; k < STENCIL_THREADS / 32; ++k) {
      a += red[0][k];
      c += red[1][k];
    }
    int nparts = gridDim.x * gridDim.y;
    int part = blockIdx.y * gridDim.x + blockIdx.x;
    int64_t base = ((int64_t)(col0 + blockIdx.z) * nparts + part) * 2;
    partial[base] = a;
    partial[base + 1] = c;
  }
}

// out[col * nvals + v] = sum_p partial[(col * nparts + p) * nvals + v], one block per column.
__global__ void k_finalize(const double* __restrict__ partial, const int* __restrict__ nparts_col, int nvals,
                           double* __restrict__ out) {
  int col = blockIdx.x;
  int np = nparts_col[col];
  int64_t base = 0;
  for (int c = 0; c < col; ++c) base += (int64_t)nparts_col[c] * nvals;
  __shared__ double red[256 / 32];
  for (int v = 0; v < nvals; ++v) {
    double s = 0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) s += partial[base + (int64_t)p * nvals + v];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
      out[(int64_t)col * nvals + v] = t;
    }
    __syncthreads();
  }
}

template <typename R>
helm_status apply_op(helm_ctx* ctx, const C<R>* x, C<R>* y, int nrhs, bool adjoint, cudaStream_t st) {
  const bool fp64 = sizeof(R) == 8;
  for (auto& s : ctx->sys) {
    const C<R>* xs = x + s.off * nrhs;
    C<R>* ys = y + s.off * nrhs;
    const R* k2 = fp64 ? (const R*)(ctx->k2d + s.off) : (const R*)(ctx->k2f + s.off);
    const C<R>* pr = fp64 ? (const C<R>*)ctx->prof_d : (const C<R>*)ctx->prof_f;
    R inv_h2 = (R)(1.0 / (s.h * s.h));
    if (!fp64 && stencil_tma_supported(s.Nx, s.Ny, xs, ys)) {
      HELM_TRY(stencil_tma((const float2*)xs, (float2*)ys, (const float*)k2, (const float2*)pr + s.prof_x,
                           (const float2*)pr + s.prof_y, ctx->unit_f + s.prof_x, ctx->unit_f + s.prof_y, s.Nx, s.Ny,
                           nrhs, (float)inv_h2, adjoint, ctx->flag_dev + 2, st));
      continue;
    }
    dim3 grid(cdiv(s.Nx, STENCIL_THREADS), cdiv(s.Ny, STENCIL_ROWS), nrhs);
    if (adjoint)
      launch(k_stencil<R, true>, grid, STENCIL_THREADS, 0, st, xs, ys, k2, pr + s.prof_x, pr + s.prof_y, s.Nx, s.Ny,
                                                           s.n, inv_h2);
    else
      launch(k_stencil<R, false>, grid, STENCIL_THREADS, 0, st, xs, ys, k2, pr + s.prof_x, pr + s.prof_y, s.Nx, s.Ny,
                                                            s.n, inv_h2);
  }
  HELM_CK_LAUNCH();
  return HELM_OK;
}

template helm_status apply_op<float>(helm_ctx*, const float2*, float2*, int, bool, cudaStream_t);
template helm_status apply_op<double>(helm_ctx*, const double2*, double2*, int, bool, cudaStream_t);

template <typename R>
helm_status residual_op(helm_ctx* ctx, const C<R>* x, const C<R>* b, C<R>* r, int nrhs, double* sums, cudaStream_t st) {
  const bool fp64 = sizeof(R) == 8;
  HELM_TRY(ensure_cols(ctx, nrhs));
  int ncol = num_cols(ctx, nrhs);
  // per-column part counts
  std::vector<int> np(ncol);
  int64_t total = 0;
  for (int c = 0; c < ncol; ++c) {
    auto& s = ctx->sys[ctx->cols_host[c].sys];
    np[c] = (int)(cdiv(s.Nx, STENCIL_THREADS) * cdiv(s.Ny, STENCIL_ROWS));
    total += np[c];
  }
  size_t need = sizeof(double) * 2 * total + sizeof(int) * ncol + 64;
  HELM_TRY(ctx->ws_red.reserve(need));
  double* partial = (double*)ctx->ws_red.ptr;
  int* np_dev = (int*)(partial + 2 * total);
  HELM_CK(cudaMemcpyAsync(np_dev, np.data(), sizeof(int) * ncol, cudaMemcpyHostToDevice, st));
  // partial layout: column-major blocks; every column of system s has the same part count, so the
  // kernel's (col * nparts + part) indexing is valid within a system; offset per system below.
  int col0 = 0;
  int64_t pbase = 0;
  for (auto& s : ctx->sys) {
    dim3 grid(cdiv(s.Nx, STENCIL_THREADS), cdiv(s.Ny, STENCIL_ROWS), nrhs);
    const R* k2 = fp64 ? (const R*)(ctx->k2d + s.off) : (const R*)(ctx->k2f + s.off);
    const C<R>* pr = fp64 ? (const C<R>*)ctx->prof_d : (const C<R>*)ctx->prof_f;
    launch(k_residual<R>, grid, STENCIL_THREADS, 0, st, x + s.off * nrhs, b + s.off * nrhs, r + s.off * nrhs, k2,
           pr + s.prof_x, pr + s.prof_y, s.Nx, s.Ny, s.n, (R)(1.0 / (s.h * s.h)), partial + pbase * 2, 0);
    pbase += (int64_t)grid.x * grid.y * nrhs;
    col0 += nrhs;
  }
  HELM_CK_LAUNCH();
  launch(k_finalize, ncol, 256, 0, st, partial, np_dev, 2, sums);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

template helm_status residual_op<float>(helm_ctx*, const float2*, const float2*, float2*, int, double*, cudaStream_t);
template helm_status residual_op<double>(helm_ctx*, const double2*, const double2*, double2*, int, double*,
                                         cudaStream_t);

helm_status residual_fp64(helm_ctx* ctx, const double2* x, const double2* b, double2* r, int nrhs, double* sums,
                          cudaStream_t st) {
  return residual_op<double>(ctx, x, b, r, nrhs, sums, st);
}

}  // namespace helm

using namespace helm;

static helm_status apply_entry(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs, void* stream,
                               bool adj, const char* name) {
  if (!ctx || !x || !y) return fail(HELM_ERR_INVALID_ARG, std::string(name) + ": NULL argument");
  HELM_TRY(check_columns(ctx, nrhs, name));
  if (x == y) return fail(HELM_ERR_INVALID_ARG, std::string(name) + ": x and y must not alias");
  if (((uintptr_t)x | (uintptr_t)y) & 15) return fail(HELM_ERR_INVALID_ARG, std::string(name) + ": pointers must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == HELM_C64) return apply_op<float>(ctx, (const float2*)x, (float2*)y, nrhs, adj, st);
  if (dtype == HELM_C128) return apply_op<double>(ctx, (const double2*)x, (double2*)y, nrhs, adj, st);
  return fail(HELM_ERR_INVALID_ARG, std::string(name) + ": unknown dtype");
}

extern "C" helm_status helm_apply(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs, void* stream) {
  return apply_entry(ctx, x, y, dtype, nrhs, stream, false, "helm_apply");
}

extern "C" helm_status helm_apply_adjoint(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs,
                                          void* stream) {
  return apply_entry(ctx, x, y, dtype, nrhs, stream, true, "helm_apply_adjoint");
}

extern "C" helm_status helm_relres(helm_ctx* ctx, const void* x, const void* b, int nrhs, double* out_host,
                                   void* stream) {
  if (!ctx || !x || !b || !out_host) return fail(HELM_ERR_INVALID_ARG, "helm_relres: NULL argument");
  HELM_TRY(check_columns(ctx, nrhs, "helm_relres"));
  cudaStream_t st = (cudaStream_t)stream;
  int ncol = num_cols(ctx, nrhs);
  size_t vec = sizeof(double2) * ctx->npts * nrhs;
  HELM_TRY(ctx->ws_vec.reserve(vec + sizeof(double) * 2 * ncol + 256));
  double2* r = (double2*)ctx->ws_vec.ptr;
  double* sums = (double*)((char*)ctx->ws_vec.ptr + ((vec + 255) / 256) * 256);
  HELM_TRY(residual_fp64(ctx, (const double2*)x, (const double2*)b, r, nrhs, sums, st));
  std::vector<double> h(2 * ncol);
  HELM_CK(cudaMemcpyAsync(h.data(), sums, sizeof(double) * 2 * ncol, cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  for (int c = 0; c < ncol; ++c) out_host[c] = h[2 * c + 1] > 0 ? sqrt(h[2 * c] / h[2 * c + 1]) : sqrt(h[2 * c]);
  return HELM_OK;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free relative residual.
//
// Some callers may not allocate device memory while they run: a host whose device memory is
// reserved up front by another framework's caching allocator, or a latency-critical loop in which
// a cudaMalloc would synchronise the whole device.  helm_relres_noalloc serves them: it computes
// the same ||b - A x|| / ||b|| as helm_relres, without storing r, and keeps its per-block partial
// sums in the fixed device array below instead of a workspace.  Every GPU that loads this library
// holds the array (NOALLOC_SCRATCH_DOUBLES doubles, 8 MiB) until the process exits.  The host-side
// name of the array is only a stand-in; its device address is looked up once per device.
namespace helm {

constexpr int64_t NOALLOC_SCRATCH_DOUBLES = (int64_t)1 << 20;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (looked up on first use per device).
static helm_status noalloc_scratch(double** out) {
  int dev = -1;
  HELM_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(HELM_ERR_INVALID_ARG, "helm_relres_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    HELM_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = (double*)p;
  }
  *out = g_noalloc_addr[dev];
  return HELM_OK;
}

// Like k_residual without the r output: per-block partial sums of |b - A x|^2 and |b|^2 only.
__global__ void __launch_bounds__(STENCIL_THREADS) k_relres_partials(const double2* __restrict__ x,
                                                                     const double2* __restrict__ b,
                                                                     const double* __restrict__ k2,
                                                                     const double2* __restrict__ px,
                                                                     const double2* __restrict__ py, int Nx, int Ny,
                                                                     int64_t rhs_stride, double inv_h2,
                                                                     double* __restrict__ partial) {
  int i = blockIdx.x * STENCIL_THREADS + threadIdx.x;
  int j0 = blockIdx.y * STENCIL_ROWS;
  const double2* xr = x + blockIdx.z * rhs_stride;
  const double2* br = b + blockIdx.z * rhs_stride;
  double sr = 0.0, sb = 0.0;
  if (i < Nx) {
    const double2 sxi = px[i], ixm = px[Nx + i], ixp = px[Nx + i + 1];
    double2 uS = ld_u<double, false>(xr, j0 - 1, i, Nx, Ny);
    double2 uC = ld_u<double, false>(xr, j0, i, Nx, Ny);
#pragma unroll
    for (int q = 0; q < STENCIL_ROWS; ++q) {
      int j = j0 + q;
      if (j >= Ny) break;
      double2 uN = ld_u<double, false>(xr, j + 1, i, Nx, Ny);
      double2 uW = ld_u<double, false>(xr, j, i - 1, Nx, Ny);
      double2 uE = ld_u<double, false>(xr, j, i + 1, Nx, Ny);
      int64_t idx = (int64_t)j * Nx + i;
      double2 Au = stencil_point<double>(uC, uE, uW, uN, uS, sxi, ixm, ixp, py[j], py[Ny + j], py[Ny + j + 1],
                                         k2[idx], inv_h2);
      double2 bv = br[idx];
      double2 res = csub(bv, Au);
      sr += res.x * res.x + res.y * res.y;
      sb += bv.x * bv.x + bv.y * bv.y;
      uS = uC;
      uC = uN;
    }
  }
  __shared__ double red[2][STENCIL_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = sr;
    red[1][w] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int k = 0; k < STENCIL_THREADS / 32; ++k) {
      a += red[0][k];
      c += red[1][k];
    }
    int64_t base = ((int64_t)blockIdx.z * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x) * 2;
    partial[base] = a;
    partial[base + 1] = c;
  }
}

// out[r] = sqrt(sum |r|^2 / sum |b|^2) for the nrhs columns of one system (one block per column).
__global__ void k_relres_finalize(const double* __restrict__ partial, int nparts, double* __restrict__ out) {
  const double* p = partial + (int64_t)blockIdx.x * nparts * 2;
  double sr = 0, sb = 0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
    sr += p[2 * k];
    sb += p[2 * k + 1];
  }
  __shared__ double red[2][256 / 32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      c += red[1][k];
    }
    out[blockIdx.x] = c > 0 ? sqrt(a / c) : sqrt(a);
  }
}

}  // namespace helm

extern "C" helm_status helm_relres_noalloc(helm_ctx* ctx, const void* x, const void* b, int nrhs,
                                           double* relres_dev, void* stream) {
  using namespace helm;
  if (!ctx || !x || !b || !relres_dev) return fail(HELM_ERR_INVALID_ARG, "helm_relres_noalloc: NULL argument");
  HELM_TRY(check_columns(ctx, nrhs, "helm_relres_noalloc"));
  if (((uintptr_t)x | (uintptr_t)b) & 15) return fail(HELM_ERR_INVALID_ARG, "helm_relres_noalloc: x, b must be 16-byte aligned");
  int64_t need = 0;
  for (auto& s : ctx->sys) need += (int64_t)cdiv(s.Nx, STENCIL_THREADS) * cdiv(s.Ny, STENCIL_ROWS) * nrhs * 2;
  if (need > NOALLOC_SCRATCH_DOUBLES)
    return fail(HELM_ERR_INVALID_ARG, "helm_relres_noalloc: the batch needs " + std::to_string(need) +
                                          " scratch doubles, more than the fixed maximum of " +
                                          std::to_string(NOALLOC_SCRATCH_DOUBLES) + "; use helm_relres");
  double* scratch = nullptr;
  HELM_TRY(noalloc_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  int64_t pbase = 0;
  int col0 = 0;
  for (auto& s : ctx->sys) {
    dim3 grid(cdiv(s.Nx, STENCIL_THREADS), cdiv(s.Ny, STENCIL_ROWS), nrhs);
    const double2* xs = (const double2*)x + s.off * nrhs;
    const double2* bs = (const double2*)b + s.off * nrhs;
    launch(k_relres_partials, grid, STENCIL_THREADS, 0, st, xs, bs, (const double*)(ctx->k2d + s.off),
           (const double2*)(ctx->prof_d + s.prof_x), (const double2*)(ctx->prof_d + s.prof_y), s.Nx, s.Ny, s.n,
           1.0 / (s.h * s.h), scratch + pbase);
    int nparts = (int)(grid.x * grid.y);
    launch(k_relres_finalize, nrhs, 256, 0, st, (const double*)(scratch + pbase), nparts, relres_dev + col0);
    pbase += (int64_t)nparts * nrhs * 2;
    col0 += nrhs;
  }
  HELM_CK_LAUNCH();
  return HELM_OK;
}
