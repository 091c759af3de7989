// Internal declarations shared by the libhelm translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/helm.h"

namespace helm {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);
helm_status fail(helm_status st, const std::string& msg);
helm_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define HELM_CK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return ::helm::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HELM_CK_LAUNCH() HELM_CK(cudaGetLastError())

#define HELM_TRY(expr)                     \
  do {                                     \
    helm_status s_ = (expr);               \
    if (s_ != HELM_OK) return s_;          \
  } while (0)

// ------------------------------------------------------------------ complex helpers

template <typename R> struct cplx;
template <> struct cplx<float> { using T = float2; };
template <> struct cplx<double> { using T = double2; };
template <typename R> using C = typename cplx<R>::T;

template <typename R> __host__ __device__ __forceinline__ C<R> mk(R a, R b) { C<R> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ T cadd(T a, T b) { a.x += b.x; a.y += b.y; return a; }
template <typename T> __host__ __device__ __forceinline__ T csub(T a, T b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
  T r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename T> __host__ __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
template <typename T, typename S> __host__ __device__ __forceinline__ T cscale(T a, S s) { a.x *= s; a.y *= s; return a; }
// conj(a) * b
template <typename T> __host__ __device__ __forceinline__ T cdotc(T a, T b) {
  T r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}

// ------------------------------------------------------------------ context

struct SysHost {
  int nx, ny, p, Nx, Ny;
  double h, omega, sigma_max;
  int64_t off;        // first point of this system within one right-hand side block set
  int64_t n;          // Nx * Ny
  int64_t prof_x, prof_y;  // offsets into the profile arrays
};

// Column = (system, right-hand side).  Device copy used by reduction kernels.
struct ColDesc {
  int64_t off;  // first element of the column in a batch vector
  int64_t len;  // points
  int sys;
  double h2;    // h^2 of the column's system (network output scale)
};

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
  helm_status reserve(size_t need);
  ~Workspace();
};

struct UnetBuffers;  // activation storage, defined in unet.cu

struct helm_ctx_impl;

}  // namespace helm

struct helm_ctx {
  int nsys = 0;
  std::vector<helm::SysHost> sys;
  int64_t npts = 0;            // sum of n_s
  // per point (npts): k^2 in both precisions, c / 1500 m/s
  float* k2f = nullptr;
  double* k2d = nullptr;
  float* chat = nullptr;
  double* chat64 = nullptr;
  // per system 1-D profiles: s(node) and 1 / s(half node) in x and y, both precisions
  double2* prof_d = nullptr;
  float2* prof_f = nullptr;
  unsigned char* unit_f = nullptr;  // per profile node: 1 where the FP32 stretch factors are all 1
  int64_t prof_len = 0;
  // per-nrhs column tables (rebuilt on demand)
  int cols_nrhs = -1;
  helm::ColDesc* cols_dev = nullptr;
  std::vector<helm::ColDesc> cols_host;
  // scratch for reductions and solver state
  helm::Workspace ws_red, ws_solver, ws_vec, ws_unet, ws_train;
  helm::UnetBuffers* ub = nullptr;
  int* flag_dev = nullptr;         // device error/status flag
  void* pinned = nullptr;          // small pinned host buffer for status reads
  size_t pinned_bytes = 0;
  // residual-estimate history of column 0 of the last solve (relative to ||b||), one entry per iteration
  std::vector<double> history;
  // phase timers: per phase a ring of event pairs, collected after each host synchronisation
  int prof_on = 0;
  cudaEvent_t prof_ev[8][32][2] = {};
  int prof_pending[8] = {};
  double prof_ms[8] = {};
  int64_t prof_cnt[8] = {};
  double prof_work[8] = {};  // algorithmic flops (preconditioner) or bytes (other phases) issued
};

namespace helm {

// ctx.cu
helm_status ensure_cols(helm_ctx* ctx, int nrhs);
helm_status ensure_pinned(helm_ctx* ctx, size_t bytes);
int num_cols(const helm_ctx* ctx, int nrhs);

// stencil.cu: y = A x (or A^H x) for all systems and right-hand sides
template <typename R>
helm_status apply_op(helm_ctx* ctx, const C<R>* x, C<R>* y, int nrhs, bool adjoint, cudaStream_t st);
// TMA-tiled FP32 stencil (stencil_tma.cu): even Nx and 16-byte aligned x, y.  A pipeline timeout
// is recorded in *err (code 21).
bool stencil_tma_supported(int Nx, int Ny, const void* x, const void* y);
helm_status stencil_tma(const float2* x, float2* y, const float* k2, const float2* px, const float2* py,
                        const unsigned char* ux, const unsigned char* uy, int Nx, int Ny, int nrhs, float inv_h2,
                        bool adjoint, int* err, cudaStream_t st);
// HELM_TIMEOUT if a stencil launch recorded a TMA wait timeout since the last check (synchronises).
helm_status stencil_check(helm_ctx* ctx, cudaStream_t st);
// r = b - A x (FP64) and per-column ||r||^2, ||b||^2 into sums[col*2 + {0,1}] (device)
helm_status residual_fp64(helm_ctx* ctx, const double2* x, const double2* b, double2* r, int nrhs,
                          double* sums, cudaStream_t st);
// the same in either precision (sums always FP64)
template <typename R>
helm_status residual_op(helm_ctx* ctx, const C<R>* x, const C<R>* b, C<R>* r, int nrhs, double* sums,
                        cudaStream_t st);

// reduce.cu: per-column sum of |v|^2 (FP64) into out[col] (device); deterministic
template <typename R>
helm_status col_norm2(helm_ctx* ctx, const C<R>* v, int nrhs, double* out, cudaStream_t st);

// out[col * nvals + v] = sum over the column's partials in a fixed order (stencil.cu)
__global__ void k_finalize(const double* __restrict__ partial, const int* __restrict__ nparts_col, int nvals,
                           double* __restrict__ out);

// Pipeline-wait budget (clock64 cycles) of the TMA / tcgen05 kernels and the host-side failure
// injection of helm_set_wait_budget / helm_inject_fault (ctx.cu).
constexpr long long DEFAULT_WAIT_BUDGET = 2000000000LL;
long long wait_budget();
bool take_fault(int site);        // consumes one armed occurrence of `site`
bool test_overrides_active();     // a fault is armed or the budget differs from the default
// HELM_ERR_INVALID_ARG unless 0 < nrhs and nsys * nrhs <= HELM_MAX_COLUMNS
helm_status check_columns(const helm_ctx* ctx, int nrhs, const char* name);

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Every kernel of the library is launched through launch(): it keeps a process-wide count of
// launches (helm_launch_count) for the benchmark's launch accounting.
void count_launch();
void count_launches(uint64_t n);    // kernels of a CUDA graph replay
void uncount_launches(uint64_t n);  // kernels captured into a graph (recorded, not run)
template <typename... KArgs, typename... Args>
inline void launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  k<<<grid, block, smem, st>>>(args...);
  count_launch();
}

// Phase timers of the solver (CUDA events on the solver's stream), enabled by helm_profile_enable.
enum Phase { PH_PRECOND = 0, PH_STENCIL, PH_ORTH, PH_LSQ, PH_RESIDUAL, PH_UPDATE, NUM_PHASES };
void prof_begin(helm_ctx* ctx, int ph, cudaStream_t st);
void prof_end(helm_ctx* ctx, int ph, cudaStream_t st);
void prof_collect(helm_ctx* ctx);  // after a stream synchronisation: add the recorded intervals

}  // namespace helm
