// Context set-up (a1): wavenumbers, PML stretch profiles, column tables, errors.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <string>

#include "helm_internal.cuh"

namespace helm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

helm_status fail(helm_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

helm_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  g_last_error = buf;
  return e == cudaErrorMemoryAllocation ? HELM_ERR_OOM : HELM_ERR_CUDA;
}

// ------------------------------------------------------------------ wait budget and fault injection

static std::atomic<long long> g_wait_budget{DEFAULT_WAIT_BUDGET};
static std::atomic<int> g_fault_site{HELM_FAULT_NONE};
static std::atomic<int> g_fault_count{0};

long long wait_budget() { return g_wait_budget.load(std::memory_order_relaxed); }

bool take_fault(int site) {
  if (g_fault_site.load() != site) return false;
  int c = g_fault_count.load();
  while (c > 0)
    if (g_fault_count.compare_exchange_weak(c, c - 1)) return true;
  return false;
}

bool test_overrides_active() {
  return (g_fault_site.load() != HELM_FAULT_NONE && g_fault_count.load() > 0) ||
         wait_budget() != DEFAULT_WAIT_BUDGET;
}

helm_status check_columns(const helm_ctx* ctx, int nrhs, const char* name) {
  if (nrhs <= 0) return fail(HELM_ERR_INVALID_ARG, std::string(name) + ": nrhs must be > 0");
  if ((int64_t)ctx->nsys * nrhs > HELM_MAX_COLUMNS)
    return fail(HELM_ERR_INVALID_ARG, std::string(name) + ": nsys * nrhs = " +
                                          std::to_string((int64_t)ctx->nsys * nrhs) + " exceeds HELM_MAX_COLUMNS (" +
                                          std::to_string(HELM_MAX_COLUMNS) + ")");
  return HELM_OK;
}

helm_status Workspace::reserve(size_t need) {
  if (need <= bytes) return HELM_OK;
  if (take_fault(HELM_FAULT_ALLOC))
    return fail(HELM_ERR_OOM, "workspace allocation of " + std::to_string(need) + " bytes failed (injected)");
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
  size_t want = need + need / 8 + 256;
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "workspace cudaMalloc", __FILE__, __LINE__);
  }
  bytes = want;
  return HELM_OK;
}

Workspace::~Workspace() {
  if (ptr) cudaFree(ptr);
}

// Depth (same unit as h) of position t (in cells; half-integers allowed) into the PML, and the
// stretch s = 1 + i sigma / omega with sigma = sigma_max (depth / ell)^2, ell = p h (eq. 2).
static std::complex<double> stretch_at(double t, int n_int, int p, double h, double omega, double sigma_max) {
  if (p <= 0) return {1.0, 0.0};
  double d = fmax(0.0, fmax((double)p - t, t - (double)(p + n_int - 1))) * h;
  double ell = p * h;
  double sigma = sigma_max * (d / ell) * (d / ell);
  return {1.0, sigma / omega};
}

__global__ void k_wavenumbers(const void* c, int c_is_fp64, int64_t n, double omega, double* k2d, float* k2f,
                              float* chat, double* chat64, int* bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double cv = c_is_fp64 ? ((const double*)c)[i] : (double)((const float*)c)[i];
  if (!(cv > 0.0) || !isfinite(cv)) {
    atomicExch(bad, 1);
    cv = 1.0;
  }
  double k = omega / cv;
  k2d[i] = k * k;
  k2f[i] = (float)(k * k);
  chat[i] = (float)(cv / 1500.0);
  chat64[i] = cv / 1500.0;
}

int num_cols(const helm_ctx* ctx, int nrhs) { return ctx->nsys * nrhs; }

helm_status ensure_cols(helm_ctx* ctx, int nrhs) {
  if (ctx->cols_nrhs == nrhs) return HELM_OK;
  std::vector<ColDesc> cols;
  for (int s = 0; s < ctx->nsys; ++s)
    for (int r = 0; r < nrhs; ++r) {
      ColDesc c;
      c.off = ctx->sys[s].off * nrhs + r * ctx->sys[s].n;
      c.len = ctx->sys[s].n;
      c.sys = s;
      c.h2 = ctx->sys[s].h * ctx->sys[s].h;
      cols.push_back(c);
    }
  if (ctx->cols_dev) cudaFree(ctx->cols_dev);
  ctx->cols_dev = nullptr;
  HELM_CK(cudaMalloc(&ctx->cols_dev, sizeof(ColDesc) * cols.size()));
  HELM_CK(cudaMemcpy(ctx->cols_dev, cols.data(), sizeof(ColDesc) * cols.size(), cudaMemcpyHostToDevice));
  ctx->cols_host = cols;
  ctx->cols_nrhs = nrhs;
  return HELM_OK;
}

helm_status ensure_pinned(helm_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->pinned_bytes) return HELM_OK;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  HELM_CK(cudaMallocHost(&ctx->pinned, bytes));
  ctx->pinned_bytes = bytes;
  return HELM_OK;
}

void unet_buffers_free(helm_ctx* ctx);  // unet.cu

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

constexpr int PROF_SLOTS = 32;  // intervals per phase between two collections

void prof_collect(helm_ctx* ctx) {
  if (!ctx->prof_on) return;
  for (int p = 0; p < NUM_PHASES; ++p) {
    for (int k = 0; k < ctx->prof_pending[p]; ++k) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ctx->prof_ev[p][k][0], ctx->prof_ev[p][k][1]) == cudaSuccess) {
        ctx->prof_ms[p] += ms;
        ctx->prof_cnt[p] += 1;
      }
    }
    ctx->prof_pending[p] = 0;
  }
}

void prof_begin(helm_ctx* ctx, int ph, cudaStream_t st) {
  if (!ctx->prof_on) return;
  if (ctx->prof_pending[ph] >= PROF_SLOTS) {  // ring full: wait for the recorded intervals and add them
    cudaEventSynchronize(ctx->prof_ev[ph][PROF_SLOTS - 1][1]);
    prof_collect(ctx);
  }
  cudaEventRecord(ctx->prof_ev[ph][ctx->prof_pending[ph]][0], st);
}

void prof_end(helm_ctx* ctx, int ph, cudaStream_t st) {
  if (!ctx->prof_on) return;
  cudaEventRecord(ctx->prof_ev[ph][ctx->prof_pending[ph]][1], st);
  ctx->prof_pending[ph] += 1;
}

}  // namespace helm

extern "C" uint64_t helm_launch_count(void) { return helm::g_launches.load(); }

extern "C" helm_status helm_profile_enable(helm_ctx* ctx, int on) {
  if (!ctx) return helm::fail(HELM_ERR_INVALID_ARG, "helm_profile_enable: NULL context");
  if (on && !ctx->prof_ev[0][0][0]) {
    for (int p = 0; p < helm::NUM_PHASES; ++p)
      for (auto& pair : ctx->prof_ev[p])
        for (auto& e : pair) HELM_CK(cudaEventCreate(&e));
  }
  ctx->prof_on = on ? 1 : 0;
  for (int p = 0; p < helm::NUM_PHASES; ++p) {
    ctx->prof_ms[p] = 0;
    ctx->prof_cnt[p] = 0;
    ctx->prof_pending[p] = 0;
    ctx->prof_work[p] = 0;
  }
  return HELM_OK;
}

extern "C" helm_status helm_profile_work(const helm_ctx* ctx, double* work_host) {
  if (!ctx || !work_host) return helm::fail(HELM_ERR_INVALID_ARG, "helm_profile_work: NULL argument");
  for (int p = 0; p < helm::NUM_PHASES; ++p) work_host[p] = ctx->prof_work[p];
  return HELM_OK;
}

extern "C" helm_status helm_profile_read(const helm_ctx* ctx, double* ms_host, int64_t* counts_host) {
  if (!ctx || !ms_host) return helm::fail(HELM_ERR_INVALID_ARG, "helm_profile_read: NULL argument");
  for (int p = 0; p < helm::NUM_PHASES; ++p) {
    ms_host[p] = ctx->prof_ms[p];
    if (counts_host) counts_host[p] = ctx->prof_cnt[p];
  }
  return HELM_OK;
}

using namespace helm;

extern "C" const char* helm_last_error(void) { return g_last_error.c_str(); }

extern "C" helm_status helm_create(helm_ctx** out, int nsys, const helm_grid* grid, const helm_pml* pml,
                                   const double* omega, const void* c_dev, int c_is_fp64, void* stream) {
  if (!out) return fail(HELM_ERR_INVALID_ARG, "helm_create: out is NULL");
  *out = nullptr;
  if (nsys <= 0 || !grid || !pml || !omega || !c_dev)
    return fail(HELM_ERR_INVALID_ARG, "helm_create: nsys must be > 0 and grid, pml, omega, c must be non-NULL");
  helm_ctx* ctx = new helm_ctx();
  ctx->nsys = nsys;
  int64_t off = 0, px = 0;
  for (int s = 0; s < nsys; ++s) {
    SysHost h{};
    h.nx = grid[s].nx;
    h.ny = grid[s].ny;
    h.p = pml[s].width;
    h.h = grid[s].h;
    h.omega = omega[s];
    if (h.nx <= 0 || h.ny <= 0 || h.p < 0 || !(h.h > 0) || !(h.omega > 0) || !std::isfinite(h.h) ||
        !std::isfinite(h.omega)) {
      delete ctx;
      return fail(HELM_ERR_INVALID_ARG, "helm_create: system " + std::to_string(s) +
                                            " needs nx, ny > 0, width >= 0, h > 0 and omega > 0");
    }
    h.sigma_max = pml[s].sigma_max > 0 ? pml[s].sigma_max : 2.0 * h.omega;
    h.Nx = h.nx + 2 * h.p;
    h.Ny = h.ny + 2 * h.p;
    if ((int64_t)h.Nx * h.Ny > (int64_t)1 << 31) {
      delete ctx;
      return fail(HELM_ERR_INVALID_ARG, "helm_create: grid larger than 2^31 points");
    }
    h.n = (int64_t)h.Nx * h.Ny;
    h.off = off;
    off += h.n;
    h.prof_x = px;
    px += 2 * h.Nx + 1;
    h.prof_y = px;
    px += 2 * h.Ny + 1;
    ctx->sys.push_back(h);
  }
  ctx->npts = off;
  ctx->prof_len = px;
  // profiles on the host in FP64: [s(node) x N][1/s(half) x (N+1)] per axis
  std::vector<double2> pd(px);
  std::vector<float2> pf(px);
  for (auto& h : ctx->sys) {
    for (int axis = 0; axis < 2; ++axis) {
      int N = axis == 0 ? h.Nx : h.Ny;
      int nint = axis == 0 ? h.nx : h.ny;
      int64_t base = axis == 0 ? h.prof_x : h.prof_y;
      for (int i = 0; i < N; ++i) {
        auto s = stretch_at((double)i, nint, h.p, h.h, h.omega, h.sigma_max);
        pd[base + i] = make_double2(s.real(), s.imag());
      }
      for (int i = 0; i <= N; ++i) {
        auto s = 1.0 / stretch_at((double)i - 0.5, nint, h.p, h.h, h.omega, h.sigma_max);
        pd[base + N + i] = make_double2(s.real(), s.imag());
      }
    }
  }
  for (int64_t i = 0; i < px; ++i) pf[i] = make_float2((float)pd[i].x, (float)pd[i].y);
  // unit[base + i] = 1 where node i of that axis has s(i) = 1/s(i - 1/2) = 1/s(i + 1/2) = 1 exactly
  // in FP32 (outside the PML), so the FP32 stencil may take its short form there
  std::vector<unsigned char> unit(px, 0);
  auto one = [](float2 v) { return v.x == 1.0f && v.y == 0.0f; };
  for (auto& h : ctx->sys)
    for (int axis = 0; axis < 2; ++axis) {
      int N = axis == 0 ? h.Nx : h.Ny;
      int64_t base = axis == 0 ? h.prof_x : h.prof_y;
      for (int i = 0; i < N; ++i)
        unit[base + i] = one(pf[base + i]) && one(pf[base + N + i]) && one(pf[base + N + i + 1]);
    }
  cudaStream_t st = (cudaStream_t)stream;
  helm_status rc = HELM_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == HELM_OK) rc = cuda_fail(e, what, __FILE__, __LINE__);
  };
  ck(cudaMalloc(&ctx->k2f, sizeof(float) * off), "cudaMalloc k2f");
  ck(cudaMalloc(&ctx->k2d, sizeof(double) * off), "cudaMalloc k2d");
  ck(cudaMalloc(&ctx->chat, sizeof(float) * off), "cudaMalloc chat");
  ck(cudaMalloc(&ctx->chat64, sizeof(double) * off), "cudaMalloc chat64");
  ck(cudaMalloc(&ctx->prof_d, sizeof(double2) * px), "cudaMalloc prof_d");
  ck(cudaMalloc(&ctx->prof_f, sizeof(float2) * px), "cudaMalloc prof_f");
  ck(cudaMalloc(&ctx->unit_f, px), "cudaMalloc unit_f");
  ck(cudaMalloc(&ctx->flag_dev, sizeof(int) * 16), "cudaMalloc flag");
  if (rc != HELM_OK) {
    helm_destroy(ctx);
    return rc;
  }
  ck(cudaMemcpyAsync(ctx->prof_d, pd.data(), sizeof(double2) * px, cudaMemcpyHostToDevice, st), "copy prof_d");
  ck(cudaMemcpyAsync(ctx->prof_f, pf.data(), sizeof(float2) * px, cudaMemcpyHostToDevice, st), "copy prof_f");
  ck(cudaMemcpyAsync(ctx->unit_f, unit.data(), px, cudaMemcpyHostToDevice, st), "copy unit_f");
  ck(cudaMemsetAsync(ctx->flag_dev, 0, sizeof(int) * 16, st), "memset flag");
  for (auto& h : ctx->sys) {
    const char* cb = (const char*)c_dev + h.off * (c_is_fp64 ? 8 : 4);
    launch(k_wavenumbers, cdiv(h.n, 256), 256, 0, st, cb, c_is_fp64, h.n, h.omega, ctx->k2d + h.off,
                                                   ctx->k2f + h.off, ctx->chat + h.off, ctx->chat64 + h.off,
                                                   ctx->flag_dev);
  }
  ck(cudaGetLastError(), "k_wavenumbers launch");
  int bad = 0;
  ck(cudaMemcpyAsync(&bad, ctx->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
  ck(cudaStreamSynchronize(st), "sync");
  if (rc == HELM_OK && bad) rc = fail(HELM_ERR_INVALID_ARG, "helm_create: c must be positive and finite everywhere");
  if (rc == HELM_OK) ck(cudaMemsetAsync(ctx->flag_dev, 0, sizeof(int) * 16, st), "memset flag");
  if (rc != HELM_OK) {
    helm_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return HELM_OK;
}

extern "C" helm_status helm_set_velocity(helm_ctx* ctx, const void* c_dev, int c_is_fp64, void* stream) {
  if (!ctx || !c_dev) return fail(HELM_ERR_INVALID_ARG, "helm_set_velocity: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  HELM_CK(cudaMemsetAsync(ctx->flag_dev, 0, sizeof(int), st));
  for (auto& h : ctx->sys) {
    const char* cb = (const char*)c_dev + h.off * (c_is_fp64 ? 8 : 4);
    launch(k_wavenumbers, cdiv(h.n, 256), 256, 0, st, cb, c_is_fp64, h.n, h.omega, ctx->k2d + h.off, ctx->k2f + h.off,
           ctx->chat + h.off, ctx->chat64 + h.off, ctx->flag_dev);
  }
  HELM_CK_LAUNCH();
  int bad = 0;
  HELM_CK(cudaMemcpyAsync(&bad, ctx->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  if (bad) {
    cudaMemsetAsync(ctx->flag_dev, 0, sizeof(int), st);
    return fail(HELM_ERR_INVALID_ARG, "helm_set_velocity: c must be positive and finite everywhere");
  }
  return HELM_OK;
}

extern "C" helm_status helm_destroy(helm_ctx* ctx) {
  if (!ctx) return HELM_OK;
  cudaDeviceSynchronize();
  unet_buffers_free(ctx);
  cudaFree(ctx->k2f);
  cudaFree(ctx->k2d);
  cudaFree(ctx->chat);
  cudaFree(ctx->chat64);
  cudaFree(ctx->prof_d);
  cudaFree(ctx->prof_f);
  cudaFree(ctx->unit_f);
  cudaFree(ctx->cols_dev);
  cudaFree(ctx->flag_dev);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (auto& pe : ctx->prof_ev)
    for (auto& pair : pe)
      for (auto& e : pair)
        if (e) cudaEventDestroy(e);
  delete ctx;
  return HELM_OK;
}

extern "C" int64_t helm_points(const helm_ctx* ctx) { return ctx ? ctx->npts : 0; }
extern "C" int helm_num_systems(const helm_ctx* ctx) { return ctx ? ctx->nsys : 0; }

extern "C" helm_status helm_set_wait_budget(int64_t cycles) {
  helm::g_wait_budget.store(cycles > 0 ? (long long)cycles : helm::DEFAULT_WAIT_BUDGET);
  return HELM_OK;
}

extern "C" helm_status helm_inject_fault(int site, int count) {
  if (site < HELM_FAULT_NONE || site > HELM_FAULT_ALLOC)
    return helm::fail(HELM_ERR_INVALID_ARG, "helm_inject_fault: unknown site");
  helm::g_fault_count.store(0);
  helm::g_fault_site.store(count > 0 ? site : HELM_FAULT_NONE);
  helm::g_fault_count.store(site == HELM_FAULT_NONE ? 0 : std::max(count, 0));
  return HELM_OK;
}
