// TMA-tiled FP32 stencil (a2, eq. 3): the complex 5-point operator with PML stretching on tiles
// staged in shared memory by the tensor-memory accelerator.
//
// A persistent CTA walks tiles of TH rows x ST_TW points of one right-hand side.  One 3-D TMA box
// per tile brings the (TH + 2) x (ST_TW + 4) halo window of u (FP32 complex viewed as floats,
// starting two points left of the tile so that the copy starts on a 16-byte boundary) into shared
// memory; out-of-range rows and columns arrive as zeros, which are exactly the homogeneous
// Dirichlet ghost values.  STAGES boxes are in flight per CTA, so the loads of later tiles
// overlap the arithmetic of the current one.  Each thread owns two adjacent points of a row (16-byte
// shared-memory reads, one 16-byte global store) and TH / 8 rows.  Per point the kernel moves the
// algorithmic 8 + 8 + 4 B of HBM traffic (u, A u, k^2); the halo re-reads come from L2.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "helm_internal.cuh"
#include "stencil_point.cuh"
#include "tc_ptx.cuh"

namespace helm {

constexpr int ST_TW = 64;                       // output points per tile row (32 lanes x 2 points)
constexpr int ST_BW = ST_TW + 4;                // loaded points per row (x0 - 2 .. x0 + ST_TW + 1)
constexpr int ST_THREADS = 256;

// Tile height TH (rows; a multiple of 8: each of the 8 warps owns TH / 8 rows) and pipeline depth.
template <int TH, int STAGES>
struct StCfg {
  static constexpr int BH = TH + 2;                                  // loaded rows (y0 - 1 .. y0 + TH)
  static constexpr int STAGE_BYTES = ST_BW * BH * 8;                 // one u box
  static constexpr int K2_BYTES = ST_TW * TH * 4;                    // one k^2 box
  static constexpr int K2_OFF = (STAGE_BYTES + 127) / 128 * 128;     // k^2 box after the u box
  static constexpr int STAGE_STRIDE = K2_OFF + K2_BYTES;             // stages start 128-byte aligned
  static constexpr int SMEM = STAGES * STAGE_STRIDE + 128;
  static_assert(TH % 8 == 0, "tile height");
};

__device__ __forceinline__ float4 conj4(float4 v) { return make_float4(v.x, -v.y, v.z, -v.w); }
__device__ __forceinline__ float2 conj2(float2 v) { return make_float2(v.x, -v.y); }

// K2T: the k^2 tile comes with the u window (second box of the stage) instead of from global loads.
// ux / uy: per-node flags, 1 where all FP32 stretch factors of that column / row are exactly 1.
template <bool ADJ, bool K2T, int TH, int ST_STAGES>
__global__ void __launch_bounds__(ST_THREADS) k_stencil_tma(const __grid_constant__ CUtensorMap tu,
                                                            const __grid_constant__ CUtensorMap tk,
                                                            float2* __restrict__ y, const float* __restrict__ k2,
                                                            const float2* __restrict__ px,
                                                            const float2* __restrict__ py,
                                                            const unsigned char* __restrict__ ux,
                                                            const unsigned char* __restrict__ uy, int Nx, int Ny,
                                                            int tiles_x, int tiles_y, int ntiles, int64_t rhs_stride,
                                                            float inv_h2, int* err, long long budget,
                                                            int skip_first) {
  using Cfg = StCfg<TH, ST_STAGES>;
  constexpr int ST_TH = TH;
  constexpr int ST_STAGE_BYTES = Cfg::STAGE_BYTES, ST_K2_BYTES = Cfg::K2_BYTES, ST_K2_OFF = Cfg::K2_OFF;
  constexpr int ST_STAGE_STRIDE = Cfg::STAGE_STRIDE;
  extern __shared__ __align__(128) unsigned char st_smem[];
  unsigned char* buf = (unsigned char*)(((uintptr_t)st_smem + 127) & ~(uintptr_t)127);
  __shared__ uint64_t full[ST_STAGES];
  __shared__ int tile_xy[ST_STAGES][3];  // (rhs, first row, first point) of the tile in each stage
  __shared__ int abort_s;
  volatile int* abort_flag = &abort_s;
  const int tid = threadIdx.x;
  const int per_rhs = tiles_x * tiles_y;
  if (tid == 0) {
    for (int s = 0; s < ST_STAGES; ++s) mbar_init(&full[s], 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  // thread 0 decodes the tile once, publishes it with the stage (the arrive below releases it)
  auto issue = [&](int t, int s) {
    const int rhs = t / per_rhs, r = t % per_rhs;
    const int y0 = (r / tiles_x) * ST_TH, x0 = (r % tiles_x) * ST_TW;
    tile_xy[s][0] = rhs;
    tile_xy[s][1] = y0;
    tile_xy[s][2] = x0;
    mbar_expect_tx(&full[s], ST_STAGE_BYTES + (K2T ? ST_K2_BYTES : 0));
    unsigned char* dst = buf + s * ST_STAGE_STRIDE;
    tma_load_3d(dst, &tu, &full[s], 2 * (x0 - 2), y0 - 1, rhs);
    if (K2T) tma_load_3d(dst + ST_K2_OFF, &tk, &full[s], x0, y0, 0);
  };
  int fills[ST_STAGES] = {};  // boxes requested per stage (thread 0's count; the drain waits for the last)
  if (tid == 0)
    for (int s = 0; s < ST_STAGES; ++s) {
      const int t = blockIdx.x + s * gridDim.x;
      if (t < ntiles && !(skip_first && t == 0)) {  // injected fault: tile 0 of CTA 0 never arrives
        issue(t, s);
        ++fills[s];
      }
    }
  const int c = tid & 31, rg = tid >> 5;  // point pair c of rows rg, rg + 8
  int stage = 0;
  uint32_t phase = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // every thread observes the stage's barrier; the block leaves the loop together (below) when
    // any thread gave up, so that no thread waits at a barrier the others have left
    const bool got = mbar_wait(&full[stage], phase, abort_flag, err, 21, budget);
    const int rhs = tile_xy[stage][0], y0 = tile_xy[stage][1];
    const int x = tile_xy[stage][2] + 2 * c;
    const unsigned char* sb = buf + stage * ST_STAGE_STRIDE;
    if (got && x < Nx) {
      const bool xunit = ux[x] && ux[x + 1];
      float2* yr = y + rhs * rhs_stride;
#pragma unroll
      for (int p = 0; p < ST_TH / 8; ++p) {
        const int rr = rg + 8 * p;
        const int j = y0 + rr;
        if (j >= Ny) break;
        const float2* row = (const float2*)sb + (rr + 1) * ST_BW + 2 * c + 2;  // the tile point x in the window
        float4 uC = *(const float4*)row, uS = *(const float4*)(row - ST_BW), uN = *(const float4*)(row + ST_BW);
        float2 w0 = row[-1], e1 = row[2];
        if (ADJ) {
          uC = conj4(uC);
          uS = conj4(uS);
          uN = conj4(uN);
          w0 = conj2(w0);
          e1 = conj2(e1);
        }
        const float2 kk = K2T ? *(const float2*)(sb + ST_K2_OFF + (rr * ST_TW + 2 * c) * 4)
                              : __ldg((const float2*)(k2 + (int64_t)j * Nx + x));
        const float2 c0 = make_float2(uC.x, uC.y), c1 = make_float2(uC.z, uC.w);
        const float2 n0 = make_float2(uN.x, uN.y), n1 = make_float2(uN.z, uN.w);
        const float2 s0 = make_float2(uS.x, uS.y), s1 = make_float2(uS.z, uS.w);
        const bool yunit = uy[j];
        float2 o0, o1;
        if (xunit && yunit) {
          o0 = stencil_point_unit<float>(c0, c1, w0, n0, s0, kk.x, inv_h2);
          o1 = stencil_point_unit<float>(c1, e1, c0, n1, s1, kk.y, inv_h2);
        } else if (yunit) {
          const float2 sx0 = px[x], sx1 = px[x + 1];
          const float2 im0 = px[Nx + x], im1 = px[Nx + x + 1], ip1 = px[Nx + x + 2];
          o0 = stencil_point_xpml<float>(c0, c1, w0, n0, s0, sx0, im0, im1, kk.x, inv_h2);
          o1 = stencil_point_xpml<float>(c1, e1, c0, n1, s1, sx1, im1, ip1, kk.y, inv_h2);
        } else if (xunit) {
          const float2 syj = py[j], iym = py[Ny + j], iyp = py[Ny + j + 1];
          o0 = stencil_point_ypml<float>(c0, c1, w0, n0, s0, syj, iym, iyp, kk.x, inv_h2);
          o1 = stencil_point_ypml<float>(c1, e1, c0, n1, s1, syj, iym, iyp, kk.y, inv_h2);
        } else {
          const float2 sx0 = px[x], sx1 = px[x + 1];
          const float2 im0 = px[Nx + x], im1 = px[Nx + x + 1], ip1 = px[Nx + x + 2];
          const float2 syj = py[j], iym = py[Ny + j], iyp = py[Ny + j + 1];
          o0 = stencil_point<float>(c0, c1, w0, n0, s0, sx0, im0, im1, syj, iym, iyp, kk.x, inv_h2);
          o1 = stencil_point<float>(c1, e1, c0, n1, s1, sx1, im1, ip1, syj, iym, iyp, kk.y, inv_h2);
        }
        if (ADJ) {
          o0.y = -o0.y;
          o1.y = -o1.y;
        }
        *(float4*)(yr + (int64_t)j * Nx + x) = make_float4(o0.x, o0.y, o1.x, o1.y);
      }
    }
    // every thread is done with this stage's window (or some thread gave up: stop issuing)
    if (__syncthreads_or(!got)) break;
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order those reads before the refill
      const int tn = t + ST_STAGES * gridDim.x;
      if (tn < ntiles) {
        issue(tn, stage);
        ++fills[stage];
      }
    }
    if (++stage == ST_STAGES) {
      stage = 0;
      phase ^= 1;
    }
  }
  // let every box requested land before the CTA exits (bounded; already done on the normal path)
  if (tid == 0)
#pragma unroll
    for (int s = 0; s < ST_STAGES; ++s) mbar_drain(&full[s], fills[s]);
}

typedef CUresult (*EncodeTiledFnS)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFnS encode_fn() {
  static EncodeTiledFnS fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFnS)p;
  });
  return fn;
}

static helm_status stencil_map(CUtensorMap* m, const void* ptr, int Nx, int Ny, int nrhs, int th) {
  EncodeTiledFnS fn = encode_fn();
  if (!fn) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  // FP32 complex viewed as floats: [nrhs][Ny][2 Nx]
  cuuint64_t dims[3] = {(cuuint64_t)2 * Nx, (cuuint64_t)Ny, (cuuint64_t)nrhs};
  cuuint64_t strides[2] = {(cuuint64_t)Nx * 8, (cuuint64_t)Nx * Ny * 8};
  cuuint32_t box[3] = {2 * ST_BW, (cuuint32_t)(th + 2), 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (stencil) failed: " + std::to_string((int)r));
  return HELM_OK;
}

// k^2 of one system as a [1][Ny][Nx] float tensor (row stride 4 Nx bytes: needs Nx % 4 == 0)
static helm_status k2_map(CUtensorMap* m, const float* k2, int Nx, int Ny, int th) {
  EncodeTiledFnS fn = encode_fn();
  if (!fn) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)Nx, (cuuint64_t)Ny, 1};
  cuuint64_t strides[2] = {(cuuint64_t)Nx * 4, (cuuint64_t)Nx * Ny * 4};
  cuuint32_t box[3] = {ST_TW, (cuuint32_t)th, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(k2), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (k^2) failed: " + std::to_string((int)r));
  return HELM_OK;
}

bool stencil_tma_supported(int Nx, int Ny, const void* x, const void* y) {
  return Nx >= 2 && Ny >= 1 && (Nx & 1) == 0 && (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
}

// One tile shape: maps, occupancy, launch.
template <bool ADJ, bool K2T, int TH, int STAGES>
static helm_status launch_stencil_tma(const float2* x, float2* y, const float* k2, const float2* px,
                                      const float2* py, const unsigned char* ux, const unsigned char* uy, int Nx,
                                      int Ny, int nrhs, float inv_h2, int* err, long long budget, int skip_first,
                                      cudaStream_t st) {
  using Cfg = StCfg<TH, STAGES>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int nsm = 148, per_sm = 1;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_stencil_tma<ADJ, K2T, TH, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Cfg::SMEM);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int a = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_stencil_tma<ADJ, K2T, TH, STAGES>, ST_THREADS, Cfg::SMEM);
    per_sm = std::max(1, a);
  });
  HELM_CK(attr_err);
  const int tiles_x = (Nx + ST_TW - 1) / ST_TW, tiles_y = (Ny + TH - 1) / TH;
  const int ntiles = tiles_x * tiles_y * nrhs;
  if (ntiles == 0) return HELM_OK;
  CUtensorMap mu, mk;
  HELM_TRY(stencil_map(&mu, x, Nx, Ny, nrhs, TH));
  if (K2T)
    HELM_TRY(k2_map(&mk, k2, Nx, Ny, TH));
  else
    mk = mu;
  const int grid = std::min(ntiles, nsm * per_sm);
  launch(k_stencil_tma<ADJ, K2T, TH, STAGES>, grid, ST_THREADS, Cfg::SMEM, st, mu, mk, y, k2, px, py, ux, uy, Nx, Ny,
         tiles_x, tiles_y, ntiles, (int64_t)Nx * Ny, inv_h2, err, budget, skip_first);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

// ------------------------------------------------------------------ tile autotuner
//
// The tile height trades halo re-reads ((TH + 2) / TH rows loaded per row) against the number of
// tiles in flight per SM (shared memory per stage).  On the first call for a grid shape (Nx, Ny,
// nrhs, adjoint, k^2 staged) every candidate runs once untimed and then three times timed with CUDA
// events on the caller's stream, in interleaved rounds, and the lowest total is kept.  Every candidate computes each point with the same
// arithmetic, so the choice never changes a result.  HELM_AUTOTUNE=0 keeps the first candidate, as do
// calls during a stream capture.

typedef helm_status (*StLaunchFn)(const float2*, float2*, const float*, const float2*, const float2*,
                                  const unsigned char*, const unsigned char*, int, int, int, float, int*, long long,
                                  int, cudaStream_t);
struct StCand {
  int th, stages;
  StLaunchFn fn;
};

template <bool ADJ, bool K2T>
static const std::vector<StCand>& st_candidates() {
  static const std::vector<StCand> c = {{32, 2, launch_stencil_tma<ADJ, K2T, 32, 2>},
                                        {16, 4, launch_stencil_tma<ADJ, K2T, 16, 4>},
                                        {32, 3, launch_stencil_tma<ADJ, K2T, 32, 3>},
                                        {64, 2, launch_stencil_tma<ADJ, K2T, 64, 2>}};
  return c;
}

struct StKey {
  int Nx, Ny, nrhs, adj, k2t;
  bool operator<(const StKey& o) const {
    return std::tie(Nx, Ny, nrhs, adj, k2t) < std::tie(o.Nx, o.Ny, o.nrhs, o.adj, o.k2t);
  }
};
static std::mutex g_st_mu;
static std::map<StKey, int> g_st_choice;
static std::atomic<int> g_st_forced{0};  // helm_set_stencil_variant: 0 = tuned, k = candidate k

static bool st_autotune_enabled() {
  static const bool on = [] {
    const char* e = getenv("HELM_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <bool ADJ, bool K2T>
static helm_status stencil_tuned(const float2* x, float2* y, const float* k2, const float2* px, const float2* py,
                                 const unsigned char* ux, const unsigned char* uy, int Nx, int Ny, int nrhs,
                                 float inv_h2, int* err, long long budget, int skip, cudaStream_t st) {
  const auto& cands = st_candidates<ADJ, K2T>();
  const int forced = g_st_forced.load();
  if (forced > 0)
    return cands[std::min<size_t>(forced, cands.size()) - 1].fn(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err,
                                                                 budget, skip, st);
  const StKey key{Nx, Ny, nrhs, ADJ ? 1 : 0, K2T ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_st_mu);
    auto it = g_st_choice.find(key);
    if (it != g_st_choice.end())
      return cands[it->second].fn(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, skip, st);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HELM_CK(cudaStreamIsCapturing(st, &cap));
  if (!st_autotune_enabled() || cap != cudaStreamCaptureStatusNone || skip)
    return cands[0].fn(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, skip, st);
  cudaEvent_t e0, e1;
  HELM_CK(cudaEventCreate(&e0));
  HELM_CK(cudaEventCreate(&e1));
  helm_status rc = HELM_OK;
  for (size_t i = 0; i < cands.size() && rc == HELM_OK; ++i)  // set-up, warm-up
    rc = cands[i].fn(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, 0, st);
  // ST_ROUNDS timed rounds over all candidates (interleaved, so that each candidate meets the same mix
  // of cache states), the lowest total wins
  constexpr int ST_ROUNDS = 3;
  std::vector<float> total(cands.size(), 0.f);
  for (int r = 0; r < ST_ROUNDS && rc == HELM_OK; ++r)
    for (size_t i = 0; i < cands.size() && rc == HELM_OK; ++i) {
      cudaEventRecord(e0, st);
      rc = cands[i].fn(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, 0, st);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (rc == HELM_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        total[i] += ms;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HELM_OK) return rc;
  int best = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (total[i] < total[best]) best = (int)i;
  std::lock_guard<std::mutex> lk(g_st_mu);
  g_st_choice[key] = best;
  return HELM_OK;
}

// Tile heights chosen so far: out[k] = {Nx, Ny, nrhs, adjoint, rows per tile, stages}.
int stencil_tuned_tiles(int (*out)[6], int max) {
  std::lock_guard<std::mutex> lk(g_st_mu);
  int k = 0;
  for (auto& kv : g_st_choice) {
    if (k >= max) break;
    const StKey& r = kv.first;
    const auto& c = (r.adj ? (r.k2t ? st_candidates<true, true>() : st_candidates<true, false>())
                           : (r.k2t ? st_candidates<false, true>() : st_candidates<false, false>()))[kv.second];
    out[k][0] = r.Nx;
    out[k][1] = r.Ny;
    out[k][2] = r.nrhs;
    out[k][3] = r.adj;
    out[k][4] = c.th;
    out[k][5] = c.stages;
    ++k;
  }
  return k;
}

helm_status stencil_tma(const float2* x, float2* y, const float* k2, const float2* px, const float2* py,
                        const unsigned char* ux, const unsigned char* uy, int Nx, int Ny, int nrhs, float inv_h2,
                        bool adjoint, int* err, cudaStream_t st) {
  const bool k2t = (Nx & 3) == 0 && ((uintptr_t)k2 & 15) == 0;
  const long long budget = wait_budget();
  const int skip = take_fault(HELM_FAULT_STENCIL_TILE) ? 1 : 0;
  if (adjoint)
    return k2t ? stencil_tuned<true, true>(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, skip, st)
               : stencil_tuned<true, false>(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, skip, st);
  return k2t ? stencil_tuned<false, true>(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, skip, st)
             : stencil_tuned<false, false>(x, y, k2, px, py, ux, uy, Nx, Ny, nrhs, inv_h2, err, budget, skip, st);
}

helm_status stencil_check(helm_ctx* ctx, cudaStream_t st) {
  int e = 0;
  HELM_CK(cudaMemcpyAsync(&e, ctx->flag_dev + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  if (e) {
    cudaMemsetAsync(ctx->flag_dev + 2, 0, sizeof(int), st);
    return fail(HELM_TIMEOUT, "stencil: a TMA wait ran out of its budget (code " + std::to_string(e) + ")");
  }
  return HELM_OK;
}

}  // namespace helm

extern "C" int helm_tuned_stencil(int* out, int max_entries) {
  if (!out || max_entries <= 0) return 0;
  return helm::stencil_tuned_tiles(reinterpret_cast<int (*)[6]>(out), max_entries);
}

extern "C" helm_status helm_set_stencil_variant(int variant) {
  if (variant < 0 || variant > 4) return helm::fail(HELM_ERR_INVALID_ARG, "helm_set_stencil_variant: 0..4");
  helm::g_st_forced.store(variant);
  return HELM_OK;
}
