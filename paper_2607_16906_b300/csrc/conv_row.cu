// Row-tile tcgen05 3x3 convolutions for the narrow layers (C_in <= 64 in 8-channel slices, C_out <= 64).
//
// The full-resolution 16- and 32-channel layers move little data per pixel, so the cost of the
// 9-box tile pipeline in conv_tc.cu (one TMA box per tap) dominates there.  Here one tile is a
// 128-pixel segment of RY consecutive image rows.  For each 8-channel slice one TMA box brings the
// RY + 2 halo rows of 130 pixels (16 bytes per pixel) into shared memory; with the innermost box
// dimension 16 bytes wide this is the non-swizzled K-major core-matrix layout (8 pixels x 16 bytes
// contiguous), so the A operand of output row r and tap (ky, dx) is the same buffer read from row
// r + ky at pixel offset dx: only the descriptor start address changes.  RY output rows share the
// RY + 2 loaded rows, cutting the L2 reads per output pixel from 3 to (RY + 2) / RY rows.  The
// weights of the layer stay resident in shared memory for the whole persistent kernel.
// Warp roles, bounded waits and the epilogue follow conv_tc.cu.
#include <cuda.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tc_ptx.cuh"
#include "unet.cuh"

namespace helm {

constexpr int ROW_PX = 128;                // output pixels per row segment (one MMA block, M = 128)
constexpr int ROW_HALO = ROW_PX + 2;       // loaded pixels per row
constexpr int ROW_PITCH = ROW_HALO * 16;   // bytes per loaded row of one slice (2080)
#ifndef ROW_EPI_BATCH
#define ROW_EPI_BATCH 2  // 16-column TMEM loads per epilogue wait
#endif

struct RowArgs {
  int B, H, W;
  int nsl0;  // 8-channel slices from source 0 (the rest from source 1)
  int tiles_x, tiles_y;
  int ntiles;
  const __nv_bfloat16* wrow;  // [tap][slice][N][8]
  const float* bias;
  __nv_bfloat16* out;  // NHWC [B][H][W][N]
  int relu;
  int* err;
  long long budget;  // clock64 cycles a pipeline wait may take before the kernel gives up
  int skip_first;    // failure injection: CTA 0 issues no loads for its first tile (its wait runs out)
  // optional fused final layer (N = 16 only): z[b][y][x] = out_scale[b] (wf^T a + bf) on the physical
  // Nx x Ny grid instead of storing the activation a
  const float* wf;  // [16][2] weights, then the 2 biases
  const double* out_scale;
  float2* z;
  int Nx, Ny;
  int64_t zstride;
  const UnetIO* io;  // non-null: z and out_scale come from this block (CUDA graph replay)
};

template <int N, int NSL, int RY>
struct RowCfg {
  static constexpr int SLB = ((RY + 2) * ROW_PITCH + 127) / 128 * 128;  // one slice of a stage
  static constexpr int STAGE_BYTES = NSL * SLB;
  static constexpr int TX_BYTES = NSL * (RY + 2) * ROW_PITCH;
  static constexpr int W_BYTES = 9 * NSL * N * 16;
  static constexpr int FIXED = W_BYTES + N * 4 + 34 * 4 + 1024 + 256;
  // two CTAs per SM when two stages fit in half the shared memory, else one CTA with more stages
  static constexpr int BUDGET = (FIXED + 2 * STAGE_BYTES <= 112 * 1024) ? 112 * 1024 : 200 * 1024;
  static constexpr int STAGES_RAW = (BUDGET - FIXED) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 4 ? 4 : (STAGES_RAW < 2 ? 2 : STAGES_RAW);
  static constexpr int ACC_COLS = RY * N;  // one accumulator: RY rows x N channels
  static constexpr int TMEM_COLS = 2 * ACC_COLS < 32 ? 32 : 2 * ACC_COLS;
  static constexpr int SMEM = STAGES * STAGE_BYTES + FIXED;
  static constexpr int THREADS = 320;  // producer, MMA issuer, two 4-warp epilogue groups
  static constexpr int MINB = 2 * (SMEM + 1024) <= 228 * 1024 ? 2 : 1;  // CTAs per SM the registers allow
  static_assert((TMEM_COLS & (TMEM_COLS - 1)) == 0 && TMEM_COLS <= 512, "TMEM allocation");
  static_assert(SLB < (1 << 18), "LBO field");
};

template <int N, int NSL, int RY>
__global__ void __launch_bounds__(320, RowCfg<N, NSL, RY>::MINB) k_conv_row(const __grid_constant__ CUtensorMap tA0,
                                                     const __grid_constant__ CUtensorMap tA1, RowArgs a) {
  using Cfg = RowCfg<N, NSL, RY>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* wsm = smem + Cfg::STAGES * Cfg::STAGE_BYTES;  // resident weights
  float* bsm = (float*)(wsm + Cfg::W_BYTES);
  float* fsm = bsm + N;  // fused final layer: 32 weights + 2 biases
  uint64_t* full = (uint64_t*)(((uintptr_t)(fsm + 34) + 7) & ~(uintptr_t)7);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdrain = tempty + 2;  // completion of the MMAs in flight when the pipeline gives up
  uint32_t* tmem_slot = (uint32_t*)(mdrain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_img = a.tiles_x * a.tiles_y;

  // weights and bias into shared memory (generic proxy), made visible to the tensor core below
  for (int i = threadIdx.x; i < Cfg::W_BYTES / 16; i += Cfg::THREADS)
    ((uint4*)wsm)[i] = ((const uint4*)a.wrow)[i];
  for (int i = threadIdx.x; i < N; i += Cfg::THREADS) bsm[i] = a.bias[i];
  if (a.z || a.io)
    for (int i = threadIdx.x; i < 34; i += Cfg::THREADS) fsm[i] = a.wf[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&tfull[k], 1);
      mbar_init(&tempty[k], 128);
    }
    mbar_init(mdrain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: one (RY + 2)-row box of the 130-pixel halo per slice per tile
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int fills[Cfg::STAGES];  // loads issued into each stage (the drain waits for the last one)
#pragma unroll
      for (int s = 0; s < Cfg::STAGES; ++s) fills[s] = 0;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int b = t / per_img;
        int r = t % per_img;
        int y0 = (r / a.tiles_x) * RY, x0 = (r % a.tiles_x) * ROW_PX;
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, 11, a.budget)) {
          ok = false;
          break;
        }
        if (a.skip_first && blockIdx.x == 0 && t == 0) {  // injected fault: this tile never arrives
          if (++stage == Cfg::STAGES) {
            stage = 0;
            phase ^= 1;
          }
          continue;
        }
        ++fills[stage];
        unsigned char* sa = smem + stage * Cfg::STAGE_BYTES;
        mbar_expect_tx(&full[stage], Cfg::TX_BYTES);
#pragma unroll
        for (int s = 0; s < NSL; ++s) {
          const bool first = s < a.nsl0;
          tma_load_4d(sa + s * Cfg::SLB, first ? &tA0 : &tA1, &full[stage], (first ? s : s - a.nsl0) * 8, x0 - 1,
                      y0 - 1, b);
        }
        if (++stage == Cfg::STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      // every load issued must land before the CTA releases its shared memory
#pragma unroll
      for (int s = 0; s < Cfg::STAGES; ++s) mbar_drain(&full[s], fills[s]);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: RY rows x 9 taps x NSL/2 MMAs (K = 16 = two slices) per tile
    constexpr uint32_t IDESC = idesc_bf16(128, N);
    const uint32_t wbase = smem_u32(wsm);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      if (!mbar_wait_warp(&tempty[acc], acc_phase ^ 1, abort_flag, a.err, 12, a.budget) ||
          !mbar_wait_warp(&full[stage], phase, abort_flag, a.err, 13, a.budget)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (lane == 0) {
        const uint32_t sa = smem_u32(smem + stage * Cfg::STAGE_BYTES);
        // rows innermost: consecutive MMAs go to different accumulators, so none waits for the
        // previous one's result
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int kk = 0; kk < NSL / 2; ++kk) {
              const int tap = ky * 3 + dx;
              const uint64_t bd = smem_desc_noswz(wbase + ((tap * NSL + 2 * kk) * N) * 16, N * 16, 128);
#pragma unroll
              for (int ry = 0; ry < RY; ++ry) {
                const uint32_t d_tmem = tmem_base + acc * Cfg::ACC_COLS + ry * N;
                const uint64_t ad =
                    smem_desc_noswz(sa + 2 * kk * Cfg::SLB + (ry + ky) * ROW_PITCH + dx * 16, Cfg::SLB, 128);
                umma_bf16(d_tmem, ad, bd, IDESC, (ky | dx | kk) ? 1u : 0u);
              }
            }
        umma_commit(&empty[stage]);
        umma_commit(&tfull[acc]);
      }
      __syncwarp();
      if (++stage == Cfg::STAGES) {
        stage = 0;
        phase ^= 1;
      }
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
    if (!ok) {
      // the MMAs already issued must complete before TMEM is released
      if (lane == 0) {
        umma_commit(mdrain);
        mbar_drain(mdrain, 1);
      }
      __syncwarp();
    }
  } else {
    // ---------------- epilogue: group e = 0 (warps 2..5) drains accumulator 0 (the CTA's even tiles),
    // e = 1 (warps 6..9) accumulator 1 (the odd ones); TMEM lane = pixel of the row segment
    const int e = (warp - 2) >> 2;
    const int q = warp & 3;
    const int p = q * 32 + lane;
    // fused output layer: this call's output pointer and scales (from the block under graph replay)
    const bool fused_out = N == 16 && (a.z != nullptr || a.io != nullptr);
    float2* const zp = a.io ? (float2*)a.io->z : a.z;
    const double* const osc = a.io ? a.io->out_scale : a.out_scale;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x + e * gridDim.x; t < a.ntiles; t += 2 * gridDim.x) {
      if (!mbar_wait_warp(&tfull[e], acc_phase, abort_flag, a.err, 14, a.budget)) break;
      tc_fence_after();
      int b = t / per_img;
      int r = t % per_img;
      int y0 = (r / a.tiles_x) * RY, x = (r % a.tiles_x) * ROW_PX + p;
      const bool inside = x < a.W;
      // the tile's RY x N accumulator columns in batches of up to four 16-column TMEM loads with
      // one wait per batch
      constexpr int NLD = Cfg::ACC_COLS / 16;
      constexpr int LB = NLD < ROW_EPI_BATCH ? NLD : ROW_EPI_BATCH;
#pragma unroll
      for (int l0 = 0; l0 < NLD; l0 += LB) {
        uint32_t v[LB][16];
#pragma unroll
        for (int l = 0; l < LB; ++l)
          tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + e * Cfg::ACC_COLS + (l0 + l) * 16, v[l]);
        tmem_ld_wait();
#pragma unroll
        for (int l = 0; l < LB; ++l) {
          const int ry = ((l0 + l) * 16) / N, cb = (((l0 + l) * 16) % N) / 16;
          const int y = y0 + ry;
          if (!inside || y >= a.H) continue;
          __align__(16) __nv_bfloat16 hv[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            float f = __uint_as_float(v[l][k]) + bsm[cb * 16 + k];
            if (a.relu) f = fmaxf(f, 0.0f);
            hv[k] = __float2bfloat16_rn(f);
          }
          if (fused_out) {
            // final 1x1 conv 16 -> 2 on the BF16 activation, then the output scale and crop
            float f0 = fsm[32], f1 = fsm[33];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const float f = __bfloat162float(hv[k]);
              f0 += f * fsm[2 * k];
              f1 += f * fsm[2 * k + 1];
            }
            if (x < a.Nx && y < a.Ny) {
              const double sc = osc ? osc[b] : 1.0;
              zp[b * a.zstride + (int64_t)y * a.Nx + x] = make_float2((float)(f0 * sc), (float)(f1 * sc));
            }
          } else {
            uint4* dst = (uint4*)(a.out + (((int64_t)b * a.H + y) * a.W + x) * N + cb * 16);
            dst[0] = ((const uint4*)hv)[0];
            dst[1] = ((const uint4*)hv)[1];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[e]);
      acc_phase ^= 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
}

// Row-kernel weights: [tap][slice][n][8] BF16 from the master layout [cout][cin][3][3]; channels
// beyond C_in (first layer: 3 used of 16) are zero.
__global__ void k_prep_row(const double* __restrict__ master, int64_t m_w, int cin, int cin_pad, int cout,
                           __nv_bfloat16* __restrict__ w) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int nsl = cin_pad / 8;
  int64_t total = (int64_t)9 * nsl * cout * 8;
  if (q >= total) return;
  int c8 = (int)(q % 8);
  int n = (int)((q / 8) % cout);
  int s = (int)((q / (8 * cout)) % nsl);
  int tap = (int)(q / ((int64_t)8 * cout * nsl));
  int ci = s * 8 + c8;
  double v = ci < cin ? master[m_w + ((int64_t)(n * cin + ci) * 3 + tap / 3) * 3 + tap % 3] : 0.0;
  w[q] = __float2bfloat16_rn((float)v);
}

typedef CUresult (*EncodeTiledFnR)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 8-channel, 130-pixel, `rows`-row non-swizzled boxes over an NHWC BF16 tensor with C channels.
static helm_status row_map(CUtensorMap* m, const void* ptr, int C, int B, int H, int W, int rows) {
  static EncodeTiledFnR fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFnR)p;
  });
  if (!fn) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  cuuint32_t box[4] = {8, (cuuint32_t)ROW_HALO, (cuuint32_t)rows, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (row boxes) failed: " + std::to_string((int)r));
  return HELM_OK;
}

template <int N, int NSL, int RY>
static helm_status launch_row(const void* in0, int C0, const void* in1, int C1, RowArgs args, cudaStream_t st) {
  using Cfg = RowCfg<N, NSL, RY>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int per_sm = 1, nsm = 148;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_conv_row<N, NSL, RY>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_conv_row<N, NSL, RY>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int by_regs = 8;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_conv_row<N, NSL, RY>) == cudaSuccess && fa.numRegs > 0)
      by_regs = 65536 / (((fa.numRegs + 7) / 8) * 8 * Cfg::THREADS);
    per_sm = std::min(std::min(smem_sm / (Cfg::SMEM + 1024), 512 / Cfg::TMEM_COLS),
                      std::min(2048 / Cfg::THREADS, by_regs));
    per_sm = std::max(1, per_sm);
  });
  HELM_CK(attr_err);
  CUtensorMap a0, a1;
  HELM_TRY(row_map(&a0, in0, C0, args.B, args.H, args.W, RY + 2));
  if (C1 > 0)
    HELM_TRY(row_map(&a1, in1, C1, args.B, args.H, args.W, RY + 2));
  else
    a1 = a0;
  args.tiles_y = (args.H + RY - 1) / RY;
  args.ntiles = args.B * args.tiles_y * args.tiles_x;
  if (args.ntiles == 0) return HELM_OK;
  int grid = std::min(args.ntiles, nsm * per_sm);
  launch(k_conv_row<N, NSL, RY>, grid, Cfg::THREADS, Cfg::SMEM, st, a0, a1, args);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

bool conv_row_supported(int cin_total, int cout) {
  int nsl = cin_total / 8;
  return (cout == 16 && (nsl == 2 || nsl == 4)) || (cout == 32 && (nsl == 2 || nsl == 4 || nsl == 8)) ||
         (cout == 64 && nsl == 4);
}

helm_status conv_row_prepare(const double* master, int64_t m_w, int cin, int cin_pad, int cout, __nv_bfloat16** w,
                             cudaStream_t st) {
  size_t n = (size_t)9 * cin_pad * cout;
  if (!*w) HELM_CK(cudaMalloc(w, sizeof(__nv_bfloat16) * n));
  launch(k_prep_row, cdiv(n, 256), 256, 0, st, master, m_w, cin, cin_pad, cout, *w);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

// ------------------------------------------------------------------ autotuner
//
// The rows per tile (RY) trade halo re-reads (RY + 2 loaded rows per RY output rows) against
// pipeline depth and CTAs per SM (shared memory, TMEM columns).  On the first call for a layer
// shape (C_out, slices, B, H, W) every candidate runs once untimed (one-time set-up) and once timed
// with CUDA events on the caller's stream; the fastest is kept for that shape.  All candidates
// produce bit-identical outputs (same MMA order per output pixel), so tuning does not perturb
// results.  HELM_AUTOTUNE=0 keeps the first candidate; calls during a CUDA-graph capture use the
// cached choice or the first candidate.

typedef helm_status (*RowLaunchFn)(const void*, int, const void*, int, RowArgs, cudaStream_t);
struct RowCand {
  int ry;
  RowLaunchFn fn;
};
struct RowKey {
  int cout, nsl, B, H, W;
  bool operator<(const RowKey& o) const {
    return std::tie(cout, nsl, B, H, W) < std::tie(o.cout, o.nsl, o.B, o.H, o.W);
  }
};

static const std::vector<RowCand>& row_candidates(int cout, int nsl) {
  static const std::vector<RowCand> none;
  static const std::vector<RowCand> c1602 = {
      {4, launch_row<16, 2, 4>}, {2, launch_row<16, 2, 2>}, {8, launch_row<16, 2, 8>}};
  static const std::vector<RowCand> c1604 = {{4, launch_row<16, 4, 4>}, {2, launch_row<16, 4, 2>}};
  static const std::vector<RowCand> c3202 = {{4, launch_row<32, 2, 4>}, {2, launch_row<32, 2, 2>}};
  static const std::vector<RowCand> c3204 = {{2, launch_row<32, 4, 2>}, {4, launch_row<32, 4, 4>}};
  static const std::vector<RowCand> c3208 = {{2, launch_row<32, 8, 2>}, {1, launch_row<32, 8, 1>}};
  static const std::vector<RowCand> c6404 = {{2, launch_row<64, 4, 2>}, {4, launch_row<64, 4, 4>}};
  switch (cout * 100 + nsl) {
    case 1602: return c1602;
    case 1604: return c1604;
    case 3202: return c3202;
    case 3204: return c3204;
    case 3208: return c3208;
    case 6404: return c6404;
    default: return none;
  }
}

static bool autotune_enabled() {
  static const bool on = [] {
    const char* e = getenv("HELM_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}

static std::mutex g_row_mu;
static std::map<RowKey, int> g_row_choice;  // index into the candidate list

static helm_status row_autotuned(const std::vector<RowCand>& cands, const RowKey& key, const void* in0, int C0,
                                 const void* in1, int C1, const RowArgs& a, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lk(g_row_mu);
    auto it = g_row_choice.find(key);
    if (it != g_row_choice.end()) return cands[it->second].fn(in0, C0, in1, C1, a, st);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HELM_CK(cudaStreamIsCapturing(st, &cap));
  if (!autotune_enabled() || cands.size() == 1 || cap != cudaStreamCaptureStatusNone)
    return cands[0].fn(in0, C0, in1, C1, a, st);
  cudaEvent_t e0, e1;
  HELM_CK(cudaEventCreate(&e0));
  HELM_CK(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  helm_status rc = HELM_OK;
  for (size_t i = 0; i < cands.size() && rc == HELM_OK; ++i) {
    rc = cands[i].fn(in0, C0, in1, C1, a, st);  // one-time set-up and warm-up
    if (rc != HELM_OK) break;
    cudaEventRecord(e0, st);
    rc = cands[i].fn(in0, C0, in1, C1, a, st);
    cudaEventRecord(e1, st);
    if (rc != HELM_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        (i == 0 || ms < best_ms)) {
      best = (int)i;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HELM_OK) return rc;
  std::lock_guard<std::mutex> lk(g_row_mu);
  g_row_choice[key] = best;
  return HELM_OK;
}

// Rows per tile chosen for each tuned layer shape so far: out[k] = {cout, slices, B, H, W, RY}.
int conv_row_tuned(int (*out)[6], int max) {
  std::lock_guard<std::mutex> lk(g_row_mu);
  int k = 0;
  for (auto& kv : g_row_choice) {
    if (k >= max) break;
    const RowKey& r = kv.first;
    out[k][0] = r.cout;
    out[k][1] = r.nsl;
    out[k][2] = r.B;
    out[k][3] = r.H;
    out[k][4] = r.W;
    out[k][5] = row_candidates(r.cout, r.nsl)[kv.second].ry;
    ++k;
  }
  return k;
}

helm_status conv_row_forward(const __nv_bfloat16* wrow, const float* bias, int* err, const void* in0, int C0,
                             const void* in1, int C1, void* out, int cout, int B, int H, int W, cudaStream_t st,
                             const RowFinal* fin, int variant, int* ry_out) {
  if (fin && !(cout == 16 && C0 + C1 == 16))
    return fail(HELM_ERR_INVALID_ARG, "conv_row_forward: the fused final layer needs a 16 -> 16 convolution");
  RowArgs a;
  a.wf = fin ? fin->wf : nullptr;
  a.out_scale = fin ? fin->out_scale : nullptr;
  a.z = fin ? fin->z : nullptr;
  a.Nx = fin ? fin->Nx : 0;
  a.Ny = fin ? fin->Ny : 0;
  a.zstride = fin ? fin->zstride : 0;
  a.io = fin ? fin->io : nullptr;
  a.B = B;
  a.H = H;
  a.W = W;
  a.nsl0 = C0 / 8;
  a.tiles_x = (W + ROW_PX - 1) / ROW_PX;
  a.tiles_y = 0;
  a.ntiles = 0;
  a.wrow = wrow;
  a.bias = bias;
  a.out = (__nv_bfloat16*)out;
  a.relu = 1;
  a.err = err;
  a.budget = wait_budget();
  a.skip_first = take_fault(HELM_FAULT_CONV_TILE) ? 1 : 0;
  const int nsl = (C0 + C1) / 8;
  const std::vector<RowCand>& cands = row_candidates(cout, nsl);
  if (cands.empty()) return fail(HELM_ERR_INVALID_ARG, "conv_row_forward: unsupported layer shape");
  if (variant > 0) {  // one fixed rows-per-tile variant (per-layer tests)
    if (variant > (int)cands.size())
      return fail(HELM_ERR_INVALID_ARG, "conv_row_forward: the layer has only " + std::to_string(cands.size()) +
                                            " rows-per-tile variants");
    if (ry_out) *ry_out = cands[variant - 1].ry;
    return cands[variant - 1].fn(in0, C0, in1, C1, a, st);
  }
  const RowKey key{cout, nsl, B, H, W};
  HELM_TRY(row_autotuned(cands, key, in0, C0, in1, C1, a, st));
  if (ry_out) {
    std::lock_guard<std::mutex> lk(g_row_mu);
    auto it = g_row_choice.find(key);
    *ry_out = cands[it != g_row_choice.end() ? it->second : 0].ry;
  }
  return HELM_OK;
}

}  // namespace helm

extern "C" int helm_tuned_tiles(int* out, int max_entries) {
  if (!out || max_entries <= 0) return 0;
  return helm::conv_row_tuned(reinterpret_cast<int (*)[6]>(out), max_entries);
}
