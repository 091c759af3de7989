// Row-tile tcgen05 3x3 convolutions for the narrow layers (C_in <= 64 in 8-channel slices, C_out <= 64).
//
// The full-resolution 16- and 32-channel layers move little data per pixel, so the cost of the
// 9-box tile pipeline in conv_tc.cu (one TMA box per tap) dominates there.  Here one tile is a
// 128-pixel segment of one image row.  For each of the three kernel rows and each 8-channel slice,
// one TMA box brings the 130-pixel halo segment (16 bytes per pixel) into shared memory in the
// non-swizzled K-major core-matrix layout (8 pixels x 16 bytes contiguous).  The three horizontal
// taps of that kernel row are then the same buffer read at pixel offsets 0, 1, 2, i.e. descriptor
// start addresses 16 bytes apart, so a tile needs 3 x slices loads instead of 9 x chunks.  The
// weights of the layer stay resident in shared memory for the whole persistent kernel.
// Warp roles, TMEM double buffering, bounded waits and the epilogue follow conv_tc.cu.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "tc_ptx.cuh"
#include "unet.cuh"

namespace helm {

constexpr int ROW_PX = 128;           // output pixels per tile (one MMA block, M = 128)
constexpr int ROW_HALO = ROW_PX + 2;  // loaded pixels per kernel row
constexpr int ROWB = 2176;            // bytes per (kernel row, slice) buffer: 130 x 16 B rounded up to 128 B

struct RowArgs {
  int B, H, W;
  int nsl0;  // 8-channel slices from source 0 (the rest from source 1)
  int tiles_x;
  int ntiles;
  const __nv_bfloat16* wrow;  // [tap][slice][N][8]
  const float* bias;
  __nv_bfloat16* out;  // NHWC [B][H][W][N]
  int relu;
  int* err;
};

template <int N, int NSL>
struct RowCfg {
  static constexpr int STAGE_BYTES = 3 * NSL * ROWB;
  static constexpr int W_BYTES = 9 * NSL * N * 16;
  static constexpr int STAGES_RAW = (100 * 1024 - W_BYTES) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 4 ? 4 : (STAGES_RAW < 2 ? 2 : STAGES_RAW);
  static constexpr int NACC = 4;  // TMEM accumulators: the MMA warp runs up to 4 tiles ahead
  static constexpr int TMEM_COLS = NACC * N < 32 ? 32 : NACC * N;
  static constexpr int SMEM = STAGES * STAGE_BYTES + W_BYTES + N * 4 + 1024 + 256;
  static constexpr int THREADS = 320;  // producer, MMA issuer, two 4-warp epilogue groups
};

template <int N, int NSL>
__global__ void __launch_bounds__(320, 1) k_conv_row(const __grid_constant__ CUtensorMap tA0,
                                                     const __grid_constant__ CUtensorMap tA1, RowArgs a) {
  using Cfg = RowCfg<N, NSL>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* wsm = smem + Cfg::STAGES * Cfg::STAGE_BYTES;  // resident weights
  float* bsm = (float*)(wsm + Cfg::W_BYTES);
  uint64_t* full = (uint64_t*)(bsm + N + (N & 1));
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + Cfg::NACC;
  uint32_t* tmem_slot = (uint32_t*)(tempty + Cfg::NACC);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // weights and bias into shared memory (generic proxy), made visible to the tensor core below
  for (int i = threadIdx.x; i < Cfg::W_BYTES / 16; i += Cfg::THREADS)
    ((uint4*)wsm)[i] = ((const uint4*)a.wrow)[i];
  for (int i = threadIdx.x; i < N; i += Cfg::THREADS) bsm[i] = a.bias[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < Cfg::NACC; ++k) {
      mbar_init(&tfull[k], 1);
      mbar_init(&tempty[k], 128);
    }
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
      // ---------------- TMA producer: 3 kernel rows x NSL slices of the 130-pixel halo per tile
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int b = t / (a.tiles_x * a.H);
        int r = t % (a.tiles_x * a.H);
        int y = r / a.tiles_x, x0 = (r % a.tiles_x) * ROW_PX;
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, 11)) {
          ok = false;
          break;
        }
        unsigned char* sa = smem + stage * Cfg::STAGE_BYTES;
        mbar_expect_tx(&full[stage], 3 * NSL * ROW_HALO * 16);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int s = 0; s < NSL; ++s) {
            const bool first = s < a.nsl0;
            tma_load_4d(sa + (ky * NSL + s) * ROWB, first ? &tA0 : &tA1, &full[stage], (first ? s : s - a.nsl0) * 8,
                        x0 - 1, y + ky - 1, b);
          }
        if (++stage == Cfg::STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
          long long t0 = clock64();
          while (!mbar_try_wait(&full[s], 0) && !mbar_try_wait(&full[s], 1) && clock64() - t0 < WAIT_CYCLES) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: 9 taps x NSL/2 MMAs (K = 16 = two slices) per tile
    constexpr uint32_t IDESC = idesc_bf16(128, N);
    const uint32_t wbase = smem_u32(wsm);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      if (!mbar_wait(&tempty[acc], acc_phase ^ 1, abort_flag, a.err, 12)) break;
      tc_fence_after();
      if (!mbar_wait(&full[stage], phase, abort_flag, a.err, 13)) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + acc * N;
      if (lane == 0) {
        const uint32_t sa = smem_u32(smem + stage * Cfg::STAGE_BYTES);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int kk = 0; kk < NSL / 2; ++kk) {
              const int tap = ky * 3 + dx;
              uint64_t ad = smem_desc_noswz(sa + (ky * NSL + 2 * kk) * ROWB + dx * 16, ROWB, 128);
              uint64_t bd = smem_desc_noswz(wbase + ((tap * NSL + 2 * kk) * N) * 16, N * 16, 128);
              umma_bf16(d_tmem, ad, bd, IDESC, (ky | dx | kk) ? 1u : 0u);
            }
        umma_commit(&empty[stage]);
        umma_commit(&tfull[acc]);
      }
      __syncwarp();
      if (++stage == Cfg::STAGES) {
        stage = 0;
        phase ^= 1;
      }
      if (++acc == Cfg::NACC) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  } else {
    // ---------------- epilogue: group e = 0 (warps 2..5) takes the CTA's even tiles, e = 1 (warps
    // 6..9) the odd ones; TMEM lane = pixel of the row segment, accumulator = tile index mod 4
    const int e = (warp - 2) >> 2;
    const int q = warp & 3;
    const int p = q * 32 + lane;
    int acc = e;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x + e * gridDim.x; t < a.ntiles; t += 2 * gridDim.x) {
      if (!mbar_wait(&tfull[acc], acc_phase, abort_flag, a.err, 14)) break;
      tc_fence_after();
      int b = t / (a.tiles_x * a.H);
      int r = t % (a.tiles_x * a.H);
      int y = r / a.tiles_x, x = (r % a.tiles_x) * ROW_PX + p;
      const bool inside = x < a.W;
      __nv_bfloat16* o = a.out + (((int64_t)b * a.H + y) * a.W + x) * N;
#pragma unroll
      for (int cb = 0; cb < N / 16; ++cb) {
        uint32_t v[16];
        tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + acc * N + cb * 16, v);
        tmem_ld_wait();
        if (inside) {
          __align__(16) __nv_bfloat16 hv[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            float f = __uint_as_float(v[k]) + bsm[cb * 16 + k];
            if (a.relu) f = fmaxf(f, 0.0f);
            hv[k] = __float2bfloat16_rn(f);
          }
          uint4* dst = (uint4*)(o + cb * 16);
          dst[0] = ((const uint4*)hv)[0];
          dst[1] = ((const uint4*)hv)[1];
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      acc += 2;
      if (acc >= Cfg::NACC) {
        acc -= Cfg::NACC;
        acc_phase ^= 1;
      }
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

// 8-channel, 130-pixel, non-swizzled boxes over an NHWC BF16 tensor with C channels.
static helm_status row_map(CUtensorMap* m, const void* ptr, int C, int B, int H, int W) {
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
  cuuint32_t box[4] = {8, (cuuint32_t)ROW_HALO, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (row boxes) failed: " + std::to_string((int)r));
  return HELM_OK;
}

template <int N, int NSL>
static helm_status launch_row(const CUtensorMap& a0, const CUtensorMap& a1, const RowArgs& args, cudaStream_t st) {
  using Cfg = RowCfg<N, NSL>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int per_sm = 1, nsm = 148;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_conv_row<N, NSL>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_conv_row<N, NSL>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int by_regs = 8;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_conv_row<N, NSL>) == cudaSuccess && fa.numRegs > 0)
      by_regs = 65536 / (((fa.numRegs + 7) / 8) * 8 * Cfg::THREADS);
    per_sm = std::min(std::min(smem_sm / (Cfg::SMEM + 1024), 512 / Cfg::TMEM_COLS),
                      std::min(2048 / Cfg::THREADS, by_regs));
    per_sm = std::max(1, per_sm);
    per_sm = std::max(1, per_sm);
  });
  HELM_CK(attr_err);
  int grid = std::min(args.ntiles, nsm * per_sm);
  launch(k_conv_row<N, NSL>, grid, Cfg::THREADS, Cfg::SMEM, st, a0, a1, args);
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

helm_status conv_row_forward(const __nv_bfloat16* wrow, const float* bias, int* err, const void* in0, int C0,
                             const void* in1, int C1, void* out, int cout, int B, int H, int W, cudaStream_t st) {
  CUtensorMap m0, m1;
  HELM_TRY(row_map(&m0, in0, C0, B, H, W));
  if (C1 > 0)
    HELM_TRY(row_map(&m1, in1, C1, B, H, W));
  else
    m1 = m0;
  RowArgs a;
  a.B = B;
  a.H = H;
  a.W = W;
  a.nsl0 = C0 / 8;
  a.tiles_x = (W + ROW_PX - 1) / ROW_PX;
  a.ntiles = B * H * a.tiles_x;
  a.wrow = wrow;
  a.bias = bias;
  a.out = (__nv_bfloat16*)out;
  a.relu = 1;
  a.err = err;
  const int nsl = (C0 + C1) / 8;
  switch (cout * 100 + nsl) {
    case 1602: return launch_row<16, 2>(m0, m1, a, st);
    case 1604: return launch_row<16, 4>(m0, m1, a, st);
    case 3202: return launch_row<32, 2>(m0, m1, a, st);
    case 3204: return launch_row<32, 4>(m0, m1, a, st);
    case 3208: return launch_row<32, 8>(m0, m1, a, st);
    case 6404: return launch_row<64, 4>(m0, m1, a, st);
    default: return fail(HELM_ERR_INVALID_ARG, "conv_row_forward: unsupported layer shape");
  }
}

}  // namespace helm
