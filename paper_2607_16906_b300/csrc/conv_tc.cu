// tcgen05 implicit-GEMM 3x3 convolutions (BF16 operands, FP32 accumulation in TMEM), sm_103a.
//
// GEMM view of one conv layer: D[pixel][co] = bias + sum_{chunk, tap} A_tap[pixel][ci] W[tap][ci][co],
// M = 128 output pixels (an 8 x 16 patch of one image), N = C_out (16..128), K = 9 taps x C_in.
// For each (input-channel chunk, tap) one TMA load brings the 8 x 16 patch shifted by the tap
// (out-of-image rows/columns arrive as zeros, which is the conv's zero padding) and one TMA load
// brings the tap's N x chunk weight tile; both land in shared memory in the swizzled K-major layout
// that tcgen05.mma reads directly.  A concat input (decoder levels) is two sources whose chunks are
// consumed one after the other, so the concat is never materialised.  The same kernel runs network
// kind 1 (unet_paper.cu): its 5x5 layers with row-reuse stages (TcCfg, KS = 5) and its first three
// encoder layers as 3x3 convolutions of a strided phase view of their input (MODE 2, ConvTcArgs::qf).
//
// Persistent kernel, one CTA per SM slot, 6 warps:
//   warp 0  TMA producer (one elected lane), STAGES-deep smem ring (full/empty mbarriers);
//   warp 1  TMEM allocator and MMA issuer (one lane issues tcgen05.mma, commits free the stage);
//   warps 2-5  epilogue: tcgen05.ld of the 128 x N accumulator (warp w reads TMEM lanes
//           32 (w % 4) .. +31), bias, ReLU, BF16 rounding, NHWC stores.
// Two TMEM accumulators alternate so the epilogue of one tile overlaps the MMAs of the next.
// Every mbarrier wait is bounded (a run-time budget of clock64 cycles, ConvTcArgs::budget, about one
// second by default; the drain waits always the full second); on a timeout the kernel records an
// error code, stops issuing work, waits (bounded) for its own copies in flight, frees TMEM and exits.
#include <cuda.h>

#include <atomic>
#include <cstdlib>
#include <mutex>

#include "tc_ptx.cuh"
#include "unet.cuh"

namespace helm {

// ------------------------------------------------------------------ kernel

struct ConvTcArgs {
  int B, H, W;            // GEMM pixel grid: the output grid (3x3 conv) or the input grid (2x2 up-conv)
  int nk0, nk1;           // input-channel chunks from source 0 / source 1
  int tiles_x, tiles_y;   // 16-wide, 8-high pixel tiles
  int ntiles;
  const float* bias;      // [N]
  __nv_bfloat16* out;     // NHWC [B][H][W][N]
  int act;               // 0 none, 1 ReLU, 2 PReLU with `slope`
  float slope;
  int* err;               // device error code (0 = ok)
  long long budget;       // clock64 cycles a pipeline wait may take before the kernel gives up
  int skip_first;         // failure injection: CTA 0 issues no loads for its first tile
  // MODE 0: source 0 is an NHWC tensor of the 2H x 2W grid read as its space-to-depth view (channel
  // chunk kc = input row phase; the map's rows are traversed with stride 2)
  int s2d;
  // MODE 2, KS = 3: source 0 is an NHWC tensor [B][qf H][qf W][32] read as its phase view (qf = 2 or 4):
  // chunk kc of GEMM pixel (y, x) is the source pixel (qf y + kc / qf, qf x + kc % qf); the map's rows
  // and columns are traversed with stride qf.  0: no phase view
  int qf;
  // optional, per image: an image whose scale is 0 (a converged column of the solver, whose network
  // input scale is zero) is skipped by every role; with the fused output layer its output is zeroed
  const double* img_scale;
  // optional (training): the BF16 pre-activation is stored here too, at the output's index
  __nv_bfloat16* pre_out;
  // MODE 2 only, optional: the network's 1x1 output layer C_out -> 2 fused into the epilogue:
  // z[b][Y][X] = out_scale[b] (wf^T a + bf) for the output pixels inside the physical Nx x Ny grid, no
  // activation stored
  const float* wf;        // [C_out][2] weights, then the 2 biases
  const double* out_scale;  // per image; null: scale 1
  float2* z;
  int Nx, Ny;
  int64_t zstride;
};

template <int N, int CHUNK, int MODE, int KS, int RB = 1>
struct TcCfg {
  // KS = 5 (the reformulated stride-2 layers): a tile is RB row blocks of 8 x 16 pixels stacked
  // vertically (RB MMA accumulators of 128 x N); one stage is one (input-channel chunk, kernel
  // column dx): the (8 RB + 4)-row patch of the column-shifted window and the KS weight tiles of that
  // column.  The A operand of row block rb and kernel row dy is the same patch 16 (8 rb + dy) pixels
  // further on (a whole number of 8-row swizzle atoms), so every input pixel is loaded
  // (8 RB + 4) / (8 RB) times per chunk instead of 25 times, and every weight tile serves RB blocks.
  // KS = 3, MODE 2 (the stride-2 layers read through a phase view): the same row reuse with a
  // (8 RB + 2)-row patch and 3 weight tiles per stage.
  // KS = 3 otherwise: one stage is one or three taps, each with its own patch and weight tile (RB = 1).
  static constexpr bool RR = KS == 5 || (KS == 3 && MODE == 2);
  static_assert(RR || RB == 1, "row blocks need the row-reuse stages");
  static constexpr int A_ROWS = RR ? 8 * RB + KS - 1 : 8;
  static constexpr int A_BYTES = A_ROWS * 16 * CHUNK * 2;
  static constexpr int B_BYTES = N * CHUNK * 2;
  // taps per pipeline stage: a whole kernel row (3 taps) for narrow chunks, so that one barrier
  // round trip carries three MMAs; one tap otherwise
  static constexpr int TPS = RR ? KS : ((MODE == 0 && KS == 3 && CHUNK <= 32) ? 3 : 1);
  static constexpr int STAGE_BYTES = RR ? A_BYTES + KS * B_BYTES : TPS * (A_BYTES + B_BYTES);
  // shared memory for the stage ring: the phase-view layers (many small stages per tile) take one
  // stage more than 200 KB would give
  static constexpr int BUDGET = RR ? (KS == 3 ? 220 * 1024 : 200 * 1024) : 96 * 1024;
  static constexpr int STAGES = (BUDGET / STAGE_BYTES) > 8 ? 8 : (BUDGET / STAGE_BYTES);
  static constexpr int ACC_COLS = RB * N;  // one tile's accumulators
  static constexpr int TMEM_COLS = 2 * ACC_COLS < 32 ? 32 : 2 * ACC_COLS;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*alignment*/ + 256 /*barriers*/;
  static constexpr int THREADS = 192;
  static_assert(STAGES >= 2, "pipeline depth");
  static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM allocation");
  static_assert(!RR || (A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0), "swizzle-atom alignment of the stage buffers");
};

// MODE 0: KS x KS conv, pad KS / 2 (KS^2 shifted taps per channel chunk), N = C_out.
// MODE 2: the same taps with the MODE 1 epilogue (a stride-2 transposed conv written as a KS x KS conv
//         with N = 4 C_out followed by depth-to-space).
// MODE 1: 2x2 stride-2 transposed conv as one GEMM with N = 4 C_out (column n = tap C_out + co); the
//         epilogue scatters column blocks to output pixel (2y + tap / 2, 2x + tap % 2); no activation.
template <int N, int CHUNK, int MODE, int KS, int RB = 1>
__global__ void __launch_bounds__(192, 1) k_conv_tc(const __grid_constant__ CUtensorMap tA0,
                                                    const __grid_constant__ CUtensorMap tA1,
                                                    const __grid_constant__ CUtensorMap tW, ConvTcArgs a) {
  using Cfg = TcCfg<N, CHUNK, MODE, KS, RB>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdrain = tempty + 2;  // completion of the MMAs in flight when the pipeline gives up
  uint32_t* tmem_slot = (uint32_t*)(mdrain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = a.nk0 + a.nk1;
  constexpr int TAPS = MODE == 1 ? 1 : KS * KS;
  constexpr int TPS = Cfg::TPS;
  // stages per tile: KS = 5, one per (chunk, kernel column); otherwise one per (chunk, tap group)
  const int ksteps = (TAPS / TPS) * nk;

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
      // ---------------- TMA producer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int fills[Cfg::STAGES];  // loads issued into each stage (the drain waits for the last one)
#pragma unroll
      for (int s = 0; s < Cfg::STAGES; ++s) fills[s] = 0;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int b = t / (a.tiles_x * a.tiles_y);
        if (a.img_scale && a.img_scale[b] == 0.0) continue;
        int r = t % (a.tiles_x * a.tiles_y);
        int y0 = (r / a.tiles_x) * 8 * RB, x0 = (r % a.tiles_x) * 16;
        for (int kc = 0; kc < nk && ok; ++kc) {
          const CUtensorMap* src = kc < a.nk0 ? &tA0 : &tA1;
          int c0 = (kc < a.nk0 ? kc : kc - a.nk0) * CHUNK;
          for (int tg = 0; tg < TAPS / TPS; ++tg) {
            if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, 1, a.budget)) {
              ok = false;
              break;
            }
            if (a.skip_first && blockIdx.x == 0 && t == 0) {  // injected fault: these loads never arrive
              if (++stage == Cfg::STAGES) {
                stage = 0;
                phase ^= 1;
              }
              continue;
            }
            ++fills[stage];
            unsigned char* sa = smem + stage * Cfg::STAGE_BYTES;
            mbar_expect_tx(&full[stage], Cfg::STAGE_BYTES);
            if constexpr (Cfg::RR) {
              // kernel column dx = tg: the (8 + KS - 1)-row patch and the KS weight tiles (dy, dx)
              unsigned char* sb = sa + Cfg::A_BYTES;
              if (MODE == 2 && a.qf)
                tma_load_4d(sa, src, &full[stage], 0, a.qf * (x0 + tg - KS / 2) + kc % a.qf,
                            a.qf * (y0 - KS / 2) + kc / a.qf, b);
              else if (MODE == 0 && a.s2d)
                tma_load_4d(sa, src, &full[stage], 0, x0 + tg - KS / 2, 2 * (y0 - KS / 2) + kc, b);
              else
                tma_load_4d(sa, src, &full[stage], c0, x0 + tg - KS / 2, y0 - KS / 2, b);
#pragma unroll
              for (int dy = 0; dy < KS; ++dy)
                tma_load_3d(sb + dy * Cfg::B_BYTES, &tW, &full[stage], 0, 0, (dy * KS + tg) * nk + kc);
              if (++stage == Cfg::STAGES) {
                stage = 0;
                phase ^= 1;
              }
              continue;
            }
            unsigned char* sb = sa + TPS * Cfg::A_BYTES;
#pragma unroll
            for (int t = 0; t < TPS; ++t) {
              const int tap = tg * TPS + t;
              if (MODE == 0 && a.s2d)
                tma_load_4d(sa + t * Cfg::A_BYTES, src, &full[stage], 0, x0 + tap % KS - KS / 2,
                            2 * (y0 + tap / KS - KS / 2) + kc, b);
              else if (MODE != 1)
                tma_load_4d(sa + t * Cfg::A_BYTES, src, &full[stage], c0, x0 + tap % KS - KS / 2,
                            y0 + tap / KS - KS / 2, b);
              else
                tma_load_4d(sa + t * Cfg::A_BYTES, src, &full[stage], c0, x0, y0, b);
              tma_load_3d(sb + t * Cfg::B_BYTES, &tW, &full[stage], 0, 0, tap * nk + kc);
            }
            if (++stage == Cfg::STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      // every load issued must land before the CTA releases its shared memory
#pragma unroll
      for (int s = 0; s < Cfg::STAGES; ++s) mbar_drain(&full[s], fills[s]);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    constexpr uint32_t IDESC = idesc_bf16(128, N);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      if (a.img_scale && a.img_scale[t / (a.tiles_x * a.tiles_y)] == 0.0) continue;
      if (!mbar_wait_warp(&tempty[acc], acc_phase ^ 1, abort_flag, a.err, 2, a.budget)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + acc * Cfg::ACC_COLS;
      for (int ks = 0; ks < ksteps; ++ks) {
        if (!mbar_wait_warp(&full[stage], phase, abort_flag, a.err, 3, a.budget)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (lane == 0 && Cfg::RR) {
          // kernel rows dy of this column: A = the patch from pixel row dy, B = weight tile dy
          const uint32_t sa = smem_u32(smem + stage * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
          for (int dy = 0; dy < KS; ++dy) {
            const uint64_t bd = smem_desc(sb + dy * Cfg::B_BYTES, CHUNK * 2);
#pragma unroll
            for (int rb = 0; rb < RB; ++rb) {
              const uint64_t ad = smem_desc(sa + (8 * rb + dy) * 16 * CHUNK * 2, CHUNK * 2);
#pragma unroll
              for (int k = 0; k < CHUNK / 16; ++k)
                umma_bf16(d_tmem + rb * N, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), IDESC,
                          (ks > 0 || dy > 0 || k > 0) ? 1u : 0u);
            }
          }
          umma_commit(&empty[stage]);
        } else if (lane == 0) {
          uint32_t sa = smem_u32(smem + stage * Cfg::STAGE_BYTES);
          uint32_t sb = sa + TPS * Cfg::A_BYTES;
#pragma unroll
          for (int t = 0; t < TPS; ++t) {
            uint64_t ad = smem_desc(sa + t * Cfg::A_BYTES, CHUNK * 2), bd = smem_desc(sb + t * Cfg::B_BYTES, CHUNK * 2);
#pragma unroll
            for (int k = 0; k < CHUNK / 16; ++k)
              umma_bf16(d_tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), IDESC,
                        (ks > 0 || t > 0 || k > 0) ? 1u : 0u);
          }
          umma_commit(&empty[stage]);
        }
        __syncwarp();
        if (++stage == Cfg::STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      if (lane == 0) umma_commit(&tfull[acc]);
      __syncwarp();
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
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
    // ---------------- epilogue (warps 2..5)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int p = q * 32 + lane;  // pixel within the tile
    const int ly = p >> 4, lx = p & 15;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      int b = t / (a.tiles_x * a.tiles_y);
      int r = t % (a.tiles_x * a.tiles_y);
      constexpr int COUT = MODE == 0 ? N : N / 4;
      const bool fused = MODE == 2 && a.z != nullptr;
      if (a.img_scale && a.img_scale[b] == 0.0) {
        // skipped image: no accumulator was filled; the fused output layer writes its zeros
        if (fused)
          for (int rb = 0; rb < RB; ++rb) {
            const int y = (r / a.tiles_x) * 8 * RB + rb * 8 + ly, x = (r % a.tiles_x) * 16 + lx;
            if (y >= a.H || x >= a.W) continue;
            for (int qy = 0; qy < 2; ++qy) {
              const int Y = 2 * y + qy, X = 2 * x;
              if (Y >= a.Ny || X >= a.Nx) continue;
              float2* zp = a.z + b * a.zstride + (int64_t)Y * a.Nx + X;
              zp[0] = make_float2(0.0f, 0.0f);
              if (X + 1 < a.Nx) zp[1] = make_float2(0.0f, 0.0f);
            }
          }
        continue;
      }
      if (!mbar_wait_warp(&tfull[acc], acc_phase, abort_flag, a.err, 4, a.budget)) break;
      tc_fence_after();
#pragma unroll 1
      for (int rb = 0; rb < RB; ++rb) {
        const int y = (r / a.tiles_x) * 8 * RB + rb * 8 + ly, x = (r % a.tiles_x) * 16 + lx;
        const bool inside = y < a.H && x < a.W;
        float f0 = 0.0f, f1 = 0.0f;
        float2 zr[2];  // the fused output of phases (qy, 0) and (qy, 1): one 16-byte store per row
#pragma unroll
        for (int cb = 0; cb < N / 16; ++cb) {
          uint32_t v[16];
          tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + acc * Cfg::ACC_COLS + rb * N + cb * 16, v);
          tmem_ld_wait();
          if (fused && inside) {
            // the output layer on the BF16-rounded activation of output phase `tap`, channels in order
            const int tap = (cb * 16) / COUT, co0 = (cb * 16) % COUT;
            if (co0 == 0) {
              f0 = a.wf[2 * COUT];
              f1 = a.wf[2 * COUT + 1];
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              float f = __uint_as_float(v[k]) + a.bias[cb * 16 + k];
              f = f > 0.0f ? f : a.slope * f;
              const float h = __bfloat162float(__float2bfloat16_rn(f));
              f0 += h * a.wf[2 * (co0 + k)];
              f1 += h * a.wf[2 * (co0 + k) + 1];
            }
            if (co0 + 16 == COUT) {
              const double sc = a.out_scale ? a.out_scale[b] : 1.0;
              zr[tap & 1] = make_float2((float)(f0 * sc), (float)(f1 * sc));
              const int Y = 2 * y + tap / 2, X = 2 * x;
              if ((tap & 1) && Y < a.Ny && X < a.Nx) {
                float2* zp = a.z + b * a.zstride + (int64_t)Y * a.Nx + X;
                if (X + 1 < a.Nx && ((((uintptr_t)zp) & 15) == 0)) {
                  *(float4*)zp = make_float4(zr[0].x, zr[0].y, zr[1].x, zr[1].y);
                } else {
                  zp[0] = zr[0];
                  if (X + 1 < a.Nx) zp[1] = zr[1];
                }
              }
            }
          } else if (inside && !fused) {
            const int tap = (cb * 16) / COUT, co0 = (cb * 16) % COUT;
            int64_t opix = MODE == 0 ? (((int64_t)b * a.H + y) * a.W + x)
                                     : (((int64_t)b * 2 * a.H + 2 * y + tap / 2) * (2 * a.W) + 2 * x + tap % 2);
            __nv_bfloat16* o = a.out + opix * COUT + co0;
            __align__(16) __nv_bfloat16 hv[16];
            __align__(16) __nv_bfloat16 hp[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              float f = __uint_as_float(v[k]) + a.bias[co0 + k];
              hp[k] = __float2bfloat16_rn(f);
              if (a.act == 1) f = fmaxf(f, 0.0f);
              else if (a.act == 2) f = f > 0.0f ? f : a.slope * f;
              hv[k] = __float2bfloat16_rn(f);
            }
            uint4* dst = (uint4*)o;
            dst[0] = ((const uint4*)hv)[0];
            dst[1] = ((const uint4*)hv)[1];
            if (a.pre_out) {
              uint4* dp = (uint4*)(a.pre_out + opix * COUT + co0);
              dp[0] = ((const uint4*)hp)[0];
              dp[1] = ((const uint4*)hp)[1];
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
}

// Weights for the tcgen05 path: [tap][chunk][N][CHUNK] BF16 (K-major per tap and chunk); input
// channels beyond the layer's C_in (first layer: 3 used of 16) are zero.
__global__ void k_prep_tc(const double* __restrict__ master, int64_t m_w, int cin, int cin_pad, int cout, int chunk,
                          __nv_bfloat16* __restrict__ wtc) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)9 * cin_pad * cout;
  if (q >= total) return;
  int nk = cin_pad / chunk;
  int c = (int)(q % chunk);
  int n = (int)((q / chunk) % cout);
  int kc = (int)((q / ((int64_t)chunk * cout)) % nk);
  int tap = (int)(q / ((int64_t)chunk * cout * nk));
  int ci = kc * chunk + c;
  double w = ci < cin ? master[m_w + ((int64_t)(n * cin + ci) * 3 + tap / 3) * 3 + tap % 3] : 0.0;
  wtc[q] = __float2bfloat16_rn((float)w);
}

// Up-conv weights for the tcgen05 path: [chunk][n = tap * cout + co][CHUNK] BF16 from the master
// layout [cin][cout][2][2].
__global__ void k_prep_tc_up(const double* __restrict__ master, int64_t m_w, int cin, int cout, int chunk,
                             __nv_bfloat16* __restrict__ wtc) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)cin * 4 * cout;
  if (q >= total) return;
  int c = (int)(q % chunk);
  int n = (int)((q / chunk) % (4 * cout));
  int kc = (int)(q / ((int64_t)chunk * 4 * cout));
  int ci = kc * chunk + c, tap = n / cout, co = n % cout;
  wtc[q] = __float2bfloat16_rn((float)master[m_w + ((int64_t)(ci * cout + co) * 2 + tap / 2) * 2 + tap % 2]);
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// conv_row.cu: row-tile kernels for the narrow 3x3 layers
bool conv_row_supported(int cin_total, int cout);
helm_status conv_row_prepare(const double* master, int64_t m_w, int cin, int cin_pad, int cout, __nv_bfloat16** w,
                             cudaStream_t st);
helm_status conv_row_forward(const __nv_bfloat16* wrow, const float* bias, int* err, const void* in0, int C0,
                             const void* in1, int C1, void* out, int cout, int B, int H, int W, cudaStream_t st,
                             const RowFinal* fin = nullptr, int variant = 0, int* ry_out = nullptr);

struct TcState {
  __nv_bfloat16* w[NUM_LAYERS] = {};
  __nv_bfloat16* wrow[NUM_LAYERS] = {};  // row-tile weights where the row kernels serve the layer
  int cin_pad[NUM_LAYERS] = {};
  int chunk[NUM_LAYERS] = {};
  int* err = nullptr;
  bool ok = false;
};

static int tc_chunk(int cin_pad) { return cin_pad >= 64 ? 64 : cin_pad; }

// The tcgen05 kernels can run: the tensor-map encoder is reachable and the current device is sm_103.
bool tc_available() {
  if (!encode_fn()) return false;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

static bool tc_disabled_by_env() {
  const char* e = getenv("HELM_DISABLE_TC");
  return e && e[0] == '1';
}

helm_status conv_tc_prepare(helm_unet* net, cudaStream_t st) {
  if (!net->tc) {
    net->tc = new TcState();
    TcState& S = *net->tc;
    if (!encode_fn() || tc_disabled_by_env()) return HELM_OK;  // path unavailable: CUDA-core kernels serve
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return HELM_OK;  // this binary holds sm_103a code only
    HELM_CK(cudaMalloc(&S.err, sizeof(int)));
    HELM_CK(cudaMemset(S.err, 0, sizeof(int)));
    for (int l = 0; l < NUM_LAYERS; ++l) {
      const LayerDesc& d = kLayers[l];
      if (d.kind == UP2) {
        S.cin_pad[l] = d.cin;
        S.chunk[l] = tc_chunk(d.cin);
        HELM_CK(cudaMalloc(&S.w[l], sizeof(__nv_bfloat16) * 4 * d.cin * d.cout));
        continue;
      }
      if (d.kind != CONV3) continue;
      int cin_pad = l == L_ENC1A ? X0_CH : d.cin;
      S.cin_pad[l] = cin_pad;
      S.chunk[l] = tc_chunk(l == L_DEC3A || l == L_DEC2A || l == L_DEC1A ? d.cin / 2 : cin_pad);
      HELM_CK(cudaMalloc(&S.w[l], sizeof(__nv_bfloat16) * 9 * cin_pad * d.cout));
    }
    S.ok = true;
  }
  TcState& S = *net->tc;
  if (!S.ok) return HELM_OK;
  const char* dr = getenv("HELM_DISABLE_ROW");
  const bool row_ok = !(dr && dr[0] == '1');
  for (int l = 0; l < NUM_LAYERS; ++l) {
    const LayerDesc& d = kLayers[l];
    if (row_ok && d.kind == CONV3 && conv_row_supported(S.cin_pad[l], d.cout))
      HELM_TRY(conv_row_prepare(net->master, net->L.m_w[l], d.cin, S.cin_pad[l], d.cout, &S.wrow[l], st));
    if (d.kind == UP2) {
      int64_t tot = (int64_t)4 * d.cin * d.cout;
      launch(k_prep_tc_up, cdiv(tot, 256), 256, 0, st, (const double*)net->master, net->L.m_w[l], d.cin, d.cout,
             S.chunk[l], S.w[l]);
      continue;
    }
    if (d.kind != CONV3) continue;
    int64_t total = (int64_t)9 * S.cin_pad[l] * d.cout;
    launch(k_prep_tc, cdiv(total, 256), 256, 0, st, (const double*)net->master, net->L.m_w[l], d.cin, S.cin_pad[l],
           d.cout, S.chunk[l], S.w[l]);
  }
  HELM_CK_LAUNCH();
  return HELM_OK;
}

void conv_tc_release(helm_unet* net) {
  if (!net->tc) return;
  for (auto* p : net->tc->w)
    if (p) cudaFree(p);
  for (auto* p : net->tc->wrow)
    if (p) cudaFree(p);
  if (net->tc->err) cudaFree(net->tc->err);
  delete net->tc;
  net->tc = nullptr;
}

template <typename T>
bool conv_tc_enabled(const helm_unet* net, int layer, int H, int W) {
  if (!std::is_same<T, __nv_bfloat16>::value) return false;
  if (!net->tc || !net->tc->ok || (kLayers[layer].kind != CONV3 && kLayers[layer].kind != UP2)) return false;
  return H >= 1 && W >= 1;
}
template bool conv_tc_enabled<double>(const helm_unet*, int, int, int);
template bool conv_tc_enabled<__nv_bfloat16>(const helm_unet*, int, int, int);

static CUtensorMapSwizzle swizzle_for(int chunk) {
  return chunk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (chunk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

static helm_status act_map(CUtensorMap* m, const void* ptr, int C, int B, int H, int W, int chunk, int rows = 8) {
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  cuuint32_t box[4] = {(cuuint32_t)chunk, 16, (cuuint32_t)rows, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(chunk), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (activations) failed: " + std::to_string((int)r));
  return HELM_OK;
}

// The space-to-depth view of an NHWC BF16 tensor [B][2H][2W][C] on the H x W grid: one box is the
// 8 x 16 patch of one row phase, each pixel's 2C values being its two column phases (contiguous in
// memory); the map's rows are the source's rows, traversed with stride 2 from 2 Y + phase.
static helm_status act_map_s2d(CUtensorMap* m, const void* ptr, int chunk, int B, int H, int W, int rows) {
  const int C = chunk / 2;
  cuuint64_t dims[4] = {(cuuint64_t)chunk, (cuuint64_t)W, (cuuint64_t)(2 * H), (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)chunk * 2, (cuuint64_t)2 * W * C * 2, (cuuint64_t)4 * H * W * C * 2};
  cuuint32_t box[4] = {(cuuint32_t)chunk, 16, (cuuint32_t)(2 * rows), 1};
  cuuint32_t es[4] = {1, 1, 2, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(chunk), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (space-to-depth view) failed: " + std::to_string((int)r));
  return HELM_OK;
}

// The phase view of an NHWC BF16 tensor [B][Hs][Ws][32] on the (Hs / f) x (Ws / f) grid: one box is the
// patch of one phase (sy, sx), its source rows and columns traversed with stride f from f Y + sy and
// f X + sx; each pixel holds the source pixel's 32 channels.
static helm_status act_map_phase(CUtensorMap* m, const void* ptr, int f, int B, int Hs, int Ws, int rows) {
  cuuint64_t dims[4] = {32, (cuuint64_t)Ws, (cuuint64_t)Hs, (cuuint64_t)B};
  cuuint64_t strides[3] = {64, (cuuint64_t)Ws * 64, (cuuint64_t)Hs * Ws * 64};
  cuuint32_t box[4] = {32, (cuuint32_t)(16 * f), (cuuint32_t)(rows * f), 1};
  cuuint32_t es[4] = {1, (cuuint32_t)f, (cuuint32_t)f, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (phase view) failed: " + std::to_string((int)r));
  return HELM_OK;
}

static helm_status weight_map(CUtensorMap* m, const void* ptr, int N, int chunk, int nk, int taps = 9) {
  cuuint64_t dims[3] = {(cuuint64_t)chunk, (cuuint64_t)N, (cuuint64_t)(taps * nk)};
  cuuint64_t strides[2] = {(cuuint64_t)chunk * 2, (cuuint64_t)N * chunk * 2};
  cuuint32_t box[3] = {(cuuint32_t)chunk, (cuuint32_t)N, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(chunk), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HELM_ERR_CUDA, "cuTensorMapEncodeTiled (weights) failed: " + std::to_string((int)r));
  return HELM_OK;
}

template <int N, int CHUNK, int MODE, int KS = 3, int RB = 1>
static helm_status launch_tc(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& w, const ConvTcArgs& args,
                             cudaStream_t st) {
  using Cfg = TcCfg<N, CHUNK, MODE, KS, RB>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int per_sm = 1, nsm = 148;
  std::call_once(once, [] {
    attr_err =
        cudaFuncSetAttribute(k_conv_tc<N, CHUNK, MODE, KS, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // resident CTAs per SM: shared memory (1 KB reserved per CTA), TMEM (512 columns), threads, and
    // the occupancy calculator (registers)
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_conv_tc<N, CHUNK, MODE, KS, RB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      100);
    int by_regs = 8;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_conv_tc<N, CHUNK, MODE, KS, RB>) == cudaSuccess && fa.numRegs > 0)
      by_regs = 65536 / (((fa.numRegs + 7) / 8) * 8 * Cfg::THREADS);
    int by_smem = smem_sm / (Cfg::SMEM + 1024);
    per_sm = std::min(std::min(by_smem, 512 / Cfg::TMEM_COLS), std::min(2048 / Cfg::THREADS, by_regs));
    per_sm = std::max(1, per_sm);
  });
  HELM_CK(attr_err);
  int grid = std::min(args.ntiles, nsm * per_sm);
  launch(k_conv_tc<N, CHUNK, MODE, KS, RB>, grid, Cfg::THREADS, Cfg::SMEM, st, a0, a1, w, args);
  HELM_CK_LAUNCH();
  return HELM_OK;
}

// The 9-box kernel for one 3x3 layer (any layer shape the chunking allows).
static helm_status conv_tc_box(const helm_unet* net, int l, const void* in0, int C0, const void* in1, int C1,
                               void* out, int B, int H, int W, cudaStream_t st) {
  const TcState& S = *net->tc;
  const LayerDesc& d = kLayers[l];
  const int chunk = S.chunk[l];
  if (C0 % chunk || C1 % chunk) return fail(HELM_ERR_INVALID_ARG, "conv_tc_forward: channel count not a chunk multiple");
  CUtensorMap m0, m1, mw;
  HELM_TRY(act_map(&m0, in0, C0, B, H, W, chunk));
  if (C1 > 0)
    HELM_TRY(act_map(&m1, in1, C1, B, H, W, chunk));
  else
    m1 = m0;
  const int nk = (C0 + C1) / chunk;
  HELM_TRY(weight_map(&mw, S.w[l], d.cout, chunk, nk));
  ConvTcArgs a{};
  a.B = B;
  a.H = H;
  a.W = W;
  a.nk0 = C0 / chunk;
  a.nk1 = C1 / chunk;
  a.tiles_x = (W + 15) / 16;
  a.tiles_y = (H + 7) / 8;
  a.ntiles = B * a.tiles_x * a.tiles_y;
  a.bias = net->w32 + net->L.c_b[l];
  a.out = (__nv_bfloat16*)out;
  a.act = 1;
  a.slope = 0.f;
  a.err = S.err;
  a.budget = wait_budget();
  a.skip_first = take_fault(HELM_FAULT_CONV_TILE) ? 1 : 0;
  switch (d.cout * 1000 + chunk) {
    case 16016: return launch_tc<16, 16, 0>(m0, m1, mw, a, st);
    case 32016: return launch_tc<32, 16, 0>(m0, m1, mw, a, st);
    case 32032: return launch_tc<32, 32, 0>(m0, m1, mw, a, st);
    case 64032: return launch_tc<64, 32, 0>(m0, m1, mw, a, st);
    case 64064: return launch_tc<64, 64, 0>(m0, m1, mw, a, st);
    case 128064: return launch_tc<128, 64, 0>(m0, m1, mw, a, st);
    default: return fail(HELM_ERR_INVALID_ARG, "conv_tc_forward: no kernel for this layer shape");
  }
}

helm_status conv_tc_forward(const helm_unet* net, int l, const void* in0, int C0, const void* in1, int C1, void* out,
                            int B, int H, int W, cudaStream_t st) {
  const TcState& S = *net->tc;
  const LayerDesc& d = kLayers[l];
  if (l == L_ENC1A) C0 = X0_CH;
  if (S.wrow[l])
    return conv_row_forward(S.wrow[l], net->w32 + net->L.c_b[l], S.err, in0, C0, in1, C1, out, d.cout, B, H, W, st);
  return conv_tc_box(net, l, in0, C0, in1, C1, out, B, H, W, st);
}

// 2x2 stride-2 transposed conv on tensor cores: in [B][Hi][Wi][cin] -> out [B][2Hi][2Wi][cout].
bool conv_tc_final_ready(const helm_unet* net) { return net->tc && net->tc->ok && net->tc->wrow[L_DEC1B]; }

helm_status conv_tc_final(const helm_unet* net, const void* in, float2* z, const double* out_scale, int Nx, int Ny,
                          int64_t zstride, int B, int H, int W, cudaStream_t st, const UnetIO* io) {
  const TcState& S = *net->tc;
  RowFinal f;
  f.wf = net->w32 + net->L.c_w[L_FINAL];  // [16][2] followed by the 2 biases
  f.out_scale = out_scale;
  f.z = z;
  f.Nx = Nx;
  f.Ny = Ny;
  f.zstride = zstride;
  f.io = io;
  return conv_row_forward(S.wrow[L_DEC1B], net->w32 + net->L.c_b[L_DEC1B], S.err, in, 16, nullptr, 0, nullptr, 16, B,
                          H, W, st, &f);
}

helm_status conv_tc_up(const helm_unet* net, int l, const void* in, void* out, int B, int Hi, int Wi, cudaStream_t st) {
  const TcState& S = *net->tc;
  const LayerDesc& d = kLayers[l];
  const int chunk = S.chunk[l];
  const int nk = d.cin / chunk;
  CUtensorMap m0, mw;
  HELM_TRY(act_map(&m0, in, d.cin, B, Hi, Wi, chunk));
  HELM_TRY(weight_map(&mw, S.w[l], 4 * d.cout, chunk, nk, 1));
  ConvTcArgs a{};
  a.B = B;
  a.H = Hi;
  a.W = Wi;
  a.nk0 = nk;
  a.nk1 = 0;
  a.tiles_x = (Wi + 15) / 16;
  a.tiles_y = (Hi + 7) / 8;
  a.ntiles = B * a.tiles_x * a.tiles_y;
  a.bias = net->w32 + net->L.c_b[l];
  a.out = (__nv_bfloat16*)out;
  a.act = 0;
  a.slope = 0.f;
  a.err = S.err;
  a.budget = wait_budget();
  a.skip_first = take_fault(HELM_FAULT_CONV_TILE) ? 1 : 0;
  switch (4 * d.cout * 1000 + chunk) {
    case 256064: return launch_tc<256, 64, 1>(m0, m0, mw, a, st);
    case 128064: return launch_tc<128, 64, 1>(m0, m0, mw, a, st);
    case 64032: return launch_tc<64, 32, 1>(m0, m0, mw, a, st);
    default: return fail(HELM_ERR_INVALID_ARG, "conv_tc_up: no kernel for this layer shape");
  }
}

// A KS x KS convolution of another network kind on the same kernels (unet_paper.cu): weights in the
// [tap][chunk][N][chunk] BF16 layout, N output columns (MODE 2: N = 4 C_out written depth-to-space to
// the 2H x 2W grid), inputs NHWC BF16 from one or two sources, epilogue bias + activation `act`.
helm_status conv_tc_generic(const __nv_bfloat16* w_tc, const float* bias, int* err, int ks, int mode, int N,
                            int chunk, const void* in0, int C0, const void* in1, int C1, void* out, int B, int H,
                            int W, int act, float slope, cudaStream_t st, bool s2d0, const RowFinal* fin,
                            const double* img_scale, void* pre_out) {
  if (C0 % chunk || C1 % chunk) return fail(HELM_ERR_INVALID_ARG, "conv_tc_generic: channels not a chunk multiple");
  if (s2d0 && (mode != 0 || C1 != 0 || C0 != 2 * chunk))
    return fail(HELM_ERR_INVALID_ARG, "conv_tc_generic: the space-to-depth view needs one source of two row phases");
  if (fin && mode != 2) return fail(HELM_ERR_INVALID_ARG, "conv_tc_generic: the fused output layer needs mode 2");
  CUtensorMap m0, m1, mw;
  // row blocks per tile (5x5 layers): 4 (narrow chunks of N = 32) or 2, the most whose last tile row
  // wastes at most an eighth of the grid's rows, else 1
  int rb = 1;
  if (ks == 5)
    for (int c : {(N == 32 && chunk == 32) ? 4 : 2, 2}) {
      const int tile_rows = 8 * c;
      if ((H + tile_rows - 1) / tile_rows * tile_rows - H <= H / 8) {
        rb = c;
        break;
      }
    }
  const int rows = ks == 5 ? 8 * rb + 4 : 8;  // patch rows of one stage (TcCfg::A_ROWS)
  if (s2d0)
    HELM_TRY(act_map_s2d(&m0, in0, chunk, B, H, W, rows));
  else
    HELM_TRY(act_map(&m0, in0, C0, B, H, W, chunk, rows));
  if (C1 > 0)
    HELM_TRY(act_map(&m1, in1, C1, B, H, W, chunk, rows));
  else
    m1 = m0;
  const int nk = (C0 + C1) / chunk;
  HELM_TRY(weight_map(&mw, w_tc, N, chunk, nk, ks * ks));
  ConvTcArgs a{};
  a.B = B;
  a.H = H;
  a.W = W;
  a.nk0 = C0 / chunk;
  a.nk1 = C1 / chunk;
  a.tiles_x = (W + 15) / 16;
  a.tiles_y = (H + 8 * rb - 1) / (8 * rb);
  a.ntiles = B * a.tiles_x * a.tiles_y;
  a.bias = bias;
  a.out = (__nv_bfloat16*)out;
  a.act = act;
  a.slope = slope;
  a.err = err;
  a.budget = wait_budget();
  a.skip_first = take_fault(HELM_FAULT_CONV_TILE) ? 1 : 0;
  a.s2d = s2d0 ? 1 : 0;
  a.img_scale = img_scale;
  a.pre_out = (__nv_bfloat16*)pre_out;
  a.wf = fin ? fin->wf : nullptr;
  a.out_scale = fin ? fin->out_scale : nullptr;
  a.z = fin ? fin->z : nullptr;
  a.Nx = fin ? fin->Nx : 0;
  a.Ny = fin ? fin->Ny : 0;
  a.zstride = fin ? fin->zstride : 0;
  const int key = rb * 10000000 + ks * 1000000 + mode * 100000 + N * 100 + chunk;
  switch (key) {
    case 15000000 + 32 * 100 + 32: return launch_tc<32, 32, 0, 5, 1>(m0, m1, mw, a, st);
    case 25000000 + 32 * 100 + 32: return launch_tc<32, 32, 0, 5, 2>(m0, m1, mw, a, st);
    case 45000000 + 32 * 100 + 32: return launch_tc<32, 32, 0, 5, 4>(m0, m1, mw, a, st);
    case 15000000 + 32 * 100 + 64: return launch_tc<32, 64, 0, 5, 1>(m0, m1, mw, a, st);
    case 25000000 + 32 * 100 + 64: return launch_tc<32, 64, 0, 5, 2>(m0, m1, mw, a, st);
    case 15200000 + 128 * 100 + 32: return launch_tc<128, 32, 2, 5, 1>(m0, m1, mw, a, st);
    case 25200000 + 128 * 100 + 32: return launch_tc<128, 32, 2, 5, 2>(m0, m1, mw, a, st);
    default: return fail(HELM_ERR_INVALID_ARG, "conv_tc_generic: no kernel for this shape");
  }
}

// An 8x8 stride-2 layer of network kind 1 as a 3x3 convolution of the phase view of its input
// (f = 2: the space-to-depth-packed network input, 32 channels = 2 x 2 phases x 8; f = 4: a 32-channel
// activation): GEMM grid H x W (the output grid is 2H x 2W), N = 128 columns = 2 x 2 output phases x 32
// channels written depth-to-space, K = f^2 chunks of 32 per tap, weights `wq` [tap][kc][n][32] BF16.
// Epilogue: bias + PReLU(slope); optional per-image skip and pre-activation store as conv_tc_generic.
helm_status conv_tc_phase(const __nv_bfloat16* wq, const float* bias, int* err, int f, const void* in, void* out,
                          int B, int H, int W, float slope, cudaStream_t st, const double* img_scale, void* pre_out) {
  if (f != 2 && f != 4) return fail(HELM_ERR_INVALID_ARG, "conv_tc_phase: phase factor must be 2 or 4");
  // two row blocks per tile unless the last tile row would waste more than an eighth of the grid's rows
  const int rb = (H + 15) / 16 * 16 - H <= H / 8 ? 2 : 1;
  CUtensorMap m0, mw;
  HELM_TRY(act_map_phase(&m0, in, f, B, f * H, f * W, 8 * rb + 2));
  HELM_TRY(weight_map(&mw, wq, 128, 32, f * f, 9));
  ConvTcArgs a{};
  a.B = B;
  a.H = H;
  a.W = W;
  a.nk0 = f * f;
  a.nk1 = 0;
  a.tiles_x = (W + 15) / 16;
  a.tiles_y = (H + 8 * rb - 1) / (8 * rb);
  a.ntiles = B * a.tiles_x * a.tiles_y;
  a.bias = bias;
  a.out = (__nv_bfloat16*)out;
  a.act = 2;
  a.slope = slope;
  a.err = err;
  a.budget = wait_budget();
  a.skip_first = take_fault(HELM_FAULT_CONV_TILE) ? 1 : 0;
  a.qf = f;
  a.img_scale = img_scale;
  a.pre_out = (__nv_bfloat16*)pre_out;
  return rb == 2 ? launch_tc<128, 32, 2, 3, 2>(m0, m0, mw, a, st) : launch_tc<128, 32, 2, 3, 1>(m0, m0, mw, a, st);
}

// Error code left by a timed-out tcgen05 kernel (0 if none); clears it.
helm_status conv_tc_check(const helm_unet* net, cudaStream_t st) {
  if (net->pn) return paper_check(net, st);
  if (!net->tc || !net->tc->err) return HELM_OK;
  int e = 0;
  HELM_CK(cudaMemcpyAsync(&e, net->tc->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  if (e) {
    cudaMemsetAsync(net->tc->err, 0, sizeof(int), st);
    return fail(HELM_TIMEOUT, "tcgen05 conv kernel: a pipeline wait ran out of its budget (code " + std::to_string(e) + ")");
  }
  return HELM_OK;
}

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_unet_layer_forward(const helm_unet* net, int layer, int variant, const void* in0,
                                               const void* in1, void* out, int B, int H, int W, int* ry_out,
                                               void* stream) {
  if (ry_out) *ry_out = 0;
  if (!net || !in0 || !out) return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: NULL argument");
  if (layer < 0 || layer > HELM_LAYER_DEC1B_FINAL)
    return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: layer out of range");
  if (B < 1 || H < 1 || W < 1 || (int64_t)B * H * W > ((int64_t)1 << 31))
    return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: bad image size");
  if (((uintptr_t)in0 | (uintptr_t)in1 | (uintptr_t)out) & 15)
    return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: pointers must be 16-byte aligned");
  if (net->kind != 0) return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: network kind 0 only");
  if (!net->tc || !net->tc->ok)
    return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: the tcgen05 path is not available on this device");
  cudaStream_t st = (cudaStream_t)stream;
  const TcState& S = *net->tc;
  const bool fused = layer == HELM_LAYER_DEC1B_FINAL;
  const int l = fused ? (int)L_DEC1B : layer;
  const LayerDesc& d = kLayers[l];
  const bool concat = l == L_DEC3A || l == L_DEC2A || l == L_DEC1A;
  if (concat != (in1 != nullptr))
    return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: in1 is required exactly for the decoder's first convs");
  const int C0 = concat ? d.cin / 2 : (l == L_ENC1A ? X0_CH : d.cin), C1 = concat ? d.cin / 2 : 0;
  if (d.kind == UP2) {
    if (variant != 0 && variant != -1)
      return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: up-convs have one kernel (variant 0 or -1)");
    return conv_tc_up(net, l, in0, out, B, H, W, st);
  }
  if (variant == -1) {
    if (fused) return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: the fused output layer is a row kernel");
    return conv_tc_box(net, l, in0, C0, in1, C1, out, B, H, W, st);
  }
  if (!S.wrow[l]) {
    if (variant != 0) return fail(HELM_ERR_INVALID_ARG, "helm_unet_layer_forward: no row-tile kernel for this layer");
    return conv_tc_box(net, l, in0, C0, in1, C1, out, B, H, W, st);
  }
  RowFinal f;
  if (fused) {
    f.wf = net->w32 + net->L.c_w[L_FINAL];
    f.out_scale = nullptr;  // scale 1
    f.z = (float2*)out;
    f.Nx = W;
    f.Ny = H;
    f.zstride = (int64_t)H * W;
    f.io = nullptr;
  }
  return conv_row_forward(S.wrow[l], net->w32 + net->L.c_b[l], S.err, in0, C0, in1, C1, fused ? nullptr : out, d.cout,
                          B, H, W, st, fused ? &f : nullptr, variant, ry_out);
}
