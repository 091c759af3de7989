// Internal network declarations: layer table, parameter layout, activation buffers.
#pragma once

#include <map>
#include <set>

#include "helm_internal.cuh"

namespace helm {

enum LayerKind { CONV3 = 0, UP2 = 1, CONV1 = 2 };
enum LayerId {
  L_ENC1A = 0, L_ENC1B, L_ENC2A, L_ENC2B, L_ENC3A, L_ENC3B, L_BOTA, L_BOTB, L_UP3, L_DEC3A, L_DEC3B,
  L_UP2, L_DEC2A, L_DEC2B, L_UP1, L_DEC1A, L_DEC1B, L_FINAL, NUM_LAYERS
};

struct LayerDesc {
  const char* name;
  int kind, cin, cout;
};
extern const LayerDesc kLayers[NUM_LAYERS];
int taps_of(int kind);

struct NetLayout {
  int64_t m_w[NUM_LAYERS], m_b[NUM_LAYERS];  // offsets in the master vector (PyTorch layouts)
  int64_t c_w[NUM_LAYERS], c_b[NUM_LAYERS];  // offsets in the CUDA-core buffers ([tap][cin][cout], bias)
  int64_t total, ctotal;
};
NetLayout make_layout();

// Activation slots (NHWC).  X0 holds the packed network input with X0_CH channel stride.
enum ActId {
  A_X0 = 0, A_E1A, A_S1, A_P1, A_E2A, A_S2, A_P2, A_E3A, A_S3, A_P3, A_BA, A_BB, A_U3, A_D3A, A_D3B,
  A_U2, A_D2A, A_D2B, A_U1, A_D1A, A_D1B, NUM_ACTS
};
constexpr int X0_CH = 16;  // input channels padded 3 -> 16 (one 32-byte row of BF16 per pixel)

// Pointers of one BF16 inference call that change from call to call (the Krylov slot read, the
// slot written, the per-column scales), read by the input and output kernels from a fixed device
// block so that a captured CUDA graph of the whole network stays valid.
struct UnetIO {
  const void* v;
  void* z;
  const double* in_scale;
  const double* out_scale;
};

// Captured network applications, keyed by (network id, system, columns, velocity stride, buffer
// generation).  A key is captured on its second use (the first runs eagerly, so that every
// allocation and one-time set-up has happened) and replayed afterwards.
struct UnetGraphKey {
  uint64_t net_id;
  int sys, B;
  int64_t c_stride;
  uint64_t gen;
  bool operator<(const UnetGraphKey& o) const {
    if (net_id != o.net_id) return net_id < o.net_id;
    if (sys != o.sys) return sys < o.sys;
    if (B != o.B) return B < o.B;
    if (c_stride != o.c_stride) return c_stride < o.c_stride;
    return gen < o.gen;
  }
};
struct UnetGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernel nodes per replay
};

struct UnetBuffers {
  struct Set {
    void* base = nullptr;
    size_t cap = 0;  // bytes allocated at base
    int B = 0, Hp = 0, Wp = 0;
    void* a[NUM_ACTS] = {};
  } set[2];  // [0] BF16, [1] FP64
  uint64_t gen = 0;  // bumped whenever an allocation moves (invalidates captured graphs)
  UnetIO* io = nullptr;  // device block read by the BF16 inference kernels
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::map<UnetGraphKey, UnetGraph> graphs;
  std::set<UnetGraphKey> seen;
};

struct TcLayer;  // tcgen05 per-layer state (conv_tc.cu)

helm_status ensure_buffers(helm_ctx* ctx, int B, int Hp, int Wp, bool fp64, UnetBuffers** out);

// tcgen05 implicit-GEMM 3x3 convolutions (conv_tc.cu)
struct TcState;
helm_status conv_tc_prepare(helm_unet* net, cudaStream_t st);
void conv_tc_release(helm_unet* net);
template <typename T> bool conv_tc_enabled(const helm_unet* net, int layer, int H, int W);
helm_status conv_tc_forward(const helm_unet* net, int layer, const void* in0, int C0, const void* in1, int C1,
                            void* out, int B, int H, int W, cudaStream_t st);
helm_status conv_tc_up(const helm_unet* net, int layer, const void* in, void* out, int B, int Hi, int Wi,
                       cudaStream_t st);
// Last 3x3 conv (16 -> 16, ReLU) with the final 1x1 conv, the output scale and the crop to the
// physical grid fused into its epilogue (inference only: the activation is not stored).
struct RowFinal {
  const float* wf;  // [16][2] weights, then the 2 biases
  const double* out_scale;
  float2* z;
  int Nx, Ny;
  int64_t zstride;
  const UnetIO* io;  // non-null: z and out_scale are read from this block at run time
};
bool conv_tc_final_ready(const helm_unet* net);
helm_status conv_tc_final(const helm_unet* net, const void* in, float2* z, const double* out_scale, int Nx, int Ny,
                          int64_t zstride, int B, int H, int W, cudaStream_t st, const UnetIO* io = nullptr);
// HELM_TIMEOUT if a tcgen05 conv kernel recorded a pipeline timeout since the last check (synchronises).
helm_status conv_tc_check(const helm_unet* net, cudaStream_t st);

// z = out_scale * N(in_scale * v, c) for B columns of system `sys` (column stride n_sys).  Velocity
// channel: c of system `sys` for every column (c_stride = 0), or of consecutive equal-size systems
// (c_stride = n_sys, one system per column, as in training batches).  keep_acts: every activation
// stays in the buffers for a backward pass (no fused last layer).
template <typename R>
helm_status unet_precondition(helm_ctx* ctx, const helm_unet* net, int sys, const C<R>* v, C<R>* z, int B,
                              const double* in_scale, const double* out_scale, cudaStream_t st, int64_t c_stride,
                              bool keep_acts = false);

// Element types of the two network paths: activations T, accumulation / weights A.
template <typename T> struct Acc;
template <> struct Acc<double> { using A = double; };
template <> struct Acc<__nv_bfloat16> { using A = float; };
template <> struct Acc<float> { using A = float; };
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ void store_act(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_act(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_act(float* p, float v) { *p = v; }
template <typename T> const typename Acc<T>::A* cc_weights(const helm_unet* net);
helm_status unet_prepare(helm_unet* net, cudaStream_t st);

// The paper's U-Net variant (unet_paper.cu): network kind 1.
constexpr int PAPER_LAYERS = 9;  // enc1..enc4, dec3..dec0, out
struct PaperNet {
  int64_t m_w[PAPER_LAYERS] = {}, m_b[PAPER_LAYERS] = {}, m_s[PAPER_LAYERS] = {};  // master offsets
  double* w5[PAPER_LAYERS] = {};          // reformulated weights [tap][k][n], FP64
  float* w5f[PAPER_LAYERS] = {};          // the same in FP32 (training path)
  double* b5[PAPER_LAYERS] = {};          // per-column bias, FP64
  __nv_bfloat16* wtc[PAPER_LAYERS] = {};  // tcgen05 layout [tap][kc][n][c], BF16
  float* b32[PAPER_LAYERS] = {};
  // encoder layers as 3x3 convolutions of the phase view of their input (conv_tc_phase): [tap][kc][n][c]
  // BF16 with N = 128 columns (2 x 2 output phases x 32 channels), bias per column in FP32
  __nv_bfloat16* wq[3] = {};  // enc1..enc3
  float* bq[3] = {};
  float* wout32 = nullptr;                // output layer, BF16-rounded weights in FP32 + 2 biases
  double slope[PAPER_LAYERS] = {};        // PReLU slopes
  int* err = nullptr;                     // tcgen05 pipeline error code
  struct Set {
    void* base = nullptr;
    size_t cap = 0;
  } act[2];  // activations: [0] BF16, [1] FP64
};
int64_t paper_param_count();
// Algorithmic flops of one network application per full-resolution pixel: kind 0, its 3x3 / 2x2 /
// 1x1 layers (2 x 35,408 MACs); kind 1, the 8x8 strided and transposed layers and the output layer
// (2 x 51,264 MACs; the BF16 path executes 88,800 MACs, structural zeros included).
inline double unet_flop_per_point(int kind) { return kind == 1 ? 102528.0 : 70816.0; }
helm_status paper_prepare(helm_unet* net, cudaStream_t st);
void paper_release(helm_unet* net);
template <typename R>
helm_status paper_precondition(helm_ctx* ctx, const helm_unet* net, int sys, const C<R>* v, C<R>* z, int B,
                               const double* in_scale, const double* out_scale, cudaStream_t st);
helm_status paper_check(const helm_unet* net, cudaStream_t st);
// Loss (eq. 9, batch mean) and its gradient into net->grad (master layout) for network kind 1:
// forward and backward on CUDA cores in FP32 (R = float, the training path) or FP64 (R = double).
template <typename R>
helm_status paper_loss_grad(helm_ctx* ctx, helm_unet* net, const C<R>* b, double* loss_host, cudaStream_t st);

}  // namespace helm

struct helm_unet {
  uint64_t id = 0;  // unique per created network (keys of captured graphs)
  int kind = 0;     // 0: the 16/32/64/128 U-Net; 1: the paper's variant (PaperNet)
  helm::PaperNet* pn = nullptr;
  helm::NetLayout L;
  double* master = nullptr;  // FP64 master weights (PyTorch layouts)
  double* w64 = nullptr;     // CUDA-core layout, FP64
  float* w32 = nullptr;      // CUDA-core layout, BF16-rounded values held in FP32 (bias unrounded)
  double* adam_m = nullptr;  // AdamW first moment
  double* adam_v = nullptr;  // AdamW second moment
  double* grad = nullptr;    // gradient scratch (FP64)
  int64_t step = 0;
  helm::TcState* tc = nullptr;
};
