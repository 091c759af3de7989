// tcgen05 implicit-GEMM 3x3 convolutions (BF16 operands, FP32 accumulation in TMEM).
// Not yet enabled: every layer takes the CUDA-core path in unet.cu.
#include "unet.cuh"

namespace helm {

struct TcState {};

helm_status conv_tc_prepare(helm_unet*, cudaStream_t) { return HELM_OK; }
void conv_tc_release(helm_unet*) {}

template <typename T> bool conv_tc_enabled(const helm_unet*, int, int, int) { return false; }
template bool conv_tc_enabled<double>(const helm_unet*, int, int, int);
template bool conv_tc_enabled<__nv_bfloat16>(const helm_unet*, int, int, int);

helm_status conv_tc_forward(const helm_unet*, int, const void*, int, const void*, int, void*, int, int, int,
                            cudaStream_t) {
  return fail(HELM_ERR_INVALID_ARG, "conv_tc_forward: not available");
}

}  // namespace helm
