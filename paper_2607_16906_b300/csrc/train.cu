// Physics-informed training step (a9, eqs. 8-9): forward, adjoint-stencil loss gradient, conv
// backward, global-norm clip and AdamW.  Filled in below; until then the entry points report
// that they are unavailable.
#include "unet.cuh"

using namespace helm;

extern "C" helm_status helm_loss_grad(helm_ctx* ctx, const helm_unet* net, const void* b, double* loss_host,
                                      double* grad_dev, void* stream) {
  (void)ctx; (void)net; (void)b; (void)loss_host; (void)grad_dev; (void)stream;
  return fail(HELM_ERR_INVALID_ARG, "helm_loss_grad: not built in this library version");
}

extern "C" helm_status helm_train_step(helm_ctx* ctx, helm_unet* net, const void* b, double lr, double wd,
                                       double clip, double* loss_host, double* grad_norm_host, void* stream) {
  (void)ctx; (void)net; (void)b; (void)lr; (void)wd; (void)clip; (void)loss_host; (void)grad_norm_host; (void)stream;
  return fail(HELM_ERR_INVALID_ARG, "helm_train_step: not built in this library version");
}
