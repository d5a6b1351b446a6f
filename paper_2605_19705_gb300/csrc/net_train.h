// Training plan of the regulariser network (see net_train.cu).
#pragma once

#include <string>
#include <vector>

#include "net.h"

namespace ideq {

struct WgTcPlan;  // tensor-core weight gradient of one (input, cotangent) pair (wgrad_tc.cu)

struct WgStep {
  int layer;            // index into NetWeights::layers
  ConvArgs a;           // the forward conv (geometry and primal input)
  int in_dt, cot_dt;
  const void* tin;      // tangent input of the conv
  const void* pcot;     // p-chain cotangent of its output
  const void* tcot;     // t-chain cotangent of its output
  // tensor-core forms (null: SIMT): [0] input x pcot, [1] tangent input x tcot,
  // [2] input x tcot (plain reverse chain)
  WgTcPlan* tc[3] = {nullptr, nullptr, nullptr};
};

struct TrainPlan {
  int n = 0, c = 0, H = 0, W = 0, prec = 0;
  NetWeights* w = nullptr;
  float *z = nullptr, *r = nullptr, *grad = nullptr;  // point, residual, grad g
  float *zd = nullptr, *rd = nullptr, *hvp = nullptr; // direction, rdot, Hess g . direction
  // warm-start mode (plain CNN x0 = z + W(z)): forward output and the cotangent
  // that starts the reverse chain
  bool warm = false;
  float* out_img = nullptr;
  float* cot_img = nullptr;
  double* gsum = nullptr;
  std::vector<Step> fwd, tchain, jvp, pchain;
  std::vector<WgStep> wg;
  float* wg_part = nullptr;
  float* wg_acc = nullptr;
  std::vector<void*> allocs;
  ~TrainPlan();
  void* alloc(size_t bytes);
  bool build(NetWeights* w, int n, int H, int W, int prec, double* gsum, std::string* err,
             bool warm = false);
  // dual: dst += scale * sum_conv [pcot (x) input + tcot (x) tangent input]
  // plain: dst += scale * sum_conv tcot (x) input (one reverse chain)
  cudaError_t run_wgrad(float* dst, float scale, bool dual, cudaStream_t st, long long* launches,
                        int* err);
};

int wgrad_splits(const ConvArgs& a);
// dst[e] += scale * sum_z part[z][e] over `splits` partial [N][K] tiles, fixed order
cudaError_t launch_wgrad_reduce(long long nk, int splits, const float* part, float scale,
                                float* dst, cudaStream_t st);
// tcgen05 weight gradient of a 3x3 or stride-2 2x2 conv with 16-bit NHWC input and
// cotangent (Cin, Cout multiples of 64); `part` holds wgrad_tc_splits(a) x N x K floats
bool wgrad_tc_supported(const ConvArgs& a, int in_dt, int cot_dt);
int wgrad_tc_splits(const ConvArgs& a);
WgTcPlan* wgrad_tc_plan_create(const ConvArgs& a, int dt, const void* in, const void* cot,
                               float* part);
void wgrad_tc_plan_destroy(WgTcPlan* p);
// dst [N][K] += scale * gradient; err: bounded-wait flag
cudaError_t launch_wgrad_tc(const WgTcPlan* p, float scale, float* dst, int* err,
                            cudaStream_t st);
cudaError_t launch_wgrad(const ConvArgs& a, int in_dt, int cot_dt, const void* cot, float scale,
                         float* part, float* dst, cudaStream_t st);
cudaError_t launch_weight_unform_scaled(int form, int cin, int cout, const float* g, float scale,
                                        float* dst, cudaStream_t st);
// cot = 2 (x - t) / numel and *loss = mean((x - t)^2) (FP64); part >= 128 doubles
cudaError_t launch_mse_grad(long long numel, const float* x, const float* t, float* cot,
                            double* part, double* loss, cudaStream_t st);
// one Adam step (bias-corrected) on n parameters; t is the 1-based step count
cudaError_t launch_adam(long long n, float* p, const float* g, float* m, float* v, int t, float lr,
                        float b1, float b2, float eps, cudaStream_t st);

}  // namespace ideq
