// Network weights and per-shape execution plans of the regulariser network.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <string>
#include <vector>

#include "ideq_internal.h"

namespace ideq {

enum LayerKind { LK_CONV3 = 0, LK_DOWN = 1, LK_UP = 2 };

struct Layer {
  int kind, cin, cout;  // cin/cout of the layer as written in PyTorch
  // stored channel counts of its input and output activations: cin/cout, or for a
  // plain CNN's hidden layers rounded up to a multiple of 32 (zero weights on the
  // padded channels) so that they fit the tensor-core conv's 32-channel rows
  int pcin, pcout;
  long long off;        // offset in the flat weight vector
  long long numel;
  int fwd_form, dg_form;
  float* fwd32 = nullptr;
  float* dg32 = nullptr;
  __nv_bfloat16* fwd16 = nullptr;  // bf16 forms
  __nv_bfloat16* dg16 = nullptr;
  __half* fwdh = nullptr;          // f16 forms
  __half* dgh = nullptr;
  // e4m3 forms with per-row (output column) scales, for the directions whose
  // input has >= 256 channels (forward: cin, input gradient: cout)
  uint8_t* fwd8 = nullptr;
  float* fwd8s = nullptr;
  uint8_t* dg8 = nullptr;
  float* dg8s = nullptr;
  // [N][32] 16-bit forms of 3x3 directions whose K = 9 x (image channels) <= 32:
  // the image-side input convs (head forward, tail input gradient) as one K chunk
  __half* i2c_fwd_h = nullptr;
  __nv_bfloat16* i2c_fwd_b = nullptr;
  __half* i2c_dg_h = nullptr;
  __nv_bfloat16* i2c_dg_b = nullptr;
};

constexpr int kFp8MinChannels = 256;  // convs with at least this many input channels

// Flat weight vector + its GEMM forms (f32, bf16, f16; forward and input-gradient).
struct NetWeights {
  ideq_net_desc desc{};
  long long nparams = 0;
  float* master = nullptr;  // device, PyTorch layout
  std::vector<Layer> layers;
  std::vector<void*> allocs;
  ~NetWeights();
  bool build(const ideq_net_desc& d, std::string* err);
  cudaError_t upload(const float* dev_weights, cudaStream_t st);  // copy + re-form
  cudaError_t reform(cudaStream_t st);
};

bool net_param_count(const ideq_net_desc& d, long long* count, std::vector<Layer>* layers,
                     std::string* err);

// One conv launch of a plan.
struct Step {
  ConvArgs a;
  int in_dt = 0, out_dt = 0;  // DT_* of the NHWC/NCHW input and output
  TcPlan* tc = nullptr;
  bool edge = false;  // image-side <-> feature-side kernel
  // FP8 convs (quant_n > 0): the 16-bit input q_src is first reduced to its
  // max |x| (q_amax) and quantised to e4m3 codes (q_dst, the conv's input) with
  // the scale q_scale that the conv's epilogue multiplies back
  long long quant_n = 0;
  const void* q_src = nullptr;
  uint8_t* q_dst = nullptr;
  float* q_amax = nullptr;
  float* q_scale = nullptr;
  // image-side input convs on the tensor cores (i2c_px > 0): the f32 planar image
  // i2c_src (i2c_c channels, i2c_H x i2c_W) is first written as im2col rows into
  // i2c_dst, the conv's 32-channel input
  long long i2c_px = 0;
  const float* i2c_src = nullptr;
  void* i2c_dst = nullptr;
  int i2c_c = 0, i2c_H = 0, i2c_W = 0;
};

// Execution plan for one (n, H, W, precision): activation buffers and the
// conv op lists of the forward pass N(z) -> r = z - N(z) and of the reverse
// pass grad = r - J_N(z)^T r.  z, r and grad are plan-owned f32 NCHW buffers.
struct NetPlan {
  int n = 0, c = 0, H = 0, W = 0, prec = 0;
  NetWeights* w = nullptr;
  float* z = nullptr;
  float* r = nullptr;
  float* grad = nullptr;
  double* gsum = nullptr;  // per-image 1/2||r||^2, accumulated by the forward pass
  const int* skip = nullptr;  // per-image skip flags of the solver (nullable)
  std::vector<Step> fwd, vjp;
  std::vector<void*> allocs;
  double fwd_flops = 0, vjp_flops = 0;
  ~NetPlan();
  bool build(NetWeights* w, int n, int H, int W, int prec, double* gsum, std::string* err,
             const int* skip = nullptr);
  void* alloc(size_t bytes);
};

struct Profiler;
cudaError_t run_steps(const std::vector<Step>& steps, int* err_flag, cudaStream_t st,
                      Profiler* prof, long long* launches);

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  size_t used = 0;
  double flops = 0;
  long long launches = 0;
  cudaEvent_t next();
  ~Profiler();
};

}  // namespace ideq
