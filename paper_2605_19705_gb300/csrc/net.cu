// Regulariser network: weight forms and the conv op lists of N and J_N^T.
//
// g(z) = 1/2 ||z - N(z)||^2 and grad g(z) = r - J_N(z)^T r with r = z - N(z)
// (Sec. 2.2, Eq. GS).  The forward list ends with the tail conv whose epilogue
// forms r = z - N(z) and accumulates 1/2||r||^2; the reverse list starts with
// the transposed tail conv applied to r and ends with the transposed head conv
// whose epilogue forms grad = r - J_N^T r.  Activation derivatives are saved by
// the forward epilogues (softplus' = logistic) and multiplied in by the reverse
// epilogues; residual and skip sums are fused into the conv that produces them.
#include "net.h"

#include <algorithm>
#include <cstdlib>

namespace ideq {

// ------------------------------------------------------------------ weights

static int conv_form(int kind, bool dgrad) {
  if (kind == LK_CONV3) return dgrad ? WF_CONV3_DGRAD : WF_CONV3_FWD;
  if (kind == LK_DOWN) return dgrad ? WF_DOWN_DGRAD : WF_DOWN_FWD;
  return dgrad ? WF_UP_DGRAD : WF_UP_FWD;
}

bool net_param_count(const ideq_net_desc& d, long long* count, std::vector<Layer>* layers,
                     std::string* err) {
  std::vector<Layer> L;
  long long off = 0;
  auto add = [&](int kind, int cin, int cout, int pcin = -1, int pcout = -1) {
    Layer l;
    l.kind = kind;
    l.cin = cin;
    l.cout = cout;
    l.pcin = pcin < 0 ? cin : pcin;
    l.pcout = pcout < 0 ? cout : pcout;
    l.off = off;
    l.numel = (long long)cin * cout * (kind == LK_CONV3 ? 9 : 4);
    l.fwd_form = conv_form(kind, false);
    l.dg_form = conv_form(kind, true);
    off += l.numel;
    L.push_back(l);
  };
  if (d.in_ch < 1 || d.in_ch > 4) {
    *err = "in_ch must be 1..4";
    return false;
  }
  if (d.kind == IDEQ_NET_UNET) {
    const int Lv = d.n_levels;
    if (Lv < 1 || Lv > 6 || d.n_rb < 0 || d.n_rb > 8) {
      *err = "bad U-Net levels/rbs";
      return false;
    }
    for (int i = 0; i < Lv; ++i)
      if (d.widths[i] < 1) {
        *err = "bad U-Net width";
        return false;
      }
    add(LK_CONV3, d.in_ch, d.widths[0]);
    for (int l = 0; l < Lv - 1; ++l) {
      for (int r = 0; r < d.n_rb; ++r) {
        add(LK_CONV3, d.widths[l], d.widths[l]);
        add(LK_CONV3, d.widths[l], d.widths[l]);
      }
      add(LK_DOWN, d.widths[l], d.widths[l + 1]);
    }
    for (int r = 0; r < d.n_rb; ++r) {
      add(LK_CONV3, d.widths[Lv - 1], d.widths[Lv - 1]);
      add(LK_CONV3, d.widths[Lv - 1], d.widths[Lv - 1]);
    }
    for (int l = Lv - 2; l >= 0; --l) {
      add(LK_UP, d.widths[l + 1], d.widths[l]);
      for (int r = 0; r < d.n_rb; ++r) {
        add(LK_CONV3, d.widths[l], d.widths[l]);
        add(LK_CONV3, d.widths[l], d.widths[l]);
      }
    }
    add(LK_CONV3, d.widths[0], d.in_ch);
  } else if (d.kind == IDEQ_NET_CNN) {
    if (d.depth < 1 || d.depth > 15) {
      *err = "bad CNN depth";
      return false;
    }
    if (d.widths[0] != d.in_ch || d.widths[d.depth] != d.in_ch) {
      *err = "CNN widths[0] and widths[depth] must equal in_ch";
      return false;
    }
    // hidden widths stored as multiples of 32 channels (the image sides as they are)
    auto pad = [](int c) { return (c + 31) / 32 * 32; };
    for (int i = 0; i < d.depth; ++i)
      add(LK_CONV3, d.widths[i], d.widths[i + 1], i == 0 ? d.widths[i] : pad(d.widths[i]),
          i == d.depth - 1 ? d.widths[i + 1] : pad(d.widths[i + 1]));
  } else {
    *err = "unknown network kind";
    return false;
  }
  *count = off;
  if (layers) *layers = L;
  return true;
}

NetWeights::~NetWeights() {
  for (void* p : allocs) cudaFree(p);
}

bool NetWeights::build(const ideq_net_desc& d, std::string* err) {
  desc = d;
  if (!net_param_count(d, &nparams, &layers, err)) return false;
  auto al = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, (bytes + 255) & ~(size_t)255) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  };
  master = (float*)al(nparams * 4);
  if (!master) {
    *err = "cudaMalloc(weights) failed";
    return false;
  }
  for (auto& l : layers) {
    // 16-bit forms keep at least 16 rows (zero rows past N): the tensor-core conv
    // that writes c <= 16 image channels runs a 16-wide N tile
    int Nf, Kf, Nd, Kd;
    weight_form_dims_padded(l.fwd_form, l.cin, l.cout, l.pcin, l.pcout, &Nf, &Kf);
    weight_form_dims_padded(l.dg_form, l.cin, l.cout, l.pcin, l.pcout, &Nd, &Kd);
    const size_t f16n = (size_t)std::max(Nf, 16) * Kf, d16n = (size_t)std::max(Nd, 16) * Kd;
    l.fwd32 = (float*)al((size_t)Nf * Kf * 4);
    l.dg32 = (float*)al((size_t)Nd * Kd * 4);
    l.fwd16 = (__nv_bfloat16*)al(f16n * 2);
    l.dg16 = (__nv_bfloat16*)al(d16n * 2);
    l.fwdh = (__half*)al(f16n * 2);
    l.dgh = (__half*)al(d16n * 2);
    if (!l.fwd32 || !l.dg32 || !l.fwd16 || !l.dg16 || !l.fwdh || !l.dgh) {
      *err = "cudaMalloc(weight forms) failed";
      return false;
    }
    if (cudaMemset(l.fwd16, 0, f16n * 2) != cudaSuccess ||
        cudaMemset(l.dg16, 0, d16n * 2) != cudaSuccess ||
        cudaMemset(l.fwdh, 0, f16n * 2) != cudaSuccess ||
        cudaMemset(l.dgh, 0, d16n * 2) != cudaSuccess) {
      *err = "cudaMemset(weight forms) failed";
      return false;
    }
    // image-side 3x3 directions with K = 9 x (image channels) <= 32: one K chunk
    if (l.fwd_form == WF_CONV3_FWD && Kf <= 32) {
      l.i2c_fwd_h = (__half*)al((size_t)Nf * 32 * 2);
      l.i2c_fwd_b = (__nv_bfloat16*)al((size_t)Nf * 32 * 2);
      if (!l.i2c_fwd_h || !l.i2c_fwd_b) {
        *err = "cudaMalloc(weight forms) failed";
        return false;
      }
    }
    if (l.dg_form == WF_CONV3_DGRAD && Kd <= 32) {
      l.i2c_dg_h = (__half*)al((size_t)Nd * 32 * 2);
      l.i2c_dg_b = (__nv_bfloat16*)al((size_t)Nd * 32 * 2);
      if (!l.i2c_dg_h || !l.i2c_dg_b) {
        *err = "cudaMalloc(weight forms) failed";
        return false;
      }
    }
    int N, K;
    if (l.cin >= kFp8MinChannels) {
      weight_form_dims(l.fwd_form, l.cin, l.cout, &N, &K);
      l.fwd8 = (uint8_t*)al(l.numel);
      l.fwd8s = (float*)al((size_t)N * 4);
      if (!l.fwd8 || !l.fwd8s) {
        *err = "cudaMalloc(weight forms) failed";
        return false;
      }
    }
    if (l.cout >= kFp8MinChannels) {
      weight_form_dims(l.dg_form, l.cin, l.cout, &N, &K);
      l.dg8 = (uint8_t*)al(l.numel);
      l.dg8s = (float*)al((size_t)N * 4);
      if (!l.dg8 || !l.dg8s) {
        *err = "cudaMalloc(weight forms) failed";
        return false;
      }
    }
  }
  return true;
}

cudaError_t NetWeights::reform(cudaStream_t st) {
  for (auto& l : layers) {
    cudaError_t e = launch_weight_form_padded(l.fwd_form, l.cin, l.cout, l.pcin, l.pcout,
                                              master + l.off, l.fwd32, l.fwd16, l.fwdh, st);
    if (e != cudaSuccess) return e;
    e = launch_weight_form_padded(l.dg_form, l.cin, l.cout, l.pcin, l.pcout, master + l.off,
                                  l.dg32, l.dg16, l.dgh, st);
    if (e != cudaSuccess) return e;
    int N, K;
    if (l.i2c_fwd_h) {
      weight_form_dims_padded(l.fwd_form, l.cin, l.cout, l.pcin, l.pcout, &N, &K);
      if ((e = launch_i2c_weights(l.fwd32, N, K, l.i2c_fwd_h, l.i2c_fwd_b, st)) != cudaSuccess)
        return e;
    }
    if (l.i2c_dg_h) {
      weight_form_dims_padded(l.dg_form, l.cin, l.cout, l.pcin, l.pcout, &N, &K);
      if ((e = launch_i2c_weights(l.dg32, N, K, l.i2c_dg_h, l.i2c_dg_b, st)) != cudaSuccess)
        return e;
    }
    if (l.fwd8) {
      weight_form_dims(l.fwd_form, l.cin, l.cout, &N, &K);
      if ((e = launch_weight_fp8(l.fwd32, N, K, l.fwd8, l.fwd8s, st)) != cudaSuccess) return e;
    }
    if (l.dg8) {
      weight_form_dims(l.dg_form, l.cin, l.cout, &N, &K);
      if ((e = launch_weight_fp8(l.dg32, N, K, l.dg8, l.dg8s, st)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t NetWeights::upload(const float* dev_weights, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(master, dev_weights, nparams * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return reform(st);
}

// ------------------------------------------------------------------ plans

NetPlan::~NetPlan() {
  for (auto& s : fwd)
    if (s.tc) tc_plan_destroy(s.tc);
  for (auto& s : vjp)
    if (s.tc) tc_plan_destroy(s.tc);
  for (void* p : allocs) cudaFree(p);
}

void* NetPlan::alloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(256, (bytes + 255) & ~(size_t)255)) != cudaSuccess)
    return nullptr;
  allocs.push_back(p);
  return p;
}

namespace {

struct Builder {
  NetPlan* P;
  std::string* err;
  bool ok = true;
  int eb;  // activation element bytes

  void* act(int h, int w, int c) {
    void* p = P->alloc((size_t)P->n * h * w * c * eb);
    if (!p) ok = false;
    return p;
  }

  // Append one conv of `layer` (forward or input-gradient form).
  // The image-side input conv (3x3, f32 planar image in, 16-bit NHWC features out,
  // K = 9 c <= 32) on the tensor cores: an im2col pass writes one 32-channel row per
  // pixel, then a 1x1 narrow-row tcgen05 conv with the [N][32] weight form.  False
  // (step unchanged) where that form or the tensor-core path does not apply.
  bool i2c_step(Step& s, const Layer& L, bool dgrad, int adt) {
    ConvArgs& a = s.a;
    if (adt == DT_F32 || !a.in_nchw || a.out_nchw || a.mode != CM_CONV3 ||
        a.outmap != OM_IDENT || 9 * a.Cin > 32)
      return false;
    // read at plan build: IDEQ_IMG_TC=1 selects this form; by default the SIMT edge
    // kernels run these layers (this form's speed is not measured yet)
    const char* env = std::getenv("IDEQ_IMG_TC");
    const bool on = env && *env && std::atoi(env) == 1;
    const __half* wh = dgrad ? L.i2c_dg_h : L.i2c_fwd_h;
    const __nv_bfloat16* wb = dgrad ? L.i2c_dg_b : L.i2c_fwd_b;
    if (!on || !wh || !wb) return false;
    ConvArgs b = a;
    b.mode = CM_PIX;
    b.Cin = 32;
    b.in_nchw = 0;
    b.k_algo = 9 * a.Cin;
    b.wB = adt == DT_F16 ? (const void*)wh : (const void*)wb;
    const long long px = (long long)P->n * a.H * a.W;
    if (!tc_supported(b, adt)) return false;  // (b.in is replaced by the im2col rows below)
    void* buf = P->alloc((size_t)px * 32 * 2);
    if (!buf) return false;
    b.in = buf;
    std::string e;
    TcPlan* tc = tc_plan_create(b, adt, adt, &e);
    if (!tc) return false;
    s.i2c_px = px;
    s.i2c_src = (const float*)a.in;
    s.i2c_dst = buf;
    s.i2c_c = a.Cin;
    s.i2c_H = a.H;
    s.i2c_W = a.W;
    s.in_dt = adt;
    s.tc = tc;
    a = b;
    return true;
  }

  void conv(std::vector<Step>& list, const Layer& L, bool dgrad, int mode, int outmap, int gh,
            int gw, int cin, int cout, const void* in, void* out, int epi,
            const void* aux0 = nullptr, void* out2 = nullptr, bool in_nchw = false,
            bool out_nchw = false, float sign = -1.f, double* sumsq = nullptr,
            const void* aux1 = nullptr, const void* aux2 = nullptr) {
    Step s;
    ConvArgs& a = s.a;
    a.mode = mode;
    a.outmap = outmap;
    a.epi = epi;
    a.act = P->w->desc.act == IDEQ_ACT_RELU ? 1 : 0;
    a.n = P->n;
    a.H = gh;
    a.W = gw;
    a.Cin = cin;
    a.Cout = cout;
    a.in_nchw = in_nchw;
    a.out_nchw = out_nchw;
    a.sign = sign;
    a.in = in;
    a.out = out;
    a.out2 = out2;
    a.aux0 = aux0;
    a.aux1 = aux1;
    a.aux2 = aux2;
    a.sumsq = sumsq;
    a.skip = P->skip;
    const int prec = P->prec;
    const int adt = prec == IDEQ_FP32
                        ? DT_F32
                        : ((prec == IDEQ_FP16 || prec == IDEQ_FP16_FP8) ? DT_F16 : DT_BF16);
    const bool fp8_form = prec == IDEQ_BF16_FP8 || prec == IDEQ_FP16_FP8;
    s.in_dt = in_nchw ? DT_F32 : adt;
    s.out_dt = out_nchw ? DT_F32 : adt;
    const uint8_t* w8 = dgrad ? L.dg8 : L.fwd8;
    const float* w8s = dgrad ? L.dg8s : L.fwd8s;
    bool use8 = fp8_form && !in_nchw && !out_nchw && w8 && cin >= kFp8MinChannels;
    if (use8) {  // e4m3 operands: quantise the 16-bit input first
      const long long in_px = mode == CM_DOWN ? 4LL * P->n * gh * gw : (long long)P->n * gh * gw;
      s.quant_n = in_px * cin;
      s.q_src = in;
      s.q_dst = (uint8_t*)P->alloc((size_t)s.quant_n);
      float* sc = (float*)P->alloc(8);
      if (!s.q_dst || !sc) {
        ok = false;
        return;
      }
      s.q_amax = sc;
      s.q_scale = sc + 1;
      a.in = s.q_dst;
      a.wB = w8;
      a.a_scale = s.q_scale;
      a.w_scale = w8s;
      use8 = tc_supported(a, DT_FP8);
      if (!use8) {
        s.quant_n = 0;
        a.in = in;
        a.a_scale = a.w_scale = nullptr;
      }
    }
    if (use8) {
      std::string e;
      s.tc = tc_plan_create(a, DT_FP8, adt, &e);
      if (!s.tc) {
        *err = e;
        ok = false;
      }
    } else if (i2c_step(s, L, dgrad, adt)) {  // image -> feature side, as im2col + 1x1
    } else if (adt != DT_F32 && !in_nchw && tc_supported(a)) {  // incl. feature -> image
      if (adt == DT_F16)
        a.wB = dgrad ? (const void*)L.dgh : (const void*)L.fwdh;
      else
        a.wB = dgrad ? (const void*)L.dg16 : (const void*)L.fwd16;
      std::string e;
      s.tc = tc_plan_create(a, adt, adt, &e);
      if (!s.tc) {
        *err = e;
        ok = false;
      }
    } else {
      a.wB = dgrad ? (const void*)L.dg32 : (const void*)L.fwd32;
      s.edge = edge_supported(a);
    }
    list.push_back(s);
  }
};

}  // namespace

bool NetPlan::build(NetWeights* wts, int n_, int H_, int W_, int prec_, double* gsum_,
                    std::string* err, const int* skip_) {
  w = wts;
  skip = skip_;
  n = n_;
  c = wts->desc.in_ch;
  H = H_;
  W = W_;
  prec = prec_;
  gsum = gsum_;
  const ideq_net_desc& d = wts->desc;
  Builder B{this, err, true, prec == IDEQ_FP32 ? 4 : 2};  // activation element bytes
  const size_t img_bytes = (size_t)n * c * H * W * 4;
  z = (float*)alloc(img_bytes);
  r = (float*)alloc(img_bytes);
  grad = (float*)alloc(img_bytes);
  if (!z || !r || !grad) {
    *err = "cudaMalloc(plan images) failed";
    return false;
  }
  const auto& Ls = wts->layers;
  size_t li = 0;
  auto next = [&]() -> const Layer& { return Ls[li++]; };

  if (d.kind == IDEQ_NET_CNN) {
    const int D = d.depth;
    std::vector<void*> a(D), s(D);
    for (int i = 0; i + 1 < D; ++i) {
      a[i] = B.act(H, W, Ls[i].pcout);
      s[i] = B.act(H, W, Ls[i].pcout);
    }
    // forward
    for (int i = 0; i < D; ++i) {
      const Layer& L = Ls[i];
      const bool first = i == 0, last = i == D - 1;
      const void* in = first ? (const void*)z : a[i - 1];
      if (last)
        B.conv(fwd, L, false, CM_CONV3, OM_IDENT, H, W, L.pcin, L.pcout, in, r, EP_AXPY_NCHW, z,
               nullptr, first, true, -1.f, gsum);
      else
        B.conv(fwd, L, false, CM_CONV3, OM_IDENT, H, W, L.pcin, L.pcout, in, a[i], EP_ACT,
               nullptr, s[i], first);
    }
    // reverse: d_h(i-1) = s(i-1) . conv_i^T(d_h(i)); the first conv's transpose forms grad
    std::vector<void*> dh(D);
    for (int i = 0; i + 1 < D; ++i) dh[i] = B.act(H, W, Ls[i].pcout);
    for (int i = D - 1; i >= 0; --i) {
      const Layer& L = Ls[i];
      const bool last = i == D - 1, first = i == 0;
      const void* in = last ? (const void*)r : dh[i];
      if (first)
        B.conv(vjp, L, true, CM_CONV3, OM_IDENT, H, W, L.pcout, L.pcin, in, grad, EP_AXPY_NCHW,
               r, nullptr, last, true, -1.f, nullptr);
      else
        B.conv(vjp, L, true, CM_CONV3, OM_IDENT, H, W, L.pcout, L.pcin, in, dh[i - 1], EP_MUL,
               s[i - 1], nullptr, last, false);
    }
  } else {
    const int Lv = d.n_levels, R = d.n_rb;
    if (H % (1 << (Lv - 1)) != 0 || W % (1 << (Lv - 1)) != 0) {
      *err = "U-Net needs H and W divisible by 2^(n_levels-1)";
      return false;
    }
    auto Hl = [&](int l) { return H >> l; };
    auto Wl = [&](int l) { return W >> l; };
    auto Cl = [&](int l) { return d.widths[l]; };
    struct RB { void *a, *s, *o; };
    std::vector<std::vector<RB>> enc(Lv), dec(Lv);
    std::vector<void*> skip(Lv, nullptr), down_out(Lv, nullptr), up_out(Lv, nullptr);
    std::vector<const Layer*> encL, decL;  // c1,c2 per rb in order
    const Layer& head = next();
    void* h0 = B.act(H, W, Cl(0));
    B.conv(fwd, head, false, CM_CONV3, OM_IDENT, H, W, c, Cl(0), z, h0, EP_STORE, nullptr,
           nullptr, true, false);
    std::vector<std::vector<std::pair<const Layer*, const Layer*>>> encW(Lv), decW(Lv);
    std::vector<const Layer*> downW(Lv, nullptr), upW(Lv, nullptr);
    std::vector<const void*> enc_in(Lv, nullptr), dec_in(Lv, nullptr);

    auto rbs_fwd = [&](int l, const void* x, std::vector<RB>& rb,
                       std::vector<std::pair<const Layer*, const Layer*>>& lw) -> const void* {
      for (int i = 0; i < R; ++i) {
        const Layer& c1 = next();
        const Layer& c2 = next();
        lw.push_back({&c1, &c2});
        RB b{B.act(Hl(l), Wl(l), Cl(l)), B.act(Hl(l), Wl(l), Cl(l)), B.act(Hl(l), Wl(l), Cl(l))};
        B.conv(fwd, c1, false, CM_CONV3, OM_IDENT, Hl(l), Wl(l), Cl(l), Cl(l), x, b.a, EP_ACT,
               nullptr, b.s);
        B.conv(fwd, c2, false, CM_CONV3, OM_IDENT, Hl(l), Wl(l), Cl(l), Cl(l), b.a, b.o, EP_ADD,
               x);
        rb.push_back(b);
        x = b.o;
      }
      return x;
    };

    const void* x = h0;
    for (int l = 0; l < Lv - 1; ++l) {
      enc_in[l] = x;
      x = rbs_fwd(l, x, enc[l], encW[l]);
      skip[l] = const_cast<void*>(x);
      const Layer& dn = next();
      downW[l] = &dn;
      down_out[l + 1] = B.act(Hl(l + 1), Wl(l + 1), Cl(l + 1));
      B.conv(fwd, dn, false, CM_DOWN, OM_IDENT, Hl(l + 1), Wl(l + 1), Cl(l), Cl(l + 1), x,
             down_out[l + 1], EP_STORE);
      x = down_out[l + 1];
    }
    enc_in[Lv - 1] = x;
    x = rbs_fwd(Lv - 1, x, enc[Lv - 1], encW[Lv - 1]);  // coarsest scale
    for (int l = Lv - 2; l >= 0; --l) {
      const Layer& up = next();
      upW[l] = &up;
      up_out[l] = B.act(Hl(l), Wl(l), Cl(l));
      // transposed conv as a pixelwise GEMM on the coarse grid, scattered 2x2,
      // plus the encoder skip of this scale
      B.conv(fwd, up, false, CM_PIX, OM_D2S, Hl(l + 1), Wl(l + 1), Cl(l + 1), Cl(l), x, up_out[l],
             EP_ADD, skip[l]);
      dec_in[l] = up_out[l];
      x = rbs_fwd(l, up_out[l], dec[l], decW[l]);
    }
    const Layer& tail = next();
    B.conv(fwd, tail, false, CM_CONV3, OM_IDENT, H, W, Cl(0), c, x, r, EP_AXPY_NCHW, z, nullptr,
           false, true, -1.f, gsum);

    // ---- reverse pass
    std::vector<void*> dA(Lv), dB(Lv), tb(Lv);
    for (int l = 0; l < Lv; ++l) {
      dA[l] = B.act(Hl(l), Wl(l), Cl(l));
      dB[l] = B.act(Hl(l), Wl(l), Cl(l));
      tb[l] = B.act(Hl(l), Wl(l), Cl(l));
    }
    // cotangent buffer ping-pong per level: returns the buffer holding the result
    auto rbs_rev = [&](int l, void* dcur, std::vector<RB>& rb,
                       std::vector<std::pair<const Layer*, const Layer*>>& lw) -> void* {
      for (int i = R - 1; i >= 0; --i) {
        void* dnext = (dcur == dA[l]) ? dB[l] : dA[l];
        // t = s . conv2^T(d);  d' = d + conv1^T(t)
        B.conv(vjp, *lw[i].second, true, CM_CONV3, OM_IDENT, Hl(l), Wl(l), Cl(l), Cl(l), dcur,
               tb[l], EP_MUL, rb[i].s);
        B.conv(vjp, *lw[i].first, true, CM_CONV3, OM_IDENT, Hl(l), Wl(l), Cl(l), Cl(l), tb[l],
               dnext, EP_ADD, dcur);
        dcur = dnext;
      }
      return dcur;
    };
    // tail^T: r (f32 NCHW) -> d at scale 0
    B.conv(vjp, tail, true, CM_CONV3, OM_IDENT, H, W, c, Cl(0), r, dA[0], EP_STORE, nullptr,
           nullptr, true, false);
    void* dcur = dA[0];
    std::vector<void*> dskip(Lv, nullptr);
    for (int l = 0; l <= Lv - 2; ++l) {
      dcur = rbs_rev(l, dcur, dec[l], decW[l]);
      dskip[l] = dcur;  // cotangent of (up + skip) flows to the skip unchanged
      // up^T: stride-2 gather on the fine grid -> coarse cotangent
      void* dn = dA[l + 1];
      B.conv(vjp, *upW[l], true, CM_DOWN, OM_IDENT, Hl(l + 1), Wl(l + 1), Cl(l), Cl(l + 1), dcur,
             dn, EP_STORE);
      dcur = dn;
    }
    dcur = rbs_rev(Lv - 1, dcur, enc[Lv - 1], encW[Lv - 1]);
    for (int l = Lv - 2; l >= 0; --l) {
      // down^T: pixelwise GEMM on the coarse grid scattered 2x2, plus the skip cotangent.
      // dskip[l] lives in dA[l] or dB[l]; write into the other one.
      void* dst = (dskip[l] == dA[l]) ? dB[l] : dA[l];
      B.conv(vjp, *downW[l], true, CM_PIX, OM_D2S, Hl(l + 1), Wl(l + 1), Cl(l + 1), Cl(l), dcur,
             dst, EP_ADD, dskip[l]);
      dcur = rbs_rev(l, dst, enc[l], encW[l]);
    }
    B.conv(vjp, head, true, CM_CONV3, OM_IDENT, H, W, Cl(0), c, dcur, grad, EP_AXPY_NCHW, r,
           nullptr, false, true, -1.f, nullptr);
  }
  if (!B.ok) {
    if (err->empty()) *err = "cudaMalloc(plan activations) failed";
    return false;
  }
  for (auto& s : fwd) fwd_flops += s.a.flops();
  for (auto& s : vjp) vjp_flops += s.a.flops();
  return true;
}

// ------------------------------------------------------------------ execution

cudaEvent_t Profiler::next() {
  if (used == ev.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ev.push_back(e);
  }
  return ev[used++];
}

Profiler::~Profiler() {
  for (auto e : ev) cudaEventDestroy(e);
}

cudaError_t run_steps(const std::vector<Step>& steps, int* err_flag, cudaStream_t st,
                      Profiler* prof, long long* launches) {
  for (const Step& s : steps) {
    cudaError_t e;
    if (s.quant_n > 0) {
      if ((e = cudaMemsetAsync(s.q_amax, 0, sizeof(float), st)) != cudaSuccess) return e;
      if ((e = launch_act_amax(s.q_src, s.in_dt, s.quant_n, s.q_amax, st)) != cudaSuccess)
        return e;
      if ((e = launch_act_fp8(s.q_src, s.in_dt, s.quant_n, s.q_amax, s.q_dst, s.q_scale, st)) !=
          cudaSuccess)
        return e;
      if (launches) *launches += 2;
    }
    if (s.i2c_px > 0) {  // im2col rows of the image-side input conv
      if ((e = launch_im2col3(s.a.n, s.i2c_c, s.i2c_H, s.i2c_W, s.i2c_src, s.a.skip, s.i2c_dst,
                              s.in_dt, st)) != cudaSuccess)
        return e;
      if (launches) *launches += 1;
    }
    if (s.tc) {
      const bool p = prof && prof->on;
      if (p) cudaEventRecord(prof->next(), st);
      e = launch_conv_tc(s.tc, s.a, err_flag, st);
      if (p) {
        cudaEventRecord(prof->next(), st);
        prof->flops += s.a.flops();
        prof->launches += 1;
      }
    } else if (s.edge) {
      e = launch_conv_edge(s.a, s.a.in_nchw ? s.out_dt : s.in_dt, st);
    } else {
      e = launch_conv_simt(s.a, s.in_dt, s.out_dt, st);
    }
    if (launches) *launches += 1;
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ideq
