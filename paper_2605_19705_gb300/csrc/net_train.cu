// Training plan of the regulariser network: the passes behind the implicit
// backward of App. D.1.2.
//
// With r = x - N(x) and a direction w (xdot):
//   fwd     N(x)            -> r = x - N(x)          (keeps every activation and
//                                                     softplus' = s of each block)
//   tchain  J_N(x)^T r      -> grad g = r - J_N^T r  (keeps every cotangent and,
//                                                     per block, ta = conv2^T(cot))
//   jvp     J_N(x) w        -> rdot = w - J_N w      (keeps hdot per block)
//   pchain  second-order reverse with cotangents (rdot, r):
//             xbar = J_N^T rdot + (d/dx[J_N w])^T r  -> hvp = rdot - xbar = Hess g . w
//           the softplus blocks use  hbar = s abar + s(1-s) hdot tbar  (EP_DUAL)
//   wgrad   for every conv: pcot (x) primal input + tcot (x) tangent input, which is
//           the weight gradient of <rdot, N> + <r, J_N w> (the reverse pass of the
//           dual-number map (x, w) -> (N(x), J_N(x) w)); the gradient of
//           <u, grad g_theta(x)> in theta is minus it (see ideq_solve_backward).
// Every pass has its own buffers (nothing is overwritten), so the weight
// gradients can run after all reverse passes.
#include <algorithm>
#include <cstdlib>

#include "net.h"
#include "net_train.h"

namespace ideq {

TrainPlan::~TrainPlan() {
  for (auto* L : {&fwd, &tchain, &jvp, &pchain})
    for (auto& s : *L)
      if (s.tc) tc_plan_destroy(s.tc);
  for (auto& g : wg)
    for (WgTcPlan* p : g.tc)
      if (p) wgrad_tc_plan_destroy(p);
  for (void* p : allocs) cudaFree(p);
}

void* TrainPlan::alloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(256, (bytes + 255) & ~(size_t)255)) != cudaSuccess)
    return nullptr;
  allocs.push_back(p);
  return p;
}

namespace {

struct TB {
  TrainPlan* P;
  std::string* err;
  bool ok = true;
  int eb, adt;

  void* act(int h, int w, int c) {
    void* p = P->alloc((size_t)P->n * h * w * c * eb);
    if (!p) ok = false;
    return p;
  }

  Step make(const Layer& L, bool dgrad, int mode, int outmap, int gh, int gw, int cin, int cout,
            const void* in, void* out, int epi, const void* aux0 = nullptr, void* out2 = nullptr,
            bool in_nchw = false, bool out_nchw = false, float sign = -1.f,
            double* sumsq = nullptr, const void* aux1 = nullptr, const void* aux2 = nullptr) {
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
    s.in_dt = in_nchw ? DT_F32 : adt;
    s.out_dt = out_nchw ? DT_F32 : adt;
    if (adt != DT_F32 && !in_nchw && !out_nchw && tc_supported(a)) {
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
    return s;
  }

  // weight-gradient record of the forward conv `f` (its ConvArgs give geometry
  // and the primal input); tin = tangent input, pcot / tcot = output cotangents
  void wg(const Layer& L, const Step& f, const void* tin, const void* pcot, const void* tcot) {
    WgStep w;
    w.layer = (int)(&L - P->w->layers.data());
    w.a = f.a;
    w.in_dt = f.in_dt;
    w.cot_dt = f.out_dt;
    w.tin = tin;
    w.pcot = pcot;
    w.tcot = tcot;
    P->wg.push_back(w);
  }
};

}  // namespace

bool TrainPlan::build(NetWeights* wts, int n_, int H_, int W_, int prec_, double* gsum_,
                      std::string* err, bool warm_) {
  w = wts;
  warm = warm_;
  n = n_;
  c = wts->desc.in_ch;
  H = H_;
  W = W_;
  prec = prec_;
  gsum = gsum_;
  const ideq_net_desc& d = wts->desc;
  // training runs the 16-bit form of the FP8 precisions
  const int adt = prec == IDEQ_FP32
                      ? DT_F32
                      : ((prec == IDEQ_FP16 || prec == IDEQ_FP16_FP8) ? DT_F16 : DT_BF16);
  TB B{this, err, true, adt == DT_F32 ? 4 : 2, adt};
  const size_t img = (size_t)n * c * H * W * 4;
  z = (float*)alloc(img);
  r = (float*)alloc(img);
  grad = (float*)alloc(img);
  zd = (float*)alloc(img);
  rd = (float*)alloc(img);
  hvp = (float*)alloc(img);
  if (!z || !r || !grad || !zd || !rd || !hvp) {
    *err = "cudaMalloc(train images) failed";
    return false;
  }
  out_img = r;
  cot_img = r;
  if (warm) {
    out_img = hvp;  // x0 = z + W(z)
    cot_img = grad; // dl/dx0, written by the loss kernel
    if (d.kind != IDEQ_NET_CNN) {
      *err = "the warm start is a plain conv net";
      return false;
    }
  }
  const auto& Ls = wts->layers;

  if (d.kind == IDEQ_NET_CNN) {
    const int D = d.depth;
    if (D < 2) {
      *err = "training plan needs depth >= 2";
      return false;
    }
    // per hidden layer i < D-1: a (act out), s (act'), ad (tangent of a), hd (pre-act tangent),
    // ta/tc: t-chain raw / scaled cotangent, pa/pc: p-chain raw / scaled cotangent
    std::vector<void*> a(D), s(D), ad(D), hd(D), ta(D), tcv(D), pa(D), pcv(D);
    for (int i = 0; i + 1 < D; ++i) {
      const int C = Ls[i].pcout;  // stored (padded) channels
      a[i] = B.act(H, W, C);
      s[i] = B.act(H, W, C);
      ad[i] = B.act(H, W, C);
      hd[i] = B.act(H, W, C);
      ta[i] = B.act(H, W, C);
      tcv[i] = B.act(H, W, C);
      pa[i] = B.act(H, W, C);
      pcv[i] = B.act(H, W, C);
    }
    std::vector<Step> fsteps(D);
    for (int i = 0; i < D; ++i) {
      const Layer& L = Ls[i];
      const bool first = i == 0, last = i == D - 1;
      const void* in = first ? (const void*)z : a[i - 1];
      const void* tin = first ? (const void*)zd : ad[i - 1];
      if (last) {
        fsteps[i] = B.make(L, false, CM_CONV3, OM_IDENT, H, W, L.pcin, L.pcout, in, out_img,
                           EP_AXPY_NCHW, z, nullptr, first, true, warm ? 1.f : -1.f,
                           warm ? nullptr : gsum);
        jvp.push_back(B.make(L, false, CM_CONV3, OM_IDENT, H, W, L.pcin, L.pcout, tin, rd,
                             EP_AXPY_NCHW, zd, nullptr, first, true, -1.f, nullptr));
      } else {
        fsteps[i] = B.make(L, false, CM_CONV3, OM_IDENT, H, W, L.pcin, L.pcout, in, a[i], EP_ACT,
                           nullptr, s[i], first);
        jvp.push_back(B.make(L, false, CM_CONV3, OM_IDENT, H, W, L.pcin, L.pcout, tin, ad[i],
                             EP_MUL_KEEP, s[i], hd[i], first));
      }
      fwd.push_back(fsteps[i]);
    }
    // reverse chains: layer i's input-gradient conv maps the cotangent of its
    // output to the raw cotangent of a[i-1]; the epilogue multiplies by s[i-1]
    // (t-chain, keeping the raw value) or adds the second-order term (p-chain).
    for (int i = D - 1; i >= 0; --i) {
      const Layer& L = Ls[i];
      const bool last = i == D - 1, first = i == 0;
      const void* tin = last ? (const void*)cot_img : tcv[i];
      const void* pin = last ? (const void*)rd : pcv[i];
      if (first && warm) {
        // the warm start needs no input gradient: the chain ends at layer 1
      } else if (first) {
        tchain.push_back(B.make(L, true, CM_CONV3, OM_IDENT, H, W, L.pcout, L.pcin, tin, grad,
                                EP_AXPY_NCHW, r, nullptr, last, true, -1.f, nullptr));
        pchain.push_back(B.make(L, true, CM_CONV3, OM_IDENT, H, W, L.pcout, L.pcin, pin, hvp,
                                EP_AXPY_NCHW, rd, nullptr, last, true, -1.f, nullptr));
      } else {
        tchain.push_back(B.make(L, true, CM_CONV3, OM_IDENT, H, W, L.pcout, L.pcin, tin, tcv[i - 1],
                                EP_MUL_KEEP, s[i - 1], ta[i - 1], last, false));
        pchain.push_back(B.make(L, true, CM_CONV3, OM_IDENT, H, W, L.pcout, L.pcin, pin, pcv[i - 1],
                                EP_DUAL, s[i - 1], nullptr, last, false, -1.f, nullptr, hd[i - 1],
                                ta[i - 1]));
      }
      // weight gradient of layer i: output cotangents (pchain, tchain) x inputs
      const void* pcot = last ? (const void*)rd : pcv[i];
      const void* tcot = last ? (const void*)cot_img : tcv[i];
      B.wg(L, fsteps[i], first ? (const void*)zd : ad[i - 1], pcot, tcot);
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
    // a value of the forward graph with its four companions
    struct V {
      void *p, *t, *tc, *pc;  // primal, tangent, t-chain cotangent, p-chain cotangent
    };
    auto val = [&](int l) { return V{B.act(Hl(l), Wl(l), Cl(l)), B.act(Hl(l), Wl(l), Cl(l)),
                                     B.act(Hl(l), Wl(l), Cl(l)), B.act(Hl(l), Wl(l), Cl(l))}; };
    struct Blk {
      const Layer *c1, *c2;
      int l;
      V x, o;                       // block input and output
      void *a, *s, *ad, *hd;        // activation, act', their tangents
      void *ta, *th, *pa, *ph;      // raw / scaled cotangents at the activation
      Step f1, f2;
    };
    size_t li = 0;
    auto next = [&]() -> const Layer& { return Ls[li++]; };
    const Layer& head = next();
    V h0 = val(0);
    Step fhead = B.make(head, false, CM_CONV3, OM_IDENT, H, W, c, Cl(0), z, h0.p, EP_STORE,
                        nullptr, nullptr, true, false);
    fwd.push_back(fhead);
    jvp.push_back(B.make(head, false, CM_CONV3, OM_IDENT, H, W, c, Cl(0), zd, h0.t, EP_STORE,
                         nullptr, nullptr, true, false));
    std::vector<std::vector<Blk>> enc(Lv), dec(Lv);
    auto blocks_fwd = [&](int l, V x, std::vector<Blk>& out) -> V {
      for (int i = 0; i < R; ++i) {
        Blk b;
        b.c1 = &next();
        b.c2 = &next();
        b.l = l;
        b.x = x;
        const int h = Hl(l), wd = Wl(l), C = Cl(l);
        b.a = B.act(h, wd, C);
        b.s = B.act(h, wd, C);
        b.ad = B.act(h, wd, C);
        b.hd = B.act(h, wd, C);
        b.ta = B.act(h, wd, C);
        b.th = B.act(h, wd, C);
        b.pa = B.act(h, wd, C);
        b.ph = B.act(h, wd, C);
        b.o = val(l);
        b.f1 = B.make(*b.c1, false, CM_CONV3, OM_IDENT, h, wd, C, C, x.p, b.a, EP_ACT, nullptr,
                      b.s);
        b.f2 = B.make(*b.c2, false, CM_CONV3, OM_IDENT, h, wd, C, C, b.a, b.o.p, EP_ADD, x.p);
        fwd.push_back(b.f1);
        fwd.push_back(b.f2);
        jvp.push_back(B.make(*b.c1, false, CM_CONV3, OM_IDENT, h, wd, C, C, x.t, b.ad,
                             EP_MUL_KEEP, b.s, b.hd));
        jvp.push_back(B.make(*b.c2, false, CM_CONV3, OM_IDENT, h, wd, C, C, b.ad, b.o.t, EP_ADD,
                             x.t));
        out.push_back(b);
        x = b.o;
      }
      return x;
    };
    std::vector<V> skip(Lv), dn(Lv), up(Lv);
    std::vector<const Layer*> downW(Lv), upW(Lv);
    std::vector<Step> fdown(Lv), fup(Lv);
    V x = h0;
    for (int l = 0; l < Lv - 1; ++l) {
      x = blocks_fwd(l, x, enc[l]);
      skip[l] = x;
      downW[l] = &next();
      dn[l + 1] = val(l + 1);
      fdown[l] = B.make(*downW[l], false, CM_DOWN, OM_IDENT, Hl(l + 1), Wl(l + 1), Cl(l),
                        Cl(l + 1), x.p, dn[l + 1].p, EP_STORE);
      fwd.push_back(fdown[l]);
      jvp.push_back(B.make(*downW[l], false, CM_DOWN, OM_IDENT, Hl(l + 1), Wl(l + 1), Cl(l),
                           Cl(l + 1), x.t, dn[l + 1].t, EP_STORE));
      x = dn[l + 1];
    }
    x = blocks_fwd(Lv - 1, x, enc[Lv - 1]);
    std::vector<V> coarse_in(Lv);
    for (int l = Lv - 2; l >= 0; --l) {
      upW[l] = &next();
      coarse_in[l] = x;
      up[l] = val(l);
      fup[l] = B.make(*upW[l], false, CM_PIX, OM_D2S, Hl(l + 1), Wl(l + 1), Cl(l + 1), Cl(l), x.p,
                      up[l].p, EP_ADD, skip[l].p);
      fwd.push_back(fup[l]);
      jvp.push_back(B.make(*upW[l], false, CM_PIX, OM_D2S, Hl(l + 1), Wl(l + 1), Cl(l + 1), Cl(l),
                           x.t, up[l].t, EP_ADD, skip[l].t));
      x = blocks_fwd(l, up[l], dec[l]);
    }
    const Layer& tail = next();
    const V xlast = x;
    Step ftail = B.make(tail, false, CM_CONV3, OM_IDENT, H, W, Cl(0), c, x.p, r, EP_AXPY_NCHW, z,
                        nullptr, false, true, -1.f, gsum);
    fwd.push_back(ftail);
    jvp.push_back(B.make(tail, false, CM_CONV3, OM_IDENT, H, W, Cl(0), c, x.t, rd, EP_AXPY_NCHW,
                         zd, nullptr, false, true, -1.f, nullptr));

    // ---- reverse chains.  Block reverse (o = x + conv2(act(conv1 x))):
    //   t-chain: th = s . (ta = conv2^T cot_o);        cot_x = cot_o + conv1^T th
    //   p-chain: ph = s . conv2^T pcot_o + s(1-s) hd ta; pcot_x = pcot_o + conv1^T ph
    auto blocks_rev = [&](std::vector<Blk>& bl) {
      for (int i = (int)bl.size() - 1; i >= 0; --i) {
        Blk& b = bl[i];
        const int h = Hl(b.l), wd = Wl(b.l), C = Cl(b.l);
        tchain.push_back(B.make(*b.c2, true, CM_CONV3, OM_IDENT, h, wd, C, C, b.o.tc, b.th,
                                EP_MUL_KEEP, b.s, b.ta));
        tchain.push_back(B.make(*b.c1, true, CM_CONV3, OM_IDENT, h, wd, C, C, b.th, b.x.tc, EP_ADD,
                                b.o.tc));
        pchain.push_back(B.make(*b.c2, true, CM_CONV3, OM_IDENT, h, wd, C, C, b.o.pc, b.ph,
                                EP_DUAL, b.s, nullptr, false, false, -1.f, nullptr, b.hd, b.ta));
        pchain.push_back(B.make(*b.c1, true, CM_CONV3, OM_IDENT, h, wd, C, C, b.ph, b.x.pc, EP_ADD,
                                b.o.pc));
        B.wg(*b.c2, b.f2, b.ad, b.o.pc, b.o.tc);
        B.wg(*b.c1, b.f1, b.x.t, b.ph, b.th);
      }
    };
    // tail^T
    tchain.push_back(B.make(tail, true, CM_CONV3, OM_IDENT, H, W, c, Cl(0), r, xlast.tc, EP_STORE,
                            nullptr, nullptr, true, false));
    pchain.push_back(B.make(tail, true, CM_CONV3, OM_IDENT, H, W, c, Cl(0), rd, xlast.pc, EP_STORE,
                            nullptr, nullptr, true, false));
    B.wg(tail, ftail, xlast.t, rd, r);
    for (int l = 0; l <= Lv - 2; ++l) {
      blocks_rev(dec[l]);
      // cotangent of up[l] (= up conv output + skip) is now in up[l].tc / .pc
      tchain.push_back(B.make(*upW[l], true, CM_DOWN, OM_IDENT, Hl(l + 1), Wl(l + 1), Cl(l),
                              Cl(l + 1), up[l].tc, coarse_in[l].tc, EP_STORE));
      pchain.push_back(B.make(*upW[l], true, CM_DOWN, OM_IDENT, Hl(l + 1), Wl(l + 1), Cl(l),
                              Cl(l + 1), up[l].pc, coarse_in[l].pc, EP_STORE));
      B.wg(*upW[l], fup[l], coarse_in[l].t, up[l].pc, up[l].tc);
    }
    blocks_rev(enc[Lv - 1]);
    for (int l = Lv - 2; l >= 0; --l) {
      // down^T plus the skip cotangent (the cotangent of up[l]) into skip[l]
      tchain.push_back(B.make(*downW[l], true, CM_PIX, OM_D2S, Hl(l + 1), Wl(l + 1), Cl(l + 1),
                              Cl(l), dn[l + 1].tc, skip[l].tc, EP_ADD, up[l].tc));
      pchain.push_back(B.make(*downW[l], true, CM_PIX, OM_D2S, Hl(l + 1), Wl(l + 1), Cl(l + 1),
                              Cl(l), dn[l + 1].pc, skip[l].pc, EP_ADD, up[l].pc));
      B.wg(*downW[l], fdown[l], skip[l].t, dn[l + 1].pc, dn[l + 1].tc);
      blocks_rev(enc[l]);
    }
    tchain.push_back(B.make(head, true, CM_CONV3, OM_IDENT, H, W, Cl(0), c, h0.tc, grad,
                            EP_AXPY_NCHW, r, nullptr, false, true, -1.f, nullptr));
    pchain.push_back(B.make(head, true, CM_CONV3, OM_IDENT, H, W, Cl(0), c, h0.pc, hvp,
                            EP_AXPY_NCHW, rd, nullptr, false, true, -1.f, nullptr));
    B.wg(head, fhead, zd, h0.pc, h0.tc);
  }
  if (!B.ok) {
    if (err->empty()) *err = "cudaMalloc(train activations) failed";
    return false;
  }
  // weight-gradient workspace: splits x N x K partials and a GEMM-form accumulator;
  // tensor-core forms for the 16-bit convs that fit them (IDEQ_WGRAD_TC=0: SIMT only)
  const char* tcv = std::getenv("IDEQ_WGRAD_TC");
  const bool use_tc = !(tcv && tcv[0] == '0');
  size_t part = 0, acc = 0;
  for (auto& g : wg) {
    const bool tc = use_tc && wgrad_tc_supported(g.a, g.in_dt, g.cot_dt);
    const int sp = std::max(wgrad_splits(g.a), tc ? wgrad_tc_splits(g.a) : 1);
    part = std::max(part, (size_t)sp * g.a.N() * g.a.K());
    acc = std::max(acc, (size_t)g.a.N() * g.a.K());
  }
  wg_part = (float*)alloc(part * 4);
  wg_acc = (float*)alloc(acc * 4);
  if (!wg_part || !wg_acc) {
    *err = "cudaMalloc(wgrad workspace) failed";
    return false;
  }
  for (auto& g : wg) {
    if (!use_tc || !wgrad_tc_supported(g.a, g.in_dt, g.cot_dt)) continue;
    const void* ins[3] = {g.a.in, g.tin, g.a.in};
    const void* cots[3] = {g.pcot, g.tcot, g.tcot};
    for (int j = 0; j < 3; ++j) {
      if ((warm && j < 2) || (!warm && j == 2) || !ins[j] || !cots[j]) continue;
      g.tc[j] = wgrad_tc_plan_create(g.a, g.in_dt, ins[j], cots[j], wg_part);
      if (!g.tc[j]) {
        *err = "tensor-core weight-gradient plan failed";
        return false;
      }
    }
  }
  return true;
}

// dst (flat, PyTorch layout) += scale * gradient in the weights of
// <pcot, out(primal)> + <tcot, out(tangent)> over every conv (dual), or of
// <tcot, out(primal)> alone (plain reverse chain, e.g. the warm start).
cudaError_t TrainPlan::run_wgrad(float* dst, float scale, bool dual, cudaStream_t st,
                                 long long* launches, int* err) {
  for (const WgStep& g : wg) {
    const Layer& L = w->layers[g.layer];
    const long long nk = (long long)g.a.N() * g.a.K();
    cudaError_t e = cudaMemsetAsync(wg_acc, 0, nk * 4, st);
    if (e != cudaSuccess) return e;
    const WgTcPlan* t0 = dual ? g.tc[0] : g.tc[2];
    if (t0)
      e = launch_wgrad_tc(t0, 1.f, wg_acc, err, st);
    else
      e = launch_wgrad(g.a, g.in_dt, g.cot_dt, dual ? g.pcot : g.tcot, 1.f, wg_part, wg_acc, st);
    if (e != cudaSuccess) return e;
    if (dual) {
      if (g.tc[1]) {
        e = launch_wgrad_tc(g.tc[1], 1.f, wg_acc, err, st);
      } else {
        ConvArgs t = g.a;
        t.in = g.tin;
        e = launch_wgrad(t, g.in_dt, g.cot_dt, g.tcot, 1.f, wg_part, wg_acc, st);
      }
      if (e != cudaSuccess) return e;
    }
    // accumulate the [N][K] forward-form gradient into the PyTorch layout
    e = launch_weight_unform_padded(L.fwd_form, L.cin, L.cout, L.pcin, L.pcout, wg_acc, scale,
                                    dst + L.off, st);
    if (e != cudaSuccess) return e;
    if (launches) *launches += dual ? 5 : 3;
  }
  return cudaSuccess;
}

}  // namespace ideq
