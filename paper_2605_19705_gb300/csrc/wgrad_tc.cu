// Weight gradients of the 3x3 and stride-2 2x2 convolutions on the tcgen05
// tensor cores (sm_103a), for 16-bit (bf16 or f16) activations.
//
// For a conv with forward GEMM out[p][co] = sum_k A[p][k] B[co][k] (ConvArgs), the
// gradient of <cot, out> in B is dB[co][k] = sum_p cot[p][co] A[p][k], with
// k = tap * Cin + ci and A[p][k] the input at the tap-shifted pixel (zero outside
// the image).  Here it runs as D[k][co] = sum_p A[p][k] cot[p][co] on the tensor
// cores: M = k (128 rows per tile), N = co (64..256 columns per tile), and the
// reduction K = pixels.  Both operands keep the NHWC layout of the activations, so
// they are "MN-major" (channels contiguous for a fixed pixel): a TMA box of 64
// pixels x 64 channels lands in shared memory as 64 rows of 128 bytes under the
// 128-byte swizzle, one MN-major swizzle atom column per 64 channels.  One tile's
// 128 M rows are two such boxes -- two taps of 64 channels, or 128 channels of one
// tap -- of the tap-shifted input (the zero padding is the TMA out-of-bounds
// fill); its N columns are BN / 64 boxes of the cotangent at the same pixels.
//
// Persistent kernel, warp-specialised like the forward conv: warp 0 is the TMA
// producer, warp 1 allocates two TMEM accumulators and issues tcgen05.mma
// (M = 128, N = BN, K = 16 pixels) from one lane, warps 2..5 read the finished
// accumulator (one M row per lane) and write it to the split's partial [N][K]
// tile.  The pixel sum is split into S contiguous ranges of 64-pixel boxes; a
// work unit is (split, N tile, M tile), and the splits are summed afterwards in
// a fixed order (deterministic), scaled and added into the [N][K] accumulator.
// Every mbarrier wait is bounded (about 2 s); an expired wait sets *err.
#include <algorithm>

#include "common.cuh"
#include "ideq_internal.h"
#include "net_train.h"
#include "tc_ptx.cuh"

namespace ideq {

constexpr int WG_THREADS = 192;  // producer, MMA issuer, 4 epilogue warps
constexpr int WG_BOX = 8192;     // one 64-pixel x 64-channel 16-bit box: 64 rows of 128 B
constexpr int WG_STAGES_MAX = 6;

struct WgTcArgs {
  int mode;              // CM_CONV3 or CM_DOWN
  int Cin, N, K;         // N = Cout, K = 9 Cin (CM_CONV3) or 4 Cin (CM_DOWN)
  int Wt, Ht, tiles_w, tiles_h, nbox;  // 64-pixel boxes (Wt x Ht) of the output grid
  int bn, mt, nt, splits, stages;
  // channels per box of A (input) and B (cotangent): 64 (128-byte rows, 128-byte
  // swizzle) or 32 (64-byte rows, 64-byte swizzle, for 32-channel sides)
  int ca, cb;
  float* part;           // [splits][N][K]
  int* err;
};

struct WgTcPlan {
  CUtensorMap tmA, tmB;
  WgTcArgs a;
  dim3 grid;
  size_t smem;
  int dt;
};

// MN-major shared-memory descriptor: rows of `c` 16-bit MN elements (64: 128-byte
// rows under the 128-byte swizzle; 32: 64-byte rows under the 64-byte swizzle); a K
// step of 8 rows is one swizzle atom (stride byte offset), consecutive MN blocks of
// c elements are one box (64 rows) apart (leading byte offset).
IDEQ_DEV uint64_t umma_desc_mn(uint32_t saddr, int c) {
  const uint32_t row = 2u * (uint32_t)c, box = 64u * row;
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(box >> 4) << 16;
  d |= (uint64_t)((8u * row) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(c == 64 ? 2 : 4) << 61;
  return d;
}

// A (input) box j of M tile mt: the (tap, first channel) it starts at.
IDEQ_DEV void wg_a_box(const WgTcArgs& a, int mt, int j, int* tap, int* c0) {
  const int taps = a.mode == CM_CONV3 ? 9 : 4;
  const int m0 = mt * 128 + a.ca * j;
  int t = m0 / a.Cin;
  if (t >= taps) t = taps - 1;  // past the last tap (9 taps of 64 channels): rows never stored
  *tap = t;
  *c0 = m0 - t * a.Cin;
  if (*c0 >= a.Cin) *c0 = 0;
}

template <typename T>
__global__ void __launch_bounds__(WG_THREADS, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB, WgTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int ST = a.stages;
  const int na = 128 / a.ca;                // input boxes per stage (128 M rows)
  const int nb = a.bn / a.cb;               // cotangent boxes per stage
  const int ABOX = 128 * a.ca, BBOX = 128 * a.cb;  // bytes of one box (64 rows)
  const int STAGE = na * ABOX + nb * BBOX;   // = 16 KB + BN x 128 B
  uint64_t* bars = (uint64_t*)(smem + ST * STAGE);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * ST + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + ST);
  const uint32_t tfull0 = smem_u32(bars + 2 * ST), tempty0 = smem_u32(bars + 2 * ST + 2);
  const uint32_t drain = smem_u32(bars + 2 * ST + 4);
  const int units = a.splits * a.nt * a.mt;
  const int my_units =
      (int)blockIdx.x < units ? (units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t tcols = (uint32_t)(2 * a.bn);  // 64, 128, 256 or 512

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 4);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // unit u -> (split, N tile, M tile); units of one split (the same pixels) are
  // neighbours in the grid, so their boxes are shared through L2
  auto unit_of = [&](int i, int* sp, int* nti, int* mti) {
    const int u = (int)blockIdx.x + i * (int)gridDim.x;
    *sp = u / (a.nt * a.mt);
    const int r = u - *sp * a.nt * a.mt;
    *nti = r / a.mt;
    *mti = r - *nti * a.mt;
  };
  auto box_range = [&](int sp, int* q0, int* q1) {
    *q0 = (int)(((long long)sp * a.nbox) / a.splits);
    *q1 = (int)(((long long)(sp + 1) * a.nbox) / a.splits);
  };

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
      int g = 0;
      bool ok = true;
      for (int i = 0; i < my_units && ok; ++i) {
        int sp, nti, mti, q0, q1;
        unit_of(i, &sp, &nti, &mti);
        box_range(sp, &q0, &q1);
        int tap[4], c0[4];
        for (int j = 0; j < na; ++j) wg_a_box(a, mti, j, &tap[j], &c0[j]);
        for (int q = q0; q < q1; ++q) {
          const int s = g % ST, ph = g / ST;
          if (ph > 0 && !mbar_wait(empty0 + 8 * s, (ph - 1) & 1, a.err, 21)) {
            ok = false;
            break;
          }
          const int per = a.tiles_w * a.tiles_h;
          const int img = q / per, rr = q - img * per;
          const int y0 = (rr / a.tiles_w) * a.Ht, x0 = (rr % a.tiles_w) * a.Wt;
          mbar_expect_tx(full0 + 8 * s, (uint32_t)(STAGE));
          const uint32_t dst = smem_u32(smem + s * STAGE);
          for (int j = 0; j < na; ++j) {
            if (a.mode == CM_CONV3)
              tma_load_4d(dst + j * ABOX, &tmA, c0[j], x0 + tap[j] % 3 - 1, y0 + tap[j] / 3 - 1,
                          img, full0 + 8 * s);
            else  // stride-2 2x2: tap q = (di, dj) of the fine grid
              tma_load_5d(dst + j * ABOX, &tmA, (tap[j] & 1) * a.Cin + c0[j], x0, tap[j] >> 1,
                          y0, img, full0 + 8 * s);
          }
          for (int j = 0; j < nb; ++j)
            tma_load_4d(dst + na * ABOX + j * BBOX, &tmB, nti * a.bn + a.cb * j, x0, y0, img,
                        full0 + 8 * s);
          ++g;
        }
      }
      // no commit arrival may be outstanding when the CTA exits
      const int first = g > ST ? g - ST : 0;
      for (int i = first; i < g; ++i) {
        const int s = i % ST, ph = i / ST;
        if (ok) ok = mbar_wait(empty0 + 8 * s, ph & 1, a.err, 22);
        if (!ok) mbar_wait(full0 + 8 * s, ph & 1, a.err, 22);  // our own copies in flight
      }
    }
  } else if (warp == 1) {
    {  // the whole warp, converged: one elected lane issues (as in the conv kernel)
      // A and B both MN-major (bits 15 and 16 of the instruction descriptor)
      const uint32_t idesc = umma_idesc_16(128, a.bn, Fmt<T>::v) | (1u << 15) | (1u << 16);
      int rs = 0;  // ring slot and phase, advanced without division
      uint32_t rph = 0u;
      bool ok = true;
      for (int i = 0; i < my_units && ok; ++i) {
        int sp, nti, mti, q0, q1;
        unit_of(i, &sp, &nti, &mti);
        box_range(sp, &q0, &q1);
        const int b = i & 1, u = i >> 1;
        if (u > 0 && !mbar_wait_warp(tempty0 + 8 * b, (u - 1) & 1, a.err, 23)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t td = tmem + (uint32_t)(b * a.bn);
        for (int q = q0; q < q1; ++q) {
          const int s = rs;
          if (!mbar_wait_warp(full0 + 8 * s, rph, a.err, 24)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * STAGE);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 16 pixels (two 8-row atoms) per MMA
            const uint64_t ad = umma_desc_mn(base + (uint32_t)(32 * a.ca * kk), a.ca);
            const uint64_t bd =
                umma_desc_mn(base + (uint32_t)(na * ABOX + 32 * a.cb * kk), a.cb);
            umma_el<T>(td, ad, bd, idesc, (q > q0 || kk > 0) ? 1u : 0u);
          }
          umma_commit_el(empty0 + 8 * s);
          if (++rs == ST) {
            rs = 0;
            rph ^= 1u;
          }
        }
        if (ok) umma_commit_el(tfull0 + 8 * b);
      }
      if (!ok) {  // let every issued MMA finish before TMEM is released
        umma_commit_el(drain);
        mbar_wait_warp(drain, 0, a.err, 25);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, one M row per lane
    const int q = warp & 3;
    bool ok = true;
    for (int i = 0; i < my_units && ok; ++i) {
      int sp, nti, mti, q0, q1;
      unit_of(i, &sp, &nti, &mti);
      box_range(sp, &q0, &q1);
      const int b = i & 1, u = i >> 1;
      ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * b, u & 1, a.err, 26));
      if (!ok) break;
      tc_fence_after();
      const int m = mti * 128 + 32 * q + lane;
      const bool valid = m < a.K;  // rows past K (a box past the 9th tap) hold no entry
      float* dst = a.part + ((size_t)sp * a.N + (size_t)nti * a.bn) * a.K + m;
      const bool empty_range = q1 <= q0;  // no pixels: the accumulator was never written
      for (int c = 0; c < a.bn; c += 32) {
        float v[32];
        tmem_ld32(tmem + (uint32_t)(b * a.bn + c) + ((uint32_t)(32 * q) << 16), v);
        if (valid) {
#pragma unroll
          for (int t = 0; t < 32; ++t) dst[(size_t)(c + t) * a.K] = empty_range ? 0.f : v[t];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols)
                 : "memory");
  }
}

// ------------------------------------------------------------------ host side

static bool wg_encode(CUtensorMap* m, CUtensorMapDataType dt, int rank, const void* base,
                      const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box,
                      bool narrow) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(m, dt, rank, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE,
             narrow ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// channels of one operand box: 64, or 32 for a side of exactly 32 channels
static int wg_box_ch(int c) { return c % 64 == 0 ? 64 : 32; }

bool wgrad_tc_supported(const ConvArgs& a, int in_dt, int cot_dt) {
  if (in_dt != cot_dt || (in_dt != DT_BF16 && in_dt != DT_F16)) return false;
  if (a.in_nchw || a.out_nchw || a.outmap != OM_IDENT) return false;
  if (a.mode != CM_CONV3 && a.mode != CM_DOWN) return false;
  if (!(a.Cin % 64 == 0 || a.Cin == 32) || !(a.Cout % 64 == 0 || a.Cout == 32)) return false;
  if (a.M() == 0) return false;
  return true;
}

static int wg_bn(int N) {
  if (N % 256 == 0) return 256;
  if (N % 128 == 0) return 128;
  if (N % 64 == 0) return 64;
  return 32;
}

int wgrad_tc_splits(const ConvArgs& a) {
  int wt = 1;
  while (wt < a.W && wt < 64) wt <<= 1;
  const int ht = 64 / wt;
  const long long nbox = (long long)a.n * ((a.H + ht - 1) / ht) * ((a.W + wt - 1) / wt);
  const int mt = (a.K() + 127) / 128, nt = a.N() / wg_bn(a.N());
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  long long s = std::max(1, sms / (mt * nt));
  if (s > nbox) s = nbox;
  return (int)s;
}

WgTcPlan* wgrad_tc_plan_create(const ConvArgs& a, int dt, const void* in, const void* cot,
                               float* part) {
  WgTcPlan* p = new WgTcPlan();
  WgTcArgs& t = p->a;
  p->dt = dt;
  t.mode = a.mode;
  t.Cin = a.Cin;
  t.N = a.N();
  t.K = a.K();
  int wt = 1;
  while (wt < a.W && wt < 64) wt <<= 1;
  t.Wt = wt;
  t.Ht = 64 / wt;
  t.tiles_w = (a.W + t.Wt - 1) / t.Wt;
  t.tiles_h = (a.H + t.Ht - 1) / t.Ht;
  t.nbox = a.n * t.tiles_w * t.tiles_h;
  t.bn = wg_bn(t.N);
  t.mt = (t.K + 127) / 128;
  t.nt = t.N / t.bn;
  t.splits = wgrad_tc_splits(a);
  t.part = part;
  t.ca = wg_box_ch(a.Cin);
  t.cb = wg_box_ch(a.Cout);
  const size_t stage = (size_t)WG_BOX * 2 + (size_t)t.bn * 128;
  const size_t fixed = 1024 + (2 * WG_STAGES_MAX + 5) * 8 + 16;
  t.stages = WG_STAGES_MAX;
  while (t.stages > 2 && fixed + t.stages * stage > 227 * 1024) --t.stages;
  p->smem = 1024 + t.stages * stage + (2 * t.stages + 5) * 8 + 16;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int units = t.splits * t.nt * t.mt;
  p->grid = dim3((unsigned)std::max(1, std::min(units, sms > 0 ? sms : 148)), 1, 1);
  const CUtensorMapDataType mdt =
      dt == DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  bool ok;
  if (a.mode == CM_DOWN) {  // fine input 2H x 2W viewed as [n][H][di][W][dj * Cin + ci]
    const cuuint64_t Hi = 2 * (cuuint64_t)a.H, Wi = 2 * (cuuint64_t)a.W, C = a.Cin;
    cuuint64_t dims[5] = {2 * C, (cuuint64_t)a.W, 2, (cuuint64_t)a.H, (cuuint64_t)a.n};
    cuuint64_t strides[4] = {2 * C * 2, Wi * C * 2, 2 * Wi * C * 2, Hi * Wi * C * 2};
    cuuint32_t box[5] = {(cuuint32_t)t.ca, (cuuint32_t)t.Wt, 1, (cuuint32_t)t.Ht, 1};
    ok = wg_encode(&p->tmA, mdt, 5, in, dims, strides, box, t.ca == 32);
  } else {
    const cuuint64_t C = a.Cin;
    cuuint64_t dims[4] = {C, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.n};
    cuuint64_t strides[3] = {C * 2, (cuuint64_t)a.W * C * 2, (cuuint64_t)a.H * a.W * C * 2};
    cuuint32_t box[4] = {(cuuint32_t)t.ca, (cuuint32_t)t.Wt, (cuuint32_t)t.Ht, 1};
    ok = wg_encode(&p->tmA, mdt, 4, in, dims, strides, box, t.ca == 32);
  }
  {
    const cuuint64_t C = a.Cout;
    cuuint64_t dims[4] = {C, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.n};
    cuuint64_t strides[3] = {C * 2, (cuuint64_t)a.W * C * 2, (cuuint64_t)a.H * a.W * C * 2};
    cuuint32_t box[4] = {(cuuint32_t)t.cb, (cuuint32_t)t.Wt, (cuuint32_t)t.Ht, 1};
    ok = ok && wg_encode(&p->tmB, mdt, 4, cot, dims, strides, box, t.cb == 32);
  }
  if (!ok) {
    delete p;
    return nullptr;
  }
  return p;
}

void wgrad_tc_plan_destroy(WgTcPlan* p) { delete p; }

template <typename T>
static cudaError_t wg_launch(const WgTcPlan* p, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  wgrad_tc_kernel<T><<<p->grid, WG_THREADS, p->smem, st>>>(p->tmA, p->tmB, p->a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad_tc(const WgTcPlan* p, float scale, float* dst, int* err,
                            cudaStream_t st) {
  WgTcPlan q = *p;
  q.a.err = err;
  cudaError_t e = p->dt == DT_BF16 ? wg_launch<__nv_bfloat16>(&q, st) : wg_launch<__half>(&q, st);
  if (e != cudaSuccess) return e;
  return launch_wgrad_reduce((long long)p->a.N * p->a.K, p->a.splits, p->a.part, scale, dst, st);
}

}  // namespace ideq
