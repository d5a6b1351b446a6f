// tcgen05 (5th-generation tensor core) implicit-GEMM convolution for sm_103a.
//
// Persistent kernel, one CTA per SM, looping over 128 x BN tiles of
// D = A * B^T (see ConvArgs):
//   warp 0      TMA producer: per K chunk of 64 channels, one box of 128 pixels
//               x 64 channels of the NHWC 16-bit (bf16 or f16) activation
//               (tap-shifted; the zero padding of the convolution is the TMA
//               out-of-bounds fill) and one box of BN x 64 weights, into a ring
//               of shared-memory stages that runs across tile boundaries.
//   warp 1      allocates 2 x BN TMEM columns (two accumulators) and issues
//               tcgen05.mma (M=128, N=BN, K=16, 16-bit x 16-bit -> f32) from one
//               elected lane; tcgen05.commit frees ring slots and hands a
//               finished accumulator to the epilogue.
//   warps 2..9  epilogue, per 64-column panel of the tile: tcgen05.ld the f32
//               accumulator (one pixel row per thread, 32 columns per warp),
//               read the auxiliary inputs (residual / skip / saved derivative)
//               from shared memory, apply the fused epilogue, write the 16-bit
//               results to shared memory, and let one thread store the panel
//               with a TMA tensor store.  The auxiliary panels are TMA-loaded
//               ahead (the next tile's while the MMAs run), the output staging
//               is double-buffered, and the accumulator is released after its
//               last read, so that the epilogue overlaps the MMAs of the next
//               tile.
// Every shared-memory matrix (operands, staging) uses the 128-byte swizzle:
// 8-row atoms of 128 B, 16-byte chunk c of row r stored at chunk c ^ (r & 7),
// which TMA writes/reads and the UMMA descriptor expects.
// Every mbarrier wait is bounded (about 2 s of %globaltimer); an expired wait
// sets *err_flag, all roles drain and the CTA returns after freeing TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "ideq_internal.h"
#include "tc_ptx.cuh"

namespace ideq {

struct TcArgs {
  int mode, outmap, epi, act;
  int n, H, W, Cin, Cout, N;
  int Wt, Ht, tiles_w, tiles_h, tiles_n, nk, cpt;
  int stages;  // ring depth
  int nout;    // staged outputs (1 or 2)
  int naux;    // auxiliary inputs (0..3)
  int nbo;     // output staging buffers (1 or 2)
  int nba;     // auxiliary staging buffers (1 or 2)
  const float* a_scale;  // FP8 operands: activation scale (device scalar)
  const float* w_scale;  // FP8 operands: weight scale per GEMM column
  int slide;             // halo form: contiguous row runs per CTA reusing row boxes
  int stream;            // streamed halo: per stage one row box and the 3 dx taps of B
  int split64;           // 64-column tiles: epilogue halves take alternate tiles
  // image-side output (BN = 16): out = aux + sign * acc, f32 planar, c <= 16 channels
  float sign;
  const float* img_aux;
  float* img_out;
  double* sumsq;
  const int* skip;  // per image, nonzero: frozen, its tiles are not computed (nullable)
  int* err;
  // direct epilogue: outputs stored and auxiliary inputs read by the epilogue
  // threads themselves (NHWC, Cout channels), no staging in shared memory
  int direct;
  void* gout0;
  void* gout1;
  const void* gaux0;
  const void* gaux1;
  const void* gaux2;
};

struct TcPlan {
  CUtensorMap tmA, tmB, tmO[2], tmX[3];
  int bn = 0, stages = 0, op_dt = DT_BF16, epi_dt = DT_BF16, nout = 1, naux = 0, nbo = 2,
      nba = 2, ms = 1;
  bool halo = false, slide = false, stream = false, nw = false;
  bool pdl = true;       // launched with programmatic stream serialisation
  bool cg2 = false;      // CTA pairs with two-SM MMAs (clusters of two)
  bool stk = false;      // halo form with stacked vertical taps (sliding row runs)
  bool direct = false;   // epilogue without shared-memory staging
  bool split64 = false;  // 64-column tiles: epilogue halves on alternate tiles
  int Wt = 0, Ht = 0, tiles_w = 0, tiles_h = 0, tiles_n = 0, nk = 0, cpt = 0;
  dim3 grid;
  size_t smem = 0;
};

constexpr int WBOX = 32 * 64;  // one warp's epilogue box: 32 rows x 32 16-bit columns

template <int EPI> struct EpiTraits {
  static constexpr int naux =
      EPI == EP_DUAL ? 3 : (EPI == EP_ADD || EPI == EP_MUL || EPI == EP_MUL_KEEP) ? 1 : 0;
  static constexpr bool out2 = EPI == EP_ACT || EPI == EP_MUL_KEEP;
};

// One value of the fused epilogue, the kind fixed at compile time (see Epi).
// softplus and its derivative share one exponential:
//   e = exp(-|v|), softplus(v) = max(v, 0) + log(1 + e),
//   logistic(v) = 1 / (1 + e) for v >= 0 and e / (1 + e) for v < 0.
template <int EPI, int ACT>
IDEQ_DEV float epi_one(float v, float x0, float x1, float x2, float& o2) {
  if (EPI == EP_ACT) {
    if (ACT == 0) {
      const float e = __expf(-fabsf(v));
      const float d = 1.f + e;
      const float rd = __fdividef(1.f, d);
      o2 = v >= 0.f ? rd : e * rd;
      return fmaxf(v, 0.f) + __logf(d);
    }
    o2 = v > 0.f ? 1.f : 0.f;
    return fmaxf(v, 0.f);
  }
  if (EPI == EP_ADD) return v + x0;
  if (EPI == EP_MUL) return v * x0;
  if (EPI == EP_MUL_KEEP) {
    o2 = v;
    return v * x0;
  }
  if (EPI == EP_DUAL) return x0 * v + x0 * (1.f - x0) * x1 * x2;
  return v;
}

// Epilogue of one warp's 32 columns of one row per thread: auxiliary values
// from the warp's staged boxes at xb (one box per input), results into the
// staging boxes at ob (the second output one box further).
template <typename T, int EPI, int ACT>
IDEQ_DEV void epi_chunk(const float (&v)[32], uint32_t xb, uint32_t ob, int row) {
  using Tr = EpiTraits<EPI>;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t off = wswz(row, c);
    float x0[8] = {}, x1[8] = {}, x2[8] = {}, r[8], r2[8] = {};
    uint4 w4;
    if (Tr::naux > 0) { lds128(xb + off, w4); unpack8<T>(w4, x0); }
    if (Tr::naux > 1) { lds128(xb + WBOX + off, w4); unpack8<T>(w4, x1); }
    if (Tr::naux > 2) { lds128(xb + 2 * WBOX + off, w4); unpack8<T>(w4, x2); }
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = epi_one<EPI, ACT>(v[8 * c + i], x0[i], x1[i], x2[i], r2[i]);
    sts128(ob + off, pack8<T>(r));
    if (Tr::out2) sts128(ob + WBOX + off, pack8<T>(r2));
  }
}

template <typename T>
IDEQ_DEV void epi_apply(int epi, int act, const float (&v)[32], uint32_t xb, uint32_t ob,
                        int row) {
  switch (epi) {
    case EP_ACT:
      if (act == 0)
        epi_chunk<T, EP_ACT, 0>(v, xb, ob, row);
      else
        epi_chunk<T, EP_ACT, 1>(v, xb, ob, row);
      break;
    case EP_ADD: epi_chunk<T, EP_ADD, 0>(v, xb, ob, row); break;
    case EP_MUL: epi_chunk<T, EP_MUL, 0>(v, xb, ob, row); break;
    case EP_MUL_KEEP: epi_chunk<T, EP_MUL_KEEP, 0>(v, xb, ob, row); break;
    case EP_DUAL: epi_chunk<T, EP_DUAL, 0>(v, xb, ob, row); break;
    default: epi_chunk<T, EP_STORE, 0>(v, xb, ob, row); break;
  }
}

struct TileCoord {
  int img, h0, w0, n0;
};

// The images a launch computes: all n, or, when the caller passes per-image skip
// flags (frozen images of a solve) and n <= 32, the nrun images whose bit is set
// in `run`, in increasing order (img(j) = the j-th set bit).
struct ImgMap {
  int nrun;
  uint32_t run;
  bool masked;
  uint64_t tbl;  // n <= 16: 4-bit image index of the j-th computed image at bits 4j..4j+3
  IDEQ_DEV int img(int j) const {
    if (!masked) return j;
    if (run < (1u << 16)) return (int)((tbl >> (4 * j)) & 15u);
    uint32_t m = run;
    for (int i = 0; i < j; ++i) m &= m - 1u;  // drop the j lowest set bits
    return __ffs(m) - 1;
  }
};
constexpr int kMaxMaskImages = 32;  // launches of more images compute every image

// The 4-bit lookup table of ImgMap for the images 0..15 set in `run`.
IDEQ_DEV uint64_t img_table(uint32_t run) {
  uint64_t t = 0;
  int j = 0;
#pragma unroll
  for (int b = 0; b < 16; ++b)
    if ((run >> b) & 1u) {
      t |= (uint64_t)b << (4 * j);
      ++j;
    }
  return t;
}

// Tile t covers MS consecutive 128-row M-tiles (sub-tiles) and BN columns of the
// computed images.  An M-tile index past the last one maps to an image index >= n,
// which the TMA loads fill with zeros and the TMA stores clip.
IDEQ_DEV TileCoord tile_coord(const TcArgs& a, const ImgMap& im, int t, int bn, int ms, int sub) {
  const int per_img = a.tiles_h * a.tiles_w;
  const int tiles_m = im.nrun * per_img;
  const int groups = (tiles_m + ms - 1) / ms;
  const int nidx = t / groups, m = (t - nidx * groups) * ms + sub;
  TileCoord c;
  const int j = m / per_img;
  c.img = j < im.nrun ? im.img(j) : a.n;
  const int rr = m - j * per_img;
  c.h0 = (rr / a.tiles_w) * a.Ht;
  c.w0 = (rr % a.tiles_w) * a.Wt;
  c.n0 = nidx * bn;
  return c;
}

constexpr int EPI_WARPS = 8;
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;
constexpr int MAX_NBA = 4;  // auxiliary staging buffers (and their barriers) per warp, at most
constexpr int PANEL = EPI_WARPS * WBOX;  // one staging buffer of one tensor, all 8 warps

// Epilogue TMA of one warp's box (load of auxiliary values, store of results):
// the 32 tile rows 32q .. 32q+31 (q = the warp's TMEM lane quadrant) and the 32
// columns starting at `col`, as a 4-D NHWC box (32 channels x min(Wt, 32) x
// 32 / min(Wt, 32) pixels), or through the 5-D depth-to-space view for OM_D2S.
// Direct form of epi_chunk: the auxiliary values of the thread's row come from
// global memory (read-only for this kernel) and the results go straight to global
// memory; every pointer is at this row's first column and 16-byte aligned.
template <typename T, int EPI, int ACT>
IDEQ_DEV void epi_chunk_g(const float (&v)[32], const T* x0p, const T* x1p, const T* x2p,
                          T* o1, T* o2) {
  using Tr = EpiTraits<EPI>;
  uint4 w0[4], w1[4], w2[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {  // all loads first: one latency for the row
    if (Tr::naux > 0) w0[c] = __ldg((const uint4*)(x0p + 8 * c));
    if (Tr::naux > 1) w1[c] = __ldg((const uint4*)(x1p + 8 * c));
    if (Tr::naux > 2) w2[c] = __ldg((const uint4*)(x2p + 8 * c));
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float x0[8] = {}, x1[8] = {}, x2[8] = {}, r[8], r2[8] = {};
    if (Tr::naux > 0) unpack8<T>(w0[c], x0);
    if (Tr::naux > 1) unpack8<T>(w1[c], x1);
    if (Tr::naux > 2) unpack8<T>(w2[c], x2);
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = epi_one<EPI, ACT>(v[8 * c + i], x0[i], x1[i], x2[i], r2[i]);
    *(uint4*)(o1 + 8 * c) = pack8<T>(r);
    if (Tr::out2) *(uint4*)(o2 + 8 * c) = pack8<T>(r2);
  }
}

template <typename T>
IDEQ_DEV void epi_apply_g(int epi, int act, const float (&v)[32], const T* x0, const T* x1,
                          const T* x2, T* o1, T* o2) {
  switch (epi) {
    case EP_ACT:
      if (act == 0)
        epi_chunk_g<T, EP_ACT, 0>(v, x0, x1, x2, o1, o2);
      else
        epi_chunk_g<T, EP_ACT, 1>(v, x0, x1, x2, o1, o2);
      break;
    case EP_ADD: epi_chunk_g<T, EP_ADD, 0>(v, x0, x1, x2, o1, o2); break;
    case EP_MUL: epi_chunk_g<T, EP_MUL, 0>(v, x0, x1, x2, o1, o2); break;
    case EP_MUL_KEEP: epi_chunk_g<T, EP_MUL_KEEP, 0>(v, x0, x1, x2, o1, o2); break;
    case EP_DUAL: epi_chunk_g<T, EP_DUAL, 0>(v, x0, x1, x2, o1, o2); break;
    default: epi_chunk_g<T, EP_STORE, 0>(v, x0, x1, x2, o1, o2); break;
  }
}

IDEQ_DEV void epi_tma(bool store, const TcArgs& a, const CUtensorMap* tm, uint32_t sm,
                      const TileCoord& tc, int q, int col, uint32_t bar) {
  const int m0 = 32 * q;
  const int w = tc.w0 + m0 % a.Wt, h = tc.h0 + m0 / a.Wt;
  if (a.outmap == OM_D2S) {
    const int sp = col / a.Cout, co = col - sp * a.Cout;
    const int c0 = (sp & 1) * a.Cout + co, di = sp >> 1;
    if (store)
      tma_store_5d(tm, sm, c0, w, di, h, tc.img);
    else
      tma_load_5d(sm, tm, c0, w, di, h, tc.img, bar);
  } else {
    if (store)
      tma_store_4d(tm, sm, col, w, h, tc.img);
    else
      tma_load_4d(sm, tm, col, w, h, tc.img, bar);
  }
}

// Halo form of the 3x3 conv (one tile = 128 pixels of one image row, all N
// columns): per channel chunk the producer loads three 130-pixel row boxes
// (rows y-1, y, y+1, pixels x0-1 .. x0+128) once, and the nine taps read them
// through descriptors shifted by dx rows; the whole weight matrix stays
// resident in shared memory.  A is fetched once instead of nine times.
constexpr int HALO_ROWS = 130;
constexpr int HALO_BOX = 17408;  // 130 rows x 128 B, rounded up to a 1024-B atom
constexpr int HALO_BOX_NW = 9216;  // 130 rows x 64 B (narrow rows), rounded the same way
constexpr int HALO_PF = 4;       // rows prefetched into L2 ahead of the row being loaded

// Halo form: tile t -> row t % tiles_h of 128-pixel column strip t / tiles_h
// (strips in (image, strip) order); the ring holds single row boxes and a tile
// reads three of them.  Tiles stride the grid (neighbouring CTAs work on
// neighbouring rows, so most row boxes are still in L2 when the second and third
// CTA need them), or, in the sliding form, each CTA runs a contiguous range of
// rows and a tile that continues its run loads only row y+1, reusing y-1 and y
// (measured slower on the U-Net's 64-channel layers: 90 vs 60 us).
IDEQ_DEV TileCoord halo_coord(const TcArgs& a, const ImgMap& im, int t) {
  const int strip = t / a.tiles_h;
  TileCoord c;
  c.h0 = t - strip * a.tiles_h;
  c.w0 = (strip % a.tiles_w) * 128;
  c.img = im.img(strip / a.tiles_w);
  c.n0 = 0;
  return c;
}

// NW ("narrow rows"): the ring's K rows are 64 bytes (32 16-bit channels, for
// layers of 32 input channels) under the 64-byte swizzle, two MMAs per K chunk.
// CG2: tiles of 256 rows computed by the CTA pair of a cluster of two with
// two-SM MMAs (tcgen05 .cta_group::2): each CTA loads its own 128 rows of A and
// half of the N rows of B (per-SM operand bytes per MMA cycle fall by a third for
// N = 256), the even CTA issues the MMAs, each CTA's epilogue drains its own rows.
// STK (stacked taps; sliding halo form, N <= 64): the three vertical taps of one
// horizontal offset are stacked along N, so one MMA of N = 3 BN reads an input row
// box once for the three output rows it feeds (rows y+1, y, y-1).  The weights
// sit in shared memory in (dx, 2 - dy) order, the accumulators of consecutive
// output rows in a ring of eight TMEM blocks; each input row box is read once.
// MMAs of N = 64 are bound by the operand reads from shared memory (A: 4 KB per
// MMA whatever N is), so this cuts those reads per output row from 216 to ~124 KB.
template <typename TA, typename T, int BN, bool HALO, int MS, bool NW, bool CG2 = false,
          bool STK = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmO0,
                   const __grid_constant__ CUtensorMap tmO1,
                   const __grid_constant__ CUtensorMap tmX0,
                   const __grid_constant__ CUtensorMap tmX1,
                   const __grid_constant__ CUtensorMap tmX2, TcArgs a) {
  static_assert(!HALO || MS == 1, "the halo form has one 128-row sub-tile");
  static_assert(!CG2 || (!HALO && !NW && MS == 1 && sizeof(TA) == 2 && BN >= 128),
                "CTA pairs: plain or streamed 16-bit tiles of 128 or 256 columns");
  static_assert(!NW || (MS == 1 && sizeof(TA) == 2), "narrow rows: 16-bit, one sub-tile");
  static_assert(!STK || (HALO && !NW && BN <= 64), "stacked taps: halo form, N <= 64");
  constexpr int RB = NW ? 64 : 128;     // bytes of one K row of a ring tile
  constexpr int A_TILE = 128 * RB;      // one 128-pixel A tile of one K chunk
  constexpr int B_BYTES = (CG2 ? BN / 2 : BN) * RB;  // this CTA's rows of B per K chunk
  constexpr int MSUB = CG2 ? 2 : MS;    // 128-row sub-tiles per tile (CTA pair: one each)
  constexpr int KSTEPS = RB / 32;       // MMAs per K chunk (32 bytes of K each)
  constexpr int HBOX = NW ? HALO_BOX_NW : HALO_BOX;  // one halo row box
  // ring slot: the A (and B) boxes of one K chunk; in the halo form the three row
  // boxes of a tile, or a single row box in the sliding form; in the streamed halo
  // form one row box and the three horizontal taps of B of one (row, channel chunk)
  const bool STREAM = !HALO && !NW && a.stream;
  const int A_STAGE =
      HALO ? (a.slide ? HBOX : 3 * HBOX) : (STREAM ? MS * HALO_BOX : MS * A_TILE);
  const int B_STAGE = STREAM ? 3 * B_BYTES : B_BYTES;
  const uint32_t STAGE_TX =
      HALO ? (a.slide ? 1u : 3u) * HALO_ROWS * (uint32_t)RB
           : (STREAM ? MS * HALO_ROWS * 128u + 3u * B_BYTES
                     : (uint32_t)(MS * A_TILE + B_BYTES));
  constexpr bool IMG = BN == 16;  // image-side output: c <= 16 planar f32 channels
  constexpr int NPANEL = (IMG || BN < 64) ? 1 : BN / 64;  // 64-column epilogue panels
  constexpr int KCH = RB / (int)sizeof(TA);  // K elements per ring row
  static_assert(!HALO || sizeof(TA) == 2, "the halo form has 16-bit operands");
  // tiles of <= 32 (optionally 64) columns: the two halves of the epilogue warps
  // take alternate tiles, half h the accumulator buffer h, so two tiles drain at once
  constexpr bool SPLIT = BN <= 32;
  const bool spl = SPLIT || (BN == 64 && MS == 1 && a.split64 != 0);
  constexpr int TCOLS = MS * BN;  // TMEM columns of one accumulator buffer (2 x >= 32 allocated)
  // accumulator buffers: two (the epilogue of one tile overlaps the MMAs of the
  // next) while they fit the 512 TMEM columns, else one (M = 256 x N = 256 tiles)
  // (stacked taps: a ring of eight, one per output row in flight)
  constexpr int NACC = STK ? 8 : (TCOLS <= 256 ? 2 : 1);
  constexpr int NTB = STK ? 8 : 2;  // accumulator full / empty barriers of each kind
  const int ST = a.stages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + ST * A_STAGE;  // ring slots, or the resident weights (HALO)
  uint8_t* sOut = sB + (HALO ? a.nk * B_BYTES : ST * B_STAGE);  // [warp][nbo][nout][WBOX]
  uint8_t* sAux = sOut + a.nbo * a.nout * PANEL;                 // [warp][nba][naux][WBOX]
  uint64_t* bars = (uint64_t*)(sAux + a.nba * a.naux * PANEL);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * ST + 2 * NTB + 2 + MAX_NBA * EPI_WARPS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + ST);
  const uint32_t tfull0 = smem_u32(bars + 2 * ST);
  const uint32_t tempty0 = smem_u32(bars + 2 * ST + NTB);
  const uint32_t drain = smem_u32(bars + 2 * ST + 2 * NTB);
  const uint32_t bres = smem_u32(bars + 2 * ST + 2 * NTB + 1);
  const uint32_t auxbar0 = smem_u32(bars + 2 * ST + 2 * NTB + 2);  // [warp][MAX_NBA]
  const uint32_t rank = CG2 ? cluster_ctarank() : 0u;  // 0: issues the pair's MMAs
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < NTB; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      // a pair's accumulator is released by the epilogue warps of both CTAs
      mbar_init(tempty0 + 8 * b, CG2 ? 2 * EPI_WARPS : (spl ? EPI_WARPS / 2 : EPI_WARPS));
    }
    for (int b = 0; b < MAX_NBA * EPI_WARPS; ++b) mbar_init(auxbar0 + 8 * b, 1);
    mbar_init(drain, 1);
    mbar_init(bres, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (CG2) {  // one warp of each CTA of the pair, collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"((uint32_t)(NACC * TCOLS))
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"((uint32_t)(NACC * TCOLS))
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  // The images to compute: every warp reads the per-image skip flags into a
  // bitmask.  The flags are written only by kernels that are not convolutions (the
  // solver's bookkeeping) or by copies, after which the first convolution starts
  // only once they have completed; convolutions never write them.  So they are
  // read before the wait below, overlapping the previous convolution's tail.
  const bool masked = a.skip != nullptr && a.n <= kMaxMaskImages;
  uint32_t run = 0u;
  if (masked) run = __ballot_sync(0xffffffffu, lane < a.n && a.skip[lane] == 0);
  tc_fence_before();
  __syncthreads();
  if constexpr (CG2) cluster_sync();  // both CTAs' barriers initialised before any remote use
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // Programmatic dependent launch: the set-up above may overlap the tail of the
  // previous kernel in the stream; every global access of this kernel to data a
  // convolution writes comes after that kernel's results are complete and visible.
  // The next conv may start its own set-up as soon as this kernel's CTAs leave
  // their SMs.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const ImgMap im{masked ? __popc(run) : a.n, run, masked, masked ? img_table(run) : 0ull};
  const int ntiles = ((im.nrun * a.tiles_h * a.tiles_w + MSUB - 1) / MSUB) * a.tiles_n;
  // this CTA's tiles: t_first + i * t_step, i < my_tiles (a contiguous range in
  // the halo form, a grid-strided sequence otherwise; a CTA pair shares its tiles)
  int t_first, t_step, my_tiles;
  if (HALO && a.slide) {
    t_first = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
    my_tiles = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x) - t_first;
    t_step = 1;
  } else {
    const int unit = CG2 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int units = CG2 ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    t_first = unit;
    t_step = units;
    my_tiles = unit < ntiles ? (ntiles - 1 - unit) / units + 1 : 0;
  }
  const int tsub0 = CG2 ? (int)rank : 0;  // this CTA's sub-tile of a pair tile
  const int bn_off = CG2 ? (int)rank * (BN / 2) : 0;  // this CTA's first row of B

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
      if (HALO) {  // resident weights: every K chunk of B once
        mbar_expect_tx(bres, (uint32_t)(a.nk * B_BYTES));
        for (int kc = 0; kc < a.nk; ++kc) {  // kc: tap 3 dy + dx (one K chunk per tap)
          const int blk = STK ? (kc % 3) * 3 + 2 - kc / 3 : kc;
          tma_load_2d(smem_u32(sB + blk * B_BYTES), &tmB, kc * KCH, 0, bres);
        }
      }
      int g = 0;  // ring position across tiles (row boxes in the halo form)
      // slot and phase of ring position g, advanced without division: a runtime
      // divide in these loops measurably slows the MMA issue and the copies
      int rs = 0;
      uint32_t rph = 0u;
      bool ok = true;
      if (HALO && !a.slide) {  // one slot of three row boxes per tile
        for (int i = 0; i < my_tiles && ok; ++i) {
          const TileCoord tc = halo_coord(a, im, t_first + i * t_step);
          const int s = rs;
          if (g >= ST && !mbar_wait(empty0 + 8 * s, rph ^ 1u, a.err, 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, STAGE_TX);
          for (int dy = 0; dy < 3; ++dy)
            tma_load_4d(smem_u32(sA + s * A_STAGE + dy * HBOX), &tmA, 0, tc.w0 - 1,
                        tc.h0 + dy - 1, tc.img, full0 + 8 * s);
          ++g;
          if (++rs == ST) {
            rs = 0;
            rph ^= 1u;
          }
        }
      } else if (HALO) {  // sliding: single row boxes, reused across consecutive rows
        for (int i = 0; i < my_tiles && ok; ++i) {
          const int t = t_first + i * t_step;
          const TileCoord tc = halo_coord(a, im, t);
          const bool fresh = i == 0 || t % a.tiles_h == 0;  // three new boxes
          // rows loaded a few tiles from now are pulled into L2 first: each row is
          // read by this CTA alone, so its load would otherwise wait on DRAM
          for (int r = fresh ? 2 : HALO_PF + 1; r <= HALO_PF + 1; ++r)
            if (tc.h0 + r < a.H) tma_prefetch_4d(&tmA, 0, tc.w0 - 1, tc.h0 + r, tc.img);
          for (int dy = fresh ? -1 : 1; dy <= 1; ++dy) {
            const int s = g % ST, j = g / ST;
            if (j > 0 && !mbar_wait(empty0 + 8 * s, (j - 1) & 1, a.err, 1)) {
              ok = false;
              break;
            }
            mbar_expect_tx(full0 + 8 * s, STAGE_TX);
            tma_load_4d(smem_u32(sA + s * A_STAGE), &tmA, 0, tc.w0 - 1, tc.h0 + dy, tc.img,
                        full0 + 8 * s);
            ++g;
          }
        }
      }
      for (int i = 0; i < my_tiles && ok && STREAM; ++i) {  // streamed halo
        const int t = t_first + i * t_step;
        for (int kc = 0, dy = 0, c = 0; kc < 3 * a.cpt; ++kc) {  // (row dy, channel chunk c)
          const int s = rs;
          if (g >= ST && !mbar_wait(empty0 + 8 * s, rph ^ 1u, a.err, 1)) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_expect_tx(full0 + 8 * s, (CG2 ? 2u : 1u) * STAGE_TX);
          if constexpr (CG2) {  // both halves of the stage complete on the even CTA's barrier
            const uint32_t fb = mapa_shared(full0 + 8 * s, 0);
            const TileCoord sc = tile_coord(a, im, t, BN, MSUB, tsub0);
            tma_load_4d_cg2(smem_u32(sA + s * A_STAGE), &tmA, c * KCH, sc.w0 - 1, sc.h0 + dy - 1,
                            sc.img, fb);
            for (int dx = 0; dx < 3; ++dx)
              tma_load_2d_cg2(smem_u32(sB + s * B_STAGE + dx * B_BYTES), &tmB,
                              ((3 * dy + dx) * a.cpt + c) * KCH, sc.n0 + bn_off, fb);
          } else {
#pragma unroll
            for (int sub = 0; sub < MS; ++sub) {  // one row box per 128-pixel sub-tile
              const TileCoord sc = tile_coord(a, im, t, BN, MSUB, sub + tsub0);
              tma_load_4d(smem_u32(sA + s * A_STAGE + sub * HALO_BOX), &tmA, c * KCH, sc.w0 - 1,
                          sc.h0 + dy - 1, sc.img, full0 + 8 * s);
            }
            const TileCoord tc = tile_coord(a, im, t, BN, MSUB, tsub0);
            for (int dx = 0; dx < 3; ++dx)
              tma_load_2d(smem_u32(sB + s * B_STAGE + dx * B_BYTES), &tmB,
                          ((3 * dy + dx) * a.cpt + c) * KCH, tc.n0, full0 + 8 * s);
          }
          ++g;
          if (++rs == ST) {
            rs = 0;
            rph ^= 1u;
          }
          if (++c == a.cpt) {
            c = 0;
            ++dy;
          }
        }
      }
      for (int i = 0; i < my_tiles && ok && !HALO && !STREAM; ++i) {
        const int t = t_first + i * t_step;
        const TileCoord tc = tile_coord(a, im, t, BN, MSUB, tsub0);
        // K position of chunk kc: tap and channel offset (3x3), or the input row di
        // of the 2x2 window and the offset in it (stride 2)
        int ktap = 0, kcc = 0;
        for (int kc = 0; kc < a.nk; ++kc) {
          const int s = rs;
          if (g >= ST && !mbar_wait(empty0 + 8 * s, rph ^ 1u, a.err, 1)) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_expect_tx(full0 + 8 * s, (CG2 ? 2u : 1u) * STAGE_TX);
          // a CTA pair's halves of the stage complete on the even CTA's barrier
          const uint32_t fb = CG2 ? mapa_shared(full0 + 8 * s, 0) : full0 + 8 * s;
          const uint32_t dA = smem_u32(sA + s * A_STAGE);
          {
            const uint32_t dB = smem_u32(sB + s * B_STAGE);
#pragma unroll
            for (int sub = 0; sub < MS; ++sub) {
              const TileCoord sc = sub == 0 ? tc : tile_coord(a, im, t, BN, MSUB, sub + tsub0);
              const uint32_t dAs = dA + sub * A_TILE;
              if (a.mode == CM_DOWN) {
                const int di = ktap, rem = kcc;
                if (CG2)
                  tma_load_5d_cg2(dAs, &tmA, rem, sc.w0, di, sc.h0, sc.img, fb);
                else
                  tma_load_5d(dAs, &tmA, rem, sc.w0, di, sc.h0, sc.img, fb);
              } else {
                int tap = 4, c0 = kc * KCH;
                if (a.mode == CM_CONV3) {
                  tap = ktap;
                  c0 = kcc;
                }
                if (CG2)
                  tma_load_4d_cg2(dAs, &tmA, c0, sc.w0 + tap % 3 - 1, sc.h0 + tap / 3 - 1,
                                  sc.img, fb);
                else
                  tma_load_4d(dAs, &tmA, c0, sc.w0 + tap % 3 - 1, sc.h0 + tap / 3 - 1, sc.img,
                              fb);
              }
            }
            if (CG2)
              tma_load_2d_cg2(dB, &tmB, kc * KCH, tc.n0 + bn_off, fb);
            else
              tma_load_2d(dB, &tmB, kc * KCH, tc.n0, fb);
          }
          ++g;
          if (++rs == ST) {
            rs = 0;
            rph ^= 1u;
          }
          // next K chunk: CM_CONV3 walks the channels of one tap, CM_DOWN the
          // 2 Cin elements of one input row of the window
          kcc += KCH;
          if (kcc == (a.mode == CM_DOWN ? 2 * a.Cin : a.Cin)) {
            kcc = 0;
            ++ktap;
          }
        }
      }
      // tail: wait until the MMA warp released every slot still in use, so no
      // tcgen05.commit arrival is outstanding when the CTA exits.
      const int first = g > ST ? g - ST : 0;
      for (int i = first; i < g; ++i) {
        const int s = i % ST, j = i / ST;
        if (ok) ok = mbar_wait(empty0 + 8 * s, j & 1, a.err, 2);
        // our own copies in flight (a CTA pair's are all counted on the even CTA's
        // barriers, which it waits for here before the pair's final cluster barrier)
        if (!ok && rank == 0) mbar_wait(full0 + 8 * s, j & 1, a.err, 2);
      }
      if (HALO && !ok) mbar_wait(bres, 0, a.err, 2);
    }
  } else if (CG2 && warp == 1) {
    if (rank == 0) {  // the whole warp, converged: one elected lane issues
      // even CTA of a pair: two-SM MMAs, M = 256 (128 rows of A from each CTA),
      // N = BN (half of B from each CTA); commits release both CTAs' stages and
      // hand both CTAs their accumulator
      constexpr uint32_t idesc = umma_idesc_16(256, BN, Fmt<TA>::v);
      bool ok = true;
      int rs = 0;  // ring slot and phase, advanced without division
      uint32_t rph = 0u;
      for (int lt = 0; lt < my_tiles && ok; ++lt) {
        const int b = lt % NACC, u = lt / NACC;
        if (u > 0 && !mbar_wait_warp(tempty0 + 8 * b, (u - 1) & 1, a.err, 5)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t td = tmem + (uint32_t)(b * TCOLS);
        const int nkc = STREAM ? 3 * a.cpt : a.nk;
        for (int kc = 0; kc < nkc; ++kc) {
          const int s = rs;
          if (!mbar_wait_warp(full0 + 8 * s, rph, a.err, 3)) {  // both CTAs' halves
            ok = false;
            break;
          }
          tc_fence_after();
          if (STREAM) {
            const uint64_t a0 = umma_desc_sw128(smem_u32(sA + s * A_STAGE));
            const uint64_t b0 = umma_desc_sw128(smem_u32(sB + s * B_STAGE));
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const uint64_t bd = b0 + (uint64_t)((dx * B_BYTES) >> 4);
              const uint64_t ad = a0 + (uint64_t)((128 * dx) >> 4);
#pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk)
                umma_cg2_el(td, ad + 2 * kk, bd + 2 * kk, idesc, (kc | dx | kk) != 0 ? 1u : 0u);
            }
          } else {
            const uint64_t bd = umma_desc_sw128(smem_u32(sB + s * B_STAGE));
            const uint64_t ad = umma_desc_sw128(smem_u32(sA + s * A_STAGE));
#pragma unroll
            for (int kk = 0; kk < KSTEPS; ++kk)
              umma_cg2_el(td, ad + 2 * kk, bd + 2 * kk, idesc, (kc | kk) != 0 ? 1u : 0u);
          }
          umma_commit_cg2_both_el(empty0 + 8 * s);
          if (++rs == ST) {
            rs = 0;
            rph ^= 1u;
          }
        }
        if (ok) umma_commit_cg2_both_el(tfull0 + 8 * b);
      }
      if (!ok) {  // let every issued MMA finish before TMEM is released
        umma_commit_cg2_el(drain);
        mbar_wait_warp(drain, 0, a.err, 6);
      }
    }
  } else if (warp == 1) {
    {  // the whole warp, converged: one elected lane issues
      constexpr uint32_t idesc = umma_idesc_16(128, BN, Fmt<TA>::v);
      bool ok = true;
      if (HALO) ok = mbar_wait_warp(bres, 0, a.err, 9);
      int g = 0, base = 0;  // base: ring position of the tile's row y-1 box (HALO)
      int rs = 0;           // ring slot and phase (all forms but the sliding one),
      uint32_t rph = 0u;    // advanced without division
      if constexpr (STK) {
        // Stacked taps: walk the input row boxes in the order the producer loads
        // them.  A run of rows of one strip (seg output rows) reads seg + 2 boxes;
        // box i (-1 <= i <= seg, local rows) feeds stack position p (0: dy = 2,
        // 1: dy = 1, 2: dy = 0) of output row i - 1 + p, where that row is in the run.
        // Row i + 1 (p = 2) gets its first product here: on the first MMA step that
        // part is issued on its own without accumulation.
        constexpr uint32_t id1 = umma_idesc_16(128, BN, Fmt<TA>::v);
        constexpr uint32_t id2 = umma_idesc_16(128, 2 * BN, Fmt<TA>::v);
        constexpr uint32_t id3 = umma_idesc_16(128, 3 * BN, Fmt<TA>::v);
        const uint64_t bw0 = umma_desc<NW>(smem_u32(sB));
        int lt = 0;
        while (lt < my_tiles && ok) {
          const int t = t_first + lt;  // contiguous runs (t_step = 1)
          const int seg = min(my_tiles - lt, a.tiles_h - t % a.tiles_h);
          for (int i = -1; i <= seg && ok; ++i) {
            const int s = rs;
            const int p_lo = i >= 1 ? 0 : 1 - i, p_hi = min(2, seg - i);
            const bool fresh = p_hi == 2;  // output row i + 1 starts here
            if (fresh) {  // its accumulator block must have been drained
              const int ln = lt + i + 1;
              if (ln >= NACC &&
                  !mbar_wait_warp(tempty0 + 8 * (ln % NACC), ((ln / NACC) - 1) & 1, a.err, 5)) {
                ok = false;
                break;
              }
            }
            if (!mbar_wait_warp(full0 + 8 * s, rph, a.err, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            // positions [pl, ph] as MMAs: one, or two where the block ring wraps
            // (d: accumulator column, bo: B descriptor offset, id: N)
            uint32_t d1 = 0, d2 = 0, bo1 = 0, bo2 = 0, i1 = 0, i2 = 0;
            auto pieces = [&](int pl, int ph) -> int {
              if (pl > ph) return 0;
              const int blk = (lt + i - 1 + pl) % NACC, c = ph - pl + 1;
              const int c1 = min(c, NACC - blk);
              d1 = tmem + (uint32_t)(blk * TCOLS);
              bo1 = (uint32_t)((pl * B_BYTES) >> 4);
              i1 = c1 == 1 ? id1 : (c1 == 2 ? id2 : id3);
              if (c1 == c) return 1;
              d2 = tmem;
              bo2 = (uint32_t)(((pl + c1) * B_BYTES) >> 4);
              i2 = c - c1 == 1 ? id1 : id2;
              return 2;
            };
            // first step: the accumulating positions, then the new row
            const int nf = pieces(p_lo, fresh ? 1 : p_hi);
            const uint32_t fd1 = d1, fd2 = d2, fbo1 = bo1, fbo2 = bo2, fi1 = i1, fi2 = i2;
            const uint32_t dn = tmem + (uint32_t)(((lt + i + 1) % NACC) * TCOLS);
            const uint32_t bon = (uint32_t)((2 * B_BYTES) >> 4);
            // the other steps: all positions, accumulating
            const int ng = pieces(p_lo, p_hi);
            const uint64_t a0 = umma_desc<NW>(smem_u32(sA + s * A_STAGE));
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk) {
                const uint64_t ad = a0 + (uint64_t)((dx * RB) >> 4) + 2 * kk;
                const uint64_t bd = bw0 + (uint64_t)((dx * 3 * B_BYTES) >> 4) + 2 * kk;
                if (dx == 0 && kk == 0) {
                  if (nf >= 1) umma_el<TA>(fd1, ad, bd + fbo1, fi1, 1u);
                  if (nf >= 2) umma_el<TA>(fd2, ad, bd + fbo2, fi2, 1u);
                  if (fresh) umma_el<TA>(dn, ad, bd + bon, id1, 0u);
                } else {
                  if (ng >= 1) umma_el<TA>(d1, ad, bd + bo1, i1, 1u);
                  if (ng >= 2) umma_el<TA>(d2, ad, bd + bo2, i2, 1u);
                }
              }
            }
            umma_commit_el(empty0 + 8 * s);  // the box is read once
            if (p_lo == 0) umma_commit_el(tfull0 + 8 * ((lt + i - 1) % NACC));  // row i-1 done
            if (++rs == ST) {
              rs = 0;
              rph ^= 1u;
            }
          }
          lt += seg;
        }
      } else
      for (int lt = 0; lt < my_tiles && ok; ++lt) {
        const int t = t_first + lt * t_step;
        const int b = lt % NACC, u = lt / NACC;
        if (u > 0 && !mbar_wait_warp(tempty0 + 8 * b, (u - 1) & 1, a.err, 5)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t td = tmem + (uint32_t)(b * TCOLS);
        if (HALO && !a.slide) {
          const int s = rs;
          if (!mbar_wait_warp(full0 + 8 * s, rph, a.err, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          // The 36 (or 18) MMAs of the tile back to back: the descriptors of the
          // taps are the slot's and the weights' base descriptors plus constant
          // address offsets (the start address field holds address / 16, and no
          // shared-memory address reaches its carry), so nothing but MMAs is issued
          // between them; the pipe drains on any gap in the issue.
          const uint64_t a0 = umma_desc<NW>(smem_u32(sA + s * A_STAGE));
          const uint64_t b0 = umma_desc<NW>(smem_u32(sB));
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap - 3 * dy;
            const uint64_t ad = a0 + (uint64_t)((dy * HBOX + dx * RB) >> 4);
            const uint64_t bd = b0 + (uint64_t)((tap * B_BYTES) >> 4);
#pragma unroll
            for (int kk = 0; kk < KSTEPS; ++kk)
              umma_el<TA>(td, ad + 2 * kk, bd + 2 * kk, idesc, (tap | kk) != 0 ? 1u : 0u);
          }
          umma_commit_el(empty0 + 8 * s);
          umma_commit_el(tfull0 + 8 * b);
          ++g;
          if (++rs == ST) {
            rs = 0;
            rph ^= 1u;
          }
        } else if (HALO) {
          const bool fresh = lt == 0 || t % a.tiles_h == 0;
          if (fresh) {
            base = g;
            g += 3;
          } else {
            base += 1;
            g += 1;
          }
          for (int dy = 0; dy < 3 && ok; ++dy) {
            const int box = base + dy;
            ok = mbar_wait_warp(full0 + 8 * (box % ST), (box / ST) & 1, a.err, 3);
          }
          if (!ok) break;
          tc_fence_after();
#pragma unroll 1
          for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap - 3 * dy;
            const uint64_t ad =
                umma_desc_rows<NW>(smem_u32(sA + ((base + dy) % ST) * A_STAGE), dx);
            const uint64_t bd = umma_desc<NW>(smem_u32(sB + tap * B_BYTES));
#pragma unroll
            for (int kk = 0; kk < KSTEPS; ++kk)
              umma_el<TA>(td, ad + 2 * kk, bd + 2 * kk, idesc, (tap | kk) != 0 ? 1u : 0u);
          }
          umma_commit_el(tfull0 + 8 * b);
          // release the boxes the next tile does not read: row y-1, or all three
          // when the next tile starts a new strip run (or there is none)
          const bool next_fresh = lt + 1 == my_tiles || (t + 1) % a.tiles_h == 0;
          for (int dy = 0; dy < (next_fresh ? 3 : 1); ++dy)
            umma_commit_el(empty0 + 8 * ((base + dy) % ST));
        } else if (STREAM) {
          for (int kc = 0; kc < 3 * a.cpt; ++kc) {
            const int s = rs;
            if (!mbar_wait_warp(full0 + 8 * s, rph, a.err, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            // three taps of one row box back to back (constant descriptor offsets)
            const uint64_t a0 = umma_desc_sw128(smem_u32(sA + s * A_STAGE));
            const uint64_t b0 = umma_desc_sw128(smem_u32(sB + s * B_STAGE));
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const uint64_t bd = b0 + (uint64_t)((dx * B_BYTES) >> 4);
#pragma unroll
              for (int sub = 0; sub < MS; ++sub) {
                const uint64_t ad = a0 + (uint64_t)((sub * HALO_BOX + 128 * dx) >> 4);
#pragma unroll
                for (int kk = 0; kk < KSTEPS; ++kk)
                  umma_el<TA>(td + sub * BN, ad + 2 * kk, bd + 2 * kk, idesc,
                           (kc | dx | kk) != 0 ? 1u : 0u);
              }
            }
            umma_commit_el(empty0 + 8 * s);
            if (++rs == ST) {
              rs = 0;
              rph ^= 1u;
            }
          }
          if (ok) umma_commit_el(tfull0 + 8 * b);
        } else {
          for (int kc = 0; kc < a.nk; ++kc) {
            const int s = rs;
            if (!mbar_wait_warp(full0 + 8 * s, rph, a.err, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t bd = umma_desc<NW>(smem_u32(sB + s * B_STAGE));
#pragma unroll
            for (int sub = 0; sub < MS; ++sub) {
              const uint64_t ad = umma_desc<NW>(smem_u32(sA + s * A_STAGE + sub * A_TILE));
#pragma unroll
              for (int kk = 0; kk < KSTEPS; ++kk)
                umma_el<TA>(td + sub * BN, ad + 2 * kk, bd + 2 * kk, idesc,
                          (kc | kk) != 0 ? 1u : 0u);
            }
            umma_commit_el(empty0 + 8 * s);
            if (++rs == ST) {
              rs = 0;
              rph ^= 1u;
            }
          }
          if (ok) umma_commit_el(tfull0 + 8 * b);
        }
      }
      if (!ok) {  // let every issued MMA finish before TMEM is released
        umma_commit_el(drain);
        mbar_wait_warp(drain, 0, a.err, 6);
      }
    }
  } else if constexpr (IMG) {
    // ---------------- image-side epilogue: half h of the warps takes the tiles
    // of accumulator buffer h; each of its four warps owns one TMEM quadrant (one
    // pixel row per lane), reads the c valid columns and writes out = aux + sign *
    // acc to the f32 planar image, adding 1/2 out^2 to the image's sum.
    const int e = warp - 2, q = warp & 3, half = e >> 2;
    bool ok = true;
    for (int lt = half; lt < my_tiles && ok; lt += 2) {
      const int t = t_first + lt * t_step;
      const int b = lt % NACC, u = lt / NACC;
      ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * b, u & 1, a.err, 4));
      if (!ok) break;
      tc_fence_after();
      {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(b * TCOLS) + ((uint32_t)(q * 32) << 16), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * b);
        const TileCoord tc = HALO ? halo_coord(a, im, t) : tile_coord(a, im, t, BN, MSUB, tsub0);
        const int m = 32 * q + lane;
        const int x = tc.w0 + m % a.Wt, y = tc.h0 + m / a.Wt;
        double ssq = 0.0;
        if (tc.img < a.n && x < a.W && y < a.H) {
#pragma unroll
          for (int o = 0; o < 16; ++o) {
            if (o < a.Cout) {
              const size_t idx = (((size_t)tc.img * a.Cout + o) * a.H + y) * a.W + x;
              const float r = a.img_aux[idx] + a.sign * v[o];
              a.img_out[idx] = r;
              ssq += 0.5 * (double)r * (double)r;
            }
          }
        }
        if (a.sumsq) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, off);
          if (lane == 0 && tc.img < a.n) atomicAdd(a.sumsq + tc.img, ssq);
        }
      }
    }
  } else {
    // ---------------- epilogue warps 2..9, each on its own: warp e owns TMEM
    // lanes (rows) 32q .. 32q+31 (q = warp % 4, the quadrant it may read) and
    // columns 32h .. 32h+31 (h = e / 4) of every 64-column panel (of 32-column
    // tiles: all columns of the tiles of accumulator buffer h), with its own
    // staging boxes, auxiliary barriers and bulk store groups.
    const int e = warp - 2, q = warp & 3, half = e >> 2;
    {
      // this warp's tiles: lt0 + j * lstep
      const int lt0 = spl ? half : 0, lstep = spl ? 2 : 1;
      const int my_n = spl ? (my_tiles > half ? (my_tiles - half + 1) / 2 : 0) : my_tiles;
      const int colh = spl ? 0 : 32 * half;
      // panels: 32 columns each when split (all of the tile), else this half's 32
      // columns of each 64-column panel
      const int PW = spl ? 32 : 64;                // column step between panels
      const int nper = spl ? BN / 32 : NPANEL;     // panels per 128-row sub-tile
      const int npan = MS * nper;                  // panels per tile
      const CUtensorMap* tmO[2] = {&tmO0, &tmO1};
      const CUtensorMap* tmX[3] = {&tmX0, &tmX1, &tmX2};
      const uint32_t sO = smem_u32(sOut) + (uint32_t)(e * a.nbo * a.nout * WBOX);
      const uint32_t sX = smem_u32(sAux) + (uint32_t)(e * a.nba * a.naux * WBOX);
      const uint32_t xbar = auxbar0 + 8 * MAX_NBA * e;
      const int npc = my_n * npan;  // panels this warp processes
      // auxiliary box of panel k -> buffer k % nba, loaded ahead by lane 0
      auto aux_load = [&](int k) {
        const int i = k / npan, r = k - i * npan, sub = r / nper, p = r - sub * nper;
        const int t = t_first + (lt0 + i * lstep) * t_step;
        const TileCoord nc = HALO ? halo_coord(a, im, t) : tile_coord(a, im, t, BN, MSUB, sub + tsub0);
        const int buf = k % a.nba;
        const uint32_t bar = xbar + 8 * buf;
        mbar_expect_tx(bar, (uint32_t)(a.naux * WBOX));
        for (int x = 0; x < a.naux; ++x)
          epi_tma(false, a, tmX[x], sX + (uint32_t)((buf * a.naux + x) * WBOX), nc, q,
                  nc.n0 + PW * p + colh, bar);
      };
      int aux_issued = 0;
      const bool direct = a.direct != 0;
      if (lane == 0 && a.naux > 0 && !direct)
        for (; aux_issued < a.nba && aux_issued < npc; ++aux_issued) aux_load(aux_issued);
      int pc = 0;
      bool ok = true;
      for (int j = 0; j < my_n && ok; ++j) {
        const int lt = lt0 + j * lstep;
        const int t = t_first + lt * t_step;
        const int b = lt % NACC, u = lt / NACC;
        ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * b, u & 1, a.err, 4));
        tc_fence_after();
        for (int pp = 0; pp < npan && ok; ++pp, ++pc) {
          const int sub = pp / nper, p = pp - sub * nper;
          if (direct) {  // no staging: TMEM -> registers -> global memory
            float v[32];
            tmem_ld32(tmem + (uint32_t)(b * TCOLS + sub * BN + PW * p + colh) +
                          ((uint32_t)(q * 32) << 16),
                      v);
            if (pp == npan - 1) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) {
                if (CG2)
                  mbar_arrive_remote(mapa_shared(tempty0 + 8 * b, 0));
                else
                  mbar_arrive(tempty0 + 8 * b);
              }
            }
            const TileCoord tc = HALO ? halo_coord(a, im, t) : tile_coord(a, im, t, BN, MSUB, sub + tsub0);
            const int m = 32 * q + lane;
            const int x = tc.w0 + m % a.Wt, y = tc.h0 + m / a.Wt;
            if (tc.img < a.n && x < a.W && y < a.H) {
              const size_t e = (((size_t)tc.img * a.H + y) * a.W + x) * (size_t)a.Cout +
                               (size_t)(tc.n0 + PW * p + colh);
              epi_apply_g<T>(a.epi, a.act, v, (const T*)a.gaux0 + e, (const T*)a.gaux1 + e,
                             (const T*)a.gaux2 + e, (T*)a.gout0 + e, (T*)a.gout1 + e);
            }
            continue;
          }
          const int sb = pc % a.nbo, ab = pc % a.nba;
          if (lane == 0 && pc >= a.nbo) bulk_wait_read(a.nbo - 1);  // staging box sb read out
          __syncwarp();
          if (a.naux > 0) {
            ok = __all_sync(0xffffffffu, mbar_wait(xbar + 8 * ab, (pc / a.nba) & 1, a.err, 7));
            if (!ok) break;
          }
          float v[32];
          tmem_ld32(tmem + (uint32_t)(b * TCOLS + sub * BN + PW * p + colh) +
                        ((uint32_t)(q * 32) << 16),
                    v);
          if (pp == npan - 1) {  // last read of this accumulator: hand it back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (CG2)  // to the CTA that issues the pair's MMAs
                mbar_arrive_remote(mapa_shared(tempty0 + 8 * b, 0));
              else
                mbar_arrive(tempty0 + 8 * b);
            }
          }
          if constexpr (sizeof(TA) == 1) {  // FP8 operands: undo the two scales
            const float sa = *a.a_scale;
            const float* ws = a.w_scale + tile_coord(a, im, t, BN, MSUB, sub + tsub0).n0 + PW * p + colh;
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] *= sa * __ldg(ws + i);
          }
          const uint32_t ob = sO + (uint32_t)(sb * a.nout * WBOX);
          epi_apply<T>(a.epi, a.act, v, sX + (uint32_t)(ab * a.naux * WBOX), ob, lane);
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            const TileCoord tc = HALO ? halo_coord(a, im, t) : tile_coord(a, im, t, BN, MSUB, sub + tsub0);
            for (int i = 0; i < a.nout; ++i)
              epi_tma(true, a, tmO[i], ob + (uint32_t)(i * WBOX), tc, q,
                      tc.n0 + PW * p + colh, 0);
            bulk_commit();
            if (a.naux > 0 && aux_issued < npc) aux_load(aux_issued++);  // into buffer ab
          }
        }
      }
      if (lane == 0) {
        bulk_wait_all();
        // on an early exit, let auxiliary loads still in flight land
        for (int k = pc; k < aux_issued; ++k)
          mbar_wait(xbar + 8 * (k % a.nba), (k / a.nba) & 1, a.err, 8);
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair's CTAs leave together: the even CTA's MMAs read the odd CTA's shared
  // memory and its commits arrive on the odd CTA's barriers until the last tile
  if constexpr (CG2) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (CG2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"((uint32_t)(NACC * TCOLS))
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"((uint32_t)(NACC * TCOLS))
                   : "memory");
  }
}

// ------------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() { return tensor_map_encoder(); }

static int tiling_override(const char* name, int dflt);

// image-side output: c <= 16 f32 planar channels out of a 16-bit NHWC input
static bool image_side(const ConvArgs& a) {
  return a.out_nchw && !a.in_nchw && a.epi == EP_AXPY_NCHW && a.mode == CM_CONV3 &&
         a.outmap == OM_IDENT && a.Cout >= 1 && a.Cout <= 16;
}

static int pick_bn(int N) {
  if (N % 64 != 0) return 32;
  // smallest N tiled 256 wide (measured: 256-wide tiles win from N = 256 up)
  const int n256 = tiling_override("IDEQ_TC_BN256_MIN", 256);
  if (N % 256 == 0 && N >= n256) return 256;
  if (N % 128 == 0) return 128;
  return 64;
}

static int epi_nout(int epi) {
  if (epi == EP_AXPY_NCHW) return 0;  // written by the image-side epilogue, not staged
  return (epi == EP_ACT || epi == EP_MUL_KEEP) ? 2 : 1;
}
static int epi_naux(int epi) {
  if (epi == EP_DUAL) return 3;
  if (epi == EP_ADD || epi == EP_MUL || epi == EP_MUL_KEEP) return 1;
  return 0;
}

// narrow rows: 16-bit operands of 32 (not 64) channels per K chunk, for inputs
// whose channel count is an odd multiple of 32
static bool narrow_rows(const ConvArgs& a, int op_dt) {
  return op_dt != DT_FP8 && a.Cin % 64 != 0 && a.Cin % 32 == 0;
}

// K elements per ring row: 128 B of e4m3 or 16-bit values, 64 B for narrow rows
static int k_chunk(int op_dt, bool nw) { return op_dt == DT_FP8 ? 128 : (nw ? 32 : 64); }

bool tc_supported(const ConvArgs& a, int op_dt) {
  if (image_side(a))  // weights padded to 16 rows [16][K] by the caller
    return op_dt != DT_FP8 && a.Cin % 32 == 0 && a.aux0 && a.out;
  if (a.in_nchw || a.out_nchw || a.epi == EP_AXPY_NCHW) return false;
  if (a.Cin % k_chunk(op_dt, narrow_rows(a, op_dt)) != 0) return false;
  if (op_dt == DT_FP8 && (!a.a_scale || !a.w_scale)) return false;
  // N tiles of 32, 64, 128 or 256 columns (e4m3: 64 up); epilogue boxes of 32 channels
  const int nq = op_dt == DT_FP8 ? 64 : 32;
  if (a.N() % nq != 0 || a.Cout % nq != 0) return false;
  if (a.mode == CM_DOWN && a.outmap != OM_IDENT) return false;
  if (epi_naux(a.epi) >= 1 && !a.aux0) return false;
  if (epi_naux(a.epi) >= 2 && (!a.aux1 || !a.aux2)) return false;
  if (epi_nout(a.epi) == 2 && !a.out2) return false;
  return true;
}

static size_t fixed_smem(int nout, int naux, int nbo, int nba, int stages, int ntb = 2) {
  return 1024 + (size_t)(nbo * nout + nba * naux) * PANEL +
         (2 * stages + 2 * ntb + 2 + MAX_NBA * EPI_WARPS) * 8 + 16;
}

constexpr size_t kMaxSmem = 227 * 1024;

static bool encode(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m, CUtensorMapDataType dt,
                   int rank, const void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                   const cuuint32_t* box,
                   CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(m, dt, rank, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// map of an epilogue tensor (output or auxiliary, both shaped like the output),
// boxed as one epilogue warp's 32 rows x 32 channels, 64-byte swizzle
static bool encode_epi(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m,
                       CUtensorMapDataType dt, const ConvArgs& a, const TcPlan* p,
                       const void* base) {
  const cuuint64_t C = (cuuint64_t)a.Cout;
  const cuuint32_t bw = (cuuint32_t)std::min(p->Wt, 32), bh = 32 / bw;
  if (a.outmap == OM_D2S) {  // output image 2H x 2W viewed as [n][H][di][W][dj*C + co]
    const cuuint64_t W2 = 2 * (cuuint64_t)a.W;
    cuuint64_t dims[5] = {2 * C, (cuuint64_t)a.W, 2, (cuuint64_t)a.H, (cuuint64_t)a.n};
    cuuint64_t strides[4] = {2 * C * 2, W2 * C * 2, 2 * W2 * C * 2, 2 * (cuuint64_t)a.H * 2 * W2 * C};
    cuuint32_t box[5] = {32, bw, 1, bh, 1};
    return encode(enc, m, dt, 5, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
  }
  cuuint64_t dims[4] = {C, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.n};
  cuuint64_t strides[3] = {C * 2, (cuuint64_t)a.W * C * 2, (cuuint64_t)a.H * a.W * C * 2};
  cuuint32_t box[4] = {32, bw, bh, 1};
  return encode(enc, m, dt, 4, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

// Integer tuning override from the environment (read at plan creation), used to
// compare tilings on a given GPU without rebuilding; `dflt` when unset.
static int tiling_override(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return (v && *v) ? std::atoi(v) : dflt;
}

TcPlan* tc_plan_create(const ConvArgs& a, int op_dt, int epi_dt, std::string* err) {
  auto enc = get_encode();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled unavailable";
    return nullptr;
  }
  if ((op_dt != DT_BF16 && op_dt != DT_F16 && op_dt != DT_FP8) ||
      (epi_dt != DT_BF16 && epi_dt != DT_F16) || (op_dt != DT_FP8 && op_dt != epi_dt)) {
    *err = "tensor-core kernel needs bf16, f16 or e4m3 operands and a 16-bit output";
    return nullptr;
  }
  if (!tc_supported(a, op_dt)) {
    *err = "layer not supported by the tensor-core kernel";
    return nullptr;
  }
  TcPlan* p = new TcPlan();
  p->op_dt = op_dt;
  p->epi_dt = epi_dt;
  p->nw = narrow_rows(a, op_dt);
  p->pdl = tiling_override("IDEQ_TC_PDL", 1) != 0;
  // measured on the 64-channel full-row layers: slower split (53.9 vs 56.1
  // restorations/s on 8 x RGB 256^2), so 64-column tiles keep both halves per tile
  p->split64 = tiling_override("IDEQ_TC_SPLIT64", 0) != 0;
  const int KCH = k_chunk(op_dt, p->nw);
  const int RB = p->nw ? 64 : 128;  // bytes per ring row
  const bool img = image_side(a);
  const int N = img ? 16 : a.N();  // image side: weight rows padded to 16
  p->bn = img ? 16 : pick_bn(N);
  p->nout = epi_nout(a.epi);
  p->naux = epi_naux(a.epi);
  // M tile: Ht x Wt pixels of the grid, Wt a power of two
  int wt = 1;
  while (wt < a.W && wt < 128) wt <<= 1;
  p->Wt = wt;
  p->Ht = 128 / wt;
  p->tiles_w = (a.W + p->Wt - 1) / p->Wt;
  p->tiles_h = (a.H + p->Ht - 1) / p->Ht;
  p->cpt = a.Cin / KCH;
  p->nk = a.K() / KCH;
  p->tiles_n = N / p->bn;
  // halo form: 3x3 conv of 64 channels over whole 128-pixel row segments, with
  // the nine 64 x 64 weight taps resident in shared memory
  const size_t bres = (size_t)p->nk * p->bn * RB;
  // (instantiated for N tiles of 16, 64 and 128 columns, narrow rows 16 to 64)
  const bool halo_bn = p->nw ? p->bn <= 64 : (p->bn == 16 || p->bn == 64 || p->bn == 128);
  // the form with resident weights (halo) is tried first; where its staging does
  // not fit (epilogues with three auxiliary inputs), the layer runs without it
  p->stages = 0;
  for (int pass = 0; pass < 2 && !p->stages; ++pass) {
    const bool no_halo = pass == 1;
    p->halo = !no_halo && op_dt != DT_FP8 && a.mode == CM_CONV3 && p->Wt == 128 &&
              p->Ht == 1 && p->tiles_n == 1 && p->cpt == 1 && halo_bn && bres <= 80 * 1024 &&
              tiling_override("IDEQ_TC_HALO", 1) != 0;
    p->slide = p->halo && !p->nw && tiling_override("IDEQ_TC_SLIDE", 0) != 0;
    // stacked vertical taps (N = 3 BN per MMA) over sliding row runs, for the
    // halo layers of <= 64 output columns, when IDEQ_TC_STACK=1.  Measured on the
    // 64-channel 256^2 layers of 8 x RGB 256^2 (C1a): 70-78 us against 63-72 us for
    // the 9-tap tiles, although the stacked MMA sequence alone runs 1.6x faster; the
    // epilogue and the sliding row runs bound these layers, so the 9-tap tiles stay.
    p->stk = p->halo && !p->nw && p->bn <= 64 && tiling_override("IDEQ_TC_STACK", 0) == 1;
    if (p->stk) p->slide = true;
    // streamed halo: full-row 3x3 convs whose weights do not stay resident
    p->stream = !p->halo && op_dt != DT_FP8 && !p->nw && a.mode == CM_CONV3 && p->Wt == 128 &&
                p->Ht == 1 && p->tiles_n == 1 && p->bn <= 128 && p->bn != 32 &&
                tiling_override("IDEQ_TC_STREAM", 1) != 0;
    // Two 128-row sub-tiles can share each weight chunk (M = 256 per CTA): a third
    // fewer operand bytes per MMA cycle into each SM, at the price of coarser tiles,
    // fewer ring stages and, for N = 256, a single accumulator buffer.
    p->ms = 1;
    {
      static int nsm = 0;
      if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 148;
      }
      const int force_ms = tiling_override("IDEQ_TC_MS", 0);
      const bool ms2_ok = !p->halo && !p->nw && op_dt != DT_FP8 && p->bn >= 64 && !img;
      const long long tm = (long long)a.n * p->tiles_h * p->tiles_w;
      const long long w1 = (tm * p->tiles_n + nsm - 1) / nsm;
      const long long w2 = (((tm + 1) / 2) * p->tiles_n + nsm - 1) / nsm;
      // measured on 8 x RGB 256^2 (C1a): the wave rule made the step slower (conv
    // launches 51.8 vs 47.1 us on average), so two sub-tiles are used only when
    // forced with IDEQ_TC_MS=2 (IDEQ_TC_MS=3 applies the wave rule)
    if (ms2_ok && (force_ms == 2 || (force_ms == 3 && w2 < w1))) p->ms = 2;
    }
    // CTA pairs with two-SM MMAs for the 128- and 256-column 16-bit tiles of the
    // plain and streamed forms.  Each SM then loads a third fewer operand bytes per
    // MMA cycle; this pays where the copies bound the main loop, i.e. long K.
    // Measured on 8 x RGB 256^2 (C1a): 256- and 512-channel 3x3 layers 12-14%
    // faster as pairs; the streamed 128-channel layers and the short-K stride-2 and
    // depth-to-space layers slower.  IDEQ_TC_CG2=1 pairs every eligible layer, 2 the
    // long-K and the streamed ones, 0 none.
    const int cg2_mode = tiling_override("IDEQ_TC_CG2", -1);
    p->cg2 = !p->halo && !p->nw && op_dt != DT_FP8 && (p->bn == 128 || p->bn == 256) &&
             p->ms == 1 && !img && cg2_mode != 0 &&
             (cg2_mode == 1 || (!p->stream && p->nk >= 32) || (cg2_mode == 2 && p->stream));
    const size_t bcta = p->cg2 ? (size_t)p->bn / 2 : (size_t)p->bn;  // rows of B per CTA
    // shared memory: ring depth and staging buffers, preferring a deep ring
    // (halo: >= 5 row boxes, three in use and two in flight; else >= 3 stages),
    // then double-buffered staging
    const size_t stage = p->halo     ? (size_t)(p->slide ? 1 : 3) * (p->nw ? HALO_BOX_NW : HALO_BOX)
                         : p->stream ? (size_t)p->ms * HALO_BOX + 3 * bcta * 128
                                     : ((size_t)p->ms * 128 + bcta) * RB;
    const size_t resident = p->halo ? bres : 0;
    p->stages = 0;
    // direct epilogue (halo and streamed forms: full-row tiles whose 64- and 128-column
    // MMAs keep the shared-memory port busy, so staged epilogue traffic waits): the
    // epilogue threads read their auxiliary values and store their results in global
    // memory themselves, and the staging space goes to the ring (IDEQ_TC_DIRECT=0
    // keeps the staged epilogue)
    p->direct = (p->halo || p->stream) && a.outmap == OM_IDENT && !img && op_dt != DT_FP8 &&
                tiling_override("IDEQ_TC_DIRECT", 1) != 0;
    if (p->direct) {
      const int min_st = p->halo ? (p->slide ? 5 : 2) : 2;
      auto total = [&](int k) {
        return fixed_smem(p->nout, p->naux, 0, 0, k, p->stk ? 8 : 2) + resident + k * stage;
      };
      int st = 8;
      while (st > min_st && total(st) > kMaxSmem) --st;
      if (total(st) <= kMaxSmem) {
        p->stages = st;
        p->nbo = 0;
        p->nba = 0;
        p->smem = total(st);
      } else {
        p->direct = false;
      }
    }
    // short K (depth-to-space, stride-2 and 1x1 layers): the epilogue paces the
    // kernel, so auxiliary boxes are fetched four panels ahead and the ring is
    // held to two stages (measured: 2% on the depth-to-space layers, 57 vs 58 us)
    if (!p->stages && p->naux > 0 && !p->halo && !p->stream && p->nk <= 4 &&
        tiling_override("IDEQ_TC_NBA", MAX_NBA) == MAX_NBA) {
      for (int st = 8; st >= 2 && !p->stages; --st) {
        const size_t tot =
            fixed_smem(p->nout, p->naux, 2, MAX_NBA, st, p->stk ? 8 : 2) + (size_t)st * stage;
        if (tot <= kMaxSmem) {
          p->stages = st;
          p->nbo = 2;
          p->nba = MAX_NBA;
          p->smem = tot;
        }
      }
    }
    const int min_stages[2] = {p->halo ? (p->slide ? 5 : 3) : (p->stream ? 2 : 3),
                               p->halo ? (p->slide ? 4 : 2) : 2};
    // staging depths (output buffers, auxiliary buffers), most preferred first: both
    // double-buffered; then, where that does not fit, a deeper auxiliary prefetch
    // before a second output buffer (an auxiliary box that is not yet loaded stalls
    // the epilogue for a full load latency; IDEQ_TC_AUXDEEP=0 keeps nbo = nba)
    static const int kStaging[][2] = {{2, 2}, {1, 2}, {1, 1}};
    const bool aux_deep = tiling_override("IDEQ_TC_AUXDEEP", 1) != 0;
    for (int min_st : min_stages) {
      if (p->stages) break;
      for (const auto& sb : kStaging) {
        const int nbo = sb[0], nba = p->naux > 0 ? sb[1] : sb[0];
        if (!aux_deep && nbo != nba) continue;
        int st = 8;
        auto total = [&](int k) {
          return fixed_smem(p->nout, p->naux, nbo, nba, k, p->stk ? 8 : 2) + resident + k * stage;
        };
        while (st > min_st && total(st) > kMaxSmem) --st;
        if (total(st) <= kMaxSmem) {
          p->stages = st;
          p->nbo = nbo;
          p->nba = nba;
          p->smem = total(st);
          break;
        }
      }
      if (p->stages) break;
    }
  }
  if (!p->stages) {
    *err = "tensor-core conv does not fit in shared memory";
    delete p;
    return nullptr;
  }
  {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 148;
    }
    const long long tiles_m = (long long)a.n * p->tiles_h * p->tiles_w;
    const int per = p->cg2 ? 2 : p->ms;  // 128-row sub-tiles per tile
    const long long tiles = ((tiles_m + per - 1) / per) * p->tiles_n;
    if (p->cg2)  // one CTA pair per tile, pairs on neighbouring SMs
      p->grid = dim3((unsigned)(2 * std::min<long long>(tiles, sms / 2)), 1, 1);
    else
      p->grid = dim3((unsigned)std::min<long long>(tiles, sms), 1, 1);
  }
  auto map_type = [](int d) {
    return d == DT_FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                       : (d == DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  };
  const CUtensorMapDataType dt = map_type(op_dt), edt = map_type(epi_dt);
  const cuuint64_t es = op_dt == DT_FP8 ? 1 : 2;  // operand element bytes
  const CUtensorMapSwizzle swz = p->nw ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  bool ok;
  if (a.mode == CM_DOWN) {
    const int Hi = 2 * a.H, Wi = 2 * a.W;
    cuuint64_t dims[5] = {(cuuint64_t)(2 * a.Cin), (cuuint64_t)a.W, 2, (cuuint64_t)a.H,
                          (cuuint64_t)a.n};
    cuuint64_t strides[4] = {(cuuint64_t)2 * a.Cin * es, (cuuint64_t)Wi * a.Cin * es,
                             (cuuint64_t)2 * Wi * a.Cin * es, (cuuint64_t)Hi * Wi * a.Cin * es};
    cuuint32_t box[5] = {(cuuint32_t)KCH, (cuuint32_t)p->Wt, 1, (cuuint32_t)p->Ht, 1};
    ok = encode(enc, &p->tmA, dt, 5, a.in, dims, strides, box, swz);
  } else {
    cuuint64_t dims[4] = {(cuuint64_t)a.Cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.n};
    cuuint64_t strides[3] = {(cuuint64_t)a.Cin * es, (cuuint64_t)a.W * a.Cin * es,
                             (cuuint64_t)a.H * a.W * a.Cin * es};
    cuuint32_t box[4] = {(cuuint32_t)KCH,
                         (cuuint32_t)((p->halo || p->stream) ? HALO_ROWS : p->Wt),
                         (cuuint32_t)p->Ht, 1};
    ok = encode(enc, &p->tmA, dt, 4, a.in, dims, strides, box, swz);
  }
  {
    const int K = a.K();
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)K * es};
    // a CTA of a pair loads half of the tile's rows of B
    cuuint32_t box[2] = {(cuuint32_t)KCH, (cuuint32_t)(p->cg2 ? p->bn / 2 : p->bn)};
    ok = ok && encode(enc, &p->tmB, dt, 2, a.wB, dims, strides, box, swz);
  }
  const void* outs[2] = {a.out, a.out2};
  const void* auxs[3] = {a.aux0, a.aux1, a.aux2};
  if (img) {  // no staged epilogue tensors: copy the A map into the unused slots
    for (int i = 0; i < 2; ++i) p->tmO[i] = p->tmA;
    for (int i = 0; i < 3; ++i) p->tmX[i] = p->tmA;
  } else {
    for (int i = 0; i < 2; ++i)
      ok = ok && encode_epi(enc, &p->tmO[i], edt, a, p, i < p->nout ? outs[i] : a.out);
    for (int i = 0; i < 3; ++i)
      ok = ok && encode_epi(enc, &p->tmX[i], edt, a, p, i < p->naux ? auxs[i] : a.out);
  }
  if (!ok) {
    *err = "cuTensorMapEncodeTiled failed";
    delete p;
    return nullptr;
  }
  return p;
}

void tc_plan_destroy(TcPlan* p) { delete p; }

template <typename TA, typename T, int BN, bool HALO, int MS, bool NW = false, bool CG2 = false,
          bool STK = false>
static cudaError_t launch_bn(const TcPlan* p, const TcArgs& ta, cudaStream_t st) {
  static bool attr_set = false;  // per instantiation; set before first launch
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<TA, T, BN, HALO, MS, NW, CG2, STK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = p->grid;
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = p->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = p->pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (CG2) {  // clusters of two CTAs (a portable cluster size)
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 2;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.numAttrs = 2;
  }
  return cudaLaunchKernelEx(&cfg, conv_tc_kernel<TA, T, BN, HALO, MS, NW, CG2, STK>, p->tmA, p->tmB,
                            p->tmO[0], p->tmO[1], p->tmX[0], p->tmX[1], p->tmX[2], ta);
}

template <typename T>
static cudaError_t launch_typed(const TcPlan* p, const TcArgs& t, cudaStream_t st) {
  if (p->op_dt == DT_FP8) {  // e4m3 operands: plain tiles only
    switch (p->bn) {
      case 64: return launch_bn<__nv_fp8_e4m3, T, 64, false, 1>(p, t, st);
      case 128: return launch_bn<__nv_fp8_e4m3, T, 128, false, 1>(p, t, st);
      default: return launch_bn<__nv_fp8_e4m3, T, 256, false, 1>(p, t, st);
    }
  }
  if (p->nw && p->halo) {  // 32-channel K rows, halo form
    switch (p->bn) {
      case 16: return launch_bn<T, T, 16, true, 1, true>(p, t, st);
      case 32: return launch_bn<T, T, 32, true, 1, true>(p, t, st);
      default: return launch_bn<T, T, 64, true, 1, true>(p, t, st);
    }
  }
  if (p->nw) {  // 32-channel K rows: plain tiles
    switch (p->bn) {
      case 16: return launch_bn<T, T, 16, false, 1, true>(p, t, st);
      case 32: return launch_bn<T, T, 32, false, 1, true>(p, t, st);
      case 64: return launch_bn<T, T, 64, false, 1, true>(p, t, st);
      case 128: return launch_bn<T, T, 128, false, 1, true>(p, t, st);
      default: return launch_bn<T, T, 256, false, 1, true>(p, t, st);
    }
  }
  if (p->bn == 32) return launch_bn<T, T, 32, false, 1>(p, t, st);
  if (p->bn == 16) {
    if (p->stk) return launch_bn<T, T, 16, true, 1, false, false, true>(p, t, st);
    if (p->halo) return launch_bn<T, T, 16, true, 1>(p, t, st);
    return launch_bn<T, T, 16, false, 1>(p, t, st);
  }
  if (p->stk) return launch_bn<T, T, 64, true, 1, false, false, true>(p, t, st);
  if (p->halo) {
    switch (p->bn) {
      case 64: return launch_bn<T, T, 64, true, 1>(p, t, st);
      default: return launch_bn<T, T, 128, true, 1>(p, t, st);
    }
  }
  if (p->cg2) {  // CTA pairs: plain or streamed tiles of 128 or 256 columns
    if (p->bn == 128) return launch_bn<T, T, 128, false, 1, false, true>(p, t, st);
    return launch_bn<T, T, 256, false, 1, false, true>(p, t, st);
  }
  if (p->ms == 2) {
    switch (p->bn) {
      case 64: return launch_bn<T, T, 64, false, 2>(p, t, st);
      case 128: return launch_bn<T, T, 128, false, 2>(p, t, st);
      default: return launch_bn<T, T, 256, false, 2>(p, t, st);
    }
  }
  switch (p->bn) {
    case 64: return launch_bn<T, T, 64, false, 1>(p, t, st);
    case 128: return launch_bn<T, T, 128, false, 1>(p, t, st);
    default: return launch_bn<T, T, 256, false, 1>(p, t, st);
  }
}

cudaError_t launch_conv_tc(const TcPlan* p, const ConvArgs& a, int* err_flag, cudaStream_t st) {
  TcArgs t;
  t.mode = a.mode;
  t.outmap = a.outmap;
  t.epi = a.epi;
  t.act = a.act;
  t.n = a.n;
  t.H = a.H;
  t.W = a.W;
  t.Cin = a.Cin;
  t.Cout = a.Cout;
  t.N = a.N();
  t.Wt = p->Wt;
  t.Ht = p->Ht;
  t.tiles_w = p->tiles_w;
  t.tiles_h = p->tiles_h;
  t.tiles_n = p->tiles_n;
  t.nk = p->nk;
  t.cpt = p->cpt;
  t.stages = p->stages;
  t.nout = p->nout;
  t.naux = p->naux;
  t.nbo = p->nbo;
  t.nba = p->nba;
  t.slide = p->slide ? 1 : 0;
  t.stream = p->stream ? 1 : 0;
  t.split64 = p->split64 ? 1 : 0;
  t.sign = a.sign;
  t.img_aux = (const float*)a.aux0;
  t.img_out = (float*)a.out;
  t.sumsq = a.sumsq;
  t.skip = a.skip;
  t.a_scale = a.a_scale;
  t.w_scale = a.w_scale;
  t.err = err_flag;
  t.direct = p->direct ? 1 : 0;
  // unused slots point at the first output (never dereferenced)
  t.gout0 = a.out;
  t.gout1 = p->nout > 1 && a.out2 ? a.out2 : a.out;
  t.gaux0 = p->naux > 0 ? a.aux0 : a.out;
  t.gaux1 = p->naux > 1 ? a.aux1 : a.out;
  t.gaux2 = p->naux > 2 ? a.aux2 : a.out;
  if (p->epi_dt == DT_F16) return launch_typed<__half>(p, t, st);
  return launch_typed<__nv_bfloat16>(p, t, st);
}

}  // namespace ideq
