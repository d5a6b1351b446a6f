// Inline-PTX helpers of the tcgen05 kernels (sm_103a): mbarriers with bounded
// waits, TMA tensor loads and stores, UMMA shared-memory and instruction
// descriptors, tcgen05.mma / commit, TMEM loads, shared-memory vector access.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>
#include <mutex>

#include "common.cuh"

namespace ideq {


IDEQ_DEV uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

IDEQ_DEV uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

IDEQ_DEV void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

IDEQ_DEV void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

IDEQ_DEV uint32_t mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}

// Bounded wait: returns false after ~2 s or once another role raised the flag.
IDEQ_DEV bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*(volatile int*)err != 0) return false;
      const uint64_t now = globaltimer();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > 2000000000ull) {
        atomicCAS(err, 0, code);
        return false;
      }
    }
  }
}

IDEQ_DEV void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

IDEQ_DEV void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

IDEQ_DEV void tma_load_5d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                          int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// Pull a tensor box into L2 ahead of its load (no shared memory, no barrier).
IDEQ_DEV void tma_prefetch_4d(const CUtensorMap* tm, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(tm),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}

IDEQ_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
IDEQ_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// UMMA shared-memory matrix descriptor, K-major, 128-byte swizzle:
// start address >> 4 in bits [0,14), leading byte offset (unused for this
// layout, 16 B) in [16,30), stride byte offset 1024 B (one 8-row atom) in
// [32,46), descriptor version 1 in [46,48), swizzle mode 2 (128 B) in [61,64).
IDEQ_DEV uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// K-major with the 64-byte swizzle (rows of 32 16-bit channels): swizzle mode 4
// in [61,64) and a stride byte offset of 512 B (8 rows x 64 B).  The K steps of
// 16 elements (32 B) inside a row advance the start address, as with 128 B.
IDEQ_DEV uint64_t umma_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

template <bool NW>
IDEQ_DEV uint64_t umma_desc(uint32_t saddr) {
  return NW ? umma_desc_sw64(saddr) : umma_desc_sw128(saddr);
}

// Same descriptor for a matrix that starts `rows` 128-byte rows into a
// 1024-byte-aligned swizzle atom.  The tensor core takes the 8-row phase of the
// 128-byte swizzle from the address bits themselves (the pattern TMA wrote is
// address-based too), so the start address simply moves by whole rows and the
// base-offset field stays 0 -- measured bit-identical to the unshifted tiles.
IDEQ_DEV uint64_t umma_desc_sw128_rows(uint32_t atom_base, int rows) {
  return umma_desc_sw128(atom_base + 128u * (uint32_t)rows);
}

// Either swizzle, `rows` K rows (128 or, for narrow rows, 64 bytes each) into an
// aligned atom; the 64-byte swizzle is address-based in the same way.
template <bool NW>
IDEQ_DEV uint64_t umma_desc_rows(uint32_t atom_base, int rows) {
  return NW ? umma_desc_sw64(atom_base + 64u * (uint32_t)rows)
            : umma_desc_sw128_rows(atom_base, rows);
}

// Instruction descriptor of kind::f16: D f32 (bits [4,6) = 1), A and B of the
// same 16-bit format (bits [7,10) and [10,13): 0 = f16, 1 = bf16), both
// K-major, N >> 3 in [17,23), M >> 4 in [24,29).
__host__ __device__ constexpr uint32_t umma_idesc_16(int M, int N, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Operand format codes of the instruction descriptor: kind::f16 takes 0 = f16,
// 1 = bf16; kind::f8f6f4 takes 0 = e4m3 (the same bit fields).
template <typename T> struct Fmt;
template <> struct Fmt<__nv_bfloat16> { static constexpr uint32_t v = 1; };
template <> struct Fmt<__half> { static constexpr uint32_t v = 0; };
template <> struct Fmt<__nv_fp8_e4m3> { static constexpr uint32_t v = 0; };

// One MMA, D (+)= A * B^T, 128 x N x (32 bytes of K): K = 16 16-bit elements
// (kind::f16) or 32 e4m3 elements (kind::f8f6f4).  Both operands of one MMA
// have the same element type.
template <typename TA>
IDEQ_DEV void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                   uint32_t accumulate) {
  if constexpr (sizeof(TA) == 1) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// The MMA-issuing form for a converged warp: all 32 lanes make the call and one
// lane, chosen by elect.sync, issues (a predicate, no branch).  Measured: with a
// barrier wait before each K chunk, MMAs issued from lane 0 of a diverged warp run
// at 67-69 cycles per 128 x 64 x 16 and 82 per 128 x 128 x 16, against 52 and 69
// from a converged warp (the tensor pipe's ideal: 48 and 64).
template <typename TA>
IDEQ_DEV void umma_el(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                      uint32_t accumulate) {
  if constexpr (sizeof(TA) == 1) {
    asm volatile(
        "{\n\t.reg .pred e, p;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred e, p;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

IDEQ_DEV void umma_commit_el(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
          bar)
      : "memory");
}

// Bounded wait by a whole converged warp; every lane gets the same answer.
IDEQ_DEV bool mbar_wait_warp(uint32_t bar, uint32_t parity, int* err, int code) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, err, code));
}

IDEQ_DEV void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 consecutive f32 accumulator columns of this warp's 32 TMEM lanes (one
// lane = one row per thread); the wait is in the same statement so that no
// use of the registers can be scheduled before the data has arrived.
IDEQ_DEV void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive f32 accumulator columns of this warp's 32 TMEM lanes.
IDEQ_DEV void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

IDEQ_DEV void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

IDEQ_DEV void tma_store_4d(const CUtensorMap* tm, uint32_t src, int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];"
      ::"l"(tm), "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

IDEQ_DEV void tma_store_5d(const CUtensorMap* tm, uint32_t src, int c0, int c1, int c2, int c3,
                           int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}],"
      " [%1];" ::"l"(tm),
      "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}

IDEQ_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
IDEQ_DEV void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
IDEQ_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
IDEQ_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Wait until at most `keep` (0 or 1) of this thread's bulk store groups still
// read shared memory.
IDEQ_DEV void bulk_wait_read(int keep) {
  if (keep > 0)
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
  else
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Byte offset of 16-byte chunk c (0..3) of row `row` in one warp's epilogue
// box: 32 rows of 64 B under the 64-byte swizzle, i.e. chunk c of row r sits
// at chunk c ^ ((r >> 1) & 3) (address bits [4,6) XOR bits [7,9)), the layout
// TMA reads and writes for CU_TENSOR_MAP_SWIZZLE_64B.  The eight rows that one
// 128-byte shared-memory wavefront serves land in eight distinct bank groups.
IDEQ_DEV uint32_t wswz(int row, int c) {
  return (uint32_t)(row * 64 + ((c ^ ((row >> 1) & 3)) << 4));
}

IDEQ_DEV void lds128(uint32_t a, uint4& v) {
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
}
IDEQ_DEV void sts128(uint32_t a, const uint4& v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

template <typename T> struct H2;
template <> struct H2<__nv_bfloat16> {
  using t = __nv_bfloat162;
  static IDEQ_DEV float2 f(t h) { return __bfloat1622float2(h); }
  static IDEQ_DEV t mk(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <> struct H2<__half> {
  using t = __half2;
  static IDEQ_DEV float2 f(t h) { return __half22float2(h); }
  static IDEQ_DEV t mk(float a, float b) { return __floats2half2_rn(a, b); }
};

template <typename T>
IDEQ_DEV void unpack8(const uint4& u, float* v) {
  const typename H2<T>::t* h = (const typename H2<T>::t*)&u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = H2<T>::f(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}
template <typename T>
IDEQ_DEV uint4 pack8(const float* v) {
  uint4 u;
  typename H2<T>::t* h = (typename H2<T>::t*)&u;
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = H2<T>::mk(v[2 * i], v[2 * i + 1]);
  return u;
}

// ---------------------------------------------------------------- CTA pairs
// Two-SM MMAs (tcgen05 with .cta_group::2): the two CTAs of a cluster of two
// compute one M = 256 tile; the even CTA issues the MMAs, each CTA holds its 128
// rows of A and half of the N rows of B at the same shared-memory offsets, and
// each CTA's tensor memory receives its 128 rows of D.

IDEQ_DEV uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address of the same shared-memory variable in CTA `rank` of the cluster.
IDEQ_DEV uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// Arrive on an mbarrier of another CTA of the cluster (cluster-scope release).
IDEQ_DEV void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

// Every thread of both CTAs: all prior shared-memory work of the cluster is done.
IDEQ_DEV void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA loads into this CTA whose completion is counted on an mbarrier of either CTA
// of the pair (bar: a shared::cluster address).
IDEQ_DEV void tma_load_2d_cg2(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

IDEQ_DEV void tma_load_4d_cg2(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                              int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

IDEQ_DEV void tma_load_5d_cg2(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                              int c3, int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// Two-SM MMA (issued by the even CTA of the pair), 16-bit operands.
IDEQ_DEV void umma_cg2(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Converged-warp forms of the pair's MMA and commits (one elected lane issues).
IDEQ_DEV void umma_cg2_el(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred e, p;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

IDEQ_DEV void umma_commit_cg2_both_el(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\t.reg .b16 m;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "mov.b16 m, 3;\n\t"
      "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], m;\n\t}" ::"r"(bar)
      : "memory");
}

IDEQ_DEV void umma_commit_cg2_el(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
          bar)
      : "memory");
}

// Arrive on the mbarrier at this offset in both CTAs of the pair once the pair's
// MMAs issued so far have completed.
IDEQ_DEV void umma_commit_cg2_both(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b16 m;\n\t"
      "mov.b16 m, 3;\n\t"
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], m;\n\t}" ::"r"(bar)
      : "memory");
}

// Arrive on this CTA's mbarrier once the pair's MMAs issued so far have completed.
IDEQ_DEV void umma_commit_cg2(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// cuTensorMapEncodeTiled from the driver, looked up once (null if unavailable).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

}  // namespace ideq
