// Inline-PTX helpers for the sm_103a tensor-core path: mbarriers with bounded
// waits, TMA tiled loads, TMEM allocation, tcgen05.mma (kind::f16 with BF16
// operands, kind::tf32), tcgen05.ld, and the BF16 slicing of FP32 values.
// Every wait gives up after a wall-clock limit and reports it through an error
// word instead of spinning forever.
#pragma once

#include <cstdint>
#include <cuda.h>

namespace g1g2 {
namespace tc {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr int kErrTimeout = 1;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Index of element (i0, i1, i2, i3) of an nb^4 tensor (nb % 4 == 0) stored in 4^4 blocks:
// block (i0/4, i1/4, i2/4, i3/4) in row-major order, 256 contiguous elements each, row-major
// inside the block.  The layout of the tensor-core form's assembly inputs and accumulator,
// so that the assembly reads and writes whole blocks.
__host__ __device__ __forceinline__ long long blk4(long long N, long long i0, long long i1, long long i2,
                                                   long long i3) {
  const long long nB = N >> 2;
  return ((((i0 >> 2) * nB + (i1 >> 2)) * nB + (i2 >> 2)) * nB + (i3 >> 2)) * 256 +
         ((((i0 & 3) * 4 + (i1 & 3)) * 4 + (i2 & 3)) * 4 + (i3 & 3));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error word set) when the phase did not complete in
// limit_ns of wall-clock time.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (globaltimer() - t0 > limit_ns) {
        atomicOr(err, kErrTimeout);
        return false;
      }
      if (*(volatile int *)err) return false;  // another role gave up: stop waiting
    }
  }
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- TMEM
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand tile written by TMA with
// 128-byte swizzling (rows of 128 B, 8-row atoms 1024 B apart).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                            // descriptor version
  d |= (uint64_t)2 << 61;                            // 128-byte swizzle
  return d;
}

// Shared-memory matrix descriptor: K-major operand tile with 64-byte rows and
// 64-byte swizzling (8-row atoms 512 B apart), the layout of the bf16 slices.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512u >> 4) << 32;                  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                            // descriptor version
  d |= (uint64_t)4 << 61;                            // 64-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulator, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                       // D format: F32
         | (1u << 7)                     // A format: BF16
         | (1u << 10)                    // B format: BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The same MMA with the A operand in tensor memory: a_tmem addresses M = 128 lanes
// (tile rows) by K/2 columns, two BF16 values per 32-bit column (the lower K index in
// the low half).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 32 lanes x 8 consecutive 32-bit columns per warp, from the calling lane's registers;
// tmem_wait_st() waits until this thread's stores are complete.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Instruction descriptor: kind::tf32, FP32 accumulator, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                       // D format: F32
         | (2u << 7)                     // A format: TF32
         | (2u << 10)                    // B format: TF32
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns per warp.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Exponent E with |x| < 2^E for every x of a tensor whose largest magnitude has
// the FP32 bit pattern mbits (0 for an all-zero tensor).
__host__ __device__ __forceinline__ int slice_exponent(int mbits) {
  return mbits > 0 ? ((mbits >> 23) & 255) - 126 : 0;
}

// Leading-slice width for an exact FP32 accumulation over K terms: with
// |q_0| <= 2^L on both operands the K products sum below 2^24 when
// K 2^(2L) < 2^24; L = 7 (8-bit slices) covers K <= 1024.
__host__ __device__ constexpr int slice_lead_for(long long K) {
  int L = 7;
  while (L > 1 && K * (1LL << (2 * L)) >= (1LL << 24)) --L;
  return L;
}
// Four slices of x (|x| < 2^E): x = v_0 + v_1 + v_2 + v_3 + O(2^(E-L-25)), where
// v_s is an integer multiple of 2^(E-L-8s) with |v_0| <= 2^E and
// |v_s| <= 2^(E-L-8s+7) for s > 0, i.e. at most 8 significant bits: exact in
// BF16.  Each cut rounds the running remainder to nearest-even on its grid by
// adding and subtracting c_s = 1.5 2^(23+E-L-8s) (the sum's ulp is the grid
// step), and the remainder r - v_s is exact in FP32.
__device__ __forceinline__ void slice4(float x, float (&v)[4], const float (&c)[4]) {
  float r = x;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    v[s] = __fsub_rn(__fadd_rn(r, c[s]), c[s]);
    r = __fsub_rn(r, v[s]);
  }
}

// Three slices of x (|x| < 2^E) with a 9-bit leading slice (L = 8): the cuts of slice4
// with c_q = 1.5 2^(15 + E - 8q) (cuts3_lead8); v_q is x's remainder rounded to
// nearest-even on the grid 2^(E - 8 - 8q), |v_0| <= 2^E, |v_1|, |v_2| <= 2^(E - 9 - 8(q - 1)),
// each exact in BF16.  The part of x below 2^(E - 25) is dropped.
__device__ __forceinline__ void cuts3_lead8(int E, float (&c)[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) c[q] = ldexpf(1.5f, 15 + E - 8 * q);
}
__device__ __forceinline__ void slice3(float x, const float (&c)[3], float (&v)[3]) {
  float r = x;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    v[q] = __fsub_rn(__fadd_rn(r, c[q]), c[q]);
    r = __fsub_rn(r, v[q]);
  }
}

// slice4 on two values at once with packed FP32x2 adds (round to nearest per lane,
// the same results as slice4 on each).  c2[s] holds c_s in both halves.
__device__ __forceinline__ void slice4x2(float2 x, float2 (&v)[4], const uint64_t (&c2)[4]) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x.x), "f"(x.y));
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    uint64_t t, vs;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(r), "l"(c2[s]));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(vs) : "l"(t), "l"(c2[s]));
    if (s < 3) asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(r), "l"(vs));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v[s].x), "=f"(v[s].y) : "l"(vs));
  }
}
__device__ __forceinline__ uint64_t splat_f32x2(float c) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(c));
  return r;
}

// two FP32 values -> packed BF16 pair (lo in the low half), round to nearest
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Round to the nearest TF32 value (10 explicit mantissa bits), kept in an FP32 container.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace g1g2
