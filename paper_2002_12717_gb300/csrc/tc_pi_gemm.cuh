// tcgen05 GEMM of the nb^2 x nb^2 x nb^2 products of the G1-G2 right-hand side:
// the GW polarisation (Eq. gwpi) and the particle-particle and particle-hole
// ladder products (Eqs. lambdapp, lambdaph), on operands sliced beforehand.
//
//   D[m][n] = sum_k A[m][k] B[n][k],   M = nb^2 rows, N' = K' = 2 nb^2
//
// Both operands arrive as three BF16 slices x = v0 + v1 + v2 (global memory,
// [slice][row][K], K contiguous), cut by the slicing passes with one power of
// two per row of A and per column of B: v_s is an integer multiple of
// 2^(E - 8 - 8 s), |v0| <= 2^E, at most 8 significant bits, exact in BF16.  So
// for one output element every order-0 product v0 v0 is an integer multiple of
// one grid, and their FP32 sum in TMEM is exact while it stays below 2^24 grid
// steps; the order-1 and order-2 products (v0 v1, v1 v0, v0 v2, v1 v1, v2 v0)
// go to a second accumulator, 2^-8 and smaller, whose truncating FP32
// accumulation then costs little.  The order-3 and order-4 products are not
// formed: with the leading slice 9 bits wide they sit near the FP32 rounding
// of the inputs.  Six BF16 MMAs per 16-element K step.
//
// No converter stage: a warp issues TMA loads of the three slices of a 128-row
// A tile and a 256-row B tile per 32-element K block into a 3-stage ring, one
// thread issues the MMAs (M = 128, N = 256) into two accumulators of 256 TMEM
// columns each (512 columns, single-buffered), and four warps drain TMEM into
// the output after the last K block of a tile.  Persistent over tiles, column
// tile outer so that the CTAs running at one time share their B column tiles
// in L2.  All mbarrier waits are bounded and report through the error word.
#pragma once

#include "tc_ptx.cuh"

namespace g1g2 {
namespace tc {

constexpr int kPiTileM = 128;
constexpr int kPiTileN = 256;
constexpr int kPiBlockK = 32;                                   // BF16 per K block (64-byte rows)
constexpr int kPiSlices = 3;
constexpr uint32_t kPiASlice = kPiTileM * kPiBlockK * 2;        // 8 KB
constexpr uint32_t kPiBSlice = kPiTileN * kPiBlockK * 2;        // 16 KB
constexpr uint32_t kPiBOff = kPiSlices * kPiASlice;             // 24 KB: B slices within a stage
constexpr uint32_t kPiStageBytes = kPiBOff + kPiSlices * kPiBSlice;  // 72 KB
constexpr int kPiStages = 3;
constexpr int kPiThreads = 192;                                 // TMA warp, MMA warp, 4 epilogue warps
constexpr uint32_t kPiD1Col = 256;                              // TMEM column of the second accumulator
constexpr size_t kPiSmemBytes = 1024 + kPiStages * kPiStageBytes + 256;

struct PiGemmParams {
  int nb;        // row m = (a, b) = a nb + b; column n = (c, d, v) = 2 (c nb + d) + v
  int M;         // rows (nb^2)
  int ncols;     // output columns (2 nb^2)
  int kblocks;   // K' / 32
  int mtiles;    // row tiles of 128
  int tiles;     // mtiles x column tiles; tile = n_tile * mtiles + m_tile
  float2 *out;   // out[a][c][d][b], complex: (D[m][2cd], D[m][2cd + 1])
  int out_blk;   // out in 4^4 blocks: blk4(nb, a, c, d, b)
  int *err;
};

__global__ void __launch_bounds__(kPiThreads, 1)
    tc_pi_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const PiGemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kPiStages * kPiStageBytes);
  uint64_t *full = bars;
  uint64_t *empty = bars + kPiStages;
  uint64_t *tfull = bars + 2 * kPiStages;
  uint64_t *tempty = tfull + 1;
  uint64_t *fin = tempty + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPiStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 128);
    mbar_init(fin, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int m0 = (tile % p.mtiles) * kPiTileM, n0 = (tile / p.mtiles) * kPiTileN;
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!mbar_wait(&empty[s], ph ^ 1u, p.err)) { ok = false; break; }
          uint8_t *st = smem + (size_t)s * kPiStageBytes;
          mbar_arrive_expect_tx(&full[s], kPiStageBytes);
          tma_load_3d(st, &tmA, &full[s], kb * kPiBlockK, m0, 0);             // three A slices
          tma_load_3d(st + kPiBOff, &tmB, &full[s], kb * kPiBlockK, n0, 0);   // three B slices
          if (++s == kPiStages) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kPiTileM, kPiTileN);
      const uint32_t d0 = tmem_base, d1 = tmem_base + kPiD1Col;
      int s = 0;
      uint32_t ph = 0, acc_ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        if (!mbar_wait(tempty, acc_ph ^ 1u, p.err)) break;   // the epilogue has drained the last tile
        tc_fence_after();
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!mbar_wait(&full[s], ph, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * kPiStageBytes), sb = sa + kPiBOff;
#pragma unroll
          for (int k = 0; k < kPiBlockK / 16; ++k) {
            uint64_t a[kPiSlices], b[kPiSlices];
#pragma unroll
            for (int q = 0; q < kPiSlices; ++q) {
              a[q] = smem_desc_sw64(sa + q * kPiASlice + 32 * k);
              b[q] = smem_desc_sw64(sb + q * kPiBSlice + 32 * k);
            }
            const uint32_t acc = (kb | k) ? 1u : 0u;
            mma_bf16(d0, a[0], b[0], idesc, acc);   // order 0: exact integer sums
            mma_bf16(d1, a[0], b[1], idesc, acc);   // order 1
            mma_bf16(d1, a[1], b[0], idesc, 1u);
            mma_bf16(d1, a[0], b[2], idesc, 1u);    // order 2
            mma_bf16(d1, a[1], b[1], idesc, 1u);
            mma_bf16(d1, a[2], b[0], idesc, 1u);
          }
          mma_commit(&empty[s]);   // the stage is free once these MMAs have read it
          if (++s == kPiStages) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull);
        acc_ph ^= 1u;
      }
      // every MMA issued by this thread has completed before TMEM is released
      mma_commit(fin);
      mbar_wait(fin, 0, p.err);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-5)
    const int r = 32 * (warp & 3) + lane;                     // TMEM lane == tile row
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const long long N = p.nb;
    uint32_t acc_ph = 0;
    for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
      // warp-uniform: the TMEM loads below are .sync.aligned
      if (!__all_sync(0xffffffffu, mbar_wait(tfull, acc_ph, p.err))) break;
      tc_fence_after();
      const int m = (tile % p.mtiles) * kPiTileM + r, n0 = (tile / p.mtiles) * kPiTileN;
      const bool valid = m < p.M;
      const long long a = m / p.nb, b = m - a * p.nb;
#pragma unroll 1
      for (int c0 = 0; c0 < kPiTileN; c0 += 32) {
        float v[32], w[32];
        tmem_ld32(tmem_base + lane_base + (uint32_t)c0, v);
        tmem_ld32(tmem_base + lane_base + kPiD1Col + (uint32_t)c0, w);
        if (!valid) continue;
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          const int col = n0 + c0 + j;
          if (col >= p.ncols) break;
          const long long cd = col >> 1;
          const long long c = cd / N, d = cd - c * N;
          p.out[p.out_blk ? blk4(N, a, c, d, b) : ((a * N + c) * N + d) * N + b] =
              make_float2(v[j] + w[j], v[j + 1] + w[j + 1]);
        }
      }
      tc_fence_before();
      mbar_arrive(tempty);
      acc_ph ^= 1u;
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

}  // namespace tc
}  // namespace g1g2
