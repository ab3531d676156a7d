// The sliced (bf16x4) nb^5 GEMM for wide outputs (128 < nout <= 192, i.e.
// nb > 64): the same arithmetic as tc_gemm_kernel<true> -- four BF16 slices of
// A and B, the order-0 product into an exact accumulator, the nine products of
// order 1-3 into a second one -- with a different data path:
//
//  * the converters write the A slices straight into tensor memory
//    (tcgen05.st) and the MMAs read A from there, so the A slices never pass
//    through shared memory (ten MMAs per 16-element K step would read them
//    ten times);
//  * one MMA spans the whole output width (N = nout): wait-time counters put
//    the tensor core near its nominal rate while it runs N = 192 MMAs, and at
//    about 60% of that rate on the same work as N = 96 MMAs, so the two
//    accumulators (2 x 192 columns) stay single-buffered and the epilogue is
//    made short instead (epi_store_tile_t): planar outputs go from TMEM
//    through a staging tile in shared memory, 16 columns at a time, and every
//    lane stores four consecutive rows of a column as one 16-byte vector;
//    interleaved complex outputs are stored per row without a branch per
//    element (one 4-byte store per row and column took 3-7 us a tile, as long
//    as the MMAs);
//  * B arrives in a ring of its own, three stages deep, filled by a producer
//    warp of its own;
//  * the FP32 A tiles land in a ring of their own slots.
//
// TMEM (512 columns): exact accumulator at column 0, lower-order one at 192,
// two A-slice buffers of 64 columns at 384 and 448: four slices of a 128 x 32
// tile, two BF16 per 32-bit column, slice q at +16 q, the 16-element K step k
// at +8 k.
//
// Warps (480 threads): 0 A producer, 1 TMEM owner and MMA issuer, 2 B
// producer, 3-10 converters (two per TMEM lane quarter, one per half of the
// 32-element K block), 11-14 epilogue.  Persistent over row tiles; every
// mbarrier wait is bounded and reports through the error word.
#pragma once

#include "tc_gemm.cuh"

namespace g1g2 {
namespace tc {

constexpr int kTsThreads = 480;
constexpr int kTsConvWarp0 = 3;
constexpr int kTsConvThreads = 256;
constexpr int kTsEpiWarp0 = 11;
constexpr int kTsBStages = 3;
// TMEM columns: exact accumulator, lower-order accumulator, A-slice buffer a
constexpr uint32_t kTsD1Col = 192;
__host__ __device__ constexpr uint32_t ts_abuf(int a) { return 384u + 64u * (uint32_t)a; }

// rows of the B box: the whole output width
__host__ __device__ constexpr int ts_nt(int nout) { return nout; }

__host__ __device__ constexpr uint32_t ts_bstage_bytes(int nout) { return (uint32_t)kSlices * nout * kBlockK * 2; }

// dynamic shared memory and FP32 slots of tc_gemm_ts_kernel for an output of nout columns
__host__ __device__ constexpr int ts_fstages(int nout) {
  return (int)((224u * 1024u - kTsBStages * ts_bstage_bytes(nout) - kStgAll) / kABytes) > 6
             ? 6
             : (int)((224u * 1024u - kTsBStages * ts_bstage_bytes(nout) - kStgAll) / kABytes);
}
__host__ __device__ constexpr size_t ts_smem_bytes(int nout) {
  return 1024 + (size_t)ts_fstages(nout) * kABytes + (size_t)kTsBStages * ts_bstage_bytes(nout) + kStgAll + 256;
}

__global__ void __launch_bounds__(kTsThreads, 1)
    tc_gemm_ts_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nf = ts_fstages(p.nout);
  const uint32_t b_bytes = (uint32_t)p.nout * kBlockK * 2;     // one slice of a B stage
  const uint32_t bstage = ts_bstage_bytes(p.nout);
  uint8_t *fring = smem;
  uint8_t *bring = smem + (size_t)nf * kABytes;
  float *stg_all = reinterpret_cast<float *>(bring + (size_t)kTsBStages * bstage);   // epilogue staging
  uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(stg_all) + kStgAll);
  uint64_t *ffull = bars;                     // FP32 A tile landed in slot
  uint64_t *fempty = ffull + nf;              // slot read by the converters
  uint64_t *bfull = fempty + nf;              // B slices landed in stage
  uint64_t *bempty = bfull + kTsBStages;      // stage read by the MMAs
  uint64_t *aready = bempty + kTsBStages;     // A slices stored in TMEM buffer
  uint64_t *afree = aready + 2;               // TMEM buffer read by the MMAs
  uint64_t *tfull = afree + 2;                // accumulators complete
  uint64_t *tempty = tfull + 1;               // accumulators drained
  uint64_t *fin = tempty + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int f = 0; f < nf; ++f) {
      mbar_init(&ffull[f], 1);
      mbar_init(&fempty[f], kTsConvThreads);
    }
    for (int b = 0; b < kTsBStages; ++b) {
      mbar_init(&bfull[b], 1);
      mbar_init(&bempty[b], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&aready[a], kTsConvThreads);
      mbar_init(&afree[a], 1);
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
    // ------------------------------------------------------------ A producer (FP32 tiles)
    if (lane == 0) {
      int f = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&fempty[f], ph ^ 1u, p.err)) { ok = false; break; }
          uint8_t *dst = fring + (size_t)f * kABytes;
          mbar_arrive_expect_tx(&ffull[f], kABytes);
          if (p.a_rows == AR_LINEAR) {
            const int u = kb / p.kb_per_plane, pb = kb % p.kb_per_plane;
            tma_load_3d(dst, &tmA, &ffull[f], pb * kBlockK, tile * kTileM, u);
          } else {  // AR_GATHER4
            const int u = kb / p.kb_per_plane, pb = kb % p.kb_per_plane;
            const int bB = tile % p.g_nb, aB = (tile / p.g_nb) % p.g_na, c = tile / (p.g_nb * p.g_na);
            tma_load_5d(dst, &tmA, &ffull[f], pb * kBlockK, c, bB * 32, aB * 4, u);
          }
          if (++f == nf) { f = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ B producer (slices)
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&bempty[s], ph ^ 1u, p.err)) { ok = false; break; }
          int bk, brow;
          b_coords(p, tile, kb, bk, brow);
          mbar_arrive_expect_tx(&bfull[s], kSlices * b_bytes);
          tma_load_3d(bring + (size_t)s * bstage, &tmB, &bfull[s], bk, brow, 0);   // all four slices
          if (++s == kTsBStages) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kTileM, p.nout);
      const uint32_t d0 = tmem_base, d1 = tmem_base + kTsD1Col;
      int s = 0, a = 0;
      uint32_t ph = 0, aph = 0, acc_ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        if (!mbar_wait(tempty, acc_ph ^ 1u, p.err)) break;   // the epilogue has drained the last tile
        tc_fence_after();
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&aready[a], aph, p.err) || !mbar_wait(&bfull[s], ph, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ab = tmem_base + ts_abuf(a);
          const uint32_t bs0 = smem_u32(bring + (size_t)s * bstage);
#pragma unroll
          for (int k = 0; k < kBlockK / 16; ++k) {
            uint32_t at[kSlices];
            uint64_t bd[kSlices];
#pragma unroll
            for (int q = 0; q < kSlices; ++q) {
              at[q] = ab + 16u * q + 8u * k;
              bd[q] = smem_desc_sw64(bs0 + q * b_bytes + 32 * k);
            }
            const uint32_t acc_in = (kb | k) ? 1u : 0u;
            mma_bf16_ts(d0, at[0], bd[0], idesc, acc_in);          // exact: integers < 2^24
            mma_bf16_ts(d1, at[0], bd[1], idesc, acc_in);          // order 1 ...
            mma_bf16_ts(d1, at[1], bd[0], idesc, 1u);
            mma_bf16_ts(d1, at[0], bd[2], idesc, 1u);              // order 2
            mma_bf16_ts(d1, at[1], bd[1], idesc, 1u);
            mma_bf16_ts(d1, at[2], bd[0], idesc, 1u);
            mma_bf16_ts(d1, at[0], bd[3], idesc, 1u);              // order 3
            mma_bf16_ts(d1, at[1], bd[2], idesc, 1u);
            mma_bf16_ts(d1, at[2], bd[1], idesc, 1u);
            mma_bf16_ts(d1, at[3], bd[0], idesc, 1u);
          }
          mma_commit(&bempty[s]);   // the B stage and the A buffer are free once these MMAs have read them
          mma_commit(&afree[a]);
          if (++s == kTsBStages) { s = 0; ph ^= 1u; }
          if (++a == 2) { a = 0; aph ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull);
        acc_ph ^= 1u;
      }
      // every MMA issued by this thread has completed before TMEM is released
      mma_commit(fin);
      mbar_wait(fin, 0, p.err);
    }
  } else if (warp < kTsEpiWarp0) {
    // ------------------------------------------------------------ converters
    const int quarter = warp & 3, half = (warp - kTsConvWarp0) >> 2;
    const int r = 32 * quarter + lane;                                   // tile row == TMEM lane
    const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
    uint64_t cut2[kSlices];
    {
      const int E = slice_exponent(p.a_amax ? *p.a_amax : 0);
      const int Ld = p.slice_lead ? p.slice_lead : 7;
#pragma unroll
      for (int q = 0; q < kSlices; ++q) cut2[q] = splat_f32x2(ldexpf(1.5f, 23 + E - Ld - 8 * q));
    }
    int f = 0, a = 0;
    uint32_t fph = 0, aph = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
      const int nkb = tile_kblocks(p, tile);
      for (int kb = 0; kb < nkb; ++kb) {
        // warp-uniform waits: the TMEM stores below are .sync.aligned
        if (!__all_sync(0xffffffffu, mbar_wait(&afree[a], aph ^ 1u, p.err) && mbar_wait(&ffull[f], fph, p.err))) {
          ok = false;
          break;
        }
        tc_fence_after();
        // this thread's half row: logical floats 16 half .. 16 half + 15 of row r, four
        // 16-byte chunks of the 128-byte-swizzled FP32 tile
        const uint8_t *rowp = fring + (size_t)f * kABytes + (size_t)r * 128;
        uint32_t w[kSlices][8];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int chunk = 4 * half + c;
          const float4 x = *reinterpret_cast<const float4 *>(rowp + ((chunk ^ (r & 7)) << 4));
          float2 lo2[kSlices], hi2[kSlices];
          slice4x2(make_float2(x.x, x.y), lo2, cut2);
          slice4x2(make_float2(x.z, x.w), hi2, cut2);
#pragma unroll
          for (int q = 0; q < kSlices; ++q) {
            w[q][2 * c] = pack_bf16(lo2[q].x, lo2[q].y);
            w[q][2 * c + 1] = pack_bf16(hi2[q].x, hi2[q].y);
          }
        }
        const uint32_t ab = tmem_base + lane_addr + ts_abuf(a) + 8u * half;
#pragma unroll
        for (int q = 0; q < kSlices; ++q) tmem_st8(ab + 16u * q, w[q]);
        tmem_wait_st();
        tc_fence_before();
        fence_proxy_async_smem();   // the FP32 slot's reads precede its next TMA write
        mbar_arrive(&aready[a]);
        mbar_arrive(&fempty[f]);
        if (++f == nf) { f = 0; fph ^= 1u; }
        if (++a == 2) { a = 0; aph ^= 1u; }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 11-14)
    const int r = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    float *stg = stg_all + (warp - kTsEpiWarp0) * (kStgCols * kStgPitch);
    uint32_t acc_ph = 0;
    float mx = 0.f;
    for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
      if (!__all_sync(0xffffffffu, mbar_wait(tfull, acc_ph, p.err))) break;
      tc_fence_after();
      epi_store_tile_t(p, tile, r, tmem_base + lane_base, kTsD1Col, mx, stg);
      tc_fence_before();
      mbar_arrive(tempty);
      acc_ph ^= 1u;
    }
    if (p.out_amax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) atomicMax(p.out_amax, __float_as_int(mx));
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
