// The split-K GEMM of the collision integral (Eq. eom_gone-I) in the sliced
// (bf16x4) form:  D_(u,split)[j][i] = sum_{c in split} G_u[j][c] w[i][c],  c =
// (k, l, p) over nb^3 terms, output nb x nb per plane u and K split, summed over
// the splits in FP64 by collision_reduce_kernel.  The arithmetic is that of
// tc_gemm_kernel<true> on AR_SPLITK tiles -- four BF16 slices of A (cut in the
// kernel, one exponent per tensor) and of w (cut beforehand), the order-0
// product into an exact accumulator, the nine products of order 1-3 into a
// second one, the accumulators drained every kb_chunks K blocks (while the
// order-0 sums stay below 2^24 grid steps) into a compensated (sum, error) FP32
// pair per output in shared memory -- with the data path of the TMEM-A kernel:
//
//  * the operands stream from HBM once (both are nb^4 tensors) and the kernel is
//    bound by keeping enough of them in flight: w's slices arrive in a ring of
//    their own (three to eight stages, as shared memory allows), filled by a
//    producer warp ahead of the MMAs, and G's FP32 tiles in a ring of four slots (in tc_gemm_kernel the B
//    load of a K block started only when an MMA stage came free, and the pass
//    ran at a fifth of the HBM rate);
//  * the converters write the A slices into tensor memory, the MMAs read A from
//    there;
//  * with N = nb <= 96 two accumulator pairs fit beside the A buffers, so the
//    drain of one K chunk overlaps the MMAs of the next.
//
// TMEM (512 columns): accumulator pair b (exact, lower-order) at columns 192 b
// and 192 b + 96; A-slice buffers at 384 and 448.  Warps (480 threads): 0 A
// producer, 1 TMEM owner and MMA issuer, 2 B producer, 3-10 converters, 11-14
// the chunk drain (TMEM lane = output row j).  Persistent over tiles (tile =
// 2 split + u); every mbarrier wait is bounded and reports through the error word.
#pragma once

#include "tc_gemm_ts.cuh"

namespace g1g2 {
namespace tc {

constexpr uint32_t kCtD1Off = 96;
constexpr int kCtFStages = 4;   // FP32 A slots
__host__ __device__ constexpr uint32_t ct_dcol(int b) { return 192u * (uint32_t)b; }

__host__ __device__ constexpr uint32_t ct_bstage_bytes(int nout) { return (uint32_t)kSlices * nout * kBlockK * 2; }
// bytes of the (sum, error) pairs: nb rows of n_valid + 1 (odd row stride: no bank conflicts)
__host__ __device__ constexpr size_t ct_acc_bytes(int nb, int n_valid) { return (size_t)nb * (n_valid + 1) * 8; }
// B stages: what shared memory holds beside four FP32 slots and the pairs, at most eight
// (a K block's MMAs take 640 cycles at N = 64, so the B ring must cover the HBM latency
// with several blocks)
__host__ __device__ constexpr int ct_bstages(int nout, size_t acc_bytes) {
  return (int)((224u * 1024u - kCtFStages * kABytes - acc_bytes) / ct_bstage_bytes(nout)) > 8
             ? 8
             : (int)((224u * 1024u - kCtFStages * kABytes - acc_bytes) / ct_bstage_bytes(nout));
}
__host__ __device__ constexpr size_t ct_smem_bytes(int nout, size_t acc_bytes) {
  return 1024 + (size_t)kCtFStages * kABytes + (size_t)ct_bstages(nout, acc_bytes) * ct_bstage_bytes(nout) +
         acc_bytes + 512;   // barriers: up to 8 B stages
}

__global__ void __launch_bounds__(kTsThreads, 1)
    tc_collision_ts_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                           const GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int N = p.nb;
  const int nv = p.n_valid;
  const int ld = nv + 1;
  const size_t acc_bytes = ct_acc_bytes(N, nv);
  const int nf = kCtFStages;
  const int nbs = ct_bstages(p.nout, acc_bytes);
  const uint32_t b_bytes = (uint32_t)p.nout * kBlockK * 2;     // one slice of a B stage
  const uint32_t bstage = ct_bstage_bytes(p.nout);
  const int C = p.kb_chunks;                                    // K blocks per TMEM accumulation
  uint8_t *fring = smem;
  uint8_t *bring = smem + (size_t)nf * kABytes;
  float2 *acc2 = reinterpret_cast<float2 *>(bring + (size_t)nbs * bstage);   // (sum, error) pairs
  uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(acc2) + acc_bytes);
  uint64_t *ffull = bars;                     // FP32 A tile landed in slot
  uint64_t *fempty = ffull + nf;              // slot read by the converters
  uint64_t *bfull = fempty + nf;              // B slices landed in stage
  uint64_t *bempty = bfull + nbs;      // stage read by the MMAs
  uint64_t *aready = bempty + nbs;     // A slices stored in TMEM buffer
  uint64_t *afree = aready + 2;               // TMEM buffer read by the MMAs
  uint64_t *tfull = afree + 2;                // accumulator pair holds a finished chunk (two)
  uint64_t *tempty = tfull + 2;               // accumulator pair drained (two)
  uint64_t *fin = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int f = 0; f < nf; ++f) {
      mbar_init(&ffull[f], 1);
      mbar_init(&fempty[f], kTsConvThreads);
    }
    for (int b = 0; b < nbs; ++b) {
      mbar_init(&bfull[b], 1);
      mbar_init(&bempty[b], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&aready[a], kTsConvThreads);
      mbar_init(&afree[a], 1);
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    mbar_init(fin, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ A producer (FP32 tiles of G)
    if (lane == 0) {
      int f = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        const int u = splitk_plane(tile), split = splitk_split(tile);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&fempty[f], ph ^ 1u, p.err)) { ok = false; break; }
          mbar_arrive_expect_tx(&ffull[f], kABytes);
          // rows j = 0..127 of plane u (rows past nb read as zero)
          tma_load_3d(fring + (size_t)f * kABytes, &tmA, &ffull[f], (split * p.kb_per_split + kb) * kBlockK, 0, u);
          if (++f == nf) { f = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ B producer (slices of w)
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
          if (++s == nbs) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kTileM, p.nout);
      int s = 0, a = 0, chunk = 0;
      uint32_t ph = 0, aph = 0;
      uint32_t d0 = tmem_base, d1 = tmem_base + kCtD1Off;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        for (int kb = 0; kb < nkb; ++kb) {
          const int kc = kb % C;
          if (kc == 0) {
            // the drain of this pair's previous chunk is done
            const int buf = chunk & 1;
            if (!mbar_wait(&tempty[buf], ((uint32_t)(chunk >> 1) & 1u) ^ 1u, p.err)) { ok = false; break; }
            tc_fence_after();
            d0 = tmem_base + ct_dcol(buf);
            d1 = d0 + kCtD1Off;
          }
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
            const uint32_t acc_in = (kc | k) ? 1u : 0u;
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
          if (++s == nbs) { s = 0; ph ^= 1u; }
          if (++a == 2) { a = 0; aph ^= 1u; }
          if (kc == C - 1 || kb == nkb - 1) {
            mma_commit(&tfull[chunk & 1]);
            ++chunk;
          }
        }
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
    // ------------------------------------------------------------ chunk drain (warps 11-14)
    const int r = 32 * (warp & 3) + lane;                      // output row j == TMEM lane
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int chunk = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
      const int nkb = tile_kblocks(p, tile);
      const int u = splitk_plane(tile), split = splitk_split(tile);
      if (r < N)
        for (int col = 0; col < nv; ++col) acc2[r * ld + col] = make_float2(0.f, 0.f);
      const int nchunks = (nkb + C - 1) / C;
      for (int ch = 0; ch < nchunks; ++ch, ++chunk) {
        const int buf = chunk & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&tfull[buf], (uint32_t)(chunk >> 1) & 1u, p.err))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem_base + lane_base + ct_dcol(buf);
        for (int c0 = 0; c0 < p.nout; c0 += 32) {
          float v[32], vl[32];
          tmem_ld32(tbase + (uint32_t)c0, v);
          tmem_ld32(tbase + kCtD1Off + (uint32_t)c0, vl);
          if (r < N) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (c0 + j < nv) {
                // Knuth's TwoSum of the running pair and this chunk's sum
                float2 a = acc2[r * ld + c0 + j];
                const float x = v[j] + vl[j];
                const float sum = a.x + x;
                const float bp = sum - a.x;
                a.y += (a.x - (sum - bp)) + (x - bp);
                a.x = sum;
                acc2[r * ld + c0 + j] = a;
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
      }
      if (!ok) break;
      if (r < N)
        for (int col = 0; col < nv; ++col) {
          const float2 a = acc2[r * ld + col];
          p.out64[(((long long)split * 2 + u) * N + r) * nv + col] = (double)a.x + (double)a.y;
        }
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
