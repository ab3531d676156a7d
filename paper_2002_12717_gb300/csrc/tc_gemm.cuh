// Persistent tcgen05 GEMM for the nb^5 contractions of the G1-G2 right-hand
// side, in two split-precision operand forms.
//
//   D[m][n] = sum_k A[m][k] B[n][k]        (both operands K-major)
//
// A is a big FP32 tensor streamed by TMA (128-row tiles, 32-float K blocks,
// 128-byte swizzle); six converter warps turn each landed A tile into the MMA
// operands; B is small and arrives pre-split in global memory.
//
// Sliced form (kSliced, the default "bf16x4"): the converters cut each A
// element, scaled by one power of two per tensor (from its largest magnitude),
// into four integer-valued BF16 slices (8 bits each, Ozaki-style), and B
// arrives as four such slices.  The leading product A_0 B_0 is a sum of
// integers below 2^24 times one common scale, so its FP32 accumulation in TMEM
// is exact whatever rounding the tensor core applies; the nine lower-order
// products (2^-8 and smaller) go to a second accumulator.  This removes the
// systematic round-toward-zero drift of long FP32 tensor-core accumulations,
// at 20 BF16 MMAs per 32-element K block.
//
// TF32 form ("tf32x3"): the converters split A into a round-to-nearest TF32
// "hi" part (in place) and a TF32 "lo" remainder, B arrives as hi and lo
// arrays, and each K step issues three MMAs, A_hi B_hi + A_lo B_hi + A_hi B_lo,
// into one FP32 accumulator (about 21 significant bits of every product).
//
// Accumulators are double-buffered in TMEM where they fit, so the epilogue of
// one tile overlaps the main loop of the next.  Warp roles (384 threads):
// warp 0 TMA producer, warp 1 TMEM owner and MMA issuer, warps 2-7
// converters, warps 8-11 epilogue (TMEM lanes 0..127: a warp reaches the lane
// quarter warp % 4).
#pragma once

#include "tc_ptx.cuh"

namespace g1g2 {
namespace tc {

constexpr int kTileM = 128;
constexpr int kBlockK = 32;                        // floats per K block (128 B)
constexpr uint32_t kABytes = kTileM * kBlockK * 4; // 16 KB
constexpr int kAccCols = 256;                      // TMEM columns per accumulator buffer
constexpr int kGemmThreads = 384;
constexpr int kConvThreads = 192;                  // warps 2-7
constexpr int kEpiWarp0 = 8;                       // first epilogue warp
constexpr int kSlices = 4;                         // BF16 slices per operand (sliced form)
constexpr uint32_t kASliceBytes = kTileM * kBlockK * 2;  // 8 KB: one slice of an A tile, 64-byte rows
constexpr uint32_t kSlicedBOff = kSlices * kASliceBytes;  // 32 KB: B slices within a sliced MMA stage

// shared memory of one MMA stage: TF32 form the FP32 A tile, its lo part and B (hi, lo);
// sliced form the four A slices and the four B slices (the FP32 A tiles land in a ring of
// their own, kABytes per slot)
__host__ __device__ constexpr uint32_t stage_bytes_for(bool sliced, int nout) {
  return sliced ? (uint32_t)kSlices * kASliceBytes + (uint32_t)kSlices * (uint32_t)nout * kBlockK * 2
                : 2 * kABytes + 2 * (uint32_t)nout * kBlockK * 4;
}

enum ARows : int {
  AR_LINEAR = 0,   // A viewed as [plane][row][k]; tile = 128 consecutive rows
  AR_GATHER4 = 1,  // A = T[plane][a][b][c][k]; tile = rows (a: 4, b: 32) at fixed c
  AR_SPLITK = 2,   // A = G[plane][j][c]; tile = 2 (K split) + plane, rows j
  AR_PI = 3,       // TF32 form: A = G[plane][i][p][k][q]; tile rows (i: 4, k: 32), K blocks over (plane, p, q)
};

// Output index maps.  In every map the fastest-varying output index is the
// tile row, so the 32 lanes of a warp store 32 consecutive floats per column.
enum Epi : int {
  EP_SWAP34 = 0,        // row (i,j,k), col l -> out[v][i][j][l][k]
  EP_EXCH_T = 1,        // row (p,q,r), col l -> out[v][q][p][l][r]
  EP_GATHER_TCONJ = 2,  // row (a,b,c), col d -> out[v][c][d][a][b], imaginary plane negated
  EP_PARTIAL = 3,       // split-K sums: partial[split][plane][row][col] (FP64 from a compensated FP32 sum)
  EP_PI = 4,            // row (i,k), col (j,l,v) interleaved -> out[i][j][l][k] interleaved complex
};

struct GemmParams {
  int nb;             // basis size N
  int a_rows;         // ARows
  int epi;            // Epi
  int tiles;          // work items
  int kb_per_plane;   // K blocks per A plane
  int a_planes;       // 1 (real A) or 2 (complex A, planar)
  int nout;           // MMA N (multiple of 16, <= 256)
  int n_valid;        // output columns that are stored
  long long rows;     // AR_LINEAR: valid rows
  int g_na, g_nb;     // AR_GATHER4: number of a-blocks (4) and b-blocks (32)
  int splits;         // AR_SPLITK: K splits per plane
  int kb_per_split;   //            K blocks per split
  int kb_all;         //            K blocks in total
  int kb_chunks;      // AR_SPLITK: K blocks per TMEM accumulation (0: one accumulation per tile),
                      //            chunks summed in shared memory
  double *out64;      //            FP64 partial sums [split][plane][row][col]
  float *out;
  long long out_plane;
  int n_tiles;        // output column tiles of width nout (B rows n_tile*nout ...); 1 for most passes
  int pi_mk, pi_kq;   // AR_PI: number of k-blocks (32) per i-block; q-blocks (32) per p
  int pi_mtiles;      // AR_PI: row tiles; tile = n_tile * pi_mtiles + m_tile (column-tile outer,
                      //        so concurrent CTAs share the B column tile in L2)
  int *err;
  const int *a_amax;  // sliced form: FP32 bit pattern of max |A| (the A slice scale)
  int slice_lead;     // sliced form: leading-slice width L (slice_lead_for(K)); 0 means 7
  int col_il;         // B rows (output columns) ordered 2 l + v instead of v nb + l
  int out_il;         // EP_SWAP34 with col_il: interleaved complex FP32 output out[i][j][l][k]
  int out_blk;        // out_il and EP_PI: that output in 4^4 blocks (blk4 of (i, j, l, k))
  int *out_amax;      // sliced form, optional: atomic max of |stored outputs| (FP32 bits)
};

// AR_SPLITK tiles: tile = 2 split + u, so the two planes of one K split are neighbouring
// tiles, which run at the same time on two SMs and read the same B K blocks: one of the
// two reads comes from L2 instead of HBM.
__device__ __forceinline__ int splitk_plane(int tile) { return tile & 1; }
__device__ __forceinline__ int splitk_split(int tile) { return tile >> 1; }

// K coordinate (elements) and first row of the B tile of K block kb of a tile
__device__ __forceinline__ void b_coords(const GemmParams &p, int tile, int kb, int &bk, int &brow) {
  bk = (p.a_rows == AR_SPLITK) ? (splitk_split(tile) * p.kb_per_split + kb) * kBlockK : kb * kBlockK;
  brow = (p.a_rows == AR_PI) ? (tile / p.pi_mtiles) * p.nout : 0;
}

__device__ __forceinline__ int tile_kblocks(const GemmParams &p, int tile) {
  if (p.a_rows == AR_SPLITK) {
    const int split = splitk_split(tile);
    const int b0 = split * p.kb_per_split;
    const int n = p.kb_all - b0;
    return n < p.kb_per_split ? (n > 0 ? n : 0) : p.kb_per_split;
  }
  if (p.a_rows == AR_PI) return 2 * p.nb * p.pi_kq;
  return p.kb_per_plane * p.a_planes;
}

// Epilogue of one tile of a pass that is not split-K: TMEM lane r (the tile row) of the
// accumulators at tbase (the exact one) and tbase + d1_off (the lower-order one, sliced
// form), summed and stored through the output map of p; mx collects max |stored|.  The
// accumulators hold output columns col0 .. col0 + ncols - 1 (ncols = 0: all p.nout).
template <bool kSliced>
__device__ __forceinline__ void epi_store_tile(const GemmParams &p, int tile, int r, uint32_t tbase,
                                               uint32_t d1_off, float &mx, int col0 = 0, int ncols = 0) {
  const int N = p.nb;
  const long long NN = N;
  // the row this thread owns
  bool valid = false;
  long long i0 = 0, i1 = 0, i2 = 0, grow = 0;
  int u = 0, split = 0;
  if (p.a_rows == AR_LINEAR) {
    grow = (long long)tile * kTileM + r;
    valid = grow < p.rows;
    i2 = grow % NN;
    i1 = (grow / NN) % NN;
    i0 = grow / (NN * NN);
  } else if (p.a_rows == AR_GATHER4) {
    const int bB = tile % p.g_nb, aB = (tile / p.g_nb) % p.g_na, c = tile / (p.g_nb * p.g_na);
    i0 = aB * 4 + r / 32;   // a
    i1 = bB * 32 + r % 32;  // b
    i2 = c;
    valid = i0 < NN && i1 < NN;
  } else if (p.a_rows == AR_PI) {
    const int mt = tile % p.pi_mtiles;
    const int kB = mt % p.pi_mk, iB = mt / p.pi_mk;
    i0 = iB * 4 + r / 32;   // i
    i2 = kB * 32 + r % 32;  // k
    grow = (long long)(tile / p.pi_mtiles) * p.nout;  // first global output column of the tile
    valid = i0 < NN && i2 < NN;
  } else {
    u = splitk_plane(tile);
    split = splitk_split(tile);
    valid = r < N;
  }
  // Store map of this row: out[base + l cs (+ plane for the imaginary part)],
  // with (l, v) decoded from the column (v nb + l, or 2 l + v with col_il).
  long long base = 0;
  int cs = 0;
  bool neg_im = false;
  if (p.epi == EP_SWAP34) {          // out[v][i][j][l][k], row (i,j,k)
    base = (i0 * NN + i1) * NN * NN + i2;
    cs = N;
  } else if (p.epi == EP_EXCH_T) {   // out[v][q][p][l][r], row (p,q,r)
    base = (i1 * NN + i0) * NN * NN + i2;
    cs = N;
  } else if (p.epi == EP_GATHER_TCONJ) {  // out[v][c][d][a][b], row (a,b,c), imaginary negated
    base = i2 * NN * NN * NN + i0 * NN + i1;
    cs = N * N;
    neg_im = true;
  }
  const int nc = ncols ? ncols : p.nout;
  for (int c0 = 0; c0 < nc; c0 += 32) {
    float v[32];
    tmem_ld32(tbase + (uint32_t)c0, v);
    if (kSliced) {
      float vl[32];
      tmem_ld32(tbase + d1_off + (uint32_t)c0, vl);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += vl[j];
    }
    if (!valid) continue;
    const int g0 = col0 + c0;                              // output column of the chunk's first
    const int nv = min(min(32, nc - c0), p.n_valid - g0);  // columns of this chunk that are stored
    if (p.epi == EP_PARTIAL) {
      float *o = p.out + (((long long)split * 2 + u) * NN + r) * p.n_valid + g0;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < nv) o[j] = v[j];
    } else if (p.epi == EP_PI) {
      // columns (j, l, v) interleaved from the even global column grow + g0: complex pairs
      float2 *o = reinterpret_cast<float2 *>(p.out);
      const long long cg0 = grow + g0;
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const long long cg = cg0 + j;
        if (j >= nv || cg >= p.rows) break;
        const long long jl = cg >> 1;
        const long long jj = jl / NN, ll = jl - jj * NN;
        o[p.out_blk ? blk4(NN, i0, jj, ll, i2) : ((i0 * NN + jj) * NN + ll) * NN + i2] =
            make_float2(v[j], v[j + 1]);
      }
    } else if (p.out_il) {
      // col_il columns (2 l, 2 l + 1) -> one interleaved complex value
      float2 *o = reinterpret_cast<float2 *>(p.out) + base;
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        if (j >= nv) break;
        const int l = (g0 + j) >> 1;
        if (p.out_blk)
          reinterpret_cast<float2 *>(p.out)[blk4(NN, i0, i1, l, i2)] = make_float2(v[j], v[j + 1]);
        else
          o[l * cs] = make_float2(v[j], v[j + 1]);
        if (kSliced) mx = fmaxf(mx, fmaxf(fabsf(v[j]), fabsf(v[j + 1])));
      }
    } else if (p.col_il) {
      float *o = p.out + base;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j >= nv) break;
        const int col = g0 + j, vv = col & 1, l = col >> 1;
        const float x = (neg_im && vv) ? -v[j] : v[j];
        o[(long long)l * cs + (vv ? p.out_plane : 0)] = x;
        if (kSliced) mx = fmaxf(mx, fabsf(x));
      }
    } else {
      float *o = p.out + base;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j >= nv) break;
        const int col = g0 + j, vv = col >= N ? 1 : 0, l = col - (vv ? N : 0);
        const float x = (neg_im && vv) ? -v[j] : v[j];
        o[(long long)l * cs + (vv ? p.out_plane : 0)] = x;
        if (kSliced) mx = fmaxf(mx, fabsf(x));
      }
    }
  }
}

// Staging tile of one epilogue warp for epi_store_tile_t: 16 columns x 32 rows of FP32,
// row pitch 36 floats (writes of one column by 32 lanes and 16-byte reads of 4 rows are
// free of bank conflicts).
constexpr int kStgCols = 16;
constexpr int kStgPitch = 36;
constexpr uint32_t kStgBytes = kStgCols * kStgPitch * 4;
constexpr uint32_t kStgAll = 4 * kStgBytes;   // four epilogue warps

// the passes epi_store_tile_t serves
__host__ __device__ __forceinline__ bool epi_transposed(const GemmParams &p) {
  return (p.a_rows == AR_LINEAR || p.a_rows == AR_GATHER4) &&
         (p.epi == EP_SWAP34 || p.epi == EP_EXCH_T || p.epi == EP_GATHER_TCONJ);
}

// Epilogue of one row tile of the sliced form (rows r, output columns 0 .. p.nout - 1) for
// the row maps AR_LINEAR, AR_GATHER4 and the stores EP_SWAP34, EP_EXCH_T, EP_GATHER_TCONJ
// (planar, col_il, or out_il complex, optionally 4^4-blocked) -- every nb^5 pass but the
// collision integral.  Planar outputs: each 32-column chunk read from TMEM goes through
// the warp's staging tile in two halves of 16 columns, so that a lane stores four
// consecutive rows of one column as one 16-byte vector: with nb % 4 == 0 and row tiles
// starting at multiples of 4, four consecutive rows of a warp are four consecutive output
// elements under every one of these maps (and 16-byte aligned); one store per four rows
// and column instead of one per row.  Interleaved complex outputs already fill a 32-byte
// sector with the 8-byte pairs of four rows and are stored per row.  No branch per
// element, and the address split into a per-row base and a per-column term.
__device__ __forceinline__ void epi_store_tile_t(const GemmParams &p, int tile, int r, uint32_t tbase,
                                                 uint32_t d1_off, float &mx, float *stg) {
  const int N = p.nb;
  const long long NN = N;
  const int lane = threadIdx.x & 31;
  // the row this lane owns
  bool valid;
  long long i0, i1, i2;
  if (p.a_rows == AR_LINEAR) {
    const long long grow = (long long)tile * kTileM + r;
    valid = grow < p.rows;
    i2 = grow % NN;
    i1 = (grow / NN) % NN;
    i0 = grow / (NN * NN);
  } else {  // AR_GATHER4
    const int bB = tile % p.g_nb, aB = (tile / p.g_nb) % p.g_na, c = tile / (p.g_nb * p.g_na);
    i0 = aB * 4 + r / 32;
    i1 = bB * 32 + r % 32;
    i2 = c;
    valid = i0 < NN && i1 < NN;
  }
  // per-row part of the output index: planar out[base + l cs (+ plane)], or for out_il the
  // float2 index base + l cs, or blk4(i0, i1, l, i2) = blk4(i0, i1, 0, i2) + blk4(0, 0, l, 0)
  long long base = 0;
  int cs = 0;
  bool neg_im = false;
  if (p.epi == EP_SWAP34) {
    base = (i0 * NN + i1) * NN * NN + i2;
    cs = N;
  } else if (p.epi == EP_EXCH_T) {
    base = (i1 * NN + i0) * NN * NN + i2;
    cs = N;
  } else {  // EP_GATHER_TCONJ
    base = i2 * NN * NN * NN + i0 * NN + i1;
    cs = N * N;
    neg_im = true;
  }
  if (p.out_il && p.out_blk) base = blk4(NN, i0, i1, 0, i2);
  // this lane stores rows 4 q .. 4 q + 3 of the warp's 32, column group jq
  const int q = lane & 7, jq = lane >> 3;
  const long long qbase = __shfl_sync(0xffffffffu, base, 4 * q);
  const bool qvalid = __shfl_sync(0xffffffffu, valid ? 1 : 0, 4 * q) != 0;
  for (int c0 = 0; c0 < p.nout; c0 += 32) {
    float v[32];
    tmem_ld32(tbase + (uint32_t)c0, v);
    {
      float vl[32];
      tmem_ld32(tbase + d1_off + (uint32_t)c0, vl);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += vl[j];
    }
    if (p.out_il) {
      // interleaved complex output: each lane stores its own row, one 8-byte pair per
      // column pair (2 l, 2 l + 1); four rows of a warp fill a 32-byte sector
      const int nv = min(32, p.n_valid - c0);
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        if (valid && j < nv) {
          const int l = (c0 + j) >> 1;
          const long long e = base + (p.out_blk ? blk4(NN, 0, 0, l, 0) : (long long)l * cs);
          reinterpret_cast<float2 *>(p.out)[e] = make_float2(v[j], v[j + 1]);
          mx = fmaxf(mx, fmaxf(fabsf(v[j]), fabsf(v[j + 1])));
        }
      }
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g0 = c0 + kStgCols * h;                       // output column of the half-chunk's first
      const int nv = min(kStgCols, p.n_valid - g0);           // columns of this half-chunk that are stored
#pragma unroll
      for (int j = 0; j < kStgCols; ++j) stg[j * kStgPitch + lane] = v[kStgCols * h + j];
      __syncwarp();
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int jj = 4 * it + jq;
        float4 x = *reinterpret_cast<const float4 *>(stg + jj * kStgPitch + 4 * q);
        if (qvalid && jj < nv) {
          const int col = g0 + jj;
          int vv, l;
          if (p.col_il) {
            vv = col & 1;
            l = col >> 1;
          } else {
            vv = col >= N ? 1 : 0;
            l = col - (vv ? N : 0);
          }
          if (neg_im && vv) x = make_float4(-x.x, -x.y, -x.z, -x.w);
          *reinterpret_cast<float4 *>(p.out + qbase + (long long)l * cs + (vv ? p.out_plane : 0)) = x;
          mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
        }
      }
      __syncwarp();   // the staging tile is read before the next half-chunk overwrites it
    }
  }
}

// tmBhi/tmBlo: TF32 hi and lo parts of B; in the sliced form tmBhi holds the
// four BF16 slices of B as [slice][row][k] (tmBlo unused).
//
// Pipeline.  TF32 form: `stages` stages, each filled by one TMA transaction (A and
// B), converted in place, consumed by the MMAs.  Sliced form: the FP32 A tiles land
// in a ring of `fstages` slots of their own, so that the TMA runs ahead of the
// conversion by the depth of that ring; the converters take an MMA stage (one of
// `stages`), have one of their threads load that K block's B slices into it, cut the
// FP32 tile of the matching slot into the stage's A slices and release the slot.
template <bool kSliced>
__global__ void __launch_bounds__(kGemmThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                   const GemmParams p, const int stages, const int fstages) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t b_bytes = kSliced ? (uint32_t)p.nout * kBlockK * 2 : (uint32_t)p.nout * kBlockK * 4;
  const uint32_t stage_bytes = stage_bytes_for(kSliced, p.nout);
  const int nf = kSliced ? fstages : 0;
  uint8_t *fring = smem;                                   // sliced form: FP32 A slots
  uint8_t *stg = smem + (size_t)nf * kABytes;              // MMA stages
  // accumulator buffers: TF32 form two (double-buffered); sliced form a pair
  // (exact leading product, lower-order products) per buffer, two buffers when they fit
  const int nbuf = (!kSliced || p.nout <= 128) ? 2 : 1;
  const uint32_t d1_off = (nbuf == 2) ? 128u : 256u;
  uint8_t *bar_area = stg + (size_t)stages * stage_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(bar_area);
  uint64_t *full = bars;                // TF32: A and B landed; sliced: B landed
  uint64_t *conv = bars + stages;
  uint64_t *empty = bars + 2 * stages;
  uint64_t *ffull = bars + 3 * stages;  // sliced: FP32 A tile landed in slot
  uint64_t *fempty = ffull + nf;        // sliced: slot read by the converters
  uint64_t *tfull = fempty + nf;
  uint64_t *tempty = tfull + 2;
  uint64_t *fin = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
  float2 *acc2 = reinterpret_cast<float2 *>(bar_area + 256);  // (sum, error) pairs
  float *stg_all = reinterpret_cast<float *>(bar_area + 256);  // or: epilogue staging (kStgAll bytes)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kConvThreads);
      mbar_init(&empty[s], 1);
    }
    for (int f = 0; f < nf; ++f) {
      mbar_init(&ffull[f], 1);
      mbar_init(&fempty[f], kConvThreads);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(fin, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 2 * kAccCols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int N = p.nb;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        for (int kb = 0; kb < nkb; ++kb) {
          // the A tile goes to the FP32 slot (sliced) or to the MMA stage (TF32)
          uint8_t *dst;
          uint64_t *bar;
          if (kSliced) {
            if (!mbar_wait(&fempty[s], ph ^ 1u, p.err)) { ok = false; break; }
            dst = fring + (size_t)s * kABytes;
            bar = &ffull[s];
            mbar_arrive_expect_tx(bar, kABytes);
          } else {
            if (!mbar_wait(&empty[s], ph ^ 1u, p.err)) { ok = false; break; }
            dst = stg + (size_t)s * stage_bytes;
            bar = &full[s];
            mbar_arrive_expect_tx(bar, kABytes + 2 * b_bytes);
          }
          if (p.a_rows == AR_LINEAR) {
            const int u = kb / p.kb_per_plane, pb = kb % p.kb_per_plane;
            tma_load_3d(dst, &tmA, bar, pb * kBlockK, tile * kTileM, u);
          } else if (p.a_rows == AR_GATHER4) {
            const int u = kb / p.kb_per_plane, pb = kb % p.kb_per_plane;
            const int bB = tile % p.g_nb, aB = (tile / p.g_nb) % p.g_na, c = tile / (p.g_nb * p.g_na);
            tma_load_5d(dst, &tmA, bar, pb * kBlockK, c, bB * 32, aB * 4, u);
          } else if (p.a_rows == AR_PI) {
            const int mt = tile % p.pi_mtiles;
            const int kB = mt % p.pi_mk, iB = mt / p.pi_mk;
            const int qb = kb % p.pi_kq, rest = kb / p.pi_kq;
            const int pp = rest % N, u = rest / N;
            tma_load_5d(dst, &tmA, bar, qb * kBlockK, kB * 32, pp, iB * 4, u);
          } else {
            const int u = splitk_plane(tile), split = splitk_split(tile);
            tma_load_3d(dst, &tmA, bar, (split * p.kb_per_split + kb) * kBlockK, 0, u);
          }
          if (!kSliced) {
            int bk, brow;
            b_coords(p, tile, kb, bk, brow);
            tma_load_3d(dst + 2 * kABytes, &tmBhi, bar, bk, brow, 0);
            tma_load_3d(dst + 2 * kABytes + b_bytes, &tmBlo, bar, bk, brow, 0);
          }
          if (++s == (kSliced ? nf : stages)) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = kSliced ? idesc_bf16(kTileM, p.nout) : idesc_tf32(kTileM, p.nout);
      int s = 0, acc = 0;
      uint32_t ph = 0, acc_ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        if (!p.kb_chunks) {
          if (!mbar_wait(&tempty[acc], acc_ph ^ 1u, p.err)) break;
          tc_fence_after();
        }
        for (int kb = 0; kb < nkb; ++kb) {
          const bool chunk_start = p.kb_chunks && (kb % p.kb_chunks == 0);
          const bool chunk_end = p.kb_chunks && (kb % p.kb_chunks == p.kb_chunks - 1 || kb == nkb - 1);
          if (chunk_start) {
            if (!mbar_wait(&tempty[acc], acc_ph ^ 1u, p.err)) { ok = false; break; }
            tc_fence_after();
          }
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kAccCols);
          const uint32_t first = p.kb_chunks ? (uint32_t)(kb % p.kb_chunks) : (uint32_t)kb;
          if (!mbar_wait(&conv[s], ph, p.err)) { ok = false; break; }
          if (kSliced && !mbar_wait(&full[s], ph, p.err)) { ok = false; break; }   // B slices landed
          tc_fence_after();
          const uint32_t sa = smem_u32(stg + (size_t)s * stage_bytes);
          if (kSliced) {
            // slice q of A at sa + q * kASliceBytes, of B at sa + kSlicedBOff + q * b_bytes
            const uint32_t as0 = sa, bs0 = sa + kSlicedBOff;
#pragma unroll
            for (int k = 0; k < kBlockK / 16; ++k) {
              uint64_t ad[kSlices], bd[kSlices];
#pragma unroll
              for (int q = 0; q < kSlices; ++q) {
                ad[q] = smem_desc_sw64(as0 + q * kASliceBytes + 32 * k);
                bd[q] = smem_desc_sw64(bs0 + q * b_bytes + 32 * k);
              }
              const uint32_t acc_in = (first | (uint32_t)k) ? 1u : 0u;
              mma_bf16(d_tmem, ad[0], bd[0], idesc, acc_in);               // exact: integers < 2^24
              mma_bf16(d_tmem + d1_off, ad[0], bd[1], idesc, acc_in);      // order 1 ...
              mma_bf16(d_tmem + d1_off, ad[1], bd[0], idesc, 1u);
              mma_bf16(d_tmem + d1_off, ad[0], bd[2], idesc, 1u);          // order 2
              mma_bf16(d_tmem + d1_off, ad[1], bd[1], idesc, 1u);
              mma_bf16(d_tmem + d1_off, ad[2], bd[0], idesc, 1u);
              mma_bf16(d_tmem + d1_off, ad[0], bd[3], idesc, 1u);          // order 3
              mma_bf16(d_tmem + d1_off, ad[1], bd[2], idesc, 1u);
              mma_bf16(d_tmem + d1_off, ad[2], bd[1], idesc, 1u);
              mma_bf16(d_tmem + d1_off, ad[3], bd[0], idesc, 1u);
            }
          } else {
            const uint32_t sal = sa + kABytes, sbh = sa + 2 * kABytes, sbl = sbh + b_bytes;
#pragma unroll
            for (int k = 0; k < kBlockK / 8; ++k) {
              const uint64_t ah = smem_desc_sw128(sa + 32 * k), al = smem_desc_sw128(sal + 32 * k);
              const uint64_t bh = smem_desc_sw128(sbh + 32 * k), bl = smem_desc_sw128(sbl + 32 * k);
              mma_tf32(d_tmem, ah, bh, idesc, (first | (uint32_t)k) ? 1u : 0u);
              mma_tf32(d_tmem, al, bh, idesc, 1u);
              mma_tf32(d_tmem, ah, bl, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
          if (++s == stages) { s = 0; ph ^= 1u; }
          if (chunk_end) {
            mma_commit(&tfull[acc]);
            if (++acc == nbuf) { acc = 0; acc_ph ^= 1u; }
          }
        }
        if (!ok) break;
        if (!p.kb_chunks) {
          mma_commit(&tfull[acc]);
          if (++acc == nbuf) { acc = 0; acc_ph ^= 1u; }
        }
      }
      // every MMA issued by this thread has completed before TMEM is released
      mma_commit(fin);
      mbar_wait(fin, 0, p.err);
    }
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------------------ converters
    const int ct = threadIdx.x - 64;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    // sliced form: rounding constants c_q = 1.5 2^(23+E-L-8q) of the four cuts
    uint64_t cut2[kSlices] = {0, 0, 0, 0};
    if (kSliced) {
      const int E = slice_exponent(p.a_amax ? *p.a_amax : 0);
      const int Ld = p.slice_lead ? p.slice_lead : 7;
#pragma unroll
      for (int q = 0; q < kSlices; ++q) cut2[q] = splat_f32x2(ldexpf(1.5f, 23 + E - Ld - 8 * q));
    }
    int f = 0;
    uint32_t fph = 0;
    for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
      const int nkb = tile_kblocks(p, tile);
      for (int kb = 0; kb < nkb; ++kb) {
        float4 *a;
        if (kSliced) {
          // take the MMA stage, start its B load, then wait for the FP32 A tile
          if (!mbar_wait(&empty[s], ph ^ 1u, p.err)) { ok = false; break; }
          if (ct == 0) {
            int bk, brow;
            b_coords(p, tile, kb, bk, brow);
            mbar_arrive_expect_tx(&full[s], kSlices * b_bytes);
            tma_load_3d(stg + (size_t)s * stage_bytes + kSlicedBOff, &tmBhi, &full[s], bk, brow, 0);
          }
          if (!mbar_wait(&ffull[f], fph, p.err)) { ok = false; break; }
          a = reinterpret_cast<float4 *>(fring + (size_t)f * kABytes);
        } else {
          if (!mbar_wait(&full[s], ph, p.err)) { ok = false; break; }
          a = reinterpret_cast<float4 *>(stg + (size_t)s * stage_bytes);
        }
        if (kSliced) {
          uint8_t *sl = stg + (size_t)s * stage_bytes;
#pragma unroll 2
          for (int i = ct; i < (int)(kABytes / 16); i += kConvThreads) {
            // 16-byte chunk i of the 128-byte-swizzled FP32 tile: row r, logical floats k0..k0+3
            const int r = i >> 3, k0 = ((i & 7) ^ (r & 7)) << 2;
            const float4 x = a[i];
            float2 lo2[kSlices], hi2[kSlices];
            slice4x2(make_float2(x.x, x.y), lo2, cut2);
            slice4x2(make_float2(x.z, x.w), hi2, cut2);
            // the same four elements in the 64-byte-swizzled BF16 slice tile
            const uint32_t off = (uint32_t)r * 64u + ((uint32_t)((k0 >> 3) ^ ((r >> 1) & 3)) << 4) + (uint32_t)(k0 & 7) * 2u;
#pragma unroll
            for (int q = 0; q < kSlices; ++q) {
              uint2 v;
              v.x = pack_bf16(lo2[q].x, lo2[q].y);
              v.y = pack_bf16(hi2[q].x, hi2[q].y);
              *reinterpret_cast<uint2 *>(sl + q * kASliceBytes + off) = v;
            }
          }
        } else {
          float4 *lo = reinterpret_cast<float4 *>(stg + (size_t)s * stage_bytes + kABytes);
#pragma unroll 4
          for (int i = ct; i < (int)(kABytes / 16); i += kConvThreads) {
            const float4 x = a[i];
            float4 h, l;
            h.x = to_tf32(x.x); l.x = to_tf32(x.x - h.x);
            h.y = to_tf32(x.y); l.y = to_tf32(x.y - h.y);
            h.z = to_tf32(x.z); l.z = to_tf32(x.z - h.z);
            h.w = to_tf32(x.w); l.w = to_tf32(x.w - h.w);
            a[i] = h;
            lo[i] = l;
          }
        }
        fence_proxy_async_smem();
        mbar_arrive(&conv[s]);
        if (++s == stages) { s = 0; ph ^= 1u; }
        if (kSliced) {
          mbar_arrive(&fempty[f]);   // the FP32 slot may be refilled
          if (++f == nf) { f = 0; fph ^= 1u; }
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int r = threadIdx.x - 32 * kEpiWarp0;       // TMEM lane == tile row
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int acc = 0;
    uint32_t acc_ph = 0;
    const long long NN = N;
    if (p.kb_chunks) {
      // split-K: every K block arrives as its own FP32 tile and is added to a
      // compensated (sum, error) FP32 pair per output (Knuth's TwoSum), which
      // keeps about twice the FP32 precision at FP32 speed
      const int nv = p.n_valid;
      const int ld = nv + 1;  // odd row stride: no shared-memory bank conflicts across rows
      bool ok = true;
      for (int tile = blockIdx.x; tile < p.tiles && ok; tile += gridDim.x) {
        const int nkb = tile_kblocks(p, tile);
        const int u = splitk_plane(tile), split = splitk_split(tile);
        if (r < N)
          for (int col = 0; col < nv; ++col) acc2[r * ld + col] = make_float2(0.f, 0.f);
        const int nchunks = (nkb + p.kb_chunks - 1) / p.kb_chunks;
        for (int ch = 0; ch < nchunks; ++ch) {
          if (!mbar_wait(&tfull[acc], acc_ph, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t tbase = tmem_base + lane_base + (uint32_t)(acc * kAccCols);
          for (int c0 = 0; c0 < p.nout; c0 += 32) {
            float v[32];
            tmem_ld32(tbase + (uint32_t)c0, v);
            if (kSliced) {
              float vl[32];
              tmem_ld32(tbase + d1_off + (uint32_t)c0, vl);
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] += vl[j];
            }
            if (r < N) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                if (c0 + j < nv) {
                  float2 a = acc2[r * ld + c0 + j];
                  const float sum = a.x + v[j];
                  const float bp = sum - a.x;
                  const float err = (a.x - (sum - bp)) + (v[j] - bp);
                  a.x = sum;
                  a.y += err;
                  acc2[r * ld + c0 + j] = a;
                }
              }
            }
          }
          tc_fence_before();
          mbar_arrive(&tempty[acc]);
          if (++acc == nbuf) { acc = 0; acc_ph ^= 1u; }
        }
        if (!ok) break;
        if (r < N)
          for (int col = 0; col < nv; ++col) {
            const float2 a = acc2[r * ld + col];
            p.out64[(((long long)split * 2 + u) * NN + r) * nv + col] = (double)a.x + (double)a.y;
          }
      }
    } else {
    float mx = 0.f;  // largest |stored value| of this thread (sliced form, out_amax)
    for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
      // warp-uniform: the TMEM loads below are .sync.aligned
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull[acc], acc_ph, p.err))) break;
      tc_fence_after();
      if (kSliced && epi_transposed(p))
        epi_store_tile_t(p, tile, r, tmem_base + lane_base + (uint32_t)(acc * kAccCols), d1_off, mx,
                         stg_all + (warp - kEpiWarp0) * (kStgCols * kStgPitch));
      else
        epi_store_tile<kSliced>(p, tile, r, tmem_base + lane_base + (uint32_t)(acc * kAccCols), d1_off, mx);
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      if (++acc == nbuf) { acc = 0; acc_ph ^= 1u; }
    }
    if (kSliced && p.out_amax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) atomicMax(p.out_amax, __float_as_int(mx));
    }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * kAccCols);
  }
}

}  // namespace tc
}  // namespace g1g2
