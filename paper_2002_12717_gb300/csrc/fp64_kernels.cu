// Plain FP64 kernels of libg1g2: the reference form of every contraction
// (CUDA-core DFMA), the Hartree-Fock build, the G1 right-hand side, the G2
// assembly with the fused RK4 update, and the FP64 observables.
#include "g1g2_internal.h"

#include <algorithm>

namespace g1g2 {

namespace {

__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx c) {
  return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.x, -a.y}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return {a.x * s, a.y * s}; }
// -i * z
__device__ __forceinline__ cplx mul_minus_i(cplx z) { return {z.y, -z.x}; }

// ---------------------------------------------------------------------------
// Strided batched complex GEMM (FP64 CUDA cores).
// Tile 32x32x16, 64 threads, each thread a 4x4 micro-tile strided by 8.
// ---------------------------------------------------------------------------
constexpr int GBM = 32, GBN = 32, GBK = 16, GTM = 4, GTN = 4;
constexpr int GNT = (GBM / GTM) * (GBN / GTN);  // 64

struct ZGemmDev {
  int M, N, K, batch;
  const cplx *A; long long sa_b, sa_m, sa_k;
  const cplx *B; long long sb_b, sb_k, sb_n;
  cplx *C; long long sc_b, sc_m, sc_n;
  cplx alpha; double beta;
  int conjA, conjB;
};

// Micro-tile product over kcount k-steps of the staged tiles: rows ty + 8 i (i < TI),
// columns tx + 8 j (j < TJ).  TI, TJ < 4 serve tiles whose valid extent is at most 8
// rows or columns, and kcount < GBK a ragged K tile, so that padding costs no DFMA
// (the FP64 pipe is the bound of this kernel).
template <int TI, int TJ, bool kFullK>
__device__ __forceinline__ void tile_fma(const cplx (*As)[GBM + 1], const cplx (*Bs)[GBN + 1], int ty, int tx,
                                         int kcount, cplx (&acc)[GTM][GTN]) {
  const int kn = kFullK ? GBK : kcount;
#pragma unroll 4
  for (int kk = 0; kk < kn; ++kk) {
    cplx a[TI], bb[TJ];
#pragma unroll
    for (int i = 0; i < TI; ++i) a[i] = As[kk][ty + i * (GBM / GTM)];
#pragma unroll
    for (int j = 0; j < TJ; ++j) bb[j] = Bs[kk][tx + j * (GBN / GTN)];
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
      for (int j = 0; j < TJ; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
  }
}

// reduce != 0: split-K form.  The reduction runs over (batch, K); it is cut
// into batch * kparts units (unit u: batch u / kparts, K range
// [(u % kparts) * klen, ...)), and split z sums units [z * per_split, ...)
// into partial[z].
// TI, TJ: micro-tile rows and columns computed per thread (GTM, GTN for operands wider
// than 8 in M and N; 1 where that extent is at most 8, chosen by the host per GEMM).
template <int TI, int TJ>
__global__ void __launch_bounds__(GNT) zgemm_kernel(ZGemmDev g, int reduce, int per_split, cplx *partial, int kparts,
                                                     int klen) {
  __shared__ cplx As[GBK][GBM + 1];
  __shared__ cplx Bs[GBK][GBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (GBN / GTN), ty = tid / (GBN / GTN);
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;

  long long b_begin, b_end, b_step;
  if (reduce) {
    b_begin = (long long)blockIdx.z * per_split;
    b_end = min((long long)g.batch * kparts, b_begin + per_split);
    b_step = 1;
  } else {
    b_begin = blockIdx.z;
    b_end = g.batch;
    b_step = gridDim.z;
  }
  for (long long b0 = b_begin; b0 < b_end; b0 += (reduce ? (b_end - b_begin) : b_step)) {
    cplx acc[GTM][GTN];
#pragma unroll
    for (int i = 0; i < GTM; ++i)
#pragma unroll
      for (int j = 0; j < GTN; ++j) acc[i][j] = {0.0, 0.0};
    const long long bl = reduce ? b_end : b0 + 1;
    for (long long u = b0; u < bl; ++u) {
      const long long b = reduce ? u / kparts : u;
      const int kbeg = reduce ? (int)(u % kparts) * klen : 0;
      const int kend = reduce ? min(g.K, kbeg + klen) : g.K;
      const cplx *A = g.A + b * g.sa_b;
      const cplx *B = g.B + b * g.sb_b;
      for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        for (int idx = tid; idx < GBM * GBK; idx += GNT) {
          int m, k;
          if (g.sa_k == 1) { m = idx / GBK; k = idx % GBK; } else { k = idx / GBM; m = idx % GBM; }
          cplx v = {0.0, 0.0};
          if (m0 + m < g.M && k0 + k < kend) v = A[(long long)(m0 + m) * g.sa_m + (long long)(k0 + k) * g.sa_k];
          if (g.conjA) v.y = -v.y;
          As[k][m] = v;
        }
        for (int idx = tid; idx < GBN * GBK; idx += GNT) {
          int n, k;
          if (g.sb_n == 1) { k = idx / GBN; n = idx % GBN; } else { n = idx / GBK; k = idx % GBK; }
          cplx v = {0.0, 0.0};
          if (n0 + n < g.N && k0 + k < kend) v = B[(long long)(k0 + k) * g.sb_k + (long long)(n0 + n) * g.sb_n];
          if (g.conjB) v.y = -v.y;
          Bs[k][n] = v;
        }
        __syncthreads();
        // the full micro-tile runs the whole (zero-padded) K tile: a runtime trip count
        // there costs registers, and wide GEMMs have few ragged K tiles
        if (TI == GTM && TJ == GTN) tile_fma<TI, TJ, true>(As, Bs, ty, tx, GBK, acc);
        else tile_fma<TI, TJ, false>(As, Bs, ty, tx, min(GBK, kend - k0), acc);
        __syncthreads();
      }
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < GTM; ++i) {
      const int m = m0 + ty + i * (GBM / GTM);
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < GTN; ++j) {
        const int n = n0 + tx + j * (GBN / GTN);
        if (n >= g.N) continue;
        if (reduce) {
          partial[((long long)blockIdx.z * g.M + m) * g.N + n] = acc[i][j];
        } else {
          cplx *c = g.C + b0 * g.sc_b + (long long)m * g.sc_m + (long long)n * g.sc_n;
          cplx r = cmul(g.alpha, acc[i][j]);
          if (g.beta != 0.0) r = cadd(r, cscale(*c, g.beta));
          *c = r;
        }
      }
    }
    if (reduce) break;
  }
}

// Block (32, 32): x = one of 32 consecutive outputs, y = a strided subset of the splits.
__global__ void __launch_bounds__(1024) zgemm_reduce_kernel(ZGemmDev g, int splits, const cplx *partial) {
  __shared__ cplx part[32][33];
  const long long mn = (long long)g.M * g.N;
  const long long idx = (long long)blockIdx.x * 32 + threadIdx.x;
  cplx s = {0.0, 0.0};
  if (idx < mn)
    for (int z = threadIdx.y; z < splits; z += 32) s = cadd(s, partial[(long long)z * mn + idx]);
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y != 0 || idx >= mn) return;
  s = {0.0, 0.0};
  for (int y = 0; y < 32; ++y) s = cadd(s, part[y][threadIdx.x]);
  const int m = (int)(idx / g.N), n = (int)(idx % g.N);
  cplx *c = g.C + (long long)m * g.sc_m + (long long)n * g.sc_n;
  cplx r = cmul(g.alpha, s);
  if (g.beta != 0.0) r = cadd(r, cscale(*c, g.beta));
  *c = r;
}

ZGemmDev to_dev(const ZGemm &g) {
  ZGemmDev d;
  d.M = g.M; d.N = g.N; d.K = g.K; d.batch = g.batch;
  d.A = g.A; d.sa_b = g.sa_b; d.sa_m = g.sa_m; d.sa_k = g.sa_k;
  d.B = g.B; d.sb_b = g.sb_b; d.sb_k = g.sb_k; d.sb_n = g.sb_n;
  d.C = g.C; d.sc_b = g.sc_b; d.sc_m = g.sc_m; d.sc_n = g.sc_n;
  d.alpha = g.alpha; d.beta = g.beta;
  d.conjA = g.conjA; d.conjB = g.conjB;
  return d;
}

// ---------------------------------------------------------------------------
// 4-index permutation, tiled over the innermost input and output axes.
// ---------------------------------------------------------------------------
constexpr int PT = 32;

__global__ void permute4_kernel(int nb, const cplx *__restrict__ in, cplx *__restrict__ out, int p0, int p1,
                                int p2, int p3, cplx alpha, double beta, int conj) {
  // out axis 3 is innermost in memory; input innermost axis is out-axis p3.
  __shared__ cplx tile[PT][PT + 1];
  const int ntile = (nb + PT - 1) / PT;
  const int tA = blockIdx.x % ntile;   // tile along out axis 3
  const int tB = blockIdx.x / ntile;   // tile along out axis p3 (when p3 != 3)
  // the two remaining out axes
  int rest[2], r = 0;
  for (int d = 0; d < 3; ++d)
    if (d != p3) rest[r++] = d;
  // when p3 == 3 the tiles run over out axis 3 only and 'rest' holds axes 0..2 minus p3 -> handle below
  const long long nb2 = (long long)nb * nb;
  const int pidx[4] = {p0, p1, p2, p3};
  if (p3 == 3) {
    // both innermost: plain gather with a 2D grid: blockIdx.y = (a0, a1), x-tiles over (a2, a3)
    const long long a01 = blockIdx.y;
    const int a0 = (int)(a01 / nb), a1 = (int)(a01 % nb);
    for (int e = threadIdx.y * blockDim.x + threadIdx.x; e < nb * nb; e += blockDim.x * blockDim.y) {
      const int a2 = e / nb, a3 = e % nb;
      const int a[4] = {a0, a1, a2, a3};
      const long long src = (((long long)a[pidx[0]] * nb + a[pidx[1]]) * nb + a[pidx[2]]) * nb + a[pidx[3]];
      const long long dst = (((long long)a0 * nb + a1) * nb + a2) * nb + a3;
      cplx v = in[src];
      if (conj) v.y = -v.y;
      cplx res = cmul(alpha, v);
      if (beta != 0.0) res = cadd(res, cscale(out[dst], beta));
      out[dst] = res;
    }
    return;
  }
  const long long ab = blockIdx.y;   // the two remaining out axes, flattened
  int a[4];
  a[rest[0]] = (int)(ab / nb);
  a[rest[1]] = (int)(ab % nb);
  // load: threadIdx.x runs over out axis p3 (input-contiguous), threadIdx.y over out axis 3
  for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
    const int x3 = tA * PT + yy;
    const int xp = tB * PT + threadIdx.x;
    if (x3 < nb && xp < nb) {
      a[3] = x3;
      a[p3] = xp;
      const long long src = (((long long)a[pidx[0]] * nb + a[pidx[1]]) * nb + a[pidx[2]]) * nb + a[pidx[3]];
      tile[yy][threadIdx.x] = in[src];
    }
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
    const int xp = tB * PT + yy;
    const int x3 = tA * PT + threadIdx.x;
    if (x3 < nb && xp < nb) {
      int b[4] = {a[0], a[1], a[2], a[3]};
      b[3] = x3;
      b[p3] = xp;
      const long long dst = (((long long)b[0] * nb + b[1]) * nb + b[2]) * nb + b[3];
      cplx v = tile[threadIdx.x][yy];
      if (conj) v.y = -v.y;
      cplx res = cmul(alpha, v);
      if (beta != 0.0) res = cadd(res, cscale(out[dst], beta));
      out[dst] = res;
    }
  }
  (void)nb2;
}

// ---------------------------------------------------------------------------
// Hartree-Fock build: one warp per (i, j).
// ---------------------------------------------------------------------------
template <bool REAL>
__global__ void hf_build_kernel(int nb, const void *__restrict__ Wm_, const cplx *__restrict__ h,
                                const cplx *__restrict__ D, double f, const cplx *__restrict__ n,
                                cplx *__restrict__ hhf) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nb2 = nb * nb;
  if (warp >= nb2) return;
  // the row of Wm streams from HBM: four independent loads per lane in flight
  cplx acc = {0.0, 0.0}, acc2 = {0.0, 0.0};
  int c = lane;
  if (REAL) {
    const double *Wm = static_cast<const double *>(Wm_) + (long long)warp * nb2;
    for (; c + 96 < nb2; c += 128) {
      const double w0 = Wm[c], w1 = Wm[c + 32], w2 = Wm[c + 64], w3 = Wm[c + 96];
      const cplx n0 = n[c], n1 = n[c + 32], n2 = n[c + 64], n3 = n[c + 96];
      acc.x = fma(w0, n0.x, acc.x);
      acc.y = fma(w0, n0.y, acc.y);
      acc2.x = fma(w1, n1.x, acc2.x);
      acc2.y = fma(w1, n1.y, acc2.y);
      acc.x = fma(w2, n2.x, acc.x);
      acc.y = fma(w2, n2.y, acc.y);
      acc2.x = fma(w3, n3.x, acc2.x);
      acc2.y = fma(w3, n3.y, acc2.y);
    }
    for (; c < nb2; c += 32) {
      const double wv = Wm[c];
      acc.x = fma(wv, n[c].x, acc.x);
      acc.y = fma(wv, n[c].y, acc.y);
    }
  } else {
    const cplx *Wm = static_cast<const cplx *>(Wm_) + (long long)warp * nb2;
    for (; c + 96 < nb2; c += 128) {
      const cplx w0 = Wm[c], w1 = Wm[c + 32], w2 = Wm[c + 64], w3 = Wm[c + 96];
      acc = cfma(w0, n[c], acc);
      acc2 = cfma(w1, n[c + 32], acc2);
      acc = cfma(w2, n[c + 64], acc);
      acc2 = cfma(w3, n[c + 96], acc2);
    }
    for (; c < nb2; c += 32) acc = cfma(Wm[c], n[c], acc);
  }
  acc = cadd(acc, acc2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) {
    cplx r = cadd(h[warp], acc);
    if (D) r = cadd(r, cscale(D[warp], f));
    hhf[warp] = r;
  }
}

// ---------------------------------------------------------------------------
// Hartree-Fock build in double-single arithmetic (the tensor-core forms).
//
// The same matrix-vector product as hf_build_kernel with every FP64 number x held
// as a pair of FP32 numbers x = x_hi + x_lo (x_hi = fl32(x), x_lo = fl32(x - x_hi)),
// evaluated on the FP32 pipe: GB300 issues FP64 instructions at a small fraction of
// its FP32 rate, and in FP64 this product takes longer than streaming Wm from HBM.
// Per term w n = w_hi n_hi + (w_hi n_lo + w_lo n_hi) + w_lo n_lo: the first product
// exactly (TwoProd with a fused multiply-add), the cross terms in FP32, the last one
// dropped (2^-48 relative); the sum in a (S, C) pair, S updated by the error-free
// TwoSum of Knuth (TAOCP vol. 2, 4.2.2) and C collecting the rounding errors.  The
// result carries about 46 bits: the tensor-core forms evaluate G2's terms to
// about 2^-24, so the mean field stays far more accurate than the rest of the step.
// Intrinsics keep the compiler from contracting the error terms into other FMAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ds_add(float &S, float &C, float p) {
  const float s = __fadd_rn(S, p);
  const float bp = __fsub_rn(s, S);
  C = __fadd_rn(C, __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp)));
  S = s;
}

// (S, C) += (wh + wl)(nh + nl)
__device__ __forceinline__ void ds_mac(float &S, float &C, float wh, float wl, float nh, float nl) {
  const float p = __fmul_rn(wh, nh);
  const float e = __fmaf_rn(wh, nh, -p);
  const float cross = __fmaf_rn(wh, nl, __fmul_rn(wl, nh));
  ds_add(S, C, p);
  C = __fadd_rn(C, __fadd_rn(e, cross));
}

// ns[c] = (Re n_hi, Im n_hi, Re n_lo, Im n_lo)
__global__ void n_split_kernel(int nb2, const cplx *__restrict__ n, float4 *__restrict__ ns) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb2) return;
  const cplx v = n[c];
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  ns[c] = make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
}

constexpr int kHfRows = 4;   // rows of Wm per CTA: each n load serves four rows

// Wds: the real Wm as float2 (hi, lo) per entry (the tensor-core forms take a real w).
// One CTA of 256 threads per kHfRows rows: thread t takes entries c = t, t + 256, ... of
// each row, four of them per iteration with all sixteen row loads and four n loads
// issued before the arithmetic (the product is bound by the bytes in flight); the partial
// pairs are reduced over the warp and the CTA in a fixed order.
__global__ void __launch_bounds__(256) hf_build_ds_kernel(int nb, const float2 *__restrict__ Wds,
                                                           const float4 *__restrict__ ns,
                                                           const cplx *__restrict__ h, const cplx *__restrict__ D,
                                                           double f, cplx *__restrict__ hhf) {
  __shared__ float4 red[8][kHfRows];   // per warp and row: (S_re, C_re, S_im, C_im)
  const int nb2 = nb * nb;
  const int row0 = blockIdx.x * kHfRows;
  const int nrow = min(kHfRows, nb2 - row0);
  float Sr[kHfRows], Cr[kHfRows], Si[kHfRows], Ci[kHfRows];
#pragma unroll
  for (int r = 0; r < kHfRows; ++r) Sr[r] = Cr[r] = Si[r] = Ci[r] = 0.f;
  // rows past the end (a ragged last CTA) repeat the last row and are not stored, so the
  // loads carry no branch
  const float2 *wbase = Wds + (long long)row0 * nb2;
  int woff[kHfRows];
#pragma unroll
  for (int r = 0; r < kHfRows; ++r) woff[r] = (min(row0 + r, nb2 - 1) - row0) * nb2;
  int c = threadIdx.x;
  for (; c + 768 < nb2; c += 1024) {
    float4 nv[4];
    float2 w[4][kHfRows];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      nv[u] = ns[c + 256 * u];
#pragma unroll
      for (int r = 0; r < kHfRows; ++r) w[u][r] = wbase[woff[r] + c + 256 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int r = 0; r < kHfRows; ++r) {
        ds_mac(Sr[r], Cr[r], w[u][r].x, w[u][r].y, nv[u].x, nv[u].z);
        ds_mac(Si[r], Ci[r], w[u][r].x, w[u][r].y, nv[u].y, nv[u].w);
      }
  }
  for (; c < nb2; c += 256) {
    const float4 nv = ns[c];
    float2 w[kHfRows];
#pragma unroll
    for (int r = 0; r < kHfRows; ++r) w[r] = wbase[woff[r] + c];
#pragma unroll
    for (int r = 0; r < kHfRows; ++r) {
      ds_mac(Sr[r], Cr[r], w[r].x, w[r].y, nv.x, nv.z);
      ds_mac(Si[r], Ci[r], w[r].x, w[r].y, nv.y, nv.w);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kHfRows; ++r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float sr = __shfl_xor_sync(0xffffffffu, Sr[r], o), cr = __shfl_xor_sync(0xffffffffu, Cr[r], o);
      const float si = __shfl_xor_sync(0xffffffffu, Si[r], o), ci = __shfl_xor_sync(0xffffffffu, Ci[r], o);
      ds_add(Sr[r], Cr[r], sr);
      Cr[r] = __fadd_rn(Cr[r], cr);
      ds_add(Si[r], Ci[r], si);
      Ci[r] = __fadd_rn(Ci[r], ci);
    }
    if (lane == 0) red[warp][r] = make_float4(Sr[r], Cr[r], Si[r], Ci[r]);
  }
  __syncthreads();
  if (threadIdx.x < nrow) {
    const int r = threadIdx.x, row = row0 + r;
    cplx acc = {0.0, 0.0};
    for (int w = 0; w < 8; ++w) {
      const float4 v = red[w][r];
      acc.x += (double)v.x + (double)v.y;
      acc.y += (double)v.z + (double)v.w;
    }
    cplx out = cadd(h[row], acc);
    if (D) out = cadd(out, cscale(D[row], f));
    hhf[row] = out;
  }
}

__global__ void one_pm_kernel(int nb, const cplx *n, double eta, cplx *nbar) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * nb) return;
  const int i = idx / nb, j = idx % nb;
  cplx v = n[idx];
  nbar[idx] = {(i == j ? 1.0 : 0.0) + eta * v.x, eta * v.y};
}

// RK4 bookkeeping for one element with derivative k.
__device__ __forceinline__ void rk4_apply(long long e, cplx k, int stage, double dt, cplx *y, cplx *ys, cplx *acc,
                                          cplx *kout) {
  if (stage < 0) {
    kout[e] = k;
    return;
  }
  const cplx y0 = y[e];
  if (stage == 0) {
    acc[e] = k;
    ys[e] = {fma(0.5 * dt, k.x, y0.x), fma(0.5 * dt, k.y, y0.y)};
  } else if (stage == 1) {
    const cplx a = acc[e];
    acc[e] = {fma(2.0, k.x, a.x), fma(2.0, k.y, a.y)};
    ys[e] = {fma(0.5 * dt, k.x, y0.x), fma(0.5 * dt, k.y, y0.y)};
  } else if (stage == 2) {
    const cplx a = acc[e];
    acc[e] = {fma(2.0, k.x, a.x), fma(2.0, k.y, a.y)};
    ys[e] = {fma(dt, k.x, y0.x), fma(dt, k.y, y0.y)};
  } else {
    const cplx a = acc[e];
    y[e] = {fma(dt / 6.0, a.x + k.x, y0.x), fma(dt / 6.0, a.y + k.y, y0.y)};
  }
}

// dn = -i[hHF, n] - (I + I^dag): one thread per element, explicit sums over p.
// dn/dt = -i [hHF, n] - (I + I^dag) (Eqs. eom_gone-2, eom_gone-I) and its RK4 stage update:
// one warp per element (i, j), the lanes splitting the sum over p and reducing in a fixed
// order, so that the nb^3 FP64 multiply-adds spread over every SM.
__global__ void __launch_bounds__(256) g1_update_kernel(int nb, const cplx *__restrict__ hhf,
                                                        const cplx *__restrict__ n, const cplx *__restrict__ I,
                                                        int stage, double dt, cplx *y, cplx *ys, cplx *acc,
                                                        cplx *kout) {
  const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= nb * nb) return;
  const int i = idx / nb, j = idx % nb;
  cplx comm = {0.0, 0.0};
  for (int p = lane; p < nb; p += 32) {
    comm = cfma(hhf[i * nb + p], n[p * nb + j], comm);
    comm = csub(comm, cmul(n[i * nb + p], hhf[p * nb + j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    comm.x += __shfl_xor_sync(0xffffffffu, comm.x, o);
    comm.y += __shfl_xor_sync(0xffffffffu, comm.y, o);
  }
  if (lane != 0) return;
  cplx k = mul_minus_i(comm);
  if (I) {
    const cplx a = I[i * nb + j];
    const cplx b = cconj(I[j * nb + i]);
    k = csub(k, cadd(a, b));
  }
  rk4_apply(idx, k, stage, dt, y, ys, acc, kout);
}

// dG = -i (Cb - Ab + conj(Ab^T)): 32x32 tiles of the (ij),(kl) matrix view.
__global__ void g2_assemble_kernel(int nb, const cplx *__restrict__ Cb, const cplx *__restrict__ Ab, int stage,
                                   double dt, cplx *y, cplx *ys, cplx *acc, cplx *kout) {
  __shared__ cplx tile[PT][PT + 1];
  const long long M = (long long)nb * nb;
  const long long r0 = (long long)blockIdx.y * PT, c0 = (long long)blockIdx.x * PT;
  // load the transposed tile Ab[(c0..), (r0..)] (no Ab: dG = -i Cb)
  if (Ab)
    for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
      const long long rr = c0 + yy, cc = r0 + threadIdx.x;
      if (rr < M && cc < M) tile[yy][threadIdx.x] = Ab[rr * M + cc];
    }
  __syncthreads();
  for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
    const long long r = r0 + yy, c = c0 + threadIdx.x;
    if (r < M && c < M) {
      const long long e = r * M + c;
      const cplx v = Ab ? cadd(csub(Cb[e], Ab[e]), cconj(tile[threadIdx.x][yy])) : Cb[e];
      rk4_apply(e, mul_minus_i(v), stage, dt, y, ys, acc, kout);
    }
  }
}

// ---------------------------------------------------------------------------
// Hubbard basis, spin-restricted SOA: the O(nb^4) forms of the G2 right-hand
// side.  With an on-site interaction w_ijkl = U_i d(i=j=k=l):
//   * the commutator [h2, G] only needs the nonzeros of h^HF (h plus the
//     diagonal Hartree term), a stencil over the sparsity pattern (CSR);
//   * in the source term, writing G^> = G^< - i 1 cancels the products of
//     four G^< (the reformulation of Sec. VI for the Hubbard basis) and
//     leaves six terms, each with one or two Kronecker deltas; with
//     G^< = i n they read Psi = -S,
//       S_ijkl = - U_j n_ij n_jk n_jl - U_i n_ji n_ik n_il + d_ij U_i n_ik n_il
//                + U_l n_il n_jl n_lk + U_k n_ik n_jk n_kl - d_kl U_k n_ik n_jk;
//   * the collision integral is I_ij = -i U_i G_iiji.
// ---------------------------------------------------------------------------
// With Go (GW, the other spin block of G2: same-spin for the opposite-spin equation and
// vice versa) the polarisation term is added, Pi_ijkl - conj(Pi_lkji) with
// Pi_ijkl = n_jl (U_j Go_ijkj - U_l Go_ilkl): the Hubbard-basis reduction of Eqs.
// (pihubbardtrans, pihubbardcis) with G^> = G^< - i and G^< = i n (U_p inside the sum
// over the site p).  psi = 0 leaves out the source term (the same-spin equation, whose
// source vanishes for an on-site interaction).
__global__ void hubbard_c_kernel(int nb, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const cplx *__restrict__ hhf, const double *__restrict__ U,
                                 const cplx *__restrict__ n, const cplx *__restrict__ G,
                                 const cplx *__restrict__ Go, int psi, cplx *C) {
  // grid: y = i nb + j, x over (k, l); index arithmetic in 32 bits where it fits
  const long long N = nb, N2 = N * N, N3 = N2 * N;
  const int ij = blockIdx.y, i = ij / nb, j = ij - i * nb;
  const int kl = blockIdx.x * blockDim.x + threadIdx.x;
  if (kl < nb * nb) {
    const int k = kl / nb, l = kl - k * nb;
    const long long e = (long long)ij * N2 + kl;
    cplx acc = {0.0, 0.0};
    // [h2, G]_ijkl = sum_p h_ip G_pjkl + h_jp G_ipkl - G_ijpl h_pk - G_ijkp h_pl
    for (int q = rp[i]; q < rp[i + 1]; ++q) {
      const int p = ci[q];
      acc = cfma(hhf[i * N + p], G[p * N3 + j * N2 + kl], acc);
    }
    for (int q = rp[j]; q < rp[j + 1]; ++q) {
      const int p = ci[q];
      acc = cfma(hhf[j * N + p], G[i * N3 + p * N2 + k * N + l], acc);
    }
    for (int q = rp[k]; q < rp[k + 1]; ++q) {
      const int p = ci[q];
      acc = csub(acc, cmul(G[i * N3 + j * N2 + p * N + l], hhf[p * N + k]));
    }
    for (int q = rp[l]; q < rp[l + 1]; ++q) {
      const int p = ci[q];
      acc = csub(acc, cmul(G[e - l + p], hhf[p * N + l]));
    }
    if (psi) {
      // Psi = -S
      const cplx nij = n[i * N + j], nji = n[j * N + i], nik = n[i * N + k], nil = n[i * N + l];
      const cplx njk = n[j * N + k], njl = n[j * N + l], nlk = n[l * N + k], nkl = n[k * N + l];
      cplx S = cscale(cmul(cmul(nij, njk), njl), -U[j]);
      S = cadd(S, cscale(cmul(cmul(nji, nik), nil), -U[i]));
      S = cadd(S, cscale(cmul(cmul(nil, njl), nlk), U[l]));
      S = cadd(S, cscale(cmul(cmul(nik, njk), nkl), U[k]));
      if (i == j) S = cadd(S, cscale(cmul(nik, nil), U[i]));
      if (k == l) S = csub(S, cscale(cmul(nik, njk), U[k]));
      acc = csub(acc, S);
    }
    if (Go) {
      auto g4 = [&](int a, int b, int c, int d) { return Go[((a * N + b) * N + c) * N + d]; };
      const cplx pi = cmul(n[j * N + l], csub(cscale(g4(i, j, k, j), U[j]), cscale(g4(i, l, k, l), U[l])));
      const cplx pt = cmul(n[k * N + i], csub(cscale(g4(l, k, j, k), U[k]), cscale(g4(l, i, j, i), U[i])));
      acc = csub(cadd(acc, pi), cconj(pt));   // + Pi_ijkl - conj(Pi_lkji)
    }
    C[e] = acc;
  }
}

__global__ void hubbard_collision_kernel(int nb, const double *__restrict__ U, const cplx *__restrict__ G, cplx *I) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb * nb) return;
  const long long N = nb;
  const int i = e / nb, j = e % nb;
  const cplx g = G[((i * N + i) * N + j) * N + i];  // G_iiji
  I[e] = cscale(mul_minus_i(g), U[i]);
}

// ---------------------------------------------------------------------------
// Observables
// ---------------------------------------------------------------------------
__global__ void obs_one_body_kernel(int nb, const cplx *h, const cplx *D, double f, const cplx *hhf, const cplx *n,
                                    double *red) {
  // single block
  __shared__ double s[4][256];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx % nb;
    const cplx nji = n[j * nb + i];
    cplx hij = h[idx];
    if (D) hij = cadd(hij, cscale(D[idx], f));
    a0 += hij.x * nji.x - hij.y * nji.y;
    const cplx dh = csub(hhf[idx], hij);
    a1 += dh.x * nji.x - dh.y * nji.y;
    if (i == j) a2 += nji.x;
    if (D) a3 += D[idx].x * nji.x - D[idx].y * nji.y;
  }
  s[0][threadIdx.x] = a0; s[1][threadIdx.x] = a1; s[2][threadIdx.x] = a2; s[3][threadIdx.x] = a3;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) red[threadIdx.x] = s[threadIdx.x][0];
}

// per-block partial sums of Re W[(ij),(kl)] G[(kl),(ij)] and of the non-finite count: each
// CTA walks the 32 x 32 tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... of the (ij),(kl)
// matrix view (G's tile read transposed through shared memory) and reduces once at the end
__global__ void __launch_bounds__(PT * 8) obs_two_body_kernel(int nb, const cplx *__restrict__ W,
                                                              const cplx *__restrict__ G, double *partials) {
  __shared__ cplx tile[PT][PT + 1];
  __shared__ double s0[8], s1[8];
  const long long M = (long long)nb * nb;
  const long long nt = (M + PT - 1) / PT;
  double acc = 0.0, bad = 0.0;
  for (long long t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const long long r0 = (t / nt) * PT, c0 = (t % nt) * PT;
    __syncthreads();   // the previous tile has been read
    for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
      const long long rr = c0 + yy, cc = r0 + threadIdx.x;
      if (rr < M && cc < M) tile[yy][threadIdx.x] = G[rr * M + cc];
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
      const long long r = r0 + yy, c = c0 + threadIdx.x;
      if (r < M && c < M) {
        const cplx w = W[r * M + c];
        const cplx g = tile[threadIdx.x][yy];   // G[(c),(r)]
        acc += w.x * g.x - w.y * g.y;
        // every element of G lands in exactly one transposed tile: count the non-finite ones there
        if (!isfinite(g.x) || !isfinite(g.y)) bad += 1.0;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (threadIdx.x == 0) {
    s0[threadIdx.y] = acc;
    s1[threadIdx.y] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += s0[w];
      b += s1[w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void sum_pairs_kernel(const double *partials, long long nblk, double *red) {
  __shared__ double s0[256], s1[256];
  double a = 0, b = 0;
  for (long long i = threadIdx.x; i < nblk; i += blockDim.x) { a += partials[2 * i]; b += partials[2 * i + 1]; }
  s0[threadIdx.x] = a; s1[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { red[0] = s0[0]; red[1] = s1[0]; }
}

// W += coeff Re sum_ij D_ij n_ji: one CTA of 1024 threads, reduced over the warps in a
// fixed order (deterministic, no atomics)
__global__ void __launch_bounds__(1024) accumulate_work_kernel(int nb, const cplx *D, const cplx *n, double coeff,
                                                               double *W) {
  __shared__ double s[32];
  double a = 0;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx % nb;
    const cplx nji = n[j * nb + i];
    a += D[idx].x * nji.x - D[idx].y * nji.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    *W += coeff * t;
  }
}

__global__ void double_occ_kernel(int nb, const cplx *n, const cplx *G, double eta, double *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb / 2) return;
  const int u = 2 * s, d = 2 * s + 1;
  const long long nb_ = nb;
  const cplx nuu = n[u * nb + u], ndd = n[d * nb + d], nud = n[u * nb + d], ndu = n[d * nb + u];
  const cplx g = G[((u * nb_ + d) * nb_ + u) * nb_ + d];
  const cplx prod = cadd(cmul(nuu, ndd), cscale(cmul(nud, ndu), eta));   // Eq. (ini-g2): the exchange term takes the ±
  out[s] = prod.x - g.x;
}

__global__ void count_nonfinite_kernel(const cplx *x, long long len, double *cnt) {
  __shared__ double s[256];
  double a = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i].x) || !isfinite(x[i].y)) a += 1.0;
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && s[0] != 0.0) atomicAdd(cnt, s[0]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Rows (columns) beyond 8 of a tile exist only when M (N) exceeds 8; narrower GEMMs
// run the 1-row (1-column) micro-tile so that no DFMA is spent on padding.
void launch_zgemm(dim3 grid, cudaStream_t st, const ZGemm &g, int reduce, int per, cplx *partial, int kparts,
                  int klen) {
  const bool mw = g.M > GBM / GTM, nw = g.N > GBN / GTN;
  if (mw && nw) zgemm_kernel<GTM, GTN><<<grid, GNT, 0, st>>>(to_dev(g), reduce, per, partial, kparts, klen);
  else if (mw) zgemm_kernel<GTM, 1><<<grid, GNT, 0, st>>>(to_dev(g), reduce, per, partial, kparts, klen);
  else if (nw) zgemm_kernel<1, GTN><<<grid, GNT, 0, st>>>(to_dev(g), reduce, per, partial, kparts, klen);
  else zgemm_kernel<1, 1><<<grid, GNT, 0, st>>>(to_dev(g), reduce, per, partial, kparts, klen);
}

void zgemm(Launcher &L, const ZGemm &g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, std::min(g.batch, 65535));
  L.before("fp64_zgemm");
  launch_zgemm(grid, L.stream, g, 0, 1, nullptr, 1, g.K);
  L.after_launch();
}

void zgemm_reduce(Launcher &L, const ZGemm &g, cplx *partial, int splits) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  // cut K as well when the batch alone gives fewer units than splits
  const int kblocks = (g.K + GBK - 1) / GBK;
  const int kparts = std::max(1, std::min(kblocks, (splits + g.batch - 1) / g.batch));
  const int klen = ((kblocks + kparts - 1) / kparts) * GBK;
  const long long units = (long long)g.batch * kparts;
  splits = (int)std::max(1LL, std::min((long long)splits, units));
  const int per = (int)((units + splits - 1) / splits);
  splits = (int)((units + per - 1) / per);
  dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, splits);
  L.before("fp64_zgemm_splitk");
  launch_zgemm(grid, L.stream, g, 1, per, partial, kparts, klen);
  L.after_launch();
  const long long mn = (long long)g.M * g.N;
  L.before("fp64_splitk_reduce");
  zgemm_reduce_kernel<<<(unsigned)((mn + 31) / 32), dim3(32, 32), 0, L.stream>>>(to_dev(g), splits, partial);
  L.after_launch();
}

void permute4(Launcher &L, int nb, const cplx *in, cplx *out, const int p[4], cplx alpha, double beta, bool conj) {
  const int nt = (nb + PT - 1) / PT;
  dim3 block(PT, 8);
  L.before("permute4");
  if (p[3] == 3) {
    dim3 grid(1, (unsigned)((long long)nb * nb));
    permute4_kernel<<<grid, block, 0, L.stream>>>(nb, in, out, p[0], p[1], p[2], p[3], alpha, beta, conj);
  } else {
    dim3 grid(nt * nt, (unsigned)((long long)nb * nb));
    permute4_kernel<<<grid, block, 0, L.stream>>>(nb, in, out, p[0], p[1], p[2], p[3], alpha, beta, conj);
  }
  L.after_launch();
}

void hf_build(Launcher &L, int nb, const void *Wm, bool wm_real, const cplx *h, const cplx *D, double f,
              const cplx *n, cplx *hhf) {
  const int warps = nb * nb;
  const int threads = 256;
  const int blocks = (warps * 32 + threads - 1) / threads;
  L.before("hf_build");
  if (wm_real)
    hf_build_kernel<true><<<blocks, threads, 0, L.stream>>>(nb, Wm, h, D, f, n, hhf);
  else
    hf_build_kernel<false><<<blocks, threads, 0, L.stream>>>(nb, Wm, h, D, f, n, hhf);
  L.after_launch();
}

void hf_build_ds(Launcher &L, int nb, const float2 *Wds, const cplx *h, const cplx *D, double f, const cplx *n,
                 float4 *nsplit, cplx *hhf) {
  const int nb2 = nb * nb;
  L.before("hf_split_n");
  n_split_kernel<<<(nb2 + 255) / 256, 256, 0, L.stream>>>(nb2, n, nsplit);
  L.after_launch();
  L.before("hf_build");
  const int blocks = (nb2 + kHfRows - 1) / kHfRows;
  hf_build_ds_kernel<<<blocks, 256, 0, L.stream>>>(nb, Wds, nsplit, h, D, f, hhf);
  L.after_launch();
}

void one_pm(Launcher &L, int nb, const cplx *n, double eta, cplx *nbar) {
  L.before("one_minus");
  one_pm_kernel<<<(nb * nb + 255) / 256, 256, 0, L.stream>>>(nb, n, eta, nbar);
  L.after_launch();
}

void g1_update(Launcher &L, int nb, const cplx *hhf, const cplx *n, const cplx *I, Rk4Stage st, cplx *y, cplx *ys,
               cplx *acc, cplx *kout) {
  L.before("g1_update");
  g1_update_kernel<<<(nb * nb + 7) / 8, 256, 0, L.stream>>>(nb, hhf, n, I, st.stage, st.dt, y, ys, acc, kout);
  L.after_launch();
}

void g2_assemble(Launcher &L, int nb, const cplx *Cb, const cplx *Ab, Rk4Stage st, cplx *y, cplx *ys, cplx *acc,
                 cplx *kout) {
  const long long M = (long long)nb * nb;
  const unsigned t = (unsigned)((M + PT - 1) / PT);
  L.before("fp64_g2_assemble_rk4");
  g2_assemble_kernel<<<dim3(t, t), dim3(PT, 8), 0, L.stream>>>(nb, Cb, Ab, st.stage, st.dt, y, ys, acc, kout);
  L.after_launch();
}

void hubbard_c(Launcher &L, int nb, const int *rp, const int *ci, const cplx *hhf, const double *U, const cplx *n,
               const cplx *G, const cplx *Go, bool psi, cplx *C) {
  L.before("hubbard_c");
  hubbard_c_kernel<<<dim3((nb * nb + 127) / 128, nb * nb), 128, 0, L.stream>>>(nb, rp, ci, hhf, U, n, G, Go, psi ? 1 : 0,
                                                                                C);
  L.after_launch();
}

void hubbard_collision(Launcher &L, int nb, const double *U, const cplx *G, cplx *I) {
  L.before("hubbard_collision");
  hubbard_collision_kernel<<<(nb * nb + 127) / 128, 128, 0, L.stream>>>(nb, U, G, I);
  L.after_launch();
}

void obs_one_body(Launcher &L, int nb, const cplx *h, const cplx *D, double f, const cplx *hhf, const cplx *n,
                  double *red) {
  L.before("obs_one_body");
  obs_one_body_kernel<<<1, 256, 0, L.stream>>>(nb, h, D, f, hhf, n, red);
  L.after_launch();
}

void obs_two_body(Launcher &L, int nb, const cplx *W, const cplx *G, double *partials, double *red) {
  const long long M = (long long)nb * nb;
  const long long t = (M + PT - 1) / PT;
  // eight CTAs of 256 threads per SM, each over several tiles (partials holds t^2 pairs)
  const unsigned blocks = (unsigned)std::min<long long>(t * t, 152 * 8);
  L.before("obs_two_body");
  obs_two_body_kernel<<<blocks, dim3(PT, 8), 0, L.stream>>>(nb, W, G, partials);
  L.after_launch();
  L.before("obs_sum");
  sum_pairs_kernel<<<1, 256, 0, L.stream>>>(partials, (long long)blocks, red);
  L.after_launch();
}

void accumulate_work(Launcher &L, int nb, const cplx *D, const cplx *n, double coeff, double *W_acc) {
  L.before("drive_work");
  accumulate_work_kernel<<<1, 1024, 0, L.stream>>>(nb, D, n, coeff, W_acc);
  L.after_launch();
}

void double_occ(Launcher &L, int nb, const cplx *n, const cplx *G, double eta, double *out) {
  L.before("double_occ");
  double_occ_kernel<<<(nb / 2 + 63) / 64, 64, 0, L.stream>>>(nb, n, G, eta, out);
  L.after_launch();
}

void count_nonfinite(Launcher &L, const cplx *x, long long len, double *cnt) {
  const unsigned blocks = (unsigned)std::min<long long>((len + 255) / 256, 4096);
  L.before("nonfinite_check");
  count_nonfinite_kernel<<<blocks, 256, 0, L.stream>>>(x, len, cnt);
  L.after_launch();
}

}  // namespace g1g2

// ---------------------------------------------------------------------------
// Kernels of the discrete adjoint (FP64)
// ---------------------------------------------------------------------------
namespace g1g2 {
namespace {

__global__ void zaxpby_kernel(long long n, cplx alpha, const cplx *__restrict__ x, cplx beta,
                              const cplx *__restrict__ y, cplx *out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    cplx r = cmul(alpha, x[e]);
    if (y) r = cadd(r, cmul(beta, y[e]));
    out[e] = r;
  }
}

// out = c * (a + a^dag) for an nb x nb matrix
__global__ void herm_sum_kernel(int nb, cplx c, const cplx *__restrict__ a, cplx *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb * nb) return;
  const int i = e / nb, j = e % nb;
  out[e] = cmul(c, cadd(a[e], cconj(a[j * nb + i])));
}

// out = c * (Y + Y^dag), (Y^dag)_ijkl = conj(Y_klij), 32x32 tiles of the (ij),(kl) view
__global__ void tconj_add_kernel(int nb, cplx c, const cplx *__restrict__ Y, cplx *out) {
  __shared__ cplx tile[PT][PT + 1];
  const long long M = (long long)nb * nb;
  const long long r0 = (long long)blockIdx.y * PT, c0 = (long long)blockIdx.x * PT;
  for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
    const long long rr = c0 + yy, cc = r0 + threadIdx.x;
    if (rr < M && cc < M) tile[yy][threadIdx.x] = Y[rr * M + cc];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < PT; yy += blockDim.y) {
    const long long r = r0 + yy, cl = c0 + threadIdx.x;
    if (r < M && cl < M) {
      const long long e = r * M + cl;
      out[e] = cmul(c, cadd(Y[e], cconj(tile[threadIdx.x][yy])));
    }
  }
}

// partial sums of Re sum conj(x) y
__global__ void real_dot_kernel(long long n, const cplx *__restrict__ x, const cplx *__restrict__ y, double *partials) {
  __shared__ double s[256];
  double a = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    a += x[e].x * y[e].x + x[e].y * y[e].y;
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

// acc[slot] += coeff * sum(partials)
__global__ void dot_accumulate_kernel(int nparts, const double *partials, double coeff, double *acc) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += partials[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += coeff * s[0];
}

// out_lk (+)= sum_ij Wm[(ij),(lk)] x_ij  (the adjoint of the Hartree-Fock build)
template <bool REAL>
__global__ void hf_build_t_kernel(int nb, const void *__restrict__ Wm_, const cplx *__restrict__ x, cplx *out,
                                  int accumulate) {
  const int nb2 = nb * nb;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb2) return;
  cplx acc = {0.0, 0.0};
  for (int r = 0; r < nb2; ++r) {
    const cplx xv = x[r];
    if (REAL) {
      const double wv = static_cast<const double *>(Wm_)[(long long)r * nb2 + c];
      acc.x = fma(wv, xv.x, acc.x);
      acc.y = fma(wv, xv.y, acc.y);
    } else {
      acc = cfma(cconj(static_cast<const cplx *>(Wm_)[(long long)r * nb2 + c]), xv, acc);
    }
  }
  // the Hartree-Fock matrix is indexed [(ij),(lk)] with column (l*nb + k) = the n_lk entry
  out[c] = accumulate ? cadd(out[c], acc) : acc;
}

}  // namespace

void zaxpby(Launcher &L, long long n, cplx alpha, const cplx *x, cplx beta, const cplx *y, cplx *out) {
  L.before("adj_axpby");
  zaxpby_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 8192), 256, 0, L.stream>>>(n, alpha, x, beta, y, out);
  L.after_launch();
}

// Cotangent of w from the Hartree-Fock build (Eq. h_HF): with Wm[(ij),(lk)] = w_ikjl + eta
// w_iklj, the cotangent x of h^HF gives Wmbar[(ij),(lk)] = x_ij conj(n_lk), so
// wbar_abcd += c (x_ac conj(n_db) + eta x_ad conj(n_cb)).  One thread per element of w.
__global__ void hf_wbar_kernel(int nb, const cplx *__restrict__ x, const cplx *__restrict__ n, double c, double eta,
                               cplx *wbar) {
  const long long N = nb, N4 = N * N * N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N4; e += (long long)gridDim.x * blockDim.x) {
    const long long d = e % N, cc = (e / N) % N, b = (e / (N * N)) % N, a = e / (N * N * N);
    const cplx x1 = x[a * N + cc], n1 = n[d * N + b];
    double re = x1.x * n1.x + x1.y * n1.y, im = x1.y * n1.x - x1.x * n1.y;   // x1 conj(n1)
    if (eta != 0.0) {
      const cplx x2 = x[a * N + d], n2 = n[cc * N + b];
      re += eta * (x2.x * n2.x + x2.y * n2.y);
      im += eta * (x2.y * n2.x - x2.x * n2.y);
    }
    wbar[e].x += c * re;
    wbar[e].y += c * im;
  }
}

// out = (X + X_jilk + conj(X_klij) + conj(X_lkji)) / 4: the orthogonal projection (for
// Re sum conj(x) y) onto the tensors with the symmetries w_ijkl = w_jilk = conj(w_klij).
__global__ void w_symmetrize_kernel(int nb, const cplx *__restrict__ X, cplx *out) {
  const long long N = nb, N4 = N * N * N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N4; e += (long long)gridDim.x * blockDim.x) {
    const long long l = e % N, k = (e / N) % N, j = (e / (N * N)) % N, i = e / (N * N * N);
    const cplx a = X[e], b = X[((j * N + i) * N + l) * N + k];
    const cplx h = X[((k * N + l) * N + i) * N + j], g = X[((l * N + k) * N + j) * N + i];
    out[e] = make_double2(0.25 * (a.x + b.x + h.x + g.x), 0.25 * (a.y + b.y - h.y - g.y));
  }
}

void hf_wbar(Launcher &L, int nb, const cplx *x, const cplx *n, double c, double eta, cplx *wbar) {
  L.before("adj_hf_wbar");
  hf_wbar_kernel<<<1024, 256, 0, L.stream>>>(nb, x, n, c, eta, wbar);
  L.after_launch();
}

void w_symmetrize(Launcher &L, int nb, const cplx *X, cplx *out) {
  L.before("adj_w_symmetrize");
  w_symmetrize_kernel<<<1024, 256, 0, L.stream>>>(nb, X, out);
  L.after_launch();
}

void herm_sum(Launcher &L, int nb, cplx c, const cplx *a, cplx *out) {
  L.before("adj_herm_sum");
  herm_sum_kernel<<<(nb * nb + 127) / 128, 128, 0, L.stream>>>(nb, c, a, out);
  L.after_launch();
}

void tconj_add(Launcher &L, int nb, cplx c, const cplx *Y, cplx *out) {
  const long long M = (long long)nb * nb;
  const unsigned t = (unsigned)((M + PT - 1) / PT);
  L.before("adj_tconj_add");
  tconj_add_kernel<<<dim3(t, t), dim3(PT, 8), 0, L.stream>>>(nb, c, Y, out);
  L.after_launch();
}

void real_dot_acc(Launcher &L, long long n, const cplx *x, const cplx *y, double coeff, double *partials, double *acc) {
  const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
  L.before("adj_dot");
  real_dot_kernel<<<blocks, 256, 0, L.stream>>>(n, x, y, partials);
  L.after_launch();
  L.before("adj_dot");
  dot_accumulate_kernel<<<1, 256, 0, L.stream>>>(blocks, partials, coeff, acc);
  L.after_launch();
}

void hf_build_t(Launcher &L, int nb, const void *Wm, bool wm_real, const cplx *x, cplx *out, bool accumulate) {
  const int nb2 = nb * nb;
  L.before("adj_hf_build_t");
  if (wm_real)
    hf_build_t_kernel<true><<<(nb2 + 127) / 128, 128, 0, L.stream>>>(nb, Wm, x, out, accumulate ? 1 : 0);
  else
    hf_build_t_kernel<false><<<(nb2 + 127) / 128, 128, 0, L.stream>>>(nb, Wm, x, out, accumulate ? 1 : 0);
  L.after_launch();
}

}  // namespace g1g2

// ---------------------------------------------------------------------------
// Kernels of the memory-integral HF-GKBA (FP64)
// ---------------------------------------------------------------------------
namespace g1g2 {
namespace {

// out_b[m][i] = sum_p in_b[p][m] op(S_b[i][p]) with m = (q, r, s) running over the
// trailing nb^3 entries: a mode-1 product whose new index i moves to the last place,
// so four calls with S1..S4 apply S1 (x) S2 (x) S3 (x) S4 to the four indices and
// return them in their original order.  One thread per (m, b); its nb inputs
// in_b[p][m] are coalesced across the warp and held in registers.
template <int NMAX>
__global__ void __launch_bounds__(128) mode_rotate_kernel(int nb, const cplx *__restrict__ in,
                                                          const cplx *__restrict__ S, int conjS,
                                                          cplx *__restrict__ out) {
  __shared__ cplx Ss[NMAX * NMAX];
  const long long N3 = (long long)nb * nb * nb, N4 = N3 * nb;
  const long long b = blockIdx.y;
  const cplx *Sb = S + b * nb * nb;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    cplx v = Sb[e];
    if (conjS) v.y = -v.y;
    Ss[e] = v;
  }
  __syncthreads();
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N3) return;
  const cplx *ib = in + b * N4 + m;
  cplx x[NMAX];
#pragma unroll
  for (int p = 0; p < NMAX; ++p) x[p] = (p < nb) ? ib[(long long)p * N3] : cplx{0.0, 0.0};
  cplx *ob = out + b * N4 + m * nb;
  for (int i = 0; i < nb; ++i) {
    cplx acc = {0.0, 0.0};
#pragma unroll
    for (int p = 0; p < NMAX; ++p)
      if (p < nb) acc = cfma(x[p], Ss[i * nb + p], acc);
    ob[i] = acc;
  }
}

// out[e] = beta out[e] + sum_b x[b len + e]: 32 consecutive entries per block, the
// batch split over the block's eight warps (b = warp + 8 r), then a fixed-order
// reduction over the warps in shared memory (deterministic).
__global__ void __launch_bounds__(256) batch_sum_kernel(long long len, int nbatch, const cplx *__restrict__ x,
                                                        double beta, cplx *out) {
  __shared__ cplx part[8][32];
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  const long long e = (long long)blockIdx.x * 32 + lane;
  cplx s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
  if (e < len) {
    int b = wv;
    for (; b + 8 < nbatch; b += 16) {
      s0 = cadd(s0, x[(long long)b * len + e]);
      s1 = cadd(s1, x[(long long)(b + 8) * len + e]);
    }
    if (b < nbatch) s0 = cadd(s0, x[(long long)b * len + e]);
  }
  part[wv][lane] = cadd(s0, s1);
  __syncthreads();
  if (wv != 0 || e >= len) return;
  cplx s = (beta != 0.0) ? cscale(out[e], beta) : cplx{0.0, 0.0};
#pragma unroll
  for (int w = 0; w < 8; ++w) s = cadd(s, part[w][lane]);
  out[e] = s;
}

__global__ void count_nonzero_kernel(const cplx *x, long long len, double *cnt) {
  __shared__ double s[256];
  double a = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    if (x[i].x != 0.0 || x[i].y != 0.0) a += 1.0;
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && s[0] != 0.0) atomicAdd(cnt, s[0]);
}

}  // namespace

int mode_rotate_max_nb() { return 32; }

void mode_rotate(Launcher &L, int nb, int batch, const cplx *in, const cplx *S, bool conjS, cplx *out) {
  if (batch <= 0) return;
  const long long N3 = (long long)nb * nb * nb;
  dim3 grid((unsigned)((N3 + 127) / 128), (unsigned)batch);
  L.before("hfgkba_mode_rotate");
  if (nb <= 8)
    mode_rotate_kernel<8><<<grid, 128, 0, L.stream>>>(nb, in, S, conjS ? 1 : 0, out);
  else if (nb <= 16)
    mode_rotate_kernel<16><<<grid, 128, 0, L.stream>>>(nb, in, S, conjS ? 1 : 0, out);
  else
    mode_rotate_kernel<32><<<grid, 128, 0, L.stream>>>(nb, in, S, conjS ? 1 : 0, out);
  L.after_launch();
}

void batch_sum(Launcher &L, long long len, int nbatch, const cplx *x, double beta, cplx *out) {
  L.before("hfgkba_batch_sum");
  batch_sum_kernel<<<(unsigned)((len + 31) / 32), 256, 0, L.stream>>>(len, nbatch, x, beta, out);
  L.after_launch();
}

void count_nonzero(Launcher &L, const cplx *x, long long len, double *cnt) {
  const unsigned blocks = (unsigned)std::min<long long>((len + 255) / 256, 4096);
  L.before("nonzero_count");
  count_nonzero_kernel<<<blocks, 256, 0, L.stream>>>(x, len, cnt);
  L.after_launch();
}

}  // namespace g1g2

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe: the ALU roofline of the FP64 form
// ---------------------------------------------------------------------------
namespace g1g2 {
namespace {

// eight independent DFMA chains per thread, no memory traffic but one store per thread
__global__ void __launch_bounds__(256) dfma_probe_kernel(int iters, double *out) {
  const double m = 0.9999999, a = 1e-9;
  double x0 = threadIdx.x * 1e-6, x1 = x0 + 0.1, x2 = x0 + 0.2, x3 = x0 + 0.3;
  double x4 = x0 + 0.4, x5 = x0 + 0.5, x6 = x0 + 0.6, x7 = x0 + 0.7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, m, a); x1 = fma(x1, m, a); x2 = fma(x2, m, a); x3 = fma(x3, m, a);
    x4 = fma(x4, m, a); x5 = fma(x5, m, a); x6 = fma(x6, m, a); x7 = fma(x7, m, a);
  }
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

double dfma_rate(cudaStream_t stream, int *err) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, iters = 16384;   // about 0.8 s per launch
  double *out = nullptr;
  *err = 0;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    *err = 1;
    return 0.0;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  for (int rep = 0; rep < 5; ++rep) {   // the first two launches bring the clocks up
    cudaEventRecord(e0, stream);
    dfma_probe_kernel<<<blocks, threads, 0, stream>>>(iters, out);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) { *err = 1; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flop = 2.0 * 8.0 * iters * (double)blocks * threads;
    if (rep > 1 && ms > 0.f) best = std::max(best, flop / (ms * 1e-3) / 1e12);
  }
  if (cudaGetLastError() != cudaSuccess) *err = 1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return best;
}

}  // namespace g1g2
