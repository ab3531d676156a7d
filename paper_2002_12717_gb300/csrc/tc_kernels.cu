// Split-precision tensor-core form of the G1-G2 right-hand side (sm_103a).
//
// The nb^5 contractions run on tcgen05 (tc_gemm.cuh); the Hartree-Fock build,
// the G1 update, the RK4 state of G2 and the observables stay FP64.  Every
// contraction is written as a right multiplication of a big tensor by a small
// nb x nb matrix over its last index, using the symmetries the exact dynamics
// keep (Eqs. Gsymm_a/b for G2, Eqs. wsymm_a/b for w):
//
//   commutator (Eqs. twopart_hamiltonian, result_eom_soa): with M = G2 as an
//     nb^2 x nb^2 Hermitian matrix, [h2, M] = U^dag - U, U = M h2, and the
//     mode-3 half of U is the exchange image of the mode-4 half:
//     U_ijkl = Z_ijkl + Z_jilk,  Z = G2 x_4 hHF                      (1 pass)
//   source term (Eqs. psi-pm-def, soa-skalierung): A = (nbar (x) nbar) w~ (n (x) n),
//     Psi = A^dag - A; the chain is evaluated as
//       B1 = w~ x_4 n            stored exchange-permuted
//       B  = B1~ x_4 n           rows gathered, stored as B^dag (transposed, conj)
//       T2 = B^dag x_4 nbar      stored exchange-permuted
//       A^dag = T2~ x_4 nbar                                          (4 passes)
//   collision integral (Eq. eom_gone-I): I_ij = -i sum_c w_ic conj(G2_jc) with
//     c = (k,l,p), both operands row-contiguous; split-K over c.
//   polarisation and ladder products (Eqs. gwpi, lambdapp, lambdaph): one
//     nb^2 x nb^2 x nb^2 GEMM each, A = G2 read through a permutation of its
//     indices, B the realified quasi-Hamiltonian (tc_pi_gemm.cuh).
//   assembly: P = U - (Q + exch Q)/2 with Q = A^dag and dG2 = -i (P^dag - P), read as
//     the orbit {X, exch X, trans X, exch trans X} of 4^4 blocks so every
//     input block is read once; the RK4 stage update is fused.
//
// Two operand forms: TF32 hi/lo (three TF32 products) and BF16 slices with an
// exact leading product.  In the nb^5 passes (tc_gemm.cuh) the converters cut
// four slices with one exponent per tensor; the sliced form needs the largest
// magnitude of every A tensor before it is read, and each producer (the
// assembly, the FP32 copy of the state, the source-term passes) folds it into
// a slot of amax with an atomic maximum.  The nb^2 x nb^2 x nb^2 products take
// both operands as three slices cut beforehand by memory-bound passes, with
// one exponent per row of A and per column of B (a_rowmax/a_slice3,
// *_colmax/realify_*_slice3 below).
#include "tc_path.h"
#include "tc_gemm.cuh"
#include "tc_pi_gemm.cuh"
#include "tc_gemm_ts.cuh"
#include "tc_coll_ts.cuh"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace g1g2 {

using namespace tc;

namespace {

constexpr int BSZ_LOG = 2;
constexpr int BSZ = 1 << BSZ_LOG;            // assembly block edge; divides nb (nb % 4 == 0 here)
constexpr int BEL = BSZ * BSZ * BSZ * BSZ;  // elements per block

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ------------------------------------------------------------------ small kernels
// B operand of "X x_4 S" for a complex (planar) X: rows (v, l), K' = (u, p):
// (a_re, a_im) * S_pl as a real 2x2 block [[S_re, S_im], [-S_im, S_re]].
// Real X: rows (v, l), K' = p: S_v[p][l].  hi = TF32(x), lo = TF32(x - hi).
// Rows are ordered v nb + l, or 2 l + v with il (the real and imaginary part
// of one output element then sit in adjacent accumulator columns).
__global__ void realify_kernel(int nb, int nout, int kpad, int complex_a, int shift, double scale, int ld, int col0,
                               int transpose, int il, const cplx *__restrict__ S, float *hi, float *lo) {
  const int kt = complex_a ? 2 * kpad : kpad;
  const int total = nout * kt;
  // optional shift S -> S - mu 1 with mu = Re Tr S / nb (the commutator does not see it)
  double mu = 0.0;
  if (shift)
    for (int i = 0; i < nb; ++i) mu += S[i * nb + i].x;
  mu /= nb;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int row = e / kt, col = e % kt;
    double x = 0.0;
    if (row < 2 * nb) {
      const int v = il ? (row & 1) : row / nb, l = il ? (row >> 1) : row % nb;
      const int u = complex_a ? col / kpad : 0;
      const int pp = complex_a ? col % kpad : col;
      if (pp < nb) {
        cplx s = transpose ? S[l * nb + pp] : S[pp * nb + l];
        if (pp == l) s.x -= mu;
        if (!complex_a) x = v ? s.y : s.x;
        else if (u == 0) x = v ? s.y : s.x;
        else x = v ? s.x : -s.y;
      }
    }
    x *= scale;
    const float h = to_tf32((float)x);
    hi[row * ld + col0 + col] = h;
    lo[row * ld + col0 + col] = to_tf32((float)(x - (double)h));
  }
}

// w (real part of the FP64 interleaved tensor) -> hi/lo TF32 arrays [i][c].
__global__ void split_real_kernel(long long n, const cplx *__restrict__ w, float *hi, float *lo) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double x = w[e].x;
    const float h = to_tf32((float)x);
    hi[e] = h;
    lo[e] = to_tf32((float)(x - (double)h));
  }
}

// block-wide maximum of v folded into *slot (FP32 bit patterns of non-negative values order as ints)
__device__ __forceinline__ void block_amax(float v, int *slot) {
  __shared__ int smx;
  if (threadIdx.x == 0) smx = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&smx, __float_as_int(v));
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(slot, smx);
}

// interleaved FP64 -> planar FP32 (re plane, im plane); amax (optional): max |out|
__global__ void to_planar_f32_kernel(long long n, const cplx *__restrict__ x, float *out, int *amax) {
  float mx = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const cplx v = x[e];
    const float re = (float)v.x, im = (float)v.y;
    out[e] = re;
    out[n + e] = im;
    mx = fmaxf(mx, fmaxf(fabsf(re), fabsf(im)));
  }
  if (amax) block_amax(mx, amax);
}

// value of the real B operand of realify_kernel at (row, col) (no scale)
__device__ __forceinline__ double realified(int nb, int kpad, int complex_a, int transpose, int il, double mu,
                                            const cplx *__restrict__ S, int row, int col) {
  if (row >= 2 * nb) return 0.0;
  const int v = il ? (row & 1) : row / nb, l = il ? (row >> 1) : row % nb;
  const int u = complex_a ? col / kpad : 0;
  const int pp = complex_a ? col % kpad : col;
  if (pp >= nb) return 0.0;
  cplx s = transpose ? S[l * nb + pp] : S[pp * nb + l];
  if (pp == l) s.x -= mu;
  if (!complex_a || u == 0) return v ? s.y : s.x;
  return v ? s.x : -s.y;
}

// Four BF16 slices of x (|x| < 2^E), cut in FP64 as slice4 does in FP32: slice q
// is x's remainder rounded to nearest-even on the grid 2^(E-L-8q) (add and
// subtract of c[q] = 1.5 2^(52+E-L-8q)), at most 8 significant bits, exact in BF16.
__device__ __forceinline__ void slice_cuts_f64(int E, int L, double (&c)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) c[q] = ldexp(1.5, 52 + E - L - 8 * q);
}
__device__ __forceinline__ void slice4_f64(double x, const double (&c)[4], __nv_bfloat16 *out, long long stride) {
  double r = x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double v = __dsub_rn(__dadd_rn(r, c[q]), c[q]);
    r = __dsub_rn(r, v);
    out[q * stride] = __float2bfloat16_rn((float)v);
  }
}

// Sliced form of realify_kernel: the same real matrix, one power-of-two scale
// from its largest magnitude, written as slices [q][row][ld].  The realified
// matrix holds +-Re and +-Im of the (shifted) entries of S, so every CTA takes
// the maximum over the nb^2 entries of S itself and slices its share.
// One operand of slice_b_kernel: the matrix S and how it is realified (see realify_kernel).
struct SliceBOp {
  const cplx *S;
  __nv_bfloat16 *out;
  long long slice_stride;
  int complex_a, shift, ld, transpose, il;
};
constexpr int kMaxSliceBOps = 8;
struct SliceBBatch {
  SliceBOp op[kMaxSliceBOps];
};

// The B operands of one right-hand side in one launch: grid row blockIdx.y slices op[y].
__global__ void __launch_bounds__(256) slice_b_kernel(int nb, int nout, int kpad, const SliceBBatch batch) {
  const SliceBOp &o = batch.op[blockIdx.y];
  const cplx *__restrict__ S = o.S;
  const int complex_a = o.complex_a, shift = o.shift, ld = o.ld, transpose = o.transpose, il = o.il;
  __nv_bfloat16 *out = o.out;
  const long long slice_stride = o.slice_stride;
  __shared__ double red[8];
  __shared__ double smu;
  const int kt = complex_a ? 2 * kpad : kpad;
  const int total = nout * kt;
  if (threadIdx.x < 32) {
    // mu = Re Tr S / nb over warp 0 (lane-strided, fixed-order shuffle reduction)
    double mu = 0.0;
    if (shift)
      for (int i = threadIdx.x; i < nb; i += 32) mu += S[i * nb + i].x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mu += __shfl_xor_sync(0xffffffffu, mu, o);
    if (threadIdx.x == 0) smu = mu / nb;
  }
  __syncthreads();
  const double mu = smu;
  double mx = 0.0;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    cplx v = S[e];
    if (e / nb == e % nb) v.x -= mu;
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  int E = 0;
  if (mx > 0.0) frexp(mx, &E);  // mx < 2^E
  double c[4];
  slice_cuts_f64(E, 7, c);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int row = e / kt, col = e % kt;
    slice4_f64(realified(nb, kpad, complex_a, transpose, il, mu, S, row, col), c, out + (long long)row * ld + col,
               slice_stride);
  }
}

// real part of w -> four BF16 slices [q][i][c] with the common exponent E
__global__ void slice_w_kernel(long long n, const cplx *__restrict__ w, int E, __nv_bfloat16 *out) {
  double c[4];
  slice_cuts_f64(E, 7, c);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    slice4_f64(w[e].x, c, out + e, n);
}

// I_ij = -D1[j][i] - i D0[j][i], summed over the K splits in FP64.  Block (32, 8):
// x runs over 32 consecutive (j, i) of the partial layout, y over the splits.
__global__ void __launch_bounds__(256) collision_reduce_kernel(int nb, int splits, const double *__restrict__ partial,
                                                              cplx *I) {
  __shared__ double2 red[8][33];
  const int e = blockIdx.x * 32 + threadIdx.x;  // j nb + i
  const long long plane = (long long)nb * nb;
  double d0 = 0.0, d1 = 0.0;
  if (e < nb * nb)
    for (int s = threadIdx.y; s < splits; s += 8) {
      d0 += partial[(long long)s * 2 * plane + e];
      d1 += partial[((long long)s * 2 + 1) * plane + e];
    }
  red[threadIdx.y][threadIdx.x] = make_double2(d0, d1);
  __syncthreads();
  if (threadIdx.y != 0 || e >= nb * nb) return;
  for (int y = 1; y < 8; ++y) {
    d0 += red[y][threadIdx.x].x;
    d1 += red[y][threadIdx.x].y;
  }
  const int j = e / nb, i = e % nb;
  I[i * nb + j] = {-d1, -d0};
}

// B operand of the polarisation GEMM: rows (j,l,v) interleaved as 2 (j nb + l) + v,
// K = (u, p, q) as (u nb + p) kpad + q, value R(hcorr_qjpl)[u][v] split into TF32
// hi/lo, with hcorr_qjpl = Y1_qjpl - Y2_plqj (Y1 = w x_4 n, Y2 = w x_4 n^T, both
// in the swapped layout [a][b][d][c]).  One CTA per (j,l) and 32x32 (p,q) tile.
__global__ void realify_pi_kernel(int nb, int kpad, const float *__restrict__ Y1s, const float *__restrict__ Y2s,
                                  long long P, float *hi, float *lo, long long ldb) {
  __shared__ float2 t1[32][33];
  const long long N = nb;
  const long long jl = blockIdx.y;
  const long long j = jl / N, l = jl % N;
  const int ntq = kpad / 32;
  const int p0 = (blockIdx.x / ntq) * 32, q0 = (blockIdx.x % ntq) * 32;
  const int tx = threadIdx.x, ty0 = threadIdx.y;
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int q = q0 + ty, pp = p0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (q < nb && pp < nb) {
      const long long g = ((q * N + j) * N + l) * N + pp;   // Y1_{q j p l} at [q][j][l][p]
      v = make_float2(Y1s[g], Y1s[P + g]);
    }
    t1[ty][tx] = v;
  }
  __syncthreads();
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int pp = p0 + ty, q = q0 + tx;
    if (pp >= nb) continue;
    float2 h = make_float2(0.f, 0.f);
    if (q < nb) {
      const long long g = ((pp * N + l) * N + j) * N + q;   // Y2_{p l q j} at [p][l][j][q]
      const float2 a = t1[tx][ty];
      h = make_float2(a.x - Y2s[g], a.y - Y2s[P + g]);
    }
    for (int u = 0; u < 2; ++u)
      for (int v = 0; v < 2; ++v) {
        const float x = (u == 0) ? (v ? h.y : h.x) : (v ? h.x : -h.y);
        const long long row = 2 * jl + v;
        const long long col = ((long long)u * N + pp) * kpad + q;
        const float hh = to_tf32(x);
        hi[row * ldb + col] = hh;
        lo[row * ldb + col] = to_tf32(x - hh);
      }
  }
}

// B operand of the polarisation GEMM (tc_pi_gemm_kernel): rows (j, l, v) interleaved as
// 2 (j nb + l) + v, K = (u, p, q) as (u nb + p) nb + q, value R(hcorr_qjpl)[u][v] (the
// real 2 x 2 block [[Re, Im], [-Im, Re]] of the complex product) with
// hcorr_qjpl = Y1_qjpl - Y2_plqj (Y1 = w x_4 n, Y2 = w x_4 n^T in the swapped layout
// [a][b][d][c]), as three BF16 slices [slice][row][K] with one exponent per column (j, l):
// that of max over (p, q) of the larger component of hcorr_qjpl.  One CTA per (j, l):
// a first sweep over the 32 x 32 tiles of (p, q) takes the maximum, a second one (its
// reads served from L2) slices; Y1 is read along p and Y2 along q, transposed in shared
// memory.
__global__ void __launch_bounds__(256) realify_pi_slice3_kernel(int nb, const float *__restrict__ Y1s,
                                                                const float *__restrict__ Y2s, long long P,
                                                                __nv_bfloat16 *out, long long slice_stride) {
  __shared__ float2 t1[32][33];
  __shared__ float red[8];
  extern __shared__ float4 hs_raw[];   // nb * nb float2 (dynamic)
  const long long N = nb, K = 2 * N * N;
  const long long jl = blockIdx.x;
  const long long j = jl / N, l = jl % N;
  const int nt = (nb + 31) / 32;
  const int tx = threadIdx.x & 31, ty0 = threadIdx.x >> 5;
  auto load_tile = [&](int p0, int q0) {
    for (int ty = ty0; ty < 32; ty += 8) {
      const int q = q0 + ty, pp = p0 + tx;
      float2 v = make_float2(0.f, 0.f);
      if (q < nb && pp < nb) {
        const long long g = ((q * N + j) * N + l) * N + pp;   // Y1_{q j p l} at [q][j][l][p]
        v = make_float2(Y1s[g], Y1s[P + g]);
      }
      t1[ty][tx] = v;
    }
  };
  auto hval = [&](int pp, int q, int ty) {   // hcorr_qjpl (after load_tile and a barrier)
    const long long g = ((pp * N + l) * N + j) * N + q;       // Y2_{p l q j} at [p][l][j][q]
    const float2 a = t1[tx][ty];
    return make_float2(a.x - Y2s[g], a.y - Y2s[P + g]);
  };
  // first sweep: hcorr of this (j, l) into shared memory (Hs[p nb + q]) and its largest
  // magnitude; the slicing sweep then reads shared memory only, so Y1 and Y2 stream once
  float2 *Hs = reinterpret_cast<float2 *>(hs_raw);
  float mx = 0.f;
  for (int tile = 0; tile < nt * nt; ++tile) {
    const int p0 = (tile / nt) * 32, q0 = (tile % nt) * 32;
    __syncthreads();
    load_tile(p0, q0);
    __syncthreads();
    for (int ty = ty0; ty < 32; ty += 8) {
      const int pp = p0 + ty, q = q0 + tx;
      if (pp < nb && q < nb) {
        const float2 h = hval(pp, q, ty);
        Hs[pp * nb + q] = h;
        mx = fmaxf(mx, fmaxf(fabsf(h.x), fabsf(h.y)));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (tx == 0) red[ty0] = mx;
  __syncthreads();   // also orders the Hs writes before the reads below
  mx = red[0];
  for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
  float cut[3];
  cuts3_lead8(slice_exponent(__float_as_int(mx)), cut);
  // slicing sweep: thread e cuts the pair q = 2 e mod nb, q + 1 of row p = 2 e / nb (nb is
  // even), so a warp stores 128 contiguous bytes per slice and output row
  for (int e = threadIdx.x; e < nb * nb / 2; e += blockDim.x) {
    const int pp = (2 * e) / nb, q = 2 * e - pp * nb;
    const float4 hv = reinterpret_cast<const float4 *>(Hs)[e];
    const float2 h0 = make_float2(hv.x, hv.y), h1 = make_float2(hv.z, hv.w);
    for (int u = 0; u < 2; ++u)
      for (int v = 0; v < 2; ++v) {
        const float x0 = (u == 0) ? (v ? h0.y : h0.x) : (v ? h0.x : -h0.y);
        const float x1 = (u == 0) ? (v ? h1.y : h1.x) : (v ? h1.x : -h1.y);
        const long long row = 2 * jl + v;
        const long long col = ((long long)u * N + pp) * N + q;
        float s0[3], s1[3];
        slice3(x0, cut, s0);
        slice3(x1, cut, s1);
#pragma unroll
        for (int z = 0; z < 3; ++z)
          *reinterpret_cast<__nv_bfloat162 *>(out + z * slice_stride + row * K + col) = __floats2bfloat162_rn(s0[z], s1[z]);
      }
  }
}

// B operand of the ladder products Lambda^dag = G2 H^dag (Eqs. lambdapp, lambdaph; G2 is
// Hermitian as an nb^2 x nb^2 matrix) for tc_pi_gemm_kernel: rows (c, d, v) interleaved as
// 2 (c nb + d) + v, K = (u, p, q) as (u nb + p) nb + q, value R(X)[u][v] with
// X = H^dag_pqcd = conj(hcorr_cdpq) = P1_pqcd - P2_pqcd, both stored as [q][p][c][d] (the
// two right-multiplication passes w x3 S x4 S with S = nbar and S = n), as three BF16
// slices with the exponent of the column's maximum colmax[c nb + d].  One CTA per (p, c)
// and a 32 x 32 tile of (q, d): read along d, transposed in shared memory, written along q.
__global__ void realify_lam_slice3_kernel(int nb, const float *__restrict__ P1s, const float *__restrict__ P2s,
                                          long long P, const int *__restrict__ colmax, __nv_bfloat16 *out,
                                          long long slice_stride) {
  __shared__ float2 t1[32][33];
  __shared__ float sc[32][3];
  const long long N = nb, K = 2 * N * N;
  const long long pc = blockIdx.y;
  const long long p = pc / N, c = pc % N;
  const int ntd = (nb + 31) / 32;
  const int q0 = (blockIdx.x / ntd) * 32, d0 = (blockIdx.x % ntd) * 32;
  const int tx = threadIdx.x, ty0 = threadIdx.y;
  if (ty0 == 0) {
    float cu[3];
    cuts3_lead8((d0 + tx < nb) ? slice_exponent(colmax[c * N + d0 + tx]) : 0, cu);
    sc[tx][0] = cu[0];
    sc[tx][1] = cu[1];
    sc[tx][2] = cu[2];
  }
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int q = q0 + ty, d = d0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (q < nb && d < nb) {
      const long long g = ((q * N + p) * N + c) * N + d;   // H^dag_{p q c d} at [q][p][c][d]
      v = make_float2(P1s[g] - P2s[g], P1s[P + g] - P2s[P + g]);
    }
    t1[ty][tx] = v;
  }
  __syncthreads();
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int d = d0 + ty, q = q0 + tx;
    if (d >= nb || q >= nb) continue;
    const float2 h = t1[tx][ty];
    const float cu[3] = {sc[ty][0], sc[ty][1], sc[ty][2]};
    for (int u = 0; u < 2; ++u)
      for (int v = 0; v < 2; ++v) {
        const float x = (u == 0) ? (v ? h.y : h.x) : (v ? h.x : -h.y);
        const long long row = 2 * (c * N + d) + v;
        const long long col = ((long long)u * N + p) * N + q;
        float sl[3];
        slice3(x, cu, sl);
#pragma unroll
        for (int z = 0; z < 3; ++z) out[z * slice_stride + row * K + col] = __float2bfloat16_rn(sl[z]);
      }
  }
}

// Per-column maxima of the ladder products' B operand: colmax[c nb + d] = max over (p, q)
// of the larger component of P1_pqcd - P2_pqcd ([q][p][c][d] layout), atomic max of FP32
// bits.  One CTA per (p, c) and 32 x 32 tile of (q, d).
__global__ void ladder_colmax_kernel(int nb, const float *__restrict__ P1s, const float *__restrict__ P2s,
                                     long long P, int *colmax) {
  __shared__ float red[8][33];
  const long long N = nb;
  const long long pc = blockIdx.y;
  const long long p = pc / N, c = pc % N;
  const int ntd = (nb + 31) / 32;
  const int q0 = (blockIdx.x / ntd) * 32, d0 = (blockIdx.x % ntd) * 32;
  float mx = 0.f;
  const int d = d0 + threadIdx.x;
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int q = q0 + ty;
    if (q < nb && d < nb) {
      const long long g = ((q * N + p) * N + c) * N + d;
      mx = fmaxf(mx, fmaxf(fabsf(P1s[g] - P2s[g]), fabsf(P1s[P + g] - P2s[P + g])));
    }
  }
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && d < nb) {
    for (int y = 1; y < (int)blockDim.y; ++y) mx = fmaxf(mx, red[y][threadIdx.x]);
    atomicMax(colmax + c * N + d, __float_as_int(mx));
  }
}

// The A operand of the nb^2 x nb^2 x nb^2 products read from the planar FP32 state G
// (plane stride P): row m = (a, b) = a nb + b, K = (u, p, q) as (u nb + p) nb + q, value
// G[u P + a sA + b sB + p sP + q sQ].  The polarisation reads G_ipkq (rows (i, k)), the
// particle-particle ladder G_ijpq (rows (i, j)), the particle-hole ladder G_ipql (rows (i, l)).
struct AOperand {
  long long sA, sB, sP, sQ;
};

// rowmax[a nb + b] = max over (u, p, q) of |G element| (FP32 bits, atomic max).  One CTA
// (32 x 8 threads) per (a, 32-row block of b) and (u, 8 values of p); the fast thread index
// runs along whichever of b and q is contiguous in memory.
__global__ void a_rowmax_kernel(int nb, const float *__restrict__ G, long long P, AOperand m, int *rowmax) {
  __shared__ float red[8][33];
  const long long N = nb;
  const int nbt = (nb + 31) / 32;
  const long long a = blockIdx.x / nbt;
  const int b0 = (blockIdx.x % nbt) * 32;
  const int npb = (nb + 7) / 8;
  const int u = blockIdx.y / npb, p0 = (blockIdx.y % npb) * 8;
  const bool b_fast = m.sB == 1;
  const float *base = G + u * P + a * m.sA;
  float mx = 0.f;  // b_fast: row b0 + x; else per-thread over its rows, reduced below
  float rmx[4] = {0.f, 0.f, 0.f, 0.f};
  for (int pp = p0; pp < min(p0 + 8, nb); ++pp)
    for (int q0 = 0; q0 < nb; q0 += 32) {
      if (b_fast) {
        const int b = b0 + threadIdx.x;
        for (int ty = threadIdx.y; ty < 32; ty += 8) {
          const int q = q0 + ty;
          if (b < nb && q < nb) mx = fmaxf(mx, fabsf(base[b * m.sB + pp * m.sP + q * m.sQ]));
        }
      } else {
        const int q = q0 + threadIdx.x;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int b = b0 + threadIdx.y + 8 * i;
          if (b < nb && q < nb) rmx[i] = fmaxf(rmx[i], fabsf(base[b * m.sB + pp * m.sP + q * m.sQ]));
        }
      }
    }
  if (b_fast) {
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && b0 + (int)threadIdx.x < nb) {
      for (int y = 1; y < 8; ++y) mx = fmaxf(mx, red[y][threadIdx.x]);
      atomicMax(rowmax + a * N + b0 + threadIdx.x, __float_as_int(mx));
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float v = rmx[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      const int b = b0 + threadIdx.y + 8 * i;
      if (threadIdx.x == 0 && b < nb) atomicMax(rowmax + a * N + b, __float_as_int(v));
    }
  }
}

// Three BF16 slices [slice][row][K] of the A operand (see AOperand) with the exponent of
// each row's maximum rowmax[row] and a 9-bit leading slice (slice3).  One CTA (32 x 8
// threads) per (a, 32-row block of b) and (u, p): a 32 x 32 tile of (b, q) is read along
// the contiguous index into shared memory; each thread then cuts two adjacent q of one row
// and stores them as BF16 pairs.
__global__ void a_slice3_kernel(int nb, const float *__restrict__ G, long long P, AOperand m,
                                const int *__restrict__ rowmax, __nv_bfloat16 *out, long long slice_stride) {
  __shared__ float t[32][34];
  __shared__ float sc[32][3];
  const long long N = nb, K = 2 * N * N;
  const int nbt = (nb + 31) / 32;
  const long long a = blockIdx.x / nbt;
  const int b0 = (blockIdx.x % nbt) * 32;
  const int u = blockIdx.y / nb, pp = blockIdx.y % nb;
  const bool b_fast = m.sB == 1;
  const float *base = G + u * P + a * m.sA + pp * m.sP;
  if (threadIdx.y == 0) {
    float cu[3];
    cuts3_lead8((b0 + (int)threadIdx.x < nb) ? slice_exponent(rowmax[a * N + b0 + threadIdx.x]) : 0, cu);
    sc[threadIdx.x][0] = cu[0];
    sc[threadIdx.x][1] = cu[1];
    sc[threadIdx.x][2] = cu[2];
  }
  const int qp = threadIdx.x & 15, rsub = threadIdx.x >> 4;   // q pair, row within the warp's pair
  for (int q0 = 0; q0 < nb; q0 += 32) {
    __syncthreads();
    for (int ty = threadIdx.y; ty < 32; ty += 8) {
      // t[b][q]
      const int b = b0 + (b_fast ? (int)threadIdx.x : ty), q = q0 + (b_fast ? ty : (int)threadIdx.x);
      const float x = (b < nb && q < nb) ? base[b * m.sB + q * m.sQ] : 0.f;
      if (b_fast) t[threadIdx.x][ty] = x;
      else t[ty][threadIdx.x] = x;
    }
    __syncthreads();
    for (int rb = 2 * threadIdx.y + rsub; rb < 32; rb += 16) {
      const int b = b0 + rb, q = q0 + 2 * qp;
      if (b >= nb || q >= nb) continue;   // nb % 4 == 0: q and q + 1 are both in range
      const float cu[3] = {sc[rb][0], sc[rb][1], sc[rb][2]};
      float s0[3], s1[3];
      slice3(t[rb][2 * qp], cu, s0);
      slice3(t[rb][2 * qp + 1], cu, s1);
      const long long o = (a * N + b) * K + ((long long)u * N + pp) * N + q;
#pragma unroll
      for (int z = 0; z < 3; ++z)
        *reinterpret_cast<__nv_bfloat162 *>(out + z * slice_stride + o) = __floats2bfloat162_rn(s0[z], s1[z]);
    }
  }
}

// Q[a][b][c][d] -= Lam[a][d][b][c] (interleaved complex FP32): the particle-hole ladder
// product from the polarisation epilogue's layout into the source-term buffer's.  One
// CTA per (a, b) and a 32 x 32 tile of (c, d), transposed in shared memory.
__global__ void sub_rot_kernel(int nb, const float2 *__restrict__ Lam, float2 *Q) {
  __shared__ float2 t1[32][33];
  const long long N = nb;
  const long long ab = blockIdx.y;
  const long long a = ab / N, b = ab % N;
  const int nt = (nb + 31) / 32;
  const int c0 = (blockIdx.x / nt) * 32, d0 = (blockIdx.x % nt) * 32;
  const int tx = threadIdx.x, ty0 = threadIdx.y;
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int d = d0 + ty, c = c0 + tx;
    if (d < nb && c < nb) t1[ty][tx] = Lam[((a * N + d) * N + b) * N + c];
  }
  __syncthreads();
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int c = c0 + ty, d = d0 + tx;
    if (c < nb && d < nb) {
      float2 *o = Q + blk4(N, a, b, c, d);
      const float2 l = t1[tx][ty];
      *o = make_float2(o->x - l.x, o->y - l.y);
    }
  }
}

// Q[a][b][c][d] -= Lam[a][d][c][b] (interleaved complex FP32): the ladder product from the
// polarisation epilogue's layout into the source-term buffer's.  One CTA per (a, c) and a
// 32 x 32 tile of (b, d), transposed in shared memory.
__global__ void sub_swap13_kernel(int nb, const float2 *__restrict__ Lam, float2 *Q) {
  __shared__ float2 t1[32][33];
  const long long N = nb;
  const long long ac = blockIdx.y;
  const long long a = ac / N, c = ac % N;
  const int nt = (nb + 31) / 32;
  const int b0 = (blockIdx.x / nt) * 32, d0 = (blockIdx.x % nt) * 32;
  const int tx = threadIdx.x, ty0 = threadIdx.y;
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int d = d0 + ty, b = b0 + tx;
    if (d < nb && b < nb) t1[ty][tx] = Lam[((a * N + d) * N + c) * N + b];
  }
  __syncthreads();
  for (int ty = ty0; ty < 32; ty += blockDim.y) {
    const int b = b0 + ty, d = d0 + tx;
    if (b < nb && d < nb) {
      float2 *o = Q + blk4(N, a, b, c, d);
      const float2 l = t1[tx][ty];
      *o = make_float2(o->x - l.x, o->y - l.y);
    }
  }
}

struct AsmParams {
  int nb, nblk;
  const int4 *blocks;
  const float *Z, *Q, *Pi;     // interleaved complex FP32, swapped layout in 4^4 blocks (blk4)
  long long P;                 // plane stride of ys and y32
  cplx *y;                     // FP64 state (interleaved): read and written at the last stage
  float *acc;                  // interleaved complex FP32 in 4^4 blocks (blk4)
  float *ys;                   // planar FP32 stage input of the next stage (stages 0-2)
  float *y32;                  // planar FP32 copy of y: read at stages 0-2, rewritten at the last
  cplx *kout;                  // write-k mode
  int stage;
  float hs;                    // stages 0-2: the stage's step (dt / 2 or dt) in FP32
  double dt6;                  // last stage: dt / 6
  int *amax;                   // optional: max |written ys or y32| (sliced form)
};

// Shared-memory slot of block element (a,b,c,d) (BSZ = 4): row (a,b) of 16 slots, and
// within the row the slot (a ^ c, b ^ d).  A half-warp (16 lanes of fixed (a,b) in
// thread order) then reads or writes 16 distinct slots mod 16 (one 128-byte wavefront
// of float2) under each of the permutations of (a,b,c,d) the assembly uses.
__device__ __forceinline__ int sidx(int a, int b, int c, int d) {
  return ((a * BSZ + b) << 4) | (((a ^ c) & (BSZ - 1)) << 2) | ((b ^ d) & (BSZ - 1));
}

// 4^4 blocks: 8 KB of shared memory and 256 threads per orbit CTA, so that eight CTAs
// share an SM and the load, combine and update phases of different orbits overlap
constexpr int ATHREADS = 256;               // assembly threads per CTA
constexpr int APER = BEL / ATHREADS;        // element orbits per thread

__device__ __forceinline__ void elem(int e, int &a, int &b, int &c, int &d) {
  a = e >> (3 * BSZ_LOG); b = (e >> (2 * BSZ_LOG)) & (BSZ - 1); c = (e >> BSZ_LOG) & (BSZ - 1); d = e & (BSZ - 1);
}

__device__ __forceinline__ float2 sval(const float2 *sm, int m, int a, int b, int c, int d, bool swap34) {
  return sm[m * BEL + (swap34 ? sidx(a, b, d, c) : sidx(a, b, c, d))];
}

// Conversions between IEEE-754 binary32 and binary64 done on the bit patterns with
// integer instructions.  GB300 issues FP64 instructions (conversions included) at a
// small fraction of its FP32 and integer rates, and the assembly would otherwise spend
// more time on them than on its HBM traffic.  Both follow the formats' definitions:
// binary32 = (s, 8-bit exponent biased by 127, 23-bit fraction), binary64 = (s, 11-bit
// exponent biased by 1023, 52-bit fraction).
//
// f32 -> f64 is exact for normal numbers, zero, infinities and NaNs; a subnormal input
// becomes a zero of the same sign.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint32_t hi = u & 0x80000000u, lo = 0u;
  if (e != 0u) {
    hi |= ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | (m >> 3);   // 896 = 1023 - 127
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// f64 -> f32, round to nearest, ties to even, for results in the binary32 normal range;
// magnitudes below 2^-126 become a zero of the same sign, magnitudes beyond the range
// infinity, and a NaN stays a NaN.
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t E = (hi >> 20) & 0x7ffu;
  // the upper 23 of the 52 fraction bits; the lower 29 decide the rounding
  uint32_t mag = ((E - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  mag += (rest > 0x10000000u || (rest == 0x10000000u && (mag & 1u))) ? 1u : 0u;   // may carry into the exponent
  if (E < 897u) mag = 0u;
  if (E >= 1151u) mag = (E == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float((hi & 0x80000000u) | mag);
}

// Stage kinds of the assembly: the plain right-hand side (k written in FP64), RK4 stages
// 0-2 (next stage input and accumulator) and the last stage (the FP64 state update).
enum AsmKind { kAsmK = 0, kAsmStage = 1, kAsmLast = 2 };

// One CTA per orbit {X, exch X, trans X, exch trans X} of BSZ^4 blocks, each thread
// APER element orbits.  Z, Q and Pi arrive in the swapped layout and enter only as
// V = Z - Q/2 - Pi/2 per element: with P = U - (Q + exch Q)/2 and U = Z + exch Z,
// dG2 = -i (P^dag - P) plus the polarisation term (Pi_ijkl - conj(Pi_lkji), symmetrised
// over the exchange) is, on the two exchange pairs (0,1) and (2,3) of the orbit,
//   k0 = -i (conj(V2 + V3) - (V0 + V1)),   k2 = -i (conj(V0 + V1) - (V2 + V3)).
// So one load phase reads Z, Q and Pi together with the RK4 state of the update, one
// shared-memory exchange forms the orbit sums, and the update stores.  The tensor-core
// form requires nb % 4 == 0 (tc_create), so BSZ = 4 blocks tile the tensor exactly and
// no element of a block lies outside it.
//
// RK4 (classical, k in FP32 from the tensor-core products):
//   stages 0-2: ys = y32 + h k (FP32; y32 the FP32 rounding of the state y),
//               acc = acc + w k (w = 1 at stage 0, else 2; FP32);
//   last stage: y = y + dt/6 (acc + k) with one FP64 fused multiply-add per component,
//               y32 = the FP32 rounding of the new y.
// The stage inputs are FP32 operands of the next products in either case; only the
// state update needs FP64, and it issues one FP64 instruction per real component.
template <int KIND>
__global__ void __launch_bounds__(ATHREADS, 4) orbit_assemble_kernel(const AsmParams p) {
  extern __shared__ float2 sm[];  // 4 * BEL
  const int4 base = p.blocks[blockIdx.x];
  const int X[4][4] = {{base.x, base.y, base.z, base.w},
                       {base.y, base.x, base.w, base.z},
                       {base.z, base.w, base.x, base.y},
                       {base.w, base.z, base.y, base.x}};
  const long long N = p.nb;
  const long long P = p.P;
  bool dup[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    dup[m] = false;
    for (int q = 0; q < m; ++q)
      dup[m] |= (X[q][0] == X[m][0] && X[q][1] == X[m][1] && X[q][2] == X[m][2] && X[q][3] == X[m][3]);
  }
  const bool acc_in = KIND == kAsmLast || (KIND == kAsmStage && p.stage > 0);
  float2 yf[4][APER];   // stages 0-2: the FP32 state
  cplx y0[4][APER];     // last stage: the FP64 state
  float2 ac[4][APER];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int t = 0; t < APER; ++t) {
      int a, b, c, d;
      elem(threadIdx.x + ATHREADS * t, a, b, c, d);
      // stored (swapped, 4^4-blocked) element of block (X0, X1, X3, X2): natural in-block index (a, b, d, c)
      const long long gs = blk4(N, X[m][0] * BSZ + a, X[m][1] * BSZ + b, X[m][3] * BSZ + c, X[m][2] * BSZ + d);
      const float2 z = reinterpret_cast<const float2 *>(p.Z)[gs];
      const float2 q = reinterpret_cast<const float2 *>(p.Q)[gs];
      float2 v = make_float2(z.x - 0.5f * q.x, z.y - 0.5f * q.y);
      if (p.Pi) {
        const float2 pi = reinterpret_cast<const float2 *>(p.Pi)[gs];
        v = make_float2(v.x - 0.5f * pi.x, v.y - 0.5f * pi.y);
      }
      sm[m * BEL + sidx(a, b, c, d)] = v;
      // RK4 state of the natural element (a, b, c, d) of member m
      const long long gn = (((X[m][0] * BSZ + a) * N + X[m][1] * BSZ + b) * N + X[m][2] * BSZ + c) * N +
                           X[m][3] * BSZ + d;
      if (KIND == kAsmStage) yf[m][t] = dup[m] ? make_float2(0.f, 0.f) : make_float2(p.y32[gn], p.y32[P + gn]);
      if (KIND == kAsmLast) y0[m][t] = dup[m] ? make_double2(0.0, 0.0) : p.y[gn];
      const long long gb = blk4(N, X[m][0] * BSZ + a, X[m][1] * BSZ + b, X[m][2] * BSZ + c, X[m][3] * BSZ + d);
      ac[m][t] = acc_in && !dup[m] ? reinterpret_cast<const float2 *>(p.acc)[gb] : make_float2(0.f, 0.f);
    }
  __syncthreads();
  float2 kx[APER], ky[APER];
#pragma unroll
  for (int t = 0; t < APER; ++t) {
    int a, b, c, d;
    elem(threadIdx.x + ATHREADS * t, a, b, c, d);
    const float2 v0 = sval(sm, 0, a, b, c, d, true), v1 = sval(sm, 1, b, a, d, c, true);
    const float2 v2 = sval(sm, 2, c, d, a, b, true), v3 = sval(sm, 3, d, c, b, a, true);
    const float2 s01 = make_float2(v0.x + v1.x, v0.y + v1.y), s23 = make_float2(v2.x + v3.x, v2.y + v3.y);
    const float2 D = make_float2(s23.x - s01.x, -s23.y - s01.y);   // conj(s23) - s01
    const float2 E = make_float2(s01.x - s23.x, -s01.y - s23.y);   // conj(s01) - s23
    kx[t] = make_float2(D.y, -D.x);
    ky[t] = make_float2(E.y, -E.x);
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < APER; ++t) {
    int a, b, c, d;
    elem(threadIdx.x + ATHREADS * t, a, b, c, d);
    sm[0 * BEL + sidx(a, b, c, d)] = kx[t];
    sm[1 * BEL + sidx(b, a, d, c)] = kx[t];
    sm[2 * BEL + sidx(c, d, a, b)] = ky[t];
    sm[3 * BEL + sidx(d, c, b, a)] = ky[t];
  }
  __syncthreads();
  // RK4 update of each distinct member block, in natural (coalesced) order
  const float w = p.stage == 0 ? 1.f : 2.f;
  float mx = 0.f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (dup[m]) continue;
#pragma unroll
    for (int t = 0; t < APER; ++t) {
      int a, b, c, d;
      elem(threadIdx.x + ATHREADS * t, a, b, c, d);
      const long long g = (((X[m][0] * BSZ + a) * N + X[m][1] * BSZ + b) * N + X[m][2] * BSZ + c) * N +
                          X[m][3] * BSZ + d;
      const float2 k = sm[m * BEL + sidx(a, b, c, d)];
      if (KIND == kAsmK) {
        p.kout[g] = make_double2(f32_to_f64_bits(k.x), f32_to_f64_bits(k.y));
      } else if (KIND == kAsmStage) {
        reinterpret_cast<float2 *>(p.acc)[blk4(N, X[m][0] * BSZ + a, X[m][1] * BSZ + b, X[m][2] * BSZ + c,
                                               X[m][3] * BSZ + d)] =
            make_float2(fmaf(w, k.x, ac[m][t].x), fmaf(w, k.y, ac[m][t].y));
        const float sx = fmaf(p.hs, k.x, yf[m][t].x), sy = fmaf(p.hs, k.y, yf[m][t].y);
        p.ys[g] = sx;
        p.ys[P + g] = sy;
        mx = fmaxf(mx, fmaxf(fabsf(sx), fabsf(sy)));
      } else {
        const double nx = fma(f32_to_f64_bits(ac[m][t].x + k.x), p.dt6, y0[m][t].x);
        const double ny = fma(f32_to_f64_bits(ac[m][t].y + k.y), p.dt6, y0[m][t].y);
        p.y[g] = make_double2(nx, ny);
        const float fx = f64_to_f32_bits(nx), fy = f64_to_f32_bits(ny);
        p.y32[g] = fx;
        p.y32[P + g] = fy;
        mx = fmaxf(mx, fmaxf(fabsf(fx), fabsf(fy)));
      }
    }
  }
  if (KIND != kAsmK && p.amax) block_amax(mx, p.amax);
}

// ------------------------------------------------------------------ tensor maps
// The tensor-map encoder is a driver entry point; it is looked up through the
// runtime so that the library does not link the driver library (it loads on
// machines without a GPU driver, where only the host-side entry points run).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int encode_map(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
               const cuuint32_t *box, bool bf16 = false) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return G1G2_ECUDA;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank,
                   const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? G1G2_OK : G1G2_ECUDA;
}

// A viewed as [planes][rows][K]
int map_linear(CUtensorMap *m, const float *base, int K, long long rows, int planes) {
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t str[2] = {(cuuint64_t)K * 4, (cuuint64_t)K * 4 * rows};
  cuuint32_t box[3] = {(cuuint32_t)kBlockK, (cuuint32_t)kTileM, 1};
  return encode_map(m, base, 3, dims, str, box);
}
// A = T[plane][a][b][c][s], box (s 32, c 1, b 32, a 4)
int map_gather(CUtensorMap *m, const float *base, int N, cuuint32_t b1 = 1, cuuint32_t b2 = 32, cuuint32_t b3 = 4) {
  const cuuint64_t n = N;
  cuuint64_t dims[5] = {n, n, n, n, 2};
  cuuint64_t str[4] = {n * 4, n * n * 4, n * n * n * 4, n * n * n * n * 4};
  cuuint32_t box[5] = {(cuuint32_t)kBlockK, b1, b2, b3, 1};
  return encode_map(m, base, 5, dims, str, box);
}
// small pre-split B operand [rows][kt]
int map_b(CUtensorMap *m, const float *base, int kt, int rows, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)kt, (cuuint64_t)rows, 1};
  cuuint64_t str[2] = {(cuuint64_t)kt * 4, (cuuint64_t)kt * 4 * rows};
  cuuint32_t box[3] = {(cuuint32_t)kBlockK, (cuuint32_t)box_rows, 1};
  return encode_map(m, base, 3, dims, str, box);
}
// B as BF16 slices [q][rows][kt] (four, or nslices); one box carries all of them
int map_bs(CUtensorMap *m, const __nv_bfloat16 *base, long long kt, int rows, int box_rows, int box_slices = kSlices,
           int nslices = kSlices) {
  cuuint64_t dims[3] = {(cuuint64_t)kt, (cuuint64_t)rows, (cuuint64_t)nslices};
  cuuint64_t str[2] = {(cuuint64_t)kt * 2, (cuuint64_t)kt * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)kBlockK, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
  return encode_map(m, base, 3, dims, str, box, true);
}

}  // namespace

struct TcPath {
  int nb = 0, se = 0, kpad = 0, nout2 = 0, nout1 = 0, sms = 0;
  bool restricted = false;
  long long N4 = 0;
  std::vector<void *> allocs;
  // FP32 planar tensors [2][nb^4]
  float *y32 = nullptr, *ys32 = nullptr, *acc = nullptr, *Z = nullptr, *buf1 = nullptr, *buf2 = nullptr;
  float *W32 = nullptr;                 // source interaction (real) [nb^4]
  float *Wh32 = nullptr;                // GW: w for the quasi-Hamiltonian (= W32 unless the source is w^-)
  float *w_hi = nullptr, *w_lo = nullptr;  // w (real) split [i][c]
  // small pre-split B operands
  float *bh_hi = nullptr, *bh_lo = nullptr;   // hHF, complex A
  float *bnr_hi = nullptr, *bnr_lo = nullptr; // n, real A
  float *bnc_hi = nullptr, *bnc_lo = nullptr; // n, complex A
  float *bnb_hi = nullptr, *bnb_lo = nullptr; // nbar, complex A
  double *partial = nullptr;
  cplx *nbar = nullptr, *I = nullptr;
  // GW: Y1 = w x_4 n, Y2 = w x_4 n^T, polarisation Pi, its B operand
  float *Y1 = nullptr, *Y2 = nullptr, *Pi = nullptr, *bpi_hi = nullptr, *bpi_lo = nullptr;
  float *bnt_hi = nullptr, *bnt_lo = nullptr;   // n^T, real A
  // particle-particle T matrix: Y1/Y2 hold the two terms of H^dag, Pi the ladder product
  __nv_bfloat16 *bnbr_s = nullptr, *bnbc_s = nullptr;  // nbar in the real-A and complex-A forms
  // particle-hole T matrix: Wp32[p][q][r][s] = w_rpqs, nbar^T in the real-A form; Lam: the
  // ladder products' output when the polarisation output Pi must survive (DSL)
  float *Wp32 = nullptr, *Lam = nullptr;
  __nv_bfloat16 *bnbt_s = nullptr;
  bool has_pi = false, has_pp = false, has_ph = false;
  double eta = -1.0;    // statistics sign: nbar = 1 + eta n (-1 fermions, +1 bosons)
  int pi_nout = 0, pi_ntiles = 0, pi_mtiles = 0;
  long long pi_ldb = 0;
  int4 *blocks = nullptr;
  int nblocks = 0;
  int *err = nullptr;
  int splits = 0, kb_all_coll = 0, kb_per_split = 0;
  // sliced form: BF16 slices [4][rows][kt] of the B operands and of w; A maxima
  bool sliced = false;
  __nv_bfloat16 *bh_s = nullptr, *bnr_s = nullptr, *bnc_s = nullptr, *bnb_s = nullptr, *bnt_s = nullptr,
                *w_s = nullptr;
  int *amax = nullptr;  // slots: see kAmax*
  // sliced nb^2 x nb^2 x nb^2 products (tc_pi_gemm_kernel): three BF16 slices of the A
  // operand [3][nb^2][2 nb^2] and of the B operand [3][2 nb^2][2 nb^2], per-row maxima of A
  // and per-column maxima of B (FP32 bits)
  __nv_bfloat16 *pa_s = nullptr, *pb_s = nullptr;
  int *rowmax = nullptr, *colmax = nullptr;
  CUtensorMap mBh_s, mBnr_s, mBnc_s, mBnb_s, mBnt_s, mW_s, mPa_s, mPb_s;
  // tensor maps
  CUtensorMap mZin_y32, mZin_ys32, mCol_y32, mCol_ys32, mW32, mWh32, mBuf1Gather, mBuf2Lin, mBuf1Lin;
  CUtensorMap mBh_hi, mBh_lo, mBnr_hi, mBnr_lo, mBnc_hi, mBnc_lo, mBnb_hi, mBnb_lo, mW_hi, mW_lo;
  CUtensorMap mPi_y32, mPi_ys32, mBpi_hi, mBpi_lo, mBnt_hi, mBnt_lo;
  CUtensorMap mBnbr_s, mBnbc_s, mWp32, mBnbt_s;
};

namespace {

// amax slots: FP32 bit patterns of the largest |A| of each A tensor of the sliced form
enum : int {
  kAmaxW = 0, kAmaxY = 1, kAmaxYs = 2, kAmaxP1 = 3, kAmaxP2 = 4, kAmaxP3 = 5, kAmaxH1 = 6, kAmaxH2 = 7,
  kAmaxWh = 8, kAmaxT1 = 9, kAmaxT2 = 10, kAmaxSlots = 16
};

template <class T>
int talloc(TcPath *p, T **ptr, size_t count) {
  void *q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return G1G2_ENOMEM;
  }
  p->allocs.push_back(q);
  *ptr = static_cast<T *>(q);
  return G1G2_OK;
}

// dynamic shared memory of one GEMM CTA; acc64_bytes > 0 adds the FP64 split-K accumulator.
// TF32 form: up to 4 stages.  Sliced form: 2 or 3 MMA stages and as many FP32 A slots
// (2..6) as the rest of the budget holds.
size_t gemm_smem(bool sliced, int nout, int *stages, int *fstages, size_t acc64_bytes = 0) {
  const size_t stage = stage_bytes_for(sliced, nout);
  const size_t budget = 224 * 1024 - acc64_bytes;
  if (sliced) {
    // a third MMA stage (more lookahead for the B loads) where it fits beside two FP32 slots
    *stages = (3 * stage + 2 * (size_t)kABytes <= budget) ? 3 : 2;
    *fstages = (int)std::max<size_t>(2, std::min<size_t>(6, (budget - std::min(budget, *stages * stage)) / kABytes));
    return 1024 + *stages * stage + (size_t)*fstages * kABytes + 256 + acc64_bytes;
  }
  int s = (int)std::min<size_t>(4, budget / stage);
  if (s < 2) s = 2;
  *stages = s;
  *fstages = 0;
  return 1024 + s * stage + 256 + acc64_bytes;
}

// The sliced passes with output tiles wider than 128 columns (nb > 64) whose rows are
// linear or gathered run on tc_gemm_ts_kernel (A slices in tensor memory).
bool use_ts_gemm(const GemmParams &g) {
  return g.nout > 128 && g.nout <= 192 && !g.kb_chunks && (g.a_rows == AR_LINEAR || g.a_rows == AR_GATHER4);
}

// The sliced collision integral (split-K over nb^3, N = nb <= 96) runs on tc_collision_ts_kernel.
bool use_collision_ts(const GemmParams &g) { return g.a_rows == AR_SPLITK && g.kb_chunks && g.nout <= 96; }

// sliced: the BF16-slice form (Bh = slices of B, Bl unused); otherwise TF32 hi/lo
void launch_gemm(TcPath *t, Launcher &L, const char *tag, const CUtensorMap &A, const CUtensorMap &Bh,
                 const CUtensorMap &Bl, GemmParams gp, bool sliced = false) {
  gp.err = t->err;
  int stages = 0, fstages = 0;
  // the region after the barriers: split-K partial pairs, or the staging of the transposed epilogue
  const size_t acc64 = gp.kb_chunks ? (size_t)gp.nb * (gp.n_valid + 1) * sizeof(float2)
                                    : ((sliced && epi_transposed(gp)) ? kStgAll : 0);
  const size_t smem = gemm_smem(sliced, gp.nout, &stages, &fstages, acc64);
  const int grid = std::max(1, std::min(gp.tiles, t->sms));
  L.before(tag);
  if (sliced && use_ts_gemm(gp)) {
    tc_gemm_ts_kernel<<<grid, kTsThreads, ts_smem_bytes(gp.nout), L.stream>>>(A, Bh, gp);
  } else if (sliced && use_collision_ts(gp)) {
    tc_collision_ts_kernel<<<grid, kTsThreads, ct_smem_bytes(gp.nout, ct_acc_bytes(gp.nb, gp.n_valid)), L.stream>>>(
        A, Bh, gp);
  } else if (sliced) {
    tc_gemm_kernel<true><<<grid, kGemmThreads, smem, L.stream>>>(A, Bh, Bl, gp, stages, fstages);
  } else {
    tc_gemm_kernel<false><<<grid, kGemmThreads, smem, L.stream>>>(A, Bh, Bl, gp, stages, fstages);
  }
  L.after_launch();
}

GemmParams linear_params(const TcPath *t, long long rows, int planes, int epi, float *out) {
  GemmParams g{};
  g.nb = t->nb;
  g.a_rows = AR_LINEAR;
  g.epi = epi;
  g.rows = rows;
  g.tiles = (int)((rows + kTileM - 1) / kTileM);
  g.kb_per_plane = t->kpad / kBlockK;
  g.a_planes = planes;
  g.nout = t->nout2;
  g.n_valid = 2 * t->nb;
  g.out = out;
  g.out_plane = t->N4;
  return g;
}

}  // namespace

int tc_create(TcPath **out, int nb, int se, bool restricted, bool sliced, bool bosons, const cplx *hw, const cplx *hsrc,
              cudaStream_t stream) {
  *out = nullptr;
  if (nb % 4 != 0) {
    set_error_detail("the tensor-core form needs nb divisible by 4 (TMA row pitch)");
    return G1G2_EUNSUPPORTED;
  }
  const bool has_pi = se == G1G2_GW || se == G1G2_DSL, has_pp = se == G1G2_TPP || se == G1G2_DSL,
             has_ph = se == G1G2_TPH || se == G1G2_DSL;
  if ((has_pp || has_ph) && !sliced) {
    set_error_detail("the tensor-core ladder product runs in the BF16-slice form");
    return G1G2_EUNSUPPORTED;
  }
  const bool big = has_pi || has_pp || has_ph;  // an nb^2 x nb^2 x nb^2 product (polarisation or ladder)
  const long long N = nb, N4 = N * N * N * N;
  for (long long e = 0; e < N4; ++e)
    if (hw[e].y != 0.0) {
      set_error_detail("the tensor-core form takes a real interaction w");
      return G1G2_EUNSUPPORTED;
    }
  TcPath *t = new TcPath;
  t->nb = nb;
  t->se = se;
  t->restricted = restricted;
  t->sliced = sliced;
  t->has_pi = has_pi;
  t->eta = bosons ? 1.0 : -1.0;
  t->has_pp = has_pp;
  t->has_ph = has_ph;
  t->N4 = N4;
  t->kpad = round_up(nb, kBlockK);
  t->nout2 = round_up(2 * nb, 16);
  t->nout1 = round_up(nb, 16);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, dev);
  int rc = G1G2_OK;
  auto bail = [&](int code) {
    tc_destroy(t);
    return code;
  };
  const int kt_c = 2 * t->kpad, kt_r = t->kpad;
  if ((rc = talloc(t, &t->y32, 2 * N4)) || (rc = talloc(t, &t->ys32, 2 * N4)) || (rc = talloc(t, &t->acc, 2 * N4)) ||
      (rc = talloc(t, &t->Z, 2 * N4)) || (rc = talloc(t, &t->buf1, 2 * N4)) || (rc = talloc(t, &t->buf2, 2 * N4)) ||
      (rc = talloc(t, &t->W32, N4)) || (rc = talloc(t, &t->w_hi, N4)) || (rc = talloc(t, &t->w_lo, N4)) ||
      (rc = talloc(t, &t->bh_hi, (size_t)t->nout2 * 2 * kt_c)) ||
      (rc = talloc(t, &t->bh_lo, (size_t)t->nout2 * 2 * kt_c)) ||
      (rc = talloc(t, &t->bnr_hi, (size_t)t->nout2 * kt_r)) || (rc = talloc(t, &t->bnr_lo, (size_t)t->nout2 * kt_r)) ||
      (rc = talloc(t, &t->bnc_hi, (size_t)t->nout2 * kt_c)) || (rc = talloc(t, &t->bnc_lo, (size_t)t->nout2 * kt_c)) ||
      (rc = talloc(t, &t->bnb_hi, (size_t)t->nout2 * kt_c)) || (rc = talloc(t, &t->bnb_lo, (size_t)t->nout2 * kt_c)) ||
      (rc = talloc(t, &t->nbar, N * N)) || (rc = talloc(t, &t->I, N * N)) || (rc = talloc(t, &t->err, 1)))
    return bail(rc);
  if (sliced) {
    const size_t bs_c = (size_t)kSlices * t->nout2 * kt_c, bs_r = (size_t)kSlices * t->nout2 * kt_r;
    if ((rc = talloc(t, &t->bh_s, bs_c)) || (rc = talloc(t, &t->bnr_s, bs_r)) || (rc = talloc(t, &t->bnc_s, bs_c)) ||
        (rc = talloc(t, &t->bnb_s, bs_c)) || (rc = talloc(t, &t->bnt_s, bs_r)) ||
        (rc = talloc(t, &t->w_s, (size_t)kSlices * N4)) || (rc = talloc(t, &t->amax, kAmaxSlots)))
      return bail(rc);
    if (cudaMemset(t->amax, 0, kAmaxSlots * sizeof(int)) != cudaSuccess) return bail(G1G2_ECUDA);
  }
  if (big) {
    const long long ncol = 2 * N * N;  // output columns (j, l, v)
    // TF32 form: the tc_gemm_kernel geometry of the polarisation (column tiles of up to 256)
    t->pi_nout = (int)std::min<long long>(256, ((ncol + 15) / 16) * 16);
    t->pi_ntiles = (int)((ncol + t->pi_nout - 1) / t->pi_nout);
    t->pi_mtiles = ((nb + 3) / 4) * ((nb + 31) / 32);
    t->pi_ldb = 2 * N * t->kpad;
    const size_t brows = (size_t)t->pi_ntiles * t->pi_nout;
    if ((rc = talloc(t, &t->Y1, 2 * N4)) || (rc = talloc(t, &t->Y2, 2 * N4)) || (rc = talloc(t, &t->Pi, 2 * N4)) ||
        (rc = talloc(t, &t->bnt_hi, (size_t)t->nout2 * kt_r)) || (rc = talloc(t, &t->bnt_lo, (size_t)t->nout2 * kt_r)))
      return bail(rc);
    if (!sliced) {
      if ((rc = talloc(t, &t->bpi_hi, brows * t->pi_ldb)) || (rc = talloc(t, &t->bpi_lo, brows * t->pi_ldb)))
        return bail(rc);
      if (cudaMemset(t->bpi_hi, 0, brows * t->pi_ldb * sizeof(float)) != cudaSuccess ||
          cudaMemset(t->bpi_lo, 0, brows * t->pi_ldb * sizeof(float)) != cudaSuccess)
        return bail(G1G2_ECUDA);
    } else {
      const size_t K = 2 * (size_t)N * N;
      if ((rc = talloc(t, &t->pa_s, (size_t)kPiSlices * N * N * K)) ||
          (rc = talloc(t, &t->pb_s, (size_t)kPiSlices * K * K)) || (rc = talloc(t, &t->rowmax, (size_t)N * N)) ||
          (rc = talloc(t, &t->colmax, (size_t)N * N)))
        return bail(rc);
    }
    if (has_pp || has_ph) {
      const size_t bs_c = (size_t)kSlices * t->nout2 * kt_c, bs_r = (size_t)kSlices * t->nout2 * kt_r;
      if ((rc = talloc(t, &t->bnbr_s, bs_r)) || (rc = talloc(t, &t->bnbc_s, bs_c)) ||
          (rc = talloc(t, &t->bnbt_s, bs_r)))
        return bail(rc);
      t->Lam = t->Pi;
      if (has_pi && (rc = talloc(t, &t->Lam, 2 * N4))) return bail(rc);
    }
    if (has_ph && (rc = talloc(t, &t->Wp32, N4))) return bail(rc);
  }
  // collision split-K geometry: K = nb^3 floats, both planes
  t->kb_all_coll = (int)((N * N * N + kBlockK - 1) / kBlockK);
  t->splits = std::max(1, std::min(t->kb_all_coll, t->sms));
  t->kb_per_split = (t->kb_all_coll + t->splits - 1) / t->splits;
  t->splits = (t->kb_all_coll + t->kb_per_split - 1) / t->kb_per_split;
  if ((rc = talloc(t, &t->partial, (size_t)t->splits * 2 * N * N))) return bail(rc);
  // canonical blocks of the assembly orbits
  {
    const int nB = (nb + BSZ - 1) / BSZ;
    std::vector<int4> blk;
    for (int a = 0; a < nB; ++a)
      for (int b = 0; b < nB; ++b)
        for (int c = 0; c < nB; ++c)
          for (int d = 0; d < nB; ++d) {
            const int m[4][4] = {{a, b, c, d}, {b, a, d, c}, {c, d, a, b}, {d, c, b, a}};
            bool canon = true;
            for (int q = 1; q < 4 && canon; ++q) {
              for (int z = 0; z < 4; ++z) {
                if (m[q][z] < m[0][z]) { canon = false; break; }
                if (m[q][z] > m[0][z]) break;
              }
            }
            if (canon) blk.push_back(make_int4(a, b, c, d));
          }
    // CTA order: the orbits of the 4^4 blocks that make up one orbit of 16^4 blocks (at most
    // 256 of them) run one after another.  The state copy and the stage input are planar
    // FP32 in natural order, so a 4^4 block covers 16 bytes of each 64-byte DRAM access
    // along the last index; the other 48 bytes lie in the neighbouring 4^4 blocks of the
    // same 16^4 block, which belong to these orbits for every member of the orbit.  Run
    // together (well within the CTAs resident at one time), they meet in L2 instead of
    // reaching HBM once each.
    auto orbit_key = [](int a, int b, int c, int d, long long K) {
      const int m[4][4] = {{a, b, c, d}, {b, a, d, c}, {c, d, a, b}, {d, c, b, a}};
      long long best = -1;
      for (int q = 0; q < 4; ++q) {
        const long long k = ((m[q][0] * K + m[q][1]) * K + m[q][2]) * K + m[q][3];
        if (best < 0 || k < best) best = k;
      }
      return best;
    };
    const long long K16 = (nB + 3) / 4;
    std::stable_sort(blk.begin(), blk.end(), [&](const int4 &x, const int4 &y) {
      return orbit_key(x.x >> 2, x.y >> 2, x.z >> 2, x.w >> 2, K16) <
             orbit_key(y.x >> 2, y.y >> 2, y.z >> 2, y.w >> 2, K16);
    });
    t->nblocks = (int)blk.size();
    if ((rc = talloc(t, &t->blocks, blk.size()))) return bail(rc);
    if (cudaMemcpy(t->blocks, blk.data(), blk.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(G1G2_ECUDA);
  }
  // fixed operands: W32 = source interaction (real), w hi/lo for the collision integral;
  // GW with a w^- source (exchange) also needs plain w for the quasi-Hamiltonian (Wh32)
  {
    std::vector<float> w32(N4);
    bool src_is_w = true;
    for (long long e = 0; e < N4; ++e) {
      w32[e] = (float)hsrc[e].x;
      if (hsrc[e].x != hw[e].x) src_is_w = false;
    }
    if (cudaMemcpy(t->W32, w32.data(), N4 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(G1G2_ECUDA);
    t->Wh32 = t->W32;
    if (big && !src_is_w) {
      std::vector<float> wh(N4);
      float hmax = 0.f;
      for (long long e = 0; e < N4; ++e) {
        wh[e] = (float)hw[e].x;
        hmax = std::max(hmax, std::fabs(wh[e]));
      }
      if ((rc = talloc(t, &t->Wh32, N4))) return bail(rc);
      if (cudaMemcpy(t->Wh32, wh.data(), N4 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(G1G2_ECUDA);
      if (sliced) {
        int bits = 0;
        std::memcpy(&bits, &hmax, sizeof(bits));
        cudaMemcpy(t->amax + kAmaxWh, &bits, sizeof(int), cudaMemcpyHostToDevice);
      }
    }
    if (has_ph) {  // Wp32[p][q][r][s] = w_rpqs: the particle-hole quasi-Hamiltonian as right multiplications
      std::vector<float> wp(N4);
      for (long long r = 0; r < N; ++r)
        for (long long p = 0; p < N; ++p)
          for (long long q = 0; q < N; ++q)
            for (long long u = 0; u < N; ++u)
              wp[((p * N + q) * N + r) * N + u] = (float)hw[((r * N + p) * N + q) * N + u].x;
      if (cudaMemcpy(t->Wp32, wp.data(), N4 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(G1G2_ECUDA);
      if (sliced && t->Wh32 == t->W32) {  // the slot of plain w must hold max|w|
        float hmax = 0.f;
        for (long long e = 0; e < N4; ++e) hmax = std::max(hmax, std::fabs(wp[e]));
        int bits = 0;
        std::memcpy(&bits, &hmax, sizeof(bits));
        cudaMemcpy(t->amax + kAmaxWh, &bits, sizeof(int), cudaMemcpyHostToDevice);
      }
    }
    cplx *wd = nullptr;
    if (cudaMalloc(&wd, N4 * sizeof(cplx)) != cudaSuccess) return bail(G1G2_ENOMEM);
    cudaMemcpy(wd, hw, N4 * sizeof(cplx), cudaMemcpyHostToDevice);
    split_real_kernel<<<1024, 256, 0, stream>>>(N4, wd, t->w_hi, t->w_lo);
    if (sliced) {
      double wmax = 0.0;
      float smax = 0.f;
      for (long long e = 0; e < N4; ++e) {
        wmax = std::max(wmax, std::fabs(hw[e].x));
        smax = std::max(smax, std::fabs(w32[e]));
      }
      int E = 0;
      if (wmax > 0.0) std::frexp(wmax, &E);
      slice_w_kernel<<<1024, 256, 0, stream>>>(N4, wd, E, t->w_s);
      int bits = 0;
      std::memcpy(&bits, &smax, sizeof(bits));
      cudaMemcpy(t->amax + kAmaxW, &bits, sizeof(int), cudaMemcpyHostToDevice);
    }
    cudaStreamSynchronize(stream);
    cudaFree(wd);
    if (cudaGetLastError() != cudaSuccess) return bail(G1G2_ECUDA);
  }
  if (cudaMemset(t->err, 0, sizeof(int)) != cudaSuccess) return bail(G1G2_ECUDA);
  // tensor maps
  const long long N3 = N * N * N;
  // B boxes of the 2 nb-column passes: the whole output, or one sub-tile of the TMEM-A kernel
  const int bbox = (sliced && t->nout2 > 128) ? ts_nt(t->nout2) : t->nout2;
  if ((rc = map_linear(&t->mZin_y32, t->y32, nb, N3, 2)) || (rc = map_linear(&t->mZin_ys32, t->ys32, nb, N3, 2)) ||
      (rc = map_linear(&t->mCol_y32, t->y32, (int)N3, N, 2)) ||
      (rc = map_linear(&t->mCol_ys32, t->ys32, (int)N3, N, 2)) || (rc = map_linear(&t->mW32, t->W32, nb, N3, 1)) ||
      (rc = map_linear(&t->mWh32, t->Wh32, nb, N3, 1)) ||
      (rc = map_gather(&t->mBuf1Gather, t->buf1, nb)) || (rc = map_linear(&t->mBuf2Lin, t->buf2, nb, N3, 2)) ||
      (rc = map_linear(&t->mBuf1Lin, t->buf1, nb, N3, 2)) ||
      (rc = map_b(&t->mBh_hi, t->bh_hi, kt_c, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBh_lo, t->bh_lo, kt_c, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBnr_hi, t->bnr_hi, kt_r, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBnr_lo, t->bnr_lo, kt_r, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBnc_hi, t->bnc_hi, kt_c, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBnc_lo, t->bnc_lo, kt_c, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBnb_hi, t->bnb_hi, kt_c, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mBnb_lo, t->bnb_lo, kt_c, t->nout2, t->nout2)) ||
      (rc = map_b(&t->mW_hi, t->w_hi, (int)N3, nb, t->nout1)) ||
      (rc = map_b(&t->mW_lo, t->w_lo, (int)N3, nb, t->nout1)) ||
      (big &&
       ((rc = map_b(&t->mBnt_hi, t->bnt_hi, kt_r, t->nout2, t->nout2)) ||
        (rc = map_b(&t->mBnt_lo, t->bnt_lo, kt_r, t->nout2, t->nout2)))) ||
      (big && !sliced &&
       ((rc = map_gather(&t->mPi_y32, t->y32, nb, 32, 1, 4)) || (rc = map_gather(&t->mPi_ys32, t->ys32, nb, 32, 1, 4)) ||
        (rc = map_b(&t->mBpi_hi, t->bpi_hi, (int)t->pi_ldb, t->pi_ntiles * t->pi_nout, t->pi_nout)) ||
        (rc = map_b(&t->mBpi_lo, t->bpi_lo, (int)t->pi_ldb, t->pi_ntiles * t->pi_nout, t->pi_nout)))) ||
      (sliced && ((rc = map_bs(&t->mBh_s, t->bh_s, kt_c, t->nout2, bbox)) ||
                  (rc = map_bs(&t->mBnr_s, t->bnr_s, kt_r, t->nout2, bbox)) ||
                  (rc = map_bs(&t->mBnc_s, t->bnc_s, kt_c, t->nout2, bbox)) ||
                  (rc = map_bs(&t->mBnb_s, t->bnb_s, kt_c, t->nout2, bbox)) ||
                  (rc = map_bs(&t->mBnt_s, t->bnt_s, kt_r, t->nout2, bbox)) ||
                  (rc = map_bs(&t->mW_s, t->w_s, N3, nb, t->nout1)) ||
                  (big &&
                   ((rc = map_bs(&t->mPa_s, t->pa_s, 2 * N * N, (int)(N * N), kPiTileM, kPiSlices, kPiSlices)) ||
                    (rc = map_bs(&t->mPb_s, t->pb_s, 2 * N * N, (int)(2 * N * N), kPiTileN, kPiSlices,
                                 kPiSlices)))) ||
                  ((has_pp || has_ph) &&
                   ((rc = map_bs(&t->mBnbr_s, t->bnbr_s, kt_r, t->nout2, bbox)) ||
                    (rc = map_bs(&t->mBnbc_s, t->bnbc_s, kt_c, t->nout2, bbox)) ||
                    (rc = map_bs(&t->mBnbt_s, t->bnbt_s, kt_r, t->nout2, bbox)))) ||
                  (has_ph && (rc = map_linear(&t->mWp32, t->Wp32, nb, N3, 1)))))) {
    set_error_detail("cuTensorMapEncodeTiled failed");
    return bail(rc);
  }
  int st = 0, fst = 0;
  const size_t acc64 = (size_t)nb * (nb + 1) * sizeof(float2);
  size_t smax = std::max(gemm_smem(sliced, t->nout2, &st, &fst, sliced ? kStgAll : 0),
                         gemm_smem(sliced, t->nout1, &st, &fst, acc64));
  if (big && !sliced) smax = std::max(smax, gemm_smem(sliced, t->pi_nout, &st, &fst));
  if (smax > 227 * 1024) {
    set_error_detail("basis too large for the FP64 split-K accumulator of the tensor-core collision integral");
    return bail(G1G2_EUNSUPPORTED);
  }
  // The limit is a property of the kernel, shared by every context of the process:
  // set it to the device maximum so that no context lowers it under another one.
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  auto raise_limit = [&](const void *fn, size_t need) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return false;
    const int dyn = optin - (int)fa.sharedSizeBytes;  // static shared memory counts against the same limit
    return dyn >= (int)need && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess;
  };
  if (!raise_limit((const void *)tc_gemm_kernel<false>, smax) || !raise_limit((const void *)tc_gemm_kernel<true>, smax) ||
      !raise_limit((const void *)orbit_assemble_kernel<kAsmK>, 4 * BEL * sizeof(float2)) ||
      !raise_limit((const void *)orbit_assemble_kernel<kAsmStage>, 4 * BEL * sizeof(float2)) ||
      !raise_limit((const void *)orbit_assemble_kernel<kAsmLast>, 4 * BEL * sizeof(float2)) ||
      (big && sliced && !raise_limit((const void *)tc_pi_gemm_kernel, kPiSmemBytes)) ||
      (has_pi && sliced && !raise_limit((const void *)realify_pi_slice3_kernel, (size_t)nb * nb * sizeof(float2))) ||
      (sliced && t->nout2 > 128 && !raise_limit((const void *)tc_gemm_ts_kernel, ts_smem_bytes(t->nout2))) ||
      (sliced && t->nout1 <= 96 &&
       !raise_limit((const void *)tc_collision_ts_kernel, ct_smem_bytes(t->nout1, ct_acc_bytes(nb, nb))))) {
    cudaGetLastError();
    set_error_detail("cannot raise the shared-memory limit of the tensor-core kernels");
    return bail(G1G2_ECUDA);
  }
  *out = t;
  return G1G2_OK;
}

void tc_destroy(TcPath *p) {
  if (!p) return;
  for (void *q : p->allocs) cudaFree(q);
  delete p;
}

namespace {
// One CTA waits on an mbarrier that nothing arrives on: the bounded wait must
// give up after limit_ns, set the error word and let the kernel return.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, err, limit_ns);
  __syncthreads();
}
}  // namespace

int tc_wait_selftest(unsigned long long limit_ns, cudaStream_t stream) {
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return G1G2_ENOMEM;
  }
  int e = 0, rc = G1G2_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) rc = G1G2_ECUDA;
  if (!rc) {
    wait_selftest_kernel<<<1, 32, 0, stream>>>(limit_ns, err);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      rc = G1G2_ECUDA;
  }
  cudaFree(err);
  if (rc) return rc;
  if (e) {
    set_error_detail("self-test: the bounded barrier wait gave up as intended");
    return G1G2_ETIMEOUT;
  }
  return G1G2_OK;
}

int tc_error(TcPath *p, cudaStream_t stream) {
  int e = 0;
  if (cudaMemcpyAsync(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return G1G2_ECUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return G1G2_ECUDA;
  if (e) {
    set_error_detail("a tensor-core kernel gave up waiting on a barrier");
    return G1G2_ETIMEOUT;
  }
  return G1G2_OK;
}

void tc_load_state(TcPath *p, Launcher &L, const cplx *G) {
  int *slot = p->sliced ? p->amax + kAmaxY : nullptr;
  if (slot) cudaMemsetAsync(slot, 0, sizeof(int), L.stream);
  L.before("tc_to_planar");
  to_planar_f32_kernel<<<2048, 256, 0, L.stream>>>(p->N4, G, p->y32, slot);
  L.after_launch();
}

namespace {
// out = A B^T for one nb^2 x nb^2 x nb^2 product of the sliced form: the A operand read from
// the planar FP32 state G32 through m, its per-row maxima and three BF16 slices, then
// tc_pi_gemm_kernel against the B slices already in pb_s (out in the layout
// out[a][c][d][b], complex; in 4^4 blocks with out_blk).
void sliced_product(TcPath *t, Launcher &L, const float *G32, AOperand m, float *out, const char *tag,
                    bool out_blk = false) {
  const int nb = t->nb;
  const long long N = nb, K = 2 * N * N;
  const int nbt = (nb + 31) / 32;
  cudaMemsetAsync(t->rowmax, 0, N * N * sizeof(int), L.stream);
  L.before("tc_product_a_rowmax");
  a_rowmax_kernel<<<dim3((unsigned)(nb * nbt), (unsigned)(2 * ((nb + 7) / 8))), dim3(32, 8), 0, L.stream>>>(
      nb, G32, t->N4, m, t->rowmax);
  L.after_launch();
  L.before("tc_product_a_slices");
  a_slice3_kernel<<<dim3((unsigned)(nb * nbt), (unsigned)(2 * nb)), dim3(32, 8), 0, L.stream>>>(
      nb, G32, t->N4, m, t->rowmax, t->pa_s, N * N * K);
  L.after_launch();
  PiGemmParams g{};
  g.nb = nb;
  g.M = nb * nb;
  g.ncols = 2 * nb * nb;
  g.kblocks = (int)(K / kPiBlockK);
  g.mtiles = (g.M + kPiTileM - 1) / kPiTileM;
  g.tiles = g.mtiles * ((g.ncols + kPiTileN - 1) / kPiTileN);
  g.out = reinterpret_cast<float2 *>(out);
  g.out_blk = out_blk ? 1 : 0;
  g.err = t->err;
  const int grid = std::max(1, std::min(g.tiles, t->sms));
  L.before(tag);
  tc_pi_gemm_kernel<<<grid, kPiThreads, kPiSmemBytes, L.stream>>>(t->mPa_s, t->mPb_s, g);
  L.after_launch();
}
}  // namespace

void tc_rhs(TcPath *t, Launcher &L, const cplx *n_in, const cplx *G_in, const cplx *hhf, Rk4Stage st, cplx *ny,
            cplx *nys, cplx *nacc, cplx *nk, cplx *Gy, cplx *Gys, cplx *Gacc, cplx *Gk) {
  (void)Gys;
  (void)Gacc;
  const int nb = t->nb;
  const long long N = nb, N3 = N * N * N;
  // stage input of G2 in FP32 planar
  const bool from_y = (st.stage == 0);
  const bool sl = t->sliced;
  int *const amax = t->amax;
  if (st.stage < 0) {
    if (sl) cudaMemsetAsync(amax + kAmaxYs, 0, sizeof(int), L.stream);
    L.before("tc_to_planar");
    to_planar_f32_kernel<<<2048, 256, 0, L.stream>>>(t->N4, G_in, t->ys32, sl ? amax + kAmaxYs : nullptr);
    L.after_launch();
  }
  const CUtensorMap &mZin = from_y ? t->mZin_y32 : t->mZin_ys32;
  const CUtensorMap &mCol = from_y ? t->mCol_y32 : t->mCol_ys32;
  const int *g2_amax = sl ? amax + (from_y ? kAmaxY : kAmaxYs) : nullptr;
  if (sl) cudaMemsetAsync(amax + kAmaxP1, 0, 3 * sizeof(int), L.stream);  // this call's source-term passes
  // small operands
  one_pm(L, nb, n_in, t->eta, t->nbar);
  if (sl) {
    const int kc = 2 * t->kpad;
    struct { const cplx *S; int complex_a, shift, ld, transpose, il; __nv_bfloat16 *out; } ops[8] = {
        {hhf, 1, 1, kc, 0, 1, t->bh_s},
        {n_in, 0, 0, t->kpad, 0, 0, t->bnr_s},
        {n_in, 1, 0, kc, 0, 0, t->bnc_s},
        {t->nbar, 1, 0, kc, 0, 1, t->bnb_s},
        {n_in, 0, 0, t->kpad, 1, 0, t->bnt_s},       // GW: n^T
        {t->nbar, 0, 0, t->kpad, 0, 0, t->bnbr_s},   // ladder: nbar, real A
        {t->nbar, 1, 0, kc, 0, 0, t->bnbc_s},        // ladder: nbar, complex A
        {t->nbar, 0, 0, t->kpad, 1, 0, t->bnbt_s}};  // particle-hole ladder: nbar^T, real A
    int sel[8] = {0, 1, 2, 3, 0, 0, 0, 0}, nops = 4;
    if (t->has_pi || t->has_ph) sel[nops++] = 4;
    if (t->has_pp) sel[nops++] = 5;
    if (t->has_pp || t->has_ph) sel[nops++] = 6;
    if (t->has_ph) sel[nops++] = 7;
    SliceBBatch batch{};
    for (int qi = 0; qi < nops; ++qi) {
      const auto &o = ops[sel[qi]];
      batch.op[qi] = SliceBOp{o.S, o.out, (long long)t->nout2 * o.ld, o.complex_a, o.shift, o.ld, o.transpose, o.il};
    }
    L.before("tc_slice_b");
    slice_b_kernel<<<dim3(64, (unsigned)nops), 256, 0, L.stream>>>(nb, t->nout2, t->kpad, batch);
    L.after_launch();
  }
  {
    const int kc = 2 * t->kpad;
    struct { const cplx *S; int complex_a, shift; double scale; int ld, col0, transpose, il; float *hi, *lo; } ops[5] = {
        {hhf, 1, 1, 1.0, kc, 0, 0, 1, t->bh_hi, t->bh_lo},
        {n_in, 0, 0, 1.0, t->kpad, 0, 0, 0, t->bnr_hi, t->bnr_lo},
        {n_in, 1, 0, 1.0, kc, 0, 0, 0, t->bnc_hi, t->bnc_lo},
        {t->nbar, 1, 0, 1.0, kc, 0, 0, 1, t->bnb_hi, t->bnb_lo},
        {n_in, 0, 0, 1.0, t->kpad, 0, 1, 0, t->bnt_hi, t->bnt_lo}};
    const int nops = sl ? 0 : t->has_pi ? 5 : 4;  // the sliced form slices these above
    for (int q = 0; q < nops; ++q) {
      const auto &o = ops[q];
      L.before("tc_realify");
      realify_kernel<<<64, 256, 0, L.stream>>>(nb, t->nout2, t->kpad, o.complex_a, o.shift, o.scale, o.ld, o.col0,
                                               o.transpose, o.il, o.S, o.hi, o.lo);
      L.after_launch();
    }
  }
  // a2: collision integral, split-K over c = (k,l,p)
  {
    GemmParams g{};
    g.nb = nb;
    g.a_rows = AR_SPLITK;
    g.epi = EP_PARTIAL;
    g.splits = t->splits;
    g.kb_per_split = t->kb_per_split;
    g.kb_all = t->kb_all_coll;
    g.tiles = 2 * t->splits;
    g.kb_per_plane = t->kb_per_split;
    g.a_planes = 1;
    g.nout = t->nout1;
    g.n_valid = nb;
    g.kb_chunks = 4;
    g.out64 = t->partial;
    g.a_amax = g2_amax;
    launch_gemm(t, L, "tc_gemm_collision", mCol, sl ? t->mW_s : t->mW_hi, t->mW_lo, g, sl);
    L.before("tc_collision_reduce");
    collision_reduce_kernel<<<(nb * nb + 31) / 32, dim3(32, 8), 0, L.stream>>>(nb, t->splits, t->partial, t->I);
    L.after_launch();
  }
  g1_update(L, nb, hhf, n_in, t->I, st, ny, nys, nacc, nk);
  // a4: the source-term chain
  // sliced-form A scales and output maxima of each pass
  auto lp = [&](long long rows, int planes, int epi, float *out, int a_slot, int out_slot) {
    GemmParams g = linear_params(t, rows, planes, epi, out);
    if (sl) {
      g.a_amax = a_slot >= 0 ? amax + a_slot : g2_amax;
      g.out_amax = out_slot >= 0 ? amax + out_slot : nullptr;
    }
    return g;
  };
  launch_gemm(t, L, "tc_gemm_psi1", t->mW32, sl ? t->mBnr_s : t->mBnr_hi, t->mBnr_lo,
              lp(N3, 1, EP_EXCH_T, t->buf1, kAmaxW, kAmaxP1), sl);
  {
    GemmParams g = lp(N3, 2, EP_GATHER_TCONJ, t->buf2, kAmaxP1, kAmaxP2);
    g.a_rows = AR_GATHER4;
    g.g_na = (nb + 3) / 4;
    g.g_nb = (nb + 31) / 32;
    g.tiles = nb * g.g_na * g.g_nb;
    launch_gemm(t, L, "tc_gemm_psi2", t->mBuf1Gather, sl ? t->mBnc_s : t->mBnc_hi, t->mBnc_lo, g, sl);
  }
  // B = nbar and B = hHF have interleaved rows (col_il); the passes feeding the
  // assembly store interleaved complex FP32 (out_il)
  auto il = [](GemmParams g, bool out_il) {
    g.col_il = 1;
    g.out_il = out_il ? 1 : 0;
    g.out_blk = out_il ? 1 : 0;   // the assembly's inputs Z and Q: 4^4 blocks
    return g;
  };
  launch_gemm(t, L, "tc_gemm_psi3", t->mBuf2Lin, sl ? t->mBnb_s : t->mBnb_hi, t->mBnb_lo,
              il(lp(N3, 2, EP_EXCH_T, t->buf1, kAmaxP2, kAmaxP3), false), sl);
  // a3: Z = G2 x_4 (hHF - mu); last a4 pass: Q = T2~ x_4 nbar = A^dag (both in the swapped layout)
  launch_gemm(t, L, "tc_gemm_commutator", mZin, sl ? t->mBh_s : t->mBh_hi, t->mBh_lo,
              il(lp(N3, 2, EP_SWAP34, t->Z, -1, -1), true), sl);
  launch_gemm(t, L, "tc_gemm_psi4", t->mBuf1Lin, sl ? t->mBnb_s : t->mBnb_hi, t->mBnb_lo,
              il(lp(N3, 2, EP_SWAP34, t->buf2, kAmaxP3, -1), true), sl);
  if (t->has_pi) {
    // a5: Y1 = w x_4 n, Y2 = w x_4 n^T (hcorr_ijkl = Y1_ijkl - Y2_klij), swapped layout
    if (sl) cudaMemsetAsync(amax + kAmaxH1, 0, 2 * sizeof(int), L.stream);
    const int wh_slot = (t->Wh32 == t->W32) ? kAmaxW : kAmaxWh;
    launch_gemm(t, L, "tc_gemm_hcorr", t->mWh32, sl ? t->mBnr_s : t->mBnr_hi, t->mBnr_lo,
                lp(N3, 1, EP_SWAP34, t->Y1, wh_slot, kAmaxH1), sl);
    launch_gemm(t, L, "tc_gemm_hcorr", t->mWh32, sl ? t->mBnt_s : t->mBnt_hi, t->mBnt_lo,
                lp(N3, 1, EP_SWAP34, t->Y2, wh_slot, kAmaxH2), sl);
    if (sl) {
      // B = R(hcorr) as three BF16 slices with per-column exponents, then the product
      L.before("tc_pi_b_slices");
      realify_pi_slice3_kernel<<<(unsigned)(N * N), 256, N * N * sizeof(float2), L.stream>>>(
          nb, t->Y1, t->Y2, t->N4, t->pb_s, 4 * N * N * N * N);
      L.after_launch();
      // a6: Pi_(ik),(jl) = sum_(pq) G_ipkq hcorr_qjpl, rows (i, k) of G_ipkq
      sliced_product(t, L, from_y ? t->y32 : t->ys32, AOperand{N * N * N, N, N * N, 1}, t->Pi, "tc_gemm_pi",
                     true);
    } else {
      const dim3 pgrid((unsigned)(((nb + 31) / 32) * (t->kpad / 32)), (unsigned)(N * N));
      L.before("tc_realify_pi");
      realify_pi_kernel<<<pgrid, dim3(32, 8), 0, L.stream>>>(nb, t->kpad, t->Y1, t->Y2, t->N4, t->bpi_hi,
                                                             t->bpi_lo, t->pi_ldb);
      L.after_launch();
      // a6: Pi_(ik),(jl) = sum_(pq) G_ipkq hcorr_qjpl, one GEMM with M = N' = K = nb^2
      GemmParams g{};
      g.nb = nb;
      g.a_rows = AR_PI;
      g.epi = EP_PI;
      g.n_tiles = t->pi_ntiles;
      g.pi_mk = (nb + 31) / 32;
      g.pi_kq = t->kpad / kBlockK;
      g.pi_mtiles = t->pi_mtiles;
      g.tiles = t->pi_mtiles * t->pi_ntiles;
      g.nout = t->pi_nout;
      g.n_valid = t->pi_nout;
      g.rows = 2 * N * N;
      g.out = t->Pi;
      g.out_plane = t->N4;
      g.out_blk = 1;
      launch_gemm(t, L, "tc_gemm_pi", from_y ? t->mPi_y32 : t->mPi_ys32, t->mBpi_hi, t->mBpi_lo, g, false);
    }
  }
  // Ladder terms (Sec. IV.D/E): H^dag as P1 - P2, each term two right multiplications of a
  // real interaction tensor Wt (x_4 S into the exchange-permuted layout, then x_4 S' again,
  // stored as [q][p][k][l] = sum_rs Wt_pqrs S'_rk S_sl in Y1, Y2), the sliced B operand, then
  // the polarisation GEMM with G2 read through a permuted copy, and the product subtracted
  // from the source-term buffer: Psi + Lambda - Lambda^dag = -(A - Lambda) + (A - Lambda)^dag.
  auto ladder = [&](const char *tag, const CUtensorMap &mWt, int wt_slot, const CUtensorMap &B1a,
                    const CUtensorMap &B1b, const CUtensorMap &B2a, const CUtensorMap &B2b) {
    cudaMemsetAsync(amax + kAmaxH1, 0, 2 * sizeof(int), L.stream);
    cudaMemsetAsync(amax + kAmaxT1, 0, 2 * sizeof(int), L.stream);
    launch_gemm(t, L, tag, mWt, B1a, B1a, lp(N3, 1, EP_EXCH_T, t->buf1, wt_slot, kAmaxT1), sl);
    launch_gemm(t, L, tag, t->mBuf1Lin, B1b, B1b, lp(N3, 2, EP_SWAP34, t->Y1, kAmaxT1, kAmaxH1), sl);
    launch_gemm(t, L, tag, mWt, B2a, B2a, lp(N3, 1, EP_EXCH_T, t->buf1, wt_slot, kAmaxT2), sl);
    launch_gemm(t, L, tag, t->mBuf1Lin, B2b, B2b, lp(N3, 2, EP_SWAP34, t->Y2, kAmaxT2, kAmaxH2), sl);
    const dim3 lgrid((unsigned)((t->kpad / 32) * ((nb + 31) / 32)), (unsigned)(N * N));
    cudaMemsetAsync(t->colmax, 0, N * N * sizeof(int), L.stream);
    L.before("tc_ladder_b_colmax");
    ladder_colmax_kernel<<<lgrid, dim3(32, 8), 0, L.stream>>>(nb, t->Y1, t->Y2, t->N4, t->colmax);
    L.after_launch();
    L.before("tc_ladder_b_slices");
    realify_lam_slice3_kernel<<<lgrid, dim3(32, 8), 0, L.stream>>>(nb, t->Y1, t->Y2, t->N4, t->colmax, t->pb_s,
                                                                    4 * N * N * N * N);
    L.after_launch();
  };
  const float *g32 = from_y ? t->y32 : t->ys32;
  const int nt32 = (nb + 31) / 32;
  if (t->has_pp) {
    // Eq. (HTPPcorr): H^dag_pqkl = sum_rs w_pqrs (nbar_rk nbar_sl - n_rk n_sl)
    const int wh_slot = (t->Wh32 == t->W32) ? kAmaxW : kAmaxWh;
    ladder("tc_gemm_ladder_h", t->mWh32, wh_slot, t->mBnbr_s, t->mBnbc_s, t->mBnr_s, t->mBnc_s);
    // Eq. (lambdapp): Lambda^dag_(ij),(kl) = sum_(pq) G_ijpq H^dag_pqkl (rows (i, j), K (p, q))
    sliced_product(t, L, g32, AOperand{N * N * N, N * N, N, 1}, t->Lam, "tc_gemm_ladder");
    L.before("tc_ladder_into_source");
    sub_swap13_kernel<<<dim3((unsigned)(nt32 * nt32), (unsigned)(N * N)), dim3(32, 8), 0, L.stream>>>(
        nb, reinterpret_cast<const float2 *>(t->Lam), reinterpret_cast<float2 *>(t->buf2));
    L.after_launch();
  }
  if (t->has_ph) {
    // Eq. (HTPHcorr): X_(pq),(kj) = conj(hcorr_kpqj) = sum_rs w_rpqs (n_rk nbar_js - nbar_rk n_js),
    // with Wp32[p][q][r][s] = w_rpqs: S' = n, S = nbar^T, then S' = nbar, S = n^T; bosons
    // (G^< = -i n, G^> = -i (1 + n)) have the opposite sign: the two terms trade places
    if (t->eta < 0)
      ladder("tc_gemm_ladder_h", t->mWp32, kAmaxWh, t->mBnbt_s, t->mBnc_s, t->mBnt_s, t->mBnbc_s);
    else
      ladder("tc_gemm_ladder_h", t->mWp32, kAmaxWh, t->mBnt_s, t->mBnbc_s, t->mBnbt_s, t->mBnc_s);
    // Eq. (lambdaph): Lambda^dag_ijkl = sum_pq G_ipql X_(pq),(kj) (rows (i, l), K (p, q))
    sliced_product(t, L, g32, AOperand{N * N * N, 1, N * N, N}, t->Lam, "tc_gemm_ladder");
    L.before("tc_ladder_into_source");
    sub_rot_kernel<<<dim3((unsigned)(nt32 * nt32), (unsigned)(N * N)), dim3(32, 8), 0, L.stream>>>(
        nb, reinterpret_cast<const float2 *>(t->Lam), reinterpret_cast<float2 *>(t->buf2));
    L.after_launch();
  }
  // a7: orbit assembly + RK4
  AsmParams a{};
  a.nb = nb;
  a.nblk = t->nblocks;
  a.blocks = t->blocks;
  a.Z = t->Z;
  a.Q = t->buf2;
  a.Pi = t->has_pi ? t->Pi : nullptr;
  a.P = t->N4;
  a.y = Gy;
  a.acc = t->acc;
  a.ys = t->ys32;
  a.y32 = t->y32;
  a.kout = Gk;
  a.stage = st.stage;
  a.hs = (float)(st.stage == 2 ? st.dt : 0.5 * st.dt);
  a.dt6 = st.dt / 6.0;
  if (sl && st.stage >= 0) {
    // the assembly writes the next stage input (ys) or, at the last stage, the new FP32 state (y32)
    a.amax = amax + (st.stage < 3 ? kAmaxYs : kAmaxY);
    cudaMemsetAsync(a.amax, 0, sizeof(int), L.stream);
  }
  L.before("tc_orbit_assemble_rk4");
  const size_t asm_smem = 4 * BEL * sizeof(float2);
  if (st.stage < 0)
    orbit_assemble_kernel<kAsmK><<<t->nblocks, ATHREADS, asm_smem, L.stream>>>(a);
  else if (st.stage < 3)
    orbit_assemble_kernel<kAsmStage><<<t->nblocks, ATHREADS, asm_smem, L.stream>>>(a);
  else
    orbit_assemble_kernel<kAsmLast><<<t->nblocks, ATHREADS, asm_smem, L.stream>>>(a);
  L.after_launch();
}

}  // namespace g1g2
