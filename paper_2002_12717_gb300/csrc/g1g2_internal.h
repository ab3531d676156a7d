// Internal declarations of libg1g2 (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/g1g2.h"

namespace g1g2 {

using cplx = double2;  // interleaved (re, im), the layout of the ABI

// ---------------------------------------------------------------------------
// Launch bookkeeping: every kernel launch goes through one of these so that a
// failed launch is turned into G1G2_ECUDA and counted.
// ---------------------------------------------------------------------------
// Optional per-kernel timing with CUDA events on the launch stream (g1g2_profile).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec { const char *tag; int start, stop; };
  std::vector<Rec> recs;
  int record(cudaStream_t s) {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
    cudaEventRecord(pool[used], s);
    return (int)used++;
  }
  void clear() { used = 0; recs.clear(); }
  ~Profiler() { for (cudaEvent_t e : pool) cudaEventDestroy(e); }
};

struct Launcher {
  cudaStream_t stream = nullptr;
  long long *counter = nullptr;
  Profiler *prof = nullptr;
  cudaError_t err = cudaSuccess;
  const char *tag = nullptr;
  int ev_start = -1;
  void before(const char *t) {
    tag = t;
    ev_start = (prof && prof->on) ? prof->record(stream) : -1;
  }
  void after_launch() {
    if (counter) ++*counter;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    if (prof && prof->on && ev_start >= 0) {
      const int stop = prof->record(stream);
      if (stop >= 0) prof->recs.push_back({tag ? tag : "kernel", ev_start, stop});
    }
    ev_start = -1;
  }
};

// Generic strided complex FP64 GEMM, batched:
//   C_b[m][n] = alpha * sum_k opA(A_b[m][k]) * opB(B_b[k][n]) + beta * C_b[m][n]
// (reduce = false), or C[m][n] = alpha * sum_b sum_k ... + beta * C (reduce = true).
struct ZGemm {
  int M = 0, N = 0, K = 0, batch = 1;
  const cplx *A = nullptr; long long sa_b = 0, sa_m = 0, sa_k = 0;
  const cplx *B = nullptr; long long sb_b = 0, sb_k = 0, sb_n = 0;
  cplx *C = nullptr;       long long sc_b = 0, sc_m = 0, sc_n = 0;
  cplx alpha{1.0, 0.0};
  double beta = 0.0;
  bool conjA = false, conjB = false;
};
void zgemm(Launcher &L, const ZGemm &g);
void zgemm_reduce(Launcher &L, const ZGemm &g, cplx *partial, int splits);

// out(a0,a1,a2,a3) = beta*out + alpha*op(in(a_p0, a_p1, a_p2, a_p3)), op = conj if conj.
void permute4(Launcher &L, int nb, const cplx *in, cplx *out, const int p[4], cplx alpha, double beta,
              bool conj);

// hHF = h + f D + Wm * vec(n), Wm[(ij),(lk)] (real or complex), Eq. (h_HF).
void hf_build(Launcher &L, int nb, const void *Wm, bool wm_real, const cplx *h, const cplx *D, double f,
              const cplx *n, cplx *hhf);
// The same product in double-single arithmetic on the FP32 pipe (tensor-core forms, real w):
// Wds holds the real Wm as (hi, lo) FP32 pairs; nsplit is scratch of nb^2 float4.
void hf_build_ds(Launcher &L, int nb, const float2 *Wds, const cplx *h, const cplx *D, double f, const cplx *n,
                 float4 *nsplit, cplx *hhf);
// nbar = 1 + eta n: 1 - n for fermions (eta = -1), 1 + n for bosons (eta = +1)
void one_pm(Launcher &L, int nb, const cplx *n, double eta, cplx *nbar);
inline void one_minus(Launcher &L, int nb, const cplx *n, cplx *nbar) { one_pm(L, nb, n, -1.0, nbar); }

// RK4 stage bookkeeping shared by the G1 and G2 updates.
struct Rk4Stage {
  int stage = -1;      // -1: write k to kout; 0..3: classical RK4 stage
  double dt = 0.0;
};
// dn = -i[hHF, n] - (I + I^dag) (I may be null); then the RK4 update of (y, ys, acc)
// or a plain write of dn to kout.
void g1_update(Launcher &L, int nb, const cplx *hhf, const cplx *n, const cplx *I, Rk4Stage st,
               cplx *y, cplx *ys, cplx *acc, cplx *kout);
// dG = -i (Cb - Ab + conj(Ab^T)) with ^T the (ij)<->(kl) transpose (dG = -i Cb when Ab is
// null); RK4 update or write k.
void g2_assemble(Launcher &L, int nb, const cplx *Cb, const cplx *Ab, Rk4Stage st, cplx *y, cplx *ys,
                 cplx *acc, cplx *kout);

// Observables.
// red[0..] = {Re Tr(h n), Re Tr((hHF-h(t)) n), Re Tr n, Re Tr(D n)} for state n;
// Hubbard basis, spin-restricted SOA (on-site w_ijkl = U_i d(i=j=k=l)): C = [h2, G] + Psi
// with the commutator over the CSR pattern (rp, ci) of h^HF, and I_ij = -i U_i G_iiji.
// GW (Go non-null: the other spin block, same-spin for the opposite-spin equation and
// vice versa) adds Pi - (Pi_lkji)^* of the reduced Hubbard polarisation; psi = false
// leaves out the source term (the same-spin equation).
void hubbard_c(Launcher &L, int nb, const int *rp, const int *ci, const cplx *hhf, const double *U, const cplx *n,
               const cplx *G, const cplx *Go, bool psi, cplx *C);
void hubbard_collision(Launcher &L, int nb, const double *U, const cplx *G, cplx *I);
void obs_one_body(Launcher &L, int nb, const cplx *h, const cplx *D, double f, const cplx *hhf,
                  const cplx *n, double *red);
// red[0] = Re sum W[(ij),(kl)] G[(kl),(ij)], red[1] = count of non-finite entries of G.
void obs_two_body(Launcher &L, int nb, const cplx *W, const cplx *G, double *partials, double *red);
// W_acc += coeff * Re Tr(D n)
void accumulate_work(Launcher &L, int nb, const cplx *D, const cplx *n, double coeff, double *W_acc);
// out[s] = double occupancy of site s (spin-orbital index 2 s + spin); eta the statistics sign.
void double_occ(Launcher &L, int nb, const cplx *n, const cplx *G, double eta, double *out);
// count non-finite entries of x (length len) into *cnt (double, accumulated)
void count_nonfinite(Launcher &L, const cplx *x, long long len, double *cnt);

// Adjoint helpers: out = alpha x + beta y (y may be null); out = c (Y + Y^dag);
// acc += coeff * Re sum conj(x) y; out (+)= Wm^T x (adjoint of the Hartree-Fock build).
void zaxpby(Launcher &L, long long n, cplx alpha, const cplx *x, cplx beta, const cplx *y, cplx *out);
void tconj_add(Launcher &L, int nb, cplx c, const cplx *Y, cplx *out);
void herm_sum(Launcher &L, int nb, cplx c, const cplx *a, cplx *out);
void real_dot_acc(Launcher &L, long long n, const cplx *x, const cplx *y, double coeff, double *partials, double *acc);
void hf_build_t(Launcher &L, int nb, const void *Wm, bool wm_real, const cplx *x, cplx *out, bool accumulate);
// Cotangent of w through the Hartree-Fock matrix Wm[(ij),(lk)] = w_ikjl + eta w_iklj given the
// cotangent x of h^HF at the state n: wbar_abcd += c (x_ac conj(n_db) + eta x_ad conj(n_cb)).
void hf_wbar(Launcher &L, int nb, const cplx *x, const cplx *n, double c, double eta, cplx *wbar);
// out = projection of X onto the symmetries of w: (X + X_jilk + conj(X_klij) + conj(X_lkji)) / 4.
void w_symmetrize(Launcher &L, int nb, const cplx *X, cplx *out);

// Memory-integral HF-GKBA: out_b[m][i] = sum_p in_b[p][m] op(S_b[i][p]) for b < batch
// (batch <= 65535, nb <= mode_rotate_max_nb()), m over the trailing nb^3 entries of the
// nb^4 tensor in_b, S_b the nb x nb matrix at S + b nb^2, op = conj when conjS;
// out[e] = beta out[e] + sum_b x[b len + e]; *cnt += number of nonzero entries of x.
int mode_rotate_max_nb();
void mode_rotate(Launcher &L, int nb, int batch, const cplx *in, const cplx *S, bool conjS, cplx *out);
void batch_sum(Launcher &L, long long len, int nbatch, const cplx *x, double beta, cplx *out);
void count_nonzero(Launcher &L, const cplx *x, long long len, double *cnt);

// Measured FP64 FMA rate of the current device in TFLOP/s (eight independent DFMA chains
// per thread, best of three timed launches after two untimed ones); *err != 0 on a CUDA failure.
double dfma_rate(cudaStream_t stream, int *err);

// Text returned by g1g2_last_error_detail on this thread.
void set_error_detail(const std::string &what);

}  // namespace g1g2
