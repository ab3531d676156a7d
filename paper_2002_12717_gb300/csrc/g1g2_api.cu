// libg1g2: the C ABI declared in include/g1g2.h.
//
// One context = one propagation on one GPU.  The RK4 driver, the drive h(t),
// validation and bookkeeping are host code here; every arithmetic step of the
// right-hand side runs in the kernels of fp64_kernels.cu (FP64 form) and
// tc_kernels.cu (split-precision tensor-core form).
#include "g1g2_internal.h"
#include "tc_path.h"

#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <unistd.h>

using namespace g1g2;

namespace {

thread_local std::string g_detail;

int fail(int code, const std::string &what) {
  g_detail = what;
  return code;
}

}  // namespace

void g1g2::set_error_detail(const std::string &what) { g_detail = what; }

struct g1g2_ctx {
  int nb = 0, se = 0, prec = 0, basis = 0;
  double eta = -1.0;                // statistics sign of the paper's ±: -1 fermions, +1 bosons
  bool w_real = false;
  cudaStream_t stream = nullptr;
  long long launches = 0;
  double t = 0.0;
  // drive h(t) = h + f(t) D
  int drive_kind = 0;
  std::vector<double> drive_params;
  bool hasD = false;
  // device memory (FP64 form)
  cplx *h = nullptr, *D = nullptr;
  void *Wm = nullptr;               // Hartree-Fock matrix [(ij),(lk)], real or complex
  bool wm_ds = false;               // real Wm held as (hi, lo) FP32 pairs (tensor-core forms)
  float4 *nsplit = nullptr;         // n as (hi, lo) FP32 pairs for the double-single build
  cplx *w = nullptr;                // w (complex), [(ij),(kl)]
  cplx *wsrc = nullptr;             // source-term interaction (w^- or w)
  bool src_pm = false;              // wsrc = w + eta w_ijlk (else wsrc = w)
  cplx *wP = nullptr;               // collision layout [(lp)][i][k] = w_iklp
  // factorised interaction w_ijkl = sum_P L^P_ik L^P_jl (FP64 form): factors [P][i][k] and
  // the per-factor products L^P n and nbar L^P n
  int nfac = 0;
  cplx *Lf = nullptr, *LfN = nullptr, *Mf = nullptr;
  cplx *n = nullptr, *ns = nullptr, *ns2 = nullptr, *nacc = nullptr;
  cplx *G = nullptr, *Gs = nullptr, *Gacc = nullptr;
  cplx *hhf = nullptr, *nbar = nullptr, *I = nullptr, *ntr = nullptr;
  cplx *Cb = nullptr, *T1 = nullptr, *T2 = nullptr, *Ab = nullptr;
  cplx *Hb = nullptr, *Gp = nullptr, *Hp = nullptr, *Pp = nullptr;
  cplx *partial = nullptr;
  int splits = 0;
  double *red = nullptr;            // small device reduction scratch
  double *obs_partials = nullptr;
  double *W_dev = nullptr;          // accumulated drive work
  std::vector<void *> allocs;
  TcPath *tc = nullptr;             // split-precision tensor-core path (precision != FP64)
  Profiler prof;
  // discrete adjoint (FP64 form), allocated on first use
  cplx *zero_h = nullptr;                       // nb*nb zeros: h for the w-part of the RHS
  cplx *AE = nullptr, *AB1 = nullptr, *AB2 = nullptr;
  double *adj_red = nullptr;                    // reduction partials
  double *adj_acc = nullptr;                    // [0] w-scale gradient, [1..] per-stage <D, hbar>
  long long adj_acc_len = 0;
  cplx *adj_hsum = nullptr;                     // accumulated cotangent of h
  cplx *adj_hbar = nullptr;                     // cotangent of hHF of one stage
  cplx *adj_wbar = nullptr;                     // accumulated cotangent of w (grad_w requested)
  std::vector<void *> adj_allocs;
  // Hubbard basis (spin-restricted SOA, on-site w): O(nb^4) right-hand side
  bool hub_ok = false, hub_on = false;
  // GW in the spin-restricted Hubbard basis (Eqs. g2-gw-hubbard1/2): G holds the opposite-spin
  // block, Gss the same-spin block that its polarisation term couples to (RK4 state Gss,
  // stage input Gss_s, accumulator Gss_acc, right-hand side Cb2)
  bool hub_gw = false;
  cplx *Gss = nullptr, *Gss_s = nullptr, *Gss_acc = nullptr, *Cb2 = nullptr;
  double *hub_U = nullptr;                      // U_i = w_iiii
  int *hub_rp = nullptr, *hub_ci = nullptr;     // CSR pattern of h^HF (h, D, diagonal), symmetric
  std::vector<unsigned char> hub_hpat;          // nonzero pattern of h (host)
  int adj_where = G1G2_CKPT_AUTO;               // where the adjoint keeps its checkpoints
  int adj_last_k = 0, adj_last_where = 0;       // plan of the last g1g2_adjoint call

  Launcher launcher() {
    Launcher L;
    L.stream = stream;
    L.counter = &launches;
    L.prof = &prof;
    return L;
  }
};

namespace {

template <class T>
int dalloc(g1g2_ctx *c, T **p, size_t count) {
  void *q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(G1G2_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return G1G2_OK;
}

int cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return G1G2_OK;
  return fail(G1G2_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int launch_status(Launcher &L, const char *what) {
  if (L.err != cudaSuccess) return fail(G1G2_ECUDA, std::string(what) + ": " + cudaGetErrorString(L.err));
  return G1G2_OK;
}

using zc = std::complex<double>;

// NVTX range for the lifetime of the object: RK4 steps and stages, observables, the
// propagation loops and the adjoint sweeps show up by name on a profiler's timeline
// (without a tool attached the calls return at once).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

bool all_finite(const double *p, size_t len) {
  for (size_t e = 0; e < len; ++e)
    if (!std::isfinite(p[e])) return false;
  return true;
}

inline zc hz(const double *a, size_t idx) { return zc(a[2 * idx], a[2 * idx + 1]); }

double drive_f(const g1g2_ctx *c, double t) {
  const std::vector<double> &p = c->drive_params;
  if (c->drive_kind == 1) {
    return p[0] * std::sin(p[1] * t) * std::exp(-(t - p[2]) * (t - p[2]) / (2.0 * p[3] * p[3]));
  }
  if (c->drive_kind == 2) {
    const double ta = p[0], tb = p[1];
    const int m = (int)p.size() - 2;
    const double hstep = (tb - ta) / (m - 1);
    const double x = (t - ta) / hstep;
    if (x <= 0) return p[2];
    if (x >= m - 1) return p[2 + m - 1];
    int s = (int)std::floor(x);
    if (s > m - 2) s = m - 2;
    const double u = x - s;
    return (1 - u) * p[2 + s] + u * p[2 + s + 1];
  }
  return 0.0;
}

double drive_dfdt(const g1g2_ctx *c, double t) {
  const std::vector<double> &p = c->drive_params;
  if (c->drive_kind == 1) {
    const double g = std::exp(-(t - p[2]) * (t - p[2]) / (2.0 * p[3] * p[3]));
    return p[0] * g * (p[1] * std::cos(p[1] * t) - std::sin(p[1] * t) * (t - p[2]) / (p[3] * p[3]));
  }
  if (c->drive_kind == 2) {
    const double ta = p[0], tb = p[1];
    const int m = (int)p.size() - 2;
    const double hstep = (tb - ta) / (m - 1);
    const double x = (t - ta) / hstep;
    if (x <= 0 || x >= m - 1) return 0.0;
    int s = (int)std::floor(x);
    if (s > m - 2) s = m - 2;
    return (p[2 + s + 1] - p[2 + s]) / hstep;
  }
  return 0.0;
}

// ---------------------------------------------------------------------------
// One right-hand side in the FP64 form.  (n_in, G_in) is the stage input; the
// G1 result goes to (ny, nys, nacc, nk) and the G2 result to (Gy, Gys, Gacc, Gk)
// according to st (RK4 stage update, or a plain write of k when st.stage < 0).
// ---------------------------------------------------------------------------
struct StageOut {
  cplx *ny, *nys, *nacc, *nk;
  cplx *Gy, *Gys, *Gacc, *Gk;
};

void mode_left1(g1g2_ctx *c, Launcher &L, const cplx *S, const cplx *X, cplx *out, cplx alpha, double beta);
void mode_left2(g1g2_ctx *c, Launcher &L, const cplx *S, const cplx *X, cplx *out, cplx alpha, double beta);
void mode_right4(g1g2_ctx *c, Launcher &L, const cplx *X, const cplx *S, cplx *out, cplx alpha, double beta);

// a2: I_ij = -i sum_(lp) sum_k wP[lp][i][k] G[lp][j][k]   (Eq. eom_gone-I) into c->I
void collision(g1g2_ctx *c, Launcher &L, const cplx *G_in) {
  const long long N = c->nb, N2 = N * N;
  ZGemm g;
  g.M = (int)N; g.N = (int)N; g.K = (int)N; g.batch = (int)N2;
  g.A = c->wP; g.sa_b = N2; g.sa_m = N; g.sa_k = 1;
  g.B = G_in; g.sb_b = N2; g.sb_k = 1; g.sb_n = N;
  g.C = c->I; g.sc_m = N; g.sc_n = 1;
  g.alpha = {0.0, -1.0};
  zgemm_reduce(L, g, c->partial, c->splits);
}

// a4: A_ijkl = sum nbar_ip nbar_jq wt_pqrs n_rk n_sl (Eq. psi-pm-def) by successive
// contractions into c->Ab (nbar into c->nbar); the source term is Psi = -A + A^dag
void source_A_factorised(g1g2_ctx *c, Launcher &L, const cplx *n_in);

void source_A(g1g2_ctx *c, Launcher &L, const cplx *n_in) {
  const int nb = c->nb;
  const long long N = nb, N2 = N * N, N3 = N2 * N;
  one_pm(L, nb, n_in, c->eta, c->nbar);
  if (c->Lf) {
    source_A_factorised(c, L, n_in);
    return;
  }
  {
    ZGemm g;  // T1_pqrl = sum_s wt_pqrs n_sl
    g.M = (int)N3; g.N = nb; g.K = nb;
    g.A = c->wsrc; g.sa_m = N; g.sa_k = 1;
    g.B = n_in; g.sb_k = N; g.sb_n = 1;
    g.C = c->T1; g.sc_m = N; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;  // T2_pqkl = sum_r n_rk T1_pqrl  (batched over (pq)), A[k][r] = n_rk
    g.M = nb; g.N = nb; g.K = nb; g.batch = (int)N2;
    g.A = n_in; g.sa_m = 1; g.sa_k = N;
    g.B = c->T1; g.sb_b = N2; g.sb_k = N; g.sb_n = 1;
    g.C = c->T2; g.sc_b = N2; g.sc_m = N; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;  // T1_pjkl = sum_q nbar_jq T2_pqkl (batched over p)
    g.M = nb; g.N = (int)N2; g.K = nb; g.batch = nb;
    g.A = c->nbar; g.sa_m = N; g.sa_k = 1;
    g.B = c->T2; g.sb_b = N3; g.sb_k = N2; g.sb_n = 1;
    g.C = c->T1; g.sc_b = N3; g.sc_m = N2; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;  // Ab_ijkl = sum_p nbar_ip T1_pjkl
    g.M = nb; g.N = (int)N3; g.K = nb;
    g.A = c->nbar; g.sa_m = N; g.sa_k = 1;
    g.B = c->T1; g.sb_k = N3; g.sb_n = 1;
    g.C = c->Ab; g.sc_m = N3; g.sc_n = 1;
    zgemm(L, g);
  }
}

// a4 for a factorised interaction w_pqrs = sum_P L^P_pr L^P_qs: the mode products act on
// each factor, sum_pr nbar_ip L^P_pr n_rk = M^P_ik with M^P = nbar L^P n, so
//   A_ijkl = sum_P M^P_ik M^P_jl            (plain w)
//          + eta sum_P M^P_il M^P_jk        (the exchange part of w^± = w_pqrs + eta w_pqsr)
// The pair product C_(ik),(jl) = sum_P M^P_ik M^P_jl is one nb^2 x nb^2 x nfac GEMM (into T1);
// A follows by two index permutations of C.  c->nbar is set by the caller.
void source_A_factorised(g1g2_ctx *c, Launcher &L, const cplx *n_in) {
  const int nb = c->nb, P = c->nfac;
  const long long N = nb, N2 = N * N;
  {
    ZGemm g;  // LfN^P_pk = sum_r L^P_pr n_rk  (batched over P)
    g.M = nb; g.N = nb; g.K = nb; g.batch = P;
    g.A = c->Lf; g.sa_b = N2; g.sa_m = N; g.sa_k = 1;
    g.B = n_in; g.sb_k = N; g.sb_n = 1;
    g.C = c->LfN; g.sc_b = N2; g.sc_m = N; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;  // M^P_ik = sum_p nbar_ip LfN^P_pk  (batched over P)
    g.M = nb; g.N = nb; g.K = nb; g.batch = P;
    g.A = c->nbar; g.sa_m = N; g.sa_k = 1;
    g.B = c->LfN; g.sb_b = N2; g.sb_k = N; g.sb_n = 1;
    g.C = c->Mf; g.sc_b = N2; g.sc_m = N; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;  // C_(ik),(jl) = sum_P M^P_(ik) M^P_(jl)
    g.M = (int)N2; g.N = (int)N2; g.K = P;
    g.A = c->Mf; g.sa_m = 1; g.sa_k = N2;
    g.B = c->Mf; g.sb_k = N2; g.sb_n = 1;
    g.C = c->T1; g.sc_m = N2; g.sc_n = 1;
    zgemm(L, g);
  }
  // A_ijkl = C(i,k,j,l) [+ eta C(i,l,j,k)]
  const int p_direct[4] = {0, 2, 1, 3};
  permute4(L, nb, c->T1, c->Ab, p_direct, {1.0, 0.0}, 0.0, false);
  if (c->src_pm) {
    const int p_exch[4] = {0, 3, 1, 2};
    permute4(L, nb, c->T1, c->Ab, p_exch, {c->eta, 0.0}, 1.0, false);
  }
}

// h^HF (Eq. h_HF) into c->hhf from the density n: FP64 in the FP64 form, double-single
// arithmetic in the tensor-core forms (where Wm is stored as FP32 pairs).
void mean_field(g1g2_ctx *c, Launcher &L, const cplx *h, const cplx *D, double f, const cplx *n) {
  if (c->wm_ds)
    hf_build_ds(L, c->nb, static_cast<const float2 *>(c->Wm), h, D, f, n, c->nsplit, c->hhf);
  else
    hf_build(L, c->nb, c->Wm, c->w_real, h, D, f, n, c->hhf);
}

void rhs_fp64(g1g2_ctx *c, Launcher &L, double t, const cplx *n_in, const cplx *G_in, Rk4Stage st,
              const StageOut &o, bool w_only = false) {
  const int nb = c->nb;
  const long long N = nb, N2 = N * N, N3 = N2 * N;
  const double f = drive_f(c, t);
  // a1: Eq. (h_HF); with w_only the one-body h(t) is left out (the part of the
  // right-hand side that is linear in w, used for the gradient by the scale of w)
  if (w_only)
    mean_field(c, L, c->zero_h, nullptr, 0.0, n_in);
  else
    mean_field(c, L, c->h, c->hasD ? c->D : nullptr, f, n_in);
  if (c->se == G1G2_HF) {
    g1_update(L, nb, c->hhf, n_in, nullptr, st, o.ny, o.nys, o.nacc, o.nk);
    return;
  }
  if (c->hub_on) {
    // Hubbard basis: I, then C = [h2, G] + Psi in O(nb^4); the assembly forms dG = -i C
    hubbard_collision(L, nb, c->hub_U, G_in, c->I);
    g1_update(L, nb, c->hhf, n_in, c->I, st, o.ny, o.nys, o.nacc, o.nk);
    if (c->hub_gw) {
      // GW: each spin block with the polarisation of the other (every read of a stage input
      // is queued before the assemblies overwrite it)
      const cplx *Gss_in = (st.stage <= 0) ? c->Gss : c->Gss_s;
      hubbard_c(L, nb, c->hub_rp, c->hub_ci, c->hhf, c->hub_U, n_in, G_in, Gss_in, true, c->Cb);
      hubbard_c(L, nb, c->hub_rp, c->hub_ci, c->hhf, c->hub_U, n_in, Gss_in, G_in, false, c->Cb2);
      g2_assemble(L, nb, c->Cb, nullptr, st, o.Gy, o.Gys, o.Gacc, o.Gk);
      g2_assemble(L, nb, c->Cb2, nullptr, st, c->Gss, c->Gss_s, c->Gss_acc, nullptr);
      return;
    }
    hubbard_c(L, nb, c->hub_rp, c->hub_ci, c->hhf, c->hub_U, n_in, G_in, nullptr, true, c->Cb);
    g2_assemble(L, nb, c->Cb, nullptr, st, o.Gy, o.Gys, o.Gacc, o.Gk);
    return;
  }
  // a2: Eq. (eom_gone-I)
  collision(c, L, G_in);
  g1_update(L, nb, c->hhf, n_in, c->I, st, o.ny, o.nys, o.nacc, o.nk);

  // a3: C = [h2, G] as four mode products (Eq. twopart_hamiltonian)
  {
    ZGemm g;  // mode 1: sum_p h_ip G_pjkl
    g.M = nb; g.N = (int)N3; g.K = nb; g.batch = 1;
    g.A = c->hhf; g.sa_m = N; g.sa_k = 1;
    g.B = G_in; g.sb_k = N3; g.sb_n = 1;
    g.C = c->Cb; g.sc_m = N3; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;  // mode 2: sum_q h_jq G_iqkl (batched over i)
    g.M = nb; g.N = (int)N2; g.K = nb; g.batch = nb;
    g.A = c->hhf; g.sa_m = N; g.sa_k = 1;
    g.B = G_in; g.sb_b = N3; g.sb_k = N2; g.sb_n = 1;
    g.C = c->Cb; g.sc_b = N3; g.sc_m = N2; g.sc_n = 1;
    g.beta = 1.0;
    zgemm(L, g);
  }
  {
    ZGemm g;  // mode 3: - sum_p G_ijpl h_pk (batched over (ij)), A[k][p] = h_pk
    g.M = nb; g.N = nb; g.K = nb; g.batch = (int)N2;
    g.A = c->hhf; g.sa_m = 1; g.sa_k = N;
    g.B = G_in; g.sb_b = N2; g.sb_k = N; g.sb_n = 1;
    g.C = c->Cb; g.sc_b = N2; g.sc_m = N; g.sc_n = 1;
    g.alpha = {-1.0, 0.0}; g.beta = 1.0;
    zgemm(L, g);
  }
  {
    ZGemm g;  // mode 4: - sum_p G_ijkp h_pl
    g.M = (int)N3; g.N = nb; g.K = nb; g.batch = 1;
    g.A = G_in; g.sa_m = N; g.sa_k = 1;
    g.B = c->hhf; g.sb_k = N; g.sb_n = 1;
    g.C = c->Cb; g.sc_m = N; g.sc_n = 1;
    g.alpha = {-1.0, 0.0}; g.beta = 1.0;
    zgemm(L, g);
  }
  // a4: Eq. (psi-pm-def) by successive contractions into A; Psi = -A + A^dag in the assembly
  source_A(c, L, n_in);
  if (c->se == G1G2_TPP || c->se == G1G2_DSL) {
    // Eq. (HTPPcorr) with G^> = -i nbar, G^< = i n: hcorr = (nbar (x) nbar - n (x) n) w
    const cplx one{1.0, 0.0}, mone{-1.0, 0.0};
    mode_left2(c, L, c->nbar, c->w, c->T1, one, 0.0);    // T1_ijkl = sum_q nbar_jq w_iqkl
    mode_left1(c, L, c->nbar, c->T1, c->Hb, one, 0.0);   // Hb_ijkl = sum_p nbar_ip T1_pjkl
    mode_left2(c, L, n_in, c->w, c->T1, one, 0.0);
    mode_left1(c, L, n_in, c->T1, c->Hb, mone, 1.0);
    // Eq. (lambdapp): Lambda = hcorr G2 as an (ij),(pq) x (pq),(kl) product.  The source term
    // is Psi = -A + A^dag, so Psi + Lambda - Lambda^dag = -(A - Lambda) + (A - Lambda)^dag:
    // subtract Lambda from A and let the assembly do the rest
    ZGemm g;
    g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
    g.A = c->Hb; g.sa_m = N2; g.sa_k = 1;
    g.B = G_in; g.sb_k = N2; g.sb_n = 1;
    g.C = c->Ab; g.sc_m = N2; g.sc_n = 1;
    g.alpha = mone; g.beta = 1.0;
    zgemm(L, g);
  }
  if (c->se == G1G2_TPH || c->se == G1G2_DSL) {
    // Eq. (HTPHcorr) with G^> = -i nbar, G^< = i n: hcorr_ijkl = sum_pq (n_ip nbar_ql - nbar_ip n_ql) w_pjkq;
    // bosons (G^< = -i n, G^> = -i nbar, nbar = 1 + n) give the opposite overall sign
    const cplx one{-c->eta, 0.0}, mone{c->eta, 0.0};
    mode_left1(c, L, n_in, c->w, c->T1, one, 0.0);       // T1_ijkq = sum_p n_ip w_pjkq
    mode_right4(c, L, c->T1, c->nbar, c->Hb, one, 0.0);  // Hb_ijkl = sum_q T1_ijkq nbar_ql
    mode_left1(c, L, c->nbar, c->w, c->T1, one, 0.0);
    mode_right4(c, L, c->T1, n_in, c->Hb, mone, 1.0);
    // Eq. (lambdaph): Lambda_ijkl = sum_pq hcorr_ipql G2_qjkp as (il),(pq) x (pq),(jk)
    const int pH[4] = {0, 2, 3, 1};  // Hp[i][l][p][q] = hcorr[i][p][q][l]
    permute4(L, nb, c->Hb, c->Hp, pH, one, 0.0, false);
    const int pG[4] = {1, 2, 3, 0};  // Gp[p][q][j][k] = G[q][j][k][p]
    permute4(L, nb, G_in, c->Gp, pG, one, 0.0, false);
    {
      ZGemm g;
      g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
      g.A = c->Hp; g.sa_m = N2; g.sa_k = 1;
      g.B = c->Gp; g.sb_k = N2; g.sb_n = 1;
      g.C = c->Pp; g.sc_m = N2; g.sc_n = 1;
      zgemm(L, g);
    }
    // A -= Lambda (as for the pp ladder term), Pp[i][l][j][k] = Lambda_ijkl
    const int pL[4] = {0, 3, 1, 2};
    permute4(L, nb, c->Pp, c->Ab, pL, mone, 1.0, false);
  }
  if (c->se == G1G2_GW || c->se == G1G2_DSL) {
    // a5: hcorr_ijkl = sum_p w_ijkp n_pl - sum_q n_jq w_iqkl (Eq. gwhcorr with the exchange symmetry of w)
    {
      ZGemm g;
      g.M = (int)N3; g.N = nb; g.K = nb;
      g.A = c->w; g.sa_m = N; g.sa_k = 1;
      g.B = n_in; g.sb_k = N; g.sb_n = 1;
      g.C = c->Hb; g.sc_m = N; g.sc_n = 1;
      zgemm(L, g);
    }
    {
      ZGemm g;
      g.M = nb; g.N = (int)N2; g.K = nb; g.batch = nb;
      g.A = n_in; g.sa_m = N; g.sa_k = 1;
      g.B = c->w; g.sb_b = N3; g.sb_k = N2; g.sb_n = 1;
      g.C = c->Hb; g.sc_b = N3; g.sc_m = N2; g.sc_n = 1;
      g.alpha = {-1.0, 0.0}; g.beta = 1.0;
      zgemm(L, g);
    }
    // a6: Pi_ijkl = sum_pq hcorr_qjpl G_ipkq (Eq. gwpi) as one (ik)x(pq) . (pq)x(jl) GEMM
    const int pG[4] = {0, 2, 1, 3};  // Gp[i][k][p][q] = G[i][p][k][q]
    permute4(L, nb, G_in, c->Gp, pG, {1.0, 0.0}, 0.0, false);
    const int pH[4] = {1, 2, 0, 3};  // Hp[p][q][j][l] = hcorr[q][j][p][l]
    permute4(L, nb, c->Hb, c->Hp, pH, {1.0, 0.0}, 0.0, false);
    {
      ZGemm g;
      g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
      g.A = c->Gp; g.sa_m = N2; g.sa_k = 1;
      g.B = c->Hp; g.sb_k = N2; g.sb_n = 1;
      g.C = c->Pp; g.sc_m = N2; g.sc_n = 1;
      zgemm(L, g);
    }
    // Cb += Pi_ijkl - conj(Pi_lkji), Pp[i][k][j][l] = Pi_ijkl
    const int pP[4] = {0, 2, 1, 3};
    permute4(L, nb, c->Pp, c->Cb, pP, {1.0, 0.0}, 1.0, false);
    const int pR[4] = {3, 1, 2, 0};
    permute4(L, nb, c->Pp, c->Cb, pR, {-1.0, 0.0}, 1.0, true);
  }
  // a7: dG = -i (C + Psi [+ Pi - Pi^*]) and the RK4 update
  g2_assemble(L, nb, c->Cb, c->Ab, st, o.Gy, o.Gys, o.Gacc, o.Gk);
}

void rhs_dispatch(g1g2_ctx *c, Launcher &L, double t, const cplx *n_in, const cplx *G_in, Rk4Stage st,
                  const StageOut &o) {
  if (c->prec == G1G2_FP64 || c->se == G1G2_HF) {
    rhs_fp64(c, L, t, n_in, G_in, st, o);
  } else {
    const double f = drive_f(c, t);
    mean_field(c, L, c->h, c->hasD ? c->D : nullptr, f, n_in);
    tc_rhs(c->tc, L, n_in, G_in, c->hhf, st, o.ny, o.nys, o.nacc, o.nk, o.Gy, o.Gys, o.Gacc, o.Gk);
  }
}

int rk4_step(g1g2_ctx *c, double dt) {
  NvtxRange step_range("g1g2 rk4 step");
  static const char *const stage_name[4] = {"g1g2 rk4 stage 1", "g1g2 rk4 stage 2", "g1g2 rk4 stage 3",
                                            "g1g2 rk4 stage 4"};
  Launcher L = c->launcher();
  const double t = c->t;
  const double cs[4] = {0.0, 0.5, 0.5, 1.0};
  const double wgt[4] = {1.0, 2.0, 2.0, 1.0};
  // G1 stage states ping-pong between ns and ns2: the G1 update of a stage
  // is queued before the G2 contractions that still read the stage input.
  cplx *n_in_of[4] = {c->n, c->ns, c->ns2, c->ns};
  cplx *n_out_of[4] = {c->ns, c->ns2, c->ns, nullptr};
  for (int s = 0; s < 4; ++s) {
    StageOut o{c->n, n_out_of[s], c->nacc, nullptr, c->G, c->Gs, c->Gacc, nullptr};
    const cplx *n_in = n_in_of[s];
    const cplx *G_in = (s == 0) ? c->G : c->Gs;
    if (c->hasD && c->drive_kind != 0) {
      const double coeff = dt / 6.0 * wgt[s] * drive_dfdt(c, t + cs[s] * dt);
      accumulate_work(L, c->nb, c->D, n_in, coeff * (c->basis == G1G2_SPIN_RESTRICTED ? 2.0 : 1.0), c->W_dev);
    }
    NvtxRange stage_range(stage_name[s]);
    Rk4Stage st{s, dt};
    rhs_dispatch(c, L, t + cs[s] * dt, n_in, G_in, st, o);
  }
  c->t = t + dt;
  return launch_status(L, "rk4 step");
}

int observables_impl(g1g2_ctx *c, g1g2_obs *out, double *density, double *nonfinite) {
  NvtxRange range("g1g2 observables");
  Launcher L = c->launcher();
  const int nb = c->nb;
  const double f = drive_f(c, c->t);
  mean_field(c, L, c->h, c->hasD ? c->D : nullptr, f, c->n);
  obs_one_body(L, nb, c->h, c->hasD ? c->D : nullptr, f, c->hhf, c->n, c->red);
  double zero2[2] = {0.0, 0.0};
  if (c->se != G1G2_HF) {
    obs_two_body(L, nb, c->w, c->G, c->obs_partials, c->red + 4);
  } else {
    cudaMemcpyAsync(c->red + 4, zero2, sizeof(zero2), cudaMemcpyHostToDevice, c->stream);
  }
  count_nonfinite(L, c->n, (long long)nb * nb, c->red + 5);
  int rc = launch_status(L, "observables");
  if (rc) return rc;
  double r[6], W = 0.0;
  if ((rc = cuda_check(cudaMemcpyAsync(r, c->red, sizeof(r), cudaMemcpyDeviceToHost, c->stream), "obs copy"))) return rc;
  if ((rc = cuda_check(cudaMemcpyAsync(&W, c->W_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "obs copy"))) return rc;
  std::vector<cplx> diag;
  if (density) {
    diag.resize(nb);
    if ((rc = cuda_check(cudaMemcpy2DAsync(diag.data(), sizeof(cplx), c->n, (nb + 1) * sizeof(cplx), sizeof(cplx), nb,
                                           cudaMemcpyDeviceToHost, c->stream), "density copy")))
      return rc;
  }
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "obs sync"))) return rc;
  if (c->tc && (rc = tc_error(c->tc, c->stream))) return rc;
  const bool restricted = c->basis == G1G2_SPIN_RESTRICTED;
  const double s = restricted ? 2.0 : 1.0;
  out->t = c->t;
  out->e_one = s * r[0];
  out->e_hf = restricted ? r[1] : 0.5 * r[1];
  out->n_particles = s * r[2];
  out->e_corr = (c->se == G1G2_HF) ? 0.0 : (restricted ? -r[4] : -0.5 * r[4]);
  out->e_total = out->e_one + out->e_hf + out->e_corr;
  out->pulse_work = W;
  if (density)
    for (int i = 0; i < nb; ++i) density[i] = s * diag[i].x;
  if (nonfinite) *nonfinite = r[5];
  return G1G2_OK;
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the FP64 form (HF and SOA).
//
// Cotangents use the real inner product <X, Y> = Re sum conj(X) Y over every
// complex entry of (n, G2); the right-hand side is not holomorphic (it contains
// I^dag, A^dag), so each term's adjoint is taken with respect to that product.
// ---------------------------------------------------------------------------

// out = alpha * (three-index contraction of X and conj(Z)) + beta * out, out nb x nb:
//   mode 1: out[i][p] = sum_jkl X_ijkl conj(Z_pjkl)   mode 2: out[j][q] = sum_ikl X_ijkl conj(Z_iqkl)
//   mode 3: out[p][k] = sum_ijl conj(Z_ijpl) X_ijkl   mode 4: out[p][l] = sum_ijk conj(Z_ijkp) X_ijkl
void contract3(g1g2_ctx *c, Launcher &L, int mode, const cplx *X, const cplx *Z, cplx alpha, double beta, cplx *out) {
  const long long N = c->nb, N2 = N * N, N3 = N2 * N;
  ZGemm g;
  g.M = c->nb; g.N = c->nb; g.C = out; g.sc_m = N; g.sc_n = 1; g.alpha = alpha; g.beta = beta;
  if (mode == 1) {
    g.K = (int)N2; g.batch = c->nb;
    g.A = X; g.sa_b = N2; g.sa_m = N3; g.sa_k = 1;
    g.B = Z; g.sb_b = N2; g.sb_k = 1; g.sb_n = N3; g.conjB = true;
  } else if (mode == 2) {
    g.K = (int)N2; g.batch = c->nb;
    g.A = X; g.sa_b = N3; g.sa_m = N2; g.sa_k = 1;
    g.B = Z; g.sb_b = N3; g.sb_k = 1; g.sb_n = N2; g.conjB = true;
  } else if (mode == 3) {
    g.K = c->nb; g.batch = (int)N2;
    g.A = Z; g.sa_b = N2; g.sa_m = N; g.sa_k = 1; g.conjA = true;
    g.B = X; g.sb_b = N2; g.sb_k = 1; g.sb_n = N;
  } else {
    g.K = (int)N2; g.batch = c->nb;
    g.A = Z; g.sa_b = N3; g.sa_m = 1; g.sa_k = N; g.conjA = true;
    g.B = X; g.sb_b = N3; g.sb_k = N; g.sb_n = 1;
  }
  zgemm_reduce(L, g, c->partial, c->splits);
}

// Mode products on nb^4 tensors: right products over index 4 or 3, left products over 1 or 2.
void mode_right4(g1g2_ctx *c, Launcher &L, const cplx *X, const cplx *S, cplx *out, cplx alpha, double beta) {
  const long long N = c->nb;
  ZGemm g;
  g.M = (int)(N * N * N); g.N = c->nb; g.K = c->nb;
  g.A = X; g.sa_m = N; g.sa_k = 1; g.B = S; g.sb_k = N; g.sb_n = 1;
  g.C = out; g.sc_m = N; g.sc_n = 1; g.alpha = alpha; g.beta = beta;
  zgemm(L, g);
}
void mode_right3(g1g2_ctx *c, Launcher &L, const cplx *X, const cplx *S, cplx *out, cplx alpha, double beta) {
  const long long N = c->nb, N2 = N * N;
  ZGemm g;
  g.M = c->nb; g.N = c->nb; g.K = c->nb; g.batch = (int)N2;
  g.A = S; g.sa_m = 1; g.sa_k = N; g.B = X; g.sb_b = N2; g.sb_k = N; g.sb_n = 1;
  g.C = out; g.sc_b = N2; g.sc_m = N; g.sc_n = 1; g.alpha = alpha; g.beta = beta;
  zgemm(L, g);
}
void mode_left2(g1g2_ctx *c, Launcher &L, const cplx *S, const cplx *X, cplx *out, cplx alpha, double beta) {
  const long long N = c->nb, N2 = N * N, N3 = N2 * N;
  ZGemm g;
  g.M = c->nb; g.N = (int)N2; g.K = c->nb; g.batch = c->nb;
  g.A = S; g.sa_m = N; g.sa_k = 1; g.B = X; g.sb_b = N3; g.sb_k = N2; g.sb_n = 1;
  g.C = out; g.sc_b = N3; g.sc_m = N2; g.sc_n = 1; g.alpha = alpha; g.beta = beta;
  zgemm(L, g);
}
void mode_left1(g1g2_ctx *c, Launcher &L, const cplx *S, const cplx *X, cplx *out, cplx alpha, double beta) {
  const long long N = c->nb, N3 = N * N * N;
  ZGemm g;
  g.M = c->nb; g.N = (int)N3; g.K = c->nb;
  g.A = S; g.sa_m = N; g.sa_k = 1; g.B = X; g.sb_k = N3; g.sb_n = 1;
  g.C = out; g.sc_m = N3; g.sc_n = 1; g.alpha = alpha; g.beta = beta;
  zgemm(L, g);
}
void matmul(g1g2_ctx *c, Launcher &L, const cplx *A, const cplx *B, cplx *out, cplx alpha, double beta) {
  const long long N = c->nb;
  ZGemm g;
  g.M = c->nb; g.N = c->nb; g.K = c->nb;
  g.A = A; g.sa_m = N; g.sa_k = 1; g.B = B; g.sb_k = N; g.sb_n = 1;
  g.C = out; g.sc_m = N; g.sc_n = 1; g.alpha = alpha; g.beta = beta;
  zgemm(L, g);
}

// Vector-Jacobian product of the FP64 right-hand side at (t, n, G): given the
// cotangents (a, Y) of (dn, dG2), write the cotangents nbar of n, Gbar of G2
// and hbar of h^HF (which is also the cotangent of the explicit h(t)); with wbar
// non-null, add the cotangent of the interaction w (every place w enters: the
// Hartree-Fock build, the collision integral, the source term, the GW
// quasi-Hamiltonian and the ladder quasi-Hamiltonians) to wbar.
void vjp_fp64(g1g2_ctx *c, Launcher &L, double t, const cplx *n, const cplx *G, const cplx *a, const cplx *Y,
              cplx *nbar, cplx *Gbar, cplx *hbar, cplx *wbar = nullptr) {
  const int nb = c->nb;
  const long long N = nb, N2 = N * N, N4 = N2 * N2;
  const cplx I1{0.0, 1.0}, mI{0.0, -1.0}, one{1.0, 0.0}, mone{-1.0, 0.0};
  const double f = drive_f(c, t);
  hf_build(L, nb, c->Wm, c->w_real, c->h, c->hasD ? c->D : nullptr, f, n, c->hhf);
  // dn = -i [hHF, n] - (I + I^dag): cotangent of hHF from the commutator: i [a, n]
  matmul(c, L, a, n, hbar, I1, 0.0);
  matmul(c, L, n, a, hbar, mI, 1.0);
  const bool corr = c->se != G1G2_HF;
  if (corr) {
    // dG2 = -i [h2(hHF), G2] - i Psi: cotangent of hHF from the commutator
    contract3(c, L, 1, Y, G, I1, 1.0, hbar);
    contract3(c, L, 2, Y, G, I1, 1.0, hbar);
    contract3(c, L, 3, Y, G, mI, 1.0, hbar);
    contract3(c, L, 4, Y, G, mI, 1.0, hbar);
  }
  // nbar = i [hHF, a] + (adjoint of the Hartree-Fock build)(hbar)
  matmul(c, L, c->hhf, a, nbar, I1, 0.0);
  matmul(c, L, a, c->hhf, nbar, mI, 1.0);
  hf_build_t(L, nb, c->Wm, c->w_real, hbar, nbar, true);
  const bool restricted = c->basis == G1G2_SPIN_RESTRICTED;
  // wbar from Eq. (h_HF): Wm[(ij),(lk)] = w_ikjl + eta w_iklj (restricted: w_ikjl)
  if (wbar) hf_wbar(L, nb, hbar, n, 1.0, restricted ? 0.0 : c->eta, wbar);
  if (!corr) {
    cudaMemsetAsync(Gbar, 0, N4 * sizeof(cplx), c->stream);
    return;
  }
  // Gbar = i [h2(hHF), Y]  (the commutator map is anti-Hermitian)
  mode_left1(c, L, c->hhf, Y, Gbar, I1, 0.0);
  mode_left2(c, L, c->hhf, Y, Gbar, I1, 1.0);
  mode_right3(c, L, Y, c->hhf, Gbar, mI, 1.0);
  mode_right4(c, L, Y, c->hhf, Gbar, mI, 1.0);
  // collision integral I_ij = -i sum w_iklp G2_lpjk, cotangent Ibar = -(a + a^dag):
  // Gbar_lpjk += i sum_i w_iklp Ibar_ij  (batched over (lp) with wP[(lp)][i][k] = w_iklp)
  herm_sum(L, nb, mone, a, c->I);
  {
    ZGemm g;
    g.M = nb; g.N = nb; g.K = nb; g.batch = (int)N2;
    g.A = c->I; g.sa_m = 1; g.sa_k = N;
    g.B = c->wP; g.sb_b = N2; g.sb_k = N; g.sb_n = 1; g.conjB = true;
    g.C = Gbar; g.sc_b = N2; g.sc_m = N; g.sc_n = 1;
    g.alpha = I1; g.beta = 1.0;
    zgemm(L, g);
  }
  if (wbar) {
    ZGemm g;  // wbar_iklp += i sum_j Ibar_ij conj(G_lpjk)  (batched over (lp), Ibar shared)
    g.M = nb; g.N = nb; g.K = nb; g.batch = (int)N2;
    g.A = c->I; g.sa_b = 0; g.sa_m = N; g.sa_k = 1;
    g.B = G; g.sb_b = N2; g.sb_k = N; g.sb_n = 1; g.conjB = true;
    g.C = wbar; g.sc_b = 1; g.sc_m = N2 * N; g.sc_n = N2;
    g.alpha = I1; g.beta = 1.0;
    zgemm(L, g);
  }
  // source term: -i Psi = i A - i A^dag, cotangent of A: E = -i (Y + Y^dag);
  // A = nbar1 nbar2 w~ n3 n4, one n-factor at a time
  tconj_add(L, nb, mI, Y, c->AE);
  one_minus(L, nb, n, c->nbar);
  mode_right4(c, L, c->wsrc, n, c->T1, one, 0.0);          // T1_pqrl = sum_s w~_pqrs n_sl
  mode_right3(c, L, c->T1, n, c->T2, one, 0.0);            // T2_pqkl = sum_r n_rk T1_pqrl
  mode_left2(c, L, c->nbar, c->T2, c->AB1, one, 0.0);      // B1 = nbar x_2 T2
  contract3(c, L, 1, c->AE, c->AB1, mone, 1.0, nbar);
  mode_left1(c, L, c->nbar, c->T2, c->AB1, one, 0.0);      // B2 = nbar x_1 T2
  contract3(c, L, 2, c->AE, c->AB1, mone, 1.0, nbar);
  mode_left2(c, L, c->nbar, c->T1, c->AB1, one, 0.0);
  mode_left1(c, L, c->nbar, c->AB1, c->AB2, one, 0.0);     // B3 = nbar x_1 nbar x_2 T1
  contract3(c, L, 3, c->AE, c->AB2, one, 1.0, nbar);
  mode_right3(c, L, c->wsrc, n, c->AB1, one, 0.0);         // T1'_pqks = sum_r w~_pqrs n_rk
  mode_left2(c, L, c->nbar, c->AB1, c->T2, one, 0.0);
  mode_left1(c, L, c->nbar, c->T2, c->AB2, one, 0.0);      // B4 = nbar x_1 nbar x_2 T1'
  contract3(c, L, 4, c->AE, c->AB2, one, 1.0, nbar);
  if (wbar) {
    // A = (nbar (x) nbar) w~ (n (x) n): w~bar_pqrs = sum_ijkl nbar_pi nbar_qj E_ijkl n_kr n_ls
    // (n, nbar Hermitian); w~ = w + eta w_pqsr (source w^±) or w
    mode_left1(c, L, c->nbar, c->AE, c->AB1, one, 0.0);
    mode_left2(c, L, c->nbar, c->AB1, c->AB2, one, 0.0);
    mode_right3(c, L, c->AB2, n, c->AB1, one, 0.0);
    mode_right4(c, L, c->AB1, n, c->AB2, one, 0.0);
    zaxpby(L, N4, one, wbar, one, c->AB2, wbar);
    const int p34[4] = {0, 1, 3, 2};
    if (c->src_pm) permute4(L, nb, c->AB2, wbar, p34, cplx{c->eta, 0.0}, 1.0, false);
  }
  // Ladder terms (Eqs. lambdapp, lambdaph): the source buffer holds A - Lambda, so the cotangent
  // of Lambda is -AE.  With nbar = 1 - n, dH^pp_ijkl = -sum_p dn_ip w_pjkl - sum_q dn_jq w_iqkl
  // and dH^ph_ijkl = sum_p dn_ip w_pjkl - sum_q dn_ql w_ijkq (Eqs. HTPPcorr, HTPHcorr).
  if (c->se == G1G2_TPP || c->se == G1G2_DSL) {
    mode_left2(c, L, c->nbar, c->w, c->T1, one, 0.0);    // Hb = (nbar (x) nbar - n (x) n) w
    mode_left1(c, L, c->nbar, c->T1, c->Hb, one, 0.0);
    mode_left2(c, L, n, c->w, c->T1, one, 0.0);
    mode_left1(c, L, n, c->T1, c->Hb, mone, 1.0);
    {
      ZGemm g;  // Gbar_(pq),(kl) -= sum_(ij) conj(H_(ij),(pq)) AE_(ij),(kl)
      g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
      g.A = c->Hb; g.sa_m = 1; g.sa_k = N2; g.conjA = true;
      g.B = c->AE; g.sb_k = N2; g.sb_n = 1;
      g.C = Gbar; g.sc_m = N2; g.sc_n = 1;
      g.alpha = mone; g.beta = 1.0;
      zgemm(L, g);
    }
    {
      ZGemm g;  // AB1 = Hbar_(ij),(pq) = -sum_(kl) AE_(ij),(kl) conj(G_(pq),(kl))
      g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
      g.A = c->AE; g.sa_m = N2; g.sa_k = 1;
      g.B = G; g.sb_k = 1; g.sb_n = N2; g.conjB = true;
      g.C = c->AB1; g.sc_m = N2; g.sc_n = 1;
      g.alpha = mone;
      zgemm(L, g);
    }
    contract3(c, L, 1, c->AB1, c->w, mone, 1.0, nbar);
    contract3(c, L, 2, c->AB1, c->w, mone, 1.0, nbar);
    if (wbar) {
      // H = (nbar (x) nbar - n (x) n) w: wbar_pqkl += sum_ij (nbar_pi nbar_qj - n_pi n_qj) Hbar_ijkl
      mode_left1(c, L, c->nbar, c->AB1, c->T1, one, 0.0);
      mode_left2(c, L, c->nbar, c->T1, wbar, one, 1.0);
      mode_left1(c, L, n, c->AB1, c->T1, one, 0.0);
      mode_left2(c, L, n, c->T1, wbar, mone, 1.0);
    }
  }
  if (c->se == G1G2_TPH || c->se == G1G2_DSL) {
    mode_left1(c, L, n, c->w, c->T1, one, 0.0);           // Hb = n w nbar - nbar w n (modes 1 and 4)
    mode_right4(c, L, c->T1, c->nbar, c->Hb, one, 0.0);
    mode_left1(c, L, c->nbar, c->w, c->T1, one, 0.0);
    mode_right4(c, L, c->T1, n, c->Hb, mone, 1.0);
    const int pH[4] = {0, 2, 3, 1};  // Hp[i][l][p][q] = H[i][p][q][l]
    permute4(L, nb, c->Hb, c->Hp, pH, one, 0.0, false);
    const int pGt[4] = {1, 2, 3, 0};  // Gp[p][q][j][k] = G[q][j][k][p]
    permute4(L, nb, G, c->Gp, pGt, one, 0.0, false);
    permute4(L, nb, c->AE, c->Pp, pH, mone, 0.0, false);  // Pp[i][l][j][k] = -AE_ijkl (cotangent of Lambda)
    {
      ZGemm g;  // AB2[(pq)][(jk)] = sum_(il) conj(Hp[(il)][(pq)]) Pp[(il)][(jk)]
      g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
      g.A = c->Hp; g.sa_m = 1; g.sa_k = N2; g.conjA = true;
      g.B = c->Pp; g.sb_k = N2; g.sb_n = 1;
      g.C = c->AB2; g.sc_m = N2; g.sc_n = 1;
      zgemm(L, g);
    }
    const int pGb[4] = {3, 0, 1, 2};  // Gbar[q][j][k][p] += AB2[p][q][j][k]
    permute4(L, nb, c->AB2, Gbar, pGb, one, 1.0, false);
    {
      ZGemm g;  // AB1[(il)][(pq)] = sum_(jk) Pp[(il)][(jk)] conj(Gp[(pq)][(jk)])
      g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
      g.A = c->Pp; g.sa_m = N2; g.sa_k = 1;
      g.B = c->Gp; g.sb_k = 1; g.sb_n = N2; g.conjB = true;
      g.C = c->AB1; g.sc_m = N2; g.sc_n = 1;
      zgemm(L, g);
    }
    const int pHb[4] = {0, 3, 1, 2};  // T2 = Hbar[i][p][q][l] = AB1[i][l][p][q]
    permute4(L, nb, c->AB1, c->T2, pHb, one, 0.0, false);
    contract3(c, L, 1, c->T2, c->w, one, 1.0, nbar);
    contract3(c, L, 4, c->T2, c->w, mone, 1.0, nbar);
    if (wbar) {
      // H = n w nbar - nbar w n (modes 1 and 4): wbar_pjks += sum_il (n_pi Hbar_ijkl nbar_ls - nbar_pi Hbar_ijkl n_ls)
      mode_left1(c, L, n, c->T2, c->T1, one, 0.0);
      mode_right4(c, L, c->T1, c->nbar, wbar, one, 1.0);
      mode_left1(c, L, c->nbar, c->T2, c->T1, one, 0.0);
      mode_right4(c, L, c->T1, n, wbar, mone, 1.0);
    }
  }
  if (c->se != G1G2_GW && c->se != G1G2_DSL) return;
  // GW: dG2 += -i (Pi - conj(Pi_lkji)), Pi_ijkl = sum_pq hcorr_qjpl G_ipkq, hcorr = w x_4 n - n x_2 w
  // (Eqs. gwpi, gwhcorr).  Cotangent of Pi: Pibar = i (Y + conj(Y_lkji)); then the transposed
  // products of the forward GEMM (Pp = Gp Hp) and of the two mode products of hcorr.
  {
    ZGemm g;  // Hb = hcorr (recomputed as in the forward pass)
    g.M = (int)(N2 * N); g.N = nb; g.K = nb;
    g.A = c->w; g.sa_m = N; g.sa_k = 1;
    g.B = n; g.sb_k = N; g.sb_n = 1;
    g.C = c->Hb; g.sc_m = N; g.sc_n = 1;
    zgemm(L, g);
  }
  {
    ZGemm g;
    g.M = nb; g.N = (int)N2; g.K = nb; g.batch = nb;
    g.A = n; g.sa_m = N; g.sa_k = 1;
    g.B = c->w; g.sb_b = N2 * N; g.sb_k = N2; g.sb_n = 1;
    g.C = c->Hb; g.sc_b = N2 * N; g.sc_m = N2; g.sc_n = 1;
    g.alpha = mone; g.beta = 1.0;
    zgemm(L, g);
  }
  const int pG[4] = {0, 2, 1, 3};  // Gp[i][k][p][q] = G[i][p][k][q]
  permute4(L, nb, G, c->Gp, pG, one, 0.0, false);
  const int pH[4] = {1, 2, 0, 3};  // Hp[p][q][j][l] = hcorr[q][j][p][l]
  permute4(L, nb, c->Hb, c->Hp, pH, one, 0.0, false);
  const int pT[4] = {3, 2, 1, 0};  // AB1 = Pibar = i Y + i conj(Y_lkji)
  permute4(L, nb, Y, c->AB1, pT, I1, 0.0, true);
  zaxpby(L, N4, I1, Y, one, c->AB1, c->AB1);
  permute4(L, nb, c->AB1, c->Pp, pG, one, 0.0, false);  // Pp[i][k][j][l] = Pibar_ijkl
  {
    ZGemm g;  // AB2[(ik)][(pq)] = sum_(jl) Pp[(ik)][(jl)] conj(Hp[(pq)][(jl)])
    g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
    g.A = c->Pp; g.sa_m = N2; g.sa_k = 1;
    g.B = c->Hp; g.sb_k = 1; g.sb_n = N2; g.conjB = true;
    g.C = c->AB2; g.sc_m = N2; g.sc_n = 1;
    zgemm(L, g);
  }
  permute4(L, nb, c->AB2, Gbar, pG, one, 1.0, false);   // Gbar[i][p][k][q] += AB2[i][k][p][q]
  {
    ZGemm g;  // AE[(pq)][(jl)] = sum_(ik) conj(Gp[(ik)][(pq)]) Pp[(ik)][(jl)]  (cotangent of Hp)
    g.M = (int)N2; g.N = (int)N2; g.K = (int)N2;
    g.A = c->Gp; g.sa_m = 1; g.sa_k = N2; g.conjA = true;
    g.B = c->Pp; g.sb_k = N2; g.sb_n = 1;
    g.C = c->AE; g.sc_m = N2; g.sc_n = 1;
    zgemm(L, g);
  }
  const int pHt[4] = {2, 0, 1, 3};  // Hb = hcorr-bar[q][j][p][l] = AE[p][q][j][l]
  permute4(L, nb, c->AE, c->Hb, pHt, one, 0.0, false);
  {
    ZGemm g;  // nbar_pl += sum_(ijk) conj(w_ijkp) hbar_ijkl
    g.M = nb; g.N = nb; g.K = (int)(N2 * N);
    g.A = c->w; g.sa_m = 1; g.sa_k = N; g.conjA = true;
    g.B = c->Hb; g.sb_k = N; g.sb_n = 1;
    g.C = nbar; g.sc_m = N; g.sc_n = 1;
    g.beta = 1.0;
    zgemm_reduce(L, g, c->partial, c->splits);
  }
  {
    ZGemm g;  // nbar_jq -= sum_i sum_(kl) hbar_ijkl conj(w_iqkl)
    g.M = nb; g.N = nb; g.K = (int)N2; g.batch = nb;
    g.A = c->Hb; g.sa_b = N2 * N; g.sa_m = N2; g.sa_k = 1;
    g.B = c->w; g.sb_b = N2 * N; g.sb_k = 1; g.sb_n = N2; g.conjB = true;
    g.C = nbar; g.sc_m = N; g.sc_n = 1;
    g.alpha = mone; g.beta = 1.0;
    zgemm_reduce(L, g, c->partial, c->splits);
  }
  if (wbar) {
    // hcorr = w x_4 n - n x_2 w: wbar_ijks += sum_l hbar_ijkl n_ls, wbar_iqkl -= sum_j n_qj hbar_ijkl
    mode_right4(c, L, c->Hb, n, wbar, one, 1.0);
    mode_left2(c, L, n, c->Hb, wbar, mone, 1.0);
  }
}

// CSR pattern of h^HF for the Hubbard path: the nonzeros of h (and of D when a
// drive is set), the diagonal, made symmetric.
int hub_upload_pattern(g1g2_ctx *c, const std::vector<cplx> *D) {
  const int N = c->nb;
  std::vector<int> rp(N + 1, 0), ci;
  for (int i = 0; i < N; ++i) {
    for (int p = 0; p < N; ++p) {
      const size_t a = (size_t)i * N + p, b = (size_t)p * N + i;
      bool nz = i == p || c->hub_hpat[a] || c->hub_hpat[b];
      if (D && !nz) nz = (*D)[a].x != 0.0 || (*D)[a].y != 0.0 || (*D)[b].x != 0.0 || (*D)[b].y != 0.0;
      if (nz) ci.push_back(p);
    }
    rp[i + 1] = (int)ci.size();
  }
  if (cudaMemcpyAsync(c->hub_rp, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->hub_ci, ci.data(), ci.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(G1G2_ECUDA, "Hubbard pattern upload");
  }
  return G1G2_OK;
}

int adj_alloc(g1g2_ctx *, std::vector<void *> &own, void **p, size_t bytes) {
  void *q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(G1G2_ENOMEM, "adjoint: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  own.push_back(q);
  *p = q;
  return G1G2_OK;
}

}  // namespace

// Helpers of the memory-integral HF-GKBA (g1g2_propagate_hfgkba).
namespace {

struct DevScratch {
  std::vector<void *> p;
  ~DevScratch() { for (void *q : p) cudaFree(q); }
  template <class T>
  int get(T **out, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return fail(G1G2_ENOMEM, "memory-integral scratch of " + std::to_string(count * sizeof(T)) + " bytes");
    }
    p.push_back(q);
    *out = static_cast<T *>(q);
    return G1G2_OK;
  }
};

// dn = -i[hHF, n] - (I + I^dag) with I from G2, du = -i hHF u (Eqs. eom_gone-2, eom_gone-I)
void gkba_derivs(g1g2_ctx *c, Launcher &L, const cplx *n, const cplx *u, const cplx *G2, cplx *dn, cplx *du) {
  const int nb = c->nb;
  hf_build(L, nb, c->Wm, c->w_real, c->h, nullptr, 0.0, n, c->hhf);
  collision(c, L, G2);
  g1_update(L, nb, c->hhf, n, c->I, Rk4Stage{-1, 0.0}, nullptr, nullptr, nullptr, dn);
  ZGemm g;
  g.M = nb; g.N = nb; g.K = nb;
  g.A = c->hhf; g.sa_m = nb; g.sa_k = 1;
  g.B = u; g.sb_k = nb; g.sb_n = 1;
  g.C = du; g.sc_m = nb; g.sc_n = 1;
  g.alpha = {0.0, -1.0};
  zgemm(L, g);
}

// Q = -i Psi(n) = -i (-A + A^dag): the assembly with a zero commutator buffer (c->Cb)
void gkba_source(g1g2_ctx *c, Launcher &L, const cplx *n, cplx *Q) {
  source_A(c, L, n);
  g2_assemble(L, c->nb, c->Cb, c->Ab, Rk4Stage{-1, 0.0}, nullptr, nullptr, nullptr, Q);
}

struct GkbaHist {
  cplx *u = nullptr, *Q = nullptr, *V = nullptr, *Vs = nullptr, *Y0 = nullptr, *Y1 = nullptr;
  int chunk = 1;
};

// G2 = sum_{k<K} w_k dt (V_k (x) V_k) Q_k (V_k (x) V_k)^dag, V_k = u_now u_k^dag, trapezoid
// weights w_0 = w_{K-1} = 1/2 (G2 = 0 for K = 1)
void gkba_memory(g1g2_ctx *c, Launcher &L, const GkbaHist &H, int K, const cplx *u_now, double dt, cplx *G2) {
  const int nb = c->nb;
  const long long N2 = (long long)nb * nb, N4 = N2 * N2;
  if (K <= 1) {
    cudaMemsetAsync(G2, 0, N4 * sizeof(cplx), L.stream);
    return;
  }
  {
    ZGemm g;  // V_k[i][j] = sum_p u_now[i][p] conj(u_k[j][p])
    g.M = nb; g.N = nb; g.K = nb; g.batch = K;
    g.A = u_now; g.sa_b = 0; g.sa_m = nb; g.sa_k = 1;
    g.B = H.u; g.sb_b = N2; g.sb_k = 1; g.sb_n = nb; g.conjB = true;
    g.C = H.V; g.sc_b = N2; g.sc_m = nb; g.sc_n = 1;
    zgemm(L, g);
  }
  zaxpby(L, (long long)K * N2, {dt, 0.0}, H.V, {0.0, 0.0}, nullptr, H.Vs);
  zaxpby(L, N2, {0.5 * dt, 0.0}, H.V, {0.0, 0.0}, nullptr, H.Vs);
  zaxpby(L, N2, {0.5 * dt, 0.0}, H.V + (K - 1) * N2, {0.0, 0.0}, nullptr, H.Vs + (K - 1) * N2);
  for (int k0 = 0; k0 < K; k0 += H.chunk) {
    const int kc = std::min(H.chunk, K - k0);
    mode_rotate(L, nb, kc, H.Q + k0 * N4, H.Vs + k0 * N2, false, H.Y0);
    mode_rotate(L, nb, kc, H.Y0, H.V + k0 * N2, false, H.Y1);
    mode_rotate(L, nb, kc, H.Y1, H.V + k0 * N2, true, H.Y0);
    mode_rotate(L, nb, kc, H.Y0, H.V + k0 * N2, true, H.Y1);
    batch_sum(L, N4, kc, H.Y1, k0 == 0 ? 0.0 : 1.0, G2);
  }
}

}  // namespace

extern "C" {

void g1g2_default_options(g1g2_options *opt) {
  if (!opt) return;
  opt->precision = G1G2_FP64;
  opt->basis = G1G2_SPIN_ORBITAL;
  opt->w_is_real = 0;
  opt->sym_tol = 1e-10;
  opt->cuda_stream = nullptr;
  opt->statistics = G1G2_FERMIONS;
}

const char *g1g2_strerror(int code) {
  switch (code) {
    case G1G2_OK: return "ok";
    case G1G2_EINVAL: return "invalid argument";
    case G1G2_ESYMM: return "input violates the symmetries of w, G1 or G2";
    case G1G2_ENOMEM: return "device allocation failed";
    case G1G2_ECUDA: return "CUDA error";
    case G1G2_ENONFINITE: return "state or input contains NaN or Inf";
    case G1G2_ETIMEOUT: return "bounded device wait timed out";
    case G1G2_EUNSUPPORTED: return "not supported by this build";
    default: return "unknown error code";
  }
}

const char *g1g2_last_error_detail(void) { return g_detail.c_str(); }

long long g1g2_launch_count(const g1g2_ctx *c) { return c ? c->launches : -1; }

int g1g2_profile(g1g2_ctx *c, int enable) {
  if (!c) return fail(G1G2_EINVAL, "ctx is NULL");
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "profile sync");
  if (rc) return rc;
  c->prof.clear();
  c->prof.on = enable != 0;
  return G1G2_OK;
}

int g1g2_profile_report(g1g2_ctx *c, g1g2_kernel_stat *out, int max_entries, int *n_entries) {
  if (!c || !n_entries || (max_entries > 0 && !out)) return fail(G1G2_EINVAL, "NULL argument");
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "profile sync");
  if (rc) return rc;
  std::vector<std::string> names;
  std::vector<long long> counts;
  std::vector<double> ms;
  for (const Profiler::Rec &r : c->prof.recs) {
    float t = 0.f;
    if ((rc = cuda_check(cudaEventElapsedTime(&t, c->prof.pool[r.start], c->prof.pool[r.stop]), "event time")))
      return rc;
    size_t k = 0;
    while (k < names.size() && names[k] != r.tag) ++k;
    if (k == names.size()) { names.push_back(r.tag); counts.push_back(0); ms.push_back(0.0); }
    ++counts[k];
    ms[k] += t;
  }
  const int n = (int)names.size();
  for (int k = 0; k < n && k < max_entries; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, names[k].c_str(), sizeof(out[k].name) - 1);
    out[k].launches = counts[k];
    out[k].total_ms = ms[k];
  }
  *n_entries = n < max_entries ? n : max_entries;
  return G1G2_OK;
}

void g1g2_destroy(g1g2_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->tc) tc_destroy(c->tc);
  for (void *p : c->adj_allocs) cudaFree(p);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

int g1g2_init(g1g2_ctx **out, int nb, const double *h, const double *w, const double *G1_0, const double *G2_0,
              int se, const g1g2_options *opt_in) {
  if (!out) return fail(G1G2_EINVAL, "out is NULL");
  *out = nullptr;
  g1g2_options opt;
  g1g2_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (nb < 1 || nb > 128) return fail(G1G2_EINVAL, "nb must be in [1, 128]");
  if (!h || !w || !G1_0) return fail(G1G2_EINVAL, "h, w and G1_0 must be non-NULL");
  if (se < G1G2_HF || se > G1G2_DSL) return fail(G1G2_EINVAL, "bad selfenergy");
  if ((se == G1G2_TPP || se == G1G2_TPH || se == G1G2_DSL) && opt.precision == G1G2_TF32X3)
    return fail(G1G2_EUNSUPPORTED, "the ladder terms run on the FP64 and BF16-slice forms");
  // GW with exchange is GW with the source term Psi^± (w^- in Psi)
  const bool gw_exchange = se == G1G2_GW_EXCHANGE;
  if (gw_exchange) se = G1G2_GW;
  if (opt.precision != G1G2_FP64 && opt.precision != G1G2_TF32X3 && opt.precision != G1G2_BF16X4)
    return fail(G1G2_EINVAL, "bad precision");
  if (opt.basis != G1G2_SPIN_ORBITAL && opt.basis != G1G2_SPIN_RESTRICTED) return fail(G1G2_EINVAL, "bad basis");
  if (opt.statistics != G1G2_FERMIONS && opt.statistics != G1G2_BOSONS) return fail(G1G2_EINVAL, "bad statistics");
  const bool bosons = opt.statistics == G1G2_BOSONS;
  if (bosons && opt.basis == G1G2_SPIN_RESTRICTED)
    return fail(G1G2_EINVAL, "the spin-restricted mode is the fermion Hubbard form; bosons run in the spin-orbital basis");
  // GW in the spin-restricted basis: only the Hubbard form, which carries the same-spin block
  // besides the opposite-spin one (Eqs. g2-gw-hubbard1/2); GW with exchange and DSL have none
  const bool restricted_gw = opt.basis == G1G2_SPIN_RESTRICTED && se == G1G2_GW && !gw_exchange;
  if (opt.basis == G1G2_SPIN_RESTRICTED && (se == G1G2_DSL || gw_exchange))
    return fail(G1G2_EINVAL, "GW couples same-spin components and has no general spin-restricted form");
  if (restricted_gw) {
    if (opt.precision != G1G2_FP64)
      return fail(G1G2_EUNSUPPORTED, "spin-restricted GW runs the Hubbard form in FP64");
    const size_t M = nb;
    bool onsite = true;
    for (size_t i = 0; i < M && onsite; ++i)
      for (size_t j = 0; j < M && onsite; ++j)
        for (size_t k = 0; k < M && onsite; ++k)
          for (size_t l = 0; l < M; ++l) {
            const size_t e = ((i * M + j) * M + k) * M + l;
            const double re = opt.w_is_real ? w[e] : w[2 * e], im = opt.w_is_real ? 0.0 : w[2 * e + 1];
            if (im != 0.0 || (!(i == j && j == k && k == l) && re != 0.0)) { onsite = false; break; }
          }
    if (!onsite)
      return fail(G1G2_EINVAL, "GW has a spin-restricted form only in the Hubbard basis (real on-site w)");
  }

  const size_t N = nb, N2 = N * N, N4 = N2 * N2;
  const bool restricted = opt.basis == G1G2_SPIN_RESTRICTED;
  // non-finite host inputs are refused before they reach the device
  {
    struct In { const double *p; size_t len; const char *name; };
    const In ins[4] = {{h, 2 * N2, "h"}, {w, (opt.w_is_real ? 1 : 2) * N4, "w"}, {G1_0, 2 * N2, "G1_0"},
                       {G2_0, G2_0 ? 2 * N4 : 0, "G2_0"}};
    for (const In &x : ins)
      if (!all_finite(x.p, x.len)) return fail(G1G2_ENONFINITE, std::string(x.name) + " contains NaN or Inf");
  }
  auto wv = [&](size_t idx) -> zc { return opt.w_is_real ? zc(w[idx], 0.0) : hz(w, idx); };
  auto at4 = [&](size_t i, size_t j, size_t k, size_t l) { return ((i * N + j) * N + k) * N + l; };

  // --- symmetry validation (Eqs. wsymm_a/b, Gsymm_a/b, n Hermitian) ---
  if (opt.sym_tol >= 0) {
    double wmax = 0, werr = 0;
    for (size_t i = 0; i < N; ++i)
      for (size_t j = 0; j < N; ++j)
        for (size_t k = 0; k < N; ++k)
          for (size_t l = 0; l < N; ++l) {
            const zc a = wv(at4(i, j, k, l));
            wmax = std::max(wmax, std::abs(a));
            werr = std::max(werr, std::abs(a - wv(at4(j, i, l, k))));
            werr = std::max(werr, std::abs(a - std::conj(wv(at4(k, l, i, j)))));
          }
    if (werr > opt.sym_tol * std::max(1.0, wmax))
      return fail(G1G2_ESYMM, "w violates w_ijkl = w_jilk or w_ijkl = conj(w_klij) by " + std::to_string(werr));
    double herr = 0, hmax = 0, nerr = 0, nmax = 0;
    for (size_t i = 0; i < N; ++i)
      for (size_t j = 0; j < N; ++j) {
        hmax = std::max(hmax, std::abs(hz(h, i * N + j)));
        herr = std::max(herr, std::abs(hz(h, i * N + j) - std::conj(hz(h, j * N + i))));
        nmax = std::max(nmax, std::abs(hz(G1_0, i * N + j)));
        nerr = std::max(nerr, std::abs(hz(G1_0, i * N + j) - std::conj(hz(G1_0, j * N + i))));
      }
    if (herr > opt.sym_tol * std::max(1.0, hmax)) return fail(G1G2_ESYMM, "h is not Hermitian");
    if (nerr > opt.sym_tol * std::max(1.0, nmax)) return fail(G1G2_ESYMM, "G1_0 is not Hermitian");
    if (G2_0) {
      double gmax = 0, gerr = 0;
      for (size_t i = 0; i < N; ++i)
        for (size_t j = 0; j < N; ++j)
          for (size_t k = 0; k < N; ++k)
            for (size_t l = 0; l < N; ++l) {
              const zc a = hz(G2_0, at4(i, j, k, l));
              gmax = std::max(gmax, std::abs(a));
              if (!restricted) gerr = std::max(gerr, std::abs(a - hz(G2_0, at4(j, i, l, k))));
              gerr = std::max(gerr, std::abs(a - std::conj(hz(G2_0, at4(k, l, i, j)))));
            }
      if (gerr > opt.sym_tol * std::max(1.0, gmax)) return fail(G1G2_ESYMM, "G2_0 violates Eqs. (Gsymm_a/b)");
    }
  }

  g1g2_ctx *c = new (std::nothrow) g1g2_ctx;
  if (!c) return fail(G1G2_ENOMEM, "host allocation failed");
  c->nb = nb; c->se = se; c->prec = opt.precision; c->basis = opt.basis;
  c->eta = bosons ? 1.0 : -1.0;
  c->hub_gw = restricted_gw;
  c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
  int rc = G1G2_OK;
  auto bail = [&](int code) { g1g2_destroy(c); return code; };

  // --- host-side layouts ---
  std::vector<cplx> hw(N4), hsrc(N4), hP(N4), tmp2(N2);
  bool real = true;
  for (size_t i = 0; i < N4; ++i) {
    const zc a = wv(i);
    hw[i] = {a.real(), a.imag()};
    if (a.imag() != 0.0) real = false;
  }
  c->w_real = real;
  // source interaction: w^± (SOA, T matrices, DSL, GW with exchange; spin-orbital), else w
  const bool use_pm =
      (se == G1G2_SOA || se == G1G2_TPP || se == G1G2_TPH || se == G1G2_DSL || gw_exchange) && !restricted;
  const double eta = bosons ? 1.0 : -1.0;
  c->src_pm = use_pm;
  for (size_t i = 0; i < N; ++i)
    for (size_t j = 0; j < N; ++j)
      for (size_t k = 0; k < N; ++k)
        for (size_t l = 0; l < N; ++l) {
          zc a = wv(at4(i, j, k, l));
          if (use_pm) a += eta * wv(at4(i, j, l, k));
          hsrc[at4(i, j, k, l)] = {a.real(), a.imag()};
          // collision layout wP[(l,p)][i][k] = w_iklp: here (i,k,l,p) = (i,j,k,l) renamed
          const zc b = wv(at4(i, j, k, l));        // w_{i j k l} with j->k', k->l', l->p'
          hP[((k * N + l) * N + i) * N + j] = {b.real(), b.imag()};
        }
  // Hartree-Fock matrix Wm[(ij),(lk)] = w_ikjl ± w_iklj = w^±_ikjl (restricted: w_ikjl)
  std::vector<double> WmR;
  std::vector<cplx> WmC;
  if (real) WmR.resize(N4); else WmC.resize(N4);
  for (size_t i = 0; i < N; ++i)
    for (size_t j = 0; j < N; ++j)
      for (size_t l = 0; l < N; ++l)
        for (size_t k = 0; k < N; ++k) {
          zc a = wv(at4(i, k, j, l));
          if (!restricted) a += eta * wv(at4(i, k, l, j));
          const size_t e = (i * N + j) * N2 + l * N + k;
          if (real) WmR[e] = a.real(); else WmC[e] = {a.real(), a.imag()};
        }

  // --- device buffers ---
  if ((rc = dalloc(c, &c->h, N2)) || (rc = dalloc(c, &c->D, N2)) || (rc = dalloc(c, &c->n, N2)) ||
      (rc = dalloc(c, &c->ns, N2)) || (rc = dalloc(c, &c->ns2, N2)) || (rc = dalloc(c, &c->nacc, N2)) || (rc = dalloc(c, &c->hhf, N2)) ||
      (rc = dalloc(c, &c->nbar, N2)) || (rc = dalloc(c, &c->I, N2)) || (rc = dalloc(c, &c->ntr, N2)) ||
      (rc = dalloc(c, &c->red, 256)) || (rc = dalloc(c, &c->W_dev, 1)) || (rc = dalloc(c, &c->w, N4)) ||
      (rc = dalloc(c, &c->G, N4)))
    return bail(rc);
  if (real) { double *p; if ((rc = dalloc(c, &p, N4))) return bail(rc); c->Wm = p; }
  else { cplx *p; if ((rc = dalloc(c, &p, N4))) return bail(rc); c->Wm = p; }
  const long long tiles = (long long)((N2 + 31) / 32) * ((N2 + 31) / 32);
  if ((rc = dalloc(c, &c->obs_partials, 2 * tiles))) return bail(rc);
  const bool correlated = se != G1G2_HF;
  if (correlated && c->prec == G1G2_FP64) {
    if ((rc = dalloc(c, &c->Gs, N4)) || (rc = dalloc(c, &c->Gacc, N4)) || (rc = dalloc(c, &c->wsrc, N4)) ||
        (rc = dalloc(c, &c->wP, N4)) || (rc = dalloc(c, &c->Cb, N4)) || (rc = dalloc(c, &c->T1, N4)) ||
        (rc = dalloc(c, &c->T2, N4)) || (rc = dalloc(c, &c->Ab, N4)))
      return bail(rc);
    c->splits = 4 * 152;
    if ((rc = dalloc(c, &c->partial, (size_t)c->splits * N2))) return bail(rc);
    if ((se == G1G2_GW && !restricted_gw) || se == G1G2_TPH || se == G1G2_DSL) {
      if ((rc = dalloc(c, &c->Hb, N4)) || (rc = dalloc(c, &c->Gp, N4)) || (rc = dalloc(c, &c->Hp, N4)) ||
          (rc = dalloc(c, &c->Pp, N4)))
        return bail(rc);
    }
    if (se == G1G2_TPP && (rc = dalloc(c, &c->Hb, N4))) return bail(rc);
    if (restricted_gw && ((rc = dalloc(c, &c->Gss, N4)) || (rc = dalloc(c, &c->Gss_s, N4)) ||
                          (rc = dalloc(c, &c->Gss_acc, N4)) || (rc = dalloc(c, &c->Cb2, N4))))
      return bail(rc);
    if (restricted_gw && (rc = cuda_check(cudaMemsetAsync(c->Gss, 0, N4 * sizeof(cplx), c->stream), "memset")))
      return bail(rc);
  }
  // uploads
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream), "upload");
  };
  for (size_t i = 0; i < N2; ++i) tmp2[i] = {h[2 * i], h[2 * i + 1]};
  if ((rc = up(c->h, tmp2.data(), N2 * sizeof(cplx)))) return bail(rc);
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "sync"))) return bail(rc);
  if ((rc = up(c->n, G1_0, N2 * sizeof(cplx)))) return bail(rc);
  if ((rc = up(c->w, hw.data(), N4 * sizeof(cplx)))) return bail(rc);
  if (correlated && c->prec != G1G2_FP64 && real) {
    // tensor-core forms (real w only): Wm as (hi, lo) FP32 pairs for the double-single
    // h^HF build, in place (entry e's pair takes the bytes of entry e)
    c->wm_ds = true;
    cplx *ns_buf = nullptr;
    if ((rc = dalloc(c, &ns_buf, N2))) return bail(rc);
    c->nsplit = reinterpret_cast<float4 *>(ns_buf);
    auto split = [](double x, float *out) {
      out[0] = (float)x;
      out[1] = (float)(x - (double)out[0]);
    };
    for (size_t e = 0; e < N4; ++e) {
      float v[2];
      split(WmR[e], v);
      std::memcpy(&WmR[e], v, sizeof(v));
    }
  }
  if (real) { if ((rc = up(c->Wm, WmR.data(), N4 * sizeof(double)))) return bail(rc); }
  else { if ((rc = up(c->Wm, WmC.data(), N4 * sizeof(cplx)))) return bail(rc); }
  if (G2_0) { if ((rc = up(c->G, G2_0, N4 * sizeof(cplx)))) return bail(rc); }
  else if ((rc = cuda_check(cudaMemsetAsync(c->G, 0, N4 * sizeof(cplx), c->stream), "memset"))) return bail(rc);
  if ((rc = cuda_check(cudaMemsetAsync(c->W_dev, 0, sizeof(double), c->stream), "memset"))) return bail(rc);
  if ((rc = cuda_check(cudaMemsetAsync(c->D, 0, N2 * sizeof(cplx), c->stream), "memset"))) return bail(rc);
  if (correlated && c->prec == G1G2_FP64) {
    if ((rc = up(c->wsrc, hsrc.data(), N4 * sizeof(cplx)))) return bail(rc);
    if ((rc = up(c->wP, hP.data(), N4 * sizeof(cplx)))) return bail(rc);
  }
  // Hubbard basis: spin-restricted SOA with an on-site interaction w_ijkl = U_i d(i=j=k=l)
  if ((se == G1G2_SOA || restricted_gw) && restricted && !bosons && c->prec == G1G2_FP64 && real) {
    bool onsite = true;
    std::vector<double> Ui(N);
    for (size_t i = 0; i < N && onsite; ++i)
      for (size_t j = 0; j < N && onsite; ++j)
        for (size_t k = 0; k < N && onsite; ++k)
          for (size_t l = 0; l < N; ++l) {
            const double v = hw[at4(i, j, k, l)].x;
            if (i == j && j == k && k == l) Ui[i] = v;
            else if (v != 0.0) { onsite = false; break; }
          }
    if (onsite) {
      c->hub_hpat.assign(N2, 0);
      for (size_t e = 0; e < N2; ++e) c->hub_hpat[e] = (h[2 * e] != 0.0 || h[2 * e + 1] != 0.0);
      if ((rc = dalloc(c, &c->hub_U, N)) || (rc = dalloc(c, &c->hub_rp, N + 1)) || (rc = dalloc(c, &c->hub_ci, N2)))
        return bail(rc);
      if ((rc = up(c->hub_U, Ui.data(), N * sizeof(double)))) return bail(rc);
      if ((rc = hub_upload_pattern(c, nullptr))) return bail(rc);
      c->hub_ok = c->hub_on = true;
    }
  }
  if (restricted_gw && !c->hub_ok) return bail(fail(G1G2_EINVAL, "spin-restricted GW needs the Hubbard form"));
  if (correlated && c->prec != G1G2_FP64) {
    if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "init sync"))) return bail(rc);
    g_detail.clear();
    rc = tc_create(&c->tc, nb, se, restricted, c->prec == G1G2_BF16X4, bosons, hw.data(), hsrc.data(), c->stream);
    if (rc) return bail(rc);
    Launcher L = c->launcher();
    tc_load_state(c->tc, L, c->G);
    if ((rc = launch_status(L, "tensor-core state"))) return bail(rc);
  }
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "init sync"))) return bail(rc);
  *out = c;
  return G1G2_OK;
}

// w_ijkl = sum_P L^P_ik L^P_jl expanded on the device (the pair product C_(ik),(jl) and one
// index permutation), then the context of g1g2_init on that w; FP64 contexts with a correlated
// selfenergy keep the factors for the factorised source term (source_A_factorised).
int g1g2_init_factorised(g1g2_ctx **out, int nb, const double *h, const double *Lh, int nfac, const double *G1_0,
                         const double *G2_0, int se, const g1g2_options *opt_in) {
  if (!out) return fail(G1G2_EINVAL, "out is NULL");
  *out = nullptr;
  if (nb < 1 || nb > 128) return fail(G1G2_EINVAL, "nb must be in [1, 128]");
  if (!h || !Lh || !G1_0) return fail(G1G2_EINVAL, "h, L and G1_0 must be non-NULL");
  if (se < G1G2_HF || se > G1G2_DSL) return fail(G1G2_EINVAL, "bad selfenergy");
  if (nfac < 1 || (long long)nfac > (long long)nb * nb) return fail(G1G2_EINVAL, "nfac must be in [1, nb^2]");
  g1g2_options opt;
  g1g2_default_options(&opt);
  if (opt_in) opt = *opt_in;
  const size_t N2 = (size_t)nb * nb, N4 = N2 * N2, NL = (size_t)nfac * N2;
  if (!all_finite(Lh, (opt.w_is_real ? 1 : 2) * NL)) return fail(G1G2_ENONFINITE, "L contains NaN or Inf");
  std::vector<cplx> hL(NL);
  for (size_t e = 0; e < NL; ++e) hL[e] = opt.w_is_real ? cplx{Lh[e], 0.0} : cplx{Lh[2 * e], Lh[2 * e + 1]};
  // each factor Hermitian or i times Hermitian (then w meets Eqs. wsymm_a/b), checked on the host
  if (opt.sym_tol >= 0) {
    for (int P = 0; P < nfac; ++P) {
      const cplx *f = hL.data() + (size_t)P * N2;
      double fmax = 0, eh = 0, ea = 0;
      for (int i = 0; i < nb; ++i)
        for (int k = 0; k < nb; ++k) {
          const cplx a = f[(size_t)i * nb + k], b = f[(size_t)k * nb + i];  // b = L_ki
          fmax = std::max(fmax, std::hypot(a.x, a.y));
          eh = std::max(eh, std::hypot(a.x - b.x, a.y + b.y));   // |L_ik - conj(L_ki)|
          ea = std::max(ea, std::hypot(a.x + b.x, a.y - b.y));   // |L_ik + conj(L_ki)|
        }
      if (std::min(eh, ea) > opt.sym_tol * std::max(1.0, fmax))
        return fail(G1G2_ESYMM, "factor " + std::to_string(P) + " is neither Hermitian nor i times Hermitian");
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(opt.cuda_stream);
  cplx *dL = nullptr, *dC = nullptr, *dW = nullptr;
  auto alloc = [](cplx **p, size_t count) -> int {
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(cplx)) != cudaSuccess) {
      cudaGetLastError();
      return fail(G1G2_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(cplx)) + " bytes failed");
    }
    *p = static_cast<cplx *>(q);
    return G1G2_OK;
  };
  auto release = [&]() {
    if (dL) cudaFree(dL);
    if (dC) cudaFree(dC);
    if (dW) cudaFree(dW);
    dL = dC = dW = nullptr;
  };
  int rc = G1G2_OK;
  if ((rc = alloc(&dL, NL)) || (rc = alloc(&dC, N4)) || (rc = alloc(&dW, N4))) {
    release();
    return rc;
  }
  std::vector<double> hw;
  rc = cuda_check(cudaMemcpyAsync(dL, hL.data(), NL * sizeof(cplx), cudaMemcpyHostToDevice, s), "factor upload");
  if (!rc) {
    Launcher L;
    L.stream = s;
    ZGemm g;  // C_(ik),(jl) = sum_P L^P_(ik) L^P_(jl)
    g.M = (int)N2; g.N = (int)N2; g.K = nfac;
    g.A = dL; g.sa_m = 1; g.sa_k = (long long)N2;
    g.B = dL; g.sb_k = (long long)N2; g.sb_n = 1;
    g.C = dC; g.sc_m = (long long)N2; g.sc_n = 1;
    zgemm(L, g);
    const int p[4] = {0, 2, 1, 3};  // w(i,j,k,l) = C(i,k,j,l)
    permute4(L, nb, dC, dW, p, {1.0, 0.0}, 0.0, false);
    rc = launch_status(L, "factorised interaction");
  }
  if (!rc) {
    hw.resize(2 * N4);
    rc = cuda_check(cudaMemcpyAsync(hw.data(), dW, N4 * sizeof(cplx), cudaMemcpyDeviceToHost, s), "w download");
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "factorised interaction sync");
  cudaFree(dC);
  cudaFree(dW);
  dC = dW = nullptr;
  if (rc) {
    release();
    return rc;
  }
  g1g2_options o2 = opt;
  o2.w_is_real = 0;
  rc = g1g2_init(out, nb, h, hw.data(), G1_0, G2_0, se, &o2);
  if (rc) {
    release();
    return rc;
  }
  g1g2_ctx *c = *out;
  if (c->T1 && c->Ab) {  // FP64 form with a source term
    c->allocs.push_back(dL);
    c->Lf = dL;
    dL = nullptr;
    c->nfac = nfac;
    if ((rc = dalloc(c, &c->LfN, NL)) || (rc = dalloc(c, &c->Mf, NL))) {
      g1g2_destroy(c);
      *out = nullptr;
      return rc;
    }
  }
  release();
  return G1G2_OK;
}

int g1g2_set_drive(g1g2_ctx *c, const double *D, int kind, const double *params, int nparams) {
  if (!c) return fail(G1G2_EINVAL, "ctx is NULL");
  if (kind == 0) {
    c->drive_kind = 0;
    c->hasD = false;
    return G1G2_OK;
  }
  if (!D || !params) return fail(G1G2_EINVAL, "D and params must be non-NULL");
  if (kind == 1 && nparams != 4) return fail(G1G2_EINVAL, "gauss-sine drive takes 4 parameters");
  if (kind == 2 && (nparams < 4 || params[1] <= params[0]))
    return fail(G1G2_EINVAL, "piecewise-linear drive takes ta < tb and at least 2 values");
  if (kind != 1 && kind != 2) return fail(G1G2_EINVAL, "bad drive kind");
  if (kind == 1 && params[3] == 0.0) return fail(G1G2_EINVAL, "sigma must be nonzero");
  const size_t N2 = (size_t)c->nb * c->nb;
  if (!all_finite(D, 2 * N2) || !all_finite(params, (size_t)nparams))
    return fail(G1G2_ENONFINITE, "D or the drive parameters contain NaN or Inf");
  int rc = cuda_check(cudaMemcpyAsync(c->D, D, N2 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "drive upload");
  if (rc) return rc;
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "drive sync"))) return rc;
  if (c->hub_ok) {  // the drive's nonzeros join the pattern of h^HF
    std::vector<cplx> Dh(N2);
    for (size_t e = 0; e < N2; ++e) Dh[e] = {D[2 * e], D[2 * e + 1]};
    if ((rc = hub_upload_pattern(c, &Dh))) return rc;
  }
  c->drive_kind = kind;
  c->drive_params.assign(params, params + nparams);
  c->hasD = true;
  return G1G2_OK;
}

int g1g2_rhs(g1g2_ctx *c, double t, const double *n_dev, const double *G2_dev, double *dn_dev, double *dG2_dev) {
  if (!c || !n_dev || !dn_dev) return fail(G1G2_EINVAL, "NULL argument");
  if (c->se != G1G2_HF && (!G2_dev || !dG2_dev)) return fail(G1G2_EINVAL, "G2 and dG2 must be non-NULL");
  if (c->hub_gw)
    return fail(G1G2_EUNSUPPORTED, "spin-restricted GW keeps its same-spin block in the context: use g1g2_step");
  Launcher L = c->launcher();
  Rk4Stage st{-1, 0.0};
  StageOut o{nullptr, nullptr, nullptr, reinterpret_cast<cplx *>(dn_dev),
             nullptr, nullptr, nullptr, reinterpret_cast<cplx *>(dG2_dev)};
  rhs_dispatch(c, L, t, reinterpret_cast<const cplx *>(n_dev), reinterpret_cast<const cplx *>(G2_dev), st, o);
  if (c->se == G1G2_HF && dG2_dev) {
    const size_t N4 = (size_t)c->nb * c->nb * c->nb * c->nb;
    int rc = cuda_check(cudaMemsetAsync(dG2_dev, 0, N4 * sizeof(cplx), c->stream), "memset dG2");
    if (rc) return rc;
  }
  return launch_status(L, "rhs");
}

int g1g2_step(g1g2_ctx *c, double dt) {
  if (!c) return fail(G1G2_EINVAL, "ctx is NULL");
  return rk4_step(c, dt);
}

int g1g2_observables(g1g2_ctx *c, g1g2_obs *out, double *density, double *dbl) {
  if (!c || !out) return fail(G1G2_EINVAL, "NULL argument");
  double bad = 0;
  int rc = observables_impl(c, out, density, &bad);
  if (rc) return rc;
  if (dbl) {
    if (c->basis != G1G2_SPIN_ORBITAL || c->nb % 2) return fail(G1G2_EINVAL, "double occupancy needs a spin-orbital basis");
    Launcher L = c->launcher();
    double_occ(L, c->nb, c->n, c->G, c->eta, c->red + 8);
    if ((rc = launch_status(L, "double occupancy"))) return rc;
    if ((rc = cuda_check(cudaMemcpyAsync(dbl, c->red + 8, sizeof(double) * (c->nb / 2), cudaMemcpyDeviceToHost,
                                         c->stream), "copy")))
      return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "sync"))) return rc;
  }
  return G1G2_OK;
}

int g1g2_propagate(g1g2_ctx *c, double dt, int nsteps, int obs_every, g1g2_obs *obs, double *density) {
  if (!c || nsteps < 0) return fail(G1G2_EINVAL, "bad argument");
  if ((obs || density) && obs_every <= 0) return fail(G1G2_EINVAL, "obs_every must be positive");
  NvtxRange range("g1g2 propagate");
  int rec = 0, rc;
  auto record = [&]() -> int {
    g1g2_obs o;
    double bad = 0;
    int r = observables_impl(c, &o, density ? density + (size_t)rec * c->nb : nullptr, &bad);
    if (r) return r;
    if (bad != 0) return fail(G1G2_ENONFINITE, "non-finite entries in G1 at t = " + std::to_string(c->t));
    if (obs) obs[rec] = o;
    ++rec;
    return G1G2_OK;
  };
  const bool recording = obs || density;
  if (recording && (rc = record())) return rc;
  for (int s = 0; s < nsteps; ++s) {
    if ((rc = rk4_step(c, dt))) return rc;
    if (recording && (s + 1) % obs_every == 0 && (rc = record())) return rc;
  }
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "propagate sync"))) return rc;
  return c->tc ? tc_error(c->tc, c->stream) : G1G2_OK;
}

// Original HF-GKBA with the SOA selfenergy, the memory-integral form the G1-G2
// equations were derived from (Sec. III.B): the correlated part at time t is
//   G2(t) = (i hbar)^3 int_{t0}^t dtb U2(t,tb) Psi(tb) U2(tb,t)   Eq. (dtilde-solution-short)
// with U2 = U (x) U (Eq. prop_two) and i hbar U(t,tb) = u(t) u(tb)^dag the Hartree-Fock
// propagator of the GKBA (Eqs. GKBA_propa/b), i du/dt = hHF u.  Every evaluation sums
// over the whole stored history (trapezoid rule): the O(N_t^2) cost of the standard
// scheme (Table I).  n and u advance by Heun's method; the memory sum at the predictor
// includes the predicted end point.  History entry k holds u(t_k) and Q_k = -i Psi(t_k),
// since (i hbar)^3 (i hbar)^-4 = -i.
int g1g2_propagate_hfgkba(g1g2_ctx *c, double dt, int nsteps, double *G1_history, size_t scratch_bytes) {
  if (!c || nsteps < 0 || !std::isfinite(dt)) return fail(G1G2_EINVAL, "bad argument");
  if (c->se != G1G2_SOA || c->prec != G1G2_FP64)
    return fail(G1G2_EUNSUPPORTED, "the memory-integral HF-GKBA covers SOA in the FP64 form");
  NvtxRange range("g1g2 hf-gkba propagate");
  if (c->hasD) return fail(G1G2_EUNSUPPORTED, "the memory-integral HF-GKBA runs without a drive");
  if (c->nb > mode_rotate_max_nb())
    return fail(G1G2_EUNSUPPORTED, "the memory-integral HF-GKBA keeps nb^4 per time step; nb <= " +
                                       std::to_string(mode_rotate_max_nb()));
  const int nb = c->nb;
  const long long N2 = (long long)nb * nb, N4 = N2 * N2;
  const long long slots = (long long)nsteps + 2;
  if (scratch_bytes == 0) scratch_bytes = (size_t)256 << 20;
  GkbaHist H;
  H.chunk = (int)std::max<long long>(
      1, std::min<long long>(std::min<long long>(slots, 65535LL), (long long)(scratch_bytes / (2 * N4 * sizeof(cplx)))));
  Launcher L = c->launcher();
  int rc;
  // the integral starts from an uncorrelated state
  if ((rc = cuda_check(cudaMemsetAsync(c->red, 0, sizeof(double), c->stream), "memset"))) return rc;
  count_nonzero(L, c->G, N4, c->red);
  double nz = 0;
  if ((rc = cuda_check(cudaMemcpyAsync(&nz, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "check")) ||
      (rc = cuda_check(cudaStreamSynchronize(c->stream), "check sync")))
    return rc;
  if (nz != 0) return fail(G1G2_EINVAL, "the memory integral starts from G2 = 0; the state has a nonzero G2");
  DevScratch S;
  cplx *nh, *np, *dn1, *dn2, *du1, *du2;
  if ((rc = S.get(&H.u, slots * N2)) || (rc = S.get(&H.Q, slots * N4)) || (rc = S.get(&H.V, slots * N2)) ||
      (rc = S.get(&H.Vs, slots * N2)) || (rc = S.get(&H.Y0, H.chunk * N4)) || (rc = S.get(&H.Y1, H.chunk * N4)) ||
      (rc = S.get(&nh, (slots - 1) * N2)) || (rc = S.get(&np, N2)) || (rc = S.get(&dn1, N2)) ||
      (rc = S.get(&dn2, N2)) || (rc = S.get(&du1, N2)) || (rc = S.get(&du2, N2)))
    return rc;
  std::vector<cplx> eye(N2, cplx{0.0, 0.0});
  for (int i = 0; i < nb; ++i) eye[(size_t)i * nb + i] = {1.0, 0.0};
  if ((rc = cuda_check(cudaMemcpyAsync(H.u, eye.data(), N2 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "u0")) ||
      (rc = cuda_check(cudaMemcpyAsync(nh, c->n, N2 * sizeof(cplx), cudaMemcpyDeviceToDevice, c->stream), "n0")) ||
      (rc = cuda_check(cudaMemsetAsync(c->Cb, 0, N4 * sizeof(cplx), c->stream), "zero")))
    return rc;
  gkba_source(c, L, nh, H.Q);
  gkba_memory(c, L, H, 1, H.u, dt, c->G);
  const cplx one{1.0, 0.0}, half{0.5 * dt, 0.0}, full{dt, 0.0};
  for (int m = 0; m < nsteps; ++m) {
    cplx *n0 = nh + m * N2, *n1 = nh + (m + 1) * N2, *u0 = H.u + m * N2, *u1 = H.u + (m + 1) * N2;
    cplx *Q1 = H.Q + (m + 1) * N4;
    gkba_derivs(c, L, n0, u0, c->G, dn1, du1);
    zaxpby(L, N2, one, n0, full, dn1, np);                 // predictor
    zaxpby(L, N2, one, u0, full, du1, u1);
    gkba_source(c, L, np, Q1);
    gkba_memory(c, L, H, m + 2, u1, dt, c->Gs);
    gkba_derivs(c, L, np, u1, c->Gs, dn2, du2);
    zaxpby(L, N2, one, n0, half, dn1, n1);                 // corrector
    zaxpby(L, N2, one, n1, half, dn2, n1);
    zaxpby(L, N2, one, u0, half, du1, u1);
    zaxpby(L, N2, one, u1, half, du2, u1);
    gkba_source(c, L, n1, Q1);
    gkba_memory(c, L, H, m + 2, u1, dt, c->G);
  }
  if ((rc = launch_status(L, "memory-integral HF-GKBA"))) return rc;
  if ((rc = cuda_check(cudaMemcpyAsync(c->n, nh + nsteps * N2, N2 * sizeof(cplx), cudaMemcpyDeviceToDevice, c->stream),
                       "state")))
    return rc;
  if (G1_history &&
      (rc = cuda_check(cudaMemcpyAsync(G1_history, nh, (size_t)(nsteps + 1) * N2 * sizeof(cplx), cudaMemcpyDeviceToHost,
                                       c->stream),
                       "history")))
    return rc;
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "memory-integral sync"))) return rc;
  c->t += nsteps * dt;
  return G1G2_OK;
}

int g1g2_get_state(g1g2_ctx *c, double *t, double *G1, double *G2) {
  if (!c) return fail(G1G2_EINVAL, "ctx is NULL");
  const size_t N2 = (size_t)c->nb * c->nb, N4 = N2 * N2;
  int rc;
  if (t) *t = c->t;
  if (G1 && (rc = cuda_check(cudaMemcpyAsync(G1, c->n, N2 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream), "get")))
    return rc;
  if (G2 && (rc = cuda_check(cudaMemcpyAsync(G2, c->G, N4 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream), "get")))
    return rc;
  return cuda_check(cudaStreamSynchronize(c->stream), "get sync");
}

int g1g2_rhs_vjp(g1g2_ctx *c, double t, const double *n_dev, const double *G2_dev, const double *dn_bar,
                 const double *dG2_bar, double *n_bar, double *G2_bar, double *h_bar) {
  if (!c || !n_dev || !G2_dev || !dn_bar || !dG2_bar || !n_bar || !G2_bar || !h_bar)
    return fail(G1G2_EINVAL, "NULL argument");
  if (c->prec != G1G2_FP64) return fail(G1G2_EUNSUPPORTED, "the vector-Jacobian product runs on the FP64 form");
  if (c->hub_gw) return fail(G1G2_EUNSUPPORTED, "the vector-Jacobian product covers the general basis");
  if (c->eta > 0) return fail(G1G2_EUNSUPPORTED, "the vector-Jacobian product covers fermions");
  const long long N2 = (long long)c->nb * c->nb, N4 = N2 * N2;
  if (!c->AE) {  // scratch of the adjoint
    void *p;
    int rc;
    for (cplx **b : {&c->AE, &c->AB1, &c->AB2}) {
      if ((rc = adj_alloc(c, c->adj_allocs, &p, N4 * sizeof(cplx)))) return rc;
      *b = (cplx *)p;
    }
    if (c->se == G1G2_HF) return fail(G1G2_EUNSUPPORTED, "call g1g2_adjoint once before the HF product");
  }
  Launcher L = c->launcher();
  vjp_fp64(c, L, t, reinterpret_cast<const cplx *>(n_dev), reinterpret_cast<const cplx *>(G2_dev),
           reinterpret_cast<const cplx *>(dn_bar), reinterpret_cast<const cplx *>(dG2_bar), reinterpret_cast<cplx *>(n_bar),
           reinterpret_cast<cplx *>(G2_bar), reinterpret_cast<cplx *>(h_bar));
  return launch_status(L, "rhs vjp");
}

// Checkpoint plan.  Every step is recomputed at most once whatever the
// interval k, so k only trades memory ((ceil(M/k) + 1) checkpoints and k + 1
// segment states) against recomputation ((k - 1)/k of a forward sweep).
// Device plan: the smallest k whose states fit in 80% of the free device
// memory (k = 1, no recomputation, when all fit), at most ceil(sqrt(M)) (the
// memory minimum).  Host plan (requested, or when no device plan fits): the
// checkpoints go to pinned host memory (at most half of the free host memory)
// and only the segment stays on the device; the smallest k that fits both.
struct AdjPlan {
  int k, where;
};
static AdjPlan adjoint_plan(int nsteps, size_t SB, int ckpt_every, int where_req) {
  const double sb = (double)SB;
  auto ckpt_bytes = [&](int k) { return (double)((nsteps + k - 1) / k + 1) * sb; };
  auto seg_bytes = [&](int k) { return (double)(k + 1) * sb; };
  size_t free_b = 0, total_b = 0;
  double dev = 0.0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) dev = 0.8 * (double)free_b - 8.0 * sb;  // minus stage buffers
  else cudaGetLastError();
  const long pages = sysconf(_SC_AVPHYS_PAGES), psz = sysconf(_SC_PAGESIZE);
  const double host = (pages > 0 && psz > 0) ? 0.5 * (double)pages * (double)psz : 0.0;
  const int kmem = std::max(1, (int)std::ceil(std::sqrt((double)nsteps)));
  if (ckpt_every > 0) {
    const int k = std::min(ckpt_every, nsteps);
    int where = where_req;
    if (where == G1G2_CKPT_AUTO) where = (ckpt_bytes(k) + seg_bytes(k) <= dev) ? G1G2_CKPT_DEVICE : G1G2_CKPT_HOST;
    return {k, where};
  }
  if (where_req != G1G2_CKPT_HOST) {
    for (int k = 1; k <= kmem; ++k)
      if (ckpt_bytes(k) + seg_bytes(k) <= dev) return {k, G1G2_CKPT_DEVICE};
    if (where_req == G1G2_CKPT_DEVICE) return {kmem, G1G2_CKPT_DEVICE};
  }
  for (int k = 1; k <= nsteps; ++k) {
    if (seg_bytes(k) > dev && k > 1) break;
    if (ckpt_bytes(k) <= host) return {k, G1G2_CKPT_HOST};
  }
  return {kmem, G1G2_CKPT_HOST};
}

int g1g2_set_hubbard_path(g1g2_ctx *c, int enable) {
  if (!c) return fail(G1G2_EINVAL, "ctx is NULL");
  if (!enable && c->hub_gw) return fail(G1G2_EUNSUPPORTED, "spin-restricted GW runs only in the Hubbard form");
  if (enable && !c->hub_ok)
    return fail(G1G2_EUNSUPPORTED, "the O(nb^4) path needs spin-restricted SOA, the FP64 form and an on-site w");
  c->hub_on = enable != 0;
  return G1G2_OK;
}

int g1g2_hubbard_path(const g1g2_ctx *c) { return c ? (c->hub_on ? 1 : 0) : G1G2_EINVAL; }

int g1g2_fp64_rate(double *tflops) {
  if (!tflops) return fail(G1G2_EINVAL, "tflops is NULL");
  int err = 0;
  *tflops = dfma_rate(nullptr, &err);
  return err ? fail(G1G2_ECUDA, "FP64 rate probe failed") : G1G2_OK;
}

int g1g2_wait_selftest(int limit_us) {
  if (limit_us < 1 || limit_us > 10000000) return fail(G1G2_EINVAL, "limit must be 1 us .. 10 s");
  return tc_wait_selftest(1000ull * (unsigned long long)limit_us, nullptr);
}

int g1g2_set_adjoint_checkpoints(g1g2_ctx *c, int where) {
  if (!c) return fail(G1G2_EINVAL, "ctx is NULL");
  if (where != G1G2_CKPT_AUTO && where != G1G2_CKPT_DEVICE && where != G1G2_CKPT_HOST)
    return fail(G1G2_EINVAL, "checkpoint location must be AUTO, DEVICE or HOST");
  c->adj_where = where;
  return G1G2_OK;
}

int g1g2_adjoint_plan(const g1g2_ctx *c, int *ckpt_every, int *where) {
  if (!c || !ckpt_every || !where) return fail(G1G2_EINVAL, "NULL argument");
  *ckpt_every = c->adj_last_k;
  *where = c->adj_last_where;
  return G1G2_OK;
}

int g1g2_adjoint(g1g2_ctx *c, double dt, int nsteps, int ckpt_every, int objective, double *J_out,
                 double *grad_drive, double *grad_wscale, double *grad_h, double *grad_w) {
  if (!c || nsteps < 1 || !J_out) return fail(G1G2_EINVAL, "bad adjoint argument");
  if (c->prec != G1G2_FP64) return fail(G1G2_EUNSUPPORTED, "the discrete adjoint runs on the FP64 form");
  NvtxRange range("g1g2 adjoint");
  if (c->hub_gw) return fail(G1G2_EUNSUPPORTED, "the discrete adjoint covers the general basis");
  if (c->eta > 0) return fail(G1G2_EUNSUPPORTED, "the discrete adjoint covers fermions");
  if (objective < 0 || objective > 2) return fail(G1G2_EINVAL, "objective must be 0, 1 or 2");
  if (objective == 0 && (c->basis != G1G2_SPIN_ORBITAL || c->nb % 2))
    return fail(G1G2_EINVAL, "double occupancy needs a spin-orbital basis with index 2*site+spin");
  const int nb = c->nb;
  const long long N = nb, N2 = N * N, N4 = N2 * N2;
  const size_t SB = (N2 + N4) * sizeof(cplx);  // one stored state (n, G2)
  const AdjPlan plan = adjoint_plan(nsteps, SB, ckpt_every, c->adj_where);
  const int k = plan.k;
  const bool host_ckpt = plan.where == G1G2_CKPT_HOST;
  c->adj_last_k = k;
  c->adj_last_where = plan.where;
  const int nseg = (nsteps + k - 1) / k;
  const bool restricted = c->basis == G1G2_SPIN_RESTRICTED;
  const double sfac = restricted ? 2.0 : 1.0;
  int rc;
  Launcher L = c->launcher();
  std::vector<void *> own;  // per-call memory
  void *host_ckpt_mem = nullptr;
  auto done = [&](int code) {
    cudaStreamSynchronize(c->stream);  // no copy may still read or write the checkpoints
    for (void *q : own) cudaFree(q);
    if (host_ckpt_mem) cudaFreeHost(host_ckpt_mem);
    return code;
  };
  // persistent adjoint scratch
  if (!c->AE) {
    void *p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N4 * sizeof(cplx)))) return rc;
    c->AE = (cplx *)p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N4 * sizeof(cplx)))) return rc;
    c->AB1 = (cplx *)p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N4 * sizeof(cplx)))) return rc;
    c->AB2 = (cplx *)p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N2 * sizeof(cplx)))) return rc;
    c->zero_h = (cplx *)p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, 1024 * sizeof(double)))) return rc;
    c->adj_red = (double *)p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N2 * sizeof(cplx)))) return rc;
    c->adj_hsum = (cplx *)p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N2 * sizeof(cplx)))) return rc;
    c->adj_hbar = (cplx *)p;
    cudaMemsetAsync(c->zero_h, 0, N2 * sizeof(cplx), c->stream);
    if (c->se == G1G2_HF) {  // the correlated buffers the adjoint touches
      for (cplx **b : {&c->Gs, &c->Gacc, &c->wsrc, &c->wP, &c->Cb, &c->T1, &c->T2, &c->Ab})
        if (!*b) {
          if ((rc = adj_alloc(c, c->adj_allocs, &p, N4 * sizeof(cplx)))) return rc;
          *b = (cplx *)p;
          cudaMemsetAsync(p, 0, N4 * sizeof(cplx), c->stream);
        }
      if (!c->partial) {
        c->splits = 4 * 152;
        if ((rc = adj_alloc(c, c->adj_allocs, &p, (size_t)c->splits * N2 * sizeof(cplx)))) return rc;
        c->partial = (cplx *)p;
      }
    }
  }
  // per-call memory: checkpoints, one segment of states, stage inputs, cotangents
  auto state_n = [&](void *base) { return (cplx *)base; };
  auto state_G = [&](void *base) { return (cplx *)base + N2; };
  void *ckpt, *seg, *Y2, *Y3, *Y4, *lam, *lam2, *kbar, *Ybar, *kk, *acc;
  if (host_ckpt) {
    if (cudaHostAlloc(&host_ckpt_mem, SB * (nseg + 1), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return done(fail(G1G2_ENOMEM, "adjoint: pinned host memory for " + std::to_string(nseg + 1) +
                                        " checkpoints failed"));
    }
    ckpt = host_ckpt_mem;
  } else if ((rc = adj_alloc(c, own, &ckpt, SB * (nseg + 1)))) {
    return done(rc);
  }
  if ((rc = adj_alloc(c, own, &seg, SB * (k + 1))) ||
      (rc = adj_alloc(c, own, &Y2, SB)) || (rc = adj_alloc(c, own, &Y3, SB)) || (rc = adj_alloc(c, own, &Y4, SB)) ||
      (rc = adj_alloc(c, own, &lam, SB)) || (rc = adj_alloc(c, own, &lam2, SB)) ||
      (rc = adj_alloc(c, own, &kbar, SB)) || (rc = adj_alloc(c, own, &Ybar, SB)) || (rc = adj_alloc(c, own, &kk, SB)) ||
      (rc = adj_alloc(c, own, &acc, sizeof(double) * (1 + 4 * (size_t)nsteps))))
    return done(rc);
  if (grad_w && !c->adj_wbar) {
    void *p;
    if ((rc = adj_alloc(c, c->adj_allocs, &p, N4 * sizeof(cplx)))) return done(rc);
    c->adj_wbar = (cplx *)p;
  }
  if (grad_w) cudaMemsetAsync(c->adj_wbar, 0, N4 * sizeof(cplx), c->stream);
  double *dacc = (double *)acc;
  cudaMemsetAsync(dacc, 0, sizeof(double) * (1 + 4 * (size_t)nsteps), c->stream);
  cudaMemsetAsync(c->adj_hsum, 0, N2 * sizeof(cplx), c->stream);
  // checkpoints may live in pinned host memory: copies use the unified address space
  auto copy_state = [&](void *dst, const cplx *n, const cplx *G) {
    cudaMemcpyAsync(state_n(dst), n, N2 * sizeof(cplx), cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(state_G(dst), G, N4 * sizeof(cplx), cudaMemcpyDefault, c->stream);
  };
  auto at = [&](void *base, long long i) { return (void *)((char *)base + SB * i); };
  // ---- forward sweep with checkpoints (the state at step m*k is kept)
  const double t0 = c->t;
  double E0 = 0.0, Eint0 = 0.0;  // E(0) and its interaction part for the energy-absorbed objective
  {
    g1g2_obs o;
    if (objective == 2 && (rc = observables_impl(c, &o, nullptr, nullptr))) return done(rc);
    if (objective == 2) {
      E0 = o.e_total;
      Eint0 = o.e_hf + o.e_corr;
    }
  }
  copy_state(at(ckpt, 0), c->n, c->G);
  for (int m = 0; m < nsteps; ++m) {
    c->t = t0 + m * dt;  // same step times as the segment recomputation below
    if ((rc = rk4_step(c, dt))) return done(rc);
    if ((m + 1) % k == 0 && m + 1 < nsteps) copy_state(at(ckpt, (m + 1) / k), c->n, c->G);
  }
  copy_state(at(ckpt, nseg), c->n, c->G);  // final state
  const double tM = c->t;
  // ---- objective and its gradient lambda_M (host side for n, sparse / device for G2)
  std::vector<cplx> hn(N2), hl(N2, cplx{0.0, 0.0});
  cudaMemcpyAsync(hn.data(), c->n, N2 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream);
  cudaMemsetAsync(state_G(lam), 0, N4 * sizeof(cplx), c->stream);
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "adjoint sync"))) return done(rc);
  double J = 0.0, EintT = 0.0;
  if (objective == 0) {
    const int Ls = nb / 2;
    std::vector<cplx> gd(Ls);
    for (int s = 0; s < Ls; ++s) {
      const long long u = 2 * s, d = 2 * s + 1;
      cudaMemcpyAsync(&gd[s], c->G + ((u * N + d) * N + u) * N + d, sizeof(cplx), cudaMemcpyDeviceToHost, c->stream);
    }
    cudaStreamSynchronize(c->stream);
    const cplx mone{-1.0 / Ls, 0.0};
    for (int s = 0; s < Ls; ++s) {
      const long long u = 2 * s, d = 2 * s + 1;
      const zc nuu(hn[u * N + u].x, hn[u * N + u].y), ndd(hn[d * N + d].x, hn[d * N + d].y);
      const zc nud(hn[u * N + d].x, hn[u * N + d].y), ndu(hn[d * N + u].x, hn[d * N + u].y);
      J += ((nuu * ndd - nud * ndu).real() - gd[s].x) / Ls;
      const zc luu = std::conj(ndd) / (double)Ls, ldd = std::conj(nuu) / (double)Ls;
      const zc lud = -std::conj(ndu) / (double)Ls, ldu = -std::conj(nud) / (double)Ls;
      hl[u * N + u] = {luu.real(), luu.imag()};
      hl[d * N + d] = {ldd.real(), ldd.imag()};
      hl[u * N + d] = {lud.real(), lud.imag()};
      hl[d * N + u] = {ldu.real(), ldu.imag()};
      cudaMemcpyAsync(state_G(lam) + ((u * N + d) * N + u) * N + d, &mone, sizeof(cplx), cudaMemcpyHostToDevice,
                      c->stream);
      cudaStreamSynchronize(c->stream);
    }
  } else if (objective == 1) {
    for (int i = 0; i < nb; ++i) {
      const int site = restricted ? i : i / 2;
      const double sgn = (site % 2 == 0) ? 1.0 : -1.0;
      J += sfac * sgn * hn[(long long)i * N + i].x;
      hl[(long long)i * N + i] = {sfac * sgn, 0.0};
    }
  } else {
    g1g2_obs o;
    if ((rc = observables_impl(c, &o, nullptr, nullptr))) return done(rc);
    J = o.e_total - E0;
    EintT = o.e_hf + o.e_corr;
    // dE/dn = s hHF(T), dE/dG2 = -(s/2) w   (s = spin factor)
    std::vector<cplx> hh(N2);
    cudaMemcpyAsync(hh.data(), c->hhf, N2 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    for (long long e = 0; e < N2; ++e) hl[e] = {sfac * hh[e].x, sfac * hh[e].y};
    zaxpby(L, N4, cplx{-0.5 * sfac, 0.0}, c->w, cplx{0.0, 0.0}, nullptr, state_G(lam));
  }
  cudaMemcpyAsync(state_n(lam), hl.data(), N2 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream);
  // ---- reverse sweep
  const cplx one{1.0, 0.0}, zero{0.0, 0.0};
  const double cs[4] = {0.0, 0.5, 0.5, 1.0};
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int m0 = sgi * k, m1 = std::min(nsteps, m0 + k);
    // recompute the segment's step states
    cudaMemcpyAsync(c->n, state_n(at(ckpt, sgi)), N2 * sizeof(cplx), cudaMemcpyDefault, c->stream);
    cudaMemcpyAsync(c->G, state_G(at(ckpt, sgi)), N4 * sizeof(cplx), cudaMemcpyDefault, c->stream);
    c->t = t0 + m0 * dt;
    copy_state(at(seg, 0), c->n, c->G);
    for (int m = m0; m < m1 - 1; ++m) {
      c->t = t0 + m * dt;
      if ((rc = rk4_step(c, dt))) return done(rc);
      copy_state(at(seg, m - m0 + 1), c->n, c->G);
    }
    for (int m = m1 - 1; m >= m0; --m) {
      const double tm = t0 + m * dt;
      void *y = at(seg, m - m0);
      // stage inputs Y1 = y, Y2, Y3, Y4
      void *Ys[4] = {y, Y2, Y3, Y4};
      const double ah[3] = {0.5 * dt, 0.5 * dt, dt};
      for (int s = 0; s < 3; ++s) {
        Rk4Stage st{-1, 0.0};
        StageOut o{nullptr, nullptr, nullptr, state_n(kk), nullptr, nullptr, nullptr, state_G(kk)};
        rhs_fp64(c, L, tm + cs[s] * dt, state_n(Ys[s]), state_G(Ys[s]), st, o);
        if (c->se == G1G2_HF) cudaMemsetAsync(state_G(kk), 0, N4 * sizeof(cplx), c->stream);
        zaxpby(L, N2, one, state_n(y), cplx{ah[s], 0.0}, state_n(kk), state_n(Ys[s + 1]));
        zaxpby(L, N4, one, state_G(y), cplx{ah[s], 0.0}, state_G(kk), state_G(Ys[s + 1]));
      }
      // lam2 accumulates the cotangent of y_m
      cudaMemcpyAsync(lam2, lam, SB, cudaMemcpyDeviceToDevice, c->stream);
      const double lw[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
      const double yw[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};  // weight of Ybar_{s+1} in kbar_s
      for (int s = 3; s >= 0; --s) {
        // kbar_s = lw_s lam + yw_s Ybar_{s+1}
        if (s == 3) {
          zaxpby(L, N2, cplx{lw[s], 0.0}, state_n(lam), zero, nullptr, state_n(kbar));
          zaxpby(L, N4, cplx{lw[s], 0.0}, state_G(lam), zero, nullptr, state_G(kbar));
        } else {
          zaxpby(L, N2, cplx{lw[s], 0.0}, state_n(lam), cplx{yw[s], 0.0}, state_n(Ybar), state_n(kbar));
          zaxpby(L, N4, cplx{lw[s], 0.0}, state_G(lam), cplx{yw[s], 0.0}, state_G(Ybar), state_G(kbar));
        }
        const double ts = tm + cs[s] * dt;
        vjp_fp64(c, L, ts, state_n(Ys[s]), state_G(Ys[s]), state_n(kbar), state_G(kbar), state_n(Ybar),
                 state_G(Ybar), c->adj_hbar, grad_w ? c->adj_wbar : nullptr);
        // parameter cotangents of this stage: <D, hbar> (drive), hbar (h), <f_w, kbar> (scale of w)
        if (c->hasD) real_dot_acc(L, N2, c->D, c->adj_hbar, 1.0, c->adj_red, dacc + 1 + 4 * (size_t)m + s);
        if (grad_h) zaxpby(L, N2, one, c->adj_hsum, one, c->adj_hbar, c->adj_hsum);
        if (grad_wscale) {
          Rk4Stage st{-1, 0.0};
          StageOut o{nullptr, nullptr, nullptr, state_n(kk), nullptr, nullptr, nullptr, state_G(kk)};
          rhs_fp64(c, L, ts, state_n(Ys[s]), state_G(Ys[s]), st, o, true);
          real_dot_acc(L, N2, state_n(kk), state_n(kbar), 1.0, c->adj_red, dacc);
          if (c->se != G1G2_HF) real_dot_acc(L, N4, state_G(kk), state_G(kbar), 1.0, c->adj_red, dacc);
        }
        zaxpby(L, N2, one, state_n(lam2), one, state_n(Ybar), state_n(lam2));
        zaxpby(L, N4, one, state_G(lam2), one, state_G(Ybar), state_G(lam2));
      }
      cudaMemcpyAsync(lam, lam2, SB, cudaMemcpyDeviceToDevice, c->stream);
    }
    if ((rc = launch_status(L, "adjoint"))) return done(rc);
  }
  // restore the final state
  cudaMemcpyAsync(c->n, state_n(at(ckpt, nseg)), N2 * sizeof(cplx), cudaMemcpyDefault, c->stream);
  cudaMemcpyAsync(c->G, state_G(at(ckpt, nseg)), N4 * sizeof(cplx), cudaMemcpyDefault, c->stream);
  c->t = tM;
  if (grad_w) {
    if (objective == 2) {
      // E(T) - E(0) depends on w directly: E_HF = (s_HF) Re sum Wm[(ij),(lk)] n_lk n_ji gives the
      // Hartree-Fock-build cotangent x = s_HF n (n Hermitian), E_corr = -(s_c) Re sum w_ijkl G_klij
      // gives wbar += -(s_c) conj(G_klij) = -(s_c) G_ijkl (G Hermitian); minus the same at t0
      const double s_hf = restricted ? 1.0 : 0.5, s_c = restricted ? 1.0 : 0.5;
      const double eta_hf = restricted ? 0.0 : c->eta;
      cudaMemcpyAsync(c->adj_hbar, c->n, N2 * sizeof(cplx), cudaMemcpyDeviceToDevice, c->stream);
      hf_wbar(L, nb, c->adj_hbar, c->n, s_hf, eta_hf, c->adj_wbar);
      zaxpby(L, N4, one, c->adj_wbar, cplx{-s_c, 0.0}, c->G, c->adj_wbar);
      cudaMemcpyAsync(c->adj_hbar, state_n(at(ckpt, 0)), N2 * sizeof(cplx), cudaMemcpyDefault, c->stream);
      hf_wbar(L, nb, c->adj_hbar, c->adj_hbar, -s_hf, eta_hf, c->adj_wbar);
      cudaMemcpyAsync(state_G(kk), state_G(at(ckpt, 0)), N4 * sizeof(cplx), cudaMemcpyDefault, c->stream);
      zaxpby(L, N4, one, c->adj_wbar, cplx{s_c, 0.0}, state_G(kk), c->adj_wbar);
    }
    // the gradient on the space of admissible w (w_ijkl = w_jilk = conj(w_klij), which g1g2_init
    // enforces): the orthogonal projection of the accumulated cotangent
    w_symmetrize(L, nb, c->adj_wbar, state_G(kk));
    cudaMemcpyAsync(grad_w, state_G(kk), N4 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream);
  }
  std::vector<double> hacc(1 + 4 * (size_t)nsteps);
  cudaMemcpyAsync(hacc.data(), dacc, hacc.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  std::vector<cplx> hg(N2);
  if (grad_h) cudaMemcpyAsync(hg.data(), c->adj_hsum, N2 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream);
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "adjoint sync"))) return done(rc);
  *J_out = J;
  // E(T) - E(0) also depends on w directly: its interaction energies are linear in w
  if (grad_wscale) *grad_wscale = hacc[0] + (objective == 2 ? EintT - Eint0 : 0.0);
  if (grad_h) {
    std::vector<cplx> hn0(N2);
    if (objective == 2) {
      // E(T) - E(0) depends on h directly: s (n(T) - n(0))
      cudaMemcpyAsync(hn0.data(), state_n(at(ckpt, 0)), N2 * sizeof(cplx), cudaMemcpyDefault, c->stream);
      cudaMemcpyAsync(hn.data(), c->n, N2 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream);
      cudaStreamSynchronize(c->stream);
    }
    std::vector<cplx> g(N2);
    for (long long e = 0; e < N2; ++e)
      g[e] = {hg[e].x + (objective == 2 ? sfac * (hn[e].x - hn0[e].x) : 0.0),
              hg[e].y + (objective == 2 ? sfac * (hn[e].y - hn0[e].y) : 0.0)};
    // Hermitian part: the gradient on the space of Hermitian h (h^dag = h is kept by the dynamics)
    for (long long i = 0; i < N; ++i)
      for (long long j = 0; j < N; ++j) {
        const cplx a = g[i * N + j], b = g[j * N + i];
        grad_h[2 * (i * N + j)] = 0.5 * (a.x + b.x);
        grad_h[2 * (i * N + j) + 1] = 0.5 * (a.y - b.y);
      }
  }
  if (grad_drive && c->hasD) {
    // dJ/dtheta = sum over steps and stages of (df/dtheta)(t_s) <D, hbar_s>, plus the
    // explicit f-dependence of the energy objective at t = T and t = 0
    const std::vector<double> &p = c->drive_params;
    const int np = (int)p.size();
    const int ng = c->drive_kind == 2 ? np - 2 : 4;
    std::vector<double> gd(ng, 0.0);
    auto add_df = [&](double tt, double wgt) {
      if (c->drive_kind == 2) {
        const double ta = p[0], tb = p[1];
        const int M = np - 2;
        const double hs = (tb - ta) / (M - 1);
        const double x = (tt - ta) / hs;
        if (x <= 0) gd[0] += wgt;
        else if (x >= M - 1) gd[M - 1] += wgt;
        else {
          int sI = (int)std::floor(x);
          if (sI > M - 2) sI = M - 2;
          const double u = x - sI;
          gd[sI] += (1 - u) * wgt;
          gd[sI + 1] += u * wgt;
        }
      } else {
        const double A = p[0], w = p[1], tc = p[2], sg = p[3];
        const double g = std::exp(-(tt - tc) * (tt - tc) / (2 * sg * sg));
        const double sn = std::sin(w * tt), cn = std::cos(w * tt);
        gd[0] += wgt * sn * g;
        gd[1] += wgt * A * tt * cn * g;
        gd[2] += wgt * A * sn * g * (tt - tc) / (sg * sg);
        gd[3] += wgt * A * sn * g * (tt - tc) * (tt - tc) / (sg * sg * sg);
      }
    };
    for (int m = 0; m < nsteps; ++m)
      for (int s = 0; s < 4; ++s) add_df(t0 + m * dt + cs[s] * dt, hacc[1 + 4 * (size_t)m + s]);
    if (objective == 2) {
      // J = E(T) - E(0) depends on f(T) and f(0) through h(t): dE/df = s Re Tr(D n)
      Launcher L2 = c->launcher();
      obs_one_body(L2, nb, c->h, c->D, drive_f(c, tM), c->hhf, c->n, c->red);
      double r[4];
      cudaMemcpyAsync(r, c->red, sizeof(r), cudaMemcpyDeviceToHost, c->stream);
      cudaStreamSynchronize(c->stream);
      add_df(tM, sfac * r[3]);
      cudaMemcpyAsync(c->adj_hsum, state_n(at(ckpt, 0)), N2 * sizeof(cplx), cudaMemcpyDefault, c->stream);
      obs_one_body(L2, nb, c->h, c->D, drive_f(c, t0), c->hhf, c->adj_hsum, c->red);
      cudaMemcpyAsync(r, c->red, sizeof(r), cudaMemcpyDeviceToHost, c->stream);
      cudaStreamSynchronize(c->stream);
      add_df(t0, -sfac * r[3]);
    }
    for (int i = 0; i < ng; ++i) grad_drive[i] = gd[i];
  }
  return done(G1G2_OK);
}

int g1g2_set_state(g1g2_ctx *c, double t, const double *G1, const double *G2) {
  if (!c || !G1) return fail(G1G2_EINVAL, "NULL argument");
  const size_t N2 = (size_t)c->nb * c->nb, N4 = N2 * N2;
  int rc;
  if ((rc = cuda_check(cudaMemcpyAsync(c->n, G1, N2 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "set")))
    return rc;
  if (G2) rc = cuda_check(cudaMemcpyAsync(c->G, G2, N4 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "set");
  else rc = cuda_check(cudaMemsetAsync(c->G, 0, N4 * sizeof(cplx), c->stream), "set");
  if (rc) return rc;
  if (c->hub_gw && (rc = cuda_check(cudaMemsetAsync(c->Gss, 0, N4 * sizeof(cplx), c->stream), "set"))) return rc;
  c->t = t;
  if (c->tc) {
    Launcher L = c->launcher();
    tc_load_state(c->tc, L, c->G);
    if ((rc = launch_status(L, "tensor-core state"))) return rc;
  }
  if ((rc = cuda_check(cudaMemsetAsync(c->W_dev, 0, sizeof(double), c->stream), "memset"))) return rc;
  return cuda_check(cudaStreamSynchronize(c->stream), "set sync");
}

}  // extern "C"
