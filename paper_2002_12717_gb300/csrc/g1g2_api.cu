// libg1g2: the C ABI declared in include/g1g2.h.
//
// One context = one propagation on one GPU.  The RK4 driver, the drive h(t),
// validation and bookkeeping are host code here; every arithmetic step of the
// right-hand side runs in the kernels of fp64_kernels.cu (FP64 form) and
// tc_kernels.cu (split-precision tensor-core form).
#include "g1g2_internal.h"
#include "tc_path.h"

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>

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
  cplx *w = nullptr;                // w (complex), [(ij),(kl)]
  cplx *wsrc = nullptr;             // source-term interaction (w^- or w)
  cplx *wP = nullptr;               // collision layout [(lp)][i][k] = w_iklp
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

void rhs_fp64(g1g2_ctx *c, Launcher &L, double t, const cplx *n_in, const cplx *G_in, Rk4Stage st,
              const StageOut &o) {
  const int nb = c->nb;
  const long long N = nb, N2 = N * N, N3 = N2 * N;
  const double f = drive_f(c, t);
  // a1: Eq. (h_HF)
  hf_build(L, nb, c->Wm, c->w_real, c->h, c->hasD ? c->D : nullptr, f, n_in, c->hhf);
  if (c->se == G1G2_HF) {
    g1_update(L, nb, c->hhf, n_in, nullptr, st, o.ny, o.nys, o.nacc, o.nk);
    return;
  }
  // a2: I_ij = -i sum_(lp) sum_k wP[lp][i][k] G[lp][j][k]   (Eq. eom_gone-I)
  {
    ZGemm g;
    g.M = nb; g.N = nb; g.K = nb; g.batch = (int)N2;
    g.A = c->wP; g.sa_b = N2; g.sa_m = N; g.sa_k = 1;
    g.B = G_in; g.sb_b = N2; g.sb_k = 1; g.sb_n = N;
    g.C = c->I; g.sc_m = N; g.sc_n = 1;
    g.alpha = {0.0, -1.0};
    zgemm_reduce(L, g, c->partial, c->splits);
  }
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
  // a4: A = sum nbar_ip nbar_jq wt_pqrs n_rk n_sl by successive contractions; Psi = -A + A^dag
  one_minus(L, nb, n_in, c->nbar);
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
  if (c->se == G1G2_GW) {
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
    hf_build(L, c->nb, c->Wm, c->w_real, c->h, c->hasD ? c->D : nullptr, f, n_in, c->hhf);
    tc_rhs(c->tc, L, n_in, G_in, c->hhf, st, o.ny, o.nys, o.nacc, o.nk, o.Gy, o.Gys, o.Gacc, o.Gk);
  }
}

int rk4_step(g1g2_ctx *c, double dt) {
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
    Rk4Stage st{s, dt};
    rhs_dispatch(c, L, t + cs[s] * dt, n_in, G_in, st, o);
  }
  c->t = t + dt;
  return launch_status(L, "rk4 step");
}

int observables_impl(g1g2_ctx *c, g1g2_obs *out, double *density, double *nonfinite) {
  Launcher L = c->launcher();
  const int nb = c->nb;
  const double f = drive_f(c, c->t);
  hf_build(L, nb, c->Wm, c->w_real, c->h, c->hasD ? c->D : nullptr, f, c->n, c->hhf);
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

}  // namespace

extern "C" {

void g1g2_default_options(g1g2_options *opt) {
  if (!opt) return;
  opt->precision = G1G2_FP64;
  opt->basis = G1G2_SPIN_ORBITAL;
  opt->w_is_real = 0;
  opt->sym_tol = 1e-10;
  opt->cuda_stream = nullptr;
}

const char *g1g2_strerror(int code) {
  switch (code) {
    case G1G2_OK: return "ok";
    case G1G2_EINVAL: return "invalid argument";
    case G1G2_ESYMM: return "input violates the symmetries of w, G1 or G2";
    case G1G2_ENOMEM: return "device allocation failed";
    case G1G2_ECUDA: return "CUDA error";
    case G1G2_ENONFINITE: return "state contains NaN or Inf";
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
  if (se < G1G2_HF || se > G1G2_GW) return fail(G1G2_EINVAL, "bad selfenergy");
  if (opt.precision != G1G2_FP64 && opt.precision != G1G2_TF32X3) return fail(G1G2_EINVAL, "bad precision");
  if (opt.basis != G1G2_SPIN_ORBITAL && opt.basis != G1G2_SPIN_RESTRICTED) return fail(G1G2_EINVAL, "bad basis");
  if (opt.basis == G1G2_SPIN_RESTRICTED && se == G1G2_GW)
    return fail(G1G2_EINVAL, "GW couples same-spin components and has no spin-restricted form");

  const size_t N = nb, N2 = N * N, N4 = N2 * N2;
  const bool restricted = opt.basis == G1G2_SPIN_RESTRICTED;
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
  // source interaction: w^- (SOA, spin-orbital), else w
  const bool use_minus = (se == G1G2_SOA && !restricted);
  for (size_t i = 0; i < N; ++i)
    for (size_t j = 0; j < N; ++j)
      for (size_t k = 0; k < N; ++k)
        for (size_t l = 0; l < N; ++l) {
          zc a = wv(at4(i, j, k, l));
          if (use_minus) a -= wv(at4(i, j, l, k));
          hsrc[at4(i, j, k, l)] = {a.real(), a.imag()};
          // collision layout wP[(l,p)][i][k] = w_iklp: here (i,k,l,p) = (i,j,k,l) renamed
          const zc b = wv(at4(i, j, k, l));        // w_{i j k l} with j->k', k->l', l->p'
          hP[((k * N + l) * N + i) * N + j] = {b.real(), b.imag()};
        }
  // Hartree-Fock matrix Wm[(ij),(lk)] = w_ikjl - w_iklj (restricted: w_ikjl)
  std::vector<double> WmR;
  std::vector<cplx> WmC;
  if (real) WmR.resize(N4); else WmC.resize(N4);
  for (size_t i = 0; i < N; ++i)
    for (size_t j = 0; j < N; ++j)
      for (size_t l = 0; l < N; ++l)
        for (size_t k = 0; k < N; ++k) {
          zc a = wv(at4(i, k, j, l));
          if (!restricted) a -= wv(at4(i, k, l, j));
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
    if (se == G1G2_GW) {
      if ((rc = dalloc(c, &c->Hb, N4)) || (rc = dalloc(c, &c->Gp, N4)) || (rc = dalloc(c, &c->Hp, N4)) ||
          (rc = dalloc(c, &c->Pp, N4)))
        return bail(rc);
    }
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
  if (correlated && c->prec != G1G2_FP64) {
    if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "init sync"))) return bail(rc);
    g_detail.clear();
    rc = tc_create(&c->tc, nb, se, restricted, hw.data(), hsrc.data(), c->stream);
    if (rc) return bail(rc);
    Launcher L = c->launcher();
    tc_load_state(c->tc, L, c->G);
    if ((rc = launch_status(L, "tensor-core state"))) return bail(rc);
  }
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "init sync"))) return bail(rc);
  *out = c;
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
  int rc = cuda_check(cudaMemcpyAsync(c->D, D, N2 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "drive upload");
  if (rc) return rc;
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "drive sync"))) return rc;
  c->drive_kind = kind;
  c->drive_params.assign(params, params + nparams);
  c->hasD = true;
  return G1G2_OK;
}

int g1g2_rhs(g1g2_ctx *c, double t, const double *n_dev, const double *G2_dev, double *dn_dev, double *dG2_dev) {
  if (!c || !n_dev || !dn_dev) return fail(G1G2_EINVAL, "NULL argument");
  if (c->se != G1G2_HF && (!G2_dev || !dG2_dev)) return fail(G1G2_EINVAL, "G2 and dG2 must be non-NULL");
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
    double_occ(L, c->nb, c->n, c->G, c->red + 8);
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

int g1g2_set_state(g1g2_ctx *c, double t, const double *G1, const double *G2) {
  if (!c || !G1) return fail(G1G2_EINVAL, "NULL argument");
  const size_t N2 = (size_t)c->nb * c->nb, N4 = N2 * N2;
  int rc;
  if ((rc = cuda_check(cudaMemcpyAsync(c->n, G1, N2 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "set")))
    return rc;
  if (G2) rc = cuda_check(cudaMemcpyAsync(c->G, G2, N4 * sizeof(cplx), cudaMemcpyHostToDevice, c->stream), "set");
  else rc = cuda_check(cudaMemsetAsync(c->G, 0, N4 * sizeof(cplx), c->stream), "set");
  if (rc) return rc;
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
