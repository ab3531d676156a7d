/*
 * g1g2.h -- C ABI of libg1g2, a GB300 (sm_103a) implementation of the time-local
 * G1-G2 scheme of Joost, Schluenzen and Bonitz (arXiv:2002.12717).
 *
 * The library propagates the one-particle density matrix n (called G1 here,
 * n_ij = <c_j^dagger c_i>, Sec. II.B Eq. g-glsymm) and the correlated
 * two-particle Green function G2 (the nb^4 tensor of Eq. gscor-def) with
 * classical RK4.  The right-hand side is
 *   G1:  Eq. (eom_gone-2) with the collision integral of Eq. (eom_gone-I)
 *   G2:  Eq. (result_eom_soa) for SOA (source term Psi^-, Eq. psi-pm-def),
 *        Eq. (g2-eq-gw-pi) for GW (plain-w Psi plus the polarisation term
 *        of Eq. gwpi), the T-matrix ladder terms of Sec. IV.D/E and their
 *        combination with GW (Sec. V), nothing for HF (time-dependent
 *        Hartree-Fock).  g1g2_propagate_hfgkba runs the memory-integral
 *        HF-GKBA the G1-G2 equations replace (Sec. III.B), for comparison.
 * Conventions: fermions, hbar = 1, h(t) = h + f(t) D.
 *
 * Layout of every complex array: row-major, interleaved (re, im) doubles.
 *   h, D, G1 : nb x nb            element (i, j) at 2*(i*nb + j)
 *   w, G2    : nb x nb x nb x nb  element (i, j, k, l) at 2*(((i*nb + j)*nb + k)*nb + l)
 * w is the pair interaction of Eq. (h): H = sum h_ij c_i^+ c_j
 *   + 1/2 sum w_ijkl c_i^+ c_j^+ c_l c_k.  With g1g2_options.w_is_real != 0,
 *   w is passed as nb^4 real doubles instead.
 *
 * Ownership: init, set_drive, set_state and get_state take HOST pointers and
 * copy; the caller keeps its buffers.  g1g2_rhs takes DEVICE pointers owned
 * by the caller.  The context owns all of its device memory until
 * g1g2_destroy.  All device work is issued on the stream given in
 * g1g2_options.cuda_stream (NULL = the legacy default stream).
 *
 * Errors: every int-returning call returns G1G2_OK (0) or a negative code;
 * nothing aborts or throws across the ABI.  g1g2_strerror gives the message,
 * g1g2_last_error_detail the detail of the last failure on this thread.
 */
#ifndef G1G2_H
#define G1G2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define G1G2_OK            0
#define G1G2_EINVAL       -1  /* bad size, NULL pointer, bad enum, unsupported combination */
#define G1G2_ESYMM        -2  /* w, G1_0 or G2_0 violates the symmetries of Sec. II (Eqs. Gsymm, wsymm) */
#define G1G2_ENOMEM       -3  /* device allocation failed */
#define G1G2_ECUDA        -4  /* a CUDA runtime call or kernel launch failed */
#define G1G2_ENONFINITE   -5  /* the state or a host input contains NaN or Inf */
#define G1G2_ETIMEOUT     -6  /* a bounded device wait gave up */
#define G1G2_EUNSUPPORTED -7  /* valid request that this build does not implement */

typedef struct g1g2_ctx g1g2_ctx;  /* opaque */

/* Selfenergy of the G2 equation. */
typedef enum {
  G1G2_HF = 0,   /* I = 0, G2 frozen: time-dependent Hartree-Fock (Eq. eom_gone-2 without I) */
  G1G2_SOA = 1,  /* second-order Born, Sec. III.C, Eq. (result_eom_soa) */
  G1G2_GW = 2,   /* GW, Sec. IV.C, Eq. (g2-eq-gw-pi); in the spin-restricted basis only for an
                    on-site w (the Hubbard form, Eqs. g2-gw-hubbard1/2, FP64): G2 is the
                    opposite-spin block, the context keeps the same-spin block its
                    polarisation couples to (zero at init and after g1g2_set_state), and
                    g1g2_rhs is refused (G1G2_EUNSUPPORTED) */
  G1G2_GW_EXCHANGE = 3, /* GW with exchange: Psi replaced by Psi^± in Eq. (g2-eq-gw-pi)
                           (end of Sec. IV.C); spin-orbital basis only */
  G1G2_TPP = 4,         /* particle-particle T matrix, Sec. IV.D, Eq. (g2-eq-tpp-lambda): the SOA
                           equation plus the ladder term Lambda - (Lambda_klij)^*, Lambda = hcorr G2
                           (Eqs. HTPPcorr, lambdapp); FP64 and BF16-slice forms */
  G1G2_TPH = 5,         /* particle-hole T matrix, Sec. IV.E, Eq. (g2-eq-tph-lambda): the same with
                           Lambda_ijkl = sum_pq hcorr_ipql G2_qjkp (Eqs. HTPHcorr, lambdaph); FP64
                           and BF16-slice forms */
  G1G2_DSL = 6          /* dynamically screened ladder, Sec. V, Eq. (g2-dsl-equation-pi-lambda):
                           Psi^± plus the GW term Pi - (Pi_lkji)^* plus the ladder term with
                           Lambda = Lambda^pp + Lambda^ph; spin-orbital basis, FP64 and
                           BF16-slice forms */
} g1g2_selfenergy;

/* Arithmetic of the contractions. The RK4 state update, the Hartree-Fock
 * build and the observables are FP64 in every mode. */
typedef enum {
  G1G2_FP64 = 0,   /* every contraction in FP64 on the CUDA cores: the reference form */
  G1G2_TF32X3 = 1, /* split-precision tensor-core contractions: hi/lo TF32 operands, FP32 accumulation */
  G1G2_BF16X4 = 2  /* tensor-core contractions on four BF16 slices per operand with one power-of-two
                      scale per tensor; the leading slice product accumulates exactly in FP32, the
                      lower-order products (2^-8 and below) in a second accumulator */
} g1g2_precision;

/* Basis. SPIN_RESTRICTED: the index runs over spatial orbitals, w is an
 * opposite-spin interaction and n_up = n_down (the Hubbard equations of
 * Sec. III.D: no exchange term in h^HF and Psi, spin factors in the energies).
 * HF, SOA and the two T matrices run in this basis for any such w; GW only in
 * the Hubbard form (an on-site w); GW with exchange and DSL not at all. */
typedef enum { G1G2_SPIN_ORBITAL = 0, G1G2_SPIN_RESTRICTED = 1 } g1g2_basis;

typedef struct {
  int precision;      /* g1g2_precision */
  int basis;          /* g1g2_basis */
  int w_is_real;      /* nonzero: w is nb^4 real doubles */
  double sym_tol;     /* absolute symmetry tolerance for w, G1_0, G2_0 (scaled by max|x|); <0 skips */
  void *cuda_stream;  /* cudaStream_t used for every launch; NULL = default stream */
  int statistics;     /* g1g2_statistics */
} g1g2_options;

/* Particle statistics: the "±" of the paper (footnote to the KBE, Sec. II.A).
 * Bosons change the exchange sign of h^HF (w^+ of Eq. h_HF) and of the energy
 * (Eq. ini-g2, upper sign), the source interaction w^+ of Psi^±, and
 * G^> = -i (1 + n) (Eq. g-glsymm) in the source term and the T-matrix
 * quasi-Hamiltonians.  The G1 equation in (n, G2), the collision integral, the
 * commutator and the GW quasi-Hamiltonian are the same for both.  Bosons run
 * in the spin-orbital basis (G1G2_EINVAL otherwise), in every precision; the
 * discrete adjoint and the Hubbard path are fermion-only. */
enum { G1G2_FERMIONS = 0, G1G2_BOSONS = 1 };

typedef struct {
  double t;
  double n_particles;  /* Re Tr n (x2 spin-restricted) */
  double e_one;        /* Re Tr(h(t) n) (x2 spin-restricted) */
  double e_hf;         /* 1/2 Re sum w^-_ijkl n_ki n_lj (w^+ for bosons; spin-restricted: Re sum w_ijkl n_ki n_lj) */
  double e_corr;       /* -1/2 Re sum w_ijkl G2_klij (spin-restricted: -Re sum w_ijkl G2_klij) */
  double e_total;      /* e_one + e_hf + e_corr */
  double pulse_work;   /* W(t) = int f'(t) Re Tr(D n) dt, RK4-weighted over the stages */
} g1g2_obs;

/* Default options: FP64, spin-orbital, complex w, sym_tol 1e-10, default stream, fermions. */
void g1g2_default_options(g1g2_options *opt);

/* Create a propagation context (Sec. III.F: the initial values n^0 and G2^0).
 *   nb         basis size, 1 <= nb <= 128
 *   h          nb*nb complex, Hermitian (host)
 *   w          nb^4 complex, or real if opt->w_is_real (host); must satisfy
 *              w_ijkl = w_jilk and w_ijkl = conj(w_klij) (Eqs. wsymm_a/b)
 *   G1_0       nb*nb complex, Hermitian (host)
 *   G2_0       nb^4 complex with Eqs. (Gsymm_a/b) (host), or NULL for G2_0 = 0
 *   se         g1g2_selfenergy
 *   opt        options, or NULL for the defaults
 * Returns G1G2_EINVAL for nb out of range, NULL arrays, bad enums, GW with
 * exchange or DSL in the spin-restricted basis, or GW there with a w that is
 * not on-site (the Hubbard form); G1G2_EUNSUPPORTED for a combination this
 * build does not run (see g1g2_selfenergy and g1g2_precision); G1G2_ESYMM
 * when a symmetry is violated beyond sym_tol; G1G2_ENONFINITE when h, w, G1_0 or G2_0 holds a NaN or an Inf
 * (checked on the host before any device work); G1G2_ENOMEM / G1G2_ECUDA on
 * device failure. t starts at 0. */
int g1g2_init(g1g2_ctx **out, int nb, const double *h, const double *w, const double *G1_0,
              const double *G2_0, int se, const g1g2_options *opt);

/* Create a context for a factorised interaction
 *   w_ijkl = sum_{P<nfac} L^P_ik L^P_jl
 * (the density-fitted / Cholesky form of a two-electron integral tensor; the
 * paper's general-basis w of Eq. (h) in the pair order (ik),(jl)).
 *   L      nfac*nb*nb, element (P, i, k) at P*nb*nb + i*nb + k: complex
 *          interleaved, or real if opt->w_is_real (host, copied).  Each L^P is
 *          Hermitian or i times Hermitian, so that w meets Eqs. (wsymm_a/b)
 *   nfac   number of factors, 1 <= nfac <= nb*nb
 * A NaN or an Inf in L returns G1G2_ENONFINITE, a factor that is neither Hermitian
 * nor i times Hermitian (beyond opt->sym_tol) G1G2_ESYMM, both before any device work.
 * The other arguments and the error codes are those of g1g2_init, which runs on
 * the w expanded on the device (one nb^2 x nb^2 x nfac product; nb^4 complex
 * doubles of host memory for the duration of the call).  In the FP64 form the
 * source term of Eq. (psi-pm-def) then runs in the factorised form: M^P = nbar
 * L^P n (two batched nb^3 products per factor) and
 *   A_ijkl = sum_P M^P_ik M^P_jl  (+ eta M^P_il M^P_jk for the source w^±),
 * an nb^2 x nb^2 x nfac product in place of four nb^5 mode products.  The
 * split-precision forms run on the expanded w. */
int g1g2_init_factorised(g1g2_ctx **out, int nb, const double *h, const double *L, int nfac,
                         const double *G1_0, const double *G2_0, int se, const g1g2_options *opt);

/* Time-dependent one-body term h(t) = h + f(t) D (the excitations of the
 * workloads; the paper's Eq. (h) allows any h(t)).
 *   D       nb*nb complex Hermitian (host), copied
 *   kind    0 none; 1 gauss-sine f = A sin(w t) exp(-(t-t0)^2/(2 s^2)) with
 *           params = {A, w, t0, s}; 2 piecewise linear through M equidistant
 *           values on [ta, tb], params = {ta, tb, v_0 .. v_{M-1}} (M >= 2),
 *           constant beyond the ends.
 * Returns G1G2_EINVAL on a bad kind or parameter count. */
int g1g2_set_drive(g1g2_ctx *c, const double *D, int kind, const double *params, int nparams);

/* One evaluation of the right-hand side at time t (device pointers, caller-owned,
 * interleaved complex, same layouts as above):
 *   n_dev, G2_dev  input state; G2_dev must be Hermitian as an nb^2 x nb^2
 *                  matrix (Eq. Gsymm_b), which the tensor-core form relies on
 *   dn_dev, dG2_dev  outputs dn/dt and dG2/dt (dG2 is zero for HF)
 * Runs on the context's stream; returns after the launches are queued. */
int g1g2_rhs(g1g2_ctx *c, double t, const double *n_dev, const double *G2_dev, double *dn_dev,
             double *dG2_dev);

/* One classical RK4 step of size dt on the context's state (no host sync). */
int g1g2_step(g1g2_ctx *c, double dt);

/* nsteps RK4 steps. When obs is non-NULL it receives 1 + nsteps/obs_every
 * records (t = start and after every obs_every-th step); when density is
 * non-NULL it receives nb doubles per record (n_ii, x2 spin-restricted).
 * Synchronises the stream at the end; checks the state for NaN/Inf at every
 * record (G1G2_ENONFINITE). */
int g1g2_propagate(g1g2_ctx *c, double dt, int nsteps, int obs_every, g1g2_obs *obs, double *density);

/* The original HF-GKBA in its memory-integral form (Sec. III.B), the scheme the
 * G1-G2 equations replace: G2(t) = (i hbar)^3 int_{t0}^t dtb U2(t,tb) Psi(tb) U2(tb,t)
 * (Eq. dtilde-solution-short, U2 = U (x) U by Eq. prop_two), with the Hartree-Fock
 * propagators of the GKBA (Eqs. GKBA_propa/b), i hbar U(t,tb) = u(t) u(tb)^dag,
 * i du/dt = hHF u.  Each evaluation of G2 sums over all earlier time steps (trapezoid
 * rule), so nsteps steps cost O(nsteps^2) (Table I); n and u advance by Heun's method
 * (second order), so the result converges to the G1-G2 one as dt^2.
 *   c            SOA context in the FP64 form, nb <= 32, no drive (G1G2_EUNSUPPORTED
 *                otherwise); its state must have G2 = 0 (uncorrelated start at the
 *                context's time, G1G2_EINVAL otherwise)
 *   G1_history   host, (nsteps+1)*nb*nb complex: n(t0 + m dt), m = 0..nsteps, or NULL
 *   scratch_bytes  device memory for the batched history products (0: 256 MiB); the
 *                history itself takes (nsteps+2) (nb^4 + 3 nb^2) complex doubles
 * Allocates its scratch on each call (G1G2_ENOMEM when it does not fit) and frees it
 * before returning.  On return the context holds n(T) and G2(T) from the memory
 * integral and t = t0 + nsteps dt.  Synchronous. */
int g1g2_propagate_hfgkba(g1g2_ctx *c, double dt, int nsteps, double *G1_history, size_t scratch_bytes);

/* Observables of the current state (synchronous). density: nb doubles or NULL.
 * double_occ: nb/2 doubles or NULL, spin-orbital basis with index 2*site+spin only
 * (E10: d_i = n_{i+,i+} n_{i-,i-} - |n_{i+,i-}|^2 - G2_{i+ i- i+ i-}; + |n_{i+,i-}|^2
 * for bosons, Eq. ini-g2). */
int g1g2_observables(g1g2_ctx *c, g1g2_obs *out, double *density, double *double_occ);

/* Vector-Jacobian product of the right-hand side (FP64 form; fermions in a general
 * basis, every selfenergy; not the spin-restricted Hubbard GW): given the
 * cotangents (dn_bar, dG2_bar) of (dn/dt, dG2/dt) at the state (n, G2) at time
 * t, write the cotangents of n, of G2 and of h^HF (= of the explicit h(t)),
 * with respect to Re sum conj(x) y.  All pointers are caller-owned device
 * arrays in the ABI layout; n must be Hermitian (the point of evaluation).
 * Not in the paper: the building block of g1g2_adjoint. */
int g1g2_rhs_vjp(g1g2_ctx *c, double t, const double *n_dev, const double *G2_dev, const double *dn_bar,
                 const double *dG2_bar, double *n_bar, double *G2_bar, double *h_bar);

/* Discrete adjoint of nsteps RK4 steps of the FP64 form (fermions, every selfenergy
 * in a general basis), starting
 * from the current state: the gradient of a final-time objective J with
 * respect to the drive parameters, a global scale of w, the entries of h and
 * the entries of w.
 * Not in the paper; the reverse sweep is the exact transpose of the discrete
 * RK4 map, with the state (n, G2) checkpointed every ckpt_every steps and
 * each segment recomputed once.  ckpt_every <= 0 chooses the interval from
 * the free memory: the smallest k whose ceil(nsteps/k) + 1 checkpoints and
 * k + 1 segment states fit (k = 1, no recomputation, when all steps fit; see
 * g1g2_set_adjoint_checkpoints for device or pinned host checkpoints).
 *   objective   0: mean double occupancy (1/L) sum_i d_i (E10; spin-orbital
 *                  basis, index 2*site+spin); 1: density imbalance
 *                  sum_i (-1)^site n_ii (x2 spin-restricted); 2: energy absorbed
 *                  E(T) - E(0) (E9)
 *   J_out       objective value at the final time
 *   grad_drive  dJ/dtheta for the drive parameters (kind 2: the M control
 *               values; kind 1: A, omega, t0, sigma), or NULL
 *   grad_wscale dJ/ds for w -> s w at s = 1 (e.g. U dJ/dU for a Hubbard w), or NULL
 *   grad_h      nb*nb interleaved gradient G on Hermitian h: for every Hermitian
 *               perturbation dh, dJ = Re sum conj(G_ij) dh_ij (G is Hermitian), or NULL
 *   grad_w      nb^4 interleaved gradient W on the interactions g1g2_init accepts
 *               (w_ijkl = w_jilk = conj(w_klij)): for every such perturbation dw,
 *               dJ = Re sum conj(W_ijkl) dw_ijkl, and W has the same symmetries (for a
 *               real w and real dw only Re W acts).  Every place w enters the right-hand
 *               side contributes: Eq. (h_HF), Eq. (eom_gone-I), the source term of
 *               Eq. (psi-pm-def), Eq. (gwhcorr) and the ladder quasi-Hamiltonians of
 *               Eqs. (HTPPcorr), (HTPHcorr), plus the interaction energies of objective 2.
 *               Host array, or NULL (then none of that work is done)
 * Cotangents use Re sum conj(x) y over every complex entry of (G1, G2).  On
 * return the context holds the final state (as after g1g2_propagate).
 * G1G2_EUNSUPPORTED for the tensor-core precision, bosons and the spin-restricted
 * Hubbard GW. */
int g1g2_adjoint(g1g2_ctx *c, double dt, int nsteps, int ckpt_every, int objective, double *J_out,
                 double *grad_drive, double *grad_wscale, double *grad_h, double *grad_w);

/* Where g1g2_adjoint keeps its checkpoints: G1G2_CKPT_AUTO (device memory when
 * the checkpoints and one segment fit in 80% of the free device memory, else
 * pinned host memory, at most half of the free host memory, with only the
 * segment on the device), G1G2_CKPT_DEVICE or G1G2_CKPT_HOST.  The choice of
 * the interval (ckpt_every <= 0) follows the location: the smallest interval
 * that fits.  Results do not depend on it.  G1G2_EINVAL on another value.
 * Not in the paper. */
enum { G1G2_CKPT_AUTO = 0, G1G2_CKPT_DEVICE = 1, G1G2_CKPT_HOST = 2 };
int g1g2_set_adjoint_checkpoints(g1g2_ctx *c, int where);

/* Interval and location (G1G2_CKPT_DEVICE / G1G2_CKPT_HOST) the last
 * g1g2_adjoint call used (0, 0 before the first). */
int g1g2_adjoint_plan(const g1g2_ctx *c, int *ckpt_every, int *where);

/* O(nb^4) right-hand side for the Hubbard basis (Sec. VI: the commutator with
 * the sparse h^HF as a stencil, and the source term with the products of four
 * G^< cancelled, Eq. (soa-cubic-scheme); the collision integral reduces to
 * I_ij = -i U_i G2_iiji).  Chosen automatically at g1g2_init when the basis is
 * spin-restricted, the selfenergy SOA, the precision FP64 and w is on-site
 * (w_ijkl = U_i when i = j = k = l, else 0); the commutator runs over the
 * nonzero pattern of h, of D (set_drive) and of the diagonal.
 *   g1g2_set_hubbard_path(c, 0) switches to the general O(nb^5) form,
 *   g1g2_set_hubbard_path(c, 1) back (G1G2_EUNSUPPORTED if the structure does
 *   not qualify); g1g2_hubbard_path returns 1 when it is in use, 0 when not,
 *   G1G2_EINVAL for a NULL context. */
/* The FP64 FMA throughput of the current device in TFLOP/s: eight independent
 * DFMA chains per thread over 8 blocks of 256 threads per SM, best of three
 * launches timed with CUDA events after two untimed ones (about 4 s in all).  The ALU roofline of
 * the FP64 form and of the memory-integral HF-GKBA.  Not part of the paper's
 * method.  G1G2_ECUDA on a CUDA failure. */
int g1g2_fp64_rate(double *tflops);

int g1g2_set_hubbard_path(g1g2_ctx *c, int enable);
int g1g2_hubbard_path(const g1g2_ctx *c);

/* Failure-detection self-test (not in the paper): launches one CTA that waits
 * on a barrier nothing arrives on, with the bounded wait the tensor-core
 * kernels use but a limit of limit_us microseconds (1 .. 1e7).  Expected
 * result: G1G2_ETIMEOUT (the wait gave up, reported through the error word,
 * and the kernel returned; the CUDA context stays usable).  G1G2_EINVAL on a
 * bad limit, G1G2_ECUDA on a launch failure.  Runs on the legacy default
 * stream of the current device. */
int g1g2_wait_selftest(int limit_us);

/* Copy the state to / from host memory (G2 may be NULL on get; NULL on set means 0). */
int g1g2_get_state(g1g2_ctx *c, double *t, double *G1, double *G2);
int g1g2_set_state(g1g2_ctx *c, double t, const double *G1, const double *G2);

/* Number of kernel launches issued by this context since creation. */
long long g1g2_launch_count(const g1g2_ctx *c);

/* Per-kernel device time, for roofline accounting (not part of the paper's
 * method).  g1g2_profile(c, 1) clears the records and brackets every later
 * launch of the context with CUDA events on its stream; g1g2_profile(c, 0)
 * stops recording.  g1g2_profile_report synchronises the stream and writes at
 * most max_entries aggregates (one per kernel name, launches and summed
 * milliseconds) to out, their number to *n_entries; the records are kept. */
typedef struct {
  char name[48];
  long long launches;
  double total_ms;
} g1g2_kernel_stat;
int g1g2_profile(g1g2_ctx *c, int enable);
int g1g2_profile_report(g1g2_ctx *c, g1g2_kernel_stat *out, int max_entries, int *n_entries);

/* G1 right-hand side without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- for example code whose device memory is owned by another
 * allocator (a framework's caching pool, a fixed arena set up at start-up),
 * or loops that must not risk the latency or failure of an allocation
 * between steps.  It returns dn/dt of Eq. (eom_gone-2), with h^HF from
 * Eq. (h_HF) and I from Eq. (eom_gone-I), the same quantity as the dn output
 * of g1g2_rhs, for one state:
 *   nb          1 <= nb <= 64 (larger nb returns G1G2_EINVAL with a detail)
 *   restricted  nonzero: spin-restricted basis (no exchange term in h^HF)
 *   h_dev       nb*nb complex one-body Hamiltonian h(t) (device)
 *   w_dev       nb^4 complex interaction in the ABI layout (device)
 *   n_dev       nb*nb complex density matrix G1 (device)
 *   G2_dev      nb^4 complex G2 (device)
 *   dn_dev      nb*nb complex output (device)
 *   cuda_stream stream for the launches (NULL = default stream)
 * All arrays are caller-owned.  Scratch (split-K partial sums, h^HF, I,
 * about 2.2 MB) is one static device array per GPU, kept until the process
 * exits and shared by every call on that GPU: calls whose kernels overlap on
 * the GPU (different streams, or threads without ordering) race on it.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture
 * (a lookup that fails is not cached: the next call tries again).  Nothing in
 * the scratch needs clearing between calls: each call writes every scratch
 * element it reads.  A non-sticky CUDA error left pending by earlier work is
 * cleared on entry, so it is not reported as this call's failure. */
int g1g2_g1_rhs_noalloc(int nb, int restricted, const double *h_dev, const double *w_dev, const double *n_dev,
                        const double *G2_dev, double *dn_dev, void *cuda_stream);

const char *g1g2_strerror(int code);
const char *g1g2_last_error_detail(void);
void g1g2_destroy(g1g2_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* G1G2_H */
