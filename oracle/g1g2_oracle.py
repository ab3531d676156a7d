"""Plain FP64 CPU oracle of the G1-G2 scheme (Joost, Schluenzen, Bonitz, arXiv:2002.12717).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this module.
It shares no code with the CUDA path and imports nothing from the product
package.

Everything is complex128 numpy; ħ = 1.  The "±" of the paper refers to
bosons/fermions (footnote to the KBE in Sec. II.A); every function that carries
one takes eta = +1 (bosons, upper sign) or eta = -1 (fermions, lower sign, the
default).  The equations are
written in the paper's own variables: the time-diagonal G^< and G^> of
Eq. (g-glsymm), the Hartree-Fock Hamiltonian of Eq. (h_HF), the two-particle
Hartree-Fock Hamiltonian of Eq. (twopart_hamiltonian), the source term Psi of
Eq. (psi-pm-def) evaluated by the successive contractions of
Eq. (soa-skalierung), the GW quasi-Hamiltonian of Eq. (gwhcorr) built from the
exchange products of Eq. (g2f-def), and the polarisation term of Eq. (gwpi).
Library einsum/matmul calls are single contraction steps; nothing is fused or
reordered beyond the formulas themselves.

State convention: the propagated variables are the density matrix n (called
G1 at the library boundary, n_ij = <c_j^dagger c_i>, Hermitian) and the
correlated two-particle function G2 = 𝒢 of Eq. (gscor-def), an nb^4 tensor
indexed [i, j, k, l].

Readings of the paper used here, where it leaves a choice open:
  * fermions by default, bosons with eta = +1 (each ± of the paper followed
    as printed: G^< of Eq. (g-glsymm), h^HF and w^± of Eq. (h_HF), I of
    Eq. (eom_gone-I), 𝔥 of Eq. (gwhcorr), the exchange term of Eq. (ini-g2));
    ħ = 1;
  * the integrator is classical RK4 on (n, 𝒢) jointly (the paper names none);
  * SOA uses Psi^- (w^- = w_pqrs - w_pqsr); GW uses the plain-w Psi
    (standard GW without exchange, Sec. IV.C);
  * the collision integral uses 𝒢_lpjk, Eq. (definition_D) / (eom_gone-I);
  * spin-restricted mode (a Hubbard-type interaction acting between opposite
    spins only, with n_up = n_down): the exchange term of h^HF and of Psi
    vanishes, the energies carry spin factors (Sec. III.D, Eqs.
    eom_g1_hubbard, colint_hubbard, g2-hubbard, phi-hubbard);
  * energies follow from the Hamiltonian Eq. (h) and the two-particle density
    matrix of Eq. (ini-g2); the paper prints no energy formula for 𝒢.
"""
from __future__ import annotations

import functools

import numpy as np

# every einsum below is one contraction step; optimize=True lets numpy hand a
# two-operand contraction to BLAS (tensordot) instead of its generic loop
einsum = functools.partial(np.einsum, optimize=True)

SOA = "SOA"
GW = "GW"
GWX = "GWX"   # GW with the exchange source term Psi^± (end of Sec. IV.C)
TPP = "TPP"   # particle-particle T matrix, Sec. IV.D, Eq. (g2-eq-tpp-lambda)
TPH = "TPH"   # particle-hole T matrix, Sec. IV.E, Eq. (g2-eq-tph-lambda)
DSL = "DSL"   # dynamically screened ladder, Sec. V, Eq. (g2-dsl-equation-pi-lambda)
HF = "HF"


# ---------------------------------------------------------------------------
# Sec. II.B: time-diagonal G^<, G^> and the Hartree-Fock Hamiltonian
# ---------------------------------------------------------------------------

def g_less(n, eta=-1):
    """Eq. (g-glsymm): G^<_ij = ±(1/iħ) n_ij, i.e. i n_ij for fermions, -i n_ij for bosons."""
    return eta * n / 1j


def g_greater(n, eta=-1):
    """Eq. (g-glsymm): G^> = G^< + delta/(i ħ) (-i (1 - n) for fermions, -i (1 + n) for bosons)."""
    return g_less(n, eta) + np.eye(n.shape[0]) / 1j


def w_pm(w, eta=-1):
    """Definition below Eq. (h_HF): w^±_ijkl = w_ijkl ± w_ijlk."""
    return w + eta * w.transpose(0, 1, 3, 2)


def w_antisym(w):
    """w^- of Eq. (h_HF), the fermion case."""
    return w_pm(w, -1)


def w_from_factors(L):
    """Factorised (density-fitted) interaction w_ijkl = Σ_P L^P_ik L^P_jl: the general-basis
    w of Eq. (h) written through nfac factors L[P] (nb x nb), each Hermitian or i times
    Hermitian so that w meets Eqs. (wsymm_a/b)."""
    return einsum("pik,pjl->ijkl", L, L)


def hf_hamiltonian(h, w, n, restricted=False, eta=-1):
    """Eq. (h_HF): h^HF_ij = h_ij ± iħ Σ_kl w^±_ikjl G^<_lk.

    In spin-restricted mode the exchange partner of the opposite-spin
    interaction vanishes and the plain w enters (Sec. III.D, h^HF of the
    Hubbard basis).
    """
    wt = w if restricted else w_pm(w, eta)
    return h + eta * 1j * einsum("ikjl,lk->ij", wt, g_less(n, eta))


def collision_integral(w, G2, eta=-1):
    """Eq. (definition_D) / (eom_gone-I): I_ij = ±iħ Σ_klp w_iklp 𝒢_lpjk."""
    return eta * 1j * einsum("iklp,lpjk->ij", w, G2)


def g1_rhs(hhf, n, I, eta=-1):
    """Eq. (eom_gone-2): i dG^</dt = [h^HF, G^<] + I + I^dagger, returned as dn/dt.

    With G^< = ±(1/i) n this is dn/dt = ±i dG^</dt.
    """
    gl = g_less(n, eta)
    dgl = -1j * (hhf @ gl - gl @ hhf + I + I.conj().T)
    return eta * 1j * dgl


# ---------------------------------------------------------------------------
# Sec. III.C: two-particle Hartree-Fock commutator and the SOA source term
# ---------------------------------------------------------------------------

def two_particle_commutator(hhf, G2):
    """[h^(2),HF, 𝒢]_ijkl with h^(2),HF_ijpq = δ_jq h_ip + δ_ip h_jq.

    Eq. (twopart_hamiltonian) inserted in Eq. (result_eom_soa); the sum over
    the Kronecker deltas is carried out, leaving the four single sums
    (the same form the paper writes for the Hubbard basis in Sec. VII.A).
    """
    return (einsum("ip,pjkl->ijkl", hhf, G2)
            + einsum("jp,ipkl->ijkl", hhf, G2)
            - einsum("ijpl,pk->ijkl", G2, hhf)
            - einsum("ijkp,pl->ijkl", G2, hhf))


def psi_source(wt, n, eta=-1):
    """Two-particle source term, Eq. (psi-pm-def) with Φ of Sec. III.B.

    Evaluated as Eq. (soa-skalierung): four independent single sums done as
    successive tensor contractions (s first, then r, q, p), once with
    (G^>, G^>, G^<, G^<) and once with (G^<, G^<, G^>, G^>), times (iħ)^2.
    `wt` is w^± for SOA (Psi^±) and the plain w for GW / spin-restricted mode.
    """
    gl, gg = g_less(n, eta), g_greater(n, eta)

    def chain(a, b, c, d):
        x = einsum("pqrs,sl->pqrl", wt, d)      # Σ_s w_pqrs d_sl
        x = einsum("rk,pqrl->pqkl", c, x)       # Σ_r c_rk (...)
        x = einsum("jq,pqkl->pjkl", b, x)       # Σ_q b_jq (...)
        return einsum("ip,pjkl->ijkl", a, x)    # Σ_p a_ip (...)

    return (1j ** 2) * (chain(gg, gg, gl, gl) - chain(gl, gl, gg, gg))


# ---------------------------------------------------------------------------
# Sec. IV.C: GW quasi-Hamiltonian and polarisation term
# ---------------------------------------------------------------------------

def g2_exchange(gx, gy):
    """Eq. (g2f-def) on the time diagonal: 𝒢^F_ijkl = G^x_il G^y_jk."""
    return einsum("il,jk->ijkl", gx, gy)


def gw_hcorr(w, n, eta=-1):
    """Eq. (gwhcorr): 𝔥_ijkl = ±(iħ)^2 Σ_pq w_qipk [𝒢^F,>_jplq - 𝒢^F,<_jplq].

    𝒢^F,> = G^> G^< and 𝒢^F,< = G^< G^> (Eq. g2f-def, time diagonal).
    """
    gl, gg = g_less(n, eta), g_greater(n, eta)
    fdiff = g2_exchange(gg, gl) - g2_exchange(gl, gg)
    return eta * (1j ** 2) * einsum("qipk,jplq->ijkl", w, fdiff)


def gw_polarisation(hcorr, G2):
    """Eq. (gwpi): Π_ijkl = Σ_pq 𝔥_qjpl 𝒢_ipkq."""
    return einsum("qjpl,ipkq->ijkl", hcorr, G2)


# ---------------------------------------------------------------------------
# Sec. IV.D: particle-particle T matrix
# ---------------------------------------------------------------------------

def tpp_hcorr(w, n, eta=-1):
    """Correlation part of the pp quasi-Hamiltonian, Eq. (HTPPcorr):
    hcorr_ijkl = (iħ)^2 Σ_pq [G^{H,>}_ijpq - G^{H,<}_ijpq] w_pqkl, with the Hartree
    product G^{H,≷}_ijpq = G^≷_ip G^≷_jq (Sec. II)."""
    gl, gg = g_less(n, eta), g_greater(n, eta)
    return (1j ** 2) * (einsum("ip,jq,pqkl->ijkl", gg, gg, w) - einsum("ip,jq,pqkl->ijkl", gl, gl, w))


def tpp_ladder(hcorr, G2):
    """Particle-particle ladder term, Eq. (lambdapp): Λ_ijkl = Σ_pq hcorr_ijpq 𝒢_pqkl."""
    return einsum("ijpq,pqkl->ijkl", hcorr, G2)


def tph_hcorr(w, n, eta=-1):
    """Correlation part of the ph quasi-Hamiltonian, Eq. (HTPHcorr):
    hcorr_ijkl = (iħ)^2 Σ_pq [G^{F,>}_iqlp - G^{F,<}_iqlp] w_pjkq, with the
    equal-time exchange product of Eq. (g2f-def), G^{F,≷}_iqlp = G^≷_ip G^≶_ql
    (the second factor is the opposite component)."""
    gl, gg = g_less(n, eta), g_greater(n, eta)
    return (1j ** 2) * (einsum("ip,ql,pjkq->ijkl", gg, gl, w) - einsum("ip,ql,pjkq->ijkl", gl, gg, w))


def tph_ladder(hcorr, G2):
    """Particle-hole ladder term, Eq. (lambdaph): Λ_ijkl = Σ_pq hcorr_ipql 𝒢_qjkp."""
    return einsum("ipql,qjkp->ijkl", hcorr, G2)


# ---------------------------------------------------------------------------
# The closed systems: SOA (Sec. III.C), GW (Sec. IV.C), HF (I = 0)
# ---------------------------------------------------------------------------

class Problem:
    """Static data of one propagation: h(t) = h + f(t) D, w, selfenergy, basis."""

    def __init__(self, h, w, selfenergy=SOA, restricted=False, D=None, drive=None, bosons=False):
        self.h = np.asarray(h, dtype=np.complex128)
        self.w = np.asarray(w, dtype=np.complex128)
        self.selfenergy = selfenergy
        self.restricted = restricted
        self.D = None if D is None else np.asarray(D, dtype=np.complex128)
        self.drive = drive  # callable f(t) -> float, or None
        self.eta = 1 if bosons else -1  # the ± of the paper
        if restricted and selfenergy in (GW, GWX, DSL):
            raise ValueError("GW couples same-spin components; no spin-restricted form")
        # source-term interaction: Psi^- for SOA in a spin-orbital basis and for
        # GW with exchange (Psi replaced by Psi^±, end of Sec. IV.C), plain w for
        # standard GW (Sec. IV.C) and for the opposite-spin restricted mode
        self.w_source = self.w if (restricted or selfenergy == GW) else w_pm(self.w, self.eta)

    def h_of_t(self, t):
        if self.D is None or self.drive is None:
            return self.h
        return self.h + self.drive(t) * self.D


def rhs(prob: Problem, t, n, G2):
    """(dn/dt, d𝒢/dt) of the G1-G2 scheme at time t.

    G1: Eq. (eom_gone-2) with I of Eq. (eom_gone-I).
    G2: SOA Eq. (result_eom_soa): i d𝒢/dt = [h2, 𝒢] + Psi^±;
        GW  Eq. (g2-eq-gw-pi):  i d𝒢/dt = [h2, 𝒢] + Psi + Π_ijkl - (Π_lkji)^*;
        GWX: the same with Psi replaced by Psi^± (end of Sec. IV.C);
        TPP Eq. (g2-eq-tpp-lambda): i d𝒢/dt = [h2, 𝒢] + Psi^± + Λ_ijkl - (Λ_klij)^*;
        TPH Eq. (g2-eq-tph-lambda): the same with the particle-hole ladder term;
        DSL Eq. (g2-dsl-equation-pi-lambda): Psi^± plus the GW polarisation term and
            both ladder terms, each once;
        HF: 𝒢 is not propagated (collision integral zero).
    """
    eta = prob.eta
    hhf = hf_hamiltonian(prob.h_of_t(t), prob.w, n, prob.restricted, eta)
    if prob.selfenergy == HF:
        I = np.zeros_like(n)
        return g1_rhs(hhf, n, I, eta), np.zeros_like(G2)
    I = collision_integral(prob.w, G2, eta)
    dn = g1_rhs(hhf, n, I, eta)
    rhs2 = two_particle_commutator(hhf, G2) + psi_source(prob.w_source, n, eta)
    if prob.selfenergy in (GW, GWX, DSL):
        pi = gw_polarisation(gw_hcorr(prob.w, n, eta), G2)
        rhs2 = rhs2 + pi - pi.transpose(3, 2, 1, 0).conj()
    if prob.selfenergy in (TPP, TPH, DSL):
        lam = np.zeros_like(G2)
        if prob.selfenergy in (TPP, DSL):
            lam = lam + tpp_ladder(tpp_hcorr(prob.w, n, eta), G2)
        if prob.selfenergy in (TPH, DSL):
            lam = lam + tph_ladder(tph_hcorr(prob.w, n, eta), G2)
        rhs2 = rhs2 + lam - lam.transpose(2, 3, 0, 1).conj()
    return dn, -1j * rhs2


def rk4_step(prob: Problem, t, n, G2, dt):
    """Classical fourth-order Runge-Kutta step on (n, 𝒢) jointly."""
    k1 = rhs(prob, t, n, G2)
    k2 = rhs(prob, t + dt / 2, n + dt / 2 * k1[0], G2 + dt / 2 * k1[1])
    k3 = rhs(prob, t + dt / 2, n + dt / 2 * k2[0], G2 + dt / 2 * k2[1])
    k4 = rhs(prob, t + dt, n + dt * k3[0], G2 + dt * k3[1])
    n_new = n + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
    G2_new = G2 + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    stage_dn = (k1[0], k2[0], k3[0], k4[0])
    return n_new, G2_new, stage_dn


# ---------------------------------------------------------------------------
# Observables: energies from Eq. (h) and the two-particle density matrix of
# Eq. (ini-g2), n_ijkl = n_ik n_jl ± n_il n_jk - 𝒢_ijkl (ħ = 1).
# ---------------------------------------------------------------------------

def energies(prob: Problem, t, n, G2):
    """Return dict with e_one, e_hf, e_corr, e_total, n_particles.

    <H> = Σ h_ij <c_i^† c_j> + ½ Σ w_ijkl <c_i^† c_j^† c_l c_k>, with
    <c_i^† c_j> = n_ji and <c_i^† c_j^† c_l c_k> = n_klij.
    Spin-restricted mode sums both spin species of an opposite-spin
    interaction: factor 2 on the one-body part and on both interaction parts.
    """
    h = prob.h_of_t(t)
    if prob.restricted:
        e1 = 2.0 * einsum("ij,ji->", h, n).real
        ehf = einsum("ijkl,ki,lj->", prob.w, n, n).real
        ecorr = -einsum("ijkl,klij->", prob.w, G2).real if prob.selfenergy != HF else 0.0
        npart = 2.0 * np.trace(n).real
    else:
        e1 = einsum("ij,ji->", h, n).real
        ehf = 0.5 * einsum("ijkl,ki,lj->", w_pm(prob.w, prob.eta), n, n).real
        ecorr = -0.5 * einsum("ijkl,klij->", prob.w, G2).real if prob.selfenergy != HF else 0.0
        npart = np.trace(n).real
    return {"e_one": e1, "e_hf": ehf, "e_corr": ecorr,
            "e_total": e1 + ehf + ecorr, "n_particles": npart}


def drive_power(prob: Problem, t, n):
    """<D> = Re Tr(D n) (times the spin factor in restricted mode).

    With h(t) = h + f(t) D the energy changes at the rate f'(t) <D>, so the
    drive work is W = ∫ f'(t) <D> dt; the caller multiplies by f'(t).
    """
    if prob.D is None:
        return 0.0
    s = 2.0 if prob.restricted else 1.0
    return s * einsum("ij,ji->", prob.D, n).real


def double_occupancy(n, G2, nsites, eta=-1):
    """E10: d_i = <n_i,up n_i,down> for spin-orbitals ordered (site, spin) = 2*site + spin.

    From Eq. (ini-g2): n_ijkl = n_ik n_jl ± n_il n_jk - 𝒢_ijkl with
    i = k = (site, up), j = l = (site, down).
    """
    d = np.empty(nsites)
    for s in range(nsites):
        u, dn = 2 * s, 2 * s + 1
        d[s] = (n[u, u] * n[dn, dn] + eta * n[u, dn] * n[dn, u] - G2[u, dn, u, dn]).real
    return d


def propagate(prob: Problem, n0, G2_0, dt, nsteps, t0=0.0, obs_every=1, dfdt=None):
    """RK4 propagation; returns (n, 𝒢, t, list of observable dicts).

    Each observable dict holds the energies, the time, the density n_ii
    (summed over spin in restricted mode) and the accumulated drive work
    W = ∫ f'(t) Re Tr(D n) dt, integrated with the RK4 weights on the stage
    states (Simpson-consistent with the step).
    """
    n, G2, t = n0.astype(np.complex128), G2_0.astype(np.complex128), t0
    work = 0.0
    obs = []

    def record():
        e = energies(prob, t, n, G2)
        e["t"] = t
        e["pulse_work"] = work
        s = 2.0 if prob.restricted else 1.0
        e["density"] = s * np.diag(n).real.copy()
        obs.append(e)

    record()
    for step in range(nsteps):
        if dfdt is not None and prob.D is not None:
            # stage states of this step for the work integral
            k1 = rhs(prob, t, n, G2)
            y2 = (n + dt / 2 * k1[0], G2 + dt / 2 * k1[1])
            k2 = rhs(prob, t + dt / 2, *y2)
            y3 = (n + dt / 2 * k2[0], G2 + dt / 2 * k2[1])
            k3 = rhs(prob, t + dt / 2, *y3)
            y4 = (n + dt * k3[0], G2 + dt * k3[1])
            k4 = rhs(prob, t + dt, *y4)
            p = [dfdt(t) * drive_power(prob, t, n),
                 dfdt(t + dt / 2) * drive_power(prob, t + dt / 2, y2[0]),
                 dfdt(t + dt / 2) * drive_power(prob, t + dt / 2, y3[0]),
                 dfdt(t + dt) * drive_power(prob, t + dt, y4[0])]
            work += dt / 6 * (p[0] + 2 * p[1] + 2 * p[2] + p[3])
            n = n + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
            G2 = G2 + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        else:
            n, G2, _ = rk4_step(prob, t, n, G2, dt)
        t = t0 + (step + 1) * dt
        if (step + 1) % obs_every == 0:
            record()
    return n, G2, t, obs
