"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Every test here checks the oracle against something other than itself:
exact many-body (Fock-space) dynamics, brute-force 8-index sums, explicit
Kronecker-product matrices, closed forms, conservation laws, the Hubbard
specialisations the paper prints, and the memory-integral HF-GKBA the
G1-G2 scheme is derived from.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import g1g2_oracle as O
from oracle.hfgkba import propagate_hfgkba
from paper_2002_12717_gb300 import inputs

from . import fock
from . import fock_bosons


def sym_w(nb, rng, real=False):
    """Random w with w_ijkl = w_jilk and w_ijkl = conj(w_klij) (Eqs. wsymm_a/b)."""
    x = rng.standard_normal((nb,) * 4)
    if not real:
        x = x + 1j * rng.standard_normal((nb,) * 4)
    x = x + x.transpose(1, 0, 3, 2)
    x = x + x.transpose(2, 3, 0, 1).conj()
    return x * 0.25


def random_fock_state(nb, npart, rng):
    dim = 1 << nb
    v = np.zeros(dim, dtype=np.complex128)
    for b in range(dim):
        if bin(b).count("1") == npart:
            v[b] = rng.standard_normal() + 1j * rng.standard_normal()
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# Exact many-body pins (Fock space, nb = 5 spin-orbitals)
# ---------------------------------------------------------------------------

def test_g1_equation_is_exact_first_hierarchy_equation():
    """Eq. (eom_gone) with I of Eq. (definition_D) is exact for any state.

    Pins h^HF (Eq. h_HF incl. the exchange term), the collision integral and
    its index order 𝒢_lpjk, and the sign conventions of Eq. (g-glsymm).
    """
    rng = np.random.default_rng(11)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    H = fock.hamiltonian(h, w)
    psi = random_fock_state(nb, 2, rng)
    n, n2 = fock.rdms(psi, nb)
    g2 = fock.correlated_g2(n, n2)
    exact = fock.time_derivative(H, psi, lambda v: fock.rdms(v, nb)[0])
    hhf = O.hf_hamiltonian(h, w, n)
    got = O.g1_rhs(hhf, n, O.collision_integral(w, g2))
    assert np.abs(got - exact).max() < 1e-8


def test_source_term_is_exact_initial_slope_from_slater_determinant():
    """From an uncorrelated state the exact d𝒢/dt equals -iΨ^- (Eq. dgdt-a).

    Pins the source term of Eq. (psi-pm-def): signs, index placement and the
    antisymmetrised w^- of the SOA.
    """
    rng = np.random.default_rng(12)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    H = fock.hamiltonian(h, w)
    orb = np.linalg.qr(rng.standard_normal((nb, 2)) + 1j * rng.standard_normal((nb, 2)))[0]
    psi = fock.slater(orb, nb)
    n, n2 = fock.rdms(psi, nb)
    assert np.abs(fock.correlated_g2(n, n2)).max() < 1e-12
    exact = fock.time_derivative(H, psi, lambda v: fock.correlated_g2(*fock.rdms(v, nb)))
    got = -1j * O.psi_source(O.w_antisym(w), n)
    assert np.abs(got - exact).max() < 1e-8
    # the plain-w source (GW reading) is a different function
    assert np.abs(-1j * O.psi_source(w, n) - exact).max() > 1e-3


def test_gw_with_exchange_has_the_exact_initial_slope():
    """GW with Psi replaced by Psi^± (end of Sec. IV.C): from an uncorrelated state
    (𝒢 = 0, so Π = 0) its full right-hand side is the exact d𝒢/dt, while standard
    GW (plain-w source) is not.  Pins the exchange variant's source and that the
    rest of its right-hand side vanishes at 𝒢 = 0."""
    rng = np.random.default_rng(21)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    H = fock.hamiltonian(h, w)
    orb = np.linalg.qr(rng.standard_normal((nb, 3)) + 1j * rng.standard_normal((nb, 3)))[0]
    psi = fock.slater(orb, nb)
    n, n2 = fock.rdms(psi, nb)
    g2 = fock.correlated_g2(n, n2)
    exact = fock.time_derivative(H, psi, lambda v: fock.correlated_g2(*fock.rdms(v, nb)))
    _, got = O.rhs(O.Problem(h, w, selfenergy=O.GWX), 0.0, n, g2)
    assert np.abs(got - exact).max() < 1e-8
    _, gw = O.rhs(O.Problem(h, w, selfenergy=O.GW), 0.0, n, g2)
    assert np.abs(gw - exact).max() > 1e-3


def test_commutator_is_exact_for_noninteracting_dynamics():
    """With w = 0 the exact correlated part obeys i d𝒢/dt = [h^(2), 𝒢] (Eq. result_eom_soa)."""
    rng = np.random.default_rng(13)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    H = fock.hamiltonian(h, np.zeros((nb,) * 4))
    psi = random_fock_state(nb, 2, rng)
    n, n2 = fock.rdms(psi, nb)
    g2 = fock.correlated_g2(n, n2)
    assert np.abs(g2).max() > 1e-2
    exact = fock.time_derivative(H, psi, lambda v: fock.correlated_g2(*fock.rdms(v, nb)))
    got = -1j * O.two_particle_commutator(h, g2)
    assert np.abs(got - exact).max() < 1e-8


def test_energy_equals_many_body_expectation():
    """E9 from the two-particle density matrix of Eq. (ini-g2) equals <ψ|H|ψ>."""
    rng = np.random.default_rng(14)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    H = fock.hamiltonian(h, w)
    psi = random_fock_state(nb, 3, rng)
    n, n2 = fock.rdms(psi, nb)
    g2 = fock.correlated_g2(n, n2)
    e = O.energies(O.Problem(h, w), 0.0, n, g2)
    assert abs(e["e_total"] - (psi.conj() @ H @ psi).real) < 1e-10
    assert abs(e["n_particles"] - 3.0) < 1e-12


def test_double_occupancy_equals_many_body_expectation():
    rng = np.random.default_rng(15)
    L = 2
    nb = 2 * L
    h = inputs.spin_orbital_h(inputs.chain_hopping(L))
    w = inputs.spin_orbital_hubbard_w(L, 2.0)
    psi = random_fock_state(nb, 2, rng)
    n, n2 = fock.rdms(psi, nb)
    g2 = fock.correlated_g2(n, n2)
    c = fock.annihilators(nb)
    for s in range(L):
        nu = c[2 * s].T @ c[2 * s]
        nd = c[2 * s + 1].T @ c[2 * s + 1]
        exact = (psi.conj() @ nu @ nd @ psi).real
        assert abs(O.double_occupancy(n, g2, L)[s] - exact) < 1e-12
    # E_corr of the Hubbard w is -U Σ_i 𝒢_{i↑i↓i↑i↓}-type terms; check E against <H>
    H = fock.hamiltonian(h, w)
    e = O.energies(O.Problem(h, w), 0.0, n, g2)
    assert abs(e["e_total"] - (psi.conj() @ H @ psi).real) < 1e-10


# ---------------------------------------------------------------------------
# Brute force and explicit matrices
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nb", [3, 4])
def test_psi_successive_contractions_equal_literal_phi_sum(nb):
    """Eq. (soa-skalierung) equals the literal Eq. (psi-pm-def) with Φ built from 𝒢^H."""
    rng = np.random.default_rng(20 + nb)
    n = inputs.random_hermitian(nb, rng) * 0.3 + 0.4 * np.eye(nb)
    w = sym_w(nb, rng)
    gl = 1j * n
    gg = gl - 1j * np.eye(nb)
    gh = lambda a: np.einsum("ip,jq->ijpq", a, a)          # 𝒢^H_ijpq = G_ip G_jq (Eq. g2h-def)
    # Φ^{ijkl}_{pqrs} = (iħ)^4 [𝒢^H,>_ijpq 𝒢^H,<_klrs - 𝒢^H,<_ijpq 𝒢^H,>_klrs]
    phi = (1j ** 4) * (np.einsum("ijpq,klrs->ijklpqrs", gh(gg), gh(gl))
                       - np.einsum("ijpq,klrs->ijklpqrs", gh(gl), gh(gg)))
    for wt in (w, O.w_antisym(w)):
        # Ψ_ijkl = (iħ)^-2 Σ_pqrs w_pqrs Φ^{ijrs}_{pqkl}
        literal = np.einsum("pqrs,ijrspqkl->ijkl", wt, phi) / (1j ** 2)
        assert np.abs(O.psi_source(wt, n) - literal).max() < 1e-12


def test_factorised_w_reproduces_the_hubbard_interactions():
    """w_from_factors against the paper's Hubbard interactions built element by element:
    the on-site opposite-spin w = U δ_ij δ_ik δ_il from the factors sqrt(U) e_a e_a^T, and
    the spin-orbital w of Eq. (wmatrix-hubbard) from two factors per site, the Hermitian
    sqrt(U/2) (E_up + E_dn) and i sqrt(U/2) (E_up - E_dn) (their same-spin parts cancel)."""
    L, U = 4, 1.7
    f = np.zeros((L, L, L), dtype=np.complex128)
    for a in range(L):
        f[a, a, a] = math.sqrt(U)
    assert np.abs(O.w_from_factors(f) - inputs.onsite_w_restricted(L, U)).max() < 1e-15
    nb = 2 * L
    f = np.zeros((2 * L, nb, nb), dtype=np.complex128)
    for s_ in range(L):
        up, dn = 2 * s_, 2 * s_ + 1
        f[2 * s_, up, up] = f[2 * s_, dn, dn] = math.sqrt(U / 2)
        f[2 * s_ + 1, up, up] = 1j * math.sqrt(U / 2)
        f[2 * s_ + 1, dn, dn] = -1j * math.sqrt(U / 2)
    assert np.abs(O.w_from_factors(f) - inputs.spin_orbital_hubbard_w(L, U)).max() < 1e-15


def test_factorised_w_symmetries_and_rank():
    """Hermitian and i-Hermitian factors give Eqs. (wsymm_a/b); real symmetric factors give a
    positive semidefinite (ik),(jl) matrix of rank nfac (a Coulomb-like integral tensor)."""
    rng = np.random.default_rng(3)
    nb, P = 5, 4
    a = rng.standard_normal((P, nb, nb)) + 1j * rng.standard_normal((P, nb, nb))
    herm = (a + a.conj().transpose(0, 2, 1)) / 2
    herm[1::2] *= 1j
    w = O.w_from_factors(herm)
    assert np.abs(w - w.transpose(1, 0, 3, 2)).max() < 1e-14
    assert np.abs(w - w.transpose(2, 3, 0, 1).conj()).max() < 1e-14
    b = rng.standard_normal((P, nb, nb))
    w = O.w_from_factors((b + b.transpose(0, 2, 1)) / 2)
    m = w.transpose(0, 2, 1, 3).reshape(nb * nb, nb * nb)
    ev = np.linalg.eigvalsh(m)
    assert ev.min() > -1e-13 * ev.max()
    assert int((ev > 1e-10 * ev.max()).sum()) == P


@pytest.mark.parametrize("eta", [-1, 1])
def test_psi_for_factorised_w_equals_factor_products(eta):
    """For w = Σ_P L^P ⊗ L^P each sum of the successive contractions of Eq. (soa-skalierung)
    acts on one factor: Σ_pqrs a_ip b_jq w_pqrs c_rk d_sl = Σ_P (a L^P c)_ik (b L^P d)_jl, and
    the exchange part of w^± pairs (a L^P d)_il with (b L^P c)_jk.  psi_source (plain w and
    w^±, fermions and bosons) against these nb^3 factor products."""
    rng = np.random.default_rng(11)
    nb, P = 5, 6
    b = rng.standard_normal((P, nb, nb))
    L = (b + b.transpose(0, 2, 1)) / 2
    w = O.w_from_factors(L)
    n, _ = inputs.random_state(nb, rng, soa=False)
    gl, gg = O.g_less(n, eta), O.g_greater(n, eta)

    def chain(a, b_, c, d, pm):
        x = sum(np.einsum("ik,jl->ijkl", a @ Lp @ c, b_ @ Lp @ d) for Lp in L)
        if pm:
            x = x + eta * sum(np.einsum("il,jk->ijkl", a @ Lp @ d, b_ @ Lp @ c) for Lp in L)
        return x
    for pm in (False, True):
        ref = -(chain(gg, gg, gl, gl, pm) - chain(gl, gl, gg, gg, pm))
        got = O.psi_source(O.w_pm(w, eta) if pm else w, n, eta)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_commutator_equals_kronecker_matrix_commutator():
    """Eq. (twopart_hamiltonian): h2 = 1⊗h + h⊗1 as an nb^2 x nb^2 matrix."""
    rng = np.random.default_rng(30)
    nb = 4
    h = inputs.random_hermitian(nb, rng)
    g2 = rng.standard_normal((nb,) * 4) + 1j * rng.standard_normal((nb,) * 4)
    eye = np.eye(nb)
    h2 = np.einsum("jl,ik->ijkl", eye, h) + np.einsum("ik,jl->ijkl", eye, h)
    m = g2.reshape(nb * nb, nb * nb)
    hm = h2.reshape(nb * nb, nb * nb)
    want = (hm @ m - m @ hm).reshape((nb,) * 4)
    assert np.abs(O.two_particle_commutator(h, g2) - want).max() < 1e-12


def test_hf_hamiltonian_is_energy_gradient():
    """h^HF - h = ∂E_HF/∂n^T for both bases (consistency of Eq. h_HF with E9)."""
    rng = np.random.default_rng(31)
    nb = 4
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng, real=True)
    n = inputs.random_hermitian(nb, rng) * 0.2 + 0.5 * np.eye(nb)
    for restricted in (False, True):
        prob = O.Problem(h, w, restricted=restricted)
        hhf = O.hf_hamiltonian(h, w, n, restricted)
        s = 2.0 if restricted else 1.0
        eps = 1e-6
        grad = np.zeros((nb, nb), dtype=np.complex128)
        for a in range(nb):
            for b in range(nb):
                for part, unit in ((0, 1.0), (1, 1j)):
                    dn = np.zeros((nb, nb), dtype=np.complex128)
                    dn[b, a] += unit * eps
                    ep = O.energies(prob, 0, n + dn, 0 * w)["e_hf"]
                    em = O.energies(prob, 0, n - dn, 0 * w)["e_hf"]
                    d = (ep - em) / (2 * eps)
                    grad[a, b] += d if part == 0 else -1j * d
        # E_HF(n + dn) - E_HF(n) = Re Σ (h^HF - h)_ab dn_ba * s  (dn Hermitian-free probe)
        assert np.abs(grad - s * (hhf - h)).max() < 1e-6


def test_gw_hcorr_matches_delta_reduction():
    """Eq. (gwhcorr) with Eq. (g2f-def): the G^>G^< - G^<G^> difference is δ-terms of n."""
    rng = np.random.default_rng(32)
    nb = 4
    w = sym_w(nb, rng)
    n = inputs.random_hermitian(nb, rng) * 0.2 + 0.5 * np.eye(nb)
    eye = np.eye(nb)
    # G^>_jq G^<_pl - G^<_jq G^>_pl = δ_jq n_pl - n_jq δ_pl  (brute force over all indices)
    want = np.zeros((nb,) * 4, dtype=np.complex128)
    for i in range(nb):
        for j in range(nb):
            for k in range(nb):
                for l in range(nb):
                    acc = 0
                    for p in range(nb):
                        for q in range(nb):
                            acc += w[q, i, p, k] * (eye[j, q] * n[p, l] - n[j, q] * eye[p, l])
                    want[i, j, k, l] = acc
    assert np.abs(O.gw_hcorr(w, n) - want).max() < 1e-12


# ---------------------------------------------------------------------------
# Hubbard specialisations printed in the paper
# ---------------------------------------------------------------------------

def test_hubbard_soa_source_matches_phi_hubbard():
    """Eq. (g2-hubbard) with Φ of Eq. (phi-hubbard) equals the restricted-mode Ψ."""
    rng = np.random.default_rng(40)
    L, U = 4, 1.7
    n = inputs.random_hermitian(L, rng) * 0.2 + 0.5 * np.eye(L)
    gl = 1j * n
    gg = gl - 1j * np.eye(L)
    phi = (1j ** 4) * (np.einsum("ip,jp,pk,pl->ijkl", gg, gg, gl, gl)
                       - np.einsum("ip,jp,pk,pl->ijkl", gl, gl, gg, gg))
    want = U * phi / (1j ** 2)
    got = O.psi_source(inputs.onsite_w_restricted(L, U).astype(complex), n)
    assert np.abs(got - want).max() < 1e-12


def test_hubbard_gw_polarisation_matches_pihubbardtrans():
    """Eq. (pihubbardtrans): the general Π with the spin-orbital Hubbard w, ↑↓↑↓ block."""
    rng = np.random.default_rng(41)
    L, U = 3, 1.3
    nb = 2 * L
    w = inputs.spin_orbital_hubbard_w(L, U).astype(complex)
    ns = inputs.random_hermitian(L, rng) * 0.2 + 0.5 * np.eye(L)
    n = np.kron(ns, np.eye(2))
    _, g2 = inputs.random_state(nb, rng, soa=False)
    pi = O.gw_polarisation(O.gw_hcorr(w, n), g2)
    g_uuuu = g2[0::2, 0::2, 0::2, 0::2]
    gl = 1j * ns
    gg = gl - 1j * np.eye(L)
    # Π^{↑↓↑↓}_ijkl = -(iħ)^2 U Σ_p [G^>_jp G^<_pl - G^<_jp G^>_pl] 𝒢^{↑↑↑↑}_ipkp
    want = np.zeros((L,) * 4, dtype=complex)
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    for p in range(L):
                        want[i, j, k, l] += -(1j ** 2) * U * (gg[j, p] * gl[p, l] - gl[j, p] * gg[p, l]) \
                            * g_uuuu[i, p, k, p]
    got = pi[0::2, 1::2, 0::2, 1::2]
    assert np.abs(got - want).max() < 1e-12
    assert np.abs(want).max() > 1e-3


def test_restricted_mode_equals_spin_orbital_hubbard():
    """Restricted chain of L sites == spin-orbital chain of 2L orbitals (SOA, Sec. III.D)."""
    L, U = 3, 1.0
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 2.0
    n_site = inputs.lowest_projector(inputs.chain_hopping(L), 1) * 0 + np.diag([0.7, 0.4, 0.4]).astype(complex)
    pr = O.Problem(hs, inputs.onsite_w_restricted(L, U), restricted=True)
    ps = O.Problem(inputs.spin_orbital_h(hs), inputs.spin_orbital_hubbard_w(L, U))
    nr, gr, _, obr = O.propagate(pr, n_site, np.zeros((L,) * 4), 0.02, 50)
    nso, gso, _, obs = O.propagate(ps, np.kron(n_site, np.eye(2)), np.zeros((2 * L,) * 4), 0.02, 50)
    assert np.abs(nso[0::2, 0::2] - nr).max() < 1e-12
    assert np.abs(gso[0::2, 1::2, 0::2, 1::2] - gr).max() < 1e-12
    assert abs(obr[-1]["e_total"] - obs[-1]["e_total"]) < 1e-12


# ---------------------------------------------------------------------------
# Closed forms and conservation laws
# ---------------------------------------------------------------------------

def test_noninteracting_closed_form():
    """w = 0: 𝒢 stays 0 and n(t) = e^{-iht} n0 e^{iht} (Eq. eom_gone-2 with I = 0)."""
    rng = np.random.default_rng(50)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    n0 = inputs.lowest_projector(inputs.random_hermitian(nb, rng), 2)
    prob = O.Problem(h, np.zeros((nb,) * 4))
    errs = []
    for dt in (0.02, 0.01):
        n, g2, t, _ = O.propagate(prob, n0, np.zeros((nb,) * 4), dt, int(round(2.0 / dt)))
        u = expm(-1j * h * t)
        errs.append(np.abs(n - u @ n0 @ u.conj().T).max())
        assert np.abs(g2).max() == 0.0
    assert errs[1] < 1e-8 and 12 < errs[0] / errs[1] < 20      # RK4: O(dt^4)


def test_hubbard_chain_initial_state_closed_form():
    """Open 8-site chain at half filling: HF ground state energies in closed form."""
    d = inputs.hubbard_chain_restricted()
    prob = O.Problem(inputs.chain_hopping(8), d["w"], restricted=True)
    e = O.energies(prob, 0.0, d["n0"], np.zeros((8,) * 4))
    e_tb = 2 * sum(-2 * math.cos(math.pi * k / 9) for k in range(1, 5))
    assert abs(e["e_one"] - e_tb) < 1e-12
    assert abs(e["e_hf"] - 8 * 0.25 * 1.0) < 1e-12          # U Σ_i n_ii^2 with n_ii = 1/2
    assert np.abs(np.diag(d["n0"]).real - 0.5).max() < 1e-12
    # the state is self-consistent: [h^HF(n0), n0] = 0
    hhf = O.hf_hamiltonian(inputs.chain_hopping(8), d["w"], d["n0"], True)
    assert np.abs(hhf @ d["n0"] - d["n0"] @ hhf).max() < 1e-12


def test_tpp_ladder_matches_lambdapp_hubbard():
    """The general ladder term (Eqs. HTPPcorr, lambdapp) with the spin-restricted
    on-site interaction equals the printed Hubbard form, Eq. (lambdapp_hubb):
    Λ_ijkl = (iħ)^2 U Σ_p [G^>_ip G^>_jp - G^<_ip G^<_jp] 𝒢_ppkl.  Pins the sign,
    the G^> / G^< order and the index placement of the quasi-Hamiltonian."""
    rng = np.random.default_rng(31)
    nb, U = 6, 1.7
    w = inputs.onsite_w_restricted(nb, U).astype(np.complex128)
    n = inputs.random_hermitian(nb, rng) * 0.3 + 0.5 * np.eye(nb)
    g2 = rng.standard_normal((nb,) * 4) + 1j * rng.standard_normal((nb,) * 4)
    got = O.tpp_ladder(O.tpp_hcorr(w, n), g2)
    gl, gg = 1j * n, 1j * n - 1j * np.eye(nb)
    printed = (1j ** 2) * U * np.einsum("ip,jp,ppkl->ijkl", gg, gg, g2) - \
        (1j ** 2) * U * np.einsum("ip,jp,ppkl->ijkl", gl, gl, g2)
    assert np.abs(got - printed).max() < 1e-13 * max(1.0, np.abs(printed).max())


def test_tpp_separated_form_equals_full_quasi_hamiltonian_form():
    """Eq. (g2-eq-tpp), written with the full pp quasi-Hamiltonian h^Ω = h^(2),HF + hcorr
    (Eq. h-om-pp-def; hcorr here as a Kronecker matrix product) and conjugated 𝒢,
    equals the separated form of Eq. (g2-eq-tpp-lambda) that the oracle evaluates
    (complex w: pins the index order of w as well)."""
    rng = np.random.default_rng(32)
    nb = 5
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    n, g2 = inputs.random_state(nb, rng, soa=True)
    prob = O.Problem(h, w, selfenergy=O.TPP)
    _, got = O.rhs(prob, 0.0, n, g2)
    hhf = O.hf_hamiltonian(h, w, n)
    eye = np.eye(nb)
    h2 = np.einsum("jl,ik->ijkl", eye, hhf) + np.einsum("ik,jl->ijkl", eye, hhf)   # Eq. (twopart_hamiltonian)
    # hcorr as the nb^2 x nb^2 matrix (iħ)^2 (G^> ⊗ G^> - G^< ⊗ G^<) W, W_(pq),(kl) = w_pqkl
    gl, gg = 1j * n, 1j * n - 1j * eye
    hc = (1j ** 2) * (np.kron(gg, gg) - np.kron(gl, gl)) @ w.reshape(nb * nb, nb * nb)
    hom = h2 + hc.reshape((nb,) * 4)
    full = O.psi_source(O.w_antisym(w), n) + np.einsum("ijpq,klpq->ijkl", hom, g2.conj()) \
        - np.einsum("ijpq,klpq->ijkl", g2, hom.conj())
    assert np.abs(-1j * full - got).max() < 1e-12 * np.abs(got).max()


def test_tph_ladder_matches_lambdaph_hubbard():
    """The general particle-hole ladder term (Eqs. HTPHcorr, lambdaph) with the
    spin-restricted on-site interaction equals the printed Hubbard form, Eq.
    (lambdaph_hubb): Λ_ijkl = (iħ)^2 U Σ_p [G^>_ip G^<_pl - G^<_ip G^>_pl] 𝒢_pjkp.
    Pins the mixed G^>/G^< exchange product and the index placement."""
    rng = np.random.default_rng(41)
    nb, U = 6, 1.3
    w = inputs.onsite_w_restricted(nb, U).astype(np.complex128)
    n = inputs.random_hermitian(nb, rng) * 0.3 + 0.5 * np.eye(nb)
    g2 = rng.standard_normal((nb,) * 4) + 1j * rng.standard_normal((nb,) * 4)
    got = O.tph_ladder(O.tph_hcorr(w, n), g2)
    gl, gg = 1j * n, 1j * n - 1j * np.eye(nb)
    printed = (1j ** 2) * U * (np.einsum("ip,pl,pjkp->ijkl", gg, gl, g2) - np.einsum("ip,pl,pjkp->ijkl", gl, gg, g2))
    assert np.abs(got - printed).max() < 1e-13 * max(1.0, np.abs(printed).max())


def test_tph_separated_form_equals_full_quasi_hamiltonian_form():
    """Eq. (g2-eq-tph) with the full ph quasi-Hamiltonian (Eq. homph-def: the HF part
    δ_jl h_ik - δ_ik h_jl plus hcorr, here summed over p, q in plain loops of the
    printed index pattern) equals the separated form of Eq. (g2-eq-tph-lambda)."""
    rng = np.random.default_rng(42)
    nb = 4
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    n, g2 = inputs.random_state(nb, rng, soa=False)
    _, got = O.rhs(O.Problem(h, w, selfenergy=O.TPH), 0.0, n, g2)
    hhf = O.hf_hamiltonian(h, w, n)
    gl, gg = 1j * n, 1j * n - 1j * np.eye(nb)
    hom = np.zeros((nb,) * 4, dtype=np.complex128)
    for i in range(nb):
        for j in range(nb):
            for k in range(nb):
                for l in range(nb):
                    v = (hhf[i, k] if j == l else 0) - (hhf[j, l] if i == k else 0)
                    for p in range(nb):
                        for q in range(nb):
                            # G^{F,>}_iqlp - G^{F,<}_iqlp = G^>_ip G^<_ql - G^<_ip G^>_ql
                            v += (1j ** 2) * (gg[i, p] * gl[q, l] - gl[i, p] * gg[q, l]) * w[p, j, k, q]
                    hom[i, j, k, l] = v
    full = O.psi_source(O.w_antisym(w), n) + np.einsum("ipql,kpqj->ijkl", hom, g2.conj()) \
        - np.einsum("ipql,kpqj->ijkl", g2, hom.conj())
    assert np.abs(-1j * full - got).max() < 1e-12 * np.abs(got).max()


def test_dsl_equals_printed_quasi_hamiltonian_form_and_is_additive():
    """Eq. (g2-dsl-equation): Psi^± plus, for each of the GW, pp and ph quasi-Hamiltonians,
    hcorr times conjugated 𝒢 minus its conjugate, in the index patterns printed there
    (the third sum is over p, q), equals the Π/Λ form the oracle evaluates (Eq.
    g2-dsl-equation-pi-lambda).  This also checks the GW polarisation term in its
    conjugated form.  And each correlation term enters once: DSL - SOA is the sum of
    (GWX - SOA), (TPP - SOA) and (TPH - SOA)."""
    rng = np.random.default_rng(51)
    nb = 4
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng)
    n, g2 = inputs.random_state(nb, rng, soa=False)
    _, got = O.rhs(O.Problem(h, w, selfenergy=O.DSL), 0.0, n, g2)
    hhf = O.hf_hamiltonian(h, w, n)
    he, hpp, hph = O.gw_hcorr(w, n), O.tpp_hcorr(w, n), O.tph_hcorr(w, n)
    gc = g2.conj()
    full = O.two_particle_commutator(hhf, g2) + O.psi_source(O.w_antisym(w), n)
    full = full + np.einsum("qjpl,qkpi->ijkl", he, gc) - np.einsum("qjpl,qkpi->ijkl", g2, he.conj())
    full = full + np.einsum("ijpq,klpq->ijkl", hpp, gc) - np.einsum("ijpq,klpq->ijkl", g2, hpp.conj())
    full = full + np.einsum("ipql,kpqj->ijkl", hph, gc) - np.einsum("ipql,kpqj->ijkl", g2, hph.conj())
    assert np.abs(-1j * full - got).max() < 1e-12 * np.abs(got).max()
    parts = {se: O.rhs(O.Problem(h, w, selfenergy=se), 0.0, n, g2)[1] for se in (O.SOA, O.GWX, O.TPP, O.TPH)}
    additive = parts[O.GWX] + parts[O.TPP] + parts[O.TPH] - 2 * parts[O.SOA]
    assert np.abs(additive - got).max() < 1e-12 * np.abs(got).max()


# ---------------------------------------------------------------------------
# Bosons (the upper sign of every ± in the paper), exact bosonic Fock space
# ---------------------------------------------------------------------------

def _random_unitary(m, rng):
    q, r = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_boson_g1_equation_and_energy_are_exact_for_any_state():
    """Bosons: the G1 equation (Eq. eom_gone-2 with I of Eq. eom_gone-I, h^HF with w^+)
    is the exact first hierarchy equation for any state, with 𝒢 from Eq. (ini-g2)
    (upper sign), and the energy equals <H>.  Three bosons in four modes, random
    superposition, complex w; the fermion signs fail the same check."""
    rng = np.random.default_rng(71)
    M = 4
    S = fock_bosons.Space(M, 3)
    psi = np.zeros(S.dim, dtype=np.complex128)
    idx = S.sector(3)
    psi[idx] = rng.standard_normal(len(idx)) + 1j * rng.standard_normal(len(idx))
    psi /= np.linalg.norm(psi)
    rho = np.outer(psi, psi.conj())
    h = inputs.random_hermitian(M, rng)
    w = sym_w(M, rng) * 0.6
    H = S.hamiltonian(h, w)
    n, n2 = S.rdms(rho)
    g2 = fock_bosons.correlated_g2(n, n2)
    assert np.abs(g2).max() > 0.1                      # a strongly correlated state
    dn_exact, _ = S.rdm_rates(rho, H)
    prob = O.Problem(h, w, "SOA", bosons=True)
    dn, _ = O.rhs(prob, 0.0, n, g2)
    assert np.abs(dn - dn_exact).max() < 1e-12 * max(1.0, np.abs(dn_exact).max())
    e = O.energies(prob, 0.0, n, g2)
    assert abs(e["e_total"] - np.trace(rho @ H).real) < 1e-12
    dn_f, _ = O.rhs(O.Problem(h, w, "SOA"), 0.0, n, g2)
    assert np.abs(dn_f - dn_exact).max() > 1e-2


def test_boson_source_term_is_exact_initial_slope_from_gaussian_state():
    """Bosons: from a quasi-free (Gaussian) state, where 𝒢 = 0, the exact d𝒢/dt is
    -iΨ^+ (Eq. psi-pm-def with G^> = -i(1 + n), G^< = -i n and w^+), and dn/dt
    follows Eq. (eom_gone-2).  Thermal state of rotated modes (non-diagonal n), three
    modes, Fock space truncated at 16 bosons (tail below 1e-15)."""
    rng = np.random.default_rng(72)
    M = 3
    S = fock_bosons.Space(M, 16)
    rho = fock_bosons.gaussian_state(S, np.array([2.3, 2.6, 3.0]), _random_unitary(M, rng))
    h = inputs.random_hermitian(M, rng)
    w = sym_w(M, rng)
    H = S.hamiltonian(h, w)
    n, n2 = S.rdms(rho)
    assert np.abs(fock_bosons.correlated_g2(n, n2)).max() < 1e-13
    assert np.abs(n - np.diag(np.diag(n))).max() > 1e-2          # not diagonal in the mode basis
    dn_exact, dn2_exact = S.rdm_rates(rho, H)
    dg_exact = fock_bosons.correlated_g2_rate(n, n2, dn_exact, dn2_exact)
    g0 = np.zeros((M,) * 4, dtype=np.complex128)
    dn, dg = O.rhs(O.Problem(h, w, "SOA", bosons=True), 0.0, n, g0)
    scale = np.abs(dg_exact).max()
    assert scale > 1e-3
    assert np.abs(dg - dg_exact).max() < 1e-11 * scale
    assert np.abs(dn - dn_exact).max() < 1e-12
    # the boson source term differs from the fermion one (w^- and 1 - n) on this state
    _, dg_f = O.rhs(O.Problem(h, w, "SOA"), 0.0, n, g0)
    assert np.abs(dg_f - dg_exact).max() > 1e-2 * scale


def test_boson_gw_quasi_hamiltonian_equals_the_fermion_one():
    """Eq. (gwhcorr) carries a ± in front and G^≷ change with the statistics; for the
    time-diagonal products the two signs cancel (G^>G^< - G^<G^> flips sign with
    the statistics), so 𝔥 is the same δ-reduction for bosons as for fermions."""
    rng = np.random.default_rng(73)
    nb = 4
    w = sym_w(nb, rng)
    n = inputs.random_hermitian(nb, rng) * 0.2 + 0.5 * np.eye(nb)
    want = np.einsum("jipk,pl->ijkl", w, n) - np.einsum("qilk,jq->ijkl", w, n)
    assert np.abs(O.gw_hcorr(w, n, eta=1) - want).max() < 1e-12
    assert np.abs(O.gw_hcorr(w, n, eta=-1) - want).max() < 1e-12


def test_boson_g1g2_equals_memory_integral_hfgkba():
    """Bosons: the G1-G2 SOA equations reproduce the memory-integral HF-GKBA at second
    order in dt (Sec. III.C), two-site Bose-Hubbard chain (spinless, w_iiii = U)."""
    hs = inputs.chain_hopping(2)
    hs[0, 0] += 1.0
    w = np.zeros((2,) * 4, dtype=np.complex128)
    w[0, 0, 0, 0] = w[1, 1, 1, 1] = 1.0
    prob = O.Problem(hs.astype(np.complex128), w, bosons=True)
    n0 = np.diag([0.6, 0.3]).astype(np.complex128)
    T = 2.0
    n_ref, _, _, _ = O.propagate(prob, n0, np.zeros((2,) * 4), 0.005, int(T / 0.005))
    errs = []
    for dt in (0.1, 0.05):
        ns = propagate_hfgkba(prob, n0, dt, int(round(T / dt)))
        errs.append(np.abs(ns[-1] - n_ref).max())
    assert errs[1] < 2e-3 and 3.0 < errs[0] / errs[1] < 5.0


def test_boson_t_matrix_quasi_hamiltonians_in_plain_loops():
    """Eqs. (HTPPcorr) and (HTPHcorr) in plain loops with the boson components of
    Eq. (g-glsymm) written out: G^< = -i n, G^> = -i (1 + n) (upper sign)."""
    rng = np.random.default_rng(74)
    nb = 3
    w = sym_w(nb, rng)
    n = inputs.random_hermitian(nb, rng) * 0.3 + 0.4 * np.eye(nb)
    gl = -1j * n
    gg = -1j * (np.eye(nb) + n)
    pp = np.zeros((nb,) * 4, dtype=np.complex128)
    ph = np.zeros((nb,) * 4, dtype=np.complex128)
    for i in range(nb):
        for j in range(nb):
            for k in range(nb):
                for l in range(nb):
                    a = b = 0
                    for p in range(nb):
                        for q in range(nb):
                            # Hartree products G^≷_ip G^≷_jq; exchange products G^≷_ip G^≶_ql
                            a += (gg[i, p] * gg[j, q] - gl[i, p] * gl[j, q]) * w[p, q, k, l]
                            b += (gg[i, p] * gl[q, l] - gl[i, p] * gg[q, l]) * w[p, j, k, q]
                    pp[i, j, k, l] = -a        # (iħ)^2 = -1
                    ph[i, j, k, l] = -b
    assert np.abs(O.tpp_hcorr(w, n, eta=1) - pp).max() < 1e-12
    assert np.abs(O.tph_hcorr(w, n, eta=1) - ph).max() < 1e-12


@pytest.mark.parametrize("se", ["HF", "SOA", "GW", "GWX", "TPP", "TPH", "DSL"])
def test_boson_conservation_laws(se):
    """Bosons, spinless Bose-Hubbard chain (w_iiii = U): particle number to round-off,
    energy to O(dt^4) with E_HF from w^+ (Eq. ini-g2, upper sign), the 𝒢 symmetries."""
    L = 4
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 1.5
    w = np.zeros((L,) * 4, dtype=np.complex128)
    for i in range(L):
        w[i, i, i, i] = 0.8
    prob = O.Problem(hs.astype(np.complex128), w, selfenergy=se, bosons=True)
    n0 = np.diag([0.9, 0.6, 0.3, 0.1]).astype(np.complex128)
    drifts = []
    for dt in (0.04, 0.02):
        steps = int(round(2.0 / dt))
        n, g2, _, obs = O.propagate(prob, n0, np.zeros((L,) * 4), dt, steps, obs_every=steps)
        assert abs(obs[-1]["n_particles"] - obs[0]["n_particles"]) < 1e-12
        drifts.append(abs(obs[-1]["e_total"] - obs[0]["e_total"]))
        assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-14
        assert np.abs(g2 - g2.transpose(2, 3, 0, 1).conj()).max() < 1e-14
    if se == "HF":
        assert drifts[1] < 1e-8
    else:
        assert np.abs(g2).max() > 1e-3
        assert drifts[0] > 0 and 10 < drifts[0] / drifts[1] < 24   # ~2^4


@pytest.mark.parametrize("se", ["HF", "SOA", "GW", "GWX", "TPP", "TPH", "DSL"])
def test_conservation_laws(se):
    """Particle number to round-off; energy to O(dt^4) (Sec. VIII: energy conserving)."""
    L = 3
    nb = 2 * L
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 2.0
    prob = O.Problem(inputs.spin_orbital_h(hs), inputs.spin_orbital_hubbard_w(L, 1.0), selfenergy=se)
    n0 = np.kron(inputs.lowest_projector(inputs.chain_hopping(L), 2) * 0 + np.diag([0.8, 0.5, 0.2]), np.eye(2))
    drifts = []
    for dt in (0.04, 0.02):
        steps = int(round(2.0 / dt))
        n, g2, _, obs = O.propagate(prob, n0.astype(complex), np.zeros((nb,) * 4), dt, steps, obs_every=steps)
        assert abs(obs[-1]["n_particles"] - obs[0]["n_particles"]) < 1e-12
        drifts.append(abs(obs[-1]["e_total"] - obs[0]["e_total"]))
        # 𝒢 symmetries of Eqs. (Gsymm_a/b)
        assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-14
        assert np.abs(g2 - g2.transpose(2, 3, 0, 1).conj()).max() < 1e-14
        if se in ("SOA", "TPP"):
            assert np.abs(g2 + g2.transpose(0, 1, 3, 2)).max() < 1e-14
    if se == "HF":
        assert drifts[1] < 1e-8
    else:
        assert drifts[0] > 0 and 10 < drifts[0] / drifts[1] < 24   # ~2^4


def test_energy_balance_with_drive():
    """E(T) - E(0) equals the drive work ∫ f'(t) <D> dt to O(dt^4)."""
    rng = np.random.default_rng(60)
    nb = 4
    h = inputs.random_hermitian(nb, rng)
    w = sym_w(nb, rng, real=True)
    D = np.diag(rng.standard_normal(nb)).astype(complex)
    drv = inputs.GaussSine(A=0.5, omega=1.5, t0=1.0, sigma=0.5)
    n0 = inputs.lowest_projector(h, 2)
    res = []
    for se in ("SOA", "GW"):
        prob = O.Problem(h, w, selfenergy=se, D=D, drive=drv.f)
        errs = []
        for dt in (0.04, 0.02):
            steps = int(round(2.0 / dt))
            _, _, _, obs = O.propagate(prob, n0, np.zeros((nb,) * 4), dt, steps, obs_every=steps,
                                       dfdt=drv.dfdt)
            errs.append(abs(obs[-1]["e_total"] - obs[0]["e_total"] - obs[-1]["pulse_work"]))
        assert abs(obs[-1]["pulse_work"]) > 1e-3
        assert errs[1] < 1e-6 and errs[0] / errs[1] > 8
        res.append(errs)


def test_g1g2_equals_memory_integral_hfgkba():
    """The G1-G2 SOA equations reproduce the non-Markovian HF-GKBA (Sec. III.C, Fig. densities).

    Hubbard dimer (4 spin-orbitals), U = J, half filling, uncorrelated start, quench.
    The memory-integral solution converges to the G1-G2 one at second order.
    """
    L = 2
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 1.0
    prob = O.Problem(inputs.spin_orbital_h(hs), inputs.spin_orbital_hubbard_w(L, 1.0))
    n0 = np.kron(inputs.lowest_projector(inputs.chain_hopping(L), 1), np.eye(2))
    T = 2.0
    n_ref, _, _, _ = O.propagate(prob, n0, np.zeros((4,) * 4), 0.005, int(T / 0.005))
    errs = []
    for dt in (0.1, 0.05):
        ns = propagate_hfgkba(prob, n0, dt, int(round(T / dt)))
        errs.append(np.abs(ns[-1] - n_ref).max())
    assert errs[1] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_g1g2_solution_satisfies_the_interval_recursion():
    """Eq. (linintG): 𝒢(T + Δ) is 𝒢(T) carried by the two-particle HF propagator,
    (u⊗u) 𝒢(T) (u⊗u)^† with u = u(T+Δ, T), plus the memory integral of Eq.
    (dtilde-solution-short) over [T, T + Δ] alone.  The G1-G2 RK4 solution (fine step)
    satisfies it up to the quadrature of the reconstruction: midpoint propagators and
    the trapezoid rule on a grid of step h, second order in h."""
    L = 2
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 1.0
    prob = O.Problem(inputs.spin_orbital_h(hs), inputs.spin_orbital_hubbard_w(L, 1.0))
    nb = 2 * L
    n = np.kron(inputs.lowest_projector(inputs.chain_hopping(L), 1), np.eye(2)).astype(np.complex128)
    g2 = np.zeros((nb,) * 4, dtype=np.complex128)
    fine, T, Delta = 0.0025, 1.0, 0.4
    for _ in range(int(round(T / fine))):
        n, g2, _ = O.rk4_step(prob, 0.0, n, g2, fine)
    traj = [(n, g2)]                                   # the fine trajectory over [T, T + Δ]
    for _ in range(int(round(Delta / fine))):
        n, g2, _ = O.rk4_step(prob, 0.0, *traj[-1], fine)
        traj.append((n, g2))
    g_end = traj[-1][1]

    def u2(u, x):
        return np.einsum("ip,jq,pqrs,kr,ls->ijkl", u, u, x, u.conj(), u.conj())

    errs = []
    for h in (0.05, 0.025):
        stride = int(round(h / fine))
        grid = traj[::stride]
        us = [np.eye(nb, dtype=np.complex128)]          # u(t_m, T) by midpoint exponentials
        for m in range(len(grid) - 1):
            nm = 0.5 * (grid[m][0] + grid[m + 1][0])
            us.append(expm(-1j * h * O.hf_hamiltonian(prob.h, prob.w, nm)) @ us[-1])
        u_end = us[-1]
        hom = u2(u_end, grid[0][1])
        mem = np.zeros_like(hom)
        for m, (nm, _) in enumerate(grid):
            wgt = 0.5 if m in (0, len(grid) - 1) else 1.0
            # (iħ)^3 𝒰2 Ψ 𝒰2 with iħ𝒰 = u(T+Δ, t_m) = u_end u_m^†: -i (u⊗u) Ψ (u⊗u)^†
            mem = mem + wgt * h * (-1j) * u2(u_end @ us[m].conj().T, O.psi_source(prob.w_source, nm))
        errs.append(np.abs(hom + mem - g_end).max())
    print(f"interval recursion: |G(T+D)| {np.abs(g_end).max():.3e}, residual at h, h/2: {errs[0]:.3e} {errs[1]:.3e}")
    assert np.abs(g_end).max() > 1e-3
    assert errs[1] < 2e-4 and 3.0 < errs[0] / errs[1] < 5.0


def test_hubbard_gw_reduced_polarisation_with_site_dependent_u():
    """Sec. VIII.B: with G^> = G^< - i the Hubbard polarisation terms (Eqs. pihubbardtrans,
    pihubbardcis) reduce to Pi^{ud ud}_ijkl = -i G^<_jl (U_j G^{uuuu}_ijkj - U_l G^{uuuu}_ilkl)
    and the same with the spin blocks exchanged; U_p sits inside the site sum.  Checked
    against the general spin-orbital polarisation (Eq. gwpi) of a 3-site cluster with
    site-dependent U; the blocks mixing the spins crosswise vanish."""
    rng = np.random.default_rng(5)
    L = 3
    nb = 2 * L
    U = np.array([1.0, 0.7, 1.3])
    w = np.zeros((nb,) * 4)
    for i in range(L):
        for a in range(2):
            w[2 * i + a, 2 * i + 1 - a, 2 * i + a, 2 * i + 1 - a] = U[i]
    ns = inputs.random_hermitian(L, rng) * 0.2 + 0.4 * np.eye(L)
    n = np.kron(ns, np.eye(2)).astype(complex)
    _, g2 = inputs.random_state(nb, rng, soa=False)
    pi = O.gw_polarisation(O.gw_hcorr(w.astype(complex), n), g2)

    def blk(t, spins):
        return t[np.ix_(*[np.arange(L) * 2 + x for x in spins])]

    gl = 1j * ns
    reduced = lambda Go: (-1j * (np.einsum("jl,j,ijkj->ijkl", gl, U, Go) - np.einsum("jl,l,ilkl->ijkl", gl, U, Go)))
    assert np.abs(blk(pi, (0, 1, 0, 1)) - reduced(blk(g2, (0, 0, 0, 0)))).max() < 1e-14
    assert np.abs(blk(pi, (0, 0, 0, 0)) - reduced(blk(g2, (0, 1, 0, 1)))).max() < 1e-14
    assert np.abs(blk(pi, (0, 1, 1, 0))).max() == 0.0


def test_correlation_terms_are_exchange_symmetric():
    """The tensor-core assembly symmetrises every G2 term over the exchange (ij) <-> (ji),
    (kl) <-> (lk), which is exact because each correlation term keeps 𝒢_ijkl = 𝒢_jilk
    (Eq. Gsymm_a): Pi - conj(Pi_lkji) and both Lambda - conj(Lambda_klij).  And the
    ladder product the tensor cores compute is Lambda^dag = 𝒢 H^dag (𝒢 Hermitian as an
    nb^2 x nb^2 matrix, Eq. Gsymm_b)."""
    rng = np.random.default_rng(6)
    nb = 4
    w = sym_w(nb, rng)
    n, g2 = inputs.random_state(nb, rng, soa=False)
    ex = lambda t: np.abs(t - t.transpose(1, 0, 3, 2)).max() / np.abs(t).max()
    pi = O.gw_polarisation(O.gw_hcorr(w, n), g2)
    assert ex(pi - pi.transpose(3, 2, 1, 0).conj()) < 1e-13
    for hc, lad in ((O.tpp_hcorr, O.tpp_ladder), (O.tph_hcorr, O.tph_ladder)):
        lam = lad(hc(w, n), g2)
        assert ex(lam - lam.transpose(2, 3, 0, 1).conj()) < 1e-13
    H = O.tpp_hcorr(w, n).reshape(nb * nb, nb * nb)
    lam_dag = O.tpp_ladder(O.tpp_hcorr(w, n), g2).transpose(2, 3, 0, 1).conj().reshape(nb * nb, nb * nb)
    assert np.abs(lam_dag - g2.reshape(nb * nb, nb * nb) @ H.conj().T).max() < 1e-13


def test_torch_restatement_matches_oracle():
    """The autograd restatement (oracle/torch_oracle.py) reproduces the numpy oracle's RK4 run."""
    import torch
    from oracle import torch_oracle as T
    d = inputs.hubbard_2d_spin_orbital(Lx=2, Ly=1, n_controls=5, ta=0.0, tb=0.4)
    prob = O.Problem(d["h"], d["w"], "SOA", False, d["D"], d["drive"].f)
    n_ref, g_ref, _, _ = O.propagate(prob, d["n0"], np.zeros((4,) * 4), 0.02, 20)
    model = T.TorchSOA(d["h"], d["w"], d["D"])
    n, g = T.propagate(model, torch.as_tensor(d["n0"]), torch.zeros((4,) * 4, dtype=torch.complex128), 0.02, 20,
                       torch.as_tensor(d["drive"].values), 0.0, 0.4, 1.0, torch.zeros((4, 4), dtype=torch.complex128))
    assert np.abs(n.numpy() - n_ref).max() < 1e-13
    assert np.abs(g.numpy() - g_ref).max() < 1e-13
