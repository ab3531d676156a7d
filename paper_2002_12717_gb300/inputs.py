"""Seeded synthetic inputs for the G1-G2 propagation (h, w, G1_0, 𝒢_0, drive).

This module builds problem data only; it holds none of the method's
arithmetic (no Hartree-Fock build, no contraction, no time stepping), so both
the CUDA path and the CPU oracle may be fed from it.

Workloads (the paper measures on synthetic Hubbard clusters, Sec. VII.C, and
has no dataset):
  * ``hubbard_chain_restricted`` -- 1D Hubbard chain, open boundaries,
    nearest-neighbour hopping J, on-site U stored as a dense w_ijkl =
    U δ_ij δ_ik δ_il in the spin-restricted basis, half filling, Hartree-Fock
    ground state, sudden quench of the on-site energy (Sec. III.D).
  * ``general_basis`` -- seeded general basis: h random Hermitian with
    entries N(0,1)/sqrt(nb) (complex), w_ijkl = Σ_P L^P_ik L^P_jl with L^P real
    symmetric, entries N(0, 0.1^2) before symmetrisation (so w carries the
    exchange and Hermitian symmetries of Sec. II.B), G1_0 the projector onto
    the n_occ lowest eigenvectors of h, 𝒢_0 = 0.
  * ``hubbard_2d_spin_orbital`` -- 2D Hubbard cluster in the spin-orbital
    basis (index = 2*site + spin), w from Eq. (wmatrix-hubbard).
  * gauss-sine and piecewise-linear drives h(t) = h + f(t) D.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Hubbard lattices
# ---------------------------------------------------------------------------

def chain_hopping(L, J=1.0, periodic=False):
    """h_ij = -J for nearest neighbours of an L-site chain (Eq. h-hubbard)."""
    h = np.zeros((L, L), dtype=np.complex128)
    for i in range(L - 1):
        h[i, i + 1] = h[i + 1, i] = -J
    if periodic and L > 2:
        h[0, L - 1] = h[L - 1, 0] = -J
    return h


def grid_hopping(Lx, Ly, J=1.0):
    """Open Lx x Ly grid, site index = x + Lx*y, nearest-neighbour hopping -J."""
    n = Lx * Ly
    h = np.zeros((n, n), dtype=np.complex128)
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            if x + 1 < Lx:
                h[s, s + 1] = h[s + 1, s] = -J
            if y + 1 < Ly:
                h[s, s + Lx] = h[s + Lx, s] = -J
    return h


def onsite_w_restricted(L, U):
    """Dense opposite-spin interaction w_ijkl = U δ_ij δ_ik δ_il (L^4, real)."""
    w = np.zeros((L, L, L, L))
    for i in range(L):
        w[i, i, i, i] = U
    return w


def spin_orbital_h(h_site):
    """h ⊗ 1_spin with spin-orbital index 2*site + spin."""
    return np.kron(h_site, np.eye(2))


def spin_orbital_hubbard_w(L, U):
    """Eq. (wmatrix-hubbard): w^{αβγδ}_ijkl = U δ_ij δ_ik δ_il δ_αγ δ_βδ (1-δ_αβ)."""
    nb = 2 * L
    w = np.zeros((nb, nb, nb, nb))
    for i in range(L):
        for a in range(2):
            b = 1 - a
            w[2 * i + a, 2 * i + b, 2 * i + a, 2 * i + b] = U
    return w


def lowest_projector(h, n_occ):
    """Projector onto the n_occ lowest eigenvectors of a Hermitian h."""
    e, v = np.linalg.eigh(h)
    vo = v[:, :n_occ]
    return vo @ vo.conj().T


def shell_projector(h, n_occ, tol=1e-9):
    """Paramagnetic ensemble for a degenerate Fermi shell.

    Levels strictly below the shell are filled, the shell (all levels within
    `tol` of the n_occ-th level) is filled uniformly with the remaining
    particles.  Equals `lowest_projector` when the shell is not degenerate.
    """
    e, v = np.linalg.eigh(h)
    ef = e[n_occ - 1]
    below = e < ef - tol
    shell = np.abs(e - ef) <= tol
    occ = np.zeros(len(e))
    occ[below] = 1.0
    occ[shell] = (n_occ - below.sum()) / shell.sum()
    return (v * occ) @ v.conj().T


# ---------------------------------------------------------------------------
# Seeded general basis
# ---------------------------------------------------------------------------

def random_hermitian(nb, rng):
    """(A + A^†)/2 with A = (X + iY)/sqrt(nb), X, Y ~ N(0,1)."""
    a = (rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))) / math.sqrt(nb)
    return (a + a.conj().T) / 2


def factors(nb, rank, rng, sigma=0.1):
    """The factors L^P = (B + B^T)/2, B ~ N(0, sigma^2), P < rank: real, shape (rank, nb, nb)."""
    b = rng.standard_normal((rank, nb, nb)) * sigma
    return (b + b.transpose(0, 2, 1)) / 2


def factor_w(nb, rank, rng, sigma=0.1):
    """w_ijkl = Σ_P L^P_ik L^P_jl with the factors of `factors`. Real, nb^4."""
    return expand_factors(factors(nb, rank, rng, sigma))


def expand_factors(lp):
    """The nb^4 tensor Σ_P L^P_ik L^P_jl of factors lp[P] (the workloads' w)."""
    rank, nb = lp.shape[0], lp.shape[1]
    flat = lp.reshape(rank, nb * nb)                  # [P, (i,k)]
    wik_jl = flat.T @ flat                            # [(i,k), (j,l)]
    return np.ascontiguousarray(wik_jl.reshape(nb, nb, nb, nb).transpose(0, 2, 1, 3))


# ---------------------------------------------------------------------------
# Drives h(t) = h + f(t) D
# ---------------------------------------------------------------------------

class GaussSine:
    """f(t) = A sin(ω t) exp(-(t - t0)^2 / (2 σ^2))."""

    kind = 1

    def __init__(self, A=0.5, omega=1.5, t0=5.0, sigma=1.5):
        self.A, self.omega, self.t0, self.sigma = A, omega, t0, sigma

    @property
    def params(self):
        return np.array([self.A, self.omega, self.t0, self.sigma])

    def f(self, t):
        return self.A * math.sin(self.omega * t) * math.exp(-(t - self.t0) ** 2 / (2 * self.sigma ** 2))

    def dfdt(self, t):
        g = math.exp(-(t - self.t0) ** 2 / (2 * self.sigma ** 2))
        return self.A * g * (self.omega * math.cos(self.omega * t)
                             - math.sin(self.omega * t) * (t - self.t0) / self.sigma ** 2)


class PiecewiseLinear:
    """f(t) linear between M equidistant control values on [ta, tb], constant outside."""

    kind = 2

    def __init__(self, values, ta=0.0, tb=10.0):
        self.values = np.asarray(values, dtype=np.float64)
        self.ta, self.tb = ta, tb

    @property
    def params(self):
        return np.concatenate([[self.ta, self.tb], self.values])

    def _seg(self, t):
        m = len(self.values)
        h = (self.tb - self.ta) / (m - 1)
        x = (t - self.ta) / h
        if x <= 0:
            return 0, 0.0, h, True
        if x >= m - 1:
            return m - 2, 1.0, h, True
        s = min(int(math.floor(x)), m - 2)
        return s, x - s, h, False

    def f(self, t):
        s, u, _, _ = self._seg(t)
        return (1 - u) * self.values[s] + u * self.values[s + 1]

    def dfdt(self, t):
        s, u, h, outside = self._seg(t)
        return 0.0 if outside else (self.values[s + 1] - self.values[s]) / h


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def hubbard_chain_restricted(L=8, J=1.0, U=1.0, quench=2.0, quench_sites=4):
    """1D chain, open, spin-restricted, half filling, HF ground state, sudden quench.

    At half filling on the bipartite open chain the paramagnetic HF state has
    n_ii = 1/2, so h^HF = h + U/2 and the HF ground state is the projector
    onto the L/2 lowest tight-binding orbitals.  The quench adds `quench` to
    the on-site energy of sites 0..quench_sites-1 at t = 0+.
    """
    h0 = chain_hopping(L, J)
    n0 = lowest_projector(h0, L // 2)
    h = h0.copy()
    for i in range(quench_sites):
        h[i, i] += quench
    return dict(name=f"hubbard-chain-restricted-nb{L}", nb=L, h=h, w=onsite_w_restricted(L, U),
                n0=n0, G2_0=None, selfenergy="SOA", restricted=True, D=None, drive=None)


def general_basis(nb, rank, n_occ, seed, selfenergy="SOA", pulse=False):
    """Seeded general basis, optional gauss-sine pulse with a random real diagonal dipole."""
    rng = np.random.default_rng(seed)
    h = random_hermitian(nb, rng)
    lp = factors(nb, rank, rng)
    w = expand_factors(lp)
    n0 = lowest_projector(h, n_occ)
    D = drive = None
    if pulse:
        D = np.diag(rng.standard_normal(nb)).astype(np.complex128)
        drive = GaussSine()
    return dict(name=f"general-{selfenergy.lower()}-nb{nb}", nb=nb, h=h, w=w, factors=lp, n0=n0, G2_0=None,
                selfenergy=selfenergy, restricted=False, D=D, drive=drive)


def hubbard_2d_spin_orbital(Lx=4, Ly=4, J=1.0, U=2.0, n_controls=64, ta=0.0, tb=10.0, seed=3):
    """2D open Hubbard cluster in the spin-orbital basis with a site-energy pulse.

    D_i = x_i - (Lx-1)/2 on both spins; f(t) piecewise linear through
    `n_controls` seeded control values (N(0, 0.1^2)) on [ta, tb].
    """
    L = Lx * Ly
    hs = grid_hopping(Lx, Ly, J)
    n_site = shell_projector(hs, L // 2)
    h = spin_orbital_h(hs)
    n0 = np.kron(n_site, np.eye(2))
    xs = np.array([s % Lx for s in range(L)], dtype=np.float64) - (Lx - 1) / 2
    D = np.kron(np.diag(xs), np.eye(2)).astype(np.complex128)
    rng = np.random.default_rng(seed)
    drive = PiecewiseLinear(0.1 * rng.standard_normal(n_controls), ta, tb)
    return dict(name=f"hubbard-2d-{Lx}x{Ly}-so", nb=2 * L, h=h, w=spin_orbital_hubbard_w(L, U),
                n0=n0, G2_0=None, selfenergy="SOA", restricted=False, D=D, drive=drive)


def workload(name):
    """The named workloads with their step size and length."""
    if name == "hubbard-chain-nb8":
        d = hubbard_chain_restricted()
        d.update(dt=0.02, nsteps=500)
    elif name == "general-soa-nb32":
        d = general_basis(32, 64, 16, seed=1)
        d.update(dt=0.01, nsteps=2000)
    elif name == "general-gw-nb48":
        d = general_basis(48, 96, 24, seed=2, selfenergy="GW", pulse=True)
        d.update(dt=0.01, nsteps=3000)
    elif name == "hubbard-2d-4x4":
        d = hubbard_2d_spin_orbital()
        d.update(dt=0.01, nsteps=1000)
    elif name == "general-soa-nb96":
        d = general_basis(96, 192, 48, seed=4, pulse=True)
        d.update(dt=0.01, nsteps=1000)
    elif name == "general-soa-nb48":
        d = general_basis(48, 96, 24, seed=7, pulse=True)
        d.update(dt=0.01, nsteps=1000)
    elif name == "general-soa-nb80":
        d = general_basis(80, 160, 40, seed=8, pulse=True)
        d.update(dt=0.01, nsteps=500)
    elif name == "general-soa-nb64":
        d = general_basis(64, 128, 32, seed=6, pulse=True)
        d.update(dt=0.01, nsteps=500)
    elif name == "general-gw-nb64":
        d = general_basis(64, 128, 32, seed=5, selfenergy="GW", pulse=True)
        d.update(dt=0.01, nsteps=500)
    else:
        raise KeyError(name)
    return d


WORKLOADS = ("hubbard-chain-nb8", "general-soa-nb32", "general-gw-nb48", "hubbard-2d-4x4",
             "general-soa-nb96", "general-gw-nb64", "general-soa-nb64", "general-soa-nb80")


def random_state(nb, rng, g2_scale=1e-2, soa=True):
    """A random admissible state (n Hermitian, 𝒢 with the symmetries of Sec. II.A).

    𝒢_ijkl = 𝒢_jilk and 𝒢_ijkl = 𝒢*_klij; for SOA additionally 𝒢_ijkl = -𝒢_ijlk.
    Used for right-hand-side parity at states away from 𝒢 = 0.
    """
    n = random_hermitian(nb, rng) * 0.3 + 0.5 * np.eye(nb)
    x = (rng.standard_normal((nb,) * 4) + 1j * rng.standard_normal((nb,) * 4)) * g2_scale
    if soa:
        x = x - x.transpose(0, 1, 3, 2)
    x = x + x.transpose(1, 0, 3, 2)
    x = x + x.transpose(2, 3, 0, 1).conj()
    return n, x
