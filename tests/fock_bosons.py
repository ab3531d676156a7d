"""Exact bosonic many-body helpers for pinning the oracle's boson branch.

Fock space of M modes truncated by the total particle number N <= Nmax: every
operator built here conserves N or lowers it before raising it again, so it is
exact on the truncated space, and the space is invariant under mode rotations.
Conventions as in the fermion helper (fock.py): H = Σ h_ij a_i^† a_j +
½ Σ w_ijkl a_i^† a_j^† a_l a_k; n_ij = <a_j^† a_i>; n2_ijkl = <a_k^† a_l^† a_j a_i>;
𝒢 from Eq. (ini-g2), bosons: 𝒢_ijkl = (1/(iħ)^2)(n_ijkl - n_ik n_jl - n_il n_jk).
"""
import itertools

import numpy as np


class Space:
    def __init__(self, M, Nmax):
        self.M = M
        self.states = [s for N in range(Nmax + 1) for s in _compositions(N, M)]
        self.index = {s: k for k, s in enumerate(self.states)}
        self.dim = len(self.states)
        # a_i as a dense matrix: a_i |..n_i..> = sqrt(n_i) |..n_i - 1..>
        self.a = []
        for i in range(M):
            op = np.zeros((self.dim, self.dim))
            for k, s in enumerate(self.states):
                if s[i] > 0:
                    t = list(s)
                    t[i] -= 1
                    op[self.index[tuple(t)], k] = np.sqrt(s[i])
            self.a.append(op)
        self.ad = [x.T for x in self.a]

    def number(self):
        return np.diag([float(sum(s)) for s in self.states])

    def sector(self, N):
        return [k for k, s in enumerate(self.states) if sum(s) == N]

    def one_body(self, m):
        """Σ_ij m_ij a_i^† a_j."""
        op = np.zeros((self.dim, self.dim), dtype=np.complex128)
        for i in range(self.M):
            for j in range(self.M):
                if m[i, j] != 0:
                    op += m[i, j] * (self.ad[i] @ self.a[j])
        return op

    def hamiltonian(self, h, w):
        H = self.one_body(h)
        M = self.M
        for i, j, k, l in itertools.product(range(M), repeat=4):
            if w[i, j, k, l] != 0:
                H += 0.5 * w[i, j, k, l] * (self.ad[i] @ self.ad[j] @ self.a[l] @ self.a[k])
        return H

    def rdms(self, rho):
        """(n, n2) of the (not necessarily Hermitian) operator rho:
        n_ij = Tr(rho a_j^† a_i) = Σ conj(a_j) * (a_i rho) and, with P_ij = a_j a_i,
        n2_ijkl = Tr(rho a_k^† a_l^† a_j a_i) = Σ conj(P_kl) * (P_ij rho)."""
        M = self.M
        n = np.zeros((M, M), dtype=np.complex128)
        arho = [self.a[i] @ rho for i in range(M)]
        for i in range(M):
            for j in range(M):
                n[i, j] = np.sum(self.a[j] * arho[i])
        P = {(i, j): self.a[j] @ self.a[i] for i in range(M) for j in range(M)}
        Prho = {key: op @ rho for key, op in P.items()}
        n2 = np.zeros((M,) * 4, dtype=np.complex128)
        for i, j, k, l in itertools.product(range(M), repeat=4):
            n2[i, j, k, l] = np.sum(P[(k, l)] * Prho[(i, j)])
        return n, n2

    def rdm_rates(self, rho, H):
        """d/dt of (n, n2) under H at rho: d<O>/dt = i Tr(rho [H, O])."""
        drho = -1j * (H @ rho - rho @ H)
        return self.rdms(drho)


def _compositions(N, M):
    if M == 1:
        yield (N,)
        return
    for first in range(N, -1, -1):
        for rest in _compositions(N - first, M - 1):
            yield (first,) + rest


def correlated_g2(n, n2):
    """Eq. (ini-g2), bosons: 𝒢 = (1/(iħ)^2) (n_ijkl - n_ik n_jl - n_il n_jk)."""
    hart = np.einsum("ik,jl->ijkl", n, n)
    fock = np.einsum("il,jk->ijkl", n, n)
    return (n2 - hart - fock) / (1j ** 2)


def correlated_g2_rate(n, n2, dn, dn2):
    """Time derivative of correlated_g2 by the product rule."""
    d_hart = np.einsum("ik,jl->ijkl", dn, n) + np.einsum("ik,jl->ijkl", n, dn)
    d_fock = np.einsum("il,jk->ijkl", dn, n) + np.einsum("il,jk->ijkl", n, dn)
    return (dn2 - d_hart - d_fock) / (1j ** 2)


def gaussian_state(space, eps, U):
    """Thermal state exp(-Σ_k eps_k b_k^† b_k) / Z of the rotated modes b = U^† a
    (a quasi-free state: its 𝒢 vanishes), on the truncated space."""
    from scipy.linalg import expm
    K = space.one_body(U @ np.diag(eps) @ U.conj().T)
    rho = expm(-K)
    return rho / np.trace(rho)
