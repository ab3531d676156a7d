"""Tiny Fock-space (exact diagonalisation) helpers for pinning the oracle.

Second quantisation by Jordan-Wigner matrices for nb <= 6 spin-orbitals.
Conventions of Eq. (h): H = Σ h_ij c_i^† c_j + ½ Σ w_ijkl c_i^† c_j^† c_l c_k;
n_ij = <c_j^† c_i>; two-particle density matrix n_ijkl = <c_k^† c_l^† c_j c_i>
(the equal-time less component of G^(2), Sec. II.A) and the correlated part
𝒢 from Eq. (ini-g2): 𝒢_ijkl = (1/(iħ)^2)(n_ijkl - n_ik n_jl + n_il n_jk).
"""
import numpy as np


def annihilators(nb):
    dim = 1 << nb
    ops = []
    for i in range(nb):
        c = np.zeros((dim, dim))
        for b in range(dim):
            if b >> i & 1:
                sign = (-1) ** bin(b & ((1 << i) - 1)).count("1")
                c[b ^ (1 << i), b] = sign
        ops.append(c)
    return ops


def hamiltonian(h, w):
    nb = h.shape[0]
    c = annihilators(nb)
    cd = [x.T for x in c]
    H = np.zeros((1 << nb, 1 << nb), dtype=np.complex128)
    for i in range(nb):
        for j in range(nb):
            if h[i, j] != 0:
                H += h[i, j] * cd[i] @ c[j]
    for i in range(nb):
        for j in range(nb):
            for k in range(nb):
                for l in range(nb):
                    if w[i, j, k, l] != 0:
                        H += 0.5 * w[i, j, k, l] * cd[i] @ cd[j] @ c[l] @ c[k]
    return H


def rdms(psi, nb):
    """(n, n2) with n_ij = <c_j^† c_i>, n2_ijkl = <c_k^† c_l^† c_j c_i>."""
    c = annihilators(nb)
    cd = [x.T for x in c]
    n = np.zeros((nb, nb), dtype=np.complex128)
    for i in range(nb):
        for j in range(nb):
            n[i, j] = psi.conj() @ (cd[j] @ c[i] @ psi)
    n2 = np.zeros((nb,) * 4, dtype=np.complex128)
    for i in range(nb):
        for j in range(nb):
            cji = c[j] @ c[i] @ psi
            for k in range(nb):
                for l in range(nb):
                    n2[i, j, k, l] = psi.conj() @ (cd[k] @ cd[l] @ cji)
    return n, n2


def correlated_g2(n, n2):
    """Eq. (ini-g2), fermions: 𝒢 = (1/(iħ)^2) (n_ijkl - n_ik n_jl + n_il n_jk)."""
    hart = np.einsum("ik,jl->ijkl", n, n)
    fock = np.einsum("il,jk->ijkl", n, n)
    return (n2 - hart + fock) / (1j ** 2)


def slater(orbitals, nb):
    """Fock vector of the Slater determinant Π_a (Σ_i φ_a(i) c_i^†)|0>."""
    c = annihilators(nb)
    v = np.zeros(1 << nb, dtype=np.complex128)
    v[0] = 1.0
    for a in range(orbitals.shape[1]):
        op = sum(orbitals[i, a] * c[i].T for i in range(nb))
        v = op @ v
    return v / np.linalg.norm(v)


def time_derivative(H, psi, op_expect):
    """d/dt f(psi(t)) at t = 0 for psi(t) = exp(-iHt) psi, by a 4th-order central difference."""
    from scipy.linalg import expm
    eps = 1e-3
    vals = []
    for s in (-2, -1, 1, 2):
        vals.append(op_expect(expm(-1j * H * s * eps) @ psi))
    return (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * eps)
