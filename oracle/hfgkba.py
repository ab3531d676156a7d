"""Original (non-Markovian) HF-GKBA propagation with the SOA selfenergy.

TEST INFRASTRUCTURE ONLY (see g1g2_oracle.py).  Used to check the G1-G2
equations against the memory-integral formulation they were derived from,
for tiny basis sizes.

The collision integral is evaluated from the two-time form of Sec. III.B:
    𝒢(t) = (iħ)^3 ∫_{t0}^t dt̄ 𝒰2(t,t̄) Ψ^±(t̄) 𝒰2(t̄,t)      Eq. (dtilde-solution-short)
with 𝒰2_ijkl(t,t') = 𝒰_ik 𝒰_jl (Eq. prop_two), 𝒰 = G^R - G^A (Eq. prop_b),
and the Hartree-Fock propagators of the GKBA (Eqs. GKBA_propa/b): iħ 𝒰(t,t')
is the unitary u(t,t') generated by h^HF, i du/dt = h^HF(t) u.  Every time
step recomputes the full memory integral over all earlier times (trapezoid
rule), which is the O(N_t^2) cost of the standard scheme (Table I);
u(t_m, t_k) = u_m u_k^† by the group property of the HF propagator.

Time stepping: Heun's method (second order) for n and u; the memory integral
at the predictor time includes the predicted end point.  The scheme is
second-order accurate in dt, so it agrees with the G1-G2 RK4 solution to
O(dt^2).
"""
from __future__ import annotations

import numpy as np

from .g1g2_oracle import Problem, collision_integral, g1_rhs, hf_hamiltonian, psi_source


def _u2_transform(u, psi):
    """(iħ)^3 𝒰2(t,t̄) Ψ 𝒰2(t̄,t) with iħ𝒰 = u(t,t̄): (iħ)^3 (iħ)^-4 (u⊗u) Ψ (u⊗u)^†."""
    x = np.einsum("ip,jq,pqrs->ijrs", u, u, psi)
    x = np.einsum("ijrs,kr,ls->ijkl", x, u.conj(), u.conj())
    return (1j ** 3) * (1j ** -4) * x


def _g2_memory(us, psis, u_now, dt):
    """Trapezoid rule over the stored history t_0..t_m (the last entries are 'now')."""
    m = len(psis) - 1
    g2 = np.zeros_like(psis[0])
    if m == 0:
        return g2
    for k in range(m + 1):
        wgt = 0.5 if k in (0, m) else 1.0
        u_mk = u_now @ us[k].conj().T          # u(t_m, t_k) = u_m u_k^†
        g2 = g2 + wgt * dt * _u2_transform(u_mk, psis[k])
    return g2


def propagate_hfgkba(prob: Problem, n0, dt, nsteps):
    """Return the list of n(t_m), m = 0..nsteps, for an initially uncorrelated state."""
    assert prob.selfenergy == "SOA" and prob.D is None
    nb = n0.shape[0]
    n = n0.astype(np.complex128)
    u = np.eye(nb, dtype=np.complex128)
    eta = prob.eta
    us, psis = [u], [psi_source(prob.w_source, n, eta)]
    out = [n.copy()]

    def derivs(n_, u_, g2_):
        hhf = hf_hamiltonian(prob.h, prob.w, n_, prob.restricted, eta)
        dn = g1_rhs(hhf, n_, collision_integral(prob.w, g2_, eta), eta)
        du = -1j * hhf @ u_
        return dn, du

    g2 = _g2_memory(us, psis, u, dt)
    for _ in range(nsteps):
        dn1, du1 = derivs(n, u, g2)
        n_p, u_p = n + dt * dn1, u + dt * du1
        g2_p = _g2_memory(us + [u_p], psis + [psi_source(prob.w_source, n_p, eta)], u_p, dt)
        dn2, du2 = derivs(n_p, u_p, g2_p)
        n = n + dt / 2 * (dn1 + dn2)
        u = u + dt / 2 * (du1 + du2)
        us.append(u)
        psis.append(psi_source(prob.w_source, n, eta))
        g2 = _g2_memory(us, psis, u, dt)
        out.append(n.copy())
    return out
