"""Reverse-mode-differentiable restatement of the CPU oracle (torch, CPU, complex128).

TEST INFRASTRUCTURE ONLY (see g1g2_oracle.py).  The same equations as
g1g2_oracle.py, written in torch so that autograd gives the gradient of a
final-time observable with respect to the drive controls, a global scale of w
and h: the independent reference for the discrete adjoint of the GPU library.
Tiny basis sizes only (the N^4 tensors of the whole trajectory are kept for
the backward pass).

Equations (fermions, hbar = 1, G^< = i n, G^> = i n - i):
  h^HF = h(t) - i sum w^-_ikjl G^<_lk                    Eq. (h_HF)
  I_ij = -i sum w_iklp G2_lpjk                            Eq. (eom_gone-I)
  dG^</dt = -i ([h^HF, G^<] + I + I^dag), dn = -i dG^<    Eq. (eom_gone-2)
  dG2/dt = -i ([h2, G2] + Psi)                            Eq. (result_eom_soa)
  Psi = (i)^2 [chain(G^>,G^>,G^<,G^<) - chain(G^<,G^<,G^>,G^>)]  Eq. (soa-skalierung)
"""
from __future__ import annotations

import torch


def _es(*a):
    return torch.einsum(*a)


class TorchSOA:
    """SOA G1-G2 right-hand side with h(t) = h + f(t) D and w -> s w."""

    def __init__(self, h, w, D, restricted=False):
        self.h = torch.as_tensor(h, dtype=torch.complex128)
        self.w = torch.as_tensor(w, dtype=torch.complex128)
        self.D = torch.as_tensor(D, dtype=torch.complex128)
        self.restricted = restricted

    def rhs(self, f, s, h_extra, n, G2):
        nb = n.shape[0]
        w = s * self.w
        wt = w if self.restricted else w - w.permute(0, 1, 3, 2)
        h = self.h + h_extra + f * self.D
        gl = 1j * n
        gg = gl - 1j * torch.eye(nb, dtype=torch.complex128)
        hhf = h - 1j * _es("ikjl,lk->ij", wt, gl)
        I = -1j * _es("iklp,lpjk->ij", w, G2)
        dgl = -1j * (hhf @ gl - gl @ hhf + I + I.conj().T)
        dn = -1j * dgl
        comm = (_es("ip,pjkl->ijkl", hhf, G2) + _es("jp,ipkl->ijkl", hhf, G2)
                - _es("ijpl,pk->ijkl", G2, hhf) - _es("ijkp,pl->ijkl", G2, hhf))

        def chain(a, b, c, d):
            x = _es("pqrs,sl->pqrl", wt, d)
            x = _es("rk,pqrl->pqkl", c, x)
            x = _es("jq,pqkl->pjkl", b, x)
            return _es("ip,pjkl->ijkl", a, x)

        psi = (1j ** 2) * (chain(gg, gg, gl, gl) - chain(gl, gl, gg, gg))
        return dn, -1j * (comm + psi)


def piecewise_linear(values, ta, tb, t):
    """Linear interpolation of control values on [ta, tb], constant outside (differentiable in values)."""
    m = values.shape[0]
    hstep = (tb - ta) / (m - 1)
    x = (t - ta) / hstep
    if x <= 0:
        return values[0]
    if x >= m - 1:
        return values[m - 1]
    sI = min(int(x), m - 2)
    u = x - sI
    return (1 - u) * values[sI] + u * values[sI + 1]


def propagate(model, n0, G2_0, dt, nsteps, controls, ta, tb, s, h_extra):
    n, G2 = n0, G2_0
    for m in range(nsteps):
        t = m * dt
        f = lambda tt: piecewise_linear(controls, ta, tb, tt)
        k1 = model.rhs(f(t), s, h_extra, n, G2)
        k2 = model.rhs(f(t + dt / 2), s, h_extra, n + dt / 2 * k1[0], G2 + dt / 2 * k1[1])
        k3 = model.rhs(f(t + dt / 2), s, h_extra, n + dt / 2 * k2[0], G2 + dt / 2 * k2[1])
        k4 = model.rhs(f(t + dt), s, h_extra, n + dt * k3[0], G2 + dt * k3[1])
        n = n + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        G2 = G2 + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return n, G2


def mean_double_occupancy(n, G2):
    """(1/L) sum_i [n_uu n_dd - n_ud n_du - G2_udud], spin-orbital index 2*site + spin (E10)."""
    L = n.shape[0] // 2
    tot = 0.0
    for s in range(L):
        u, d = 2 * s, 2 * s + 1
        tot = tot + (n[u, u] * n[d, d] - n[u, d] * n[d, u] - G2[u, d, u, d]).real
    return tot / L
