"""Planted mistakes in the oracle: each one must make at least one of its pins fail.

Every mutant replaces one function of the oracle (or its Problem class) by a copy
with one plausible error — a flipped sign, a dropped term, a wrong index or a
transposed operand — and runs the pins of tests/test_oracle_pins.py, cheapest
first, until one of them fails.  A mutant that no pin catches is a gap in the
pins.  All on the CPU; the mistakes are planted in the oracle only.
"""
import inspect

import numpy as np
import pytest

from oracle import g1g2_oracle as O

from . import test_oracle_pins as P

ein = O.einsum
_orig = {name: getattr(O, name) for name in
         ("g_less", "g_greater", "w_pm", "hf_hamiltonian", "collision_integral", "g1_rhs",
          "two_particle_commutator", "psi_source", "gw_hcorr", "gw_polarisation", "tpp_hcorr", "tpp_ladder",
          "tph_hcorr", "tph_ladder", "energies", "double_occupancy", "w_from_factors", "rk4_step", "Problem")}


def _psi_wrong_index(wt, n, eta=-1):
    """psi_source with the last sum over the transposed d (d_ls instead of d_sl)."""
    gl, gg = O.g_less(n, eta), O.g_greater(n, eta)

    def chain(a, b, c, d):
        x = ein("pqrs,ls->pqrl", wt, d)
        x = ein("rk,pqrl->pqkl", c, x)
        x = ein("jq,pqkl->pjkl", b, x)
        return ein("ip,pjkl->ijkl", a, x)
    return -(chain(gg, gg, gl, gl) - chain(gl, gl, gg, gg))


def _g1_rhs_no_idag(hhf, n, I, eta=-1):
    gl = O.g_less(n, eta)
    return eta * 1j * (-1j * (hhf @ gl - gl @ hhf + I))


def _energies_factor(prob, t, n, G2):
    e = _orig["energies"](prob, t, n, G2)
    e["e_total"] += e["e_corr"]
    e["e_corr"] *= 2.0
    return e


def _energies_plain_w(prob, t, n, G2):
    e = _orig["energies"](prob, t, n, G2)
    if not prob.restricted:
        d = 0.5 * ein("ijkl,ki,lj->", prob.w - O.w_pm(prob.w, prob.eta), n, n).real
        e["e_hf"] += d
        e["e_total"] += d
    return e


def _rk4_weights(prob, t, n, G2, dt):
    k1 = O.rhs(prob, t, n, G2)
    k2 = O.rhs(prob, t + dt / 2, n + dt / 2 * k1[0], G2 + dt / 2 * k1[1])
    k3 = O.rhs(prob, t + dt / 2, n + dt / 2 * k2[0], G2 + dt / 2 * k2[1])
    k4 = O.rhs(prob, t + dt, n + dt * k3[0], G2 + dt * k3[1])
    n_new = n + dt / 6 * (k1[0] + 3 * k2[0] + 1 * k3[0] + k4[0])
    G2_new = G2 + dt / 6 * (k1[1] + 3 * k2[1] + 1 * k3[1] + k4[1])
    return n_new, G2_new, (k1[0], k2[0], k3[0], k4[0])


class _ProblemPlainSource(_orig["Problem"]):
    """Psi with the plain w everywhere (w^- dropped from the SOA source term)."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.w_source = self.w


MUTANTS = {
    "G^< sign": ("g_less", lambda n, eta=-1: -eta * n / 1j),
    "G^> without the delta": ("g_greater", lambda n, eta=-1: _orig["g_less"](n, eta)),
    "G^> delta sign": ("g_greater", lambda n, eta=-1: _orig["g_less"](n, eta) - np.eye(n.shape[0]) / 1j),
    "w^± sign": ("w_pm", lambda w, eta=-1: w - eta * w.transpose(0, 1, 3, 2)),
    "w^± partner index": ("w_pm", lambda w, eta=-1: w + eta * w.transpose(0, 2, 1, 3)),
    "h^HF exchange dropped": ("hf_hamiltonian", lambda h, w, n, restricted=False, eta=-1:
                              h + eta * 1j * ein("ikjl,lk->ij", w, O.g_less(n, eta))),
    "h^HF transposed density": ("hf_hamiltonian", lambda h, w, n, restricted=False, eta=-1:
                                h + eta * 1j * ein("ikjl,kl->ij", w if restricted else O.w_pm(w, eta),
                                                   O.g_less(n, eta))),
    "I: index order of G2": ("collision_integral", lambda w, G2, eta=-1: eta * 1j * ein("iklp,lpkj->ij", w, G2)),
    "I: sign": ("collision_integral", lambda w, G2, eta=-1: -eta * 1j * ein("iklp,lpjk->ij", w, G2)),
    "G1 equation: I^dagger dropped": ("g1_rhs", _g1_rhs_no_idag),
    "commutator: a term dropped": ("two_particle_commutator", lambda hhf, G2:
                                   _orig["two_particle_commutator"](hhf, G2) + ein("ijkp,pl->ijkl", G2, hhf)),
    "commutator: transposed h": ("two_particle_commutator", lambda hhf, G2:
                                 _orig["two_particle_commutator"](hhf.T, G2)),
    "source: chains swapped": ("psi_source", lambda wt, n, eta=-1: -_orig["psi_source"](wt, n, eta)),
    "source: transposed n": ("psi_source", _psi_wrong_index),
    "source: plain w in SOA": ("Problem", _ProblemPlainSource),
    "GW hcorr: sign": ("gw_hcorr", lambda w, n, eta=-1: -_orig["gw_hcorr"](w, n, eta)),
    "GW hcorr: index of the exchange product": (
        "gw_hcorr", lambda w, n, eta=-1: eta * (1j ** 2) * ein(
            "qipk,jpql->ijkl", w, O.g2_exchange(O.g_greater(n, eta), O.g_less(n, eta))
            - O.g2_exchange(O.g_less(n, eta), O.g_greater(n, eta)))),
    "Pi: transposed operand": ("gw_polarisation", lambda hc, G2: ein("qjpl,ipqk->ijkl", hc, G2)),
    "TPP hcorr: mixed components": ("tpp_hcorr", lambda w, n, eta=-1: (1j ** 2) * (
        ein("ip,jq,pqkl->ijkl", O.g_greater(n, eta), O.g_less(n, eta), w)
        - ein("ip,jq,pqkl->ijkl", O.g_less(n, eta), O.g_greater(n, eta), w))),
    "TPP ladder: transposed pair": ("tpp_ladder", lambda hc, G2: ein("ijpq,qpkl->ijkl", hc, G2)),
    "TPH hcorr: same components": ("tph_hcorr", lambda w, n, eta=-1: (1j ** 2) * (
        ein("ip,ql,pjkq->ijkl", O.g_greater(n, eta), O.g_greater(n, eta), w)
        - ein("ip,ql,pjkq->ijkl", O.g_less(n, eta), O.g_less(n, eta), w))),
    "TPH ladder: index": ("tph_ladder", lambda hc, G2: ein("ipql,qjpk->ijkl", hc, G2)),
    "E_corr factor": ("energies", _energies_factor),
    "E_HF with w instead of w^±": ("energies", _energies_plain_w),
    "double occupancy: exchange sign": ("double_occupancy", lambda n, G2, ns, eta=-1:
                                        _orig["double_occupancy"](n, G2, ns, -eta)),
    "factorised w: pairing": ("w_from_factors", lambda L: ein("pij,pkl->ijkl", L, L)),
    "RK4 weights": ("rk4_step", _rk4_weights),
}

# propagations (tenths of a second each) after the single-evaluation pins, the pins that
# take seconds last
_PROPAGATING = ("conservation", "hfgkba", "interval", "noninteracting", "energy_balance", "propagation")
_SLOW = ("test_boson_source_term_is_exact_initial_slope_from_gaussian_state", "test_torch_restatement_matches_oracle")


def _tier(name):
    if name in _SLOW:
        return 2
    return 1 if any(k in name for k in _PROPAGATING) else 0


def _pins():
    out = []
    for name, fn in inspect.getmembers(P, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != P.__name__:
            continue
        params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if params:
            argname, values = params[0].args
            out.extend((name, (lambda f=fn, a=argname, v=v: f(**{a: v}))) for v in values)
        else:
            out.append((name, fn))
    return sorted(out, key=lambda p: _tier(p[0]))


PINS = _pins()


@pytest.mark.parametrize("mutant", list(MUTANTS))
def test_planted_mistake_is_caught(mutant, monkeypatch):
    target, replacement = MUTANTS[mutant]
    monkeypatch.setattr(O, target, replacement)
    for name, pin in PINS:
        try:
            pin()
        except AssertionError:      # caught by a pin's assertion, not by a broken call
            return
    pytest.fail(f"no pin catches the planted mistake: {mutant}")


def test_unmutated_oracle_passes_every_pin():
    """The runner itself: with nothing planted every pin passes (so a caught mutant is the
    mutant's doing)."""
    assert len(PINS) >= 50
    for name, pin in PINS:
        pin()
