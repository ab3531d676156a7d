"""The memory-integral HF-GKBA on the GPU (g1g2_propagate_hfgkba) against the
oracle's restatement of Sec. III.B, and its second-order convergence to the
G1-G2 solution (Sec. III.C)."""
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from oracle.hfgkba import propagate_hfgkba
from paper_2002_12717_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _uncorrelated(nb, rng, n_occ):
    """Slater-determinant n0 (a projector) in a random orbital basis."""
    return inputs.lowest_projector(inputs.random_hermitian(nb, rng), n_occ)


def _dimer():
    hs = inputs.chain_hopping(2)
    hs[0, 0] += 1.0
    h, w = inputs.spin_orbital_h(hs), inputs.spin_orbital_hubbard_w(2, 1.0)
    n0 = np.kron(inputs.lowest_projector(inputs.chain_hopping(2), 1), np.eye(2)).astype(np.complex128)
    return h, w, n0, False


def _general(nb, seed):
    rng = np.random.default_rng(seed)
    h = inputs.random_hermitian(nb, rng)
    w = inputs.factor_w(nb, max(2, nb), rng, sigma=0.3)
    return h, w, _uncorrelated(nb, rng, max(1, nb // 2)), False


def _restricted_chain(L):
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 1.5
    n0 = inputs.lowest_projector(inputs.chain_hopping(L), L // 2).astype(np.complex128)
    return hs.astype(np.complex128), inputs.onsite_w_restricted(L, 1.0), n0, True


@pytest.mark.parametrize("case,dt,steps,scratch", [
    ("dimer", 0.1, 20, 0),
    ("general5", 0.05, 12, 3 * 2 * 5 ** 4 * 16),   # three history points per chunk
    ("general9", 0.05, 8, 0),                      # nb^3 = 729: ragged thread tiles
    ("general17", 0.05, 4, 2 * 17 ** 4 * 16),      # widest register tile, one point per chunk
    ("restricted3", 0.1, 15, 0),                   # spin-restricted Hubbard chain (on-site w)
])
def test_memory_integral_matches_oracle(case, dt, steps, scratch):
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n0, restricted = {"dimer": _dimer, "general5": lambda: _general(5, 1), "general9": lambda: _general(9, 2),
                            "general17": lambda: _general(17, 3), "restricted3": lambda: _restricted_chain(3)}[case]()
    ref = propagate_hfgkba(O.Problem(h, w, "SOA", restricted), n0, dt, steps)
    with Propagator(h, w, n0, None, "SOA", "fp64", restricted) as p:
        got = p.propagate_hfgkba(dt, steps, scratch_bytes=scratch)
        t, n_end, _ = p.get_state()
    scale = max(1.0, np.abs(n0).max())
    assert np.abs(got - np.array(ref)).max() < 1e-12 * scale
    assert np.array_equal(n_end, got[-1]) and abs(t - steps * dt) < 1e-12
    assert np.abs(got[-1] - n0).max() > 1e-3   # the state moved


def test_memory_integral_converges_to_g1g2_at_second_order():
    """8-site spin-restricted Hubbard chain after a quench: n(T) and G2(T) of the
    memory-integral HF-GKBA approach the G1-G2 RK4 solution as dt^2."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n0, _ = _restricted_chain(8)
    T = 2.0
    with Propagator(h, w, n0, None, "SOA", "fp64", True) as p:
        p.propagate(0.005, int(round(T / 0.005)))
        _, n_ref, g_ref = p.get_state()
    errs = []
    for dt in (0.04, 0.02):
        with Propagator(h, w, n0, None, "SOA", "fp64", True) as p:
            p.propagate_hfgkba(dt, int(round(T / dt)))
            _, n, g = p.get_state()
        errs.append((np.abs(n - n_ref).max(), np.abs(g - g_ref).max()))
    assert np.abs(g_ref).max() > 1e-3
    for a, b in zip(errs[0], errs[1]):
        assert b < 5e-3 and 3.0 < a / b < 5.0


def test_memory_integral_rejections():
    from paper_2002_12717_gb300.g1g2 import G1G2Error, Propagator
    h, w, n0, _ = _general(4, 5)
    with Propagator(h, w, n0, None, "GW") as p, pytest.raises(G1G2Error):
        p.propagate_hfgkba(0.1, 2)
    g2 = np.zeros((4,) * 4, dtype=np.complex128)
    g2[0, 1, 0, 1] = g2[1, 0, 1, 0] = 1e-3
    g2[0, 1, 1, 0] = g2[1, 0, 0, 1] = -1e-3
    with Propagator(h, w, n0, g2, "SOA") as p, pytest.raises(G1G2Error):
        p.propagate_hfgkba(0.1, 2)                 # the integral starts from G2 = 0
    with Propagator(h, w, n0, None, "SOA") as p:
        p.set_drive(np.diag([1.0, -1.0, 0.5, 0.0]).astype(np.complex128), inputs.GaussSine(0.1, 1.0, 0.5, 0.3))
        with pytest.raises(G1G2Error):
            p.propagate_hfgkba(0.1, 2)
    with Propagator(h, w, n0, None, "SOA", "bf16x4") as p, pytest.raises(G1G2Error):
        p.propagate_hfgkba(0.1, 2)
