"""The factorised interaction w_ijkl = sum_P L^P_ik L^P_jl (g1g2_init_factorised): the w
expanded on the device and, in the FP64 form, the source term of Eq. (psi-pm-def) from
the per-factor products M^P = nbar L^P n.  Parity with the oracle's right-hand side on
w = w_from_factors(L), element by element: real symmetric factors and Hermitian /
i-Hermitian complex ones, every selfenergy with a source term, bosons, the spin-restricted
mode, sizes from one orbital to nb = 33 (ragged GEMM tiles, nfac up to 2 nb); a driven
propagation, the memory-integral HF-GKBA (whose history source runs through the same
factorised product) and the split-precision form on the expanded w."""
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from oracle.hfgkba import propagate_hfgkba
from paper_2002_12717_gb300 import inputs

from .helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def run_rhs(prop, t, n, g2):
    nb = n.shape[0]
    dn = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
    dg = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
    prop.rhs(t, gpu(n), gpu(g2), dn, dg)
    torch.cuda.synchronize()
    return dn.cpu().numpy(), dg.cpu().numpy()


def complex_factors(nb, nfac, rng, sigma=0.1):
    """Hermitian factors, every second one times i (w stays complex with Eqs. wsymm_a/b)."""
    a = (rng.standard_normal((nfac, nb, nb)) + 1j * rng.standard_normal((nfac, nb, nb))) * sigma
    f = (a + a.conj().transpose(0, 2, 1)) / 2
    f[1::2] *= 1j
    return f


def state(nb, nfac, se, seed, complex_l=False, restricted=False):
    rng = np.random.default_rng(seed)
    h = inputs.random_hermitian(nb, rng)
    L = complex_factors(nb, nfac, rng) if complex_l else inputs.factors(nb, nfac, rng)
    n, g2 = inputs.random_state(nb, rng, soa=(se == "SOA" and not restricted))
    return h, L, n, g2


# (selfenergy, nb, nfac, complex factors, bosons, spin-restricted)
CASES = [("SOA", 1, 1, False, False, False), ("SOA", 5, 3, False, False, False), ("SOA", 6, 4, True, False, False),
         ("SOA", 17, 34, False, False, False), ("SOA", 33, 66, False, False, False),
         ("SOA", 9, 81, False, False, False),                   # nfac = nb^2
         ("GW", 7, 4, True, False, False), ("GW", 17, 20, False, False, False),
         ("GWX", 9, 18, False, False, False), ("TPP", 6, 5, True, False, False), ("TPH", 8, 7, False, False, False),
         ("DSL", 8, 6, True, False, False), ("HF", 5, 3, False, False, False),
         ("SOA", 6, 5, True, True, False), ("GW", 7, 6, False, True, False), ("DSL", 6, 4, False, True, False),
         ("SOA", 8, 6, False, False, True), ("TPH", 7, 5, False, False, True)]


@pytest.mark.parametrize("se,nb,nfac,complex_l,bosons,restricted", CASES)
def test_factorised_rhs_matches_oracle(se, nb, nfac, complex_l, bosons, restricted):
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, L, n, g2 = state(nb, nfac, se, 100 + nb, complex_l, restricted)
    w = O.w_from_factors(L)
    prob = O.Problem(h, w, se, restricted, bosons=bosons)
    dn_ref, dg_ref = O.rhs(prob, 0.3, n, g2)
    with Propagator(h, None, n, None, se, "fp64", restricted, bosons=bosons, factors=L) as p:
        dn, dg = run_rhs(p, 0.3, n, g2)
    assert rel_err(dn, dn_ref) < TOL_FP64
    if se == "HF":
        assert np.abs(dg).max() == 0.0
    else:
        assert rel_err(dg, dg_ref) < TOL_FP64


def test_factorised_propagation_with_pulse_matches_oracle():
    """nb = 10, 20 real factors, the gauss-sine pulse, 40 RK4 steps: state and energies."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    nb, nfac, dt, steps = 10, 20, 0.01, 40
    h, L, _, _ = state(nb, nfac, "SOA", 7)
    n0 = inputs.lowest_projector(h, 5)
    rng = np.random.default_rng(8)
    D = np.diag(rng.standard_normal(nb)).astype(np.complex128)
    drv = inputs.GaussSine(A=0.5, omega=1.5, t0=0.2, sigma=0.15)
    prob = O.Problem(h, O.w_from_factors(L), "SOA", False, D, drv.f)
    n_ref, g_ref, _, obs_ref = O.propagate(prob, n0, np.zeros((nb,) * 4), dt, steps, obs_every=steps,
                                           dfdt=drv.dfdt)
    with Propagator(h, None, n0, None, "SOA", factors=L) as p:
        p.set_drive(D, drv)
        obs, _ = p.propagate(dt, steps, steps)
        _, n, g = p.get_state()
    assert rel_err(n, n_ref) < 1e-11
    assert rel_err(g, g_ref) < 1e-10
    for k in ("e_one", "e_hf", "e_corr", "e_total", "pulse_work"):
        assert abs(obs[-1][k] - obs_ref[-1][k]) < 1e-11, k
    assert np.abs(g_ref).max() > 1e-4


def test_factorised_memory_integral_hfgkba_matches_oracle():
    from paper_2002_12717_gb300.g1g2 import Propagator
    nb, nfac = 5, 4
    h, L, _, _ = state(nb, nfac, "SOA", 12)
    n0 = inputs.lowest_projector(h, 2)
    ref = propagate_hfgkba(O.Problem(h, O.w_from_factors(L)), n0, 0.05, 20)
    with Propagator(h, None, n0, None, "SOA", factors=L) as p:
        got = p.propagate_hfgkba(0.05, 20)
    assert np.abs(got - np.array(ref)).max() < 1e-12


@pytest.mark.parametrize("se,nb", [("SOA", 16), ("GW", 12)])
def test_factorised_split_precision_form(se, nb):
    """The BF16-slice form runs on the expanded w: the bar of its right-hand side (1e-6)."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, L, n, g2 = state(nb, 2 * nb, se, 30 + nb)
    dn_ref, dg_ref = O.rhs(O.Problem(h, O.w_from_factors(L), se), 0.0, n, g2)
    with Propagator(h, None, n, None, se, "bf16x4", factors=L) as p:
        dn, dg = run_rhs(p, 0.0, n, g2)
    assert rel_err(dn, dn_ref) < 1e-6
    assert rel_err(dg, dg_ref) < 1e-6
