"""Parity of the plain FP64 GPU form with the CPU oracle, element by element."""
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from paper_2002_12717_gb300 import inputs

from .helpers import problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12   # FP64 contractions of length <= nb^2 on O(1) data


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def run_rhs(prop, t, n, g2):
    nb = n.shape[0]
    dn = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
    dg = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
    prop.rhs(t, gpu(n), gpu(g2), dn, dg)
    torch.cuda.synchronize()
    return dn.cpu().numpy(), dg.cpu().numpy()


CASES = [
    ("HF", 5, False, False), ("SOA", 1, False, False), ("SOA", 2, False, False), ("SOA", 5, False, True),
    ("SOA", 17, False, False), ("SOA", 33, False, False), ("SOA", 8, True, False), ("SOA", 13, True, False),
    ("GW", 2, False, False), ("GW", 7, False, True), ("GW", 17, False, False), ("GW", 33, False, False),
    ("GWX", 7, False, True), ("GWX", 17, False, False),
    ("TPP", 6, False, True), ("TPP", 17, False, False), ("TPP", 9, True, False),
    ("TPH", 6, False, True), ("TPH", 17, False, False), ("TPH", 9, True, False),
    ("DSL", 1, False, False), ("DSL", 6, False, True), ("DSL", 17, False, False), ("DSL", 33, False, False),
]


@pytest.mark.parametrize("se,nb,restricted,complex_w", CASES)
def test_rhs_parity(se, nb, restricted, complex_w):
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, restricted, complex_w, seed=nb)
    prob = O.Problem(h, w, se, restricted, D, drv.f)
    t = 0.7
    dn_ref, dg_ref = O.rhs(prob, t, n, g2)
    with Propagator(h, w, n, None, se, "fp64", restricted) as p:
        p.set_drive(D, drv)
        dn, dg = run_rhs(p, t, n, g2)
    assert rel_err(dn, dn_ref) < TOL_FP64
    if se == "HF":
        assert np.abs(dg).max() == 0.0
    else:
        assert rel_err(dg, dg_ref) < TOL_FP64


def test_hubbard_chain_full_run_matches_oracle():
    """8-site restricted Hubbard chain, quench, 500 RK4 steps, observables every step."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.workload("hubbard-chain-nb8")
    prob = O.Problem(d["h"], d["w"], "SOA", True)
    _, _, _, obs_ref = O.propagate(prob, d["n0"], np.zeros((8,) * 4), d["dt"], d["nsteps"])
    with from_workload(d) as p:
        obs, dens = p.propagate(d["dt"], d["nsteps"], 1)
    e_ref = np.array([o["e_total"] for o in obs_ref])
    e = np.array([o["e_total"] for o in obs])
    d_ref = np.array([o["density"] for o in obs_ref])
    assert np.abs(dens - d_ref).max() < 1e-11
    assert np.abs(e - e_ref).max() < 1e-11
    assert abs(e[-1] - e[0]) < 1e-6                     # energy conserved after the quench
    assert np.abs(np.array([o["n_particles"] for o in obs]) - 8.0).max() < 1e-12


@pytest.mark.parametrize("se", ["SOA", "GW"])
def test_propagation_with_pulse_matches_oracle(se):
    """General basis nb=12 with the gauss-sine pulse: state, energies and drive work."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    nb = 12
    d = inputs.general_basis(nb, 24, 6, seed=9, selfenergy=se, pulse=True)
    d["drive"] = inputs.GaussSine(A=0.5, omega=1.5, t0=0.3, sigma=0.2)
    prob = O.Problem(d["h"], d["w"], se, False, d["D"], d["drive"].f)
    dt, steps = 0.01, 60
    n_ref, g_ref, _, obs_ref = O.propagate(prob, d["n0"], np.zeros((nb,) * 4), dt, steps, obs_every=20,
                                           dfdt=d["drive"].dfdt)
    with Propagator(d["h"], d["w"], d["n0"], None, se) as p:
        p.set_drive(d["D"], d["drive"])
        obs, dens = p.propagate(dt, steps, 20)
        _, n, g = p.get_state()
    assert rel_err(n, n_ref) < 1e-11
    assert rel_err(g, g_ref) < 1e-10
    for a, b in zip(obs, obs_ref):
        for k in ("e_one", "e_hf", "e_corr", "e_total", "n_particles", "pulse_work"):
            assert abs(a[k] - b[k]) < 1e-11, k
    assert abs(obs[-1]["pulse_work"]) > 1e-4


def test_double_occupancy_and_energies_spin_orbital():
    from paper_2002_12717_gb300.g1g2 import Propagator
    L = 3
    nb = 2 * L
    rng = np.random.default_rng(4)
    h = inputs.spin_orbital_h(inputs.chain_hopping(L))
    w = inputs.spin_orbital_hubbard_w(L, 2.0)
    n, g2 = inputs.random_state(nb, rng, soa=True)
    with Propagator(h, w, n, g2, "SOA") as p:
        o = p.observables(double_occ=True)
    ref = O.energies(O.Problem(h, w), 0.0, n, g2)
    for k in ("e_one", "e_hf", "e_corr", "e_total", "n_particles"):
        assert abs(o[k] - ref[k]) < 1e-12
    assert np.abs(o["double_occ"] - O.double_occupancy(n, g2, L)).max() < 1e-12


def test_state_roundtrip_and_launch_count():
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, _, _ = problem(6, "SOA", seed=3, drive=False)
    with Propagator(h, w, n, g2, "SOA") as p:
        t, n1, g1 = p.get_state()
        assert t == 0.0 and np.array_equal(n1, n) and np.array_equal(g1, g2)
        c0 = p.launch_count
        p.step(0.01)
        torch.cuda.synchronize()
        assert p.launch_count > c0
        p.set_state(2.5, n, None)
        t, n2, gz = p.get_state()
        assert t == 2.5 and np.abs(gz).max() == 0.0


@pytest.mark.parametrize("se", ["TPP", "TPH", "DSL"])
def test_t_matrix_propagation_matches_oracle(se):
    """T-matrix and screened-ladder selfenergies: 3-site Hubbard chain in the spin-orbital basis,
    100 RK4 steps on the GPU against the oracle (state and energy)."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    L = 3
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 2.0
    h, w = inputs.spin_orbital_h(hs), inputs.spin_orbital_hubbard_w(L, 1.0)
    n0 = np.kron(np.diag([0.8, 0.5, 0.2]), np.eye(2)).astype(np.complex128)
    prob = O.Problem(h, w, se)
    n_ref, g_ref, _, obs_ref = O.propagate(prob, n0, np.zeros((2 * L,) * 4), 0.02, 100, obs_every=100)
    with Propagator(h, w, n0, None, se, "fp64") as p:
        obs, _ = p.propagate(0.02, 100, 100)
        _, n, g = p.get_state()
    assert np.abs(n - n_ref).max() < 1e-12 and np.abs(g - g_ref).max() < 1e-12
    assert abs(obs[-1]["e_total"] - obs_ref[-1]["e_total"]) < 1e-12


def test_dsl_rejects_the_spin_restricted_basis_and_the_tf32_form():
    from paper_2002_12717_gb300.g1g2 import G1G2Error, Propagator
    h, w, n, g2, _, _ = problem(8, "DSL", seed=2, drive=False)
    for kw in (dict(restricted=True), dict(precision="tf32x3")):
        with pytest.raises(G1G2Error):
            Propagator(h, w, n, g2, "DSL", **kw)


BOSON_CASES = [("HF", 5, False), ("SOA", 1, False), ("SOA", 6, True), ("SOA", 17, False), ("GW", 6, True),
               ("GWX", 9, False), ("TPP", 6, True), ("TPH", 6, True), ("TPH", 17, False), ("DSL", 7, True)]


@pytest.mark.parametrize("se,nb,complex_w", BOSON_CASES)
def test_boson_rhs_parity(se, nb, complex_w):
    """Bosons (statistics G1G2_BOSONS): w^+ in h^HF and Psi^±, nbar = 1 + n, the ph sign."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, False, complex_w, seed=40 + nb)
    prob = O.Problem(h, w, se, False, D, drv.f, bosons=True)
    dn_ref, dg_ref = O.rhs(prob, 0.4, n, g2)
    with Propagator(h, w, n, None, se, "fp64", bosons=True) as p:
        p.set_drive(D, drv)
        dn, dg = run_rhs(p, 0.4, n, g2)
    assert rel_err(dn, dn_ref) < TOL_FP64
    if se != "HF":
        assert rel_err(dg, dg_ref) < TOL_FP64
        if nb > 1:   # one mode: A is a real number and Psi = A^dag - A vanishes for both
            _, dg_f = O.rhs(O.Problem(h, w, se, False, D, drv.f), 0.4, n, g2)
            assert rel_err(dg_f, dg_ref) > 1e-3        # the boson form differs from the fermion one


@pytest.mark.parametrize("se", ["SOA", "GW", "TPH"])
def test_boson_hubbard_propagation_matches_oracle(se):
    """Two-component Bose-Hubbard dimer with intra- and inter-component on-site
    interaction, 100 RK4 steps: state, energies and double occupancy."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    L = 2
    hs = inputs.chain_hopping(L)
    hs[0, 0] += 1.0
    h = inputs.spin_orbital_h(hs)
    w = inputs.spin_orbital_hubbard_w(L, 0.7).astype(np.complex128)
    for i in range(2 * L):
        w[i, i, i, i] += 0.5
    n0 = np.diag([0.8, 0.6, 0.3, 0.2]).astype(np.complex128)
    prob = O.Problem(h, w, se, bosons=True)
    n_ref, g_ref, _, obs_ref = O.propagate(prob, n0, np.zeros((4,) * 4), 0.02, 100, obs_every=100)
    with Propagator(h, w, n0, None, se, "fp64", bosons=True) as p:
        obs, _ = p.propagate(0.02, 100, 100)
        _, n, g = p.get_state()
        o = p.observables(double_occ=True)
    assert np.abs(n - n_ref).max() < 1e-12 and np.abs(g - g_ref).max() < 1e-12
    for k in ("e_one", "e_hf", "e_corr", "e_total", "n_particles"):
        assert abs(obs[-1][k] - obs_ref[-1][k]) < 1e-12, k
    assert np.abs(o["double_occ"] - O.double_occupancy(n_ref, g_ref, L, eta=1)).max() < 1e-12
    assert np.abs(g_ref).max() > 1e-3


def test_boson_memory_integral_hfgkba_matches_oracle():
    from oracle.hfgkba import propagate_hfgkba
    from paper_2002_12717_gb300.g1g2 import Propagator
    hs = inputs.chain_hopping(3)
    hs[0, 0] += 1.0
    w = np.zeros((3,) * 4, dtype=np.complex128)
    for i in range(3):
        w[i, i, i, i] = 1.0
    n0 = np.diag([0.7, 0.4, 0.2]).astype(np.complex128)
    ref = propagate_hfgkba(O.Problem(hs.astype(np.complex128), w, bosons=True), n0, 0.05, 20)
    with Propagator(hs.astype(np.complex128), w, n0, None, "SOA", "fp64", bosons=True) as p:
        got = p.propagate_hfgkba(0.05, 20)
    assert np.abs(got - np.array(ref)).max() < 1e-12


def test_boson_rejections():
    from paper_2002_12717_gb300.g1g2 import G1G2Error, Propagator
    h, w, n, g2, _, _ = problem(4, "SOA", seed=8, drive=False)
    with pytest.raises(G1G2Error):
        Propagator(h, w, n, g2, "SOA", bosons=True, restricted=True)
    with Propagator(h, w, n, None, "SOA", bosons=True) as p, pytest.raises(G1G2Error):
        p.adjoint(0.01, 2, objective=0, ckpt_every=1, n_drive_params=0)


def test_non_finite_state_and_drive_are_reported():
    """A NaN planted in the state through g1g2_set_state (which does not scan its input) is
    caught at the next observable record of g1g2_propagate (G1G2_ENONFINITE); a drive with an
    Inf is refused by g1g2_set_drive; the context stays usable afterwards."""
    from paper_2002_12717_gb300.g1g2 import ENONFINITE, G1G2Error, Propagator
    h, w, n, g2, D, drv = problem(6, "SOA", seed=21)
    with Propagator(h, w, n, None, "SOA") as p:
        bad = n.copy()
        bad[1, 2] = bad[2, 1] = np.nan
        p.set_state(0.0, bad)
        with pytest.raises(G1G2Error) as e:
            p.propagate(0.01, 3, 1)
        assert e.value.code == ENONFINITE
        Dbad = D.copy()
        Dbad[0, 0] = np.inf
        with pytest.raises(G1G2Error) as e:
            p.set_drive(Dbad, drv)
        assert e.value.code == ENONFINITE
        p.set_state(0.0, n)
        obs, _ = p.propagate(0.01, 3, 1)
        assert np.isfinite(obs[-1]["e_total"])
