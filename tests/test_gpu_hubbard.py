"""The O(nb^4) Hubbard-basis right-hand side (spin-restricted SOA, on-site w):
parity with the oracle's general O(nb^5) equations and with the library's own
general path, at random admissible states, with a drive."""
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from paper_2002_12717_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12   # FP64 throughout: relative to the largest entry


def _case(Lx, Ly, U=2.0, seed=0):
    rng = np.random.default_rng(seed)
    h = inputs.grid_hopping(Lx, Ly, 1.0)
    L = Lx * Ly
    h = h + np.diag(rng.uniform(-0.5, 0.5, L))           # site energies
    w = inputs.onsite_w_restricted(L, U)
    n, g2 = inputs.random_state(L, rng, soa=False)
    D = np.diag(np.arange(L, dtype=float) - (L - 1) / 2).astype(np.complex128)
    return h, w, n, g2, D


def _rhs(p, t, n, g2):
    nb = n.shape[0]
    dn = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
    dg = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
    p.rhs(t, torch.from_numpy(n).cuda(), torch.from_numpy(np.ascontiguousarray(g2)).cuda(), dn, dg)
    torch.cuda.synchronize()
    return dn.cpu().numpy(), dg.cpu().numpy()


@pytest.mark.parametrize("Lx,Ly", [(4, 1), (8, 1), (13, 1), (3, 3), (4, 4)])
def test_hubbard_path_matches_oracle_and_general_path(Lx, Ly):
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D = _case(Lx, Ly, seed=Lx * 10 + Ly)
    drv = inputs.GaussSine(A=0.4, omega=1.3, t0=0.2, sigma=0.5)
    prob = O.Problem(h, w, "SOA", True, D, drv.f)
    dn_ref, dg_ref = O.rhs(prob, 0.3, n, g2)
    with Propagator(h, w, n, None, "SOA", "fp64", restricted=True) as p:
        p.set_drive(D, drv)
        assert p.hubbard_path
        dn, dg = _rhs(p, 0.3, n, g2)
        p.hubbard_path = False
        dn_g, dg_g = _rhs(p, 0.3, n, g2)
        p.hubbard_path = True
        dn2, dg2 = _rhs(p, 0.3, n, g2)
    s = np.abs(dg_ref).max()
    assert np.abs(dg - dg_ref).max() <= TOL * s and np.abs(dn - dn_ref).max() <= TOL * np.abs(dn_ref).max()
    assert np.abs(dg - dg_g).max() <= TOL * s
    assert np.array_equal(dg, dg2) and np.array_equal(dn, dn2)   # switching back is exact


def test_hubbard_path_propagation_matches_general_path():
    """8-site chain workload, 200 RK4 steps on each path from the same state."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.workload("hubbard-chain-nb8")
    res = []
    for hub in (True, False):
        with from_workload(d, precision="fp64") as p:
            p.hubbard_path = hub
            obs, dens = p.propagate(d["dt"], 200, 50)
            _, n, g = p.get_state()
        res.append((n, g, obs[-1]["e_total"]))
    assert np.abs(res[0][0] - res[1][0]).max() < 1e-12
    assert np.abs(res[0][1] - res[1][1]).max() < 1e-12
    assert abs(res[0][2] - res[1][2]) < 1e-11


def test_hubbard_path_only_where_it_applies():
    from paper_2002_12717_gb300.g1g2 import EUNSUPPORTED, G1G2Error, Propagator
    h, w, n, g2, D = _case(4, 1)
    w2 = w.copy()
    w2[0, 1, 0, 1] = w2[1, 0, 1, 0] = 0.3                   # not on-site
    with Propagator(h, w2, n, None, "SOA", "fp64", restricted=True) as p:
        assert not p.hubbard_path
        with pytest.raises(G1G2Error) as e:
            p.hubbard_path = True
        assert e.value.code == EUNSUPPORTED
    with Propagator(h, w, n, None, "HF", "fp64", restricted=True) as p:
        assert not p.hubbard_path


def test_restricted_gw_hubbard_matches_spin_orbital_gw():
    """GW in the spin-restricted Hubbard basis (Eqs. g2-gw-hubbard1/2 with the reduced
    polarisation of Sec. VIII.B, U_i site-dependent) against the general spin-orbital GW
    oracle on the 2L-orbital problem: the density, the opposite-spin block of G2 and the
    energies over 100 RK4 steps after a quench; the same-spin block enters through the
    polarisation coupling, and the run differs from SOA."""
    from paper_2002_12717_gb300.g1g2 import G1G2Error, Propagator
    L = 4
    U = np.array([1.0, 0.6, 1.4, 0.9])
    hs = inputs.chain_hopping(L).astype(np.complex128)
    n0 = inputs.lowest_projector(hs, L // 2).astype(np.complex128)
    hs[0, 0] += 1.5
    wr = np.zeros((L,) * 4)
    wso = np.zeros((2 * L,) * 4)
    for i in range(L):
        wr[i, i, i, i] = U[i]
        for a in range(2):
            wso[2 * i + a, 2 * i + 1 - a, 2 * i + a, 2 * i + 1 - a] = U[i]
    dt, steps = 0.02, 100
    res = {}
    for se in ("GW", "SOA"):
        prob = O.Problem(inputs.spin_orbital_h(hs), wso, se)
        res[se] = O.propagate(prob, np.kron(n0, np.eye(2)).astype(np.complex128), np.zeros((2 * L,) * 4), dt, steps,
                              obs_every=steps)
    n_so, g_so, _, obs_so = res["GW"]
    with Propagator(hs, wr, n0, None, "GW", "fp64", restricted=True) as p:
        assert p.hubbard_path
        obs, _ = p.propagate(dt, steps, steps)
        _, n, g = p.get_state()
        with pytest.raises(G1G2Error):
            p.hubbard_path = False
    up, dn = slice(0, None, 2), slice(1, None, 2)
    assert np.abs(n - n_so[up, up]).max() < 1e-12
    assert np.abs(g - g_so[up, dn, up, dn]).max() < 1e-12
    assert abs(obs[-1]["e_total"] - obs_so[-1]["e_total"]) < 1e-12
    assert np.abs(g_so[up, up, up, up]).max() > 1e-4                 # the same-spin block is active
    assert np.abs(g_so - res["SOA"][1]).max() > 1e-4                 # GW differs from SOA here
    # what the mode refuses: a w that is not on-site, and the caller-buffer right-hand side
    with pytest.raises(G1G2Error):
        Propagator(hs, wr + 0.01 * np.ones((L,) * 4), n0, None, "GW", "fp64", restricted=True)
    with Propagator(hs, wr, n0, None, "GW", "fp64", restricted=True) as p:
        z = torch.zeros((L, L), dtype=torch.complex128, device="cuda")
        zg = torch.zeros((L,) * 4, dtype=torch.complex128, device="cuda")
        with pytest.raises(G1G2Error):
            p.rhs(0.0, torch.from_numpy(n0).cuda(), zg, z, zg.clone())
