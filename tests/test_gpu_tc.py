"""Parity of the split-precision tensor-core form with the CPU oracle.

TF32x3 operands with FP32 accumulation carry about 21 significant bits per
product; the chained source term goes through four FP32 intermediates.  The
longest FP32 accumulation in a right-hand side runs over K' real products
(K' = 2 nb for SOA, 2 nb^2 for the GW polarisation), i.e. 3 K'/8 tcgen05 MMA
steps, each rounding at 2^-24; its random-walk error is 2^-24 sqrt(3 K'/8).
The bar for one right-hand side (max |Δ| / max |ref|) is eight times that,
and never below 2e-6.
"""
import math
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from paper_2002_12717_gb300 import inputs

from .helpers import problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



def tol_rhs(se, nb):
    kp = 2 * nb * nb if se == "GW" else 2 * nb
    return max(2e-6, 8 * 2.0 ** -24 * math.sqrt(3 * kp / 8))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def run_rhs(prop, t, n, g2):
    nb = n.shape[0]
    dn = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
    dg = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
    prop.rhs(t, gpu(n), gpu(g2), dn, dg)
    torch.cuda.synchronize()
    return dn.cpu().numpy(), dg.cpu().numpy()


@pytest.mark.parametrize("se,nb,restricted", [("SOA", 4, False), ("SOA", 8, False), ("SOA", 12, False),
                                              ("SOA", 20, False), ("SOA", 32, False), ("SOA", 36, False),
                                              ("SOA", 48, False), ("SOA", 8, True), ("SOA", 12, True),
                                              ("GW", 4, False), ("GW", 8, False), ("GW", 12, False),
                                              ("GW", 20, False), ("GW", 32, False), ("GW", 36, False)])
def test_tc_rhs_parity(se, nb, restricted):
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, restricted, False, seed=100 + nb)
    prob = O.Problem(h, w, se, restricted, D, drv.f)
    t = 0.4
    dn_ref, dg_ref = O.rhs(prob, t, n, g2)
    with Propagator(h, w, n, None, se, "tf32x3", restricted) as p:
        p.set_drive(D, drv)
        dn, dg = run_rhs(p, t, n, g2)
    e1, e2 = rel_err(dn, dn_ref), rel_err(dg, dg_ref)
    print(f"{se} nb={nb} restricted={restricted}: dn {e1:.2e} dG2 {e2:.2e}")
    assert e1 < tol_rhs(se, nb) and e2 < tol_rhs(se, nb)


@pytest.mark.parametrize("se", ["SOA", "GW"])
def test_tc_propagation_tracks_fp64_form(se):
    """nb=16 seeded general basis, 100 RK4 steps: tensor-core vs FP64 GPU form."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.general_basis(16, 32, 8, seed=11, selfenergy=se, pulse=True)
    d["drive"] = inputs.GaussSine(A=0.5, omega=1.5, t0=0.5, sigma=0.3)
    res = {}
    for prec in ("fp64", "tf32x3"):
        with from_workload(d, precision=prec) as p:
            obs, dens = p.propagate(0.01, 100, 10)
            _, n, g = p.get_state()
        res[prec] = (obs, n, g)
    dn = np.abs(res["tf32x3"][1] - res["fp64"][1]).max()
    dg = np.abs(res["tf32x3"][2] - res["fp64"][2]).max()
    de = max(abs(a["e_total"] - b["e_total"]) for a, b in zip(res["tf32x3"][0], res["fp64"][0]))
    print(f"max|dG1| {dn:.2e}  max|dG2| {dg:.2e}  max|dE| {de:.2e}")
    assert dn < 1e-6 and dg < 1e-6 and de < 1e-6


def test_tc_hubbard_chain_full_run():
    """8-site restricted chain, 500 steps, tensor-core form against the oracle densities."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.workload("hubbard-chain-nb8")
    prob = O.Problem(d["h"], d["w"], "SOA", True)
    _, _, _, obs_ref = O.propagate(prob, d["n0"], np.zeros((8,) * 4), d["dt"], d["nsteps"], obs_every=10)
    with from_workload(d, precision="tf32x3") as p:
        obs, dens = p.propagate(d["dt"], d["nsteps"], 10)
    d_ref = np.array([o["density"] for o in obs_ref])
    e = np.array([o["e_total"] for o in obs])
    print(f"max|d density| {np.abs(dens - d_ref).max():.2e}  energy drift {abs(e[-1] - e[0]):.2e}")
    assert np.abs(dens - d_ref).max() < 1e-6
    assert abs(e[-1] - e[0]) < 1e-6


def test_tc_rejects_what_it_does_not_cover():
    from paper_2002_12717_gb300.g1g2 import EUNSUPPORTED, G1G2Error, Propagator
    h, w, n, g2, _, _ = problem(6, "SOA", seed=1, drive=False)
    with pytest.raises(G1G2Error) as e:
        Propagator(h, w, n, None, "SOA", "tf32x3")
    assert e.value.code == EUNSUPPORTED
    h, w, n, g2, _, _ = problem(8, "SOA", complex_w=True, seed=1, drive=False)
    with pytest.raises(G1G2Error) as e:
        Propagator(h, w, n, None, "SOA", "tf32x3")
    assert e.value.code == EUNSUPPORTED
