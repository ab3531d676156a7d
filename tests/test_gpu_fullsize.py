"""Parity at the full sizes of the bench workloads (SOA nb = 96, GW nb = 64) in the
form the bench times (BF16 slices): one right-hand side at a seeded correlated state
against the oracle's full right-hand side, element by element (the oracle takes
seconds per right-hand side here), plus what holds at any size: the trace of dn
(particle number) and the symmetries of d𝒢 (Eqs. Gsymm_a/b)."""
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from paper_2002_12717_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def tol_bf16x4(se, nb):
    """The BF16-slice bar of one right-hand side (test_gpu_tc.py): 1e-6 for every
    selfenergy, the nb^2 x nb^2 x nb^2 products included."""
    return 1e-6


@pytest.mark.parametrize("name,se", [("general-soa-nb96", "SOA"), ("general-gw-nb64", "GW"),
                                     ("general-gw-nb64", "TPP"), ("general-gw-nb64", "TPH")])
def test_full_size_rhs_matches_oracle(name, se):
    """The two bench workloads, and the T matrices on the GW workload's basis (nb = 64)."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = dict(inputs.workload(name), selfenergy=se)
    nb = d["nb"]
    rng = np.random.default_rng(17)
    _, g2 = inputs.random_state(nb, rng, g2_scale=1e-3, soa=(se == "SOA"))
    g2 = np.ascontiguousarray(g2)
    n = np.ascontiguousarray(d["n0"], dtype=np.complex128)
    t = 0.3
    with from_workload(d, precision="bf16x4") as p:
        dn_d = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
        dg_d = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
        p.rhs(t, torch.from_numpy(n).cuda(), torch.from_numpy(g2).cuda(), dn_d, dg_d)
        torch.cuda.synchronize()
        dn, dg = dn_d.cpu().numpy(), dg_d.cpu().numpy()
    del dn_d, dg_d
    prob = O.Problem(d["h"], d["w"], se, False, d["D"], d["drive"].f)
    dn_ref, dg_ref = O.rhs(prob, t, n, g2)
    tol = tol_bf16x4(se, nb)
    e_dn = np.abs(dn - dn_ref).max() / np.abs(dn_ref).max()
    e_dg = np.abs(dg - dg_ref).max() / np.abs(dg_ref).max()
    print(f"{name} {se} bf16x4: dn {e_dn:.2e}  dG2 {e_dg:.2e} (bar {tol:.1e})")
    assert e_dn < tol and e_dg < tol
    # any size: Tr dn = dN/dt = 0 (a sum of nb elements), and d𝒢 keeps the symmetries
    assert abs(np.trace(dn)) < nb * tol * np.abs(dn).max()
    scale = np.abs(dg).max()
    assert np.abs(dg - dg.transpose(1, 0, 3, 2)).max() < tol * scale
    assert np.abs(dg - dg.transpose(2, 3, 0, 1).conj()).max() < tol * scale
