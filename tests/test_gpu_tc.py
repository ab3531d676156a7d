"""Parity of the split-precision tensor-core form with the CPU oracle.

TF32x3 operands with FP32 accumulation carry about 21 significant bits per
product; the chained source term goes through four FP32 intermediates.  The
longest FP32 accumulation in a right-hand side runs over K' real products
(K' = 2 nb for SOA, 2 nb^2 for the GW polarisation), i.e. 3 K'/8 tcgen05 MMA
steps, each rounding at 2^-24; its random-walk error is 2^-24 sqrt(3 K'/8).
The bar for one right-hand side (max |Δ| / max |ref|) is eight times that,
and never below 2e-6.

The BF16-slice form (bf16x4) accumulates its leading products exactly.  Its
nb^5 passes carry 27-32 bits of every operand relative to the tensor's largest
entry; its nb^2 x nb^2 x nb^2 products (polarisation, ladders) carry 25 bits
relative to the largest entry of each row of A and each column of B and drop
only the order-3 and order-4 slice products, which sit near the FP32 rounding
of the inputs.  What remains is the FP32 storage of the state and of the
intermediates (2^-24 each, round to nearest).  The bar is 1e-6 for every
selfenergy and size (measured: at most 2.4e-7, at the full nb = 64).
"""
import math
import numpy as np
import pytest

from oracle import g1g2_oracle as O
from paper_2002_12717_gb300 import inputs

from .helpers import problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



def tol_rhs(se, nb, prec="tf32x3"):
    if prec == "bf16x4":
        return 1e-6
    kp = 2 * nb * nb if se in ("GW", "GWX") else 2 * nb
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


CASES = [("SOA", 4, False), ("SOA", 8, False), ("SOA", 12, False), ("SOA", 20, False), ("SOA", 32, False),
         ("SOA", 36, False), ("SOA", 48, False), ("SOA", 8, True), ("SOA", 12, True), ("GW", 4, False),
         ("GW", 8, False), ("GW", 12, False), ("GW", 20, False), ("GW", 32, False), ("GW", 36, False),
         ("GWX", 12, False), ("GWX", 32, False),
         # output tiles wider than 128 columns (nb > 64): the tensor-memory A path
         ("SOA", 68, False), ("GW", 68, False), ("SOA", 80, True)]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x4"])
@pytest.mark.parametrize("se,nb,restricted", CASES)
def test_tc_rhs_parity(se, nb, restricted, prec):
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, restricted, False, seed=100 + nb)
    prob = O.Problem(h, w, se, restricted, D, drv.f)
    t = 0.4
    dn_ref, dg_ref = O.rhs(prob, t, n, g2)
    with Propagator(h, w, n, None, se, prec, restricted) as p:
        p.set_drive(D, drv)
        dn, dg = run_rhs(p, t, n, g2)
    e1, e2 = rel_err(dn, dn_ref), rel_err(dg, dg_ref)
    print(f"{prec} {se} nb={nb} restricted={restricted}: dn {e1:.2e} dG2 {e2:.2e}")
    assert e1 < tol_rhs(se, nb, prec) and e2 < tol_rhs(se, nb, prec)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x4"])
@pytest.mark.parametrize("se,nb,restricted", [("SOA", 16, False), ("GW", 20, False), ("GWX", 12, False),
                                              ("SOA", 12, True), ("SOA", 36, False)])
def test_tc_mean_field_is_double_single_accurate(se, nb, restricted, prec):
    """The tensor-core forms build h^HF (Eq. h_HF) in double-single arithmetic on the FP32
    pipe.  At G2 = 0 the collision integral vanishes exactly in every form, so dn/dt =
    -i[h^HF, n] isolates the mean field: it must match the oracle to about 2^-46, far
    below the FP32-level bar of the G2 terms (a plain FP32 build would miss by ~1e-7)."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, _, D, drv = problem(nb, se, restricted, False, seed=300 + nb)
    g0 = np.zeros((nb,) * 4, dtype=np.complex128)
    prob = O.Problem(h, w, se, restricted, D, drv.f)
    dn_ref, _ = O.rhs(prob, 0.9, n, g0)
    with Propagator(h, w, n, None, se, prec, restricted) as p:
        p.set_drive(D, drv)
        dn, _ = run_rhs(p, 0.9, n, g0)
    e = rel_err(dn, dn_ref)
    print(f"{prec} {se} nb={nb} restricted={restricted}: mean-field dn {e:.2e}")
    assert np.abs(dn_ref).max() > 0.1 and e < 1e-11


LADDER_CASES = [("TPP", 4, False), ("TPP", 8, False), ("TPP", 12, False), ("TPP", 20, False), ("TPP", 32, False),
                ("TPP", 36, False), ("TPP", 8, True), ("TPH", 4, False), ("TPH", 8, False), ("TPH", 12, False),
                ("TPH", 20, False), ("TPH", 36, False), ("TPH", 8, True), ("DSL", 4, False), ("DSL", 12, False),
                ("DSL", 32, False)]


@pytest.mark.parametrize("se,nb,restricted", LADDER_CASES)
def test_tc_ladder_rhs_parity(se, nb, restricted):
    """T matrices and DSL in the BF16-slice form: each ladder product sums K' = 2 nb^2
    products of two FP32-stored tensors, the bar of the polarisation."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, restricted, False, seed=300 + nb)
    prob = O.Problem(h, w, se, restricted, D, drv.f)
    dn_ref, dg_ref = O.rhs(prob, 0.4, n, g2)
    with Propagator(h, w, n, None, se, "bf16x4", restricted) as p:
        p.set_drive(D, drv)
        dn, dg = run_rhs(p, 0.4, n, g2)
    e1, e2 = rel_err(dn, dn_ref), rel_err(dg, dg_ref)
    print(f"bf16x4 {se} nb={nb} restricted={restricted}: dn {e1:.2e} dG2 {e2:.2e}")
    assert e1 < tol_rhs("GW", nb, "bf16x4") and e2 < tol_rhs("GW", nb, "bf16x4")


BOSON_TC_CASES = [("SOA", 8, "tf32x3"), ("SOA", 12, "bf16x4"), ("GW", 12, "tf32x3"), ("GW", 12, "bf16x4"),
                  ("GWX", 8, "bf16x4"), ("TPP", 12, "bf16x4"), ("TPH", 12, "bf16x4"), ("DSL", 8, "bf16x4")]


@pytest.mark.parametrize("se,nb,prec", BOSON_TC_CASES)
def test_tc_boson_rhs_parity(se, nb, prec):
    """Bosons in the tensor-core forms (nbar = 1 + n, w^+ source, the ph sign)."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, False, False, seed=500 + nb)
    prob = O.Problem(h, w, se, False, D, drv.f, bosons=True)
    dn_ref, dg_ref = O.rhs(prob, 0.4, n, g2)
    with Propagator(h, w, n, None, se, prec, bosons=True) as p:
        p.set_drive(D, drv)
        dn, dg = run_rhs(p, 0.4, n, g2)
    e1, e2 = rel_err(dn, dn_ref), rel_err(dg, dg_ref)
    print(f"{prec} {se} bosons nb={nb}: dn {e1:.2e} dG2 {e2:.2e}")
    tol = tol_rhs("GW" if se != "SOA" else "SOA", nb, prec)
    assert e1 < tol and e2 < tol


@pytest.mark.parametrize("se", ["TPP", "TPH", "DSL"])
def test_tc_ladder_propagation_tracks_fp64_form(se):
    """nb=16 seeded general basis, 100 RK4 steps of the T matrices and DSL."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.general_basis(16, 32, 8, seed=12, selfenergy=se, pulse=True)
    d["drive"] = inputs.GaussSine(A=0.5, omega=1.5, t0=0.5, sigma=0.3)
    res = {}
    for pr in ("fp64", "bf16x4"):
        with from_workload(d, precision=pr) as p:
            obs, _ = p.propagate(0.01, 100, 10)
            _, n, g = p.get_state()
        res[pr] = (obs, n, g)
    dn = np.abs(res["bf16x4"][1] - res["fp64"][1]).max()
    dg = np.abs(res["bf16x4"][2] - res["fp64"][2]).max()
    de = max(abs(a["e_total"] - b["e_total"]) for a, b in zip(res["bf16x4"][0], res["fp64"][0]))
    print(f"bf16x4 {se}: max|dG1| {dn:.2e}  max|dG2| {dg:.2e}  max|dE| {de:.2e}")
    assert np.abs(res["fp64"][2]).max() > 1e-3
    assert dn < 1e-6 and dg < 1e-6 and de < 1e-6


def test_tc_ladder_rejects_tf32():
    from paper_2002_12717_gb300.g1g2 import EUNSUPPORTED, G1G2Error, Propagator
    h, w, n, _, _, _ = problem(8, "TPP", seed=2, drive=False)
    for se, prec in (("TPP", "tf32x3"), ("TPH", "tf32x3"), ("DSL", "tf32x3")):
        with pytest.raises(G1G2Error) as e:
            Propagator(h, w, n, None, se, prec)
        assert e.value.code == EUNSUPPORTED


@pytest.mark.parametrize("prec,bound", [("tf32x3", 2e-6), ("bf16x4", 5e-8)])
def test_tc_accumulation_is_unbiased(prec, bound):
    """A coherent sum: with w = 0, dG2 = -i [h2, G2]; G2 = 1e-2 a(x)a(x)a(x)a with a > 0 and
    h >= 0 off the diagonal make every entry of Z = G2 x_4 h a sum of positive terms.  A
    rounding that shrinks partial sums shows up as a negative regression coefficient of
    the error on the exact result (about -9e-9 nb for TF32 products accumulated in
    TMEM); the exact leading product of the slice form leaves only unbiased rounding."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    nb = 64
    rng = np.random.default_rng(0)
    a = 0.5 + rng.random(nb)
    h = rng.random((nb, nb))
    h = 0.5 * (h + h.T)
    np.fill_diagonal(h, 0.0)
    h = h.astype(np.complex128)
    w = np.zeros((nb,) * 4)
    n0 = np.diag(rng.random(nb)).astype(np.complex128)
    g2 = 1e-2 * np.einsum("i,j,k,l->ijkl", a, a, a, a).astype(np.complex128)
    prob = O.Problem(h, w, "GW", False)
    _, ref = O.rhs(prob, 0.0, n0, g2)
    with Propagator(h, w, n0, g2, "GW", prec) as p:
        _, dg = run_rhs(p, 0.0, n0, g2)
    err = dg - ref
    c = (np.vdot(ref, err) / np.vdot(ref, ref)).real
    print(f"{prec}: regression coefficient {c:+.2e}, max rel err {np.abs(err).max() / np.abs(ref).max():.2e}")
    assert abs(c) < bound


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x4"])
@pytest.mark.parametrize("se", ["SOA", "GW"])
def test_tc_propagation_tracks_fp64_form(se, prec):
    """nb=16 seeded general basis, 100 RK4 steps: tensor-core vs FP64 GPU form."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.general_basis(16, 32, 8, seed=11, selfenergy=se, pulse=True)
    d["drive"] = inputs.GaussSine(A=0.5, omega=1.5, t0=0.5, sigma=0.3)
    res = {}
    for pr in ("fp64", prec):
        with from_workload(d, precision=pr) as p:
            obs, dens = p.propagate(0.01, 100, 10)
            _, n, g = p.get_state()
        res[pr] = (obs, n, g)
    dn = np.abs(res[prec][1] - res["fp64"][1]).max()
    dg = np.abs(res[prec][2] - res["fp64"][2]).max()
    de = max(abs(a["e_total"] - b["e_total"]) for a, b in zip(res[prec][0], res["fp64"][0]))
    print(f"{prec} {se}: max|dG1| {dn:.2e}  max|dG2| {dg:.2e}  max|dE| {de:.2e}")
    assert dn < 1e-6 and dg < 1e-6 and de < 1e-6


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x4"])
@pytest.mark.parametrize("se", ["SOA", "GW"])
def test_tc_fp32_state_copy_is_the_rounding_of_the_state(se, prec):
    """The last RK4 stage writes the FP32 copy of the new state (the operand of the next
    step's products, and at stages 0-2 the base of the stage input) with integer bit
    operations; g1g2_set_state writes it with CUDA's double-to-float conversion.  Steps
    taken from either copy agree bit for bit: the tensor-core form has no floating-point
    atomics, so any difference would be a conversion that is not round-to-nearest-even."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.general_basis(16, 32, 8, seed=11, selfenergy=se, pulse=True)
    d["drive"] = inputs.GaussSine(A=0.5, omega=1.5, t0=0.5, sigma=0.3)
    out = []
    for reload in (False, True):
        with from_workload(d, precision=prec) as p:
            p.propagate(0.01, 6)
            if reload:
                t, n, g = p.get_state()
                p.set_state(t, n, g)
            p.propagate(0.01, 3)
            out.append(p.get_state())
    assert np.abs(out[0][2]).max() > 1e-4   # a correlated state, not a trivial one
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x4"])
def test_tc_hubbard_chain_full_run(prec):
    """8-site restricted chain, 500 steps, tensor-core form against the oracle densities."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d = inputs.workload("hubbard-chain-nb8")
    prob = O.Problem(d["h"], d["w"], "SOA", True)
    _, _, _, obs_ref = O.propagate(prob, d["n0"], np.zeros((8,) * 4), d["dt"], d["nsteps"], obs_every=10)
    with from_workload(d, precision=prec) as p:
        obs, dens = p.propagate(d["dt"], d["nsteps"], 10)
    d_ref = np.array([o["density"] for o in obs_ref])
    e = np.array([o["e_total"] for o in obs])
    print(f"max|d density| {np.abs(dens - d_ref).max():.2e}  energy drift {abs(e[-1] - e[0]):.2e}")
    assert np.abs(dens - d_ref).max() < 1e-6
    assert abs(e[-1] - e[0]) < 1e-6


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x4"])
def test_tc_rejects_what_it_does_not_cover(prec):
    from paper_2002_12717_gb300.g1g2 import EUNSUPPORTED, G1G2Error, Propagator
    h, w, n, g2, _, _ = problem(6, "SOA", seed=1, drive=False)
    with pytest.raises(G1G2Error) as e:
        Propagator(h, w, n, None, "SOA", prec)
    assert e.value.code == EUNSUPPORTED
    h, w, n, g2, _, _ = problem(8, "SOA", complex_w=True, seed=1, drive=False)
    with pytest.raises(G1G2Error) as e:
        Propagator(h, w, n, None, "SOA", prec)
    assert e.value.code == EUNSUPPORTED


def test_contexts_of_different_forms_coexist():
    """Kernel launch limits are per process: a second context with other tile sizes
    must not break the first one."""
    from paper_2002_12717_gb300.g1g2 import from_workload
    d1 = inputs.general_basis(64, 128, 32, seed=6, pulse=True)
    d2 = inputs.general_basis(16, 32, 8, seed=11, pulse=True)
    with from_workload(d1, precision="tf32x3") as p1, from_workload(d2, precision="bf16x4") as p2, \
            from_workload(d1, precision="bf16x4") as p3:
        for p in (p1, p2, p3, p1):
            p.step(0.01)
        o1, o3 = p1.observables(), p3.observables()
    assert abs(o1["e_total"] - o3["e_total"]) < 1e-6 * abs(o1["e_total"])


def test_bounded_wait_reports_timeout_and_context_survives():
    """A barrier that nothing arrives on: the wait gives up after its limit, the
    kernel returns ETIMEOUT through its error word, and later work still runs."""
    import time
    from paper_2002_12717_gb300 import g1g2
    t0 = time.perf_counter()
    assert g1g2.wait_selftest(20000) == g1g2.ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    d = inputs.general_basis(16, 32, 8, seed=3, pulse=False)
    with g1g2.from_workload(d, precision="bf16x4") as p:
        p.step(0.01)
        assert np.isfinite(p.observables()["e_total"])
