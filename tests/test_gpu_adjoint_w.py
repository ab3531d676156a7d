"""The gradient of the discrete adjoint with respect to the entries of the
interaction w (g1g2_adjoint's grad_w, FP64 form).

w enters the right-hand side through the Hartree-Fock build (Eq. h_HF), the
collision integral (Eq. eom_gone-I), the source term (Eq. psi-pm-def), the GW
quasi-Hamiltonian (Eq. gwhcorr) and the ladder quasi-Hamiltonians (Eqs.
HTPPcorr, HTPHcorr); the energy objective also holds w explicitly.  The
library returns the gradient on the interactions g1g2_init accepts
(w_ijkl = w_jilk = conj(w_klij)), so it is checked along perturbations with
those symmetries:
  * central differences (eps = 1e-5) of J along random symmetric directions and
    along the orbit of one entry, for every selfenergy, all three objectives,
    real and complex w and the spin-restricted basis;
  * the derivative along w itself is the w-scale gradient, which the library
    computes by a separate route (the right-hand side's linearity in w);
  * reverse-mode autograd of the oracle's torch restatement (SOA, 2-site
    cluster), projected onto the same symmetric subspace.
"""
import numpy as np
import pytest

from paper_2002_12717_gb300 import inputs

from .helpers import problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-6   # relative, against a required 1e-5


def rdot(x, y):
    return float((np.conj(x) * y).real.sum())


def sym_direction(nb, rng, complex_=False):
    """A random tensor with w's symmetries, built exactly (sums of its images)."""
    x = rng.standard_normal((nb,) * 4)
    if complex_:
        x = x + 1j * rng.standard_normal((nb,) * 4)
    x = x + x.transpose(1, 0, 3, 2)
    x = x + x.transpose(2, 3, 0, 1).conj()
    return x / 4


def orbit_direction(nb, idx):
    """The real perturbation of one entry of w together with its symmetry images."""
    e = np.zeros((nb,) * 4)
    i, j, k, l = idx
    for a in ((i, j, k, l), (j, i, l, k), (k, l, i, j), (l, k, j, i)):
        e[a] = 1.0
    return e


def symmetrize(x):
    return 0.25 * (x + x.transpose(1, 0, 3, 2) + x.transpose(2, 3, 0, 1).conj() + x.transpose(3, 2, 1, 0).conj())


def _hubbard_case(ncontrols=4, nsteps=30, dt=0.02):
    d = inputs.hubbard_2d_spin_orbital(Lx=2, Ly=2, U=2.0, n_controls=ncontrols, ta=0.0, tb=nsteps * dt)
    d["drive"] = inputs.PiecewiseLinear(0.3 * np.sin(np.arange(ncontrols) + 1.0), 0.0, nsteps * dt)
    return d


def _J(d, w, se, objective, nsteps, dt, restricted=False):
    from paper_2002_12717_gb300.g1g2 import Propagator
    with Propagator(d["h"], w, d["n0"], None, se, "fp64", restricted) as p:
        p.set_drive(d["D"], d["drive"])
        return p.adjoint(dt, nsteps, objective=objective, ckpt_every=nsteps)[0]


def _check(d, se, objective, nsteps, dt, dirs, restricted=False, ckpt=7):
    from paper_2002_12717_gb300.g1g2 import Propagator
    w = d["w"]
    with Propagator(d["h"], w, d["n0"], None, se, "fp64", restricted) as p:
        p.set_drive(d["D"], d["drive"])
        J, _, gws, _, gw = p.adjoint(dt, nsteps, objective=objective, ckpt_every=ckpt, grad_w=True)
    # the returned gradient has w's symmetries
    assert np.abs(gw - symmetrize(gw)).max() <= 1e-12 * np.abs(gw).max()
    # the derivative along w is the w-scale gradient (computed by a separate route)
    assert abs(rdot(gw, w) - gws) <= 1e-9 * max(abs(gws), 1e-6), (rdot(gw, w), gws)
    eps = 1e-5
    for E in dirs:
        fd = (_J(d, w + eps * E, se, objective, nsteps, dt, restricted)
              - _J(d, w - eps * E, se, objective, nsteps, dt, restricted)) / (2 * eps)
        want = rdot(gw, E)
        assert abs(fd - want) <= TOL_GRAD * max(abs(fd), 1e-3), (fd, want)
    return gw


@pytest.mark.parametrize("objective", [0, 1, 2])
def test_grad_w_soa_hubbard_cluster(objective):
    """2x2 Hubbard cluster (8 spin-orbitals, real on-site w): dense random symmetric
    directions and the orbit of an entry that is zero in w and of an on-site entry."""
    dt, nsteps = 0.02, 30
    d = _hubbard_case(4, nsteps, dt)
    nb = d["nb"]
    rng = np.random.default_rng(11 + objective)
    dirs = [0.1 * sym_direction(nb, rng), orbit_direction(nb, (0, 3, 2, 5)), orbit_direction(nb, (2, 3, 2, 3))]
    _check(d, "SOA", objective, nsteps, dt, dirs)


@pytest.mark.parametrize("se", ["GW", "GWX", "TPP", "TPH", "DSL"])
def test_grad_w_correlated_selfenergies(se):
    """GW (Eqs. gwpi, gwhcorr), GW with exchange, the T matrices and DSL: the extra places
    w enters (the quasi-Hamiltonians) against central differences."""
    dt, nsteps = 0.02, 24
    d = _hubbard_case(4, nsteps, dt)
    nb = d["nb"]
    rng = np.random.default_rng(23)
    dirs = [0.1 * sym_direction(nb, rng), orbit_direction(nb, (0, 3, 2, 5))]
    _check(d, se, 0, nsteps, dt, dirs, ckpt=5)


@pytest.mark.parametrize("se,objective", [("SOA", 1), ("SOA", 2), ("GW", 2), ("TPH", 1)])
def test_grad_w_complex_general_basis(se, objective):
    """A general basis with a complex w (nb = 6) and complex symmetric directions."""
    dt, nsteps, nb = 0.02, 20, 6
    h, w, n, _, D, drv = problem(nb, se, False, True, seed=41)
    d = dict(h=h, w=w, n0=n, D=D, drive=drv, nb=nb)
    rng = np.random.default_rng(43)
    dirs = [0.1 * sym_direction(nb, rng, complex_=True), 0.1 * sym_direction(nb, rng, complex_=False)]
    _check(d, se, objective, nsteps, dt, dirs, ckpt=6)


def test_grad_w_spin_restricted():
    """The spin-restricted basis (no exchange term in h^HF, plain w in the source term)."""
    dt, nsteps, nb = 0.02, 20, 5
    h, w, n, _, D, drv = problem(nb, "SOA", True, False, seed=47)
    d = dict(h=h, w=w, n0=n, D=D, drive=drv, nb=nb)
    rng = np.random.default_rng(53)
    _check(d, "SOA", 1, nsteps, dt, [0.1 * sym_direction(nb, rng)], restricted=True, ckpt=4)


def test_grad_w_matches_oracle_autograd():
    """Reverse-mode autograd of the oracle's torch restatement with w as the leaf, on the
    2-site cluster, projected onto w's symmetric subspace; and the same gradient through
    the torch.autograd.Function with w as an input."""
    from oracle import torch_oracle as T
    from paper_2002_12717_gb300.autograd import final_time_objective
    from paper_2002_12717_gb300.g1g2 import Propagator
    dt, nsteps, M = 0.02, 20, 5
    d = inputs.hubbard_2d_spin_orbital(Lx=2, Ly=1, U=2.0, n_controls=M, ta=0.0, tb=nsteps * dt)
    d["drive"] = inputs.PiecewiseLinear(0.3 * np.cos(np.arange(M)), 0.0, nsteps * dt)
    wl = torch.tensor(d["w"], dtype=torch.complex128, requires_grad=True)
    model = T.TorchSOA(d["h"], wl, d["D"])
    ctrl = torch.tensor(d["drive"].values, dtype=torch.float64)
    n, g = T.propagate(model, torch.as_tensor(d["n0"]), torch.zeros((4,) * 4, dtype=torch.complex128), dt, nsteps,
                       ctrl, 0.0, nsteps * dt, torch.tensor(1.0, dtype=torch.float64), torch.zeros((4, 4),
                                                                                             dtype=torch.complex128))
    J_ref = T.mean_double_occupancy(n, g)
    J_ref.backward()
    ref = symmetrize(wl.grad.numpy())
    with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        J, _, _, _, gw = p.adjoint(dt, nsteps, objective=0, ckpt_every=6, grad_w=True)
    assert abs(J - J_ref.item()) < 1e-12
    assert np.abs(gw - ref).max() <= TOL_GRAD * np.abs(ref).max()
    # through the torch.autograd.Function: a real w leaf receives Re of the gradient
    problem_ = dict(w=d["w"], n0=d["n0"], D=d["D"], drive_kind=2, ta=0.0, tb=nsteps * dt, selfenergy="SOA")
    wr = torch.tensor(d["w"].real, dtype=torch.float64, requires_grad=True)
    Jf = final_time_objective(ctrl, 1.0, torch.as_tensor(d["h"]), problem_, dt, nsteps, "double_occupancy",
                              ckpt_every=5, w=wr)
    Jf.backward()
    assert abs(Jf.item() - J_ref.item()) < 1e-12
    assert np.abs(wr.grad.numpy() - ref.real).max() <= TOL_GRAD * np.abs(ref).max()
