"""The discrete adjoint of the FP64 form: vector-Jacobian products, gradients
against central finite differences of the GPU propagation and against
reverse-mode autograd of the oracle's torch restatement."""
import numpy as np
import pytest

from paper_2002_12717_gb300 import inputs

from .helpers import problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-6   # relative, against a required 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def rdot(x, y):
    return float((x.conj() * y).real.sum())


@pytest.mark.parametrize("nb,restricted,se", [(6, False, "SOA"), (8, False, "SOA"), (5, True, "SOA"),
                                              (6, False, "GW"), (7, False, "GWX"), (6, False, "TPP"),
                                              (6, False, "TPH"), (5, True, "TPP"), (5, False, "DSL")])
def test_vjp_dot_product(nb, restricted, se):
    """<J d, ybar> by central differences of g1g2_rhs equals <d, VJP(ybar)>."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    h, w, n, g2, D, drv = problem(nb, se, restricted, False, seed=70 + nb)
    rng = np.random.default_rng(5)
    cn = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    dn_dir, dg_dir = cn(nb, nb), 0.1 * cn(*(nb,) * 4)
    a, Y = cn(nb, nb), cn(*(nb,) * 4)
    t = 0.3
    with Propagator(h, w, n, None, se, "fp64", restricted) as p:
        p.set_drive(D, drv)
        eps = 1e-5

        def f(nn, gg):
            dn = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
            dg = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
            p.rhs(t, dev(nn), dev(gg), dn, dg)
            torch.cuda.synchronize()
            return dn.cpu().numpy(), dg.cpu().numpy()

        fp, fm = f(n + eps * dn_dir, g2 + eps * dg_dir), f(n - eps * dn_dir, g2 - eps * dg_dir)
        lhs = (rdot((fp[0] - fm[0]) / (2 * eps), a) + rdot((fp[1] - fm[1]) / (2 * eps), Y))
        nbar = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
        gbar = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
        hbar = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
        if restricted:
            p.adjoint(0.01, 1, objective=1)   # allocates the adjoint scratch
        p.rhs_vjp(t, dev(n), dev(g2), dev(a), dev(Y), nbar, gbar, hbar)
        torch.cuda.synchronize()
        rhs = rdot(dn_dir, nbar.cpu().numpy()) + rdot(dg_dir, gbar.cpu().numpy())
        assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1.0), (lhs, rhs)
        # the h^HF cotangent: direction D through the drive value f(t)
        fa = drv.f(t)
        ds = 1e-5
        drv_p = inputs.GaussSine(A=drv.A * (1 + ds / fa), omega=drv.omega, t0=drv.t0, sigma=drv.sigma)
        drv_m = inputs.GaussSine(A=drv.A * (1 - ds / fa), omega=drv.omega, t0=drv.t0, sigma=drv.sigma)
        p.set_drive(D, drv_p)
        fp = f(n, g2)
        p.set_drive(D, drv_m)
        fm = f(n, g2)
        lhs_h = rdot((fp[0] - fm[0]) / (2 * ds), a) + rdot((fp[1] - fm[1]) / (2 * ds), Y)
        assert abs(lhs_h - rdot(D, hbar.cpu().numpy())) <= 1e-7 * max(abs(lhs_h), 1.0)


def _hubbard_case(ncontrols=6, nsteps=50, dt=0.02):
    d = inputs.hubbard_2d_spin_orbital(Lx=2, Ly=2, U=2.0, n_controls=ncontrols, ta=0.0, tb=nsteps * dt)
    d["drive"] = inputs.PiecewiseLinear(0.3 * np.sin(np.arange(ncontrols) + 1.0), 0.0, nsteps * dt)
    return d


def _run_J(d, objective, nsteps, dt, h=None, wscale=1.0, controls=None, se="SOA"):
    from paper_2002_12717_gb300.g1g2 import Propagator
    drv = d["drive"] if controls is None else inputs.PiecewiseLinear(controls, d["drive"].ta, d["drive"].tb)
    with Propagator(d["h"] if h is None else h, d["w"] * wscale, d["n0"], None, se, "fp64") as p:
        p.set_drive(d["D"], drv)
        J, _, _, _ = p.adjoint(dt, nsteps, objective=objective, ckpt_every=nsteps)
    return J


@pytest.mark.parametrize("objective", [0, 1, 2])
def test_adjoint_matches_central_differences(objective):
    from paper_2002_12717_gb300.g1g2 import Propagator
    dt, nsteps, M = 0.02, 50, 6
    d = _hubbard_case(M, nsteps, dt)
    with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        J, gdrive, gws, gh = p.adjoint(dt, nsteps, objective=objective, ckpt_every=7, n_drive_params=M)
    eps = 1e-5
    vals = d["drive"].values
    for m in range(M):
        vp, vm = vals.copy(), vals.copy()
        vp[m] += eps
        vm[m] -= eps
        fd = (_run_J(d, objective, nsteps, dt, controls=vp) - _run_J(d, objective, nsteps, dt, controls=vm)) / (2 * eps)
        assert abs(fd - gdrive[m]) <= TOL_GRAD * max(abs(fd), 1e-3), (m, fd, gdrive[m])
    fd = (_run_J(d, objective, nsteps, dt, wscale=1 + eps) - _run_J(d, objective, nsteps, dt, wscale=1 - eps)) / (2 * eps)
    assert abs(fd - gws) <= TOL_GRAD * max(abs(fd), 1e-3), (fd, gws)
    # h entries through Hermitian perturbations (real and imaginary part of one hopping)
    i, j = 0, 2
    for kind in ("re", "im"):
        dh = np.zeros_like(d["h"])
        if kind == "re":
            dh[i, j] = dh[j, i] = 1.0
            want = gh[i, j].real + gh[j, i].real
        else:
            dh[i, j], dh[j, i] = 1j, -1j
            want = gh[i, j].imag - gh[j, i].imag
        fd = (_run_J(d, objective, nsteps, dt, h=d["h"] + eps * dh)
              - _run_J(d, objective, nsteps, dt, h=d["h"] - eps * dh)) / (2 * eps)
        assert abs(fd - want) <= TOL_GRAD * max(abs(fd), 1e-3), (kind, fd, want)


@pytest.mark.parametrize("se", ["GW", "TPP", "TPH", "DSL"])
def test_correlated_adjoint_matches_central_differences(se):
    """GW (Eqs. g2-eq-gw-pi, gwpi, gwhcorr), the T matrices (Eqs. g2-eq-tpp-lambda,
    g2-eq-tph-lambda) and DSL: the adjoint's gradients with respect to the drive
    controls, the scale of w and a hopping against central differences."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    dt, nsteps, M = 0.02, 40, 4
    d = _hubbard_case(M, nsteps, dt)
    with Propagator(d["h"], d["w"], d["n0"], None, se, "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        J, gdrive, gws, gh = p.adjoint(dt, nsteps, objective=0, ckpt_every=9, n_drive_params=M)
    eps = 1e-5
    vals = d["drive"].values
    run = lambda **kw: _run_J(d, 0, nsteps, dt, se=se, **kw)
    for m in range(M):
        vp, vm = vals.copy(), vals.copy()
        vp[m] += eps
        vm[m] -= eps
        fd = (run(controls=vp) - run(controls=vm)) / (2 * eps)
        assert abs(fd - gdrive[m]) <= TOL_GRAD * max(abs(fd), 1e-3), (m, fd, gdrive[m])
    fd = (run(wscale=1 + eps) - run(wscale=1 - eps)) / (2 * eps)
    assert abs(fd - gws) <= TOL_GRAD * max(abs(fd), 1e-3), (fd, gws)
    i, j = 0, 2
    dh = np.zeros_like(d["h"])
    dh[i, j] = dh[j, i] = 1.0
    fd = (run(h=d["h"] + eps * dh) - run(h=d["h"] - eps * dh)) / (2 * eps)
    assert abs(fd - (gh[i, j].real + gh[j, i].real)) <= TOL_GRAD * max(abs(fd), 1e-3)
    # the gradients differ from the SOA ones on this cluster
    with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        _, gdrive_soa, _, _ = p.adjoint(dt, nsteps, objective=0, ckpt_every=9, n_drive_params=M)
    assert np.abs(gdrive - gdrive_soa).max() > 1e-3 * np.abs(gdrive).max()


def test_adjoint_independent_of_checkpoint_interval():
    from paper_2002_12717_gb300.g1g2 import Propagator
    dt, nsteps, M = 0.02, 30, 4
    d = _hubbard_case(M, nsteps, dt)
    res = []
    for k in (1, 7, 30):
        with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
            p.set_drive(d["D"], d["drive"])
            res.append(p.adjoint(dt, nsteps, objective=0, ckpt_every=k, n_drive_params=M))
    for r in res[1:]:
        assert r[0] == res[0][0]
        assert np.array_equal(r[1], res[0][1]) and r[2] == res[0][2]


def test_adjoint_matches_oracle_autograd():
    """Reverse-mode autograd of the oracle's torch restatement on a 2-site cluster."""
    from oracle import torch_oracle as T
    from paper_2002_12717_gb300.g1g2 import Propagator
    dt, nsteps, M = 0.02, 20, 5
    d = inputs.hubbard_2d_spin_orbital(Lx=2, Ly=1, U=2.0, n_controls=M, ta=0.0, tb=nsteps * dt)
    d["drive"] = inputs.PiecewiseLinear(0.3 * np.cos(np.arange(M)), 0.0, nsteps * dt)
    model = T.TorchSOA(d["h"], d["w"], d["D"])
    ctrl = torch.tensor(d["drive"].values, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    hx = torch.zeros((4, 4), dtype=torch.complex128, requires_grad=True)
    n, g = T.propagate(model, torch.as_tensor(d["n0"]), torch.zeros((4,) * 4, dtype=torch.complex128), dt, nsteps,
                       ctrl, 0.0, nsteps * dt, s, hx)
    J_ref = T.mean_double_occupancy(n, g)
    J_ref.backward()
    with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        J, gdrive, gws, gh = p.adjoint(dt, nsteps, objective=0, ckpt_every=6, n_drive_params=M)
    assert abs(J - J_ref.item()) < 1e-12
    assert np.abs(gdrive - ctrl.grad.numpy()).max() <= TOL_GRAD * np.abs(ctrl.grad.numpy()).max()
    assert abs(gws - s.grad.item()) <= TOL_GRAD * abs(s.grad.item())
    # torch's gradient of a real loss w.r.t. a complex leaf is dJ/dRe + i dJ/dIm; on
    # Hermitian perturbations only its Hermitian part acts
    g = hx.grad.numpy()
    gherm = 0.5 * (g + g.conj().T)
    assert np.abs(gh - gherm).max() <= TOL_GRAD * np.abs(gherm).max()


def test_autograd_function_chain_rule():
    """The torch.autograd.Function composes with surrounding torch code: controls built
    from two amplitudes, U as a leaf, a hopping shift as a leaf; compared with the
    oracle's reverse-mode autograd through the same parameterisation."""
    from oracle import torch_oracle as T
    from paper_2002_12717_gb300.autograd import final_time_objective
    dt, nsteps, M = 0.02, 20, 5
    tb = nsteps * dt
    d = inputs.hubbard_2d_spin_orbital(Lx=2, Ly=1, U=1.0, n_controls=M, ta=0.0, tb=tb)
    basis = torch.tensor(np.stack([np.cos(np.arange(M)), np.sin(0.5 * np.arange(M))]), dtype=torch.float64)

    def leaves():
        a = torch.tensor([0.3, -0.2], dtype=torch.float64, requires_grad=True)
        U = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
        tau = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
        return a, U, tau

    hop = np.zeros((4, 4), dtype=np.complex128)
    hop[0, 2] = hop[2, 0] = hop[1, 3] = hop[3, 1] = -1.0
    hop_t = torch.as_tensor(hop)

    a, U, tau = leaves()
    ctrl = a @ basis
    h = torch.as_tensor(d["h"]) + tau * hop_t
    problem = dict(w=d["w"], n0=d["n0"], D=d["D"], drive_kind=2, ta=0.0, tb=tb, selfenergy="SOA")
    J = final_time_objective(ctrl, U, h, problem, dt, nsteps, "double_occupancy", ckpt_every=4)
    (J ** 2).backward()
    got = (J.item(), a.grad.numpy().copy(), U.grad.item(), tau.grad.item())

    a, U, tau = leaves()
    model = T.TorchSOA(d["h"], d["w"], d["D"])
    n, g = T.propagate(model, torch.as_tensor(d["n0"]), torch.zeros((4,) * 4, dtype=torch.complex128), dt, nsteps,
                       a @ basis, 0.0, tb, U, tau * hop_t)
    Jr = T.mean_double_occupancy(n, g)
    (Jr ** 2).backward()
    assert abs(got[0] - Jr.item()) < 1e-12
    assert np.abs(got[1] - a.grad.numpy()).max() <= TOL_GRAD * np.abs(a.grad.numpy()).max()
    assert abs(got[2] - U.grad.item()) <= TOL_GRAD * abs(U.grad.item())
    assert abs(got[3] - tau.grad.item()) <= TOL_GRAD * abs(tau.grad.item())


def test_host_checkpoints_give_identical_gradients():
    """Checkpoints in pinned host memory: the same reverse sweep, bit for bit."""
    from paper_2002_12717_gb300.g1g2 import Propagator
    dt, nsteps, M = 0.02, 24, 4
    d = _hubbard_case(M, nsteps, dt)
    res = {}
    for where in ("device", "host"):
        with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
            p.set_drive(d["D"], d["drive"])
            p.set_adjoint_checkpoints(where)
            res[where] = p.adjoint(dt, nsteps, objective=0, ckpt_every=5, n_drive_params=M)
            assert p.adjoint_plan() == (5, where)
    a, b = res["device"], res["host"]
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2] and np.array_equal(a[3], b[3])
    with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        p.adjoint(dt, nsteps, objective=0, n_drive_params=M)
        k, where = p.adjoint_plan()
        assert where == "device" and k == 1     # everything fits: no recomputation
