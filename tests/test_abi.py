"""The C-ABI library: it loads, exports every symbol include/g1g2.h declares, and
rejects bad arguments before touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2002_12717_gb300 import g1g2, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "g1g2.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(g1g2_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(g1g2.LIB_PATH):
        from paper_2002_12717_gb300 import build
        build.build()
    return g1g2.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_and_defaults(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.g1g2_strerror(code)
    assert b"unknown" in lib.g1g2_strerror(42)
    opt = g1g2.Options()
    lib.g1g2_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.basis == 0 and opt.sym_tol == pytest.approx(1e-10) and opt.statistics == 0


def _init(lib, nb, h, w, n0, se=1, opt=None, g2=None):
    ctx = ctypes.c_void_p()
    o = g1g2.Options()
    lib.g1g2_default_options(ctypes.byref(o))
    if opt:
        for k, v in opt.items():
            setattr(o, k, v)
    ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return lib.g1g2_init(ctypes.byref(ctx), nb, ptr(h), ptr(w), ptr(n0), ptr(g2), se, ctypes.byref(o))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _valid(nb):
    rng = np.random.default_rng(0)
    h = inputs.random_hermitian(nb, rng)
    w = inputs.factor_w(nb, 3, rng).astype(np.complex128)
    n0 = inputs.lowest_projector(h, 1)
    return h, w, n0


def test_invalid_arguments_rejected_on_host(lib):
    h, w, n0 = _valid(3)
    assert _init(lib, 0, h, w, n0) == g1g2.EINVAL
    assert _init(lib, 129, h, w, n0) == g1g2.EINVAL
    assert _init(lib, 3, None, w, n0) == g1g2.EINVAL
    assert _init(lib, 3, h, None, n0) == g1g2.EINVAL
    assert _init(lib, 3, h, w, None) == g1g2.EINVAL
    assert _init(lib, 3, h, w, n0, se=7) == g1g2.EINVAL
    assert _init(lib, 3, h, w, n0, opt={"precision": 9}) == g1g2.EINVAL
    assert _init(lib, 3, h, w, n0, opt={"basis": 5}) == g1g2.EINVAL
    assert _init(lib, 3, h, w, n0, se=2, opt={"basis": 1}) == g1g2.EINVAL   # GW has no restricted form
    assert b"restricted" in lib.g1g2_last_error_detail()
    assert _init(lib, 3, h, w, n0, se=3, opt={"basis": 1}) == g1g2.EINVAL   # nor GW with exchange
    assert b"restricted" in lib.g1g2_last_error_detail()
    assert _init(lib, 3, h, w, n0, se=6, opt={"basis": 1}) == g1g2.EINVAL   # nor the screened ladder
    assert b"restricted" in lib.g1g2_last_error_detail()
    assert _init(lib, 3, h, w, n0, se=7) == g1g2.EINVAL
    assert _init(lib, 4, *_valid(4), se=4, opt={"precision": 1}) == g1g2.EUNSUPPORTED   # T matrix: FP64 only
    assert _init(lib, 4, *_valid(4), se=5, opt={"precision": 1}) == g1g2.EUNSUPPORTED
    assert _init(lib, 4, *_valid(4), se=6, opt={"precision": 1}) == g1g2.EUNSUPPORTED
    assert _init(lib, 3, h, w, n0, opt={"statistics": 2}) == g1g2.EINVAL
    assert _init(lib, 3, h, w, n0, opt={"statistics": 1, "basis": 1}) == g1g2.EINVAL   # bosons: spin-orbital only


def test_factorised_arguments_rejected_on_host(lib):
    """g1g2_init_factorised checks its arguments before any device work."""
    h, _, n0 = _valid(3)
    L = np.zeros((2, 3, 3))
    ctx = ctypes.c_void_p()
    o = g1g2.Options()
    lib.g1g2_default_options(ctypes.byref(o))
    o.w_is_real = 1
    ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def init(nb, hh, LL, nfac, nn, se=1):
        return lib.g1g2_init_factorised(ctypes.byref(ctx), nb, ptr(hh), ptr(LL), nfac, ptr(nn), None, se,
                                        ctypes.byref(o))
    assert init(0, h, L, 2, n0) == g1g2.EINVAL
    assert init(129, h, L, 2, n0) == g1g2.EINVAL
    assert init(3, h, None, 2, n0) == g1g2.EINVAL
    assert init(3, None, L, 2, n0) == g1g2.EINVAL
    assert init(3, h, L, 2, None) == g1g2.EINVAL
    assert init(3, h, L, 0, n0) == g1g2.EINVAL
    assert init(3, h, L, 10, n0) == g1g2.EINVAL           # more than nb^2 factors
    assert b"nfac" in lib.g1g2_last_error_detail()
    assert init(3, h, L, 2, n0, se=9) == g1g2.EINVAL
    assert not ctx.value
    with pytest.raises(ValueError):
        g1g2.Propagator(h, None, n0)                        # neither w nor factors
    with pytest.raises(ValueError):
        g1g2.Propagator(h, None, n0, factors=np.zeros((2, 3, 4)))


def test_factor_symmetry_checked_on_host(lib):
    """g1g2_init_factorised accepts Hermitian and i-Hermitian factors (the ones whose w meets
    Eqs. wsymm_a/b) and refuses others with G1G2_ESYMM before any device work; the factors of
    the GPU parity tests pass the check."""
    from .test_gpu_factorised import CASES, complex_factors, state
    nb = 4
    h, _, n0 = _valid(nb)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((2, nb, nb)) + 1j * rng.standard_normal((2, nb, nb))
    herm = (a + a.conj().transpose(0, 2, 1)) / 2
    b = rng.standard_normal((2, nb, nb))
    ptr = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def init(L):
        o = g1g2.Options()
        lib.g1g2_default_options(ctypes.byref(o))
        real = np.isrealobj(L)
        o.w_is_real = int(real)
        buf = np.ascontiguousarray(L, dtype=np.float64 if real else np.complex128)
        ctx = ctypes.c_void_p()
        rc = lib.g1g2_init_factorised(ctypes.byref(ctx), nb, ptr(h), ptr(buf), L.shape[0], ptr(n0), None, 1,
                                      ctypes.byref(o))
        if ctx.value:
            lib.g1g2_destroy(ctx)
        return rc
    valid = [herm, 1j * herm, inputs.factors(nb, 3, rng), b - b.transpose(0, 2, 1), np.zeros((1, nb, nb)),
             np.concatenate([herm, 1j * herm]), complex_factors(nb, 5, rng)]
    for L in valid:
        assert init(L) in (g1g2.OK, g1g2.ENOMEM)
    for se, nb_, nfac, complex_l, _, restricted in CASES:   # the inputs of the GPU parity tests
        hh, L, nn, _ = state(nb_, nfac, se, 100 + nb_, complex_l, restricted)
        o = g1g2.Options()
        lib.g1g2_default_options(ctypes.byref(o))
        o.w_is_real = int(np.isrealobj(L))
        buf = np.ascontiguousarray(L, dtype=np.float64 if np.isrealobj(L) else np.complex128)
        ctx = ctypes.c_void_p()
        rc = lib.g1g2_init_factorised(ctypes.byref(ctx), nb_, ptr(_c(hh)), ptr(buf), nfac, ptr(_c(nn)), None, 1,
                                      ctypes.byref(o))
        if ctx.value:
            lib.g1g2_destroy(ctx)
        assert rc in (g1g2.OK, g1g2.ENOMEM), (se, nb_, rc)
    sym = a + a.transpose(0, 2, 1)                        # complex symmetric, not Hermitian
    for L in (sym, b, (1 + 1j) * herm, np.concatenate([herm, sym[:1]])):
        assert init(L) == g1g2.ESYMM
        assert b"Hermitian" in lib.g1g2_last_error_detail()


def test_non_finite_inputs_rejected_on_host(lib):
    """A NaN or an Inf in any host input of g1g2_init / g1g2_init_factorised is refused
    (G1G2_ENONFINITE) before any device work."""
    h, w, n0 = _valid(3)
    g2 = np.zeros((3,) * 4, dtype=np.complex128)
    for name in ("h", "w", "n0", "g2"):
        args = dict(h=h.copy(), w=w.copy(), n0=n0.copy(), g2=g2.copy())
        args[name].flat[4] = np.nan if name != "w" else complex(0.0, np.inf)
        assert _init(lib, 3, args["h"], args["w"], args["n0"], g2=args["g2"]) == g1g2.ENONFINITE, name
        assert name.replace("n0", "G1_0").replace("g2", "G2_0").encode() in lib.g1g2_last_error_detail()
    wr = w.real.copy()
    wr[1, 2, 1, 2] = -np.inf
    assert _init(lib, 3, h, wr, n0, opt={"w_is_real": 1}) == g1g2.ENONFINITE
    L = np.zeros((2, 3, 3))
    L[1, 0, 0] = np.nan
    ctx = ctypes.c_void_p()
    o = g1g2.Options()
    lib.g1g2_default_options(ctypes.byref(o))
    o.w_is_real = 1
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.g1g2_init_factorised(ctypes.byref(ctx), 3, ptr(h), ptr(L), 2, ptr(n0), None, 1,
                                    ctypes.byref(o)) == g1g2.ENONFINITE
    assert b"L contains" in lib.g1g2_last_error_detail()


def test_device_allocation_failure_is_an_error_code(lib):
    """Where no device memory can be had (here: a host without a GPU), init and
    init_factorised return G1G2_ENOMEM with the failed size in the detail and leave the
    context NULL; a repeated call fails the same way (nothing half-built is kept)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: cudaMalloc succeeds")
    h, w, n0 = _valid(3)
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o = g1g2.Options()
    lib.g1g2_default_options(ctypes.byref(o))
    for _ in range(2):
        ctx = ctypes.c_void_p()
        assert lib.g1g2_init(ctypes.byref(ctx), 3, ptr(h), ptr(w), ptr(n0), None, 1, ctypes.byref(o)) == g1g2.ENOMEM
        assert ctx.value is None and b"cudaMalloc" in lib.g1g2_last_error_detail()
    o.w_is_real = 1
    L = inputs.factors(3, 2, np.random.default_rng(1))
    ctx = ctypes.c_void_p()
    assert lib.g1g2_init_factorised(ctypes.byref(ctx), 3, ptr(h), ptr(L), 2, ptr(n0), None, 1,
                                    ctypes.byref(o)) == g1g2.ENOMEM
    assert ctx.value is None


def test_symmetry_violations_rejected_on_host(lib):
    h, w, n0 = _valid(3)
    bad = w.copy()
    bad[0, 1, 2, 0] += 0.1                       # breaks w_ijkl = w_jilk
    assert _init(lib, 3, h, bad, n0) == g1g2.ESYMM
    bad = w.copy()
    bad[0, 1, 0, 2] += 0.1j                      # breaks w_ijkl = conj(w_klij)
    bad[1, 0, 2, 0] += 0.1j
    assert _init(lib, 3, h, bad, n0) == g1g2.ESYMM
    hb = h.copy()
    hb[0, 1] += 0.3
    assert _init(lib, 3, hb, w, n0) == g1g2.ESYMM
    nb_ = n0.copy()
    nb_[0, 2] += 0.3j
    assert _init(lib, 3, h, w, nb_) == g1g2.ESYMM
    g2 = np.zeros((3,) * 4, dtype=np.complex128)
    g2[0, 1, 2, 2] = 0.5
    assert _init(lib, 3, h, w, n0, g2=g2) == g1g2.ESYMM


def test_null_context_calls(lib):
    assert lib.g1g2_step(None, 0.1) == g1g2.EINVAL
    assert lib.g1g2_rhs(None, 0.0, None, None, None, None) == g1g2.EINVAL
    assert lib.g1g2_propagate(None, 0.1, 1, 1, None, None) == g1g2.EINVAL
    assert lib.g1g2_propagate_hfgkba(None, 0.1, 1, None, 0) == g1g2.EINVAL
    assert lib.g1g2_observables(None, None, None, None) == g1g2.EINVAL
    assert lib.g1g2_get_state(None, None, None, None) == g1g2.EINVAL
    assert lib.g1g2_set_state(None, 0.0, None, None) == g1g2.EINVAL
    assert lib.g1g2_set_drive(None, None, 1, None, 0) == g1g2.EINVAL
    assert lib.g1g2_launch_count(None) == -1
    lib.g1g2_destroy(None)


def test_adjoint_and_selftest_arguments_rejected_on_host(lib):
    k, w = ctypes.c_int(), ctypes.c_int()
    assert lib.g1g2_set_adjoint_checkpoints(None, 0) == g1g2.EINVAL
    assert lib.g1g2_adjoint_plan(None, ctypes.byref(k), ctypes.byref(w)) == g1g2.EINVAL
    assert lib.g1g2_adjoint(None, 0.01, 10, 0, 0, None, None, None, None, None) == g1g2.EINVAL
    assert lib.g1g2_wait_selftest(0) == g1g2.EINVAL
    assert lib.g1g2_wait_selftest(20000000) == g1g2.EINVAL


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(g1g2, "_lib", None)
    monkeypatch.setattr(g1g2, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        g1g2.load()
