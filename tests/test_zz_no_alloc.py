"""g1g2_g1_rhs_noalloc, the G1 right-hand side that allocates no device memory.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or loops that must not allocate between steps): its scratch is a
static device array.  The GPU tests call it through the C ABI twice in a row,
on different states and sizes up to the largest the scratch holds (nb = 64),
and compare each result with the oracle's G1 right-hand side and with the dn
output of the context-based g1g2_rhs; they check that the calls leave the
device's free memory and torch's reserved memory unchanged, and run it on a
non-default stream.  The CPU tests check that the binding rejects a wrong
dtype, shape or device before anything is launched.  This file is named to be
collected last.
"""
import ctypes
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import g1g2_oracle as O
from paper_2002_12717_gb300 import g1g2

from .helpers import problem, rel_err

TOL_FP64 = 1e-12


def _noalloc_fn():
    lib = g1g2.load()
    fn = lib.g1g2_g1_rhs_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 6
    return lib, fn


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _oracle_dn(h, w, n, g2, restricted):
    """dn/dt of Eq. (eom_gone-2) from the oracle, with h^HF of Eq. (h_HF) and I of Eq. (eom_gone-I)."""
    hhf = O.hf_hamiltonian(h, w, n, restricted)
    return O.g1_rhs(hhf, n, O.collision_integral(w, g2))


@pytest.mark.gpu
@pytest.mark.parametrize("cases", [[(24, False, 31), (17, True, 32)], [(64, False, 33), (64, False, 34)]])
def test_noalloc_matches_oracle_and_context_rhs_on_two_calls(cases):
    torch = pytest.importorskip("torch")
    lib, fn = _noalloc_fn()
    for nb, restricted, seed in cases:
        h, w, n, g2, _, _ = problem(nb, "SOA", restricted=restricted, complex_w=not restricted, seed=seed,
                                    drive=False)
        n_d, g_d = _dev(torch, n), _dev(torch, g2)
        dn_ref = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
        dg_ref = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
        with g1g2.Propagator(h, w, n, None, "SOA", "fp64", restricted) as p:
            p.rhs(0.0, n_d, g_d, dn_ref, dg_ref)
        torch.cuda.synchronize()
        h_d, w_d = _dev(torch, h), _dev(torch, w)
        dn = torch.full((nb, nb), np.nan, dtype=torch.complex128, device="cuda")
        rc = fn(nb, 1 if restricted else 0, h_d.data_ptr(), w_d.data_ptr(), n_d.data_ptr(), g_d.data_ptr(),
                dn.data_ptr(), None)
        torch.cuda.synchronize()
        assert rc == g1g2.OK, lib.g1g2_last_error_detail()
        got = dn.cpu().numpy()
        assert rel_err(got, _oracle_dn(h, w, n, g2, restricted)) < TOL_FP64
        assert rel_err(got, dn_ref.cpu().numpy()) < TOL_FP64


@pytest.mark.gpu
def test_noalloc_allocates_nothing_and_runs_on_a_side_stream():
    torch = pytest.importorskip("torch")
    nb = 32
    h, w, n, g2, _, _ = problem(nb, "SOA", complex_w=True, seed=35, drive=False)
    ref = _oracle_dn(h, w, n, g2, False)
    h_d, w_d, n_d, g_d = (_dev(torch, a) for a in (h, w, n, g2))
    dn = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    side = torch.cuda.Stream()
    # first calls: the scratch address lookup and the lazy loading of every kernel involved
    # (the library's and torch's fill) may allocate; only the calls after them are measured
    for stream in (None, side):
        dn.fill_(float("nan"))
        g1g2.g1_rhs_noalloc(h_d, w_d, n_d, g_d, dn, stream=stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for stream in (None, side, side.cuda_stream):
        dn.fill_(float("nan"))
        torch.cuda.synchronize()
        with torch.cuda.stream(side if stream is not None else torch.cuda.current_stream()):
            g1g2.g1_rhs_noalloc(h_d, w_d, n_d, g_d, dn, stream=stream)
        torch.cuda.synchronize()
        assert rel_err(dn.cpu().numpy(), ref) < TOL_FP64
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    lib, fn = _noalloc_fn()
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    p = x.data_ptr()
    assert fn(65, 0, p, p, p, p, p, None) == g1g2.EINVAL
    assert b"no-allocation scratch" in lib.g1g2_last_error_detail()
    assert fn(0, 0, p, p, p, p, p, None) == g1g2.EINVAL


def _fake(shape, dtype, device=0, cuda=True, contiguous=True):
    """Stand-in with the tensor attributes the binding inspects (no device needed)."""
    numel = int(np.prod(shape))
    return SimpleNamespace(shape=tuple(shape), dtype=dtype, is_cuda=cuda, device=SimpleNamespace(index=device),
                           dim=lambda: len(shape), numel=lambda: numel, is_contiguous=lambda: contiguous)


def test_noalloc_binding_rejects_bad_tensors_before_any_launch():
    torch = pytest.importorskip("torch")
    c128, nb = torch.complex128, 8
    good = dict(h=_fake((nb, nb), c128), w=_fake((nb,) * 4, c128), n=_fake((nb, nb), c128),
                g2=_fake((nb,) * 4, c128), dn=_fake((nb, nb), c128))
    assert g1g2.check_noalloc_args(**good, current_device=0) == nb
    flat = dict(good, w=_fake((nb ** 4,), c128), g2=_fake((nb ** 4,), c128))
    assert g1g2.check_noalloc_args(**flat, current_device=0) == nb
    bad = [
        ("w", _fake((nb,) * 4, torch.complex64), "complex128"),
        ("g2", _fake((nb, nb, nb, nb - 1), c128), "elements"),
        ("dn", _fake((nb, nb + 1), c128), "elements"),
        ("n", _fake((nb * nb,), c128), "elements"),
        ("h", _fake((nb, nb), c128, cuda=False), "CUDA"),
        ("w", _fake((nb,) * 4, c128, contiguous=False), "contiguous"),
        ("g2", _fake((nb,) * 4, c128, device=1), "current device"),
    ]
    for name, x, msg in bad:
        with pytest.raises(ValueError, match=msg):
            g1g2.check_noalloc_args(**dict(good, **{name: x}), current_device=0)
