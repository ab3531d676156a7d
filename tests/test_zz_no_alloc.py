"""g1g2_g1_rhs_noalloc, the G1 right-hand side that allocates no device memory.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or loops that must not allocate between steps): its scratch is a
static device array.  Here it is called through the C ABI twice in a row, on
different states and sizes, and each result is compared with the dn output of
the context-based g1g2_rhs at the FP64 parity tolerance.  This file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2002_12717_gb300 import g1g2

from .helpers import problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


def _noalloc_fn():
    lib = g1g2.load()
    fn = lib.g1g2_g1_rhs_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 6
    return lib, fn


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("cases", [[(24, False, 31), (17, True, 32)]])
def test_noalloc_matches_context_rhs_on_two_calls(cases):
    lib, fn = _noalloc_fn()
    for nb, restricted, seed in cases:
        h, w, n, g2, _, _ = problem(nb, "SOA", restricted=restricted, complex_w=not restricted, seed=seed,
                                    drive=False)
        n_d, g_d = _dev(n), _dev(g2)
        dn_ref = torch.zeros((nb, nb), dtype=torch.complex128, device="cuda")
        dg_ref = torch.zeros((nb,) * 4, dtype=torch.complex128, device="cuda")
        with g1g2.Propagator(h, w, n, None, "SOA", "fp64", restricted) as p:
            p.rhs(0.0, n_d, g_d, dn_ref, dg_ref)
        torch.cuda.synchronize()
        h_d, w_d = _dev(h), _dev(w)
        dn = torch.full((nb, nb), np.nan, dtype=torch.complex128, device="cuda")
        rc = fn(nb, 1 if restricted else 0, h_d.data_ptr(), w_d.data_ptr(), n_d.data_ptr(), g_d.data_ptr(),
                dn.data_ptr(), None)
        torch.cuda.synchronize()
        assert rc == g1g2.OK, lib.g1g2_last_error_detail()
        assert rel_err(dn.cpu().numpy(), dn_ref.cpu().numpy()) < TOL_FP64


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib, fn = _noalloc_fn()
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    p = x.data_ptr()
    assert fn(65, 0, p, p, p, p, p, None) == g1g2.EINVAL
    assert b"no-allocation scratch" in lib.g1g2_last_error_detail()
    assert fn(0, 0, p, p, p, p, p, None) == g1g2.EINVAL
