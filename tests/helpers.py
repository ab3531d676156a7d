"""Shared test helpers: seeded problems for the parity tests."""
import numpy as np

from paper_2002_12717_gb300 import inputs


def sym_w_complex(nb, rng, scale=0.1):
    """Random complex w with w_ijkl = w_jilk and w_ijkl = conj(w_klij)."""
    x = rng.standard_normal((nb,) * 4) + 1j * rng.standard_normal((nb,) * 4)
    x = x + x.transpose(1, 0, 3, 2)
    x = x + x.transpose(2, 3, 0, 1).conj()
    return x * scale / 4


def problem(nb, se, restricted=False, complex_w=False, seed=0, drive=True):
    """h, w, (n, G2) random admissible state, D and a gauss-sine drive."""
    rng = np.random.default_rng(seed)
    h = inputs.random_hermitian(nb, rng)
    if restricted:
        w = inputs.onsite_w_restricted(nb, 1.3) + 0.05 * inputs.factor_w(nb, 2, rng)
    elif complex_w:
        w = sym_w_complex(nb, rng)
    else:
        w = inputs.factor_w(nb, max(2, nb), rng)
    n, g2 = inputs.random_state(nb, rng, soa=(se == "SOA" and not restricted))
    D = np.diag(rng.standard_normal(nb)).astype(np.complex128) if drive else None
    drv = inputs.GaussSine(A=0.5, omega=1.5, t0=1.0, sigma=0.8) if drive else None
    return h, w, n, g2, D, drv


def rel_err(a, b, floor=1e-6):
    """max|a - b| / max|b|, with max|b| floored (some tiny cases have an exactly vanishing result)."""
    den = max(np.abs(b).max(), floor)
    return float(np.abs(a - b).max() / den)
