"""The 2-D block-distributed product of the partition module (shard.summa_matmul: SUMMA on a
q x q process grid, gloo CPU ranks): a ragged complex product against numpy, and the GW
polarisation (Eq. gwpi) and the particle-particle and particle-hole ladder terms
(Eqs. lambdapp, lambdaph) in their nb^2 x nb^2 matrix views against the oracle, on 2 x 2
and 3 x 3 grids."""
import os
import socket
import tempfile

import numpy as np
import pytest

from oracle import g1g2_oracle as O

from .helpers import problem

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrices(nb):
    """A ragged random product (7 x 5 times 5 x 6) and the polarisation's operands as matrices:
    A_(ik),(pq) = G2_ipkq and B_(pq),(jl) = hcorr_qjpl, so that (A B)_(ik),(jl) = Pi_ijkl."""
    rng = np.random.default_rng(5)
    A1 = rng.standard_normal((7, 5)) + 1j * rng.standard_normal((7, 5))
    B1 = rng.standard_normal((5, 6)) + 1j * rng.standard_normal((5, 6))
    h, w, n, g2, _, _ = problem(nb, "GW", complex_w=True, seed=71, drive=False)
    hc = O.gw_hcorr(w, n)
    A2 = g2.transpose(0, 2, 1, 3).reshape(nb * nb, nb * nb)
    B2 = hc.transpose(2, 0, 1, 3).reshape(nb * nb, nb * nb)
    # Eq. (lambdapp): Lambda_(ij),(kl) = sum_(pq) hpp_(ij),(pq) G_(pq),(kl)
    hpp = O.tpp_hcorr(w, n)
    A3, B3 = hpp.reshape(nb * nb, nb * nb), g2.reshape(nb * nb, nb * nb)
    # Eq. (lambdaph): Lambda_ijkl = sum_pq hph_ipql G_qjkp, rows (i,l), K (p,q), columns (j,k)
    hph = O.tph_hcorr(w, n)
    A4 = hph.transpose(0, 3, 1, 2).reshape(nb * nb, nb * nb)
    B4 = g2.transpose(3, 0, 1, 2).reshape(nb * nb, nb * nb)
    refs = {1: O.gw_polarisation(hc, g2), 2: O.tpp_ladder(hpp, g2), 3: O.tph_ladder(hph, g2)}
    return [(A1, B1), (A2, B2), (A3, B3), (A4, B4)], refs


def _worker(rank, world, port, outdir, nb):
    import torch.distributed as dist

    from paper_2002_12717_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = shard.Grid(world, rank)
        q, a, b = grid.q, grid.a, grid.b
        pairs, _ = _matrices(nb)
        for ci, (A, B) in enumerate(pairs):
            M, K = A.shape
            N = B.shape[1]
            r0, r1 = shard._block(M, q, a)
            k0, k1 = shard._block(K, q, b)
            ka, kb_ = shard._block(K, q, a)
            c0, c1 = shard._block(N, q, b)
            t = lambda x: torch.from_numpy(np.ascontiguousarray(x))
            C = shard.summa_matmul(grid, t(A[r0:r1, k0:k1]), t(B[ka:kb_, c0:c1]), M, K, N)
            np.savez(os.path.join(outdir, f"r{rank}_c{ci}.npz"), C=C.numpy(), r=(r0, r1), c=(c0, c1))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [4, 9])
def test_summa_matches_dense_product(world):
    import torch.multiprocessing as mp
    nb = 5
    with tempfile.TemporaryDirectory() as outdir:
        mp.spawn(_worker, args=(world, _free_port(), outdir, nb), nprocs=world, join=True)
        pairs, refs = _matrices(nb)
        for ci, (A, B) in enumerate(pairs):
            ref = A @ B
            got = np.full(ref.shape, np.nan, dtype=np.complex128)
            for r in range(world):
                z = np.load(os.path.join(outdir, f"r{r}_c{ci}.npz"))
                (r0, r1), (c0, c1) = z["r"], z["c"]
                got[r0:r1, c0:c1] = z["C"]
            assert np.isfinite(got).all()                      # every block written
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
            if ci:
                g4 = got.reshape(nb, nb, nb, nb)
                # the matrix views: Pi_ijkl = C_(ik),(jl) (Eq. gwpi), Lambda^pp_ijkl = C_(ij),(kl)
                # (Eq. lambdapp), Lambda^ph_ijkl = C_(il),(jk) (Eq. lambdaph)
                got4 = {1: g4.transpose(0, 2, 1, 3), 2: g4, 3: g4.transpose(0, 2, 3, 1)}[ci]
                assert np.abs(got4 - refs[ci]).max() <= 1e-12 * np.abs(refs[ci]).max(), ci
