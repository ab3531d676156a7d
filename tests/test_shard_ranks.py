"""The partition of the right-hand side over ranks (G2 and w split along their first
index, paper_2002_12717_gb300/shard.py) on CPU ranks with the gloo backend: every
rank's slab of dG2/dt, the replicated dn/dt and the correlation energy against the
oracle's full right-hand side, element by element, for every selfenergy, fermions and
bosons, spin-orbital and (not GW) spin-restricted, on 2 ranks
(nb = 6, and nb = 5 with a ragged last block), 3 ranks (nb = 5: blocks 2, 2, 1) and
4 ranks (nb = 5: blocks 2, 2, 1, 0, an empty slab and an empty SUMMA panel); and the
partitioned RK4 step over several driven steps against the oracle's propagation."""
import os
import socket
import tempfile

import numpy as np
import pytest

from oracle import g1g2_oracle as O

from paper_2002_12717_gb300 import inputs

from .helpers import problem

torch = pytest.importorskip("torch")

# (selfenergy, nb, bosons, spin-restricted)
CASES = [("SOA", 6, False, False), ("SOA", 5, False, False), ("GW", 6, False, False), ("GW", 5, False, False),
         ("GWX", 5, False, False), ("HF", 5, False, False), ("TPP", 6, False, False), ("TPP", 5, False, False),
         ("TPH", 6, False, False), ("TPH", 5, False, False), ("DSL", 6, False, False), ("DSL", 5, False, False),
         ("SOA", 5, True, False), ("GW", 5, True, False), ("GWX", 6, True, False), ("HF", 5, True, False),
         ("TPP", 5, True, False), ("TPH", 6, True, False), ("DSL", 5, True, False),
         ("SOA", 5, False, True), ("SOA", 6, False, True), ("HF", 5, False, True), ("TPP", 5, False, True),
         ("TPH", 6, False, True)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _state(nb, se, seed, restricted=False):
    se_ = se if se != "HF" else "SOA"
    if restricted:
        h, w, n, g2, _, _ = problem(nb, se_, restricted=True, seed=seed, drive=False)
    else:
        h, w, n, g2, _, _ = problem(nb, se_, complex_w=True, seed=seed, drive=False)
    return h, w, n, g2


def _worker(rank, world, port, outdir, cases):
    import torch.distributed as dist

    from paper_2002_12717_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for ci, (se, nb, bosons, rs) in enumerate(cases):
            h, w, n, g2 = _state(nb, se, 60 + ci, rs)
            part = shard.Partition(nb, world, rank)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
            dn, dg = shard.rhs_sharded(part, t(h), part.slab(t(w)), t(n), part.slab(t(g2)), se, bosons=bosons,
                                       restricted=rs)
            ec = shard.correlation_energy_sharded(part, part.slab(t(w)), part.slab(t(g2)), restricted=rs)
            np.savez(os.path.join(outdir, f"r{rank}_c{ci}.npz"), dn=dn.numpy(), dg=dg.numpy(), ec=ec,
                     lo=part.lo, hi=part.hi)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sharded_rhs_matches_oracle(world):
    import torch.multiprocessing as mp
    cases = CASES if world == 2 else [c for c in CASES if c[1] == 5]
    with tempfile.TemporaryDirectory() as outdir:
        mp.spawn(_worker, args=(world, _free_port(), outdir, cases), nprocs=world, join=True)
        for ci, (se, nb, bosons, rs) in enumerate(cases):
            h, w, n, g2 = _state(nb, se, 60 + ci, rs)
            prob = O.Problem(h, w, se, rs, bosons=bosons)
            dn_ref, dg_ref = O.rhs(prob, 0.0, n, g2)
            e_ref = -(1.0 if rs else 0.5) * np.real(np.einsum("ijkl,klij->", w, g2))
            covered = np.zeros(nb, dtype=bool)
            for r in range(world):
                z = np.load(os.path.join(outdir, f"r{r}_c{ci}.npz"))
                lo, hi = int(z["lo"]), int(z["hi"])
                covered[lo:hi] = True
                scale = max(np.abs(dg_ref).max(), 1e-300)
                assert z["dg"].shape == dg_ref[lo:hi].shape, (se, nb, r)
                if hi > lo:
                    assert np.abs(z["dg"] - dg_ref[lo:hi]).max() <= 1e-12 * scale, (se, nb, r)
                assert np.abs(z["dn"] - dn_ref).max() <= 1e-12 * np.abs(dn_ref).max(), (se, nb, r)
                assert abs(float(z["ec"]) - e_ref) <= 1e-12 * max(abs(e_ref), 1e-12)
            assert covered.all()


# (selfenergy, nb, bosons, spin-restricted, complex factors)
FACTOR_CASES = [("SOA", 5, False, False, False), ("SOA", 6, False, False, True), ("GW", 5, False, False, True),
                ("GWX", 5, False, False, False), ("TPP", 5, False, False, True), ("TPH", 5, False, False, False),
                ("DSL", 5, True, False, True), ("SOA", 5, True, False, False), ("SOA", 5, False, True, False)]


def _factor_state(nb, seed, complex_l):
    rng = np.random.default_rng(seed)
    h = inputs.random_hermitian(nb, rng)
    if complex_l:
        a = (rng.standard_normal((4, nb, nb)) + 1j * rng.standard_normal((4, nb, nb))) * 0.1
        L = (a + a.conj().transpose(0, 2, 1)) / 2
        L[1::2] *= 1j                                   # Hermitian and i-Hermitian factors
    else:
        L = inputs.factors(nb, 4, rng)
    n, g2 = inputs.random_state(nb, rng, soa=False)
    return h, L, n, g2


def _factor_worker(rank, world, port, outdir):
    import torch.distributed as dist

    from paper_2002_12717_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = {"n": 0}
    a2a = shard.dist.all_to_all_single

    def counted(*args, **kw):
        calls["n"] += 1
        return a2a(*args, **kw)
    shard.dist.all_to_all_single = counted
    try:
        for ci, (se, nb, bosons, rs, cl) in enumerate(FACTOR_CASES):
            h, L, n, g2 = _factor_state(nb, 120 + ci, cl)
            part = shard.Partition(nb, world, rank)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
            counts = []
            for use_factors in (True, False):
                calls["n"] = 0
                w_slab = None if use_factors else part.slab(t(np.einsum("pik,pjl->ijkl", L, L)))
                Lt = (torch.from_numpy(L) if np.isrealobj(L) else t(L)) if use_factors else None  # real stays real
                dn, dg = shard.rhs_sharded(part, t(h), w_slab, t(n), part.slab(t(g2)), se, bosons=bosons,
                                           restricted=rs, factors=Lt)
                counts.append(calls["n"])
                if use_factors:
                    out = dict(dn=dn.numpy(), dg=dg.numpy())
            np.savez(os.path.join(outdir, f"f{rank}_c{ci}.npz"), counts=counts, lo=part.lo, hi=part.hi, **out)
    finally:
        shard.dist.all_to_all_single = a2a
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sharded_rhs_with_factors_matches_oracle(world):
    """w given as replicated factors (each rank forms w[I_r] itself): every rank's slab of
    dG2/dt and dn/dt against the oracle's right-hand side on w = w_from_factors(L), and the
    source term's two all-to-alls gone (counted on every rank); 4 ranks at nb = 5 include an
    empty slab."""
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as outdir:
        mp.spawn(_factor_worker, args=(world, _free_port(), outdir), nprocs=world, join=True)
        for ci, (se, nb, bosons, rs, cl) in enumerate(FACTOR_CASES):
            h, L, n, g2 = _factor_state(nb, 120 + ci, cl)
            prob = O.Problem(h, O.w_from_factors(L), se, rs, bosons=bosons)
            dn_ref, dg_ref = O.rhs(prob, 0.0, n, g2)
            for r in range(world):
                z = np.load(os.path.join(outdir, f"f{r}_c{ci}.npz"))
                lo, hi = int(z["lo"]), int(z["hi"])
                assert z["dg"].shape == dg_ref[lo:hi].shape, (se, r)
                if hi > lo:
                    assert np.abs(z["dg"] - dg_ref[lo:hi]).max() <= 1e-12 * np.abs(dg_ref).max(), (se, r)
                assert np.abs(z["dn"] - dn_ref).max() <= 1e-12 * np.abs(dn_ref).max(), (se, r)
                with_f, without = z["counts"]
                assert with_f == without - 2, (se, r, with_f, without)


STEP_CASES = [("SOA", 5, False), ("GW", 5, False), ("DSL", 5, True), ("GWX", 5, False)]


def _step_worker(rank, world, port, outdir, nsteps, dt):
    import torch.distributed as dist

    from paper_2002_12717_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for ci, (se, nb, bosons) in enumerate(STEP_CASES):
            h, w, n, g2, D, drv = problem(nb, se, complex_w=True, seed=90 + ci)
            part = shard.Partition(nb, world, rank)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
            h_of_t = lambda tt: t(h + drv.f(tt) * D)
            nn, gg = t(n), part.slab(t(g2))
            L = None
            if ci == len(STEP_CASES) - 1:       # the last case: w given as factors
                L = t(inputs.factors(nb, 3, np.random.default_rng(91)))
            for m in range(nsteps):
                nn, gg = shard.rk4_step_sharded(part, h_of_t, m * dt, None if L is not None else part.slab(t(w)),
                                                nn, gg, dt, se, bosons=bosons, factors=L)
            np.savez(os.path.join(outdir, f"s{rank}_c{ci}.npz"), n=nn.numpy(), g=gg.numpy(), lo=part.lo,
                     hi=part.hi)
    finally:
        dist.destroy_process_group()


def test_sharded_rk4_steps_match_oracle():
    """Three driven RK4 steps with G2 partitioned over 3 ranks (nb = 5: blocks 2, 2, 1) against
    the oracle's steps on the whole state: SOA, GW, DSL for bosons, and GWX with w given as
    three factors."""
    import torch.multiprocessing as mp
    world, nsteps, dt = 3, 3, 0.02
    with tempfile.TemporaryDirectory() as outdir:
        mp.spawn(_step_worker, args=(world, _free_port(), outdir, nsteps, dt), nprocs=world, join=True)
        for ci, (se, nb, bosons) in enumerate(STEP_CASES):
            h, w, n, g2, D, drv = problem(nb, se, complex_w=True, seed=90 + ci)
            if ci == len(STEP_CASES) - 1:
                w = O.w_from_factors(inputs.factors(nb, 3, np.random.default_rng(91)))
            prob = O.Problem(h, w, se, False, D, drv.f, bosons=bosons)
            for m in range(nsteps):
                n, g2, _ = O.rk4_step(prob, m * dt, n, g2, dt)
            for r in range(world):
                z = np.load(os.path.join(outdir, f"s{r}_c{ci}.npz"))
                lo, hi = int(z["lo"]), int(z["hi"])
                assert np.abs(z["n"] - n).max() <= 1e-12 * np.abs(n).max(), (se, r)
                assert np.abs(z["g"] - g2[lo:hi]).max() <= 1e-12 * np.abs(g2).max(), (se, r)


def test_partition_blocks():
    from paper_2002_12717_gb300.shard import Partition
    for nb, world in ((5, 2), (5, 3), (6, 4), (7, 7), (3, 4)):
        ranges = [Partition(nb, world, r).range(r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == nb
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
