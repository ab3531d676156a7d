"""The G1-G2 right-hand side with G2 and w partitioned over P ranks along their first index.

This is the multi-rank partition of the hot path, written with torch.distributed
collectives and torch contractions on whatever device the tensors live on: rank r
holds the slabs G2[i in I_r] and w[i in I_r] (I_r a contiguous block of
ceil(nb/P) orbital indices, the last one ragged), and n, h replicated.  Every run
of this repository uses one GPU, where the CUDA library evaluates the whole
right-hand side; this module is the specification of the exchange steps that a
multi-GPU run needs and is exercised on CPU ranks (gloo) against the oracle.

Where each term of the right-hand side (Eqs. eom_gone-2, result_eom_soa,
g2-eq-gw-pi) needs data of other ranks, and the collective that supplies it:

  h^HF (Eq. h_HF)       rows i in I_r from w[I_r]; all-reduce of the nb x nb matrix
  I (Eq. eom_gone-I)    partial sum over l in I_r with w_iklp = conj(w_lpik) taken
                        from w[I_r]; all-reduce of the nb x nb matrix
  [h2, G2]              = X + exch X with X = G2 x_2 h - G2 x_4 h (local), where
                        exch X_ijkl = X_jilk; one all-to-all (re-shard on index 2)
  source A              B = w~ x_2 nbar x_3 n x_4 n on w~[I_r] (local); A = nbar x_1 B
                        needs all p: one all-to-all (B re-sharded on index 2), after
                        which A's slab follows from its exchange symmetry
  A^dag                 conj(A_klij): one all-to-all (A re-sharded on index 3)
  GW hcorr (Eq. gwhcorr) w x_4 n - n x_2 w on w[I_r] (local); the polarisation
                        Pi_ijkl = sum_pq G2_ipkq hcorr_qjpl needs all of hcorr:
                        all-gather (the one-dimensional form of the block GEMM)
  conj(Pi_lkji)         one all-to-all (Pi re-sharded on index 4)
  E_corr                local partial sum, scalar all-reduce

Selfenergies: HF, SOA, GW and GW with exchange (fermions, spin-orbital basis).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class Partition:
    """Block partition of the orbital index over `world` ranks: I_r = [lo, hi)."""

    def __init__(self, nb: int, world: int, rank: int):
        self.nb, self.world, self.rank = nb, world, rank
        self.block = -(-nb // world)
        self.lo, self.hi = self.range(rank)

    def range(self, r):
        lo = min(self.nb, r * self.block)
        return lo, min(self.nb, lo + self.block)

    def slab(self, x):
        """This rank's slab of a full nb^4 tensor (first index)."""
        return x[self.lo:self.hi]


def _pad0(x, n):
    """Zero-pad the first axis of x to length n."""
    if x.shape[0] == n:
        return x
    pad = torch.zeros((n - x.shape[0],) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
    return torch.cat([x, pad], 0)


def reshard(x, part: Partition, axis: int, group=None):
    """From the slab x[a in I_r, ...] (first index) to the slab on `axis` (1, 2 or 3):
    returns y with y[a, ...] = X[a, ...] for every a and the index on `axis` restricted
    to I_r (X the full tensor).  One all_to_all_single of equal padded blocks."""
    P, b = part.world, part.block
    xs = _pad0(x, b)                                      # [a (padded)][...]
    xs = torch.movedim(xs, axis, 0)                       # [axis][a][rest]
    xs = _pad0(xs, P * b)
    rest = tuple(xs.shape[2:])
    send = xs.reshape((P, b, b) + rest).contiguous()      # send[s]: the axis block of rank s
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)       # recv[s]: rank s's slab, axis in I_r
    y = recv.transpose(1, 2).reshape((P * b, b) + rest)   # [a (padded per rank)][axis (local)][rest]
    keep = torch.cat([torch.arange(s * b, s * b + (part.range(s)[1] - part.range(s)[0]), device=x.device)
                      for s in range(P)])
    y = y[keep][:, : part.hi - part.lo]
    return torch.movedim(y, 1, axis)


def allgather_slabs(x, part: Partition, group=None):
    """The full tensor from the first-index slabs of all ranks."""
    P, b = part.world, part.block
    xs = _pad0(x, b).contiguous()
    outs = [torch.empty_like(xs) for _ in range(P)]
    dist.all_gather(outs, xs, group=group)
    return torch.cat([outs[s][: part.range(s)[1] - part.range(s)[0]] for s in range(P)], 0)


def _es(*a):
    return torch.einsum(*a)


def rhs_sharded(part: Partition, h, w_slab, n, G_slab, selfenergy="SOA", group=None):
    """(dn/dt, the slab of dG2/dt) at the state (n, G2) for fermions in a spin-orbital basis.

    h, n: replicated nb x nb; w_slab = w[I_r], G_slab = G2[I_r] (complex tensors).  dn is
    the same on every rank.  The arithmetic is that of the oracle's right-hand side with
    the index ranges of the partition; the collectives are listed in the module header."""
    nb, lo, hi = part.nb, part.lo, part.hi
    cd = n.dtype
    eye = torch.eye(nb, dtype=cd, device=n.device)
    nbar = eye - n
    # Eq. (h_HF): hHF_ij = h_ij + sum_kl (w_ikjl - w_iklj) n_lk, rows i in I_r
    wm = w_slab - w_slab.permute(0, 1, 3, 2)
    hhf = torch.zeros((nb, nb), dtype=cd, device=n.device)
    hhf[lo:hi] = _es("ikjl,lk->ij", wm, n)
    dist.all_reduce(hhf, group=group)
    hhf = hhf + h
    if selfenergy == "HF":
        return -1j * (hhf @ n - n @ hhf), torch.zeros_like(G_slab)
    # Eq. (eom_gone-I): I_ij = -i sum_klp w_iklp G_lpjk, the part l in I_r; w_iklp = conj(w_lpik)
    w_t = w_slab.conj().permute(2, 3, 0, 1)               # [i][k][l in I_r][p] = w_iklp
    I = -1j * _es("iklp,lpjk->ij", w_t, G_slab)
    dist.all_reduce(I, group=group)
    dn = -1j * (hhf @ n - n @ hhf) - (I + I.conj().T)
    # two-particle commutator: [h2, G] = X + exch X, X = G x_2 h - G x_4 h
    X = _es("jp,ipkl->ijkl", hhf, G_slab) - _es("ijkp,pl->ijkl", G_slab, hhf)
    Xj = reshard(X, part, 1, group)                       # X[a][b in I_r][c][d]
    C = X + Xj.permute(1, 0, 3, 2)                        # exch X_abcd = X_badc, a in I_r
    # source term, Eq. (psi-pm-def): A = nbar x1 nbar x2 w~ x3 n x4 n, Psi = -A + A^dag
    wsrc = w_slab if selfenergy == "GW" else wm           # plain w for standard GW, w^- otherwise
    B = _es("jq,pqrs,rk,sl->pjkl", nbar, wsrc, n, n)      # p in I_r
    Bj = reshard(B, part, 1, group)                       # B[p (all)][j in I_r][k][l]
    Aj = _es("ip,pjkl->ijkl", nbar, Bj)                   # A[i (all)][j in I_r][k][l]
    A = Aj.permute(1, 0, 3, 2)                            # A_abcd = A_badc (exchange symmetry), a in I_r
    A3 = reshard(A, part, 2, group)                       # A[a][b][c in I_r][d]
    A_dag = A3.permute(2, 3, 0, 1).conj()                 # conj(A_cdab), first index in I_r
    rhs2 = C - A + A_dag
    if selfenergy in ("GW", "GWX"):
        # Eq. (gwhcorr): hcorr = w x4 n - n x2 w (w's exchange symmetry), all of it for Pi
        hc = _es("ijks,sl->ijkl", w_slab, n) - _es("jq,iqkl->ijkl", n, w_slab)
        hc_full = allgather_slabs(hc, part, group)
        Pi = _es("ipkq,qjpl->ijkl", G_slab, hc_full)      # Eq. (gwpi), rows i in I_r
        Pi4 = reshard(Pi, part, 3, group)                 # Pi[a][b][c][d in I_r]
        rhs2 = rhs2 + Pi - Pi4.permute(3, 2, 1, 0).conj()
    return dn, -1j * rhs2


def correlation_energy_sharded(part: Partition, w_slab, G_slab, group=None):
    """E_corr = -1/2 Re sum_ijkl w_ijkl G2_klij (spin-orbital basis), with
    G2_klij = conj(G2_ijkl): a local partial sum and one scalar all-reduce."""
    e = torch.tensor([(w_slab * G_slab.conj()).sum().real.item()], dtype=torch.float64)
    dist.all_reduce(e, group=group)
    return -0.5 * e.item()
