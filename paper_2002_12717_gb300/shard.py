"""The G1-G2 right-hand side with G2 and w partitioned over P ranks along their first index.

This is the multi-rank partition of the hot path, written with torch.distributed
collectives and torch contractions on whatever device the tensors live on: rank r
holds the slabs G2[i in I_r] and w[i in I_r] (I_r a contiguous block of
ceil(nb/P) orbital indices, the last one ragged), and n, h replicated.  Every run
of this repository uses one GPU, where the CUDA library evaluates the whole
right-hand side; this module is the specification of the exchange steps that a
multi-GPU run needs and is exercised on CPU ranks (gloo) against the oracle.

Where each term of the right-hand side (Eqs. eom_gone-2, result_eom_soa,
g2-eq-gw-pi, g2-eq-tpp-lambda, g2-eq-tph-lambda, g2-dsl-equation-pi-lambda) needs
data of other ranks, and the collective that supplies it:

  h^HF (Eq. h_HF)       rows i in I_r from w[I_r]; all-reduce of the nb x nb matrix
  I (Eq. eom_gone-I)    partial sum over l in I_r with w_iklp = conj(w_lpik) taken
                        from w[I_r]; all-reduce of the nb x nb matrix
  [h2, G2]              = X + exch X with X = G2 x_2 h - G2 x_4 h (local), where
                        exch X_ijkl = X_jilk; one all-to-all (re-shard on index 2)
  source A              B = w~ x_2 nbar x_3 n x_4 n on w~[I_r] (local); A = nbar x_1 B
                        needs all p: one all-to-all (B re-sharded on index 2), after
                        which A's slab follows from its exchange symmetry
  A^dag                 conj(A_klij): one all-to-all (A re-sharded on index 3)
  A, A^dag (factorised) with w = sum_P L^P (x) L^P and L replicated: from M^P = nbar L^P n,
                        A_ijkl = sum_P M^P_ik M^P_jl (+ eta M^P_il M^P_jk) for any
                        index range: no exchange (w's slab is formed from L as well)
  GW hcorr (Eq. gwhcorr) w x_4 n - n x_2 w on w[I_r] (local)
  Pi (Eq. gwpi)         Pi_ijkl = sum_pq G2_ipkq hcorr_qjpl, rows i in I_r: SUMMA
                        over the 1-D row blocks, P broadcasts of one rank's hcorr
                        slab (the K panel q in I_s) each; no rank holds all of hcorr
  conj(Pi_lkji)         one all-to-all (Pi re-sharded on index 4)
  TPP hcorr (HTPPcorr)  Y = G x_2 w on w[I_r] (local); the sum over p: one all-to-all
                        (Y re-sharded on index 2), the i-slab by hcorr's exchange symmetry
  TPH hcorr (HTPHcorr)  Z = w x_4 G on w[I_r] (local); the sum over p: one all-to-all,
                        and one more back to i-slabs
  Lambda (lambdapp/ph)  rows i in I_r: SUMMA with G2's slabs as the K panels (p resp.
                        q in I_s), P broadcasts
  conj(Lambda_klij)     one all-to-all (Lambda re-sharded on index 3)
  E_corr                local partial sum, scalar all-reduce

Selfenergies: HF, SOA, GW, GW with exchange, the particle-particle and particle-hole T
matrices and DSL; fermions and bosons; spin-orbital basis or (not GW) spin-restricted.

`rk4_step_sharded` takes one classical RK4 step on the slabs: four partitioned right-hand
sides, the stage states formed locally (G2 on each rank's slab, n replicated), no
exchange beyond those of the right-hand sides.

`summa_matmul` is the 2-D block-distributed form of the nb^2 x nb^2 x nb^2 products on a
q x q process grid (panels of about N^4 / q elements broadcast along grid rows and
columns), for a partition that keeps those operands in 2-D blocks.
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


def panel_broadcast(part: Partition, own, group=None):
    """The panels of a SUMMA product: yields (lo, hi, panel) for every rank s in turn, panel being
    rank s's first-index slab `own` (first index in I_s = [lo, hi)), broadcast from s to every
    rank.  A rank holds its own slab and one panel at a time (at most ceil(nb/P) leading rows),
    never the whole tensor."""
    P, b = part.world, part.block
    shape = (b,) + tuple(own.shape[1:])
    for s in range(P):
        lo, hi = part.range(s)
        buf = _pad0(own, b).contiguous() if s == part.rank else torch.empty(shape, dtype=own.dtype, device=own.device)
        src = s if group is None else dist.get_global_rank(group, s)
        dist.broadcast(buf, src=src, group=group)
        yield lo, hi, buf[: hi - lo]


def polarisation_sharded(part: Partition, hc_slab, G_slab, group=None):
    """Pi_ijkl = sum_pq hcorr_qjpl G_ipkq (Eq. gwpi) for the rows i in I_r: the sum over (p, q)
    split by q over the ranks, rank s's slab of hcorr (q in I_s) the panel of step s."""
    Pi = torch.zeros_like(G_slab)
    for lo, hi, H in panel_broadcast(part, hc_slab, group):
        if hi > lo:
            Pi = Pi + _es("qjpl,ipkq->ijkl", H, G_slab[:, :, :, lo:hi])
    return Pi


def tpp_hcorr_sharded(part: Partition, w_slab, gl, gg, group=None):
    """hcorr_ijkl = (i hbar)^2 sum_pq (G>_ip G>_jq - G<_ip G<_jq) w_pqkl (Eq. HTPPcorr), rows i in
    I_r: Y_pjkl = sum_q G_jq w_pqkl on w's slab (p in I_r), one re-shard to j-slabs for the sum
    over p, and the exchange symmetry hcorr_ijkl = hcorr_jilk (inherited from w_ijkl = w_jilk)
    for the i-slab."""
    Y = torch.stack([_es("jq,pqkl->pjkl", gg, w_slab), _es("jq,pqkl->pjkl", gl, w_slab)], -1)
    Yj = reshard(Y, part, 1, group)                       # [p (all)][j in I_r][k][l][>, <]
    Hj = -(_es("ip,pjkl->ijkl", gg, Yj[..., 0]) - _es("ip,pjkl->ijkl", gl, Yj[..., 1]))
    return Hj.permute(1, 0, 3, 2)                         # hcorr_jilk, first index in I_r


def tph_hcorr_sharded(part: Partition, w_slab, gl, gg, group=None):
    """hcorr_ijkl = (i hbar)^2 sum_pq (G>_ip G<_ql - G<_ip G>_ql) w_pjkq (Eq. HTPHcorr), rows i in
    I_r: Z_pjkl = sum_q G_ql w_pjkq on w's slab, a re-shard to j-slabs for the sum over p and one
    back to i-slabs."""
    Z = torch.stack([_es("ql,pjkq->pjkl", gl, w_slab), _es("ql,pjkq->pjkl", gg, w_slab)], -1)
    Zj = reshard(Z, part, 1, group)                       # [p (all)][j in I_r][k][l][<, >]
    Hj = -(_es("ip,pjkl->ijkl", gg, Zj[..., 0]) - _es("ip,pjkl->ijkl", gl, Zj[..., 1]))
    Hi = reshard(Hj.transpose(0, 1).contiguous(), part, 1, group)   # [j (all)][i in I_r][k][l]
    return Hi.transpose(0, 1)


def tpp_ladder_sharded(part: Partition, H_slab, G_slab, group=None):
    """Lambda_ijkl = sum_pq hcorr_ijpq G_pqkl (Eq. lambdapp), rows i in I_r: the sum split by p,
    rank s's slab of G2 (p in I_s) the panel of step s."""
    L = torch.zeros_like(G_slab)
    for lo, hi, Gp in panel_broadcast(part, G_slab, group):
        if hi > lo:
            L = L + _es("ijpq,pqkl->ijkl", H_slab[:, :, lo:hi, :], Gp)
    return L


def tph_ladder_sharded(part: Partition, H_slab, G_slab, group=None):
    """Lambda_ijkl = sum_pq hcorr_ipql G_qjkp (Eq. lambdaph), rows i in I_r: the sum split by q,
    rank s's slab of G2 (q in I_s) the panel of step s."""
    L = torch.zeros_like(G_slab)
    for lo, hi, Gq in panel_broadcast(part, G_slab, group):
        if hi > lo:
            L = L + _es("ipql,qjkp->ijkl", H_slab[:, :, lo:hi, :], Gq)
    return L


def _es(eq, *ops):
    """torch.einsum, with an empty operand (a rank whose slab is empty) giving the zeros the
    contraction defines (an empty sum, or an empty output axis) directly."""
    if any(o.numel() == 0 for o in ops):
        ins, out = eq.split("->")
        sizes = {}
        for spec, o in zip(ins.split(","), ops):
            sizes.update(zip(spec, o.shape))
        dtype = ops[0].dtype
        for o in ops[1:]:
            dtype = torch.promote_types(dtype, o.dtype)
        return torch.zeros([sizes[c] for c in out], dtype=dtype, device=ops[0].device)
    return torch.einsum(eq, *ops)


def rhs_sharded(part: Partition, h, w_slab, n, G_slab, selfenergy="SOA", group=None, bosons=False,
                restricted=False, factors=None):
    """(dn/dt, the slab of dG2/dt) at the state (n, G2), for fermions or (bosons=True) bosons:
    eta = -1 or +1 in the +/- of the paper (G^< = -i eta n, G^> = -i nbar with nbar = 1 + eta n,
    w^+/- = w + eta w_ijlk).  In a spin-orbital basis h^HF and the source term take w^+/-; in
    the spin-restricted mode (restricted=True, one spin species of an opposite-spin
    interaction; not GW) both take the plain w.

    h, n: replicated nb x nb; w_slab = w[I_r], G_slab = G2[I_r] (complex tensors).  dn is
    the same on every rank.  The arithmetic is that of the oracle's right-hand side with
    the index ranges of the partition; the collectives are listed in the module header.

    factors: the replicated factors L (nfac x nb x nb) of w_ijkl = sum_P L^P_ik L^P_jl, or
    None.  With factors, w_slab may be None (each rank forms w[I_r] from L), and the source
    term and its conjugate transpose come from the replicated M^P = nbar L^P n with no
    exchange: A_ijkl = sum_P M^P_ik M^P_jl (+ eta M^P_il M^P_jk for w^+/-) for any index
    range."""
    nb, lo, hi = part.nb, part.lo, part.hi
    cd = n.dtype
    if factors is not None:
        factors = factors.to(cd)
    if factors is not None and w_slab is None:
        w_slab = _es("pik,pjl->ijkl", factors[:, lo:hi], factors)
    eye = torch.eye(nb, dtype=cd, device=n.device)
    eta = 1.0 if bosons else -1.0
    nbar = eye + eta * n
    # Eq. (h_HF): hHF_ij = h_ij + sum_kl (w_ikjl +/- w_iklj) n_lk, rows i in I_r
    if restricted and selfenergy in ("GW", "GWX", "DSL"):
        raise ValueError("GW couples same-spin components; no spin-restricted form")
    wpm = w_slab if restricted else w_slab + eta * w_slab.permute(0, 1, 3, 2)
    hhf = torch.zeros((nb, nb), dtype=cd, device=n.device)
    hhf[lo:hi] = _es("ikjl,lk->ij", wpm, n)
    dist.all_reduce(hhf, group=group)
    hhf = hhf + h
    if selfenergy == "HF":
        return -1j * (hhf @ n - n @ hhf), torch.zeros_like(G_slab)
    # Eq. (eom_gone-I): I_ij = +/- i sum_klp w_iklp G_lpjk, the part l in I_r; w_iklp = conj(w_lpik)
    w_t = w_slab.conj().permute(2, 3, 0, 1)               # [i][k][l in I_r][p] = w_iklp
    I = eta * 1j * _es("iklp,lpjk->ij", w_t, G_slab)
    dist.all_reduce(I, group=group)
    dn = -1j * (hhf @ n - n @ hhf) + eta * (I + I.conj().T)
    # two-particle commutator: [h2, G] = X + exch X, X = G x_2 h - G x_4 h
    X = _es("jp,ipkl->ijkl", hhf, G_slab) - _es("ijkp,pl->ijkl", G_slab, hhf)
    Xj = reshard(X, part, 1, group)                       # X[a][b in I_r][c][d]
    C = X + Xj.permute(1, 0, 3, 2)                        # exch X_abcd = X_badc, a in I_r
    # source term, Eq. (psi-pm-def): A = nbar x1 nbar x2 w~ x3 n x4 n, Psi = -A + A^dag
    if factors is not None:
        pm = selfenergy != "GW" and not restricted        # w~ = w^+/- (else the plain w)
        M = nbar @ factors @ n                            # M^P = nbar L^P n, replicated
        Mr, Mc = M[:, lo:hi], M[:, :, lo:hi]              # rows / columns in I_r
        A = _es("pik,pjl->ijkl", Mr, M)                   # i in I_r
        A_dag = _es("pki,plj->ijkl", Mc, M).conj()        # conj(A_klij): sum_P M^P_ki M^P_lj
        if pm:
            A = A + eta * _es("pil,pjk->ijkl", Mr, M)
            A_dag = A_dag + eta * _es("pli,pkj->ijkl", Mc, M).conj()   # eta M^P_kj M^P_li
    else:
        wsrc = w_slab if selfenergy == "GW" else wpm      # plain w for standard GW, w^+/- otherwise
        B = _es("jq,pqrs,rk,sl->pjkl", nbar, wsrc, n, n)  # p in I_r
        Bj = reshard(B, part, 1, group)                   # B[p (all)][j in I_r][k][l]
        Aj = _es("ip,pjkl->ijkl", nbar, Bj)               # A[i (all)][j in I_r][k][l]
        A = Aj.permute(1, 0, 3, 2)                        # A_abcd = A_badc (exchange symmetry), a in I_r
        A3 = reshard(A, part, 2, group)                   # A[a][b][c in I_r][d]
        A_dag = A3.permute(2, 3, 0, 1).conj()             # conj(A_cdab), first index in I_r
    rhs2 = C - A + A_dag
    if selfenergy in ("GW", "GWX", "DSL"):
        # Eq. (gwhcorr): hcorr = w x4 n - n x2 w (w's exchange symmetry; the eta terms of
        # nbar cancel, so the same for bosons), on w's slab
        hc = _es("ijks,sl->ijkl", w_slab, n) - _es("jq,iqkl->ijkl", n, w_slab)
        Pi = polarisation_sharded(part, hc, G_slab, group)   # Eq. (gwpi), rows i in I_r
        Pi4 = reshard(Pi, part, 3, group)                 # Pi[a][b][c][d in I_r]
        rhs2 = rhs2 + Pi - Pi4.permute(3, 2, 1, 0).conj()
    if selfenergy in ("TPP", "TPH", "DSL"):
        # the T-matrix ladder terms (Eqs. lambdapp, lambdaph; DSL takes both, each once)
        gl, gg = -1j * eta * n, -1j * nbar                # G^< and G^> at equal times
        lam = torch.zeros_like(G_slab)
        if selfenergy in ("TPP", "DSL"):
            lam = lam + tpp_ladder_sharded(part, tpp_hcorr_sharded(part, w_slab, gl, gg, group), G_slab, group)
        if selfenergy in ("TPH", "DSL"):
            lam = lam + tph_ladder_sharded(part, tph_hcorr_sharded(part, w_slab, gl, gg, group), G_slab, group)
        L3 = reshard(lam, part, 2, group)                 # Lambda[a][b][c in I_r][d]
        rhs2 = rhs2 + lam - L3.permute(2, 3, 0, 1).conj()  # - conj(Lambda_klij)
    return dn, -1j * rhs2


def rk4_step_sharded(part: Partition, h_of_t, t, w_slab, n, G_slab, dt, selfenergy="SOA", group=None,
                     bosons=False, restricted=False, factors=None):
    """One classical RK4 step of (n, G2) with G2 partitioned (the slab G2[i in I_r], n replicated):
    four right-hand sides of rhs_sharded at t, t + dt/2, t + dt/2, t + dt (h_of_t(t) the
    replicated one-body Hamiltonian at time t), the stage states formed on each rank's slab.
    With factors (and w_slab None) w's slab is formed once from them for the whole step.
    Returns (n, the slab of G2) at t + dt."""
    if factors is not None:
        factors = factors.to(n.dtype)
    if factors is not None and w_slab is None:
        w_slab = _es("pik,pjl->ijkl", factors[:, part.lo:part.hi], factors)

    def f(tt, nn, gg):
        return rhs_sharded(part, h_of_t(tt), w_slab, nn, gg, selfenergy, group, bosons, restricted, factors)
    k1 = f(t, n, G_slab)
    k2 = f(t + dt / 2, n + dt / 2 * k1[0], G_slab + dt / 2 * k1[1])
    k3 = f(t + dt / 2, n + dt / 2 * k2[0], G_slab + dt / 2 * k2[1])
    k4 = f(t + dt, n + dt * k3[0], G_slab + dt * k3[1])
    n_new = n + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
    G_new = G_slab + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return n_new, G_new


def correlation_energy_sharded(part: Partition, w_slab, G_slab, group=None, restricted=False):
    """E_corr = -1/2 Re sum_ijkl w_ijkl G2_klij in a spin-orbital basis (-Re sum in the
    spin-restricted mode, both spin species of the opposite-spin interaction), with
    G2_klij = conj(G2_ijkl): a local partial sum and one scalar all-reduce."""
    e = torch.tensor([(w_slab * G_slab.conj()).sum().real.item()], dtype=torch.float64)
    dist.all_reduce(e, group=group)
    return -(1.0 if restricted else 0.5) * e.item()


# ---------------------------------------------------------------------------
# The 2-D block-distributed form of the nb^2 x nb^2 x nb^2 products (SUMMA)
# ---------------------------------------------------------------------------

def _block(n, q, x):
    """[lo, hi) of block x when n indices are cut into q blocks of ceil(n / q)."""
    b = -(-n // q)
    lo = min(n, x * b)
    return lo, min(n, lo + b)


class Grid:
    """q x q process grid over P = q^2 ranks: rank a q + b holds block (a, b) of every matrix.
    The row and column communicators are created collectively (every rank, the same order)."""

    def __init__(self, world: int, rank: int):
        q = int(round(world ** 0.5))
        if q * q != world:
            raise ValueError("the 2-D grid needs a square number of ranks")
        self.q, self.a, self.b = q, rank // q, rank % q
        self.rows = [dist.new_group([a * q + b for b in range(q)]) for a in range(q)]
        self.cols = [dist.new_group([a * q + b for a in range(q)]) for b in range(q)]


def summa_matmul(grid: Grid, A_blk, B_blk, M: int, K: int, N: int):
    """C = A B for A (M x K), B (K x N) in q x q blocks (rows, columns and K cut into blocks of
    ceil(n / q)): rank (a, b) holds A[block a, block b] and B[block a, block b] and returns
    C[block a, block b].  Step c broadcasts A[a, c] along grid row a and B[c, b] along grid
    column b (panels of about M K / q and K N / q elements), and every rank adds their product."""
    q, a, b = grid.q, grid.a, grid.b
    mb, kb, nbk = -(-M // q), -(-K // q), -(-N // q)
    r0, r1 = _block(M, q, a)
    c0, c1 = _block(N, q, b)
    C = torch.zeros((r1 - r0, c1 - c0), dtype=torch.promote_types(A_blk.dtype, B_blk.dtype), device=A_blk.device)
    for c in range(q):
        k0, k1 = _block(K, q, c)
        Abuf = torch.zeros((mb, kb), dtype=A_blk.dtype, device=A_blk.device)
        if b == c:
            Abuf[: A_blk.shape[0], : A_blk.shape[1]] = A_blk
        dist.broadcast(Abuf, src=a * q + c, group=grid.rows[a])
        Bbuf = torch.zeros((kb, nbk), dtype=B_blk.dtype, device=B_blk.device)
        if a == c:
            Bbuf[: B_blk.shape[0], : B_blk.shape[1]] = B_blk
        dist.broadcast(Bbuf, src=c * q + b, group=grid.cols[b])
        C = C + Abuf[: r1 - r0, : k1 - k0] @ Bbuf[: k1 - k0, : c1 - c0]
    return C
