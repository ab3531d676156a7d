"""The oracle's work against the scaling the paper prints in Table I (tests/golden/
table1_scaling.txt).  Every contraction of the oracle is costed exactly along the plan
numpy executes for it (np.einsum_path, the plan of optimize=True): each pairwise step costs
the product of the sizes of all its indices.  The total for one right-hand side is then a
polynomial in N_b, and its degree -- found from finite differences of exact integers --
must be the G1-G2 exponent of Table I: 5 for SOA, 6 for GW, TPP, TPH and DSL.  The
G1-G2 propagation is of degree 1 in N_t, the memory-integral HF-GKBA (SOA) of degree 5 in
N_b and 2 in N_t.  An evaluation that goes through a costlier intermediate than the
paper's successive sums (e.g. the source term through the nb^4 outer product of two G's,
an nb^6 step) fails here."""
import os

import numpy as np
import pytest

from oracle import g1g2_oracle as O
from oracle import hfgkba
from paper_2002_12717_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_scaling.txt")


def table1():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        se, *vals = line.split()
        rows[se] = [None if v == "-" else int(v) for v in vals]
    return rows


def plan_cost(eq, *ops):
    """Exact multiply-add count of einsum(eq, *ops) along numpy's contraction plan."""
    path = np.einsum_path(eq, *ops, optimize="greedy")[0][1:]
    ins, out = eq.replace(" ", "").split("->")
    terms = ins.split(",")
    size = {}
    for t, o in zip(terms, ops):
        size.update(zip(t, o.shape))
    cost = 0
    for step in path:
        idx = set().union(*(terms[i] for i in step))
        rest = [t for k, t in enumerate(terms) if k not in step]
        keep = "".join(sorted(c for c in idx if c in out or any(c in t for t in rest)))
        c = 1
        for ch in idx:
            c *= size[ch]
        cost += c
        terms = rest + [keep]
    return cost


class FlopCounter:
    """Wraps einsum: runs it and adds the exact cost of the plan numpy uses for it."""

    def __init__(self, einsum):
        self.einsum, self.cost = einsum, 0

    def __call__(self, eq, *ops, **kw):
        self.cost += plan_cost(eq, *ops)
        return self.einsum(eq, *ops, **kw)


def degree(values):
    """Degree of the polynomial through equidistant exact integer samples (finite differences)."""
    d, k = list(values), 0
    while any(d) and len(d) > 1:
        d = [b - a for a, b in zip(d, d[1:])]
        k += 1
    assert not any(d), "too few samples for the degree"
    return k - 1


def _counted(monkeypatch, fn):
    c_oracle = FlopCounter(O.einsum)
    c_np = FlopCounter(np.einsum)
    monkeypatch.setattr(O, "einsum", c_oracle)
    monkeypatch.setattr(hfgkba.np, "einsum", c_np)
    try:
        fn()
    finally:
        monkeypatch.undo()
    return c_oracle.cost + c_np.cost


def _rhs_cost(monkeypatch, se, nb):
    rng = np.random.default_rng(nb)
    h = inputs.random_hermitian(nb, rng)
    w = inputs.factor_w(nb, 2, rng)
    n, g2 = inputs.random_state(nb, rng, soa=False)
    prob = O.Problem(h, w, se)
    return _counted(monkeypatch, lambda: O.rhs(prob, 0.0, n, g2))


@pytest.mark.parametrize("se", ["SOA", "GW", "TPP", "TPH", "DSL"])
def test_rhs_work_has_the_degree_of_table1(se, monkeypatch):
    costs = [_rhs_cost(monkeypatch, se, nb) for nb in range(3, 12)]
    assert degree(costs) == table1()[se][0]


def test_g1g2_propagation_is_linear_in_nt(monkeypatch):
    nb = 4
    rng = np.random.default_rng(1)
    h = inputs.random_hermitian(nb, rng)
    prob = O.Problem(h, inputs.factor_w(nb, 2, rng), "GW")
    n0 = inputs.lowest_projector(h, 2)
    costs = [_counted(monkeypatch, lambda: O.propagate(prob, n0, np.zeros((nb,) * 4), 0.02, nt, obs_every=nt))
             for nt in range(1, 6)]
    assert degree(costs) == table1()["GW"][1] == 1


def test_memory_integral_hfgkba_has_the_degrees_of_table1(monkeypatch):
    """SOA, standard HF-GKBA: degree 5 in N_b at fixed N_t, degree 2 in N_t at fixed N_b."""
    nb_exp, nt_exp = table1()["SOA"][2:]

    def cost(nb, nt):
        rng = np.random.default_rng(nb)
        h = inputs.random_hermitian(nb, rng)
        prob = O.Problem(h, inputs.factor_w(nb, 2, rng), "SOA")
        n0 = inputs.lowest_projector(h, max(1, nb // 2))
        return _counted(monkeypatch, lambda: hfgkba.propagate_hfgkba(prob, n0, 0.02, nt))
    assert degree([cost(nb, 3) for nb in range(2, 10)]) == nb_exp
    assert degree([cost(3, nt) for nt in range(2, 7)]) == nt_exp
