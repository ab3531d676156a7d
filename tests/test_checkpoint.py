"""Checkpoint and resume of the propagated state (g1g2.save_checkpoint / load_checkpoint)
on the host: the archive round-trips t, G1 and G2 bit for bit and refuses a propagator of
another size, selfenergy or basis.  A stand-in with the Propagator's get_state/set_state
interface keeps this on the CPU; the two calls themselves are covered by the GPU tests."""
import numpy as np
import pytest

from paper_2002_12717_gb300 import g1g2


class StandIn:
    def __init__(self, nb, selfenergy="SOA", restricted=False, seed=0):
        rng = np.random.default_rng(seed)
        self.nb, self.selfenergy, self.restricted = nb, selfenergy, restricted
        self.t = float(rng.standard_normal())
        self.n = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
        self.g = rng.standard_normal((nb,) * 4) + 1j * rng.standard_normal((nb,) * 4)

    def get_state(self, with_g2=True):
        return self.t, self.n.copy(), self.g.copy()

    def set_state(self, t, n, G2=None):
        self.t, self.n, self.g = t, np.array(n), np.array(G2)


def test_checkpoint_round_trip(tmp_path):
    src, dst = StandIn(5, "GW", seed=1), StandIn(5, "GW", seed=2)
    path = tmp_path / "state.npz"
    g1g2.save_checkpoint(src, path)
    assert g1g2.load_checkpoint(dst, path) == src.t
    assert np.array_equal(dst.n, src.n) and np.array_equal(dst.g, src.g)
    assert dst.n.dtype == np.complex128 and dst.g.shape == (5,) * 4


@pytest.mark.parametrize("other", [dict(nb=4), dict(nb=5, selfenergy="SOA"), dict(nb=5, selfenergy="GW",
                                                                                 restricted=True)])
def test_checkpoint_refuses_another_problem(tmp_path, other):
    path = tmp_path / "state.npz"
    g1g2.save_checkpoint(StandIn(5, "GW"), path)
    dst = StandIn(**other)
    before = dst.get_state()
    with pytest.raises(ValueError):
        g1g2.load_checkpoint(dst, path)
    assert dst.t == before[0] and np.array_equal(dst.n, before[1])    # untouched
