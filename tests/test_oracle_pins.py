"""The oracle against closed forms, brute force and invariants (CPU only)."""
import pytest

import oracle

from tests.oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.load())


def test_intra_chirp_motion_at_rest_is_stop_and_hop():
    """The simulator's moving-antenna branch with zero velocity reproduces the
    stop-and-hop cube, with and without the residual video phase."""
    import numpy as np
    import synth
    radar = synth.Radar(n_samples=32, n_rx=3, os=2)
    q_tx, q_rx = synth.trajectory(radar, 5, jitter=0.02,
                                  rng=np.random.Generator(np.random.PCG64(2)))
    tg = np.array([[0.4, 3.0], [-1.0, 5.5]])
    am = np.array([1.0, 0.5j])
    for rvp in (False, True):
        a = synth.beat_signal(radar, q_tx, q_rx, tg, am, rvp=rvp)
        b = synth.beat_signal(radar, q_tx, q_rx, tg, am, rvp=rvp,
                              intra_chirp_velocity=np.zeros(2))
        assert np.max(np.abs(a - b)) < 1e-9
