"""Pins of the oracle's visibility integrator (Section 3: the correlator's 0.5 s
samples are integrated into 2, 4 and 8 s groups, shorter for widely separated
tiles; reading R19: per-baseline group length, mean per group).

Independent of the oracle's loops: numpy's reshape-and-mean, constant and
linear-in-time inputs (the mean of a linear signal is its value at the group
centre), and conservation of the sum over each baseline's cadence.
"""
import numpy as np

import oracle


def cube(n_fine=16, n_bl=7, n_chan=5, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n_fine, n_bl, n_chan, 4)) + 1j * rng.normal(size=(n_fine, n_bl, n_chan, 4))


def test_integrate_equals_numpy_group_means():
    fine = cube()
    L = np.array([4, 8, 16, 4, 2, 1, 8])
    out = oracle.integrate(fine, L, n_slot=16)
    for b, l in enumerate(L):
        ref = fine[:, b].reshape(16 // l, l, 5, 4).mean(axis=1)
        np.testing.assert_allclose(out[:16 // l, b], ref, rtol=0, atol=1e-14)
        assert np.all(out[16 // l:, b] == 0)


def test_constant_and_linear_signals():
    t = np.arange(16, dtype=np.float64)
    fine = np.zeros((16, 3, 2, 4), np.complex128)
    fine[:, 0] = 2.5 - 1j                                   # constant
    fine[:, 1] = (0.3 + 0.7j) * t[:, None, None]            # linear in time
    fine[:, 2] = (1.0 + 0.5j) * t[:, None, None] ** 2       # quadratic
    out = oracle.integrate(fine, np.array([8, 4, 2]), n_slot=8)
    np.testing.assert_allclose(out[:2, 0], 2.5 - 1j, rtol=0, atol=1e-15)
    centres = np.array([4 * s + 1.5 for s in range(4)])
    np.testing.assert_allclose(out[:4, 1, 0, 0], (0.3 + 0.7j) * centres, rtol=1e-15)
    # mean of t^2 over {2s, 2s+1} = (2s)^2 + 2s + 1/2
    s = np.arange(8)
    np.testing.assert_allclose(out[:8, 2, 1, 3], (1.0 + 0.5j) * ((2 * s) ** 2 + 2 * s + 0.5), rtol=1e-15)


def test_sum_over_the_cadence_is_conserved():
    fine = cube(seed=3)
    L = np.array([1, 2, 4, 8, 16, 2, 4])
    out = oracle.integrate(fine, L, n_slot=16)
    np.testing.assert_allclose((out * L[None, :, None, None]).sum(axis=0), fine.sum(axis=0), rtol=1e-13, atol=1e-13)
