"""The phase step (S0/S1) against a direct FP64 evaluation.

The kernels form each channel's phase in Q0.64 fixed point, A + c B modulo one
turn with A = frac(tau nu_0 / c) and B = frac(tau dnu / c) from an FP64 delay
(the blocked schedule takes A and B as differences of the two antennas' Q0.64
phases), and hand it to the hardware sin/cos rounded to Q0.32 and converted to
FP32.
The oracle evaluates tau nu_c / c in FP64 and reduces it by x - round(x).  At
the benchmark's geometry (512 antennas within 750 m, 768 channels 167-197.7 MHz,
8 times) and at directions with large |w (n - 1)| terms, on sampled
(time, baseline) pairs including the longest baselines:
  * Q0.64 phase, both forms: |dphi| <= (n_chan + 1) 2^-33 turns (the error
    bound of a Q0.32 accumulator over n_chan channels), and in fact <= 1e-10
    turns (FP64 rounding of the products);
  * the FP32 value given to sin/cos: |dphi| <= 2^-33 (Q0.32 rounding) + 2^-25
    (FP32 rounding of a number below 1/2) + 1e-10.
"""
import numpy as np
import pytest

import oracle
from synth import config

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()


def wrap(x):
    return (x + 0.5) % 1.0 - 0.5


@pytest.mark.parametrize("l,m", [(0.3, -0.3), (0.0, 0.0), (-0.25, 0.28), (0.7, 0.69)])
def test_fixed_point_phase_matches_fp64_phase(built, l, m):
    from paper_1003_5575_gb300 import Peeler
    cad = config(3).with_(n_src=1)
    uvw, freq = cad.uvw(), cad.freqs()
    p = Peeler(uvw, freq, n_iter=20, precision="mixed", max_sources=1, sources_per_pass=1)
    ai, aj = oracle.baseline_antennas(cad.n_ant)
    rng = np.random.default_rng(7)
    bl_len = np.linalg.norm(uvw[0, ai] - uvw[0, aj], axis=1)
    longest = np.argsort(bl_len)[-64:]
    bls = np.concatenate([longest, rng.integers(0, len(ai), 192)])
    ts = rng.integers(0, cad.n_time, len(bls))
    tb = np.stack([ts, bls], axis=1)
    q64 = p.phases(l, m, tb).cpu().numpy()
    f32 = p.phases(l, m, tb, form=1).cpu().numpy()
    ant = p.phases(l, m, tb, form=2).cpu().numpy()
    p.close()
    ref = np.empty_like(q64)
    for r, (t, b) in enumerate(tb):
        tau = oracle.delay_m(uvw, int(t), int(ai[b]), int(aj[b]), l, m)
        ref[r] = [oracle.phase_turns(tau, f) for f in freq]
    d64 = np.abs(wrap(q64 - ref)).max()
    d32 = np.abs(wrap(f32 - ref)).max()
    dant = np.abs(wrap(ant - ref)).max()
    print(f"(l, m) = ({l}, {m}): Q0.64 phase {d64:.2e} turns, from antenna phases {dant:.2e}, "
          f"FP32 sin/cos argument {d32:.2e} turns")
    for d in (d64, dant):
        assert d <= (cad.n_chan + 1) * 2.0 ** -33
        assert d <= 1e-10
    assert d32 <= 2.0 ** -33 + 2.0 ** -25 + 1e-10
    assert np.all(np.abs(q64) <= 0.5) and np.all(np.abs(f32) <= 0.5)


def test_out_of_range_pairs_give_nan(built):
    from paper_1003_5575_gb300 import Peeler
    cad = config(1)
    p = Peeler(cad.uvw(), cad.freqs(), n_iter=20, precision="mixed", max_sources=1, sources_per_pass=1)
    out = p.phases(0.1, 0.1, [[0, 0], [cad.n_time, 0], [0, cad.n_bl], [-1, 3]]).cpu().numpy()
    p.close()
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1:]))
