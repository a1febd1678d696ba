"""GPU parity of the visibility integrator (Section 3's first stage; reading
R19) through the C ABI against the oracle: FP32 sums of at most 16 samples
against FP64, |d| <= 1e-6 x max |input| element by element; slots past a
baseline's group count are exactly zero."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()


@pytest.mark.parametrize("n_fine,n_bl,n_chan,lens,n_slot", [
    (16, 45, 37, [4, 8, 16], 4),        # 0.5 s samples into 2, 4 and 8 s groups, ragged channels
    (16, 21, 1, [1, 2, 4, 8, 16], 16),  # one channel, every group length
    (12, 10, 64, [3, 4, 6, 12], 6),     # lengths that are not powers of two
])
def test_integrate_matches_oracle(n_fine, n_bl, n_chan, lens, n_slot):
    from paper_1003_5575_gb300 import Integrator
    rng = np.random.default_rng(n_fine * 1000 + n_bl)
    fine = (rng.normal(size=(n_fine, n_bl, n_chan, 4)) + 1j * rng.normal(size=(n_fine, n_bl, n_chan, 4))).astype(np.complex64)
    L = np.array([lens[b % len(lens)] for b in range(n_bl)], np.int32)
    ig = Integrator(n_fine, n_chan, L, n_slot)
    out = ig.run(torch.from_numpy(fine).cuda()).cpu().numpy()
    ig.close()
    ref = oracle.integrate(fine.astype(np.complex128), L, n_slot)
    assert np.abs(out - ref).max() <= 1e-6 * np.abs(fine).max()
    for b in range(n_bl):
        assert np.all(out[n_fine // L[b]:, b] == 0)


def test_integration_lengths_and_rejections():
    from paper_1003_5575_gb300 import Integrator, integration_lengths
    pos = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0], [0.0, 800.0, 0.0], [1500.0, 0.0, 0.0]])
    L = integration_lengths(pos, [700.0, 1400.0], [16, 8, 4])
    d = [np.linalg.norm(pos[i] - pos[j]) for i in range(4) for j in range(i + 1, 4)]
    np.testing.assert_array_equal(L, [16 if x < 700 else (8 if x < 1400 else 4) for x in d])
    with pytest.raises(RuntimeError, match="divide"):
        Integrator(16, 4, np.array([3, 4], np.int32))
    with pytest.raises(RuntimeError, match="n_slot"):
        Integrator(16, 4, np.array([4, 8], np.int32), n_slot=2)
