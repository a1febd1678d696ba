"""GPU parity of the gridder (Section 6) through the C ABI against the FP64
oracle's scatter on the same inputs.

Tolerance: |d grid| <= 1e-5 x max |grid| element by element (FP32 sums of
the ~60-450 contributions of a pixel, weights <= 1, against FP64).  The
convolution function used vanishes at r_max, so a pixel whose distance rounds
to the other side of r_max in FP32 and FP64 differs only at the FP32 level.
The grid is bitwise reproducible (fixed summation order); the sort's bin
tables are exact integers.
"""
import zlib

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


def tapered_kb(n_tab, beta=8.0):
    """Kaiser-Bessel profile shifted to vanish at r_max, 1 at r = 0."""
    r = np.linspace(0.0, 1.0, n_tab)
    k = np.i0(beta * np.sqrt(np.clip(1.0 - r * r, 0.0, None)))
    return (k - k[-1]) / (k[0] - k[-1])


def inputs(n_pix, n_vis, n_pol, seed, spread="uniform"):
    rng = np.random.default_rng(seed)
    if spread == "uniform":
        xy = rng.uniform(-3.0, n_pix + 3.0, size=(n_vis, 2))
    else:                                    # concentrated towards the centre, like a u-v plane
        r = np.abs(rng.normal(scale=n_pix / 6, size=n_vis))
        th = rng.uniform(0, 2 * np.pi, size=n_vis)
        xy = np.stack([n_pix / 2 + r * np.cos(th), n_pix / 2 + r * np.sin(th)], axis=1)
    xy = xy.astype(np.float32)
    vis = (rng.normal(size=(n_vis, n_pol)) + 1j * rng.normal(size=(n_vis, n_pol))).astype(np.complex64)
    return xy, vis


def run_gpu(n_pix, r_max, gcf, bin, xy, vis):
    from paper_1003_5575_gb300 import Gridder
    g = Gridder(n_pix, r_max, gcf, bin=bin, n_pol=vis.shape[1], max_vis=max(len(xy), 1))
    out = g.run(torch.from_numpy(xy).cuda(), torch.from_numpy(vis).cuda())
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    g.close()
    return res


CASES = [
    # name, n_pix, r_max, bin, n_vis, n_pol, spread
    ("paper-bins-uv", 200, 12.0, 24, 4000, 4, "uv"),
    ("ragged-grid", 101, 5.0, 7, 1500, 2, "uniform"),
    ("one-pol", 64, 3.5, 4, 800, 1, "uniform"),
    ("three-pol-dense", 48, 8.0, 9, 6000, 3, "uv"),
    ("bin-equals-rmax", 90, 9.0, 9, 2000, 4, "uniform"),
]


@pytest.mark.parametrize("name,n_pix,r_max,bin,n_vis,n_pol,spread", CASES, ids=[c[0] for c in CASES])
def test_grid_matches_oracle(name, n_pix, r_max, bin, n_vis, n_pol, spread):
    xy, vis = inputs(n_pix, n_vis, n_pol, seed=zlib.crc32(name.encode()) % 1000, spread=spread)
    gcf = tapered_kb(257)
    G = run_gpu(n_pix, r_max, gcf, bin, xy, vis)
    R = oracle.grid(n_pix, r_max, gcf, xy.astype(np.float64), vis.astype(np.complex128))
    assert np.abs(G - R).max() <= 1e-5 * np.abs(R).max()


def test_grid_is_reproducible_and_handles_empty_input():
    from paper_1003_5575_gb300 import Gridder
    xy, vis = inputs(150, 3000, 4, seed=5, spread="uv")
    gcf = tapered_kb(129)
    g = Gridder(150, 12.0, gcf, bin=24, n_pol=4, max_vis=3000)
    a = g.run(torch.from_numpy(xy).cuda(), torch.from_numpy(vis).cuda()).clone()
    b = g.run(torch.from_numpy(xy).cuda(), torch.from_numpy(vis).cuda())
    assert torch.equal(a, b)
    e = g.run(torch.zeros((0, 2), dtype=torch.float32, device="cuda"),
              torch.zeros((0, 4), dtype=torch.complex64, device="cuda"),
              out=torch.full((4, 150, 150), 7.0, dtype=torch.complex64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.count_nonzero(e).item() == 0
    ms = g.last_ms()
    assert ms[0] >= 0 and ms[1] >= 0
    g.close()


def test_grid_rejects_bad_configurations():
    from paper_1003_5575_gb300 import Gridder
    gcf = tapered_kb(33)
    for kw, needle in ((dict(n_pix=64, r_max=12.0, bin=8), "bin"),
                       (dict(n_pix=64, r_max=4.0, bin=50), "bin"),
                       (dict(n_pix=16384, r_max=4.0, bin=8), "8192"),
                       (dict(n_pix=64, r_max=-1.0, bin=8), "r_max")):
        with pytest.raises(RuntimeError, match=needle):
            Gridder(gcf=gcf, **kw)
    g = Gridder(64, 4.0, gcf, bin=8, n_pol=2, max_vis=10)
    with pytest.raises(RuntimeError, match="max_vis"):
        g.run(torch.zeros((11, 2), dtype=torch.float32, device="cuda"),
              torch.zeros((11, 2), dtype=torch.complex64, device="cuda"))
    g.close()


def test_grid_full_size_matches_oracle():
    """The benchmark's shape for one channel: 1125 x 1125 pixels, r_max 12 in
    24 x 24 bins, one visibility per baseline of the 512-antenna array (130 816)
    at the cadence's middle time, 4 polarisations, every pixel against the
    oracle's FP64 scatter."""
    import math
    from synth import config, baseline_pairs
    cad = config(3)
    pairs = baseline_pairs(cad.n_ant)
    uvw = cad.uvw()[cad.n_time // 2]
    duv = uvw[pairs[:, 0]] - uvw[pairs[:, 1]]
    xy = (duv[:, :2] * (cad.freqs()[0] / 299792458.0) * math.radians(21.4) + 1125 / 2.0).astype(np.float32)
    rng = np.random.default_rng(12)
    vis = (rng.normal(size=(len(xy), 4)) + 1j * rng.normal(size=(len(xy), 4))).astype(np.complex64)
    gcf = tapered_kb(1025)
    G = run_gpu(1125, 12.0, gcf, 24, xy, vis)
    R = oracle.grid(1125, 12.0, gcf, xy.astype(np.float64), vis.astype(np.complex128))
    assert np.abs(G - R).max() <= 1e-5 * np.abs(R).max()
