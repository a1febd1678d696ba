"""GPU parity of the ionospheric position-offset step (Section 3, Section 3.1)
through the C ABI, against the FP64 oracle on the oracle's own simulations.

Tolerances: the normal matrix H is FP64 on both sides from the same inputs
(relative 1e-12); the gradient g and the loss follow the adjoint's targets
(mixed 1e-4 / 1e-5 relative, FP64 1e-9 / 1e-10); the step -H^-1 g may then
differ by at most ||H^-1||_2 times the bound on g's error.
"""
import numpy as np
import pytest

import oracle
from synth import Cadence

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CDT = {"mixed": (np.complex64, torch.complex64), "fp64": (np.complex128, torch.complex128)}
NU_REF = 150e6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()


def _peeler(uvw, freq, prec, n_src):
    from paper_1003_5575_gb300 import Peeler
    return Peeler(uvw, freq, precision=prec, max_sources=max(n_src, 1))


def _dev(a, prec=None):
    a = a.astype(CDT[prec][0]) if prec else a
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _predict_shifted(cad, src, J, shifts, alpha):
    """Model with every source k moved by (NU_REF/nu_c)^alpha shifts[k] at each
    channel: one single-channel oracle prediction per channel."""
    freq = cad.freqs()
    parts = []
    for c in range(cad.n_chan):
        s = src.copy()
        s[:, :2] += (NU_REF / freq[c]) ** alpha * shifts
        parts.append(oracle.predict(cad.uvw(), freq[c:c + 1], s, J))
    return np.concatenate(parts, axis=2)


def _case(cad, prec, alpha, zero_flux=()):
    """Cube simulated with the true gains at the catalogue positions moved by a
    per-source shift under the (NU_REF/nu)^alpha law; returns (V, J, catalogue, shift)."""
    cat = cad.sources().copy()
    for k in zero_flux:
        cat[k, 2] = 0.0
    shift = cad.perturbed_sources()[:, :2] - cad.sources()[:, :2]
    J = cad.jones().astype(CDT[prec][0]).astype(np.complex128)
    V = _predict_shifted(cad, cat, J, shift, alpha)
    V = V.astype(CDT[prec][0]).astype(np.complex128)
    return V, J, cat, shift


def _check_against_oracle(out, off, out_ref, off_ref, prec):
    np.testing.assert_allclose(out[:, :3], out_ref[:, :3], rtol=1e-12)
    gtol, ltol = (1e-4, 1e-5) if prec == "mixed" else (1e-9, 1e-10)
    for col in (3, 4):
        assert np.abs(out[:, col] - out_ref[:, col]).max() <= gtol * np.abs(out_ref[:, col]).max(), col
    assert np.abs(out[:, 5] - out_ref[:, 5]).max() <= ltol * out_ref[0, 5]
    # |d delta_k| <= ||H_k^-1||_2 |d g_k|, |d g_k| <= sqrt(2) gtol max|g|
    gmax = np.abs(out_ref[:, 3:5]).max()
    for k in range(len(out_ref)):
        if out_ref[k, 0] * out_ref[k, 2] - out_ref[k, 1] ** 2 <= 0:
            assert np.all(off[k] == 0.0) and np.all(off_ref[k] == 0.0)
            continue
        H = np.array([[out_ref[k, 0], out_ref[k, 1]], [out_ref[k, 1], out_ref[k, 2]]])
        bound = np.linalg.norm(np.linalg.inv(H), 2) * np.sqrt(2) * gtol * gmax
        assert np.linalg.norm(off[k] - off_ref[k]) <= bound + 1e-12 * np.abs(off_ref).max(), k


@pytest.mark.parametrize("alpha", [0.0, 2.0])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("shape", [(10, 90, 3, 5), (9, 37, 2, 3), (33, 600, 2, 2)],
                         ids=["10ant-5src", "ragged", "two-channel-tiles"])
def test_offsets_match_oracle(alpha, prec, shape):
    cad = Cadence(*shape, precision=prec, pos_sigma_rad=2e-5, seed=77)
    V, J, cat, _ = _case(cad, prec, alpha)
    out_ref, off_ref = oracle.offsets(cad.uvw(), cad.freqs(), V, cat, J, alpha=alpha, nu_ref=NU_REF)
    p = _peeler(cad.uvw(), cad.freqs(), prec, cad.n_src)
    out, off = p.offsets(_dev(V, prec), _dev(J, prec), _dev(cat), alpha=alpha, nu_ref_hz=NU_REF)
    torch.cuda.synchronize()
    p.close()
    _check_against_oracle(out.cpu().numpy(), off.cpu().numpy(), out_ref, off_ref, prec)


@pytest.mark.parametrize("alpha", [0.0, 2.0])
def test_offsets_recover_the_position_shifts(alpha):
    """Well-separated sources, shifts of about 4 arcsec under the frequency law,
    known gains: the step returns every source's shift to a few per cent."""
    cad = Cadence(32, 128, 4, 3, precision="fp64", pos_sigma_rad=2e-5, seed=78)
    V, J, cat, shift = _case(cad, "fp64", alpha)
    p = _peeler(cad.uvw(), cad.freqs(), "fp64", cad.n_src)
    _, off = p.offsets(_dev(V), _dev(J), _dev(cat), alpha=alpha, nu_ref_hz=NU_REF)
    off = off.cpu().numpy()
    p.close()
    assert np.abs(off - shift).max() <= 0.05 * np.abs(shift).max()


def test_channel_groups_add_up_to_the_full_band():
    """Two handles over the two halves of the band (as two GPUs would hold
    them): their six numbers add to the full band's, and rts_offsets_solve on
    the sum gives the full-band step of the oracle."""
    from paper_1003_5575_gb300 import offsets_solve
    cad = Cadence(12, 64, 3, 4, precision="fp64", pos_sigma_rad=2e-5, seed=80)
    V, J, cat, _ = _case(cad, "fp64", 2.0)
    f = cad.freqs()
    out_ref, off_ref = oracle.offsets(cad.uvw(), f, V, cat, J, alpha=2.0, nu_ref=NU_REF)
    six = torch.zeros((cad.n_src, 6), dtype=torch.float64, device="cuda")
    for lo, hi in ((0, 27), (27, 64)):
        p = _peeler(cad.uvw(), f[lo:hi], "fp64", cad.n_src)
        out, _ = p.offsets(_dev(V[:, :, lo:hi].copy()), _dev(J), _dev(cat), alpha=2.0, nu_ref_hz=NU_REF)
        six += out
        torch.cuda.synchronize()
        p.close()
    off = offsets_solve(six)
    torch.cuda.synchronize()
    np.testing.assert_allclose(six.cpu().numpy(), out_ref, rtol=1e-9, atol=1e-12 * np.abs(out_ref).max())
    np.testing.assert_allclose(off.cpu().numpy(), off_ref, rtol=1e-8, atol=1e-12)


def test_solve_of_oracle_statistics_matches_oracle_step():
    from paper_1003_5575_gb300 import offsets_solve
    cad = Cadence(10, 40, 2, 5, precision="fp64", pos_sigma_rad=2e-5, seed=81)
    V, J, cat, _ = _case(cad, "fp64", 2.0, zero_flux=(2,))
    out_ref, off_ref = oracle.offsets(cad.uvw(), cad.freqs(), V, cat, J, alpha=2.0, nu_ref=NU_REF)
    off = offsets_solve(_dev(out_ref)).cpu().numpy()
    np.testing.assert_allclose(off, off_ref, rtol=1e-13, atol=0)
    assert np.all(off[2] == 0.0)


def test_zero_flux_source_gets_no_step_and_zero_sources_is_noop():
    cad = Cadence(8, 40, 2, 3, precision="fp64", pos_sigma_rad=2e-5, seed=79)
    V, J, cat, _ = _case(cad, "fp64", 2.0, zero_flux=(1,))
    out_ref, off_ref = oracle.offsets(cad.uvw(), cad.freqs(), V, cat, J, alpha=2.0, nu_ref=NU_REF)
    p = _peeler(cad.uvw(), cad.freqs(), "fp64", cad.n_src)
    out, off = p.offsets(_dev(V), _dev(J), _dev(cat), alpha=2.0, nu_ref_hz=NU_REF)
    torch.cuda.synchronize()
    out, off = out.cpu().numpy(), off.cpu().numpy()
    assert np.all(out[1, :3] == 0.0) and np.all(off[1] == 0.0) and np.all(off_ref[1] == 0.0)
    _check_against_oracle(out, off, out_ref, off_ref, "fp64")
    o0, d0 = p.offsets(_dev(V), _dev(J[:0]), torch.zeros((0, 3), dtype=torch.float64).cuda())
    assert o0.shape == (0, 6) and d0.shape == (0, 2)
    p.close()


def test_bad_offset_arguments_rejected():
    from paper_1003_5575_gb300 import RtsError, RTS_EINVAL
    cad = Cadence(6, 16, 2, 2, precision="fp64", seed=82)
    V = oracle.simulate(cad)
    p = _peeler(cad.uvw(), cad.freqs(), "fp64", cad.n_src)
    args = (_dev(V), _dev(cad.jones()), _dev(cad.sources()))
    for kw in ({"alpha": float("nan")}, {"alpha": 2.0, "nu_ref_hz": 0.0},
               {"alpha": 2.0, "nu_ref_hz": float("inf")}):
        with pytest.raises(RtsError) as e:
            p.offsets(*args, **kw)
        assert e.value.code == RTS_EINVAL
    with pytest.raises(RtsError):
        p.offsets(_dev(V), _dev(np.zeros((3, 6, 4), np.complex128)), _dev(np.zeros((3, 3))))
    p.close()
