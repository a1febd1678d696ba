"""The adjoint at the shape of the adjoint-calibration workload: 128 antennas
(8128 baselines), 256 channels of 40 kHz from 150 MHz, 8 times, 100 sources,
source positions perturbed by N(0, (1 arcmin)^2) per coordinate, the cube
simulated from the unperturbed sky.

  * the mixed-precision loss and gradient (dL/dJ, dL/dl, dL/dm, dL/dS) through
    rts_peel_grad against the oracle's analytic gradient of the same loss:
    loss 1e-5 relative, every gradient entry within 1e-4 of its block's largest
    magnitude;
  * 10 random parameters against central differences of the FP64 GPU loss,
    Richardson-extrapolated from steps h and h/2 (truncation O(h^4)): 1e-4
    relative (the floor of the denominator is 1e-2 of the block's largest
    gradient, for entries near zero).
"""
import numpy as np
import pytest

import oracle
from synth import config

torch = pytest.importorskip("torch")
from _parity import make_peeler, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()
    cad = config(4)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0)).astype(np.complex64).astype(np.complex128)
    src = cad.perturbed_sources()
    J = cad.jones().astype(np.complex64).astype(np.complex128)
    return cad, V, src, J


def test_mixed_gradient_matches_oracle_gradient_at_config4(case):
    cad, V, src, J = case
    L_ref, gJ_ref, gl_ref, gm_ref, gS_ref = oracle.loss_grad(cad.uvw(), cad.freqs(), V, src, J)
    p = make_peeler(cad, "mixed")
    loss, gJ, gs = p.grad(to_dev(V, "mixed"), torch.from_numpy(J.astype(np.complex64)).cuda(),
                          torch.from_numpy(src).cuda())
    torch.cuda.synchronize()
    p.close()
    gJ, gs = gJ.cpu().numpy(), gs.cpu().numpy()
    errs = [abs(loss.item() - L_ref) / L_ref, np.abs(gJ - gJ_ref).max() / np.abs(gJ_ref).max()]
    for col, ref in ((0, gl_ref), (1, gm_ref), (2, gS_ref)):
        errs.append(np.abs(gs[:, col] - ref).max() / np.abs(ref).max())
    print("config 4 adjoint: loss %.2e, dL/dJ %.2e, dL/dl %.2e, dL/dm %.2e, dL/dS %.2e" % tuple(errs))
    assert errs[0] <= 1e-5
    assert max(errs[1:]) <= 1e-4


def test_gradient_matches_central_differences_at_config4(case):
    cad, V, src, J = case
    pm = make_peeler(cad, "mixed")
    _, gJ, gs = pm.grad(to_dev(V, "mixed"), torch.from_numpy(J.astype(np.complex64)).cuda(),
                        torch.from_numpy(src).cuda())
    gJ, gs = gJ.cpu().numpy(), gs.cpu().numpy()
    pm.close()
    p64 = make_peeler(cad.with_(precision="fp64"), "fp64")
    v64 = to_dev(V, "fp64")
    J64 = torch.from_numpy(J).cuda()

    def L(Jt, s):
        return p64.grad(v64, Jt, torch.from_numpy(s).cuda(), want_grad=False)[0].item()

    def central(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    rng = np.random.default_rng(2024)
    worst = 0.0
    for _ in range(10):
        k = int(rng.integers(cad.n_src))
        kind = int(rng.integers(5))
        if kind < 2:
            a, e = int(rng.integers(cad.n_ant)), int(rng.integers(4))

            def f(h, a=a, e=e, k=k, kind=kind):
                d = torch.zeros_like(J64)
                d[k, a, e] = h if kind == 0 else 1j * h
                return L(J64 + d, src)
            fd = central(f, 1e-4)
            an = gJ[k, a, e].real if kind == 0 else gJ[k, a, e].imag
            scale = np.abs(gJ).max()
        else:
            col = kind - 2

            def f(h, k=k, col=col):
                s = src.copy()
                s[k, col] += h
                return L(J64, s)
            fd = central(f, 2e-7 if col < 2 else 1e-5)
            an = gs[k, col]
            scale = np.abs(gs[:, col]).max()
        err = abs(an - fd) / max(abs(fd), 1e-2 * scale)
        worst = max(worst, err)
        assert err <= 1e-4, (kind, k, an, fd)
    print(f"config 4 central differences: worst relative error {worst:.2e} over 10 parameters")
    p64.close()
