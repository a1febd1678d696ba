"""The benchmark's launch configuration against the oracle on a slice of the
benchmark's shape that the oracle can peel.

The benchmark peels 512 antennas x 768 channels (167-197.7 MHz) x 8 times with
the library defaults: blocks of 64 sources per pass, the tcgen05 pass (a
768-channel strip: two 128-row subtraction tiles, N = 192 in the average) and
the cooperative block solve.  Here the same defaults peel 128 antennas (8128
baselines) x 768 channels x 8 times x 130 sources (blocks of 64, 64 and 2), and
every residual element, every source's Jones matrices, statuses and last
relative changes are compared with the FP64 oracle's sequential peel at the
tolerances of test_gpu_parity.py.  The cadence's conditioning (how far the
oracle's own results move when its input moves by 1e-7 x rms) is printed
beside the errors.
"""
import numpy as np
import pytest

from synth import Cadence

torch = pytest.importorskip("torch")
from _parity import TOL, check_status, conditioning, jones_rel, make_peeler, oracle_case, rms_of, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

SLICE = Cadence(128, 768, 8, 130, freq0_hz=167e6, seed=103)


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import _abi, build
    build.build()
    return _abi


def test_default_configuration_matches_oracle_on_128_antennas(built):
    cad = SLICE
    V, R_ref, J_ref, st_ref, rel_ref = oracle_case(cad)
    p = make_peeler(cad, "mixed")                      # library defaults, as the benchmark
    assert built.rts_peel_kernels(p.h)[0] == built.RTS_BLOCK_TCGEN05
    vis = to_dev(V, "mixed")
    resid, jones, st = p.cadence(vis, cad.sources())
    torch.cuda.synchronize()
    assert built.rts_peel_kernels(p.h)[1] == built.RTS_SOLVE_AUTO    # the cooperative solve ran
    rel = p.rel(cad.n_src)
    err_r = np.abs(resid.cpu().numpy() - R_ref).max() / rms_of(V)
    err_j = jones_rel(jones.cpu().numpy(), J_ref)
    dj, dr = conditioning(cad, V)
    print(f"128x768x8x130: residual {err_r:.2e} x rms, Jones {err_j:.2e}; oracle moved by "
          f"{dj:.2e} (Jones) / {dr:.2e} (residual) under a 1e-7 x rms input perturbation")
    p.close()
    assert err_r <= TOL["mixed"]
    assert err_j <= TOL["mixed"]
    check_status("128x768x8x130", st, st_ref, rel, rel_ref)
