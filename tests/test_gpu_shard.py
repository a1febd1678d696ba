"""Channel-sharded cadences (Section 3.1: channel groups processed by separate
workers, their numbers combined centrally) on one GPU.

Two handles hold the two halves of a band (band_n_chan = the whole band,
band_chan0 = 0 and half); they run the channel-shard calls in lockstep and their
partial averages are summed (in place, into both) before every block's solve,
as an all-reduce over two GPUs would.  The residual (both halves together) and
the Jones matrices are compared with the FP64 oracle's sequential peel of the
whole band at the tolerances of test_gpu_parity.py.  The two handles' Jones
matrices agree to FP32 rounding, not bit for bit: each shard forms the band's
closed-form in-block corrections from its own channel frequencies in FP64, and
differences of 1e-16 relative there reach the solve's FP32 iterates.  A handle
that holds the whole band gives, through the same calls with no exchange, the
bits of rts_peel_cadence.
"""
import numpy as np
import pytest

from synth import Cadence

torch = pytest.importorskip("torch")
from _parity import TOL, check_status, jones_rel, oracle_case, rms_of, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    ("two-halves", Cadence(48, 160, 4, 100, freq0_hz=167e6, seed=104), 80, 64),
    ("ragged-split", Cadence(20, 75, 3, 21, seed=105), 37, 8),     # 37 + 38 channels, blocks of 8
]


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()


def shard(cad, lo, hi, per_pass):
    from paper_1003_5575_gb300 import Peeler
    return Peeler(cad.uvw(), cad.freqs()[lo:hi], n_iter=20, precision="mixed", max_sources=cad.n_src,
                  sources_per_pass=per_pass, band_n_chan=cad.n_chan, band_chan0=lo)


@pytest.mark.parametrize("name,cad,split,per_pass", CASES, ids=[c[0] for c in CASES])
def test_two_shards_equal_the_whole_band_oracle(built, name, cad, split, per_pass):
    V, R_ref, J_ref, st_ref, rel_ref = oracle_case(cad)
    halves = [(0, split), (split, cad.n_chan)]
    ps = [shard(cad, lo, hi, per_pass) for lo, hi in halves]
    vis = [to_dev(np.ascontiguousarray(V[:, :, lo:hi]), "mixed") for lo, hi in halves]
    outs = [p.shard_begin(v, cad.sources()) for p, v in zip(ps, vis)]
    n_ex = 0
    while True:
        a, b = ps[0].shard_partials(), ps[1].shard_partials()
        a.add_(b)
        b.copy_(a)
        n_ex += 1
        rc = [p.shard_step() for p in ps]
        assert rc[0] == rc[1]
        if rc[0] == 0:
            break
    torch.cuda.synchronize()
    assert n_ex == (cad.n_src + per_pass - 1) // per_pass
    R = np.concatenate([o[0].cpu().numpy() for o in outs], axis=2)
    J0, J1 = (o[1].cpu().numpy() for o in outs)
    st0, st1 = ps[0].shard_status(), ps[1].shard_status()
    err_r = np.abs(R - R_ref).max() / rms_of(V)
    err_j = max(jones_rel(J0, J_ref), jones_rel(J1, J_ref))
    print(f"{name}: residual {err_r:.2e} x rms, Jones {err_j:.2e} (shards apart {jones_rel(J0, J1):.2e}), "
          f"{n_ex} exchanges")
    assert err_r <= TOL["mixed"]
    assert err_j <= TOL["mixed"]
    for p, st in zip(ps, (st0, st1)):
        check_status(name, st, st_ref, p.rel(cad.n_src), rel_ref)
    for p in ps:
        p.close()


def test_whole_band_shard_equals_cadence(built):
    from paper_1003_5575_gb300 import Peeler
    cad = Cadence(16, 96, 3, 20, seed=106)
    V = oracle_case(cad)[0]
    vis = to_dev(V, "mixed")
    p = Peeler(cad.uvw(), cad.freqs(), n_iter=20, precision="mixed", max_sources=cad.n_src, sources_per_pass=8)
    r0, j0, s0 = p.cadence(vis, cad.sources())
    r1, j1, s1, n = p.cadence_sharded(vis, cad.sources(), exchange=lambda t: t)
    torch.cuda.synchronize()
    assert n == 3
    assert torch.equal(r0, r1) and torch.equal(j0, j1)
    np.testing.assert_array_equal(s0, s1)
    p.close()


def test_shard_handles_refuse_the_whole_band_calls(built):
    from paper_1003_5575_gb300 import RtsError, RTS_EINVAL
    cad = Cadence(8, 32, 2, 4, seed=107)
    p = shard(cad, 0, 16, 8)
    vis = to_dev(np.ascontiguousarray(oracle_case(cad)[0][:, :, :16]), "mixed")
    with pytest.raises(RtsError) as e:
        p.cadence(vis, cad.sources())
    assert e.value.code == RTS_EINVAL
    with pytest.raises(RtsError):
        p.shard_step()                                    # no cadence in progress
    p.close()
