"""Failure detection of the cooperative block solve's grid barrier, on the GPU
without a fault: a barrier that expects one CTA more than were launched cannot
complete, so every CTA's wait must run out its time limit (or see another CTA's
abort flag) and the kernel must return, with the failure reported to the host
instead of a hang.  Through the C ABI (rts_barrier_selftest)."""
import time

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build, _abi
    build.build()
    return _abi


@pytest.mark.gpu
def test_barrier_completes_when_every_cta_arrives(abi):
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert abi.rts_barrier_selftest(n_sm, 0, 200) == n_sm


@pytest.mark.gpu
def test_barrier_gives_up_when_a_cta_never_arrives(abi):
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    t0 = time.perf_counter()
    done = abi.rts_barrier_selftest(n_sm, 1, 3)
    dt = time.perf_counter() - t0
    assert done == 0                       # no CTA got past the first barrier
    assert dt < 20.0                       # bounded: one 2 s wait limit, then the abort flag
    # the context stays usable
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0
    assert abi.rts_barrier_selftest(8, 0, 10) == 8


@pytest.mark.gpu
def test_barrier_selftest_rejects_bad_arguments(abi):
    from paper_1003_5575_gb300 import RtsError, RTS_EINVAL
    for args in ((0, 0, 1), (8, 2, 1), (8, 0, 0)):
        with pytest.raises(RtsError) as e:
            abi.rts_barrier_selftest(*args)
        assert e.value.code == RTS_EINVAL


@pytest.mark.gpu
def test_fp64_rate_probe_is_plausible(abi):
    """The FP64 FMA rate probe (the FP64 path's roofline denominator) returns a
    rate between GB300's nominal FP64 figure's order of magnitude bounds."""
    r = abi.rts_fp64_rate()
    assert 0.1 < r < 100.0, r
