"""The allocation-free solve entry point (rts_peel_solve_noalloc).

It serves callers that may not allocate device memory or create a handle (a
pipeline whose memory is fixed at start-up, code running inside another
framework's memory pool, code inside a stream-capture region).  It keeps its
scratch in one static device array, so this file checks that it gives the
same Jones matrices as the handle-based rts_peel_solve and as the oracle's
solve, through the C ABI, on two calls in a row (the second call reuses the
scratch the first one left), and that arrays larger than the static limit and
misaligned buffers are refused.  The file name
makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import config

torch = pytest.importorskip("torch")

TOL = {"mixed": 1e-5, "fp64": 1e-10}
CDT = {"mixed": np.complex64, "fp64": np.complex128}


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_solve_matches_handle_solve_on_two_calls(built, prec):
    from paper_1003_5575_gb300 import Peeler, _abi
    cad = config(2).with_(n_src=3)
    V = oracle.simulate(cad)
    p = Peeler(cad.uvw(), cad.freqs(), n_iter=20, precision=prec, max_sources=cad.n_src)
    prec_code = _abi.RTS_PREC_MIXED if prec == "mixed" else _abi.RTS_PREC_FP64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for l, m, S in cad.sources()[:2]:                    # two calls in a row
        avg = oracle.rotate_average(cad.uvw(), cad.freqs(), V, l, m).astype(CDT[prec])
        d_avg = torch.from_numpy(avg).cuda()
        J_ref, st_ref = p.solve(d_avg, S)
        J = torch.empty((cad.n_ant, 4), dtype=J_ref.dtype, device="cuda")
        st = np.zeros(1, np.int32)
        _abi.rts_peel_solve_noalloc(ctypes.c_void_p(d_avg.data_ptr()), cad.n_ant, float(S), 20,
                                    prec_code, ctypes.c_void_p(J.data_ptr()),
                                    st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), stream)
        torch.cuda.synchronize()
        Jr, Jn = J_ref.cpu().numpy(), J.cpu().numpy()
        assert np.linalg.norm(Jn - Jr) / np.linalg.norm(Jr) <= TOL[prec]
        assert int(st[0]) == st_ref
        # and the oracle's solve of the same (rounded) average
        Jo, _, _ = oracle.als(avg.astype(np.complex128), S, cad.n_ant, n_iter=20)
        assert np.linalg.norm(Jn - Jo) / np.linalg.norm(Jo) <= TOL[prec]
    p.close()


@pytest.mark.gpu
def test_noalloc_solve_rejects_arrays_above_the_static_limit(built):
    from paper_1003_5575_gb300 import _abi
    L = _abi.lib()
    dummy = torch.zeros(8, dtype=torch.complex64, device="cuda")
    rc = L.rts_peel_solve_noalloc(ctypes.c_void_p(dummy.data_ptr()), 1025, 1.0, 20, 0,
                                  ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert rc == _abi.RTS_EINVAL
    assert "static scratch limit" in _abi.rts_peel_last_error(None)


@pytest.mark.gpu
def test_noalloc_solve_rejects_misaligned_buffers(built):
    """A buffer that does not start on a 16-byte boundary is refused on the host
    (nothing is launched with it)."""
    from paper_1003_5575_gb300 import _abi
    L = _abi.lib()
    buf = torch.zeros(64, dtype=torch.complex64, device="cuda")
    good, odd = buf.data_ptr(), buf.data_ptr() + 8
    for d_avg, d_jones in ((odd, good), (good, odd)):
        rc = L.rts_peel_solve_noalloc(ctypes.c_void_p(d_avg), 4, 1.0, 20, 0, ctypes.c_void_p(d_jones), None, None)
        assert rc == _abi.RTS_EINVAL
        assert "16-byte" in _abi.rts_peel_last_error(None)
