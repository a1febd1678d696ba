"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Inputs are the oracle's own simulation of seeded synthetic cadences (never the
CUDA path's output).  Tolerances (written here, from the stated targets):
  mixed path  residual |dR| <= 1e-5 x rms of the input cube's real components,
              Jones ||dJ_k||_F / ||J_k||_F <= 1e-5 per source,
              averages |dA| <= 1e-5 x rms, loss <= 1e-5 relative,
              gradients <= 1e-4 relative (vs the oracle's analytic gradient);
  FP64 path   1e-10 on all of these.
Integer/index work (baseline order, status codes) is exact: a source's status
is compared wherever the oracle's last relative change is farther from the 1e-6
threshold than the tolerance on that change (rel_tol), and the change itself is
compared with the oracle's.
"""
import numpy as np
import pytest

import oracle
from synth import Cadence, config

torch = pytest.importorskip("torch")
from _parity import (CDT, TOL, check_status, jones_rel, make_peeler, oracle_case, rms_of,  # noqa: E402
                     to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_5575_gb300 import build
    build.build()


# ---------------------------------------------------------------------------
# full peel

PEEL_CASES = [
    ("cfg1-fp64", config(1), "fp64"),
    ("cfg1-mixed", config(1, precision="mixed"), "mixed"),
    ("cfg2-mixed", config(2), "mixed"),
    ("ragged-mixed", Cadence(9, 37, 3, 4, seed=91), "mixed"),
    ("ragged-fp64", Cadence(9, 37, 3, 4, precision="fp64", seed=91), "fp64"),
    ("one-channel", Cadence(6, 1, 5, 2, seed=92), "mixed"),
    ("one-time", Cadence(7, 300, 1, 2, seed=93), "mixed"),
    ("two-antennas", Cadence(2, 64, 4, 1, seed=94), "mixed"),
]


@pytest.mark.parametrize("name,cad,prec", PEEL_CASES, ids=[c[0] for c in PEEL_CASES])
def test_peel_matches_oracle(name, cad, prec):
    V, R_ref, J_ref, st_ref, rel_ref = oracle_case(cad)
    p = make_peeler(cad, prec, per_pass=1)
    vis = to_dev(V, prec)
    resid, jones, st = p.cadence(vis, cad.sources())
    torch.cuda.synchronize()
    rel = p.rel(cad.n_src)
    R = resid.cpu().numpy()
    J = jones.cpu().numpy()
    tol = TOL[prec]
    err_r = np.abs(R - R_ref).max() / rms_of(V)
    err_j = jones_rel(J, J_ref)
    print(f"{name}: residual {err_r:.2e} x rms, Jones {err_j:.2e} relative")
    assert err_r <= tol
    assert err_j <= tol
    check_status(name, st, st_ref, rel, rel_ref, prec)
    # input untouched by the out-of-place call
    np.testing.assert_array_equal(vis.cpu().numpy(), V.astype(CDT[prec][0]))
    p.close()


# Cases for the blocked peel.  Each one is well conditioned: the FP64 oracle's
# Jones matrices move by well under 1e-6 when its input is perturbed by
# 1e-7 x rms, so a 1e-5 parity bound is meaningful.  Narrow-band cases with many
# sources on few antennas amplify FP32-level perturbations beyond 1e-5 whatever
# the pass structure; test_gpu_conditioning.py checks one of them against a
# bound scaled by its measured conditioning.
BLOCK_CASES = [
    ("wide768-block64", Cadence(64, 768, 4, 150, freq0_hz=167e6, seed=101), 64),  # the bench's 768-channel
    #   strip: two 128-row subtraction tiles and N = 192 in the tcgen05 pass; 64, 64, 22
    ("cfg2-blocked", config(2), 16),                                # 50 sources: blocks of 16
    ("cfg2-block64", config(2), 64),                                # one block of 50
    ("wide-blocked", Cadence(64, 384, 4, 150, freq0_hz=167e6, seed=98), 16),
    ("wide-block64", Cadence(64, 384, 4, 150, freq0_hz=167e6, seed=98), 64),   # 64, 64, 22
    ("cfg1-blocked", config(1, precision="mixed"), 16),             # 5 sources, 16 channels
    ("ragged-blocked", Cadence(9, 37, 3, 4, seed=91), 8),           # 37 channels, ragged tiles
    ("max-channels", Cadence(8, 960, 2, 5, freq0_hz=167e6, seed=99), 64),    # largest tensor-core strip
    ("odd-channels", Cadence(12, 203, 3, 9, seed=97), 64),          # ragged 16-channel row tiles
    ("odd-antennas", Cadence(40, 256, 4, 70, freq0_hz=167e6, seed=105), 64),   # 40 antennas: partial
    #   32-antenna correction tiles off the diagonal, CTAs whose share of tile rows spans two tiles;
    #   64 + 6 (256 channels: the oracle moves by 3.5e-8 under a 1e-7 x rms input perturbation, where
    #   64 channels gave 8.7e-7, too ill-conditioned for the 1e-5 bound)
]
# (pass kernel, solve kernel): FP32 FMA or tensor-core pass; the block's solve
# chain as one cooperative launch (0) or as one launch per step (1)
KERNELS = [((1, 0), "fma"), ((2, 0), "tensor"), ((2, 1), "tensor-launches"), ((3, 0), "tcgen05")]


@pytest.mark.parametrize("kernel", [k for k, _ in KERNELS], ids=[n for _, n in KERNELS])
@pytest.mark.parametrize("name,cad,per_pass", BLOCK_CASES, ids=[c[0] for c in BLOCK_CASES])
def test_blocked_peel_matches_sequential_oracle(name, cad, per_pass, kernel):
    """One HBM pass per block of RTS_BLOCK sources with in-block closed-form
    corrections, with the FP32 FMA pass or the tensor-core pass, and the solve
    chain of a block in one cooperative launch or in one launch per step: the
    same results as the oracle's one-source-at-a-time peel."""
    if kernel[0] == 3 and cad.n_chan > 768:
        pytest.skip("the tcgen05 pass holds at most 768 channels")
    V, R_ref, J_ref, st_ref, rel_ref = oracle_case(cad)
    p = make_peeler(cad, "mixed", per_pass=per_pass, block_kernel=kernel[0], solve_kernel=kernel[1])
    vis = to_dev(V, "mixed")
    resid, jones, st = p.cadence(vis, cad.sources())
    torch.cuda.synchronize()
    rel = p.rel(cad.n_src)
    err_r = np.abs(resid.cpu().numpy() - R_ref).max() / rms_of(V)
    err_j = jones_rel(jones.cpu().numpy(), J_ref)
    print(f"{name}: residual {err_r:.2e} x rms, Jones {err_j:.2e} relative")
    assert err_r <= TOL["mixed"]
    assert err_j <= TOL["mixed"]
    check_status(name, st, st_ref, rel, rel_ref)
    # in place gives the same bits
    work = vis.clone()
    r2, j2, _ = p.cadence(work, cad.sources(), resid=work)
    torch.cuda.synchronize()
    assert torch.equal(r2, resid) and torch.equal(j2, jones)
    np.testing.assert_array_equal(vis.cpu().numpy(), V.astype(np.complex64))
    p.close()


def test_in_place_equals_out_of_place_and_is_deterministic():
    cad = config(2).with_(n_src=6)
    V = oracle_case(config(2))[0]
    p = make_peeler(cad, "mixed", per_pass=1)
    vis = to_dev(V, "mixed")
    r1, j1, _ = p.cadence(vis, cad.sources())
    r2, j2, _ = p.cadence(vis, cad.sources())
    work = vis.clone()
    r3, j3, _ = p.cadence(work, cad.sources(), resid=work)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2) and torch.equal(j1, j2)
    assert torch.equal(r1, r3) and torch.equal(j1, j3)
    p.close()


def test_zero_sources_copies_input():
    cad = Cadence(5, 8, 2, 1, seed=5)
    V = oracle.simulate(cad)
    p = make_peeler(cad, "mixed")
    vis = to_dev(V, "mixed")
    resid, jones, st = p.cadence(vis, np.zeros((0, 3)))
    torch.cuda.synchronize()
    assert torch.equal(resid, vis) and jones.shape[0] == 0 and len(st) == 0
    p.close()


# ---------------------------------------------------------------------------
# single steps


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_rotate_average_matches_oracle(prec):
    cad = config(2).with_(precision=prec, n_src=8)
    V = oracle.simulate(cad)
    V = V.astype(CDT[prec][0]).astype(np.complex128)
    p = make_peeler(cad, prec)
    vis = to_dev(V, prec)
    for (l, m, _) in cad.sources()[:3]:
        ref = oracle.rotate_average(cad.uvw(), cad.freqs(), V, l, m)
        got = p.rotate_average(vis, l, m).cpu().numpy()
        assert np.abs(got - ref).max() <= TOL[prec] * rms_of(V)
    p.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_solve_matches_oracle_on_oracle_average(prec):
    cad = config(2).with_(precision=prec)
    V = oracle.simulate(cad)
    l, m, S = cad.sources()[0]
    avg = oracle.rotate_average(cad.uvw(), cad.freqs(), V, l, m)
    avg_in = avg.astype(CDT[prec][0]).astype(np.complex128)
    J_ref, st_ref, rel_ref = oracle.als(avg_in, S, cad.n_ant, n_iter=20)
    p = make_peeler(cad, prec)
    J, st = p.solve(torch.from_numpy(avg_in.astype(CDT[prec][0])).cuda(), S)
    J = J.cpu().numpy()
    assert np.linalg.norm(J - J_ref) / np.linalg.norm(J_ref) <= TOL[prec]
    check_status(f"solve-{prec}", [st], [st_ref], p.rel(1), [rel_ref], prec)
    p.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_predict_matches_oracle(prec):
    cad = Cadence(11, 70, 3, 40, precision=prec, seed=55)
    p = make_peeler(cad, prec)
    J = torch.from_numpy(cad.jones().astype(CDT[prec][0])).cuda()
    Jr = J.cpu().numpy().astype(np.complex128)
    ref = oracle.predict(cad.uvw(), cad.freqs(), cad.sources(), Jr)
    got = p.predict(cad.sources(), J).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL[prec] * rms_of(ref)
    # accumulate = add to what is there
    base = torch.ones(p.cube_shape, dtype=CDT[prec][1], device="cuda")
    got2 = p.predict(cad.sources(), J, out=base, accumulate=True).cpu().numpy()
    assert np.abs(got2 - (ref + 1.0)).max() <= TOL[prec] * rms_of(ref) + 1e-6
    p.close()


# ---------------------------------------------------------------------------
# adjoint


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_loss_and_gradient_match_oracle(prec):
    cad = Cadence(10, 90, 3, 5, precision=prec, pos_sigma_rad=2.909e-4, seed=66)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    V = V.astype(CDT[prec][0]).astype(np.complex128)
    src = cad.perturbed_sources()
    J = cad.jones().astype(CDT[prec][0]).astype(np.complex128)
    L_ref, gJ_ref, gl_ref, gm_ref, gS_ref = oracle.loss_grad(cad.uvw(), cad.freqs(), V, src, J)
    p = make_peeler(cad, prec)
    loss, gJ, gs = p.grad(to_dev(V, prec), torch.from_numpy(J.astype(CDT[prec][0])).cuda(),
                          torch.from_numpy(src).cuda())
    torch.cuda.synchronize()
    gtol = 1e-4 if prec == "mixed" else 1e-9
    assert abs(loss.item() - L_ref) <= TOL[prec] * L_ref
    gJ = gJ.cpu().numpy()
    assert np.abs(gJ - gJ_ref).max() <= gtol * np.abs(gJ_ref).max()
    gs = gs.cpu().numpy()
    for col, ref in ((0, gl_ref), (1, gm_ref), (2, gS_ref)):
        assert np.abs(gs[:, col] - ref).max() <= gtol * np.abs(ref).max(), col
    p.close()


# the mixed adjoint's two sweeps: factorised phasor tables (default) and one
# sin/cos per sample; shapes with several channel tiles of the factorised sweep
# (384 channels), ragged 16-channel groups, a source count whose tables do not
# fit in shared memory (the default then takes the per-sample sweep), and one source
ADJ_CASES = [
    ("two-tiles-ragged", Cadence(6, 410, 2, 7, pos_sigma_rad=2.909e-4, seed=68)),
    ("one-channel", Cadence(5, 1, 3, 4, pos_sigma_rad=2.909e-4, seed=69)),
    ("one-source", Cadence(7, 100, 2, 1, pos_sigma_rad=2.909e-4, seed=70)),
    ("600-sources", Cadence(3, 24, 1, 600, pos_sigma_rad=2.909e-4, seed=71)),
]


@pytest.mark.parametrize("grad_kernel", [0, 1], ids=["auto", "direct"])
@pytest.mark.parametrize("name,cad", ADJ_CASES, ids=[c[0] for c in ADJ_CASES])
def test_mixed_adjoint_sweeps_match_oracle(name, cad, grad_kernel):
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0)).astype(np.complex64).astype(np.complex128)
    src = cad.perturbed_sources()
    J = cad.jones().astype(np.complex64).astype(np.complex128)
    L_ref, gJ_ref, gl_ref, gm_ref, gS_ref = oracle.loss_grad(cad.uvw(), cad.freqs(), V, src, J)
    p = make_peeler(cad, "mixed", grad_kernel=grad_kernel)
    loss, gJ, gs = p.grad(to_dev(V, "mixed"), torch.from_numpy(J.astype(np.complex64)).cuda(),
                          torch.from_numpy(src).cuda())
    torch.cuda.synchronize()
    p.close()
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    gJ = gJ.cpu().numpy()
    assert np.abs(gJ - gJ_ref).max() <= 1e-4 * np.abs(gJ_ref).max()
    gs = gs.cpu().numpy()
    for col, ref in ((0, gl_ref), (1, gm_ref), (2, gS_ref)):
        assert np.abs(gs[:, col] - ref).max() <= 1e-4 * np.abs(ref).max(), col


def test_misaligned_cube_rejected():
    """A cube or a Jones array that does not start on a 16-byte boundary is refused on the host."""
    cad = Cadence(4, 16, 2, 2, seed=72)
    p = make_peeler(cad, "mixed")
    buf = torch.zeros(cad.n_vis * 4 + 1, dtype=torch.complex64, device="cuda")
    v = buf[1:].view(p.cube_shape)
    J = torch.from_numpy(cad.jones().astype(np.complex64)).cuda()
    src = torch.from_numpy(cad.sources()).cuda()
    with pytest.raises(RuntimeError, match="16-byte"):
        p.grad(v, J, src)
    with pytest.raises(RuntimeError, match="16-byte"):
        p.cadence(v, cad.sources())
    # a Jones array one complex64 past a 16-byte boundary (never launched on)
    vis = torch.zeros(p.cube_shape, dtype=torch.complex64, device="cuda")
    jbuf = torch.zeros(cad.n_src * cad.n_ant * 4 + 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError, match="16-byte"):
        p.cadence(vis, cad.sources(), jones=jbuf[1:].view(cad.n_src, cad.n_ant, 4))
    p.close()


def test_gradient_matches_central_differences_of_gpu_loss():
    """Central differences of the FP64 GPU loss against the mixed-path gradient."""
    cad = Cadence(8, 64, 2, 4, precision="fp64", pos_sigma_rad=2.909e-4, seed=67)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    src = cad.perturbed_sources()
    J = cad.jones()
    p64 = make_peeler(cad, "fp64")
    pm = make_peeler(cad.with_(precision="mixed"), "mixed")
    v64 = to_dev(V, "fp64")
    _, gJ, gs = pm.grad(to_dev(V, "mixed"), torch.from_numpy(J.astype(np.complex64)).cuda(),
                        torch.from_numpy(src).cuda())
    gJ, gs = gJ.cpu().numpy(), gs.cpu().numpy()
    J64 = torch.from_numpy(J.astype(np.complex64).astype(np.complex128)).cuda()

    def L(Jt, s):
        return p64.grad(v64, Jt, torch.from_numpy(s).cuda(), want_grad=False)[0].item()

    rng = np.random.default_rng(8)
    for _ in range(10):
        k = int(rng.integers(cad.n_src))
        kind = int(rng.integers(5))
        if kind < 2:
            a, e = int(rng.integers(cad.n_ant)), int(rng.integers(4))
            h = 1e-6
            d = torch.zeros_like(J64)
            d[k, a, e] = h if kind == 0 else 1j * h
            fd = (L(J64 + d, src) - L(J64 - d, src)) / (2 * h)
            an = gJ[k, a, e].real if kind == 0 else gJ[k, a, e].imag
            scale = np.abs(gJ).max()
        else:
            col = kind - 2
            h = 1e-7 if col < 2 else 1e-6
            s1, s2 = src.copy(), src.copy()
            s1[k, col] += h
            s2[k, col] -= h
            fd = (L(J64, s1) - L(J64, s2)) / (2 * h)
            an = gs[k, col]
            scale = np.abs(gs[:, col]).max()
        assert abs(an - fd) <= 1e-4 * max(abs(fd), 1e-2 * scale), (kind, an, fd)
    p64.close()
    pm.close()


def test_peel_loss_autograd_function():
    from paper_1003_5575_gb300 import PeelLoss
    cad = Cadence(8, 32, 2, 3, pos_sigma_rad=2.909e-4, seed=68)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    p = make_peeler(cad, "mixed")
    vis = to_dev(V, "mixed")
    J = torch.from_numpy(cad.jones().astype(np.complex64)).cuda().requires_grad_(True)
    src = torch.from_numpy(cad.perturbed_sources()).cuda().requires_grad_(True)
    loss = PeelLoss.apply(p, vis, J, src)
    (3.0 * loss).backward()
    _, gJ, gs = p.grad(vis, J.detach(), src.detach())
    assert torch.allclose(J.grad, 3.0 * gJ) and torch.allclose(src.grad, 3.0 * gs)
    p.close()


# ---------------------------------------------------------------------------
# errors (raised on the host or reported through status; nothing faults)


def test_bad_sources_rejected():
    from paper_1003_5575_gb300 import RtsError, RTS_EINVAL
    cad = Cadence(5, 8, 2, 1, seed=5)
    p = make_peeler(cad, "mixed", max_sources=2)
    vis = to_dev(oracle.simulate(cad), "mixed")
    for bad in ([[0.9, 0.9, 1.0]], [[0.1, 0.1, 0.0]], [[np.nan, 0.0, 1.0]], [[0.0, 0.0, 1.0]] * 3):
        with pytest.raises(RtsError) as e:
            p.cadence(vis, np.array(bad))
        assert e.value.code == RTS_EINVAL
    p.close()


def test_nonfinite_input_reported():
    from paper_1003_5575_gb300 import RtsError, RTS_ENONFINITE
    cad = Cadence(6, 16, 2, 2, seed=6)
    V = oracle.simulate(cad)
    V[0, 3, 5, 0] = np.nan
    p = make_peeler(cad, "mixed")
    with pytest.raises(RtsError) as e:
        p.cadence(to_dev(V, "mixed"), cad.sources())
    assert e.value.code == RTS_ENONFINITE
    p.close()


def test_pipelined_host_cadences_equal_device_cadences():
    """rts_peel_pipeline_submit/wait (copies of one cadence overlapping the peel
    of the other) give the same bits as rts_peel_cadence on the device."""
    import ctypes
    from paper_1003_5575_gb300 import _abi
    cad = Cadence(16, 64, 3, 20, seed=71)
    V1 = oracle.simulate(cad).astype(np.complex64)
    V2 = oracle.simulate(cad.with_(seed=72)).astype(np.complex64)
    p = make_peeler(cad, "mixed")
    refs = []
    for V in (V1, V2, V1):
        r, j, st = p.cadence(torch.from_numpy(V).cuda(), cad.sources())
        refs.append((r.cpu().numpy(), j.cpu().numpy(), st.copy()))
    nbytes = V1.nbytes
    bufs = [_abi.rts_host_alloc(nbytes) for _ in range(5)]
    try:
        def view(ptr):
            return np.ctypeslib.as_array((ctypes.c_float * (V1.size * 2)).from_address(ptr)).view(np.complex64).reshape(V1.shape)
        ins = [view(bufs[0]), view(bufs[1])]
        ins[0][...] = V1
        ins[1][...] = V2
        outs = [view(bufs[2]), view(bufs[3]), view(bufs[4])]
        jones = [np.zeros((cad.n_src, cad.n_ant, 4), np.complex64) for _ in range(3)]
        sts = [np.zeros(cad.n_src, np.int32) for _ in range(3)]
        src = np.ascontiguousarray(cad.sources())
        for i, vin in enumerate((ins[0], ins[1], ins[0])):
            _abi.rts_peel_pipeline_submit(p.h, ctypes.c_void_p(vin.ctypes.data), ctypes.c_void_p(outs[i].ctypes.data),
                                          cad.n_src, src.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.c_void_p(jones[i].ctypes.data),
                                          sts[i].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        _abi.rts_peel_pipeline_wait(p.h)
        for i in range(3):
            np.testing.assert_array_equal(outs[i], refs[i][0])
            np.testing.assert_array_equal(jones[i], refs[i][1])
            np.testing.assert_array_equal(sts[i], refs[i][2])
    finally:
        for b in bufs:
            _abi.rts_host_free(b)
        p.close()


def test_tcgen05_pass_channel_limit():
    """The tcgen05 pass holds a strip of up to 768 channels: above that the
    automatic choice is the mma.sync pass (same results), an explicit request fails."""
    from paper_1003_5575_gb300 import RtsError, RTS_EINVAL
    cad = Cadence(8, 800, 2, 5, freq0_hz=167e6, seed=95)
    with pytest.raises(RtsError) as e:
        make_peeler(cad, "mixed", per_pass=64, block_kernel=3)
    assert e.value.code == RTS_EINVAL
    V, R_ref, J_ref, _, _ = oracle_case(cad)
    p = make_peeler(cad, "mixed", per_pass=64)
    resid, jones, _ = p.cadence(to_dev(V, "mixed"), cad.sources())
    torch.cuda.synchronize()
    assert np.abs(resid.cpu().numpy() - R_ref).max() <= TOL["mixed"] * rms_of(V)
    assert jones_rel(jones.cpu().numpy(), J_ref) <= TOL["mixed"]
    p.close()


def test_tensor_pass_channel_limit():
    """The tensor-core pass holds a strip of up to 960 channels: above that the
    automatic choice is the FP32 pass (same results), an explicit request fails."""
    from paper_1003_5575_gb300 import RtsError, RTS_EINVAL
    cad = Cadence(6, 976, 2, 3, freq0_hz=150e6, seed=96)
    with pytest.raises(RtsError) as e:
        make_peeler(cad, "mixed", per_pass=64, block_kernel=2)
    assert e.value.code == RTS_EINVAL
    V, R_ref, J_ref, _, _ = oracle_case(cad)
    p = make_peeler(cad, "mixed", per_pass=64)
    resid, jones, _ = p.cadence(to_dev(V, "mixed"), cad.sources())
    torch.cuda.synchronize()
    assert np.abs(resid.cpu().numpy() - R_ref).max() <= TOL["mixed"] * rms_of(V)
    assert jones_rel(jones.cpu().numpy(), J_ref) <= TOL["mixed"]
    p.close()


def test_persistent_solve_equals_per_step_launches():
    """The cooperative block solve and the per-step launches compute the same
    corrected averages, sweeps and model matrices; only the grouping of the FP32
    partial sums of the normal equations differs, so Jones matrices and
    residuals agree to FP32 rounding (far inside the oracle tolerance)."""
    cad = Cadence(64, 384, 4, 150, freq0_hz=167e6, seed=98)
    V = oracle.simulate(cad)
    vis = to_dev(V, "mixed")
    out = []
    for solve in (0, 1):
        p = make_peeler(cad, "mixed", per_pass=64, block_kernel=2, solve_kernel=solve)
        r, j, st = p.cadence(vis, cad.sources())
        torch.cuda.synchronize()
        out.append((r.cpu().numpy(), j.cpu().numpy(), st, p.rel(cad.n_src)))
        p.close()
    (r0, j0, s0, rel0), (r1, j1, s1, rel1) = out
    assert jones_rel(j0, j1) <= 3e-6
    assert np.abs(r0 - r1).max() <= 3e-6 * rms_of(V)
    # the per-step launches solve in FP64 from FP64 iterates: their changes
    # stand in for the reference
    check_status("coop-vs-launches", s0, s1, rel0, rel1)

