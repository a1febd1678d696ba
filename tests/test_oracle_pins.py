"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one oracle function to something independent of its code: a
number the paper prints (Table 1), a closed form (geometric series, a
constant visibility), an invariant (antenna relabelling), a special case that
reduces to a textbook routine, brute-force least squares, or finite
differences / automatic differentiation of the loss.
"""
import math

import numpy as np
import pytest

import oracle
from synth import Cadence, config, baseline_pairs
from tests.conftest import golden

C_LIGHT = 299792458.0


def small(n_ant=8, n_chan=12, n_time=3, n_src=1, **kw):
    kw.setdefault("freq0_hz", 150e6)
    kw.setdefault("seed", 4242)
    return Cadence(n_ant, n_chan, n_time, n_src, **kw)


def mats(J):
    return np.asarray(J).reshape(*np.shape(J)[:-1], 2, 2)


def herm(a):
    return np.conj(np.swapaxes(a, -1, -2))


def pair_products(J, n_ant):
    """J_i J_j^H for every baseline (numpy matmul, not the oracle)."""
    pairs = baseline_pairs(n_ant)
    M = mats(J)
    return M[pairs[:, 0]] @ herm(M[pairs[:, 1]])


# ---------------------------------------------------------------------------
# baselines (bit exact) and the paper's Table 1


def test_baseline_count_matches_paper_table():
    g = golden("mwa_vital_statistics.txt")
    assert oracle.n_baselines(int(g["tiles"])) == int(g["baselines"])


@pytest.mark.parametrize("n_ant", [2, 3, 4, 32, 128, 512])
def test_baseline_map_bit_exact(n_ant):
    expect = {}
    b = 0
    for i in range(n_ant):
        for j in range(i + 1, n_ant):
            expect[(i, j)] = b
            b += 1
    assert oracle.n_baselines(n_ant) == b
    ai, aj = oracle.baseline_antennas(n_ant)
    for (i, j), idx in list(expect.items())[:: max(1, len(expect) // 2000)]:
        assert oracle.baseline_index(n_ant, i, j) == idx
        assert (ai[idx], aj[idx]) == (i, j)
    np.testing.assert_array_equal(np.stack([ai, aj], 1), baseline_pairs(n_ant))


# ---------------------------------------------------------------------------
# phase


def test_phase_reduction_in_turns():
    nu = 150e6
    for whole, frac in [(2, 0.25), (-3, -0.125), (0, 0.375), (7, -0.4375)]:
        tau = (whole + frac) * C_LIGHT / nu
        assert oracle.phase_turns(tau, nu) == pytest.approx(frac, abs=1e-12)
        assert -0.5 <= oracle.phase_turns(tau, nu) <= 0.5


def test_point_source_at_phase_centre_is_constant():
    """l = m = 0: zero delay for every baseline, so V is constant over (t, c)
    and equals S J_i J_j^H."""
    cad = small(n_src=1)
    J = cad.jones()
    src = np.array([[0.0, 0.0, 3.5]])
    V = oracle.predict(cad.uvw(), cad.freqs(), src, J)
    expect = 3.5 * pair_products(J[0], cad.n_ant).reshape(-1, 4)
    np.testing.assert_allclose(V, np.broadcast_to(expect[None, :, None, :], V.shape),
                               rtol=0, atol=1e-14)


def test_rotation_to_source_direction_removes_phase():
    """Rotating a one-source cube to that source's direction and averaging
    returns S J_i J_j^H on every baseline (rotate o unrotate = identity)."""
    cad = small(n_src=1)
    J = cad.jones()
    src = np.array([[0.21, -0.13, 2.0]])
    V = oracle.predict(cad.uvw(), cad.freqs(), src, J)
    A = oracle.rotate_average(cad.uvw(), cad.freqs(), V, 0.21, -0.13)
    np.testing.assert_allclose(A, 2.0 * pair_products(J[0], cad.n_ant).reshape(-1, 4),
                               rtol=0, atol=1e-12)


def _dirichlet_average(uvw, freq, l1, m1, l2, m2):
    """mean_{t,c} exp(-2 pi i (tau1 - tau2) nu_c / c) by the geometric series
    sum_{c<N} r^c = (1 - r^N)/(1 - r), independent of the oracle's loops."""
    n_time, n_ant = uvw.shape[:2]
    pairs = baseline_pairs(n_ant)
    nu0, dnu, N = freq[0], freq[1] - freq[0], len(freq)
    n1, n2 = math.sqrt(1 - l1 * l1 - m1 * m1), math.sqrt(1 - l2 * l2 - m2 * m2)
    acc = np.zeros(len(pairs), np.complex128)
    for t in range(n_time):
        b = uvw[t, pairs[:, 0]] - uvw[t, pairs[:, 1]]
        dtau = b[:, 0] * (l1 - l2) + b[:, 1] * (m1 - m2) + b[:, 2] * (n1 - n2)
        r = np.exp(-2j * np.pi * dtau * dnu / C_LIGHT)
        acc += np.exp(-2j * np.pi * dtau * nu0 / C_LIGHT) * (1 - r ** N) / (1 - r)
    return acc / (n_time * N)


def test_offset_source_average_is_dirichlet_closed_form():
    cad = small(n_ant=10, n_chan=24, n_time=4)
    uvw, freq = cad.uvw(), cad.freqs()
    l1, m1, l2, m2 = 0.12, -0.05, -0.02, 0.09
    src = np.array([[l1, m1, 1.0]])
    eye = np.zeros((1, cad.n_ant, 4), np.complex128)
    eye[..., 0] = eye[..., 3] = 1.0
    V = oracle.predict(uvw, freq, src, eye)
    A = oracle.rotate_average(uvw, freq, V, l2, m2)
    D = _dirichlet_average(uvw, freq, l1, m1, l2, m2)
    np.testing.assert_allclose(A[:, 0], D, rtol=0, atol=1e-11)
    np.testing.assert_allclose(A[:, 3], D, rtol=0, atol=1e-11)
    np.testing.assert_allclose(A[:, 1:3], 0, atol=1e-15)
    assert np.abs(D).min() < 0.9          # the case really decorrelates


# ---------------------------------------------------------------------------
# the solve


def test_identity_gains_one_source_recovered_exactly():
    cad = small(n_src=1)
    eye = np.zeros((1, cad.n_ant, 4), np.complex128)
    eye[..., 0] = eye[..., 3] = 1.0
    src = np.array([[0.1, 0.2, 5.0]])
    V = oracle.predict(cad.uvw(), cad.freqs(), src, eye)
    R, J, st = oracle.peel(cad.uvw(), cad.freqs(), V, src, n_iter=20)
    np.testing.assert_allclose(J, eye, atol=1e-13)
    assert st[0] == 0
    assert np.abs(R).max() < 1e-12 * np.abs(V).max()


def test_true_jones_one_source_recovered():
    """Noise-free single source: the gauge-invariant J_i J_j^H match the truth."""
    cad = small(n_ant=12, n_src=1)
    Jt = cad.jones()
    src = np.array([[-0.15, 0.07, 3.0]])
    V = oracle.predict(cad.uvw(), cad.freqs(), src, Jt)
    R, J, st = oracle.peel(cad.uvw(), cad.freqs(), V, src, n_iter=200)
    np.testing.assert_allclose(pair_products(J[0], cad.n_ant), pair_products(Jt[0], cad.n_ant),
                               rtol=0, atol=1e-10)
    assert st[0] == 0
    assert np.abs(R).max() < 1e-9


def test_als_first_iterations_closed_form():
    """From J = I one Jacobi sweep gives J_p = sum_{q!=p} A_pq / ((N-1) S); the
    second sweep is the textbook normal-equation solve, then the average."""
    rng = np.random.default_rng(7)
    n_ant, S = 6, 2.5
    nb = n_ant * (n_ant - 1) // 2
    avg = rng.normal(size=(nb, 4)) + 1j * rng.normal(size=(nb, 4))
    pairs = baseline_pairs(n_ant)
    full = np.zeros((n_ant, n_ant, 2, 2), np.complex128)
    for b, (i, j) in enumerate(pairs):
        full[i, j] = avg[b].reshape(2, 2)
        full[j, i] = herm(avg[b].reshape(2, 2))
    J1 = np.stack([sum(full[p, q] for q in range(n_ant) if q != p) / ((n_ant - 1) * S)
                   for p in range(n_ant)])
    got1, _, _ = oracle.als(avg, S, n_ant, n_iter=1)
    np.testing.assert_allclose(mats(got1), J1, rtol=1e-13, atol=1e-13)
    J2 = []
    for p in range(n_ant):
        A = sum(full[p, q] @ (S * J1[q]) for q in range(n_ant) if q != p)
        C = sum(S * S * herm(J1[q]) @ J1[q] for q in range(n_ant) if q != p)
        J2.append(np.linalg.solve(C.T, A.T).T)            # A C^-1
    J2 = 0.5 * (np.stack(J2) + J1)
    got2, _, _ = oracle.als(avg, S, n_ant, n_iter=2)
    np.testing.assert_allclose(mats(got2), J2, rtol=1e-12, atol=1e-12)


def test_als_invariant_under_antenna_relabelling():
    """Reversing the antenna order (which swaps which triangle is stored, so
    A_qp = A_pq^H is exercised) permutes the solution and nothing else."""
    rng = np.random.default_rng(3)
    n_ant, S = 7, 1.7
    Jt = np.eye(2)[None] + 0.1 * (rng.normal(size=(n_ant, 2, 2)) + 1j * rng.normal(size=(n_ant, 2, 2)))
    pairs = baseline_pairs(n_ant)
    avg = S * (Jt[pairs[:, 0]] @ herm(Jt[pairs[:, 1]])).reshape(-1, 4)
    avg += 0.01 * (rng.normal(size=avg.shape) + 1j * rng.normal(size=avg.shape))
    perm = np.arange(n_ant)[::-1]                        # new label of old antenna
    avg2 = np.zeros_like(avg)
    for b, (i, j) in enumerate(pairs):
        a, c = perm[i], perm[j]
        v = avg[b].reshape(2, 2)
        if a < c:
            avg2[oracle.baseline_index(n_ant, a, c)] = v.reshape(4)
        else:
            avg2[oracle.baseline_index(n_ant, c, a)] = herm(v).reshape(4)
    J1, _, _ = oracle.als(avg, S, n_ant, n_iter=30)
    J2, _, _ = oracle.als(avg2, S, n_ant, n_iter=30)
    np.testing.assert_allclose(J2[perm], J1, rtol=0, atol=1e-12)


def test_als_matches_brute_force_least_squares_4_antennas():
    """Four antennas, noisy data: the ALS fixed point reaches the global
    least-squares minimum found by Levenberg-Marquardt from 50 random starts."""
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)
    n_ant, S = 4, 3.0
    pairs = baseline_pairs(n_ant)
    Jt = np.eye(2)[None] + 0.2 * (rng.normal(size=(n_ant, 2, 2)) + 1j * rng.normal(size=(n_ant, 2, 2)))
    avg = S * (Jt[pairs[:, 0]] @ herm(Jt[pairs[:, 1]])).reshape(-1, 4)
    avg += 0.05 * (rng.normal(size=avg.shape) + 1j * rng.normal(size=avg.shape))

    def unpack(x):
        return (x[:16] + 1j * x[16:]).reshape(n_ant, 2, 2)

    def resid(x):
        J = unpack(x)
        r = (avg - S * (J[pairs[:, 0]] @ herm(J[pairs[:, 1]])).reshape(-1, 4)).ravel()
        return np.concatenate([r.real, r.imag])

    best = None
    for s in range(50):
        x0 = np.concatenate([np.eye(2).ravel().repeat(1)[None].repeat(n_ant, 0).ravel(),
                             np.zeros(16)]) + 0.5 * np.random.default_rng(100 + s).normal(size=32)
        r = opt.least_squares(resid, x0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                              max_nfev=20000)
        if best is None or r.cost < best.cost:
            best = r
    J, st, _ = oracle.als(avg, S, n_ant, n_iter=2000)
    x_als = np.concatenate([J.real.ravel(), J.imag.ravel()])
    cost_als = 0.5 * np.sum(resid(x_als) ** 2)
    assert cost_als <= best.cost * (1 + 1e-9) + 1e-14
    Jl = unpack(best.x)
    np.testing.assert_allclose(pair_products(J.reshape(n_ant, 4), n_ant),
                               Jl[pairs[:, 0]] @ herm(Jl[pairs[:, 1]]), atol=1e-6)


# ---------------------------------------------------------------------------
# the sequential peel


def test_sequential_subtraction_equals_dirichlet_correction():
    """The k-th averaged visibility of the sequential peel equals the plain
    average of the input in direction k minus, for every earlier source j,
    M_j(bl) times the closed-form Dirichlet average of exp(2 pi i (phi_k - phi_j))."""
    cad = small(n_ant=10, n_chan=32, n_time=3, n_src=3)
    uvw, freq = cad.uvw(), cad.freqs()
    src = cad.sources()
    V = oracle.predict(uvw, freq, src, cad.jones())
    R, J, st, avg = oracle.peel(uvw, freq, V, src, n_iter=20, keep_avg=True)
    for k in range(3):
        expect = oracle.rotate_average(uvw, freq, V, src[k, 0], src[k, 1])
        for j in range(k):
            M = src[j, 2] * pair_products(J[j], cad.n_ant).reshape(-1, 4)
            D = _dirichlet_average(uvw, freq, src[j, 0], src[j, 1], src[k, 0], src[k, 1])
            expect = expect - M * D[:, None]
        np.testing.assert_allclose(avg[k], expect, rtol=0, atol=1e-11)


def test_residual_noise_level_single_source():
    """One source plus noise: after the peel the residual carries the noise
    (E|n|^2 = 2 sigma^2 per complex element) less the few fitted parameters."""
    cad = small(n_ant=16, n_chan=32, n_time=4, n_src=1, noise_sigma=0.01)
    V = oracle.simulate(cad)
    R, J, st = oracle.peel(cad.uvw(), cad.freqs(), V, cad.sources(), n_iter=50)
    ratio = np.sqrt(np.mean(np.abs(R) ** 2)) / (cad.noise_sigma * math.sqrt(2))
    assert 0.95 < ratio < 1.02


# ---------------------------------------------------------------------------
# the adjoint


def _loss_params(cad):
    src = cad.perturbed_sources() if cad.pos_sigma_rad else cad.sources()
    return cad.uvw(), cad.freqs(), src, cad.jones()


def test_gradient_matches_central_differences():
    cad = small(n_ant=6, n_chan=10, n_time=2, n_src=3, pos_sigma_rad=1e-3)
    uvw, freq, src, J = _loss_params(cad)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    L, gJ, gl, gm, gS = oracle.loss_grad(uvw, freq, V, src, J)
    rng = np.random.default_rng(5)
    checks = []
    for _ in range(10):
        kind = rng.integers(0, 5)
        k = int(rng.integers(0, cad.n_src))
        if kind < 2:
            a, e = int(rng.integers(0, cad.n_ant)), int(rng.integers(0, 4))
            unit = 1.0 if kind == 0 else 1j
            analytic = gJ[k, a, e].real if kind == 0 else gJ[k, a, e].imag

            def f(h, k=k, a=a, e=e, unit=unit):
                J2 = J.copy()
                J2[k, a, e] += h * unit
                return oracle.loss_grad(uvw, freq, V, src, J2)[0]
            h = 1e-6
        else:
            col = {2: 0, 3: 1, 4: 2}[int(kind)]
            analytic = {0: gl, 1: gm, 2: gS}[col][k]

            def f(h, k=k, col=col):
                s2 = src.copy()
                s2[k, col] += h
                return oracle.loss_grad(uvw, freq, V, s2, J)[0]
            h = 1e-6 * max(1.0, abs(src[k, col]))
        fd = (f(h) - f(-h)) / (2 * h)
        checks.append((analytic, fd))
    for analytic, fd in checks:
        assert abs(analytic - fd) <= 1e-4 * max(abs(fd), 1e-3 * L)


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    cad = small(n_ant=4, n_chan=6, n_time=2, n_src=2, pos_sigma_rad=2e-3)
    uvw, freq, src, J = _loss_params(cad)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    L, gJ, gl, gm, gS = oracle.loss_grad(uvw, freq, V, src, J)

    pairs = baseline_pairs(cad.n_ant)
    Jt = torch.tensor(J, dtype=torch.complex128, requires_grad=True)
    lt = torch.tensor(src[:, 0], requires_grad=True)
    mt = torch.tensor(src[:, 1], requires_grad=True)
    St = torch.tensor(src[:, 2], requires_grad=True)
    U = torch.tensor(uvw)
    b = U[:, pairs[:, 0]] - U[:, pairs[:, 1]]                        # [t][bl][3]
    n = torch.sqrt(1 - lt ** 2 - mt ** 2)
    tau = (b[..., 0, None] * lt + b[..., 1, None] * mt + b[..., 2, None] * (n - 1))  # [t][bl][k]
    phi = tau[:, :, None, :] * torch.tensor(freq)[None, None, :, None] / C_LIGHT    # [t][bl][c][k]
    Jm = Jt.reshape(cad.n_src, cad.n_ant, 2, 2)
    M = St[:, None, None, None] * (Jm[:, pairs[:, 0]] @ Jm[:, pairs[:, 1]].conj().transpose(-1, -2))
    model = torch.einsum("kbxy,tbck->tbcxy", M.to(torch.complex128), torch.exp(-2j * np.pi * phi))
    R = torch.tensor(V).reshape(model.shape) - model
    loss = (R.abs() ** 2).sum()
    loss.backward()
    assert loss.item() == pytest.approx(L, rel=1e-12)
    np.testing.assert_allclose(Jt.grad.numpy(), gJ, rtol=1e-8, atol=1e-9 * abs(L))
    np.testing.assert_allclose(lt.grad.numpy(), gl, rtol=1e-8, atol=1e-9 * abs(L))
    np.testing.assert_allclose(mt.grad.numpy(), gm, rtol=1e-8, atol=1e-9 * abs(L))
    np.testing.assert_allclose(St.grad.numpy(), gS, rtol=1e-8, atol=1e-9 * abs(L))


def test_loss_is_zero_at_truth_without_noise():
    cad = small(n_ant=5, n_chan=8, n_time=2, n_src=2, noise_sigma=0.0)
    uvw, freq, src, J = cad.uvw(), cad.freqs(), cad.sources(), cad.jones()
    V = oracle.simulate(cad, noise=False)
    L, gJ, gl, gm, gS = oracle.loss_grad(uvw, freq, V, src, J)
    assert L < 1e-20
    assert np.abs(gJ).max() < 1e-9 and np.abs(gl).max() < 1e-6


# ---------------------------------------------------------------------------
# ionospheric position offsets (Gauss-Newton normal equations in l, m)


def _predict_shifted(cad, src, J, k, dl, dm, alpha, nu_ref):
    """Model with source k moved by (nu_ref/nu_c)^alpha (dl, dm) at each channel:
    one single-channel prediction per channel (independent of the offset code)."""
    freq = cad.freqs()
    parts = []
    for c in range(cad.n_chan):
        s = src.copy()
        sc = (nu_ref / freq[c]) ** alpha
        s[k, 0] += sc * dl
        s[k, 1] += sc * dm
        parts.append(oracle.predict(cad.uvw(), freq[c:c + 1], s, J))
    return np.concatenate(parts, axis=2)


def _richardson(f, h):
    """(4 D(h/2) - D(h)) / 3 with D the central difference: cancels the h^2 term."""
    d = lambda hh: (f(hh) - f(-hh)) / (2 * hh)
    return (4 * d(h / 2) - d(h)) / 3


@pytest.mark.parametrize("alpha", [0.0, 2.0])
def test_offset_normal_matrix_equals_jacobian_products(alpha):
    """H = 2 Re J^H J with J = d(model)/d(dl, dm) by extrapolated central
    differences of per-channel predictions (no use of the derivative formula)."""
    cad = small(n_ant=6, n_chan=10, n_time=2, n_src=2)
    src, J = cad.sources(), cad.jones()
    nu_ref = 160e6
    V = oracle.simulate(cad, noise=False)
    out, _ = oracle.offsets(cad.uvw(), cad.freqs(), V, src, J, alpha=alpha, nu_ref=nu_ref)
    for k in range(cad.n_src):
        jac = [_richardson(lambda h: _predict_shifted(cad, src[k:k + 1], J[k:k + 1], 0, h, 0.0, alpha,
                                                      nu_ref).ravel(), 1e-6),
               _richardson(lambda h: _predict_shifted(cad, src[k:k + 1], J[k:k + 1], 0, 0.0, h, alpha,
                                                      nu_ref).ravel(), 1e-6)]
        H = np.array([[2 * np.real(np.vdot(a, b)) for b in jac] for a in jac])
        np.testing.assert_allclose(out[k, [0, 1, 2]], [H[0, 0], H[0, 1], H[1, 1]], rtol=1e-6)


@pytest.mark.parametrize("alpha", [0.0, 2.0])
def test_offset_gradient_equals_loss_differences(alpha):
    """g = dL/d(dl, dm) of L = sum |V - model|^2 (numpy), all sources in the model."""
    cad = small(n_ant=6, n_chan=8, n_time=2, n_src=3, pos_sigma_rad=2e-4)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    src, J = cad.perturbed_sources(), cad.jones()
    nu_ref = 155e6
    out, _ = oracle.offsets(cad.uvw(), cad.freqs(), V, src, J, alpha=alpha, nu_ref=nu_ref)
    L0 = np.sum(np.abs(V - oracle.predict(cad.uvw(), cad.freqs(), src, J)) ** 2)
    assert out[0, 5] == pytest.approx(L0, rel=1e-12)
    for k in range(cad.n_src):
        for col, (ul, um) in ((3, (1, 0)), (4, (0, 1))):
            g = _richardson(lambda h: np.sum(np.abs(
                V - _predict_shifted(cad, src, J, k, ul * h, um * h, alpha, nu_ref)) ** 2), 1e-6)
            assert out[k, col] == pytest.approx(g, rel=1e-6, abs=1e-9 * abs(out[:, 3:5]).max())


def test_offset_gradient_without_frequency_law_equals_adjoint_gradient():
    """alpha = 0: the shift is a plain change of (l, m), so g is the adjoint's dL/dl, dL/dm."""
    cad = small(n_ant=7, n_chan=9, n_time=2, n_src=3, pos_sigma_rad=2e-4)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    src, J = cad.perturbed_sources(), cad.jones()
    out, _ = oracle.offsets(cad.uvw(), cad.freqs(), V, src, J, alpha=0.0)
    L, _, gl, gm, _ = oracle.loss_grad(cad.uvw(), cad.freqs(), V, src, J)
    np.testing.assert_allclose(out[:, 3], gl, rtol=1e-10)
    np.testing.assert_allclose(out[:, 4], gm, rtol=1e-10)
    assert out[0, 5] == pytest.approx(L, rel=1e-12)


def test_offset_is_zero_at_the_exact_model():
    cad = small(n_ant=6, n_chan=10, n_time=2, n_src=2)
    V = oracle.simulate(cad, noise=False)
    out, off = oracle.offsets(cad.uvw(), cad.freqs(), V, cad.sources(), cad.jones(), alpha=2.0)
    assert np.abs(off).max() < 1e-12
    assert out[0, 5] < 1e-20


@pytest.mark.parametrize("alpha", [0.0, 2.0])
def test_offset_recovers_a_shifted_source_with_known_gains(alpha):
    """A source observed 0.1 arcmin from its catalogue position (scaled by
    (nu_ref/nu)^alpha per channel): one Gauss-Newton step with the true gains
    returns the shift (first-order accurate: error of the order of the shift's
    phase, here < 1 %)."""
    cad = small(n_ant=16, n_chan=32, n_time=4, n_src=1, noise_sigma=0.0)
    cat = np.array([[0.12, -0.07, 4.0]])
    shift = np.array([2.0e-5, -3.0e-5])
    J = cad.jones()
    nu_ref = 150e6
    V = _predict_shifted(cad, cat, J, 0, shift[0], shift[1], alpha, nu_ref)
    _, off = oracle.offsets(cad.uvw(), cad.freqs(), V, cat, J, alpha=alpha, nu_ref=nu_ref)
    np.testing.assert_allclose(off[0], shift, rtol=1e-2)


def test_offset_statistics_add_over_channel_groups():
    """The six numbers are sums over channels: two halves of the band add up to
    the full band (what lets channel groups on different GPUs be combined)."""
    cad = small(n_ant=8, n_chan=12, n_time=2, n_src=3, pos_sigma_rad=2e-4)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    src, J, f = cad.perturbed_sources(), cad.jones(), cad.freqs()
    full, _ = oracle.offsets(cad.uvw(), f, V, src, J, alpha=2.0, nu_ref=150e6)
    lo, _ = oracle.offsets(cad.uvw(), f[:5], V[:, :, :5], src, J, alpha=2.0, nu_ref=150e6)
    hi, _ = oracle.offsets(cad.uvw(), f[5:], V[:, :, 5:], src, J, alpha=2.0, nu_ref=150e6)
    np.testing.assert_allclose(lo + hi, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
