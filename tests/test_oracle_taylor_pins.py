"""Pins of the oracle's gains Taylor-expanded in frequency (Section 3.1: the
gain of a tile may be Taylor-expanded in frequency when consecutive channels
are combined; reading R16: J_p(c) = G_p + x_c H_p, x_c the channel's offset
from the band centre in band widths).

Each test ties the oracle's Taylor functions to something outside their code:
the already-pinned constant-gain oracle applied channel by channel, exact
recovery of noise-free frequency-linear gains, the closed form of the first
Jacobi sweep from G = I, H = 0, and the global least-squares minimum found by
Levenberg-Marquardt from many starts.
"""
import numpy as np
import pytest

import oracle
from synth import Cadence, baseline_pairs


def mats(J):
    return np.asarray(J).reshape(*np.shape(J)[:-1], 2, 2)


def herm(a):
    return np.conj(np.swapaxes(a, -1, -2))


def xc(freq):
    """Offset of each channel from the band centre in band widths (numpy, from the definition)."""
    f = np.asarray(freq, np.float64)
    dnu = (f[-1] - f[0]) / (len(f) - 1)
    return (f - 0.5 * (f[0] + f[-1])) / (len(f) * dnu)


def channel_products(G, H, x, n_ant):
    """(G_i + x H_i)(G_j + x H_j)^H per baseline at offset x."""
    pairs = baseline_pairs(n_ant)
    J = mats(G) + x * mats(H)
    return J[pairs[:, 0]] @ herm(J[pairs[:, 1]])


def small(n_ant=6, n_chan=9, n_time=2, n_src=1, seed=5151):
    return Cadence(n_ant, n_chan, n_time, n_src, freq0_hz=150e6, seed=seed)


def test_taylor_prediction_is_the_constant_gain_prediction_channel_by_channel():
    cad = small(n_src=3)
    G, H = cad.jones(), cad.jones_slope()
    src, freq = cad.sources(), cad.freqs()
    V = oracle.predict_taylor(cad.uvw(), freq, src, G, H)
    x = xc(freq)
    assert abs(x[len(x) // 2]) < 1e-15 and np.isclose(x[-1] - x[0], (len(x) - 1) / len(x))
    for c in range(cad.n_chan):
        Vc = oracle.predict(cad.uvw(), freq[c:c + 1], src, G + x[c] * H)
        np.testing.assert_allclose(V[:, :, c:c + 1], Vc, rtol=0, atol=1e-13)


def test_taylor_peel_recovers_frequency_linear_gains():
    """Noise-free single source with gains linear in frequency: the fitted model
    (G_i + x H_i)(G_j + x H_j)^H equals the truth at every channel and the
    residual vanishes.  A rotation common to all slopes, H_p -> H_p + i G_p K,
    changes the model only at second order in x, so the Jacobi sweeps alone
    took 8000 sweeps here; with the slope-rotation Newton step after each sweep
    (reading R27) 60 sweeps recover the truth to 1e-9."""
    cad = small(n_ant=7, n_chan=11, n_time=3)
    Gt, Ht = cad.jones(), cad.jones_slope()
    src = np.array([[0.12, -0.05, 4.0]])
    V = oracle.predict_taylor(cad.uvw(), cad.freqs(), src, Gt, Ht)
    R, G, H, st = oracle.peel_taylor(cad.uvw(), cad.freqs(), V, src, n_iter=60)
    for x in xc(cad.freqs()):
        np.testing.assert_allclose(channel_products(G[0], H[0], x, cad.n_ant),
                                   channel_products(Gt[0], Ht[0], x, cad.n_ant), rtol=0, atol=1e-9)
    assert st[0] == 0
    assert np.abs(R).max() < 1e-9 * np.abs(V).max()


def test_taylor_peel_of_constant_gains_has_no_slope():
    """Gains constant over the band: the Taylor fit reproduces the constant-gain
    products and its slope terms vanish."""
    cad = small(n_ant=7, n_chan=8, n_time=2)
    Jt = cad.jones()
    src = np.array([[-0.2, 0.1, 2.5]])
    V = oracle.predict(cad.uvw(), cad.freqs(), src, Jt)
    R, G, H, st = oracle.peel_taylor(cad.uvw(), cad.freqs(), V, src, n_iter=400)
    pairs = baseline_pairs(cad.n_ant)
    Gm, Hm, Jm = mats(G[0]), mats(H[0]), mats(Jt[0])
    np.testing.assert_allclose(Gm[pairs[:, 0]] @ herm(Gm[pairs[:, 1]]),
                               Jm[pairs[:, 0]] @ herm(Jm[pairs[:, 1]]), rtol=0, atol=1e-9)
    slope = Gm[pairs[:, 0]] @ herm(Hm[pairs[:, 1]]) + Hm[pairs[:, 0]] @ herm(Gm[pairs[:, 1]])
    assert np.abs(slope).max() < 1e-9
    assert np.abs(R).max() < 1e-9 * np.abs(V).max()


def test_taylor_first_sweep_closed_form():
    """From G = I, H = 0 (and channels symmetric about the centre, so sum_c x_c = 0)
    the normal matrix is block diagonal and one sweep gives
      G_p = sum_q mean_{t,c} R~_pq / ((N-1) S),
      H_p = sum_q mean_{t,c} x_c R~_pq / ((N-1) S mean_c x_c^2),
    R~ the residual rotated to the source; the means come from the pinned
    constant-gain rotate + average applied to R and to x_c R."""
    cad = small(n_ant=5, n_chan=10, n_time=2, n_src=2)
    V = oracle.simulate(cad)
    l, m, S = 0.07, -0.11, 3.3
    x = xc(cad.freqs())
    A0 = oracle.rotate_average(cad.uvw(), cad.freqs(), V, l, m)
    A1 = oracle.rotate_average(cad.uvw(), cad.freqs(), V * x[None, None, :, None], l, m)
    n = cad.n_ant
    pairs = baseline_pairs(n)
    full0 = np.zeros((n, n, 2, 2), np.complex128)
    full1 = np.zeros((n, n, 2, 2), np.complex128)
    for b, (i, j) in enumerate(pairs):
        full0[i, j], full0[j, i] = A0[b].reshape(2, 2), herm(A0[b].reshape(2, 2))
        full1[i, j], full1[j, i] = A1[b].reshape(2, 2), herm(A1[b].reshape(2, 2))
    G1 = np.stack([sum(full0[p, q] for q in range(n) if q != p) for p in range(n)]) / ((n - 1) * S)
    H1 = np.stack([sum(full1[p, q] for q in range(n) if q != p) for p in range(n)]) / (
        (n - 1) * S * np.mean(x ** 2))
    G, H, _, _ = oracle.als_taylor(cad.uvw(), cad.freqs(), V, l, m, S, n_iter=1)
    np.testing.assert_allclose(mats(G), G1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(mats(H), H1, rtol=1e-12, atol=1e-12)


def test_taylor_als_matches_brute_force_least_squares():
    """Four antennas, a source at the phase centre (no rotation), noisy data: the
    Taylor ALS (Jacobi sweeps and slope-rotation steps) converges within 200
    sweeps to the least-squares minimum over all (G, H) found by
    Levenberg-Marquardt from 30 starts."""
    opt = pytest.importorskip("scipy.optimize")
    cad = Cadence(4, 6, 1, 1, freq0_hz=150e6, noise_sigma=0.05, seed=7373)
    S = 3.0
    src = np.array([[0.0, 0.0, S]])
    V = oracle.predict_taylor(cad.uvw(), cad.freqs(), src, cad.jones(), cad.jones_slope(0.4))
    V = V + cad.noise().reshape(V.shape)
    x = xc(cad.freqs())
    n = cad.n_ant
    pairs = baseline_pairs(n)
    data = V[0]                                         # [bl][c][4], no rotation at l = m = 0

    def unpack(p):                                      # 8 n complex = 16 n reals
        z = p[:8 * n] + 1j * p[8 * n:]
        return z[:4 * n].reshape(n, 2, 2), z[4 * n:].reshape(n, 2, 2)

    def resid(p):
        G, H = unpack(p)
        out = []
        for c in range(cad.n_chan):
            J = G + x[c] * H
            M = S * (J[pairs[:, 0]] @ herm(J[pairs[:, 1]])).reshape(-1, 4)
            out.append((data[:, c] - M).ravel())
        r = np.concatenate(out)
        return np.concatenate([r.real, r.imag])

    eye = np.concatenate([np.tile(np.eye(2).ravel(), n), np.zeros(4 * n)])
    best = None
    for s in range(30):
        p0 = np.concatenate([eye, np.zeros(8 * n)]) + 0.3 * np.random.default_rng(900 + s).normal(size=16 * n)
        r = opt.least_squares(resid, p0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=40000)
        if best is None or r.cost < best.cost:
            best = r
    G, H, st, _ = oracle.als_taylor(cad.uvw(), cad.freqs(), V, 0.0, 0.0, S, n_iter=200)
    assert st == 0
    p_als = np.concatenate([np.concatenate([G.ravel(), H.ravel()]).real,
                            np.concatenate([G.ravel(), H.ravel()]).imag])
    cost_als = 0.5 * np.sum(resid(p_als) ** 2)
    assert cost_als <= best.cost * (1 + 1e-9) + 1e-14
    Gl, Hl = unpack(best.x)
    for xx in x:
        np.testing.assert_allclose(channel_products(G, H, xx, n),
                                   channel_products(Gl.reshape(n, 4), Hl.reshape(n, 4), xx, n), atol=1e-6)


def test_taylor_moments_and_pair_terms_reduce_to_pinned_averages():
    """The Taylor moments are the pinned constant-gain rotate + average of x_c^n V,
    and the pair terms D^(p)_jk the average in direction k of x_c^p times a unit
    point source at j (identity gains, S = 1)."""
    cad = small(n_ant=5, n_chan=10, n_time=2, n_src=2)
    V = oracle.simulate(cad)
    x = xc(cad.freqs())
    l, m = 0.05, -0.08
    M = oracle.taylor_moments(cad.uvw(), cad.freqs(), V, l, m)
    for n in range(3):
        ref = oracle.rotate_average(cad.uvw(), cad.freqs(), V * (x ** n)[None, None, :, None], l, m)
        np.testing.assert_allclose(M[n], ref, rtol=0, atol=1e-13)
    lj, mj, lk, mk = -0.1, 0.12, 0.07, 0.02
    eye = np.zeros((1, cad.n_ant, 4), np.complex128)
    eye[..., 0] = eye[..., 3] = 1.0
    unit = oracle.predict(cad.uvw(), cad.freqs(), np.array([[lj, mj, 1.0]]), eye)
    D = oracle.taylor_dterm(cad.uvw(), cad.freqs(), lj, mj, lk, mk)
    for p in range(5):
        ref = oracle.rotate_average(cad.uvw(), cad.freqs(), unit * (x ** p)[None, None, :, None], lk, mk)
        np.testing.assert_allclose(D[p], ref[:, 0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(ref[:, 1], 0, atol=1e-15)


def test_sequential_taylor_moments_equal_pair_term_corrections():
    """The identity a blocked Taylor schedule rests on: the moments of source k
    over the residual of the earlier sources of its block equal the plain
    moments minus sum_j sum_m P_m,j D^(n+m)_jk, with P_0 = S G_i G_j^H,
    P_1 = S (G_i H_j^H + H_i G_j^H), P_2 = S H_i H_j^H per baseline."""
    cad = small(n_ant=6, n_chan=12, n_time=2, n_src=4)
    src, G, H = cad.sources(), cad.jones(), cad.jones_slope()
    V = oracle.predict_taylor(cad.uvw(), cad.freqs(), src, G, H) + cad.noise().reshape(cad.n_time, cad.n_bl, cad.n_chan, 4)
    pairs = baseline_pairs(cad.n_ant)
    herm_ = lambda a: np.conj(np.swapaxes(a, -1, -2))
    for k in range(1, cad.n_src):
        l, m, _ = src[k]
        neg = src[:k].copy()
        neg[:, 2] *= -1.0
        R = oracle.predict_taylor(cad.uvw(), cad.freqs(), neg, G[:k], H[:k], vis=V)
        got = oracle.taylor_moments(cad.uvw(), cad.freqs(), R, l, m)
        ref = oracle.taylor_moments(cad.uvw(), cad.freqs(), V, l, m)
        for j in range(k):
            Gm, Hm, S = mats(G[j]), mats(H[j]), src[j, 2]
            P = [S * Gm[pairs[:, 0]] @ herm_(Gm[pairs[:, 1]]),
                 S * (Gm[pairs[:, 0]] @ herm_(Hm[pairs[:, 1]]) + Hm[pairs[:, 0]] @ herm_(Gm[pairs[:, 1]])),
                 S * Hm[pairs[:, 0]] @ herm_(Hm[pairs[:, 1]])]
            D = oracle.taylor_dterm(cad.uvw(), cad.freqs(), src[j, 0], src[j, 1], l, m)
            for n in range(3):
                for mm in range(3):
                    ref[n] -= P[mm].reshape(-1, 4) * D[n + mm][:, None]
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_slope_rotation_step_is_the_newton_step_of_the_cost():
    """The slope-rotation step (reading R27): its gradient g and Hessian h are
    the derivatives at K = 0 of the cost along H_p -> H_p + i G_p K (K Hermitian,
    K = sum_a k_a B_a), taken here by central differences of the plain cost
    sum |V - predict_taylor|^2 over every sample; the step -h^-1 g lowers the
    cost and is applied to every slope."""
    cad = small(n_ant=6, n_chan=9, n_time=2)
    l, m, S = 0.09, -0.04, 3.0
    Gt, Ht = cad.jones(), cad.jones_slope(0.3)
    V = oracle.predict_taylor(cad.uvw(), cad.freqs(), np.array([[l, m, S]]), Gt, Ht)
    V = V + cad.noise().reshape(V.shape)
    # an iterate off the optimum: a few sweeps of the solve
    G, H, _, _ = oracle.als_taylor(cad.uvw(), cad.freqs(), V, l, m, S, n_iter=3)
    B = [np.array([[1, 0], [0, 0]]), np.array([[0, 0], [0, 1]]), np.array([[0, 1], [1, 0]]),
         np.array([[0, -1j], [1j, 0]])]

    def cost(k):
        K = sum(c * b for c, b in zip(k, B))
        Hk = (mats(H) + 1j * mats(G) @ K).reshape(-1, 4)
        P = oracle.predict_taylor(cad.uvw(), cad.freqs(), np.array([[l, m, S]]), G[None], Hk[None])
        return float(np.sum(np.abs(V - P) ** 2))

    Hn, taken, g, h = oracle.taylor_rotation(cad.uvw(), cad.freqs(), V, l, m, S, G, H)
    eps = 1e-4
    e = np.eye(4)
    g_fd = np.array([(cost(eps * e[a]) - cost(-eps * e[a])) / (2 * eps) for a in range(4)])
    h_fd = np.array([[(cost(eps * (e[a] + e[b])) - cost(eps * (e[a] - e[b])) - cost(eps * (e[b] - e[a]))
                       + cost(-eps * (e[a] + e[b]))) / (4 * eps * eps) for b in range(4)] for a in range(4)])
    np.testing.assert_allclose(g, g_fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())
    np.testing.assert_allclose(h, h_fd, rtol=1e-4, atol=1e-5 * np.abs(h).max())
    assert taken
    k = -np.linalg.solve(h, g)
    np.testing.assert_allclose(Hn, (mats(H) + 1j * mats(G) @ sum(c * b for c, b in zip(k, B))).reshape(-1, 4),
                               rtol=0, atol=1e-12)
    assert cost(k) < cost(np.zeros(4))
