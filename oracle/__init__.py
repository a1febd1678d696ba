"""ctypes binding of the FP64 CPU oracle (``rts_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use it; the product path never does.  It shares
no code with the CUDA library.  All arrays are numpy complex128 / float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rts_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i32 = ctypes.c_int32


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rts_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_n_baselines.restype = ctypes.c_int64
            L.orc_n_baselines.argtypes = [_i32]
            L.orc_baseline_index.restype = ctypes.c_int64
            L.orc_baseline_index.argtypes = [_i32, _i32, _i32]
            L.orc_baseline_antennas.argtypes = [_i32, _ip, _ip]
            L.orc_delay_m.restype = ctypes.c_double
            L.orc_delay_m.argtypes = [_dp, _i32, _i32, _i32, _i32, ctypes.c_double, ctypes.c_double]
            L.orc_phase_turns.restype = ctypes.c_double
            L.orc_phase_turns.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_predict.argtypes = [_i32, _i32, _i32, _dp, _dp, _i32, _dp, _dp, _dp, _i32]
            L.orc_rotate_average.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp,
                                             ctypes.c_double, ctypes.c_double, _dp]
            L.orc_als.restype = _i32
            L.orc_als.argtypes = [_i32, _dp, ctypes.c_double, _i32, _dp, _dp]
            L.orc_subtract.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _dp]
            L.orc_peel.restype = _i32
            L.orc_peel.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, _i32, _dp, _i32, _dp, _ip, _dp, _dp]
            L.orc_loss_grad.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, _i32, _dp, _dp,
                                        _dp, _dp, _dp, _dp, _dp]
            L.orc_offsets.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, _i32, _dp, _dp, ctypes.c_double,
                                      ctypes.c_double, _dp, _dp]
            L.orc_predict_taylor.argtypes = [_i32, _i32, _i32, _dp, _dp, _i32, _dp, _dp, _dp, _dp, _i32]
            L.orc_als_taylor.restype = _i32
            L.orc_als_taylor.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, _i32, _dp, _dp, _dp]
            L.orc_peel_taylor.restype = _i32
            L.orc_peel_taylor.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, _i32, _dp, _i32, _dp, _dp, _ip, _dp]
            L.orc_taylor_moments.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
            L.orc_taylor_rotation.restype = _i32
            L.orc_taylor_rotation.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, _dp, _dp, _dp, _dp]
            L.orc_taylor_dterm.argtypes = [_i32, _i32, _i32, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _dp]
            L.orc_grid.argtypes = [_i32, ctypes.c_double, _dp, _i32, _i32, _i32, _dp, _dp, _dp]
            L.orc_integrate.argtypes = [_i32, ctypes.c_int64, _i32, _ip, _i32, _dp, _dp]
            L.orc_num_threads.restype = _i32
            L.orc_set_num_threads.argtypes = [_i32]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's later calls (results do not depend on it)."""
    lib().orc_set_num_threads(int(n))


def n_baselines(n_ant: int) -> int:
    return int(lib().orc_n_baselines(n_ant))


def baseline_index(n_ant: int, i: int, j: int) -> int:
    return int(lib().orc_baseline_index(n_ant, i, j))


def baseline_antennas(n_ant: int):
    nb = n_baselines(n_ant)
    ai = np.zeros(max(nb, 1), np.int32)
    aj = np.zeros(max(nb, 1), np.int32)
    lib().orc_baseline_antennas(n_ant, ai.ctypes.data_as(_ip), aj.ctypes.data_as(_ip))
    return ai[:nb], aj[:nb]


def delay_m(uvw, t, i, j, l, m) -> float:
    uvw = _f64(uvw)
    return float(lib().orc_delay_m(_d(uvw), uvw.shape[1], t, i, j, l, m))


def phase_turns(tau_m, freq_hz) -> float:
    return float(lib().orc_phase_turns(tau_m, freq_hz))


def predict(uvw, freq, lmS, jones, vis=None):
    """[n_time][n_bl][n_chan][4] complex128 model visibilities (+= vis if given)."""
    uvw, freq, lmS = _f64(uvw), _f64(freq), _f64(lmS)
    jones = _f64(jones, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    n_chan, n_src = freq.shape[0], lmS.shape[0]
    nb = n_ant * (n_ant - 1) // 2
    acc = vis is not None
    out = _f64(vis, np.complex128).copy() if acc else np.zeros((n_time, nb, n_chan, 4), np.complex128)
    lib().orc_predict(n_ant, n_chan, n_time, _d(uvw), _d(freq), n_src, _d(lmS),
                      _d(jones), _d(out), int(acc))
    return out


def rotate_average(uvw, freq, vis, l, m):
    uvw, freq = _f64(uvw), _f64(freq)
    vis = _f64(vis, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    nb = n_ant * (n_ant - 1) // 2
    avg = np.zeros((nb, 4), np.complex128)
    lib().orc_rotate_average(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(vis),
                             float(l), float(m), _d(avg))
    return avg


def als(avg, S, n_ant, n_iter=20):
    """Jones [n_ant][4] from one source's averaged visibilities; (J, status, rel)."""
    avg = _f64(avg, np.complex128)
    J = np.zeros((n_ant, 4), np.complex128)
    rel = ctypes.c_double(0.0)
    st = lib().orc_als(n_ant, _d(avg), float(S), n_iter, _d(J), ctypes.byref(rel))
    return J, int(st), rel.value


def subtract(uvw, freq, vis, l, m, S, jones_k):
    uvw, freq = _f64(uvw), _f64(freq)
    out = _f64(vis, np.complex128).copy()
    J = _f64(jones_k, np.complex128)
    lib().orc_subtract(uvw.shape[1], freq.shape[0], uvw.shape[0], _d(uvw), _d(freq),
                       _d(out), float(l), float(m), float(S), _d(J))
    return out


def peel(uvw, freq, vis, lmS, n_iter=20, keep_avg=False, with_rel=False):
    """Sequential peel.  Returns (residual, jones [n_src][n_ant][4], status[, avg][, rel]),
    rel [n_src] = each source's last relative change ||J_n - J_(n-1)||_F / ||J_n||_F."""
    uvw, freq, lmS = _f64(uvw), _f64(freq), _f64(lmS)
    R = _f64(vis, np.complex128).copy()
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    n_src = lmS.shape[0]
    nb = n_ant * (n_ant - 1) // 2
    J = np.zeros((n_src, n_ant, 4), np.complex128)
    st = np.zeros(max(n_src, 1), np.int32)
    avg = np.zeros((n_src, nb, 4), np.complex128) if keep_avg else None
    rel = np.zeros(max(n_src, 1))
    lib().orc_peel(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(R), n_src, _d(lmS),
                   n_iter, _d(J), st.ctypes.data_as(_ip), _d(avg) if keep_avg else None, _d(rel))
    out = (R, J, st[:n_src])
    if keep_avg:
        out += (avg,)
    if with_rel:
        out += (rel[:n_src],)
    return out


def loss_grad(uvw, freq, vis, lmS, jones):
    """(loss, dL/dJ [n_src][n_ant][4] complex, dL/dl, dL/dm, dL/dS)."""
    uvw, freq, lmS = _f64(uvw), _f64(freq), _f64(lmS)
    vis = _f64(vis, np.complex128)
    jones = _f64(jones, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    n_src = lmS.shape[0]
    loss = ctypes.c_double(0.0)
    gJ = np.zeros((n_src, n_ant, 4), np.complex128)
    gl, gm, gS = (np.zeros(max(n_src, 1)) for _ in range(3))
    lib().orc_loss_grad(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(vis), n_src,
                        _d(lmS), _d(jones), ctypes.byref(loss), _d(gJ), _d(gl), _d(gm), _d(gS))
    return loss.value, gJ, gl[:n_src], gm[:n_src], gS[:n_src]


def offsets(uvw, freq, vis, lmS, jones, alpha=0.0, nu_ref=None):
    """Position-offset normal equations per source, shift (nu_ref/nu)^alpha (dl, dm).
    Returns (out [n_src][6] = H_ll, H_lm, H_mm, dL/dl, dL/dm, L; offsets [n_src][2])."""
    uvw, freq, lmS = _f64(uvw), _f64(freq), _f64(lmS)
    vis = _f64(vis, np.complex128)
    jones = _f64(jones, np.complex128)
    nu_ref = float(np.mean(freq)) if nu_ref is None else float(nu_ref)
    n_src = lmS.shape[0]
    out = np.zeros((max(n_src, 1), 6))
    off = np.zeros((max(n_src, 1), 2))
    lib().orc_offsets(uvw.shape[1], freq.shape[0], uvw.shape[0], _d(uvw), _d(freq), _d(vis), n_src,
                      _d(lmS), _d(jones), float(alpha), nu_ref, _d(out), _d(off))
    return out[:n_src], off[:n_src]


def predict_taylor(uvw, freq, lmS, gain, slope, vis=None):
    """Model with gains linear in frequency, J_p(c) = G_p + x_c H_p,
    x_c = (nu_c - nu_mid) / (n_chan dnu): [n_time][n_bl][n_chan][4] complex128."""
    uvw, freq, lmS = _f64(uvw), _f64(freq), _f64(lmS)
    gain, slope = _f64(gain, np.complex128), _f64(slope, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    n_chan, n_src = freq.shape[0], lmS.shape[0]
    nb = n_ant * (n_ant - 1) // 2
    acc = vis is not None
    out = _f64(vis, np.complex128).copy() if acc else np.zeros((n_time, nb, n_chan, 4), np.complex128)
    lib().orc_predict_taylor(n_ant, n_chan, n_time, _d(uvw), _d(freq), n_src, _d(lmS),
                             _d(gain), _d(slope), _d(out), int(acc))
    return out


def als_taylor(uvw, freq, vis, l, m, S, n_iter=20):
    """Frequency-linear gains of one source from the residual cube: (G, H, status, rel)."""
    uvw, freq = _f64(uvw), _f64(freq)
    vis = _f64(vis, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    G = np.zeros((n_ant, 4), np.complex128)
    H = np.zeros((n_ant, 4), np.complex128)
    rel = ctypes.c_double(0.0)
    st = lib().orc_als_taylor(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(vis), float(l),
                              float(m), float(S), n_iter, _d(G), _d(H), ctypes.byref(rel))
    return G, H, int(st), rel.value


def peel_taylor(uvw, freq, vis, lmS, n_iter=20, with_rel=False):
    """Sequential peel with gains linear in frequency: (residual, G, H, status[, rel]),
    rel [n_src] = each source's last relative change ||X_n - X_(n-1)||_F / ||X_n||_F."""
    uvw, freq, lmS = _f64(uvw), _f64(freq), _f64(lmS)
    R = _f64(vis, np.complex128).copy()
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    n_src = lmS.shape[0]
    G = np.zeros((n_src, n_ant, 4), np.complex128)
    H = np.zeros((n_src, n_ant, 4), np.complex128)
    st = np.zeros(max(n_src, 1), np.int32)
    rel = np.zeros(max(n_src, 1))
    lib().orc_peel_taylor(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(R), n_src, _d(lmS),
                          n_iter, _d(G), _d(H), st.ctypes.data_as(_ip), _d(rel))
    out = (R, G, H, st[:n_src])
    return out + (rel[:n_src],) if with_rel else out


def taylor_rotation(uvw, freq, vis, l, m, S, gain, slope):
    """One common slope-rotation Newton step at the iterate (gain, slope)
    [n_ant][4]: (new slope, taken, g [4], h [4][4])."""
    uvw, freq = _f64(uvw), _f64(freq)
    vis = _f64(vis, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    G = np.ascontiguousarray(np.asarray(gain, np.complex128).reshape(n_ant, 4))
    H = np.ascontiguousarray(np.asarray(slope, np.complex128).reshape(n_ant, 4)).copy()
    g = np.zeros(4)
    h = np.zeros(16)
    taken = lib().orc_taylor_rotation(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(vis), float(l),
                                      float(m), float(S), _d(G), _d(H), _d(g), _d(h))
    return H, bool(taken), g, h.reshape(4, 4)


def taylor_moments(uvw, freq, vis, l, m):
    """[3][n_bl][4]: mean_{t,c} x_c^n R exp(+2 pi i phi) of the cube in direction (l, m)."""
    uvw, freq = _f64(uvw), _f64(freq)
    vis = _f64(vis, np.complex128)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    nb = n_ant * (n_ant - 1) // 2
    out = np.zeros((3, nb, 4), np.complex128)
    lib().orc_taylor_moments(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), _d(vis), float(l), float(m), _d(out))
    return out


def taylor_dterm(uvw, freq, lj, mj, lk, mk):
    """[5][n_bl]: mean_{t,c} x_c^p exp(2 pi i (phi_k - phi_j)), p = 0..4."""
    uvw, freq = _f64(uvw), _f64(freq)
    n_time, n_ant = uvw.shape[0], uvw.shape[1]
    nb = n_ant * (n_ant - 1) // 2
    out = np.zeros((5, nb), np.complex128)
    lib().orc_taylor_dterm(n_ant, freq.shape[0], n_time, _d(uvw), _d(freq), float(lj), float(mj), float(lk),
                           float(mk), _d(out))
    return out


def grid(n_pix, r_max, gcf, xy, vis):
    """Gridded visibilities [n_pol][n_pix][n_pix] complex128: each visibility i at
    pixel coordinates xy[i] adds f(r) vis[i] to every pixel centre within r < r_max,
    f the linear interpolation of the radial table gcf on [0, r_max]."""
    gcf = _f64(gcf)
    xy = _f64(xy).reshape(-1, 2)
    vis = _f64(vis, np.complex128)
    vis = vis.reshape(vis.shape[0], -1)
    n_vis, n_pol = vis.shape
    out = np.zeros((n_pol, n_pix, n_pix), np.complex128)
    lib().orc_grid(int(n_pix), float(r_max), _d(gcf), gcf.shape[0], n_vis, n_pol, _d(xy), _d(vis), _d(out))
    return out


def integrate(fine, lengths, n_slot):
    """Per-baseline time averaging: fine [n_fine][n_bl][n_chan][4] complex, lengths [n_bl]
    (fine samples per output, dividing n_fine) -> [n_slot][n_bl][n_chan][4]; slot s of
    baseline b is the mean of fine samples s L_b .. (s+1) L_b - 1, zero past n_fine / L_b."""
    fine = _f64(fine, np.complex128)
    n_fine, n_bl, n_chan = fine.shape[0], fine.shape[1], fine.shape[2]
    L = np.ascontiguousarray(lengths, dtype=np.int32)
    out = np.zeros((n_slot, n_bl, n_chan, 4), np.complex128)
    lib().orc_integrate(n_fine, n_bl, n_chan, L.ctypes.data_as(_ip), n_slot, _d(fine), _d(out))
    return out


def simulate(cad, noise=True, sources=None, jones=None):
    """Visibility cube of a synthetic cadence: oracle prediction + generator noise."""
    src = cad.sources() if sources is None else sources
    J = cad.jones() if jones is None else jones
    V = predict(cad.uvw(), cad.freqs(), src, J)
    if noise and cad.noise_sigma > 0:
        V += cad.noise().reshape(V.shape)
    return V
