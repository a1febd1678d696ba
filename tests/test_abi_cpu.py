"""Host-side tests of the C ABI: no GPU needed.

The library loads, exports every symbol include/*.h declares (the peel, the
gridder, the integrator), and rejects bad configurations on the host before
touching CUDA.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_1003_5575_gb300 import build, _abi
    build.build()
    return _abi


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rts_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("rts_peel_init", "rts_peel_cadence", "rts_peel_grad", "rts_peel_destroy",
              "rts_peel_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(abi):
    L = abi.lib()
    for name in sorted(declared_symbols()):
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
    assert set(abi.EXPORTS) == declared_symbols()


def _cfg(abi, n_ant=8, n_chan=16, n_time=2, n_iter=20, precision=0, max_sources=4, freq=None, uvw=None,
         **fields):
    uvw = np.zeros((n_time, max(n_ant, 1), 3)) if uvw is None else uvw
    freq = 150e6 + 40e3 * np.arange(max(n_chan, 1)) if freq is None else freq
    cfg = abi.rts_peel_config()
    cfg.n_ant, cfg.n_chan, cfg.n_time = n_ant, n_chan, n_time
    cfg.n_iter, cfg.precision, cfg.max_sources = n_iter, precision, max_sources
    dp = ctypes.POINTER(ctypes.c_double)
    cfg.uvw = uvw.ctypes.data_as(dp) if uvw is not False else None
    cfg.freq_hz = freq.ctypes.data_as(dp)
    for k, v in fields.items():
        setattr(cfg, k, v)
    return cfg, (uvw, freq)


@pytest.mark.parametrize("kw,needle", [
    (dict(n_ant=1), "n_ant"),
    (dict(n_chan=0), "n_chan"),
    (dict(n_time=0), "n_time"),
    (dict(n_iter=0), "n_iter"),
    (dict(precision=7), "precision"),
    (dict(max_sources=0), "max_sources"),
    (dict(freq=150e6 + 40e3 * np.arange(16) ** 1.01), "uniformly"),
    (dict(freq=np.full(16, -1.0)), "frequencies"),
    (dict(uvw=np.full((2, 8, 3), np.nan)), "non-finite"),
    (dict(sources_per_pass=3), "sources_per_pass"),
    (dict(sources_per_pass=64, block_kernel=5), "block_kernel"),
    (dict(sources_per_pass=64, solve_kernel=7), "solve_kernel"),
    (dict(grad_kernel=2), "grad_kernel"),
])
def test_init_rejects_bad_config_on_host(abi, kw, needle):
    cfg, keep = _cfg(abi, **kw)
    h = ctypes.c_void_p()
    rc = abi.lib().rts_peel_init(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == abi.RTS_EINVAL
    assert not h.value
    assert needle in abi.rts_peel_last_error(None)


def test_null_handle_is_rejected(abi):
    assert abi.lib().rts_peel_cadence(None, None, None, 0, None, None, None, None) == abi.RTS_EINVAL
    assert abi.lib().rts_peel_grad(None, None, 0, None, None, None, None, None, None) == abi.RTS_EINVAL
    assert abi.lib().rts_peel_kernels(None, None, None) == abi.RTS_EINVAL
    assert abi.lib().rts_peel_cadence_taylor(None, None, None, 0, None, None, None, None, None) == abi.RTS_EINVAL
    assert abi.lib().rts_fp64_rate(None) == abi.RTS_EINVAL
    out = ctypes.c_int32()
    assert abi.lib().rts_barrier_selftest(0, 0, 1, ctypes.byref(out)) == abi.RTS_EINVAL
    assert abi.lib().rts_barrier_selftest(8, 2, 1, ctypes.byref(out)) == abi.RTS_EINVAL
    abi.lib().rts_peel_destroy(None)


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1003_5575_gb300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _abi.lib()


# ---- gridder and integrator: host-side validation (no CUDA call is reached) ----

def _grid_cfg(abi, **kw):
    gcf = np.asarray(kw.pop("gcf", np.linspace(1.0, 0.0, 33)), np.float64)
    cfg = abi.rts_grid_config()
    cfg.n_pix, cfg.bin, cfg.r_max = kw.get("n_pix", 64), kw.get("bin", 8), kw.get("r_max", 4.0)
    cfg.gcf = gcf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.n_tab = kw.get("n_tab", len(gcf))
    cfg.n_pol, cfg.max_vis = kw.get("n_pol", 4), kw.get("max_vis", 100)
    return cfg, gcf


@pytest.mark.parametrize("kw,needle", [
    (dict(n_pix=0), "n_pix"),
    (dict(r_max=-1.0), "r_max"),
    (dict(r_max=float("nan")), "r_max"),
    (dict(bin=3, r_max=4.0), "bin"),
    (dict(bin=41, r_max=4.0), "bin"),
    (dict(n_pix=16384, bin=8), "8192"),
    (dict(n_tab=1), "n_tab"),
    (dict(gcf=np.array([1.0, np.nan, 0.0])), "non-finite"),
    (dict(n_pol=5), "n_pol"),
    (dict(max_vis=0), "max_vis"),
])
def test_grid_init_rejects_bad_config_on_host(abi, kw, needle):
    cfg, keep = _grid_cfg(abi, **kw)
    h = ctypes.c_void_p()
    assert abi.lib().rts_grid_init(ctypes.byref(cfg), ctypes.byref(h)) == abi.RTS_EINVAL
    assert not h.value
    assert needle in abi.rts_grid_last_error(None)


def test_grid_and_integrator_null_handles(abi):
    L = abi.lib()
    assert L.rts_grid_run(None, None, None, 0, None, None) == abi.RTS_EINVAL
    assert L.rts_grid_last_ms(None, None, None) == abi.RTS_EINVAL
    assert L.rts_integrate_run(None, None, None, None) == abi.RTS_EINVAL
    L.rts_grid_destroy(None)
    L.rts_integrate_destroy(None)


def test_integration_lengths_on_host(abi):
    rng = np.random.default_rng(5)
    pos = rng.uniform(-800.0, 800.0, size=(9, 3))
    cut = np.array([500.0, 1000.0])
    lf = np.array([16, 8, 4], np.int32)
    out = np.zeros(36, np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = abi.lib().rts_integrate_lengths(9, pos.ctypes.data_as(dp), 2, cut.ctypes.data_as(dp),
                                         lf.ctypes.data_as(ip), out.ctypes.data_as(ip))
    assert rc == abi.RTS_OK
    ref = [16 if d < 500 else (8 if d < 1000 else 4)
           for d in (np.linalg.norm(pos[i] - pos[j]) for i in range(9) for j in range(i + 1, 9))]
    np.testing.assert_array_equal(out, ref)
    bad = np.array([1000.0, 500.0])
    assert abi.lib().rts_integrate_lengths(9, pos.ctypes.data_as(dp), 2, bad.ctypes.data_as(dp),
                                           lf.ctypes.data_as(ip), out.ctypes.data_as(ip)) == abi.RTS_EINVAL


@pytest.mark.parametrize("n_fine,lens,n_slot,needle", [
    (16, [3, 4], 4, "divide"),
    (16, [4, 0], 4, "divide"),
    (16, [4, 8], 2, "n_slot"),
    (16, [4, 8], 17, "n_slot"),
    (0, [1], 1, "n_fine"),
])
def test_integrate_init_rejects_bad_lengths_on_host(abi, n_fine, lens, n_slot, needle):
    L = np.asarray(lens, np.int32)
    h = ctypes.c_void_p()
    rc = abi.lib().rts_integrate_init(n_fine, len(L), 8, L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n_slot,
                                      ctypes.byref(h))
    assert rc == abi.RTS_EINVAL and not h.value
    assert needle in abi.lib().rts_integrate_last_error(None).decode()
