"""Host-side tests of the C ABI: no GPU needed.

The library loads, exports every symbol include/rts_peel.h declares, and
rejects bad configurations on the host before touching CUDA.
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
