"""Torch-facing wrapper of the C ABI: device buffers and streams come from
PyTorch, every computation from librtspeel's CUDA kernels.

    p = Peeler(uvw, freq_hz, n_iter=20, precision="mixed", max_sources=1000)
    resid, jones, status = p.cadence(vis, sources)     # vis: cuda complex64 [t][bl][c][4]
    loss = PeelLoss.apply(p, vis, jones, src)          # src: cuda float64 [K][3]
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _host_f64(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


class _DeviceFloats:
    """A float32 device buffer of the library, seen by torch without a copy."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


class Peeler:
    """One array configuration (antennas, channels, times) on the current CUDA device."""

    def __init__(self, uvw, freq_hz, n_iter: int = 20, precision: str = "mixed",
                 max_sources: int = 1024, sources_per_pass: int = 0, block_kernel: int = 0,
                 solve_kernel: int = 0, grad_kernel: int = 0, band_n_chan: int = 0, band_chan0: int = 0):
        uvw = _host_f64(uvw)
        freq = _host_f64(freq_hz)
        if uvw.ndim != 3 or uvw.shape[2] != 3:
            raise ValueError("uvw must be [n_time][n_ant][3]")
        self.n_time, self.n_ant = int(uvw.shape[0]), int(uvw.shape[1])
        self.n_chan = int(freq.shape[0])
        self.freq_hz = freq
        self.n_bl = self.n_ant * (self.n_ant - 1) // 2
        self.n_iter = int(n_iter)
        self.precision = precision
        self.max_sources = int(max_sources)
        self.cdtype = torch.complex64 if precision == "mixed" else torch.complex128
        cfg = _abi.rts_peel_config()
        cfg.n_ant, cfg.n_chan, cfg.n_time = self.n_ant, self.n_chan, self.n_time
        cfg.n_iter = self.n_iter
        cfg.precision = _abi.RTS_PREC_MIXED if precision == "mixed" else _abi.RTS_PREC_FP64
        cfg.max_sources = self.max_sources
        cfg.uvw = uvw.ctypes.data_as(_dp)
        cfg.freq_hz = freq.ctypes.data_as(_dp)
        cfg.sources_per_pass = int(sources_per_pass)
        cfg.block_kernel = int(block_kernel)
        cfg.solve_kernel = int(solve_kernel)
        cfg.grad_kernel = int(grad_kernel)
        cfg.band_n_chan = int(band_n_chan)
        cfg.band_chan0 = int(band_chan0)
        self.sources_per_pass = int(sources_per_pass)
        self._keep = (uvw, freq)
        self._shard_status = np.zeros(1, np.int32)
        self._shard_k = 0
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.h = _abi.rts_peel_init(cfg)

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            _abi.rts_peel_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes -------------------------------------------------------------
    @property
    def cube_shape(self):
        return (self.n_time, self.n_bl, self.n_chan, 4)

    def empty_cube(self) -> torch.Tensor:
        return torch.empty(self.cube_shape, dtype=self.cdtype, device=self.device)

    def _check_cube(self, v: torch.Tensor, name="vis"):
        if v.dtype != self.cdtype or tuple(v.shape) != self.cube_shape or not v.is_contiguous() \
                or v.device.type != "cuda":
            raise ValueError(f"{name} must be a contiguous cuda {self.cdtype} tensor of shape {self.cube_shape}")

    # -- calls --------------------------------------------------------------
    def set_uvw(self, uvw, stream=None):
        u = _host_f64(uvw)
        if u.shape != (self.n_time, self.n_ant, 3):
            raise ValueError("uvw shape mismatch")
        _abi.rts_peel_set_uvw(self.h, u.ctypes.data_as(_dp), _stream(stream))

    def cadence(self, vis: torch.Tensor, sources, resid: torch.Tensor | None = None,
                jones: torch.Tensor | None = None, status: bool = True, stream=None):
        """Peel every source of `sources` ([K][3] l, m, S) from `vis`.
        Returns (resid, jones [K][n_ant][4], status int32[K] or None)."""
        self._check_cube(vis)
        src = _host_f64(sources).reshape(-1, 3)
        k = src.shape[0]
        if resid is None:
            resid = self.empty_cube()
        self._check_cube(resid, "resid")
        if jones is None:
            jones = torch.empty((k, self.n_ant, 4), dtype=self.cdtype, device=self.device)
        st = np.zeros(max(k, 1), np.int32) if status else None
        _abi.rts_peel_cadence(self.h, _ptr(vis), _ptr(resid), k, src.ctypes.data_as(_dp),
                              _ptr(jones), st.ctypes.data_as(_ip) if status else None, _stream(stream))
        return resid, jones, (st[:k] if status else None)

    # -- channel shards (band_n_chan > 0) --------------------------------------
    def shard_begin(self, vis: torch.Tensor, sources, resid: torch.Tensor | None = None, stream=None):
        """Start a channel-shard cadence (first pass: the partial averages of the
        first block).  Returns (resid, jones [K][n_ant][4]), filled as it runs."""
        self._check_cube(vis)
        src = _host_f64(sources).reshape(-1, 3)
        k = src.shape[0]
        if resid is None:
            resid = self.empty_cube()
        self._check_cube(resid, "resid")
        jones = torch.empty((k, self.n_ant, 4), dtype=self.cdtype, device=self.device)
        self._shard_status = np.zeros(max(k, 1), np.int32)
        self._shard_k = k
        _abi.rts_peel_shard_begin(self.h, _ptr(vis), _ptr(resid), k, src.ctypes.data_as(_dp), _ptr(jones),
                                  _stream(stream))
        return resid, jones

    def shard_partials(self) -> torch.Tensor:
        """The current block's partial averages (float32, a view of the
        library's workspace, valid until the next shard_step)."""
        ptr, n = _abi.rts_peel_shard_partials(self.h)
        self._shard_view = _DeviceFloats(ptr, n)
        return torch.as_tensor(self._shard_view, device=self.device)

    def shard_step(self, stream=None) -> int:
        """Solve the block from the summed partials, subtract it, leave the next
        block's partials: 1 while another exchange is needed, 0 when the cadence
        is done (shard_status() then holds the statuses)."""
        return _abi.rts_peel_shard_step(self.h, self._shard_status.ctypes.data_as(_ip), _stream(stream))

    def shard_status(self) -> np.ndarray:
        return self._shard_status[:self._shard_k]

    def cadence_sharded(self, vis: torch.Tensor, sources, exchange, resid: torch.Tensor | None = None):
        """One cadence of this handle's channel shard.  Before each block's
        solve, exchange(partial) must sum the float32 tensor `partial` in place
        over all shards of the band, on the current stream (e.g.
        replicas.sum_over_ranks).  Returns (resid, jones, status, exchanges)."""
        from .replicas import run_sharded_cadence
        out = {}

        def begin():
            out["r"], out["j"] = self.shard_begin(vis, sources, resid)

        n = run_sharded_cadence(begin, self.shard_partials, self.shard_step, exchange)
        return out["r"], out["j"], self.shard_status(), n

    def cadence_taylor(self, vis: torch.Tensor, sources, resid: torch.Tensor | None = None,
                       status: bool = True, stream=None):
        """Peel with gains linear in frequency, J(c) = G + x_c H (x_c the channel's
        offset from the band centre in band widths).  Returns (resid, G, H
        [K][n_ant][4], status int32[K] or None)."""
        self._check_cube(vis)
        src = _host_f64(sources).reshape(-1, 3)
        k = src.shape[0]
        if resid is None:
            resid = self.empty_cube()
        self._check_cube(resid, "resid")
        gain = torch.empty((k, self.n_ant, 4), dtype=self.cdtype, device=self.device)
        slope = torch.empty_like(gain)
        st = np.zeros(max(k, 1), np.int32) if status else None
        _abi.rts_peel_cadence_taylor(self.h, _ptr(vis), _ptr(resid), k, src.ctypes.data_as(_dp),
                                     _ptr(gain), _ptr(slope), st.ctypes.data_as(_ip) if status else None,
                                     _stream(stream))
        return resid, gain, slope, (st[:k] if status else None)

    def cadence_host(self, h_vis: torch.Tensor, sources, d_work: torch.Tensor,
                     h_resid: torch.Tensor | None = None, stream=None):
        """The same peel on host (ideally pinned) tensors, copies included."""
        src = _host_f64(sources).reshape(-1, 3)
        k = src.shape[0]
        if h_resid is None:
            h_resid = torch.empty_like(h_vis)
        h_jones = torch.empty((k, self.n_ant, 4), dtype=self.cdtype)
        st = np.zeros(max(k, 1), np.int32)
        self._check_cube(d_work, "d_work")
        for t, nm in ((h_vis, "h_vis"), (h_resid, "h_resid")):
            if t.device.type != "cpu" or tuple(t.shape) != self.cube_shape or t.dtype != self.cdtype \
                    or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous host {self.cdtype} tensor {self.cube_shape}")
        _abi.rts_peel_cadence_host(self.h, _ptr(h_vis), _ptr(h_resid), k, src.ctypes.data_as(_dp),
                                   _ptr(h_jones), st.ctypes.data_as(_ip), _ptr(d_work), _stream(stream))
        return h_resid, h_jones, st[:k]

    def predict(self, sources, jones: torch.Tensor, out: torch.Tensor | None = None,
                accumulate: bool = False, stream=None) -> torch.Tensor:
        src = _host_f64(sources).reshape(-1, 3)
        if out is None:
            out = self.empty_cube()
        self._check_cube(out, "out")
        jones = jones.to(device=self.device, dtype=self.cdtype).contiguous()
        _abi.rts_peel_predict(self.h, _ptr(out), src.shape[0], src.ctypes.data_as(_dp), _ptr(jones),
                              int(accumulate), _stream(stream))
        return out

    def rotate_average(self, vis: torch.Tensor, l: float, m: float, stream=None) -> torch.Tensor:
        self._check_cube(vis)
        avg = torch.empty((self.n_bl, 4), dtype=self.cdtype, device=self.device)
        _abi.rts_peel_rotate_average(self.h, _ptr(vis), float(l), float(m), _ptr(avg), _stream(stream))
        return avg

    def solve(self, avg: torch.Tensor, S: float, stream=None):
        avg = avg.to(device=self.device, dtype=self.cdtype).contiguous()
        J = torch.empty((self.n_ant, 4), dtype=self.cdtype, device=self.device)
        st = np.zeros(1, np.int32)
        _abi.rts_peel_solve(self.h, _ptr(avg), float(S), _ptr(J), st.ctypes.data_as(_ip), _stream(stream))
        return J, int(st[0])

    def rel(self, n_src: int, stream=None) -> np.ndarray:
        """Last relative change of each source's ALS solve in the last cadence
        (the number its status compares with 1e-6), float64[n_src]."""
        out = np.zeros(max(n_src, 1))
        _abi.rts_peel_rel(self.h, n_src, out.ctypes.data_as(_dp), _stream(stream))
        return out[:n_src]

    def phases(self, l: float, m: float, tb, form: int = 0, stream=None) -> torch.Tensor:
        """The peel's per-channel phase of direction (l, m), in turns, on the
        (time, baseline) pairs tb ([n][2] int): float64 [n][n_chan].  form 0:
        Q0.64 phase of the baseline delay; 1: its FP32 sin/cos argument; 2: the
        blocked schedule's difference of antenna phases."""
        tb = torch.as_tensor(np.ascontiguousarray(tb, dtype=np.int32).reshape(-1, 2), device=self.device)
        out = torch.empty((tb.shape[0], self.n_chan), dtype=torch.float64, device=self.device)
        _abi.rts_peel_phases(self.h, l, m, tb.shape[0], _ptr(tb), int(form), _ptr(out), _stream(stream))
        return out

    def grad(self, vis: torch.Tensor, jones: torch.Tensor, src: torch.Tensor,
             want_grad: bool = True, stream=None):
        """(loss, dL/dJ, dL/d(l, m, S)) with loss and gradients as cuda tensors."""
        self._check_cube(vis)
        k = int(src.shape[0])
        jones = jones.detach().to(device=self.device, dtype=self.cdtype).contiguous()
        src = src.detach().to(device=self.device, dtype=torch.float64).contiguous()
        loss = torch.empty((), dtype=torch.float64, device=self.device)
        gJ = torch.empty_like(jones) if want_grad else None
        gs = torch.empty((k, 3), dtype=torch.float64, device=self.device) if want_grad else None
        _abi.rts_peel_grad(self.h, _ptr(vis), k, _ptr(jones), _ptr(src), _ptr(loss),
                           _ptr(gJ) if want_grad else None, _ptr(gs) if want_grad else None,
                           _stream(stream))
        return loss, gJ, gs

    def offsets(self, vis: torch.Tensor, jones: torch.Tensor, src: torch.Tensor, alpha: float = 0.0,
                nu_ref_hz: float | None = None, stream=None):
        """Ionospheric position offsets with the shift law (nu_ref/nu)^alpha:
        (six numbers [K][6] = H_ll, H_lm, H_mm, dL/d dl, dL/d dm, L;
        offsets [K][2] = -H^-1 g), float64 cuda tensors.  nu_ref defaults to the
        band centre; channel groups that are combined must share it."""
        self._check_cube(vis)
        k = int(src.shape[0])
        jones = jones.detach().to(device=self.device, dtype=self.cdtype).contiguous()
        src = src.detach().to(device=self.device, dtype=torch.float64).contiguous()
        nu_ref = float(np.mean(self.freq_hz)) if nu_ref_hz is None else float(nu_ref_hz)
        out = torch.empty((k, 6), dtype=torch.float64, device=self.device)
        off = torch.empty((k, 2), dtype=torch.float64, device=self.device)
        _abi.rts_peel_offsets(self.h, _ptr(vis), k, _ptr(jones), _ptr(src), float(alpha), nu_ref,
                              _ptr(out), _ptr(off), _stream(stream))
        return out, off


def offsets_solve(six: torch.Tensor, stream=None) -> torch.Tensor:
    """(dl, dm) = -H^-1 g per source from summed six numbers [K][6] (cuda float64)."""
    six = six.to(dtype=torch.float64).contiguous()
    if not six.is_cuda:
        raise ValueError("offsets_solve needs a cuda tensor")
    off = torch.empty((six.shape[0], 2), dtype=torch.float64, device=six.device)
    _abi.rts_offsets_solve(_ptr(six), int(six.shape[0]), _ptr(off), _stream(stream))
    return off

class PeelLoss(torch.autograd.Function):
    """L(J, l, m, S) = sum ||V - sum_k S_k J_i J_j^H exp(-2 pi i phi_k)||^2.

    forward runs the fused loss + adjoint kernel once (phasors recomputed,
    never stored) when any input needs a gradient; backward scales the kept
    gradients by grad_output."""

    @staticmethod
    def forward(ctx, peeler: Peeler, vis: torch.Tensor, jones: torch.Tensor, src: torch.Tensor):
        want = ctx.needs_input_grad[2] or ctx.needs_input_grad[3]
        loss, gJ, gs = peeler.grad(vis, jones, src, want_grad=want)
        if want:
            ctx.save_for_backward(gJ.to(jones.dtype), gs.to(src.dtype))
        return loss

    @staticmethod
    def backward(ctx, g):
        gJ, gs = ctx.saved_tensors
        return None, None, g * gJ, g * gs


def peel(vis: torch.Tensor, uvw, freq_hz, sources, n_iter: int = 20, precision: str = "mixed",
         sources_per_pass: int = 0):
    """One-shot peel of a cuda cube; returns (resid, jones, status)."""
    p = Peeler(uvw, freq_hz, n_iter=n_iter, precision=precision,
               max_sources=max(1, len(_host_f64(sources).reshape(-1, 3))),
               sources_per_pass=sources_per_pass)
    try:
        return p.cadence(vis, sources)
    finally:
        p.close()
