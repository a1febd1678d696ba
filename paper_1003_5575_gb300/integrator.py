"""Torch-tensor convenience over the visibility integrator's C ABI
(include/rts_integrate.h).  Argument marshalling only: the averaging runs in
the library's CUDA kernel."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from .peeler import _ptr, _stream


def integration_lengths(uvw_ant, cut_m, len_for):
    """Group length (fine samples) per baseline from antenna positions [n_ant][3]:
    len_for[k] for baselines in [cut_m[k-1], cut_m[k]) metres (cut_m ascending)."""
    uvw = np.ascontiguousarray(uvw_ant, dtype=np.float64)
    cut = np.ascontiguousarray(cut_m, dtype=np.float64)
    lf = np.ascontiguousarray(len_for, dtype=np.int32)
    n_ant = uvw.shape[0]
    out = np.zeros(n_ant * (n_ant - 1) // 2, np.int32)
    _abi.rts_integrate_lengths(n_ant, uvw.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(cut),
                               cut.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if len(cut) else None,
                               lf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


class Integrator:
    """Per-baseline time integration of [n_fine][n_bl][n_chan][4] complex64 cubes
    into [n_slot][n_bl][n_chan][4] (group lengths `lengths` [n_bl], dividing n_fine)."""

    def __init__(self, n_fine: int, n_chan: int, lengths, n_slot: int | None = None):
        self.lengths = np.ascontiguousarray(lengths, dtype=np.int32)
        self.n_fine, self.n_chan, self.n_bl = int(n_fine), int(n_chan), int(self.lengths.shape[0])
        self.n_slot = int(n_slot) if n_slot is not None else self.n_fine // int(self.lengths.min())
        self.h = _abi.rts_integrate_init(self.n_fine, self.n_bl, self.n_chan,
                                         self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.n_slot)

    def close(self):
        if self.h:
            _abi.rts_integrate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, fine: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        shape = (self.n_fine, self.n_bl, self.n_chan, 4)
        if fine.dtype != torch.complex64 or tuple(fine.shape) != shape or not fine.is_contiguous() or not fine.is_cuda:
            raise ValueError(f"fine must be a contiguous cuda complex64 tensor of shape {shape}")
        if out is None:
            out = torch.empty((self.n_slot, self.n_bl, self.n_chan, 4), dtype=torch.complex64, device=fine.device)
        _abi.rts_integrate_run(self.h, _ptr(fine), _ptr(out), _stream(stream))
        return out
