"""Torch-tensor convenience over the gridder's C ABI (include/rts_grid.h).

Argument marshalling only: the sort and the gather run in the library's CUDA
kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from .peeler import _ptr, _stream


class Gridder:
    """Gridder of Section 6 on the current CUDA device: n_pix x n_pix grid, radial
    gridding convolution function given by `gcf` samples on [0, r_max], bins of
    `bin` pixels, `n_pol` complex values per visibility."""

    def __init__(self, n_pix: int, r_max: float, gcf, bin: int = 24, n_pol: int = 4, max_vis: int = 1 << 20):
        self._gcf = np.ascontiguousarray(gcf, dtype=np.float64)
        cfg = _abi.rts_grid_config()
        cfg.n_pix, cfg.bin, cfg.r_max = int(n_pix), int(bin), float(r_max)
        cfg.gcf = self._gcf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.n_tab, cfg.n_pol, cfg.max_vis = int(self._gcf.shape[0]), int(n_pol), int(max_vis)
        self.n_pix, self.n_pol, self.max_vis = int(n_pix), int(n_pol), int(max_vis)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.h = _abi.rts_grid_init(cfg)

    def close(self):
        if self.h:
            _abi.rts_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, xy: torch.Tensor, vis: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """xy: cuda float32 [n_vis][2] pixel coordinates; vis: cuda complex64
        [n_vis][n_pol]; returns the grid, complex64 [n_pol][n_pix][n_pix]."""
        n = int(xy.shape[0])
        if xy.dtype != torch.float32 or tuple(xy.shape) != (n, 2) or not xy.is_contiguous() or not xy.is_cuda:
            raise ValueError("xy must be a contiguous cuda float32 tensor [n_vis][2]")
        if vis.dtype != torch.complex64 or tuple(vis.shape) != (n, self.n_pol) or not vis.is_contiguous() \
                or not vis.is_cuda:
            raise ValueError(f"vis must be a contiguous cuda complex64 tensor [n_vis][{self.n_pol}]")
        if out is None:
            out = torch.empty((self.n_pol, self.n_pix, self.n_pix), dtype=torch.complex64, device=self.device)
        _abi.rts_grid_run(self.h, _ptr(xy), _ptr(vis), n, _ptr(out), _stream(stream))
        return out

    def last_ms(self):
        """(sort ms, gather ms) of the last run."""
        return _abi.rts_grid_last_ms(self.h)
