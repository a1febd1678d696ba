"""GB300-native calibrate-and-peel (MWA Real Time System, Calibration-Measurement Loop).

The compute lives in librtspeel.so (hand-written sm_103a CUDA behind the C ABI of
include/rts_peel.h); this package is its binding.  Importing it does not load
the library; the first call does, and raises if the library was not built.
"""
from ._abi import (  # noqa: F401
    RTS_OK, RTS_NOT_CONVERGED, RTS_EINVAL, RTS_ENOMEM, RTS_ECUDA, RTS_ENONFINITE,
    RTS_PREC_MIXED, RTS_PREC_FP64, RtsError, rts_peel_config,
    rts_peel_init, rts_peel_set_uvw, rts_peel_cadence, rts_peel_cadence_host, rts_peel_cadence_taylor, rts_peel_predict,
    rts_peel_rotate_average, rts_peel_solve, rts_peel_solve_noalloc, rts_peel_grad,
    rts_peel_offsets, rts_offsets_solve,
    rts_peel_pipeline_submit, rts_peel_pipeline_wait, rts_peel_last_error, rts_peel_destroy,
    rts_peel_timing, rts_peel_timing_read, rts_peel_kernels, rts_host_alloc, rts_host_free, KERNEL_CLASSES, RTS_BLOCK,
    RTS_BLOCK_AUTO, RTS_BLOCK_FMA, RTS_BLOCK_TENSOR, RTS_BLOCK_TCGEN05, RTS_SOLVE_AUTO, RTS_SOLVE_LAUNCHES,
    RTS_GRAD_AUTO, RTS_GRAD_DIRECT,
)


def __getattr__(name):
    if name in ("Peeler", "PeelLoss", "peel", "offsets_solve"):
        from . import peeler
        return getattr(peeler, name)
    if name == "Gridder":
        from . import gridder
        return gridder.Gridder
    if name in ("Integrator", "integration_lengths"):
        from . import integrator
        return getattr(integrator, name)
    raise AttributeError(name)
