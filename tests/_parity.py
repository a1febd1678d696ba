"""Helpers shared by the GPU parity tests: tolerances, error measures, the
status comparison and a cache of the oracle's peels (test infrastructure)."""
import math

import numpy as np
import torch

import oracle

TOL = {"mixed": 1e-5, "fp64": 1e-10}
CDT = {"mixed": (np.complex64, torch.complex64), "fp64": (np.complex128, torch.complex128)}


def rms_of(V):
    return math.sqrt(float(np.mean(V.real.astype(np.float64) ** 2 + V.imag.astype(np.float64) ** 2) / 2))


def to_dev(V, prec):
    return torch.from_numpy(np.ascontiguousarray(V.astype(CDT[prec][0]))).cuda()


def jones_rel(Jg, Jr):
    return max(np.linalg.norm(Jg[k] - Jr[k]) / np.linalg.norm(Jr[k]) for k in range(len(Jr)))


STATUS_THRESHOLD = 1e-6   # a source is "not converged" when its last relative change exceeds this


def rel_tol(rel_ref, prec="mixed"):
    """Allowed |rel - rel_ref| of a source's last relative change
    ||J_n - J_(n-1)||_F / ||J_n||_F.  Mixed: 1 % of it plus 1e-7 (the iterate
    before the last sweep is FP32, rounded to ~2^-24 of each entry, and that
    sweep's FP32 products carry ~1e-7 of the normal-equation sums; the input
    differences of FP32 averages move the change itself by far less than 1 %).
    FP64: 1e-8 of it plus 1e-13 (summation order only).  Taylor gains
    ("taylor", X = [G H]): 2 % of it plus 4e-7 -- every sweep of the 4x4 solve
    and every slope-rotation step reads FP32 iterates and sums FP32 products,
    and the 4x4 normal matrix (channel moments up to x_c^4) amplifies their
    rounding more than the 2x2 one; measured differences stay below 3.1e-7."""
    rel_ref = np.abs(np.asarray(rel_ref, dtype=np.float64))
    if prec == "taylor":
        return 0.02 * rel_ref + 4e-7
    return 0.01 * rel_ref + 1e-7 if prec == "mixed" else 1e-8 * rel_ref + 1e-13


def check_status(name, st, st_ref, rel, rel_ref, prec="mixed"):
    """Statuses equal the oracle's wherever the oracle's relative change is
    farther from the threshold than rel_tol; the changes agree within rel_tol.
    Returns the number of sources inside that band (status not compared)."""
    st, st_ref = np.asarray(st), np.asarray(st_ref)
    rel, rel_ref = np.asarray(rel, np.float64), np.asarray(rel_ref, np.float64)
    tol = rel_tol(rel_ref, prec)
    decided = np.abs(rel_ref - STATUS_THRESHOLD) > tol
    worst = float(np.max(np.abs(rel - rel_ref) / tol)) if len(rel) else 0.0
    print(f"{name}: status {int(np.sum(st == st_ref))}/{len(st)} equal, {int(np.sum(~decided))} in the band, "
          f"{int(np.sum(st_ref == 1))} not converged (oracle), rel error {worst:.3f} of its tolerance")
    assert np.all(np.abs(rel - rel_ref) <= tol), (rel, rel_ref)
    np.testing.assert_array_equal(st[decided], st_ref[decided])
    return int(np.sum(~decided))


_cache = {}


def oracle_case(cad, n_iter=20):
    """(V as the GPU sees it, residual, Jones, status, last relative change) of the oracle's peel."""
    key = (cad, n_iter)
    if key not in _cache:
        V = oracle.simulate(cad)
        if cad.precision == "mixed":
            V = V.astype(np.complex64).astype(np.complex128)   # what the GPU sees
        R, J, st, rel = oracle.peel(cad.uvw(), cad.freqs(), V, cad.sources(), n_iter=n_iter, with_rel=True)
        _cache[key] = (V, R, J, st, rel)
    return _cache[key]



def make_peeler(cad, prec, n_iter=20, max_sources=None, per_pass=0, block_kernel=0, solve_kernel=0,
                grad_kernel=0):
    from paper_1003_5575_gb300 import Peeler
    return Peeler(cad.uvw(), cad.freqs(), n_iter=n_iter, precision=prec,
                  max_sources=max_sources or max(cad.n_src, 1), sources_per_pass=per_pass,
                  block_kernel=block_kernel, solve_kernel=solve_kernel, grad_kernel=grad_kernel)


def conditioning(cad, V, eps=1e-7, seed=12345, n_iter=20):
    """How far the oracle's own results move when its input moves by eps x rms:
    (max relative Jones change per source, max residual change beyond the
    perturbation itself / rms).  A path that works on FP32 data perturbs its
    input at that level, so these set how closely any FP32 path can agree."""
    _, R_ref, J_ref, _, _ = oracle_case(cad, n_iter)
    rng = np.random.default_rng(seed)
    d = eps * rms_of(V) * (rng.standard_normal(V.shape) + 1j * rng.standard_normal(V.shape))
    R, J, _ = oracle.peel(cad.uvw(), cad.freqs(), V + d, cad.sources(), n_iter=n_iter)
    return jones_rel(J, J_ref), float(np.abs(R - d - R_ref).max() / rms_of(V))
