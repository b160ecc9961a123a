"""Parity tolerances of the GPU tests against the FP64 oracle (relative L2).

FP64 problems: 1e-10 for operators and FB iterates (rounding order only).
FP32 and FP32-Kahan problems: 2e-5 for every result -- one application of A,
A^T, W, W^T, P^T, Lambda, the FB iterates after their iterations, the FB
history (objective, residual norm, iterate norm) and the gradients; their
inputs are the oracle's inputs rounded to FP32.
"""
FP64_TOL = 1e-10
FP64_HIST_TOL = 1e-9
FP32_TOL = 2e-5


def tol(prec, fp64_code=0):
    """Relative L2 tolerance of a result of precision `prec` (0 = FP64)."""
    return FP64_TOL if prec == fp64_code else FP32_TOL


def hist_tol(prec, fp64_code=0):
    return FP64_HIST_TOL if prec == fp64_code else FP32_TOL


def hist_dev(hist, hist_or, cols=(0, 1, 3)):
    """Largest relative deviation of the GPU FB history from the oracle's over
    the given columns (objective, residual norm, rel. change, iterate norm)."""
    import numpy as np
    return max(float(np.max(np.abs(hist[:, c] - hist_or[:, c]) / np.abs(hist_or[:, c])))
               for c in cols)
