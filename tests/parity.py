"""Helpers of the CUDA-vs-oracle parity tests.

A residual is a sum of Gauss-point fluxes that cancel to a small value, and in directions where the
exact solution has no flow it is pure discretisation noise around zero; the error of two different
FP64 evaluations is then rounding of the summed terms.  So residuals are compared relative to the
magnitude of the terms they sum (per component, the largest over cells of sum |weight x flux|), and
Gauss-Green gradients relative to sum |weight x interface state| / |Omega|; other arrays relative
to their own largest entry per component."""
import numpy as np


def _rows(a):
    a = np.asarray(a, float)
    return a[None, :] if a.ndim == 1 else a.reshape(a.shape[0], -1)


def normwise_err(got, ref, scale=None):
    """max over components of max |got - ref| / (scale of the component); scale defaults to the
    component's max |ref|, floored at 1e-8 of the largest component scale."""
    got, ref = _rows(got), _rows(ref)
    if scale is None:
        s = np.abs(ref).max(axis=1)
        s = np.maximum(s, max(1e-8 * s.max(), 1e-300))
    else:
        s = _rows(scale).max(axis=1)
    return (np.abs(got - ref).max(axis=1) / s).max()


def assert_normwise(got, ref, rtol, what="", scale=None):
    e = normwise_err(got, ref, scale)
    assert e <= rtol, f"{what}: normwise relative error {e:.3e} > {rtol:.1e}"
    return e


def grad_scale(gscale):
    """[15][N] scale of the gradient components from the [5][N] per-variable scale; the three
    momentum components share the largest of their scales (frame rotations mix them, so rounding in
    one component follows the magnitude of the momentum vector)."""
    g = np.array(gscale, dtype=float)
    g[1:4] = g[1:4].max(axis=0)
    return np.repeat(g, 3, axis=0)
