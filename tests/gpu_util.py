"""Shared helpers of the GPU tests (tolerances, comparisons, library set-up)."""
import numpy as np

# rho tolerance (FP32 path vs FP64 oracle): |d| <= RHO_TOL * max(|rho_ref|, rms(rho_ref)).
# An elementwise relative bound alone fails on delta-strong edges whose rho is
# far below the typical distance: the FP32 sweep error is absolute in the
# rescaled [-1/2, 1/2] range, not relative to each rho.
RHO_TOL = 1e-5


def rho_error(rho, ref):
    scale = max(float(np.sqrt(np.mean(np.asarray(ref, np.float64) ** 2))), 1e-30)
    d = np.abs(np.asarray(rho, np.float64) - ref)
    return float(np.max(d / np.maximum(np.abs(ref), scale))) if len(ref) else 0.0


def assert_rho_close(rho, ref, tol=RHO_TOL):
    err = rho_error(rho, ref)
    assert err <= tol, f"rho error {err:.3e} > {tol:.1e}"
    return err


def jaccard(a, b):
    a = np.asarray(a, bool)
    b = np.asarray(b, bool)
    u = np.logical_or(a, b).sum()
    return 1.0 if u == 0 else float(np.logical_and(a, b).sum() / u)


def lib():
    from paper_1601_05527_gb300 import build, _lib
    build.build()
    L = _lib
    L.load()
    L.use_torch_allocator()
    return L


def entry_weights_f64(g):
    return None if g.weight is None else g.weight.astype(np.float64)
