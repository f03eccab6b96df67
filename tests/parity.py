"""Comparison rules between the CUDA path and the FP64 oracle.

Floating point: an FP32 output passes when |gpu - ref| <= 1e-5 * max(1, |ref|)
(max abs error 1e-5, relative 1e-5 above magnitude 1).  NaN must match NaN;
a reference beyond the float range must come back as an infinity of the same
sign.  Integer work (order, levels, edge lists, status) must match exactly.
"""
import numpy as np

TOL = 1e-5
FLT_MAX = float(np.finfo(np.float32).max)


def compare_outputs(gpu, ref, tol=TOL):
    """Return (n_bad, max_abs_err, max_scaled_err, n_compared)."""
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    assert gpu.shape == ref.shape
    nan_ref = np.isnan(ref)
    bad = int(np.sum(nan_ref != np.isnan(gpu)))
    big = ~nan_ref & (np.abs(ref) > FLT_MAX)
    bad += int(np.sum(big & ~(np.isinf(gpu) & (np.sign(gpu) == np.sign(ref)))))
    fin = ~nan_ref & ~big
    err = np.abs(gpu[fin] - ref[fin])
    scaled = err / np.maximum(1.0, np.abs(ref[fin]))
    bad += int(np.sum(~(scaled <= tol)))
    return bad, (float(err.max()) if err.size else 0.0), (float(scaled.max()) if err.size else 0.0), int(fin.sum())


def assert_outputs_close(gpu, ref, tol=TOL, what=""):
    bad, mabs, mscaled, n = compare_outputs(gpu, ref, tol)
    assert bad == 0, f"{what}: {bad} outputs outside tolerance (max abs {mabs:.3g}, max scaled {mscaled:.3g})"
    return mabs, mscaled


def assert_topology_equal(dec, ref, pop, what=""):
    """Transform outputs: status everywhere; order/levels/edge lists where valid."""
    np.testing.assert_array_equal(dec.status, ref["status"], err_msg=f"{what}: status")
    ok = (ref["status"] & 0xFF) == 0
    for name in ("n_nodes",):
        np.testing.assert_array_equal(getattr(dec, name), ref[name], err_msg=f"{what}: {name}")
    np.testing.assert_array_equal(dec.n_levels[ok], ref["n_levels"][ok], err_msg=f"{what}: n_levels")
    np.testing.assert_array_equal(dec.n_edges[ok], ref["n_edges"][ok], err_msg=f"{what}: n_edges")
    np.testing.assert_array_equal(dec.order[ok], ref["order"][ok], err_msg=f"{what}: order")
    np.testing.assert_array_equal(dec.level_ptr[ok], ref["level_ptr"][ok], err_msg=f"{what}: level_ptr")
    np.testing.assert_array_equal(dec.in_ptr[ok], ref["in_ptr"][ok], err_msg=f"{what}: in_ptr")
    np.testing.assert_array_equal(dec.in_src[ok], ref["in_src"][ok], err_msg=f"{what}: in_src")
    np.testing.assert_array_equal(dec.in_w[ok].astype(np.float64), np.where(ref["in_src"][ok] >= 0, ref["in_w"][ok], 0.0),
                                  err_msg=f"{what}: in_w")
