"""Shared helpers for GPU-vs-oracle parity tests.

Tolerance: max |dRGBA| <= 1e-3 per channel over non-ambiguous pixels and RMS
<= 1e-5 over all pixels, FP32 GPU against the FP64 oracle.  A pixel is
ambiguous when FP32 and FP64 may legitimately take a different discrete
decision: its ray length / step is within 1e-4 of an integer (one sample more
or less), or an opacity compared against the termination threshold came
within AMB_ALPHA of it.
"""
import numpy as np

MAX_TOL = 1e-3
RMS_TOL = 1e-5
AMB_ALPHA = 1e-5
AMB_STEPS = 1e-4


def compare(gpu, ref, amb):
    gpu = np.asarray(gpu, dtype=np.float64).reshape(ref.shape)
    err = np.abs(gpu - ref)
    ok = (np.asarray(amb).reshape(ref.shape[:-1]) == 0)
    max_err = float(err[ok].max()) if ok.any() else 0.0
    rms = float(np.sqrt(np.mean(err ** 2)))
    return {"max": max_err, "rms": rms, "ambiguous": int((~ok).sum()),
            "max_all": float(err.max()), "pixels": int(ok.size)}


def assert_parity(gpu, ref, amb, max_tol=MAX_TOL, rms_tol=RMS_TOL, min_signal=0.05):
    r = compare(gpu, ref, amb)
    assert np.abs(ref).max() > min_signal, "degenerate case: the reference image is empty"
    assert r["max"] <= max_tol and r["rms"] <= rms_tol, r
    assert r["ambiguous"] <= 0.01 * r["pixels"] + 4, r
    return r
