"""Error measures used by the GPU parity tests.

Means are compared normwise per step, relative to the larger of the mean's
magnitude and the largest posterior standard deviation at that step
(elementwise relative error is meaningless for components near zero, and the
positions of a Wiener-velocity model grow like T^1.5).  Covariances are
compared per step relative to their largest entry.  The reported figure is
the maximum over steps.
"""
import numpy as np

# FP32 arithmetic over a log-depth scan: errors are a few hundred ulp of the
# per-step scale at most for the well-conditioned models used here, so 1e-4
# leaves a wide margin while still catching any wrong term (which shows up at
# O(1)).
TOL = 1e-4

# nx = 32: the operators chain 32 x 32 products and pivoted inverses, so the
# FP32 rounding grows with the dimension (about n eps per product, times the
# conditioning of I + C J, which is O(10) for the stable models used here):
# ~1e-5 at most, so the same 1e-4 applies.
TOL_NX32 = 1e-4


def mean_err(got, ref, Pref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sd = np.sqrt(np.abs(np.diagonal(Pref, axis1=-2, axis2=-1))).max(-1)
    scale = np.maximum(np.abs(ref).max(-1), sd)
    return float((np.abs(got - ref).max(-1) / scale).max())


def cov_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float((np.abs(got - ref).max((-2, -1)) / np.abs(ref).max((-2, -1))).max())


def errors(gpu, ref):
    """gpu, ref: (fmean, fcov, smean, scov) tuples -> dict of max errors."""
    fm, fP, sm, sP = (np.asarray(x.detach().cpu().numpy() if hasattr(x, "detach") else x) for x in gpu)
    rfm, rfP, rsm, rsP = ref
    return {"fmean": mean_err(fm, rfm, rfP), "fcov": cov_err(fP, rfP),
            "smean": mean_err(sm, rsm, rsP), "scov": cov_err(sP, rsP)}
