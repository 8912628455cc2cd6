"""Helpers shared by the GPU parity tests: seeded inputs and the comparison
rule between the CUDA path and the FP64 oracle.

Tolerance (F, per particle):  |F_gpu - F_or| <= 1e-4 |F_or| + 1e-4 rms(F_or)
Scale index: equal on >= 99.99 % of particles; every other particle must be a
near-tie (the oracle's F at the GPU's index is within the F tolerance of its
own maximum).

Conditioning (a reading of the tolerance for an FP32 path): F is not a
continuous function of the Hessian everywhere.  Where the first axis crossing
is near-tangent, or the largest eigenvalue is a tiny fraction of the field's
scale (F then goes as its cube root), a change of the Hessian at the size of
single-precision rounding moves F by more than the tolerance.  So a particle
that misses the rule above passes only if the ORACLE, on its own FP64
Hessians of that particle at every radius (the direct sum over modes), finds
it ill-conditioned and the GPU's result inside the oracle's range:
  - per radius s, the range [lo_s, hi_s] of F over eigenvalue errors of
    half-width U_FP32 (hrms_s + max |lambda|) (oracle.collapse_interval);
  - F_gpu within [max_s lo_s - tol, max_s hi_s + tol] (the range of F_max);
  - the GPU's radius index I able to hold the maximum: F_gpu within
    [lo_I - tol, hi_I + tol] (or I = -1, F_gpu = 0, and max_s lo_s <= tol).
Such conditioned particles must stay at or below 1e-4 of the grid (at least
one is allowed); every parity test prints how many there were.  Nothing of
the GPU's intermediate values enters the rule.
"""
import numpy as np

from paper_1305_1505_gb300 import ic

REL = 1e-4
ABS_FRAC = 1e-4
# Half-width of the eigenvalue errors the conditioning range allows, relative
# to the field's rms tensor norm plus the local one: about 64 units of FP32
# rounding (2^-24), above the measured transform error (a few 1e-7 of the rms
# at 768 points) and the trigonometric eigenvalue error (about 1e-6 of the
# matrix norm).
U_FP32 = 4e-6


def inputs(n, box, seed):
    """(delta_k complex64 for the GPU, the same values as complex128 for the oracle)."""
    d32 = ic.delta_k(n, box, seed, dtype=np.complex64)
    return d32, d32.astype(np.complex128)


def tolerance(f_or, rms, rel=REL, abs_frac=ABS_FRAC):
    return rel * np.abs(f_or) + abs_frac * rms


def classify(F_gpu, idx_gpu, F_or, idx_or, f2=None, idx2=None, f_all=None, rel=REL, abs_frac=ABS_FRAC):
    """Returns (bad_mask, report) under the F and index rules."""
    F_gpu = np.asarray(F_gpu, dtype=np.float64).ravel()
    idx_gpu = np.asarray(idx_gpu).ravel()
    F_or = np.asarray(F_or, dtype=np.float64).ravel()
    idx_or = np.asarray(idx_or).ravel()
    rms = float(np.sqrt(np.mean(F_or ** 2))) if F_or.size else 0.0
    tol = tolerance(F_or, rms, rel, abs_frac)
    err = np.abs(F_gpu - F_or)
    f_bad = err > tol
    mism = idx_gpu != idx_or
    tie_ok = np.zeros_like(mism)
    if mism.any():
        where = np.nonzero(mism)[0]
        for q in where:
            g = idx_gpu[q]
            if f_all is not None:
                fg = f_all[g, q] if g >= 0 else 0.0
                tie_ok[q] = abs(fg - F_or[q]) <= tol[q]
            elif f2 is not None:
                tie_ok[q] = (g == idx2[q]) and abs(f2[q] - F_or[q]) <= tol[q]
    idx_bad = mism & ~tie_ok
    bad = f_bad | idx_bad
    rep = dict(n=F_or.size, rms=rms, max_rel_err=float(np.max(err / np.maximum(np.abs(F_or), rms))) if F_or.size else 0.0,
               p99_err=float(np.percentile(err, 99)) if F_or.size else 0.0,
               f_bad=int(f_bad.sum()), idx_mismatch=int(mism.sum()), idx_bad=int(idx_bad.sum()),
               idx_equal_frac=float(1 - mism.mean()) if F_or.size else 1.0)
    return bad, rep


def within_conditioning(F_gpu, I_gpu, lo, hi, tol):
    """The conditioning rule for particles p (columns of lo/hi, (S, npts)):
    True where the GPU's F_max and radius index lie inside the oracle's
    range."""
    F_gpu = np.asarray(F_gpu, dtype=np.float64)
    I_gpu = np.asarray(I_gpu)
    Lo, Hi = lo.max(axis=0), hi.max(axis=0)
    ok = (F_gpu >= Lo - tol) & (F_gpu <= Hi + tol)
    cols = np.arange(F_gpu.size)
    Ic = np.clip(I_gpu, 0, lo.shape[0] - 1)
    at_i = (F_gpu >= lo[Ic, cols] - tol) & (F_gpu <= hi[Ic, cols] + tol)
    never = (I_gpu == -1) & (F_gpu == 0.0) & (Lo <= tol)
    return ok & np.where(I_gpu >= 0, at_i, never)


def conditioned(q_bad, F_gpu, I_gpu, d64, box, radii, hrms, correction, tol, u=U_FP32):
    """Oracle-side conditioning of the particles q_bad: (ok mask, lo, hi)."""
    import oracle
    h = oracle.hessians_at(d64, box, radii, q_bad)
    lo, hi = oracle.collapse_interval(h, hrms, u, correction)
    return within_conditioning(F_gpu, I_gpu, lo, hi, tol), lo, hi


def assert_parity(F, I, orc, d64, box, radii, correction=1, label="", rel=REL, abs_frac=ABS_FRAC, u=U_FP32):
    """The whole rule: every particle within the F tolerance with an equal or
    near-tie index, or (at most 1e-4 of the grid) ill-conditioned by the
    oracle's own measure with the GPU's result inside the oracle's range; the
    index equal on >= 99.99 % of particles.  d64, box, radii and correction
    are the oracle's inputs of this run; orc its collapse_times result.
    rel, abs_frac and u set the tolerance and the conditioning half-width
    (the FP32 path's by default)."""
    F = np.asarray(F).ravel()
    I = np.asarray(I).ravel()
    bad, rep = classify(F, I, orc["fmax"], orc["idx"], orc.get("f2"), orc.get("idx2"), orc.get("f_all"),
                        rel, abs_frac)
    bq = np.nonzero(bad)[0]
    rep["conditioned"] = int(bq.size)
    print("parity %s:" % label, rep)
    if bq.size:
        tol = tolerance(orc["fmax"][bq], rep["rms"], rel, abs_frac)
        ok, lo, hi = conditioned(bq, F[bq], I[bq], d64, box, radii, orc["hrms"], correction, tol, u)
        for j, q in enumerate(bq):
            print("  conditioned q=%d: gpu F=%.7g idx=%d, oracle F=%.7g idx=%d, range [%.7g, %.7g] %s"
                  % (q, F[q], I[q], orc["fmax"][q], orc["idx"][q], lo[:, j].max(), hi[:, j].max(),
                     "inside" if ok[j] else "OUTSIDE"))
        assert ok.all(), "mismatches outside the oracle's conditioning range at %s" % bq[~ok][:10]
        assert bq.size <= max(1, 1e-4 * F.size), "too many ill-conditioned particles: %d" % bq.size
    assert rep["idx_mismatch"] <= max(1, 1e-4 * F.size), rep
    return rep
