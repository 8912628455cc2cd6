"""Helpers shared by the GPU parity tests: seeded inputs and the comparison
rule between the CUDA path and the FP64 oracle.

Tolerance (F, per particle):  |F_gpu - F_or| <= 1e-4 |F_or| + 1e-4 rms(F_or)
Scale index: equal on >= 99.99 % of particles; every other particle must be a
near-tie (the oracle's F at the GPU's index is within the F tolerance of its
own maximum).

A particle that misses either rule is accepted only if the oracle, run on the
GPU's own FP32 Hessians of that particle (all radii), reproduces the GPU's
F_max within tolerance: the discrepancy then comes from the FP32 rounding of
the transforms feeding an ill-conditioned collapse (a near-tangent crossing,
where F jumps), not from the kernel's eigenvalue or root arithmetic.  Such
particles must stay below 1e-4 of the grid (and are reported).
"""
import numpy as np

from paper_1305_1505_gb300 import ic

REL = 1e-4
ABS_FRAC = 1e-4


def inputs(n, box, seed):
    """(delta_k complex64 for the GPU, the same values as complex128 for the oracle)."""
    d32 = ic.delta_k(n, box, seed, dtype=np.complex64)
    return d32, d32.astype(np.complex128)


def tolerance(f_or, rms):
    return REL * np.abs(f_or) + ABS_FRAC * rms


def classify(F_gpu, idx_gpu, F_or, idx_or, f2=None, idx2=None, f_all=None):
    """Returns (bad_mask, report) under the F and index rules."""
    F_gpu = np.asarray(F_gpu, dtype=np.float64).ravel()
    idx_gpu = np.asarray(idx_gpu).ravel()
    F_or = np.asarray(F_or, dtype=np.float64).ravel()
    idx_or = np.asarray(idx_or).ravel()
    rms = float(np.sqrt(np.mean(F_or ** 2))) if F_or.size else 0.0
    tol = tolerance(F_or, rms)
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


def explain_with_gpu_hessians(plan, bad_q, F_gpu, nscales, rms, correction=1):
    """Oracle collapse on the GPU's FP32 Hessians of the given particles."""
    import torch
    import oracle
    q = torch.as_tensor(np.asarray(bad_q, dtype=np.int64), device="cuda")
    hs = np.empty((nscales, len(bad_q), 6))
    for s in range(nscales):
        h = plan.hessian(s).reshape(6, -1)
        hs[s] = h[:, q].T.double().cpu().numpy()
    out = oracle.collapse_from_hessians(hs, correction)
    F_gpu = np.asarray(F_gpu, dtype=np.float64).ravel()[bad_q]
    ok = np.abs(F_gpu - out["fmax"]) <= tolerance(out["fmax"], rms)
    return ok, out


def assert_parity(plan, F, I, orc, nscales, correction=1, label=""):
    """The whole rule: every particle within the F tolerance with an equal
    or near-tie index, or explained by the oracle on the GPU's own FP32
    Hessians (FP32 rounding of the transforms feeding an ill-conditioned
    collapse), such particles below 1e-4 of the grid, and the index equal on
    >= 99.99 % of particles."""
    F = np.asarray(F).ravel()
    I = np.asarray(I).ravel()
    bad, rep = classify(F, I, orc["fmax"], orc["idx"], orc.get("f2"), orc.get("idx2"), orc.get("f_all"))
    print("parity %s:" % label, rep, plan.stats())
    bq = np.nonzero(bad)[0]
    if bq.size:
        ok, _ = explain_with_gpu_hessians(plan, bq, F, nscales, rep["rms"], correction)
        assert ok.all(), "unexplained mismatches at %s" % bq[~ok][:10]
        assert bq.size <= max(1, 1e-4 * F.size), "too many ill-conditioned particles: %d" % bq.size
    assert rep["idx_mismatch"] <= max(1, 1e-4 * F.size), rep
    return rep
