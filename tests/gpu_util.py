"""Helpers shared by the GPU tests: run a transform through the C ABI on torch
device memory, and compare with the oracle under the stated tolerances."""
import numpy as np
import torch

import paper_2211_13706_gb300 as mz

# Tolerances, componentwise relative to the magnitude d_i of the terms the
# transform adds (zeta: d = Z|f|; Moebius residual: d = Z|f_out| + |g|):
#   int64 : bit-exact;
#   fp64  : 1e-12 (plain fp64: at most a few hundred roundings of 2^-53 each
#           along a chain prefix plus k gathered terms);
#   F32C  : 1e-10 (the target for double-word fp32; Sum2 / DW bounds are
#           ~k^2 u^2 and ~L u^2 with u = 2^-24).
TOL = {mz.MZ_F64: 1e-12, mz.MZ_F32C: 1e-10}


def to_device(x, dtype):
    """numpy [n] / [n, B] values -> the device tensor of the ABI layout."""
    if dtype == mz.MZ_I64:
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.int64)).cuda()
    if dtype == mz.MZ_F64:
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    if isinstance(x, tuple):
        hi, lo = x
    else:
        hi = np.asarray(x, dtype=np.float32)
        lo = np.zeros_like(hi)
    return torch.from_numpy(np.ascontiguousarray(np.stack([hi, lo]), dtype=np.float32)).cuda()


def from_device(t, dtype):
    """device tensor -> numpy; F32C returns (hi, lo) and their exact-ish fp64 sum."""
    a = t.cpu().numpy()
    if dtype == mz.MZ_F32C:
        return a[0].astype(np.float64) + a[1].astype(np.float64)
    return a


def run(plan, name, x_np, dtype):
    x = to_device(x_np, dtype)
    y = getattr(plan, name)(x)
    plan.check()
    return from_device(y, dtype)


def exact_input(x_np, dtype):
    """The input as the oracle sees it: int64, fp64, or the F32C pair."""
    if dtype == mz.MZ_F32C:
        if isinstance(x_np, tuple):
            return x_np
        hi = np.asarray(x_np, dtype=np.float32)
        return (hi, np.zeros_like(hi))
    if dtype == mz.MZ_F64:
        return np.asarray(x_np, dtype=np.float64)
    return np.asarray(x_np, dtype=np.int64)


def assert_close(got, ref, mag, dtype, what=""):
    if dtype == mz.MZ_I64:
        bad = np.flatnonzero(np.ravel(got != ref))
        assert bad.size == 0, f"{what}: {bad.size} int64 mismatches, first at {bad[:5]}"
        return 0.0
    err = np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))
    rel = err / np.maximum(np.asarray(mag, np.float64), np.finfo(np.float64).tiny)
    worst = float(rel.max()) if rel.size else 0.0
    assert worst <= TOL[dtype], f"{what}: componentwise error {worst:.3e} > {TOL[dtype]:.0e}"
    return worst
