"""Shared helpers for the parity tests (comparison metrics, library loading)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Acceptance bound of the FP32 GPU path against the FP64 oracle: normwise
# relative error, and every element within the same fraction of the largest
# output magnitude.
TOL = 1e-5


def rel_err(got, ref):
    got = np.asarray(got).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / den) if den > 0 else float(np.linalg.norm(got))


def assert_parity(got, ref, tol=TOL, what=""):
    got = np.asarray(got).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    if ref.size == 0:
        return
    e = rel_err(got, ref)
    scale = np.abs(ref).max()
    emax = float(np.abs(got - ref).max())
    assert e <= tol, f"{what}: normwise relative error {e:.3e} > {tol:.0e}"
    assert emax <= tol * max(scale, 1e-30), f"{what}: max element error {emax:.3e} > {tol:.0e} * {scale:.3e}"


def header_functions(header="dpd.h"):
    """Names of the functions declared in include/<header> (the GPU library's
    dpd.h by default; dpd_cpu.h is the CPU library's)."""
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn != header:
            continue
        src = open(os.path.join(inc, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(dpd_\w+)\s*\(", src, flags=re.M)
    return names
