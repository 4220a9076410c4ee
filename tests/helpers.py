"""Shared test helpers: tolerance grading and tensor transfer."""
import numpy as np

# Tolerances stated by the method's accuracy targets: P_l within 1e-5 of the
# FP64 oracle, graded against max(|X_oracle|, raw monopole <|F_0|^2>/I_22)
# because P_2, P_4 (and P_0 after shot-noise subtraction) cross zero.
P_TOL = 1e-5


def p_errors(got, ref, keys=("P0", "P2", "P4", "P4b")):
    """Per-key max error relative to max(|ref|, raw monopole) over bins with modes."""
    m = ref["nmodes"] > 0
    den = np.maximum(np.abs(ref["P0"][m]), np.abs(ref["mono_raw"][m]))
    out = {}
    for k in keys:
        d = np.maximum(np.abs(ref[k][m]), den)
        out[k] = float(np.max(np.abs(got[k][m] - ref[k][m]) / d))
    return out


def to_device(cat, device="cuda"):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in cat.items() if v is not None}
