"""Shared helpers of the GPU tests (imports torch and the CUDA binding lazily)."""
import numpy as np


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


# Tolerances on the relative L2 error against the FP64 oracle, per form.
# FP32 / TF32x3 forms: 1e-5 and BF16x3: 1e-3 (the stated accuracy targets).
# FP64 form: its output is rounded to float32, so the floor is the float32
# unit roundoff 2^-24 ~ 6e-8 per entry; 2e-7 leaves room for the input cast.
TOL = {"fp64": 2e-7, "fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-3}
