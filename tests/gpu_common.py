"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np


def to_np(t):
    return t.detach().double().cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, float); b = np.asarray(b, float)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def max_rel(a, b, floor):
    """max |a - b| / max(|b|, floor)"""
    a = np.asarray(a, float); b = np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def state_to_torch(st, dtype, device="cuda"):
    import torch
    out = {}
    for k in ("u", "v", "a", "d"):
        out[k] = torch.tensor(np.asarray(st[k]), dtype=dtype, device=device).contiguous()
    out["H"] = torch.tensor(np.asarray(st["H"]), dtype=torch.float64, device=device).contiguous()
    return out
