"""Helpers shared by the GPU parity tests (imported only by tests marked gpu)."""

from __future__ import annotations

import numpy as np


def torch_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def dev_block(x: np.ndarray, ld: int, dtype: str):
    """n x ld device block (zero padded) holding x (n x c) in the given dtype."""
    torch = torch_mod()
    n, c = x.shape
    t = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    out = torch.zeros((n, ld), dtype=t, device="cuda")
    out[:, :c] = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=t)
    return out


def to_np(t) -> np.ndarray:
    return t.detach().float().cpu().numpy().astype(np.float64) if t.dtype.is_floating_point and \
        t.dtype != __import__("torch").float64 else t.detach().cpu().numpy()


def bf16_round(x: np.ndarray) -> np.ndarray:
    torch = torch_mod()
    return torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)
