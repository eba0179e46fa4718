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


def abs_operator(lmat):
    """|L| entry by entry (a copy of the scipy matrix with absolute values)."""
    a = lmat.copy()
    a.data = np.abs(a.data)
    return a


def assert_elementwise(got: np.ndarray, ref: np.ndarray, bound: np.ndarray, what: str = "") -> None:
    """|got - ref| <= bound element by element; the message names how many
    elements fail and the worst one relative to its own bound."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    bound = np.broadcast_to(np.asarray(bound, dtype=np.float64), got.shape)
    err = np.abs(got - ref)
    bad = ~(err <= bound)
    if bad.any():
        ratio = err / np.maximum(bound, 1e-300)
        i = np.unravel_index(int(np.argmax(np.where(np.isfinite(ratio), ratio, np.inf))), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {err.size} elements exceed their bound; worst at {i}: "
                             f"got {got[i]!r}, ref {ref[i]!r}, |diff| {err[i]:.3e} > bound {bound[i]:.3e}")


def spmm_bound(lmat, xin: np.ndarray, u: float, c: float = 2.0) -> np.ndarray:
    """Forward-error bound of Y = L X computed row by row in unit roundoff u:
    c (t_i + 6) u (|L| |X|)_ij with t_i the terms row i adds (its entries);
    the extra 6 covers the float coefficient and epilogue roundings."""
    terms = np.diff(lmat.indptr).astype(np.float64)
    return c * u * (terms + 6.0)[:, None] * (abs_operator(lmat) @ np.abs(xin))
