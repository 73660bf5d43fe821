"""Rotational K-SVD (Sec. II-C, R-K-SVD pseudocode of Fig. "code") driven
through the C ABI: each iteration codes the patches with rotational OMP
(rsc_encode) and updates every atom from the aligned residuals
(rsc_ksvd_update); a final OMP codes the patches with the last dictionary.
This module only sequences the calls and keeps the history; all arithmetic
runs in librsc's kernels."""
from __future__ import annotations

import numpy as np

from . import Dictionary, encode, ksvd_update


def learn(x, d0, R: int, K: int, iters: int, precision: str = "f16", callback=None):
    """x: CUDA float32 [P, kmax+1, J, 2] patches; d0: CUDA float32 initial
    unit-norm atoms [M, kmax+1, J, 2].  Returns (d, codes, history) with
    history[i] = {"iter", "mse", "unused"} where mse is the mean squared
    coding error per real coefficient before the i-th update."""
    import torch
    d = d0.contiguous()
    n = d.shape[2] * (2 * (d.shape[1] - 1) + 1)
    history = []
    for it in range(iters):
        dic = Dictionary(d, R)
        codes = encode(dic, x, K, precision)
        new, used = ksvd_update(dic, x, codes)
        torch.cuda.current_stream().synchronize()
        rec = {"iter": it, "mse": float(codes["resid_norm2"].double().mean().item()) / n,
               "unused": int((used == 0).sum().item())}
        history.append(rec)
        if callback:
            callback(rec, new)
        dic.close()
        d = new
    dic = Dictionary(d, R)
    codes = encode(dic, x, K, precision)
    torch.cuda.current_stream().synchronize()
    history.append({"iter": iters, "mse": float(codes["resid_norm2"].double().mean().item()) / n,
                    "unused": None})
    dic.close()
    return d, codes, history
