"""Rotational K-SVD (Sec. II-C, R-K-SVD pseudocode of Fig. "code") driven
through the C ABI: each iteration codes the patches with rotational OMP
(rsc_encode) and updates every atom from the aligned residuals
(rsc_ksvd_update); a final OMP codes the patches with the last dictionary.
With patches spread over ranks, the update is rsc_ksvd_accumulate on each
rank, one exchange (an all-reduce of the per-atom covariances and counts, an
all-gather of the largest-error patches) and rsc_ksvd_finish.  This module
only sequences the calls, the collectives and the merge of a short list;
the arithmetic runs in librsc's kernels."""
from __future__ import annotations

import json
import os

import numpy as np

from . import KSVD_TOP, Dictionary, encode, ksvd_accumulate, ksvd_finish, ksvd_update


def merge_top(errs, gidxs, vecs, ntop: int = KSVD_TOP):
    """Host merge of the ranks' lists of largest-error patches (numpy): all
    valid entries (global index >= 0) in descending error, ties: smaller
    global index, the first ntop kept, padded with index -1 and zero
    vectors.  Returns (global indices [ntop] int64, vectors [ntop, ...])."""
    err = np.concatenate([np.asarray(e, np.float32) for e in errs])
    gid = np.concatenate([np.asarray(g, np.int64) for g in gidxs])
    vec = np.concatenate([np.asarray(v, np.float32) for v in vecs])
    ok = gid >= 0
    err, gid, vec = err[ok], gid[ok], vec[ok]
    order = np.lexsort((gid, -err.astype(np.float64)))[:ntop]
    out_idx = np.full(ntop, -1, np.int64)
    out_vec = np.zeros((ntop,) + vec.shape[1:], np.float32)
    out_idx[:order.size] = gid[order]
    out_vec[:order.size] = vec[order]
    return out_idx, out_vec


def _all_reduce_sum(t, group):
    """Sum of a CUDA tensor over the ranks of `group` (through host memory
    unless the group's backend is NCCL)."""
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        dist.all_reduce(t, group=group)
        return t
    h = t.cpu()
    dist.all_reduce(h, group=group)
    t.copy_(h)
    return t


def update_distributed(dic: Dictionary, x, codes: dict, group=None, offset: int = 0):
    """One R-K-SVD update with this rank's patches x (global indices start at
    `offset`) and codes: accumulate here, sum the covariances and counts over
    `group`, merge the largest-error lists, finish.  With group None it is
    the single-GPU update.  Returns (new atoms, n_used)."""
    import torch
    acc = ksvd_accumulate(dic, x, codes)
    if group is None:
        return ksvd_finish(dic, acc["C"], acc["count"], acc["top_idx"], acc["top_vec"])
    _all_reduce_sum(acc["C"], group)
    cnt = acc["count"].to(torch.int64)
    _all_reduce_sum(cnt, group)
    top_idx, top_vec = gather_top(acc["top_err"].cpu(), acc["top_idx"].cpu(),
                                  acc["top_vec"].cpu(), offset, group)
    dev = x.device
    return ksvd_finish(dic, acc["C"], cnt.to(torch.int32), torch.from_numpy(top_idx).to(dev),
                       torch.from_numpy(top_vec).to(dev))


def gather_top(err, idx, vec, offset: int, group):
    """All-gather of the ranks' largest-error lists (host tensors; local
    indices shifted by `offset` to global ones) and their merge."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gidx = torch.where(idx >= 0, idx + int(offset), idx)
    gathered = {}
    for k, v in (("err", err), ("gidx", gidx), ("vec", vec)):
        bufs = [torch.empty_like(v) for _ in range(world)]
        dist.all_gather(bufs, v.contiguous(), group=group)
        gathered[k] = [b.numpy() for b in bufs]
    return merge_top(gathered["err"], gathered["gidx"], gathered["vec"], ntop=int(err.shape[0]))


def save_checkpoint(path: str, d: np.ndarray, it: int, history: list, R: int, K: int):
    """Writes the loop's state after `it` updates (dictionary [M, kmax+1, J,
    2] float32, the iteration count, the history, R and K) to `path` (npz,
    written beside it and renamed, so a crash leaves the previous one)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, d=np.asarray(d, np.float32), iter=np.int64(it), R=np.int64(R), K=np.int64(K),
             history=np.array(json.dumps(history)))
    os.replace(tmp, path)


def load_checkpoint(path: str, R: int, K: int):
    """(dictionary, iterations done, history) from `path`; raises ValueError
    when it was written for another R or K."""
    with np.load(path, allow_pickle=False) as z:
        if int(z["R"]) != R or int(z["K"]) != K:
            raise ValueError(f"checkpoint {path} is for R={int(z['R'])}, K={int(z['K'])}")
        return z["d"].copy(), int(z["iter"]), json.loads(str(z["history"]))


def learn(x, d0, R: int, K: int, iters: int, precision: str = "f16", callback=None,
          group=None, offset: int = 0, checkpoint: str | None = None, resume: bool = False):
    """x: CUDA float32 [P, kmax+1, J, 2] patches; d0: CUDA float32 initial
    unit-norm atoms [M, kmax+1, J, 2].  Returns (d, codes, history) with
    history[i] = {"iter", "mse", "unused"} where mse is the mean squared
    coding error per real coefficient before the i-th update (this rank's
    patches).  With a process group, x holds this rank's patches (global
    indices from `offset`) and every rank ends with the same dictionary.

    checkpoint: a file written after every update with the dictionary, the
    iteration count and the history (save_checkpoint; give each rank its own
    file).  The loop draws no random numbers and its kernels give the same
    result on every run, so that is its whole state: with resume=True and an
    existing file, learning continues after the saved iteration and ends
    with the atoms of an uninterrupted run, bit for bit."""
    import torch
    d = d0.contiguous()
    n = d.shape[2] * (2 * (d.shape[1] - 1) + 1)
    history = []
    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        dn, start, history = load_checkpoint(checkpoint, R, K)
        if dn.shape != tuple(d.shape):
            raise ValueError(f"checkpoint {checkpoint} holds atoms of shape {dn.shape}")
        d = torch.from_numpy(dn).to(d.device)
    for it in range(start, iters):
        dic = Dictionary(d, R)
        codes = encode(dic, x, K, precision)
        if group is None:
            new, used = ksvd_update(dic, x, codes)
        else:
            new, used = update_distributed(dic, x, codes, group, offset)
        torch.cuda.current_stream().synchronize()
        rec = {"iter": it, "mse": float(codes["resid_norm2"].double().mean().item()) / n,
               "unused": int((used == 0).sum().item())}
        history.append(rec)
        if callback:
            callback(rec, new)
        dic.close()
        d = new
        if checkpoint:
            save_checkpoint(checkpoint, d.cpu().numpy(), it + 1, history, R, K)
    dic = Dictionary(d, R)
    codes = encode(dic, x, K, precision)
    torch.cuda.current_stream().synchronize()
    history.append({"iter": iters, "mse": float(codes["resid_norm2"].double().mean().item()) / n,
                    "unused": None})
    dic.close()
    return d, codes, history
