"""Shared parity rule between a GPU result and the FP64 oracle (test helper).

Rotational OMP is greedy, so several results can be correct when two scores
tie.  The rule (selection margin 1e-6 relative, coefficient tolerance per
path) is:

1. Free oracle run: at each step, if the exact top-two margin (s1 - s2)/s1
   exceeds ``margin``, the GPU pick (atom, angle) must equal the oracle's
   (and a stop must match a stop); at the first step whose margin is within
   it, the rest of that patch is unpinned.
2. Forced-path oracle run along the GPU's own picks: every GPU pick must score
   within ``margin`` (relative) of the best exact score of its step, and the
   GPU weights must match the FP64 least-squares weights of that path:
   ||a_gpu - a_ref|| <= coef_tol ||a_ref|| per patch.
3. The residual norm^2 matches the forced path within 1e-5 ||x||^2 (float32
   output).
"""
import numpy as np

import oracle


def check(x, d, R, K, gpu, coef_tol, margin=1e-6, nthreads=0):
    """gpu: dict of numpy arrays atom, angle_idx, coef, resid_norm2.  Returns a
    summary dict; raises AssertionError on a violation."""
    x = np.asarray(x, np.float32)
    ga = np.asarray(gpu["atom"]).reshape(-1, K)
    gr = np.asarray(gpu["angle_idx"]).reshape(-1, K)
    gc = np.asarray(gpu["coef"]).reshape(-1, K)
    gn = np.asarray(gpu["resid_norm2"]).reshape(-1)
    P = x.shape[0]
    free = oracle.romp(x, d, R, K, nthreads=nthreads)
    forced = oracle.romp(x, d, R, K, nthreads=nthreads, forced_atom=ga, forced_angle=gr)
    xn2 = np.einsum("phjc,phjc->p", x.astype(np.float64), x.astype(np.float64)) * 2 - \
        np.einsum("pjc,pjc->p", x[:, 0].astype(np.float64), x[:, 0].astype(np.float64))
    pinned_steps = 0
    unpinned_patches = 0
    max_coef_err = 0.0
    for p in range(P):
        # 1. selections where the oracle's margin pins them
        for t in range(K):
            fa, fr = free["atom"][p, t], free["angle"][p, t]
            if fa < 0:
                assert ga[p, t] < 0, (p, t, "oracle stopped, GPU did not")
                pinned_steps += 1
                continue
            if free["margin"][p, t] <= margin:
                unpinned_patches += 1
                break
            assert ga[p, t] == fa and gr[p, t] == fr, (
                p, t, (ga[p, t], gr[p, t]), (fa, fr), free["margin"][p, t])
            pinned_steps += 1
        # 2. forced path: each GPU pick within the margin of the best score
        for t in range(K):
            if ga[p, t] < 0:
                assert np.all(ga[p, t:] < 0) and np.all(gr[p, t:] < 0), (p, t)
                assert np.all(gc[p, t:] == 0.0), (p, t)
                # a stop is legitimate when nothing scores above the stop level
                stop_level = oracle.STOP_REL * np.sqrt(max(xn2[p], 0.0))
                assert forced["best_score"][p, t] <= stop_level * 1.01 + 1e-300, (
                    p, t, forced["best_score"][p, t], stop_level)
                break
            bs, ps = forced["best_score"][p, t], forced["pick_score"][p, t]
            assert ps >= bs * (1.0 - margin) - 1e-300, (p, t, ps, bs)
            assert forced["atom"][p, t] == ga[p, t], (p, t, "forced path stopped (degenerate)")
        ref = forced["coef"][p]
        nref = np.linalg.norm(ref)
        err = np.linalg.norm(gc[p] - ref)
        assert err <= coef_tol * max(nref, 1e-300) or err == 0.0, (p, err, nref, gc[p], ref)
        if nref > 0:
            max_coef_err = max(max_coef_err, err / nref)
        # 3. residual norm
        assert abs(gn[p] - forced["rn2"][p]) <= 1e-5 * max(xn2[p], 1e-30) + 1e-30, (
            p, gn[p], forced["rn2"][p])
    return {"patches": P, "pinned_steps": pinned_steps, "unpinned_patches": unpinned_patches,
            "max_rel_coef_err": max_coef_err}
