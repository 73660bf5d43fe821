"""Autotuner of the FP16 coding path: measures each candidate tuning (stream
groups, refine blocks per SM, depth of the scoring kernel's dictionary ring)
with CUDA events on a synthetic workload of the given sizes and writes the
fastest per (n, M, R, K) to the table librsc reads when a dictionary is
created (rsc_tuning.txt beside librsc.so; see include/rsc.h, "Tuning").

A tuning never changes a result, so a candidate is judged on time alone.

Usage (on the GPU):
    python -m paper_1806_04374_gb300.autotune [--workload NAME ...] [--out PATH]
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import time

import numpy as np

import paper_1806_04374_gb300 as rsc
from paper_1806_04374_gb300 import synth

# the coder sizes of the workloads (J, kmax, M, R, K, patches timed)
WORKLOADS = {
    "omp_small": (6, 8, 16, 32, 3, 200_000),
    "omp_1m": (6, 8, 64, 64, 5, 1_000_000),
    "serve_11x11": (6, 8, 128, 64, 5, 400_000),
    "images_21x21": (10, 12, 256, 128, 8, 400_000),
}
TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rsc_tuning.txt")


def stage_options(dic) -> list[int]:
    """The ring depths the dictionary's layout is built with, default first
    (found by asking librsc to set each depth; clears the dictionary's tuning
    overrides)."""
    rsc.rsc_dict_set_tuning(dic.handle, clear=True)
    dflt = rsc.rsc_dict_tuning(dic.handle, 1)["score_stages"]
    out = [dflt]
    for s in range(2, 7):
        if s == dflt:
            continue
        try:
            rsc.rsc_dict_set_tuning(dic.handle, score_stages=s)
            out.append(s)
        except rsc.RscError:
            pass
    rsc.rsc_dict_set_tuning(dic.handle, clear=True)
    return out


def candidates(dic) -> list[dict]:
    """The grid searched: groups 1-3, refine blocks per SM 8/16/32, both ring
    depths the dictionary's layout is built with."""
    stages = stage_options(dic)
    return [{"groups": g, "refine_blocks_per_sm": b, "score_stages": s}
            for g, b, s in itertools.product((1, 2, 3), (8, 16, 32), stages)]


def time_encode(dic, xd, K, reps: int) -> float:
    """Milliseconds per rsc_encode (FP16 path), median of `reps` calls timed
    with CUDA events after one warm-up call."""
    import torch
    rsc.encode(dic, xd, K, "f16")
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        rsc.encode(dic, xd, K, "f16")
        ev[1].record()
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
    return float(np.median(ms))


def tune(name: str, reps: int = 3) -> dict:
    """Times every candidate on `name`'s sizes; returns the table entry of the
    fastest and every measurement."""
    import torch
    J, kmax, M, R, K, P = WORKLOADS[name]
    d = synth.make_dictionary(M, J, kmax, 20180901)
    x, _ = synth.make_patches(d, P, 3, 0.1, 20180902)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
    xd = torch.from_numpy(x).cuda()
    results = []
    for c in candidates(dic):
        rsc.rsc_dict_set_tuning(dic.handle, **c)
        results.append(dict(c, ms=time_encode(dic, xd, K, reps)))
    rsc.rsc_dict_set_tuning(dic.handle, clear=True)
    dic.close()
    best = min(results, key=lambda r: r["ms"])
    n = J * (2 * kmax + 1)
    return {"workload": name, "n": n, "M": M, "R": R, "K": K, "patches": P,
            "best": best, "default_ms": next(r["ms"] for r in results
                                             if r["groups"] == 2 and r["refine_blocks_per_sm"] == 32
                                             and r["score_stages"] == results[0]["score_stages"]),
            "results": results}


def table_lines(entries) -> list[str]:
    """Lines of the table format librsc reads (n M R K groups group_min
    refine_blocks_per_sm score_stages), with the measurement as a comment."""
    out = []
    for e in entries:
        b = e["best"]
        out.append(f"{e['n']} {e['M']} {e['R']} {e['K']} {b['groups']} 0 "
                   f"{b['refine_blocks_per_sm']} {b['score_stages']}"
                   f"  # {e['workload']}: {b['ms']:.3f} ms per call of {e['patches']} patches "
                   f"(default {e['default_ms']:.3f} ms)")
    return out


def write_table(path: str, entries, device_name: str = "") -> None:
    head = ["# librsc tuning table: n M R K groups group_min refine_blocks_per_sm score_stages",
            f"# written by paper_1806_04374_gb300.autotune on {device_name} "
            f"({time.strftime('%Y-%m-%d')}); 0 = default"]
    with open(path, "w") as f:
        f.write("\n".join(head + table_lines(entries)) + "\n")


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", nargs="*", default=list(WORKLOADS))
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--json", default=None, help="also write every measurement here")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    rsc.load_library()
    entries = [tune(w, args.reps) for w in args.workload]
    write_table(args.out, entries, torch.cuda.get_device_name(0))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(entries, f, indent=1)
    for e in entries:
        print(e["workload"], "best", e["best"], "default %.3f ms" % e["default_ms"])


if __name__ == "__main__":
    main()
