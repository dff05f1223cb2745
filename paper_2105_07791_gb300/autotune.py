"""Tile-shape autotuner of the 32-column apply (ndhss_apply_multi).

Times the multi apply of the 64-problem Helmholtz batch (uneven P1 grids of
64..256 cells, leaf 64) for every assignment of tile rows (32 or 64) to the
four front-size buckets of csrc/mapply_tune.h, through NDHSS_MAPPLY_TILES,
and writes the fastest assignment into that header (rebuild afterwards):

    python -m paper_2105_07791_gb300.autotune [--write]

`current_table()` reads the committed table (the bench prints it).
"""
from __future__ import annotations

import argparse
import itertools
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "mapply_tune.h")


def current_table() -> dict:
    txt = open(HEADER).read()
    edges = [int(v) for v in re.search(r"MAPPLY_BUCKET_EDGES\[[^\]]*\]\s*=\s*\{([^}]*)\}", txt).group(1).split(",")]
    rows = [int(v) for v in re.search(r"MAPPLY_TILE_ROWS\[[^\]]*\]\s*=\s*\{([^}]*)\}", txt).group(1).split(",")]
    names = [f"rows < {edges[0]}"] + [f"{a} <= rows < {b}" for a, b in zip(edges, edges[1:])] + [f"rows >= {edges[-1]}"]
    return {"bucket_edges": edges, "tile_rows": dict(zip(names, rows))}


def tune(reps: int = 10):
    import numpy as np
    import torch

    from ndhss_inputs import helmholtz_batch
    from paper_2105_07791_gb300 import ndhss

    ndhss.load()
    probs = helmholtz_batch(64, 0, nmin=64, nmax=256, nsrc=32)
    tree = ndhss.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices) for P in probs], 64)
    A, _ = ndhss.batch_csr([P.A for P in probs])
    M = ndhss.DeviceCSR(A)
    n = A.shape[0]
    X = torch.randn((n, 32), dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    opts = ndhss.make_factor_opts(prec=ndhss.NDHSS_FP32, hss_levels=-1)
    results = []
    for combo in itertools.product((32, 64), repeat=4):
        os.environ["NDHSS_MAPPLY_TILES"] = ",".join(str(v) for v in combo)
        f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts)
        for _ in range(2):
            ndhss.ndhss_apply_multi(f, X, Y)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ndhss.ndhss_apply_multi(f, X, Y)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        del f
        results.append((float(np.median(ts)), combo))
        print("tiles %s: %.3f ms" % (combo, results[-1][0]), flush=True)
    os.environ.pop("NDHSS_MAPPLY_TILES", None)
    results.sort()
    return results


def write_header(best: tuple, results: list) -> None:
    txt = open(HEADER).read()
    txt = re.sub(r"(MAPPLY_TILE_ROWS\[[^\]]*\]\s*=\s*\{)[^}]*(\})", lambda m: m.group(1) + ", ".join(str(v) for v in best) + m.group(2), txt)
    open(HEADER, "w").write(txt)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true", help="write the fastest assignment into csrc/mapply_tune.h")
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args()
    results = tune(a.reps)
    best_ms, best = results[0]
    worst_ms, worst = results[-1]
    print("fastest", best, "%.3f ms; slowest" % best_ms, worst, "%.3f ms" % worst_ms)
    if a.write:
        write_header(best, results)
        print("wrote", HEADER)


if __name__ == "__main__":
    main()
