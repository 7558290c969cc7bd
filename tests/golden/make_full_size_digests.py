"""Writes ``full_size_digests.json``: SHA-256 digests of the CPU oracle's
output on the full-size workloads, so that GPU tests and the benchmark can
compare complete outputs bit for bit without re-running the oracle (minutes of
CPU time) on the GPU machine.

Only ``oracle/`` computes anything here; ``paper_1503_06029_gb300.inputs``
supplies the seeded inputs (it holds none of the method's arithmetic).

Workloads:
  * chains: l = 1024 bits (16 x uint64), 2^18 Bernoulli(1/2) seeds with
    15-step single-flip chains, 25 % duplicated, N = 5,242,880, seed 3;
  * batch: the 1,024 scenes of ``inputs.scene_batch_spec()`` (3-D planes,
    l log-uniform in 8..256, N log-uniform in 1e3..1e6, seed 4), 64-bit words;
    the serving stream draws its requests from the first of these scenes;
  * planes_3d (l = 64, N = 2^24, seed 2) and lines_2d (l = 16, N = 20,000,
    seed 1, 32-bit words);
  * spheres_3d: l = 64 spheres as quadric constraints, N = 2^24, seed 13.

Digest convention (shared with the checks that read the file): the cells are
hashed as their little-endian words, row-major [U][W] (W words of word_bits
bits), the edges as little-endian uint32 pairs [E][2] in canonical (i, j)
order; cells and edges have separate digests.

Run: ``python tests/golden/make_full_size_digests.py [--jobs J]``. The oracle
is single-threaded; scenes are spread over J worker processes. ``--only
NAME`` recomputes one of the single-workload entries (planes_3d, lines_2d,
chains, spheres_3d) and keeps the others.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "full_size_digests.json")


def digest(arr) -> str:
    import numpy as np

    return hashlib.sha256(np.ascontiguousarray(arr).tobytes()).hexdigest()


def _entry(cells, edges, **extra) -> dict:
    return {**extra, "n_cells": int(cells.shape[0]), "n_edges": int(edges.shape[0]),
            "cells_sha256": digest(cells), "edges_sha256": digest(edges)}


def _scene_job(s: int) -> dict:
    import oracle
    from paper_1503_06029_gb300 import inputs

    spec = inputs.scene_batch_spec()
    sc = inputs.batch_scene(spec, s)
    cells, edges = oracle.build(sc.pts, sc.a, sc.b, 64)
    return _entry(cells, edges, scene=s, ell=int(spec.ell[s]), n=int(spec.n[s]))


def _chains_job(_=None) -> dict:
    import oracle
    from paper_1503_06029_gb300 import inputs

    ch = inputs.chains()
    cells = oracle.dedup(ch.keys, 1024, 64)
    edges = oracle.neighbors(cells, 1024, 64)
    return _entry(cells, edges, ell=1024, n=int(ch.keys.shape[0]), seed=3)


def _spheres_job(_=None) -> dict:
    import oracle
    from paper_1503_06029_gb300 import inputs

    sc = inputs.spheres_3d()
    cells, edges = oracle.build_quadric(sc.pts, sc.q, sc.a, sc.b, 64)
    return _entry(cells, edges, ell=int(sc.ell), n=int(sc.n), seed=13, word_bits=64)


def _plain_job(name: str) -> dict:
    import oracle
    from paper_1503_06029_gb300 import inputs

    if name == "planes_3d":
        sc, wb, seed = inputs.planes_3d(), 64, 2
    else:
        sc, wb, seed = inputs.lines_2d(), 32, 1
    cells, edges = oracle.build(sc.pts, sc.a, sc.b, wb)
    return _entry(cells, edges, ell=int(sc.a.shape[0]), n=int(sc.pts.shape[0]), seed=seed,
                  word_bits=wb)


SINGLE = ("convention", "planes_3d", "lines_2d", "chains", "spheres_3d", "batch")


def _write(out: dict, scenes_out: list) -> None:
    with open(OUT, "w") as f:
        # One line per record keeps the file diffable.
        f.write("{\n")
        for k in SINGLE:
            if k in out:
                f.write(f"{json.dumps(k)}: {json.dumps(out[k], sort_keys=True)},\n")
        f.write('"batch_scenes": [\n')
        f.write(",\n".join(json.dumps(e, sort_keys=True) for e in scenes_out))
        f.write("\n]\n}\n")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--only", choices=["planes_3d", "lines_2d", "chains", "spheres_3d"])
    args = ap.parse_args()
    import oracle

    oracle.compile_library()
    t0 = time.time()
    if args.only:
        with open(OUT) as f:
            out = json.load(f)
        job = {"chains": _chains_job, "spheres_3d": _spheres_job}.get(args.only)
        out[args.only] = job() if job else _plain_job(args.only)
        _write(out, out.pop("batch_scenes"))
        print(f"updated {args.only} in {OUT} in {time.time() - t0:.0f} s")
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        chains = pool.apply_async(_chains_job)
        plain = {k: pool.apply_async(_plain_job, (k,)) for k in ("planes_3d", "lines_2d")}
        # Largest scenes first, so the pool ends evenly.
        from paper_1503_06029_gb300 import inputs

        spec = inputs.scene_batch_spec()
        order = sorted(range(len(spec.n)), key=lambda s: -int(spec.n[s]) * int(spec.ell[s]))
        scenes = {s: pool.apply_async(_scene_job, (s,)) for s in order}
        batch = [scenes[s].get() for s in range(len(spec.n))]
        spheres = pool.apply_async(_spheres_job)
        out = {
            "convention": "sha256 of little-endian cells [U][W] words and of uint32 edges "
                          "[E][2] in canonical (i, j) order, from the CPU oracle",
            "planes_3d": plain["planes_3d"].get(),
            "lines_2d": plain["lines_2d"].get(),
            "batch": {"seed": 4, "word_bits": 64},
            "chains": chains.get(),
            "spheres_3d": spheres.get(),
        }
    _write(out, batch)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
