"""Tile autotuner of the batched step.

A batched step concatenates every system's grid in one launch per stage.
Its one free shape parameter is the tile: how many blocks the per-atom
kernels give one system at most (the blocks then walk that system's atoms
grid-stride).  The default (0) is the single-context grid; smaller tiles
put more atoms on each block, trading parallelism inside a large system for
fewer, fuller blocks across many small ones.  No setting changes a result:
those kernels carry no reduction and the pass with the CV sums keeps a grid
fixed by the atom count, so every system stays bit-identical to stepping it
alone.

`tune_batch` times each candidate over a few batched steps of the caller's
own inputs with CUDA events on the batch's stream and keeps the fastest.
The steps it runs deposit nothing and reuse the same positions, so they
change no state (the neighbour lists are not rebuilt).
"""
from __future__ import annotations

import torch

DEFAULT_CANDIDATES = (0, 2432, 1216, 608, 304, 152)


def tune_batch(batch, pos_list, force_list, stream: torch.cuda.Stream, candidates=DEFAULT_CANDIDATES,
               steps: int = 3, warmup: int = 1) -> dict:
    """Time each tile candidate; set and return the fastest.

    Returns {"tile": best, "ms_per_step": {tile: ms}}."""
    timings = {}
    with torch.cuda.stream(stream):
        for cand in candidates:
            batch.set_tile(int(cand))
            for _ in range(warmup):
                batch.step(pos_list, force_list)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                batch.step(pos_list, force_list)
            e1.record(stream)
            e1.synchronize()
            timings[int(cand)] = e0.elapsed_time(e1) / steps
    best = min(timings, key=lambda c: (timings[c], c != 0))
    batch.set_tile(best)
    return {"tile": best, "ms_per_step": timings}


def tile_table(results) -> str:
    """One line per tuned batch: tile and ms per step of each candidate."""
    lines = []
    for name, r in results.items():
        cells = " ".join(f"{c}:{v:.3f}" for c, v in sorted(r["ms_per_step"].items()))
        lines.append(f"{name}: best {r['tile']}  ({cells})")
    return "\n".join(lines)

