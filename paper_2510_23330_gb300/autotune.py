"""Choice of the group size n_g on the data.

Sec. 5.2.2 and 5.2.4 of the paper: a larger n_g shortens the tree walk per
particle but lengthens the shared interaction list, and the best value depends
on the hardware (2048 on Fugaku, 65536 on a GH200).  Here the candidates are
timed on the actual particles with the library's phase timers (tree build +
gravity kernel) and the fastest is kept in the context.
"""
from __future__ import annotations

from . import galnb


def tune_group_size(ctx: "galnb.Context", mode: int = galnb.GNB_GRAV_TREE,
                    candidates=(16, 32, 64, 128, 256), repeats: int = 2):
    """Returns (best n_group, {n_group: ms per gravity evaluation})."""
    was_timing = False
    ctx.set_timing(True)
    table = {}
    for ng in candidates:
        ctx.set_params(n_group=int(ng))
        ctx.compute_gravity(mode)           # warm-up (kernel attributes, caches)
        ctx.phase_times(reset=True)
        for _ in range(repeats):
            ctx.set_params(n_group=int(ng))  # forces a rebuild of tree and groups
            ctx.compute_gravity(mode)
        ms, calls, _ = ctx.phase_times(reset=True)
        k = max(calls["GRAVITY"], 1)
        table[int(ng)] = (ms["GRAVITY"] + ms["TREE"]) / k
    best = min(table, key=table.get)
    ctx.set_params(n_group=best)
    ctx.set_timing(was_timing)
    return best, table
