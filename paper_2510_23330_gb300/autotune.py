"""Choice of the group size n_g and the leaf size n_leaf on the data.

Sec. 5.2.2 and 5.2.4 of the paper: a larger n_g shortens the tree walk per
particle but lengthens the shared interaction list, and the best value depends
on the hardware (2048 on Fugaku, 65536 on a GH200).  The leaf size moves work
between the two lists: a larger n_leaf opens fewer, larger leaves (more
particle-particle terms, fewer particle-cell terms and tree nodes).  The
candidates are timed on the actual particles with the library's phase timers
and the fastest is kept in the context.
"""
from __future__ import annotations

from . import galnb

# phases a full force evaluation runs
_FORCE_PHASES = ("SORT", "TREE", "GRAVITY", "EXTERNAL", "HYDRO_TREE", "KNN", "FORCE")


def tune_group_size(ctx: "galnb.Context", mode: int = galnb.GNB_GRAV_TREE,
                    candidates=(32, 64, 128, 192, 256, 384, 512), repeats: int = 2):
    """Returns (best n_group, {n_group: ms per gravity evaluation}), tree
    build + gravity, at the context's n_leaf."""
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
    ctx.set_timing(False)
    return best, table


def tune_tree(ctx: "galnb.Context", mode: int = galnb.GNB_GRAV_TREE, leaves=(16, 32),
              groups=(128, 192, 256, 384), repeats: int = 2):
    """Joint choice of (n_leaf, n_group) by the time of a whole force
    evaluation (sort, trees, gravity, kernel size and density, hydro force),
    since the leaf size also shapes the hydro tree.  Returns
    ((n_leaf, n_group), {"n_leaf/n_group": ms per evaluation})."""
    ctx.set_timing(True)
    table = {}
    for nl in leaves:
        for ng in groups:
            ctx.set_params(n_leaf=int(nl), n_group=int(ng))
            ctx.compute_forces(mode)         # warm-up
            ctx.phase_times(reset=True)
            for _ in range(repeats):
                ctx.set_params(n_leaf=int(nl), n_group=int(ng))  # forces new trees
                ctx.compute_forces(mode)
            ms, calls, _ = ctx.phase_times(reset=True)
            k = max(calls["GRAVITY"], 1)
            table[(int(nl), int(ng))] = sum(ms[p] for p in _FORCE_PHASES) / k
    best = min(table, key=table.get)
    ctx.set_params(n_leaf=best[0], n_group=best[1])
    ctx.set_timing(False)
    return best, {f"{a}/{b}": v for (a, b), v in table.items()}
