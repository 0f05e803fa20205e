"""Host model of the fused kernel's balanced tile schedule (for_warp_tiles in
csrc/mst_single.cu): each warp runs its static tiles, then one fixed tile,
then tiles drawn from the phase's counter, taking the next ticket before it
works on the current tile.  Under any interleaving of the warps' draws every
tile must run exactly once, and phases with few tiles per warp must take no
ticket at all."""
import random

import pytest

K_NUM, K_DEN, DYN_MIN = 3, 4, 4  # kStaticShareNum, kStaticShareDen, kDynMinShare


def schedule(ntiles, nw, rng):
    small = ntiles < DYN_MIN * nw
    k_static = (ntiles + nw - 1) // nw if small else (ntiles * K_NUM) // (nw * K_DEN)
    dyn0 = k_static * nw
    counter = 0
    tickets = 0
    ran = []
    # per warp: (k, t); a warp's step = take ticket (if k >= k_static), run t, advance
    state = {gw: [0, gw if k_static else dyn0 + gw] for gw in range(nw)}
    live = [gw for gw in range(nw) if state[gw][1] < ntiles]
    while live:
        gw = rng.choice(live)
        k, t = state[gw]
        nx = None
        if k >= k_static:
            nx = counter
            counter += 1
            tickets += 1
        ran.append(t)
        k += 1
        if k < k_static:
            t = gw + k * nw
        elif k == k_static:
            t = dyn0 + gw
        else:
            t = nx + dyn0 + nw
        state[gw] = [k, t]
        if t >= ntiles:
            live.remove(gw)
    return ran, tickets, small


@pytest.mark.parametrize("ntiles,nw", [(0, 8), (1, 8), (7, 8), (8, 8), (31, 8), (32, 8),
                                       (33, 8), (100, 8), (1000, 8), (131072 // 64, 152),
                                       (4864 * 27, 4864), (5, 1), (64, 1)])
def test_every_tile_exactly_once(ntiles, nw):
    for seed in range(5):
        ran, tickets, small = schedule(ntiles, nw, random.Random(seed))
        assert sorted(ran) == list(range(ntiles))
        if small:
            assert tickets == 0
        else:  # about a quarter of the tiles, plus one overshooting draw per warp at most
            assert tickets <= ntiles - (ntiles * K_NUM) // (nw * K_DEN) * nw + nw
