"""Host logic of the owner-computes partition, in one process: the slab cuts
and the pairing of every rank's halo plan with its neighbours' plans."""
import numpy as np
import pytest

import gen
from paper_2111_03541_gb300 import partition as pt


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_node_starts_are_balanced_whole_layers(world):
    n = 64
    layer = (n + 1) ** 2
    nn = (n + 1) ** 3
    s = pt.node_starts(nn, world, layer)
    assert s[0] == 0 and s[-1] == nn and len(s) == world + 1
    assert np.all(np.diff(s) >= 0)
    assert np.all(s[1:-1] % layer == 0)  # cuts between z-layers
    sizes = np.diff(s) // layer
    assert sizes.max() - sizes.min() <= 1


@pytest.mark.parametrize("world,form", [(2, "elastic"), (3, "elastic"), (4, "thermal")])
def test_halo_plans_pair_up(world, form):
    """What rank r sends to rank q is, node for node and in the same
    (ascending global) order, what q receives from r; a rank receives exactly
    the nodes of its local problem that it does not own."""
    n = 8
    prob = gen.elastic_problem(n) if form == "elastic" else gen.thermal_q1_problem(n)
    starts = pt.node_starts(prob["coords"].shape[0], world, (n + 1) ** 2)
    locs = [pt.local_problem(prob, starts, r) for r in range(world)]
    plans = [pt.halo_plan(prob["conn"], starts, r, locs[r]) for r in range(world)]
    for r in range(world):
        nodes = locs[r]["nodes"]
        own0, nown = locs[r]["own"]
        assert np.array_equal(nodes[own0:own0 + nown], np.arange(starts[r], starts[r + 1]))
        halo = np.setdiff1d(nodes, np.arange(starts[r], starts[r + 1]))
        got = np.sort(np.concatenate([nodes[v] for v in plans[r]["recv"].values()])) if plans[r]["recv"] else \
            np.empty(0, dtype=nodes.dtype)
        assert np.array_equal(got, halo)
        for q in range(world):
            if q == r:
                continue
            sent = locs[r]["nodes"][plans[r]["send"][q]] if q in plans[r]["send"] else np.empty(0, int)
            recvd = locs[q]["nodes"][plans[q]["recv"][r]] if r in plans[q]["recv"] else np.empty(0, int)
            assert np.array_equal(sent, recvd), (r, q)
            assert np.all(np.diff(sent) > 0)
