"""Owner-computes partition over ranks (multi-GPU design), run as CPU
processes under gloo: each rank assembles its local problem (owned nodes'
elements plus one ghost layer) with the oracle, and its owned rows must equal
the single-domain rows bit for bit (pattern, values, right-hand side); a
distributed Jacobi-PCG with a halo exchange per SpMV and all-reduced scalars
must reach the single-domain solution."""
import os
import socket

import numpy as np
import pytest

import gen


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, form):
    import scipy.sparse as sp
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2111_03541_gb300 import partition as pt
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if form == "elastic_box":  # the weak-scaling workload: cubes stacked along z
            prob = gen.elastic_box_problem(n, n, n * world)
        else:
            prob = gen.elastic_problem(n) if form == "elastic" else gen.thermal_q1_problem(n)
        layer = (n + 1) * (n + 1)
        starts = pt.node_starts(prob["coords"].shape[0], world, layer)
        loc = pt.local_problem(prob, starts, rank)
        g = oracle.assemble(prob)
        l = oracle.assemble(loc)
        rp, col, val, d = pt.owned_rows(loc, l["row_ptr"], l["col"], l["val"], l["d"])
        k = loc["dofs_per_node"]
        r0 = k * int(starts[rank])
        r1 = k * int(starts[rank + 1])
        grp = g["row_ptr"][r0:r1 + 1]
        assert np.array_equal(rp, grp - grp[0]), "row pointers"
        assert np.array_equal(col, g["col"][grp[0]:grp[-1]]), "columns"
        assert np.array_equal(val, g["val"][grp[0]:grp[-1]]), "values (bit for bit)"
        assert np.array_equal(d, g["d"][r0:r1]), "right-hand side (bit for bit)"
        # distributed PCG on the owned rows (local columns)
        own0, nown = loc["own"]
        lrp = np.asarray(l["row_ptr"])
        s0, s1 = lrp[k * own0], lrp[k * (own0 + nown)]
        n_local = k * loc["nodes"].shape[0]
        Kown = sp.csr_matrix((l["val"][s0:s1], l["col"][s0:s1], lrp[k * own0:k * (own0 + nown) + 1] - s0),
                             shape=(k * nown, n_local))
        diag = np.array([Kown[i, k * own0 + i] for i in range(k * nown)])
        plan = pt.halo_plan(prob["conn"], starts, rank, loc)
        ex = pt.HaloExchange(plan, k, "cpu")

        def spmv(xl):
            return torch.from_numpy(Kown @ xl.numpy())

        x, its, rel = pt.dist_pcg(spmv, torch.from_numpy(1.0 / diag), torch.from_numpy(d.copy()), n_local,
                                  slice(k * own0, k * (own0 + nown)), ex, 1e-12, 100000)
        xg, _, _ = oracle.pcg(g, tol=1e-13, maxit=100000)
        xo = xg[r0:r1]
        num = torch.tensor([float(np.sum((x.numpy() - xo) ** 2)), float(np.sum(xg[r0:r1] ** 2))],
                           dtype=torch.float64)
        dist.all_reduce(num)
        err = float(np.sqrt(num[0] / num[1]))
        assert err <= 1e-8, err
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,form,n", [(2, "elastic", 6), (3, "elastic", 6), (2, "thermal", 9),
                                          (2, "elastic_box", 4)])
def test_partitioned_assembly_and_pcg(world, form, n):
    import torch.multiprocessing as tmp
    tmp.spawn(_rank_main, args=(world, _free_port(), n, form), nprocs=world, join=True)
