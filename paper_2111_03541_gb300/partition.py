"""Owner-computes partition of one mesh over ranks (one process per GPU).

Rank r owns the contiguous node range [starts[r], starts[r + 1]); on the
lexicographic structured boxes (x fastest, z slowest) these are z-slabs.
Its local problem holds every element that touches an owned node (the owned
elements plus one ghost layer) and every node of those elements, numbered in
ascending global order: the halo nodes below, the owned nodes, the halo
nodes above.  Every row of an owned node is then complete locally, so the
assembly needs no exchange (each CSR row is summed from the same elements in
the same ascending order as on one domain, hence bit for bit the same), and
a Krylov iteration needs one halo exchange of the search direction per SpMV
plus all-reduces of its scalars.

Host logic only (numpy index work and torch.distributed point-to-point
calls); the assembly and the SpMV are the library's kernels.
"""
from __future__ import annotations

import numpy as np


def node_starts(n_nodes: int, world: int, layer: int = 1) -> np.ndarray:
    """Balanced contiguous node ranges, cut at multiples of `layer` nodes (a
    z-layer of a structured box keeps the slabs whole)."""
    layers = -(-n_nodes // layer)
    cuts = [min(n_nodes, (layers * r // world) * layer) for r in range(world + 1)]
    cuts[-1] = n_nodes
    return np.array(cuts, dtype=np.int64)


def local_problem(prob: dict, starts: np.ndarray, rank: int) -> dict:
    """The rank's local problem (a problem dict of the same form) with the
    partition metadata: 'nodes' (global ids of the local nodes, ascending),
    'elems' (global ids of the local elements), 'own' (first local node and
    count of the owned nodes), 'dofs_per_node'."""
    conn = np.asarray(prob["conn"])
    n0, n1 = int(starts[rank]), int(starts[rank + 1])
    touch = ((conn >= n0) & (conn < n1)).any(axis=1)
    elems = np.nonzero(touch)[0]
    nodes = np.unique(conn[elems])
    lconn = np.searchsorted(nodes, conn[elems]).astype(np.int32)
    k = 3 if prob["form"] == "elastic" else 1
    dofs = (k * nodes[:, None] + np.arange(k)[None, :]).ravel()
    own0 = int(np.searchsorted(nodes, n0))
    loc = dict(prob)
    loc.update(coords=np.ascontiguousarray(prob["coords"][nodes]), conn=lconn,
               coef=np.ascontiguousarray(np.asarray(prob["coef"])[elems]),
               bc_mask=np.ascontiguousarray(np.asarray(prob["bc_mask"])[dofs]),
               bc_val=np.ascontiguousarray(np.asarray(prob["bc_val"])[dofs]),
               nodes=nodes, elems=elems, own=(own0, n1 - n0), dofs_per_node=k)
    loc.pop("facets", None)
    return loc


def owned_rows(loc: dict, row_ptr, col, val, d):
    """The owned rows of a locally assembled CSR system, columns in global dof
    numbers: (row_ptr (from 0), col, val, d) of dofs starting at the first
    owned dof."""
    k = loc["dofs_per_node"]
    own0, nown = loc["own"]
    r0, r1 = k * own0, k * (own0 + nown)
    rp = np.asarray(row_ptr)
    s0, s1 = int(rp[r0]), int(rp[r1])
    lcol = np.asarray(col)[s0:s1]
    gcol = k * loc["nodes"][lcol // k] + lcol % k
    return rp[r0:r1 + 1] - s0, gcol.astype(np.int64), np.asarray(val)[s0:s1], np.asarray(d)[r0:r1]


def halo_plan(conn: np.ndarray, starts: np.ndarray, rank: int, loc: dict) -> dict:
    """For one rank: which local nodes it receives from each other rank
    (halo) and which owned nodes it sends to each (their halo), as local node
    indices in ascending global order on both sides."""
    world = len(starts) - 1
    nodes = loc["nodes"]
    owner = np.searchsorted(starts, nodes, side="right") - 1
    recv = {int(q): np.nonzero(owner == q)[0] for q in range(world) if q != rank and np.any(owner == q)}
    # the owned nodes another rank needs: those sharing an element with its
    # owned range (exactly its halo from this rank)
    send = {}
    conn = np.asarray(conn)
    n0, n1 = int(starts[rank]), int(starts[rank + 1])
    for q in range(world):
        if q == rank:
            continue
        q0, q1 = int(starts[q]), int(starts[q + 1])
        touch_q = ((conn >= q0) & (conn < q1)).any(axis=1)
        need = np.unique(conn[touch_q])
        mine = need[(need >= n0) & (need < n1)]
        if mine.size:
            send[q] = np.searchsorted(nodes, mine)
    return {"recv": recv, "send": send}


class HaloExchange:
    """Exchanges the halo entries of a local vector (dofs_per_node entries per
    node) with torch.distributed point-to-point calls: every rank posts its
    receives and sends to all neighbours at once (isend/irecv), then waits.
    Works on CPU tensors under gloo and on GPU tensors under NCCL."""

    def __init__(self, plan: dict, dofs_per_node: int, device):
        import torch
        k = dofs_per_node

        def dof_index(nidx):
            return torch.as_tensor((k * nidx[:, None] + np.arange(k)[None, :]).ravel(), dtype=torch.long,
                                   device=device)

        self.recv = {q: dof_index(v) for q, v in sorted(plan["recv"].items())}
        self.send = {q: dof_index(v) for q, v in sorted(plan["send"].items())}

    def __call__(self, x):
        import torch
        import torch.distributed as dist
        bufs_out = {q: x.index_select(0, idx).contiguous() for q, idx in self.send.items()}
        bufs_in = {q: torch.empty(idx.numel(), dtype=x.dtype, device=x.device) for q, idx in self.recv.items()}
        reqs = [dist.isend(b, q) for q, b in bufs_out.items()] + [dist.irecv(b, q) for q, b in bufs_in.items()]
        for r in reqs:
            r.wait()
        for q, idx in self.recv.items():
            x.index_copy_(0, idx, bufs_in[q])
        return x


def dist_pcg(spmv_owned, dinv_owned, d_owned, n_local: int, own_slice: slice, exchange, tol: float,
             max_iter: int, device=None, dtype=None):
    """Jacobi-PCG on the distributed system: spmv_owned(x_local) returns K x
    on the owned rows from a local vector whose halo entries are current;
    dots are summed over ranks with all_reduce.  Returns (x_owned,
    iterations, relative residual of the recursion)."""
    import torch
    import torch.distributed as dist

    def dot(a, b):
        t = torch.dot(a, b).reshape(1)
        dist.all_reduce(t)
        return t[0]

    x = torch.zeros_like(d_owned)
    r = d_owned.clone()
    z = dinv_owned * r
    p_loc = torch.zeros(n_local, dtype=d_owned.dtype, device=d_owned.device)
    p_loc[own_slice] = z
    rz = dot(r, z)
    dd = dot(d_owned, d_owned)
    rr = dot(r, r)
    it = 0
    while it < max_iter and rr > tol * tol * dd:
        exchange(p_loc)
        q = spmv_owned(p_loc)
        alpha = rz / dot(p_loc[own_slice], q)
        x += alpha * p_loc[own_slice]
        r -= alpha * q
        z = dinv_owned * r
        rz_new = dot(r, z)
        rr = dot(r, r)
        beta = rz_new / rz
        rz = rz_new
        p_loc[own_slice] = z + beta * p_loc[own_slice]
        it += 1
    return x, it, float((rr / dd).sqrt())
