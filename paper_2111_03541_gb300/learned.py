"""Learned preconditioner correction: training data from the assembler,
training on the GPU by the library's BF16 kernels, and flexible CG.

Every arithmetic step (assembly, Jacobi-PCG, residuals, network forward and
backward, AdamW, flexible CG) runs in libmf's kernels; this module only
allocates buffers, draws the seeded inputs (``gen``) and loops.

Training systems: 3D thermal conduction on unjittered Q1 boxes of n^3 cells
(default 32^3) with k = exp(GRF) of correlation length 0.1 measured in units
of the 128^3 workload's domain (0.4 of a 32-cell box), f = 1, u = 0 on the
boundary.  Samples are the residuals r_k of Jacobi-PCG after 1, 2, 4, ..., 128
iterations with their errors e_k = x* - x_k = K^-1 r_k.  Loss: the share of
the error energy left after one optimally scaled step along the preconditioned
residual z, 1 - (z.Ke)^2 / ((z.Kz)(e.Ke)) (CG picks the step length, so the
scale of z does not matter), or the residual form ||K z - r||^2 / ||r||^2.
Iterates already converged to 1e-9 are not sampled (their error is round-off).
Training and validation systems use disjoint seeds.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

import gen

from . import (MF_PREC_FP64, MF_SOLVER_PCG, Problem, mf_axpby, mf_cnn_create, mf_cnn_destroy, mf_cnn_get_params,
               mf_cnn_input, mf_cnn_node_logk, mf_cnn_num_params, mf_cnn_train_step, mf_solve_fcg_cnn, mf_spmv)

LAYERS = [(2, 16), (16, 16), (16, 16), (16, 1)]
PCG_ITERS = (1, 2, 4, 8, 16, 32, 64, 128)
TRAIN_SEED0 = gen.SEED_GRF + 100_000
VALID_SEED0 = gen.SEED_GRF + 900_000


def init_params(seed: int = gen.SEED_CNN) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (27 ci))), zero biases; the last layer
    is scaled by 1e-2 so that the untrained correction is small."""
    parts = []
    offset = 0
    for li, (ci, co) in enumerate(LAYERS):
        nw = co * ci * 27
        w = gen.normal(seed, nw, offset) * np.sqrt(2.0 / (27 * ci))
        if li == len(LAYERS) - 1:
            w *= 1e-2
        offset += nw
        parts += [w, np.zeros(co)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == mf_cnn_num_params()
    return p


def save_params(path: str, params: np.ndarray, meta: dict) -> None:
    """Raw little-endian float32 parameters plus a JSON header next to them."""
    np.asarray(params, dtype="<f4").tofile(path)
    with open(path + ".json", "w") as f:
        json.dump(dict(meta, layers=LAYERS, n_params=int(params.size), dtype="float32-le"), f, indent=1)


def load_params(path: str) -> np.ndarray:
    p = np.fromfile(path, dtype="<f4")
    assert p.size == mf_cnn_num_params(), "parameter file does not match the network"
    return p


def grid_of(prob) -> tuple[int, int, int]:
    n = prob["n"] + 1
    return n, n, n


class Dataset:
    """Device-resident samples: per system its K values; per residual sample
    the residual (FP64) and the network input (BF16 pairs)."""

    def __init__(self, n_systems: int, n: int = 32, seed0: int = TRAIN_SEED0, corr_len: float = 0.4,
                 iters=PCG_ITERS, device="cuda"):
        import torch
        self.n = n
        base = gen.thermal_q1_problem(n, jitter=0.0, coef=np.ones(n ** 3))
        self.P = Problem(base, device=device)
        self.grid = grid_of(base)
        nv = self.P.n
        self.kvals, self.r, self.e, self.x, self.sys_of = [], [], [], [], []
        tmp = torch.empty(nv, dtype=torch.float64, device=device)
        logk = torch.empty(nv, dtype=torch.float32, device=device)
        for s in range(n_systems):
            kc = np.exp(gen.grf_cells(n, corr_len=corr_len, seed=seed0 + s))
            self.P.coef.copy_(torch.from_numpy(kc))
            self.P.assemble(MF_PREC_FP64)
            self.kvals.append(self.P.values.clone())
            mf_cnn_node_logk(*self.grid, self.P.coef, logk)
            xs, _, _ = self.P.solve(tol=1e-13, max_iter=100000)  # x*: errors of the iterates
            for it in iters:
                x, st, info = self.P.solve(tol=1e-14, max_iter=it, check_every=it)
                if info.rel_residual < 1e-9:
                    break  # converged: later iterates carry round-off only
                mf_spmv(self.P.csr, x, tmp)
                r = self.P.d.clone()
                mf_axpby(nv, -1.0, tmp, 1.0, r)
                e = xs.clone()
                mf_axpby(nv, -1.0, x, 1.0, e)  # e = x* - x_k = K^-1 r_k
                xin = torch.empty(2 * nv, dtype=torch.bfloat16, device=device)
                mf_cnn_input(nv, r, logk, xin)
                self.r.append(r)
                self.e.append(e)
                self.x.append(xin)
                self.sys_of.append(s)
        torch.cuda.synchronize()

    def __len__(self):
        return len(self.r)

    def batch(self, idx):
        return ([self.kvals[self.sys_of[i]] for i in idx], [self.r[i] for i in idx], [self.x[i] for i in idx],
                [self.e[i] for i in idx])


def loss_of(cnn, ds: Dataset, idx, energy: bool = True) -> float:
    kv, r, x, e = ds.batch(idx)
    nz, ny, nx = ds.grid
    return mf_cnn_train_step(cnn, nz, ny, nx, ds.P.csr, kv, r, x, ds.P.bc_mask, 0.0, 0.0, err=e if energy else None)


def train(train_ds: Dataset, valid_ds: Dataset, steps: int = 3000, batch: int = 16, lr: float = 2e-3,
          weight_decay: float = 1e-4, seed: int = gen.SEED_CNN, init=None, log=print, energy: bool = True):
    """AdamW on random minibatches (sample order drawn from the seeded stream);
    cosine learning-rate decay.  energy=True trains on the error energy left
    after one optimally scaled step, 1 - (z.Ke)^2 / ((z.Kz)(e.Ke)), else on the
    residual ||K z - r||^2 / ||r||^2.  Returns (cnn handle, history)."""
    cnn = mf_cnn_create(init_params(seed) if init is None else init)
    nz, ny, nx = train_ds.grid
    order = (gen.uniform(seed + 1, steps * batch) * len(train_ds)).astype(np.int64)
    vidx = list(range(len(valid_ds)))
    hist = []
    t0 = time.time()
    for k in range(steps):
        idx = order[k * batch:(k + 1) * batch]
        lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / steps))
        kv, r, x, e = train_ds.batch(idx)
        L = mf_cnn_train_step(cnn, nz, ny, nx, train_ds.P.csr, kv, r, x, train_ds.P.bc_mask, lr_k, weight_decay,
                              err=e if energy else None)
        if k % 200 == 0 or k == steps - 1:
            vl = np.mean([loss_of(cnn, valid_ds, vidx[i:i + batch], energy) for i in range(0, len(vidx), batch)])
            hist.append({"step": k, "train_loss": L, "valid_loss": float(vl), "s": time.time() - t0})
            log(f"step {k}: train {L:.4f} valid {vl:.4f} ({time.time() - t0:.0f}s)")
    return cnn, hist


def jacobi_loss(ds: Dataset, batch: int = 16, energy: bool = True) -> float:
    """Validation loss of the plain Jacobi step (the network output held at 0)."""
    p = init_params()
    p[:] = 0.0
    cnn = mf_cnn_create(p)
    idx = list(range(len(ds)))
    v = float(np.mean([loss_of(cnn, ds, idx[i:i + batch], energy) for i in range(0, len(idx), batch)]))
    mf_cnn_destroy(cnn)
    return v


def fcg(P: Problem, cnn, logk, tol: float = 1e-8, max_iter: int = 100000, x=None, m_dirs: int = 256):
    """Flexible CG with the network correction on a structured Q1 thermal
    problem; each direction is K-orthogonalised against the last m_dirs (the
    network is not a fixed linear operator, and truncated histories of 8 or 32
    directions stall on the 128^3 workload while 64 and more converge)."""
    import torch
    nz, ny, nx = grid_of(P.prob)
    if x is None:
        x = torch.zeros(P.n, dtype=torch.float64, device=P.device)
    st, info, fb = mf_solve_fcg_cnn(P.csr, P.d, x, cnn, nz, ny, nx, logk, P.bc_mask, tol, max_iter, m_dirs)
    return x, st, info, fb


def node_logk(P: Problem):
    import torch
    logk = torch.empty(P.n, dtype=torch.float32, device=P.device)
    mf_cnn_node_logk(*grid_of(P.prob), P.coef, logk)
    return logk


def main(argv=None):
    import argparse

    import torch
    ap = argparse.ArgumentParser(description="train the learned preconditioner correction")
    ap.add_argument("--systems", type=int, default=2000)
    ap.add_argument("--valid", type=int, default=64)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--loss", choices=("energy", "residual"), default="energy")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "cnn_q1_thermal.f32"))
    a = ap.parse_args(argv)
    t = time.time()
    tr = Dataset(a.systems, seed0=TRAIN_SEED0)
    va = Dataset(a.valid, seed0=VALID_SEED0)
    print(f"data: {len(tr)} train / {len(va)} valid samples in {time.time() - t:.0f}s", flush=True)
    energy = a.loss == "energy"
    jl = jacobi_loss(va, energy=energy)
    print(f"Jacobi-only validation loss {jl:.4f}", flush=True)
    cnn, hist = train(tr, va, steps=a.steps, batch=a.batch, lr=a.lr, log=lambda s: print(s, flush=True),
                      energy=energy)
    params = mf_cnn_get_params(cnn)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    save_params(a.out, params, {"systems": a.systems, "valid": a.valid, "steps": a.steps, "batch": a.batch,
                                "lr": a.lr, "loss": a.loss, "jacobi_valid_loss": jl, "history": hist})
    print(f"saved {a.out}", flush=True)
    mf_cnn_destroy(cnn)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
