"""Batched assembly (many uneven thermal problems, mixed P1/P2/Q1) on the GPU.

Each problem's K and d from the batched persistent launches must be bitwise
equal to the single-problem path, which the parity tests tie to the oracle;
a few problems are also compared with the oracle directly.
"""
import json
import os

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_03541_gb300 as mf
    mf.lib()
    return mf


def small_specs(n=24):
    # the batched workload's generator, scaled down (1e2 .. 5e3 elements)
    return gen.batch_specs(n, lo=1e2, hi=5e3)


def test_batch_matches_single_problem_path_bitwise(mf, orc, tmp_path):
    import torch
    specs = small_specs()
    assert {s["type"] for s in specs} == {"P1", "P2", "Q1"}
    probs = [gen.batch_problem(s) for s in specs]
    # unjittered Q1 boxes (every element a translate of element 0) in the mix
    probs.insert(3, gen.thermal_q1_problem(6, jitter=0.0))
    probs.append(gen.thermal_q1_problem(9, jitter=0.0))
    # power-of-two boxes: exact translates of a cubic cell (the box row routine)
    probs.insert(5, gen.thermal_q1_problem(8, jitter=0.0))
    probs.append(gen.thermal_q1_problem(16, jitter=0.0))
    single = []
    for pr in probs:
        P = mf.Problem(pr)
        v, d = P.assemble()
        single.append((v.clone(), d.clone()))
    batch_P = [mf.Problem(pr) for pr in probs]
    for P in batch_P:
        P.values.fill_(float("nan"))
        P.d.fill_(float("nan"))
    B = mf.mf_batch_create(batch_P)
    for tiling in (mf.BatchTiling(64, 64, 16, 2), mf.BatchTiling(4096, 256, 1024, 8)):
        mf.mf_batch_set_tiling(B, tiling)
        mf.mf_batch_assemble(B)
        torch.cuda.synchronize()
        for P, (v, d) in zip(batch_P, single):
            assert torch.equal(P.values, v) and torch.equal(P.d, d)
    mf.mf_sync_status()
    # a few problems against the oracle
    for i in (0, 3, len(probs) // 2, len(probs) - 1):
        ref = orc.assemble(probs[i])
        P = batch_P[i]
        val = P.values.cpu().numpy()
        rp = ref["row_ptr"]
        rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
        emax = np.zeros(rp.shape[0] - 1)
        rmax = np.zeros(rp.shape[0] - 1)
        np.maximum.at(emax, rows, np.abs(val - ref["val"]))
        np.maximum.at(rmax, rows, np.abs(ref["val"]))
        assert (emax / rmax).max() <= 1e-12
    mf.mf_batch_destroy(B)


def test_autotuner_picks_and_caches_a_tiling(mf, tmp_path):
    import torch
    probs = [gen.batch_problem(s) for s in small_specs(12)]
    Ps = [mf.Problem(pr) for pr in probs]
    B = mf.mf_batch_create(Ps)
    cache = str(tmp_path / "tiling.json")
    t1 = mf.mf_batch_autotune(B, cache)
    assert t1.elem_tile > 0 and t1.elem_block % 32 == 0 and t1.node_tile > 0 and t1.grid_per_sm > 0
    data = json.load(open(cache))
    assert len(data) == 1 and list(data.values())[0] == [t1.elem_tile, t1.elem_block, t1.node_tile, t1.grid_per_sm]
    # a second tuner run reuses the cached entry
    B2 = mf.mf_batch_create(Ps)
    t2 = mf.mf_batch_autotune(B2, cache)
    assert (t2.elem_tile, t2.elem_block, t2.node_tile, t2.grid_per_sm) == \
        (t1.elem_tile, t1.elem_block, t1.node_tile, t1.grid_per_sm)
    mf.mf_batch_assemble(B2)
    torch.cuda.synchronize()
    mf.mf_batch_destroy(B)
    mf.mf_batch_destroy(B2)


def test_batch_rejects_non_thermal(mf):
    P = mf.Problem(gen.elastic_problem(3))
    with pytest.raises(mf.MFError) as ei:
        mf.mf_batch_create([P])
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
