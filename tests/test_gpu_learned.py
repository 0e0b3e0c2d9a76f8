"""Learned preconditioner correction: BF16 CNN kernels against the FP64 oracle,
training, and flexible CG against Jacobi-PCG.

Forward/backward: the GPU computes in BF16 with FP32 accumulation and rounds
the activations to BF16 between layers; the oracle convolutions run in FP64 on
the same BF16-rounded weights and inputs with the same rounding of the
activations, so the remaining difference is the accumulation order and the
BF16 rounding decisions it flips.  A flipped rounding moves one activation by
one BF16 unit (2^-8 of it) and reaches a later entry through |w| |a|
products, so every entry is compared on its own against the same network run
on |w| and |x| (its magnitude scale s_i): |y_gpu - y_oracle| <= 2^-6 s_i for
the output (up to four layers of flips), |g_gpu - g_oracle| <= 2^-5 s_i for
every weight and bias gradient (the GPU backward pass also rounds the masked
gradients entering the two 16-channel layers to BF16, 2^-9 of s_i per layer).
A wrong halo, plane or channel moves entries by O(s_i) and fails; the
(4, 5, 37) grid spans three 16-node runs along x with a ragged last one.
"""
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


def bf16(a):
    """Round float64/float32 values to BF16 (nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


LAYERS = [(2, 16), (16, 16), (16, 16), (16, 1)]


def split_params(p):
    out, o = [], 0
    for ci, co in LAYERS:
        w = p[o:o + co * ci * 27].reshape(co, ci, 27)
        o += co * ci * 27
        b = p[o:o + co]
        o += co
        out.append((w, b))
    return out


def oracle_forward(orc, x, params):
    acts = [x]
    h = x
    for li, (w, b) in enumerate(split_params(params)):
        last = li == len(LAYERS) - 1
        h = orc.conv3d_fwd(h, bf16(w), b.astype(np.float64), relu=not last)
        if not last:
            h = bf16(h)
        acts.append(h)
    return acts


def oracle_backward(orc, acts, params, gy):
    ps = split_params(params)
    grads = [None] * 4
    g = gy
    for li in range(3, -1, -1):
        w, b = ps[li]
        if li < 3:
            g = g * (acts[li + 1] > 0)
        gw, gb = orc.conv3d_bwd_weight(acts[li], g)
        grads[li] = (gw, gb)
        if li > 0:
            g = orc.conv3d_bwd_data(g, bf16(w), LAYERS[li][0])
    return grads


def rand_params(mf, seed):
    rng = np.random.default_rng(seed)
    p = []
    for ci, co in LAYERS:
        p += [rng.normal(size=co * ci * 27) * np.sqrt(2.0 / (27 * ci)), rng.normal(size=co) * 0.1]
    return np.concatenate(p).astype(np.float32)


def oracle_scale_forward(orc, x, params):
    """The network on |w|, |b| and |x| with the same layers (ReLU of a
    non-negative value is the identity): the magnitude scale of every entry."""
    acts = [np.abs(x)]
    h = np.abs(x)
    for w, b in split_params(params):
        h = orc.conv3d_fwd(h, np.abs(bf16(w)), np.abs(b.astype(np.float64)), relu=False)
        acts.append(h)
    return acts


def oracle_scale_backward(orc, sacts, params, gy):
    ps = split_params(params)
    grads = [None] * 4
    g = np.abs(gy)
    for li in range(3, -1, -1):
        w, _ = ps[li]
        gw, gb = orc.conv3d_bwd_weight(sacts[li], g)
        grads[li] = (gw, gb)
        if li > 0:
            g = orc.conv3d_bwd_data(g, np.abs(bf16(w)), LAYERS[li][0])
    return grads


@pytest.mark.parametrize("shape", [(5, 6, 7), (9, 4, 11), (4, 5, 37)])
def test_cnn_forward_backward_against_oracle(mf, orc, shape):
    import torch
    nz, ny, nx = shape
    B = 2
    params = rand_params(mf, 3)
    cnn = mf.mf_cnn_create(params)
    rng = np.random.default_rng(4)
    xh = rng.normal(size=(B, nz, ny, nx, 2))
    x = torch.from_numpy(xh.reshape(-1)).to("cuda", torch.bfloat16)
    xr = x.float().cpu().numpy().astype(np.float64).reshape(B, nz, ny, nx, 2)
    y = torch.empty(B * nz * ny * nx, dtype=torch.float32, device="cuda")
    mf.mf_cnn_forward(cnn, B, nz, ny, nx, x, y)
    gyh = rng.normal(size=(B, nz, ny, nx)).astype(np.float32)
    gy = torch.from_numpy(gyh.reshape(-1)).cuda()
    mf.mf_cnn_backward(cnn, B, nz, ny, nx, x, gy)
    torch.cuda.synchronize()
    yg = y.cpu().numpy().reshape(B, nz, ny, nx)
    gg = mf.mf_cnn_get_grads(cnn)
    tot = [None] * 4
    tsc = [None] * 4
    for b in range(B):
        acts = oracle_forward(orc, xr[b], params)
        sacts = oracle_scale_forward(orc, xr[b], params)
        yo, ys = acts[-1][..., 0], sacts[-1][..., 0]
        assert np.all(np.abs(yg[b] - yo) <= 2.0 ** -6 * ys), np.max(np.abs(yg[b] - yo) / ys)
        g64 = gyh[b][..., None].astype(np.float64)
        gr = oracle_backward(orc, acts, params, g64)
        gs = oracle_scale_backward(orc, sacts, params, g64)
        for li in range(4):
            tot[li] = gr[li] if tot[li] is None else (tot[li][0] + gr[li][0], tot[li][1] + gr[li][1])
            tsc[li] = gs[li] if tsc[li] is None else (tsc[li][0] + gs[li][0], tsc[li][1] + gs[li][1])
    o = 0
    for li, (ci, co) in enumerate(LAYERS):
        gw = gg[o:o + co * ci * 27].reshape(co, ci, 27)
        o += co * ci * 27
        gb = gg[o:o + co]
        o += co
        assert np.all(np.abs(gw - tot[li][0]) <= 2.0 ** -5 * tsc[li][0]), \
            (li, np.max(np.abs(gw - tot[li][0]) / tsc[li][0]))
        assert np.all(np.abs(gb - tot[li][1]) <= 2.0 ** -5 * tsc[li][1]), \
            (li, np.max(np.abs(gb - tot[li][1]) / tsc[li][1]))
    mf.mf_cnn_destroy(cnn)


@pytest.fixture(scope="module")
def small_data(mf):
    from paper_2111_03541_gb300 import learned
    tr = learned.Dataset(24, n=16, seed0=learned.TRAIN_SEED0, iters=(1, 4, 16, 64))
    va = learned.Dataset(6, n=16, seed0=learned.VALID_SEED0, iters=(1, 4, 16, 64))
    return learned, tr, va


def test_training_reduces_loss_below_jacobi(mf, small_data):
    learned, tr, va = small_data
    jl = learned.jacobi_loss(va)
    cnn, hist = learned.train(tr, va, steps=300, batch=8, lr=3e-3, log=lambda s: None)
    assert hist[-1]["valid_loss"] < 0.9 * jl, (jl, hist)
    mf.mf_cnn_destroy(cnn)


def test_fcg_with_network_matches_oracle_solution(mf, orc, small_data):
    import torch
    learned, tr, va = small_data
    cnn, _ = learned.train(tr, va, steps=200, batch=8, lr=3e-3, log=lambda s: None)
    kc = np.exp(gen.grf_cells(16, corr_len=0.4, seed=learned.VALID_SEED0 + 77))
    prob = gen.thermal_q1_problem(16, jitter=0.0, coef=kc)
    P = mf.Problem(prob)
    P.assemble()
    logk = learned.node_logk(P)
    x, st, info, fb = learned.fcg(P, cnn, logk, tol=1e-10)
    assert st == mf.MF_OK and info.rel_residual <= 1e-10
    ref = orc.assemble(prob)
    xo, it_o, _ = orc.pcg(ref, tol=1e-13)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)
    # a network that points the wrong way triggers the Jacobi fallback and still converges
    p = learned.init_params()
    p[-(16 * 27 + 1):-1] = -50.0
    bad = mf.mf_cnn_create(p)
    x2, st2, info2, fb2 = learned.fcg(P, bad, logk, tol=1e-10)
    assert st2 == mf.MF_OK and fb2 > 0
    assert np.linalg.norm(x2.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)
    mf.mf_cnn_destroy(cnn)
    mf.mf_cnn_destroy(bad)
