"""The dispatch MLP: CPU oracle pins and GPU kernel parity.

The oracle (oracle/mlp.py, FP64) is pinned by central finite differences
and by a one-neuron network whose gradient is written out by hand.  The
GPU kernels (afmm_mlp_forward / loss_grad / adam) are compared with it.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as M


def _net(rng, F=5, H=7, V=2, rows=23):
    p = rng.standard_normal(M.param_count(F, H, V)) * 0.5
    X = rng.standard_normal((rows, F))
    T = rng.standard_normal((rows, V))
    Mk = (rng.random((rows, V)) < 0.7).astype(np.float64)
    return p, X, T, Mk, F, H, V


def test_oracle_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p, X, T, Mk, F, H, V = _net(rng)
    count = Mk.sum()
    _, g = M.loss_and_grads(p, X, T, Mk, count, F, H, V)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = M.loss_and_grads(p + e, X, T, Mk, count, F, H, V)
        lm, _ = M.loss_and_grads(p - e, X, T, Mk, count, F, H, V)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_oracle_one_neuron_by_hand():
    """F = H = V = 1, all weights positive: P = w3 * (w2 * (w1 x + b1) + b2)
    + b3 and dL/dw1 = 2 (P - T) w3 w2 x for one sample (count 1)."""
    w1, b1, w2, b2, w3, b3 = 0.5, 0.1, 2.0, -0.3, 1.5, 0.2
    p = np.array([w1, b1, w2, b2, w3, b3])
    x, t = 3.0, 1.0
    h1 = w1 * x + b1
    h2 = w2 * h1 + b2
    P = w3 * h2 + b3
    loss, g = M.loss_and_grads(p, [[x]], [[t]], [[1.0]], 1.0, 1, 1, 1)
    assert loss == pytest.approx((P - t) ** 2)
    d = 2 * (P - t)
    assert g == pytest.approx([d * w3 * w2 * x, d * w3 * w2, d * w3 * h1, d * w3,
                               d * h2, d])


@pytest.mark.gpu
def test_gpu_forward_and_gradients_match_oracle():
    import torch
    from paper_1308_2400_gb300.afmm import (afmm_mlp_forward, afmm_mlp_loss_grad,
                                            afmm_mlp_param_count,
                                            afmm_mlp_work_floats, mlp_shape)
    rng = np.random.default_rng(1)
    for F, H, V, rows in [(8, 32, 2, 300), (5, 7, 3, 23), (8, 64, 2, 1000)]:
        p, X, T, Mk, F, H, V = _net(rng, F, H, V, rows)
        shape = mlp_shape(F, H, V)
        assert afmm_mlp_param_count(shape) == p.size
        d = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
        pd, Xd, Td, Md = d(p), d(X), d(T), d(Mk)
        work = torch.empty(afmm_mlp_work_floats(shape, rows), device="cuda")
        P = torch.empty((rows, V), device="cuda")
        afmm_mlp_forward(shape, pd, Xd, rows, P, work)
        torch.cuda.synchronize()
        P_ref, _, _ = M.forward(p.astype(np.float32), X.astype(np.float32), F, H, V)
        assert np.max(np.abs(P.cpu().numpy() - P_ref)) <= 1e-4 * max(1, np.abs(P_ref).max())
        grads = torch.empty_like(pd)
        loss = torch.empty(1, device="cuda")
        count = float(Mk.sum())
        afmm_mlp_loss_grad(shape, pd, Xd, Td, Md, rows, count, grads, work, loss)
        torch.cuda.synchronize()
        l_ref, g_ref = M.loss_and_grads(p.astype(np.float32), X.astype(np.float32),
                                        T.astype(np.float32), Mk, count, F, H, V)
        assert abs(loss.item() - l_ref) <= 1e-4 * max(1.0, l_ref)
        g = grads.cpu().numpy().astype(np.float64)
        for a, b in ((0, F * H), (F * H, F * H + H), (F * H + H, F * H + H + H * H)):
            ref = g_ref[a:b]
            assert np.linalg.norm(g[a:b] - ref) <= 1e-4 * max(1e-6, np.linalg.norm(ref))
        assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


@pytest.mark.gpu
def test_gpu_adam_matches_oracle():
    import torch
    from paper_1308_2400_gb300.afmm import afmm_mlp_adam
    rng = np.random.default_rng(2)
    n = 777
    p, g = rng.standard_normal(n), rng.standard_normal(n)
    m, v = rng.standard_normal(n) * 0.1, rng.random(n) * 0.1
    d = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    pd, gd, md, vd = d(p), d(g), d(m), d(v)
    afmm_mlp_adam(n, pd, gd, md, vd, 1e-3, 0.9, 0.999, 1e-8, 5)
    torch.cuda.synchronize()
    pr, mr, vr = M.adam_step(p, g, m, v, 1e-3, 0.9, 0.999, 1e-8, 5)
    assert np.allclose(pd.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    assert np.allclose(md.cpu().numpy(), mr, rtol=1e-5, atol=1e-6)
    assert np.allclose(vd.cpu().numpy(), vr, rtol=1e-5, atol=1e-7)


def test_host_dispatch_uses_the_installed_model():
    """afmm_dispatch_variant evaluates the installed model on the host: a
    network whose output 1 (tensor cores) is always lower picks them, and
    removing the model restores the built-in rule."""
    from paper_1308_2400_gb300.afmm import (afmm_dispatch_features,
                                            afmm_dispatch_variant,
                                            afmm_set_dispatch_model, make_desc,
                                            mlp_shape)
    F, H, V = 8, 4, 2
    p = np.zeros(M.param_count(F, H, V), np.float32)
    p[-2:] = [5.0, -5.0]                  # b3: output 0 high, output 1 low
    d = make_desc(256, "A", "f32", "u8", "f32", "fp32", d1=0.01, d2=0.5,
                  mu_prime=2.0)
    f = afmm_dispatch_features(d)
    assert f[0] == 8.0 and f[4] == 0.0 and abs(f[1] - 0.01) < 1e-7
    assert afmm_dispatch_variant(d) == 0           # rule: very sparse Base
    afmm_set_dispatch_model(mlp_shape(F, H, V), p, np.zeros(F), np.ones(F), [0, 1])
    try:
        assert afmm_dispatch_variant(d) == 1
    finally:
        afmm_set_dispatch_model(None, None, None, None, None)
    assert afmm_dispatch_variant(d) == 0


def test_dispatch_features_and_narrow_tile_route():
    """The two tile-padding features, and a three-output model whose third
    output (the 128 x 128 tensor-core tiles) is the lowest."""
    from paper_1308_2400_gb300.afmm import (AFMM_DISPATCH_FEATURES,
                                            AFMM_VARIANT_TC_BF16X3_N128,
                                            afmm_dispatch_features,
                                            afmm_dispatch_variant,
                                            afmm_set_dispatch_model, make_desc,
                                            mlp_shape)
    assert AFMM_DISPATCH_FEATURES == 10
    d = make_desc(300, "B", "u8", "f32", "f32", "fp32", d1=0.5, d2=0.5, mu_prime=2.0)
    f = afmm_dispatch_features(d)
    assert abs(f[8] - 512 / 300) < 1e-6 and abs(f[9] - 384 / 300) < 1e-6
    F, H, V = 10, 4, 3
    p = np.zeros(M.param_count(F, H, V), np.float32)
    p[-3:] = [5.0, 4.0, -5.0]
    afmm_set_dispatch_model(mlp_shape(F, H, V), p, np.zeros(F), np.ones(F),
                            [0, 1, AFMM_VARIANT_TC_BF16X3_N128])
    try:
        assert afmm_dispatch_variant(d) == AFMM_VARIANT_TC_BF16X3_N128
    finally:
        afmm_set_dispatch_model(None, None, None, None, None)


def test_autotuner_copies_fill_the_grouped_launch():
    """The in-batch cost of an instance is timed on copies of it that give
    the grouped launch about four waves of 128 x 256 tiles on 152 SMs."""
    from paper_1308_2400_gb300.tune import copies_for
    assert copies_for(64) == 64                     # one tile: capped at 64
    assert copies_for(2048) == 5                    # 128 tiles: ceil(608 / 128)
    assert copies_for(4096) == 2                    # 512 tiles
    assert copies_for(8192) == 1
    for n in (1, 100, 129, 257, 700, 1500, 2047):
        r = copies_for(n)
        tiles = -(-n // 128) * -(-n // 256)
        assert 1 <= r <= 64
        assert r == 64 or (r * tiles >= 608 and (r - 1) * tiles < 608)
