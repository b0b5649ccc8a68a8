"""Pins of the oracle's surrogate pieces: features, targets, network gradients, Adam."""
import math

import numpy as np
import pytest
import torch

from oracle import surrogate as S
from workloads import grid_global


def _params(seed=0, scale=1.0):
    P = S.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    P["b1"] = rng.standard_normal(S.HIDDEN) * 0.1
    P["b2"] = rng.standard_normal(S.HIDDEN) * 0.1
    P["b3"] = rng.standard_normal(S.NOUT) * 0.1
    return {k: v * scale for k, v in P.items()}


def test_gelu_matches_torch():
    x = np.linspace(-6, 6, 1001)
    ref = torch.nn.functional.gelu(torch.from_numpy(x), approximate="none").numpy()
    np.testing.assert_allclose(S.gelu(x), ref, rtol=1e-14, atol=1e-15)
    xt = torch.from_numpy(x).requires_grad_(True)
    torch.nn.functional.gelu(xt, approximate="none").sum().backward()
    np.testing.assert_allclose(S.gelu_grad(x), xt.grad.numpy(), rtol=1e-12, atol=1e-14)


def test_forward_backward_match_torch_autograd():
    rng = np.random.default_rng(3)
    P = _params(0)
    xh = rng.standard_normal((64, S.KPAD))
    xh[:, S.NFEAT:] = 0
    yt = rng.standard_normal((64, S.NOUT))
    loss, g = S.loss_and_grads(P, xh, yt)
    T = {k: torch.from_numpy(v.copy()).requires_grad_(True) for k, v in P.items()}
    x = torch.from_numpy(xh)
    gel = lambda z: torch.nn.functional.gelu(z, approximate="none")
    y = gel(gel(x @ T["W1"] + T["b1"]) @ T["W2"] + T["b2"]) @ T["W3"] + T["b3"]
    tl = ((y - torch.from_numpy(yt)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12
    for k in T:
        np.testing.assert_allclose(g[k], T[k].grad.numpy(), rtol=1e-10, atol=1e-13, err_msg=k)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(4)
    P = _params(1)
    xh = rng.standard_normal((16, S.KPAD))
    yt = rng.standard_normal((16, S.NOUT))
    _, g = S.loss_and_grads(P, xh, yt)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in P[name].shape)
            if name == "W1":
                idx = (rng.integers(0, S.NFEAT), idx[1])
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += h
            Pm[name][idx] -= h
            fd = (S.loss_and_grads(Pp, xh, yt)[0] - S.loss_and_grads(Pm, xh, yt)[0]) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    t = torch.from_numpy(theta.copy()).requires_grad_(True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 4):
        grad = rng.standard_normal(50)
        theta, m, v = S.adam_step(theta, grad, m, v, step, 3e-3)
        t.grad = torch.from_numpy(grad)
        opt.step()
        np.testing.assert_allclose(theta, t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_features_of_a_node_indexed_field():
    """With f = 1000*var + 100*snap + 10*k + 0.01*j + 1e-4*i the stencil values name their nodes."""
    grid = grid_global(8, 7, 6)
    kk, jj, ii = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    f = []
    for snap in (0, 1):
        f.append({var: 1000.0 * c + 100.0 * snap + 10.0 * kk + 0.01 * jj + 1e-4 * ii
                  for c, var in enumerate(("u", "v", "w"))})
    # a point nearest to node (i=0, j=3, k=2): lon 10 deg (x = 0.22), lat 3 (y = 3.1)
    lon, lat = np.array([10.0]), np.array([3.0])
    p = np.array([0.7 * grid.plev[2] + 0.3 * grid.plev[3]])    # z = 2 + fz, fz = 0.3 (linear in p)
    X = S.features(grid, f[0], f[1], 5400.0, 0.0, 21600.0, lon, lat, p)[0]
    i0, j0, k0, ox, oy, oz = S.nearest_node(grid, lon, lat, p)
    assert (i0[0], j0[0], k0[0]) == (0, 3, 2)
    col = 0
    for snap in (0, 1):
        for c in range(3):
            for dk in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    for di in (-1, 0, 1):
                        i = (0 + di) % 8
                        assert X[col] == 1000.0 * c + 100.0 * snap + 10.0 * (2 + dk) + 0.01 * (3 + dj) + 1e-4 * i
                        col += 1
    assert abs(X[162] - 10.0 / 45.0) < 1e-15 and abs(X[163] - (93.0 / 30.0 - 3)) < 1e-12
    assert abs(X[164] - 0.3) < 1e-12
    assert X[165] == 0.25
    assert abs(X[166] - math.sin(math.radians(3.0))) < 1e-15
    assert np.all(X[168:] == 0)


def test_targets_apply_roundtrip():
    rng = np.random.default_rng(6)
    n = 1000
    lon0, lat0 = rng.uniform(0, 360, n), rng.uniform(-80, 80, n)
    p0 = rng.uniform(2e3, 9e4, n)
    lon1 = lon0 + rng.uniform(-1, 1, n)
    lat1 = lat0 + rng.uniform(-0.5, 0.5, n)
    p1 = p0 * np.exp(rng.uniform(-0.1, 0.1, n))
    y = S.targets(lon0, lat0, p0, lon1, lat1, p1)
    a, b, c = S.apply_displacement(lon0, lat0, p0, y)
    np.testing.assert_allclose(a, lon1, atol=1e-10)
    np.testing.assert_allclose(b, lat1, atol=1e-10)
    np.testing.assert_allclose(c, p1, rtol=1e-12)
    # 1 degree of latitude is R pi / 180 metres north
    y1 = S.targets(np.array([0.0]), np.array([10.0]), np.array([5e4]), np.array([0.0]), np.array([11.0]),
                   np.array([5e4]))
    assert abs(y1[0, 1] - 6371000.0 * math.pi / 180) < 1e-6 and y1[0, 0] == 0 and y1[0, 2] == 0


def test_envelope():
    xh = np.zeros((4, S.KPAD))
    xh[1, 10] = 4.5
    xh[3, 170] = 99.0        # padding is ignored
    lat = np.array([10.0, 10.0, 85.0, -20.0])
    np.testing.assert_array_equal(S.in_envelope(xh, lat), [True, False, False, True])


def test_bf16_round_matches_torch_and_ties():
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(x.astype(np.float64)), ref)
    # ties go to the even neighbour; 8 significant bits
    cases = {1 + 2.0**-8: 1.0, 1 + 3 * 2.0**-8: 1 + 2.0**-6, 1 + 2.0**-7: 1 + 2.0**-7,
             -(1 + 2.0**-8): -1.0, 0.0: 0.0, 3 * 2.0**-9: 3 * 2.0**-9, 255.5: 256.0, 257.0: 256.0}
    for a, b in cases.items():
        assert S.bf16_round(np.array([a]))[0] == b, (a, b)


class _RoundValue(torch.autograd.Function):
    """Rounds the value to bfloat16 (torch's cast); the gradient passes unchanged."""
    @staticmethod
    def forward(ctx, x):
        return x.to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g


class _RoundGrad(torch.autograd.Function):
    """Passes the value unchanged; rounds the incoming gradient to bfloat16."""
    @staticmethod
    def forward(ctx, x):
        return x.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(torch.float64)


def test_bf16_network_matches_torch_autograd_with_rounding_hooks():
    """The BF16 network (rounded activations forward, rounded upstream gradients backward)
    against torch autograd, whose chain rule sees the roundings only as value hooks."""
    rng = np.random.default_rng(12)
    P = {k: (S.bf16_round(v) if k.startswith("W") else v) for k, v in _params(2).items()}
    xh = S.bf16_round(rng.standard_normal((96, S.KPAD)))
    xh[:, S.NFEAT:] = 0
    yt = rng.standard_normal((96, S.NOUT))
    trace = {}
    loss, g = S.loss_and_grads(P, xh, yt, rnd=S.bf16_round, trace=trace)
    T = {k: torch.from_numpy(v.copy()).requires_grad_(True) for k, v in P.items()}
    gel = lambda z: torch.nn.functional.gelu(z, approximate="none")
    z1 = _RoundGrad.apply(torch.from_numpy(xh) @ T["W1"] + T["b1"])
    z2 = _RoundGrad.apply(_RoundValue.apply(gel(z1)) @ T["W2"] + T["b2"])
    y = _RoundGrad.apply(_RoundValue.apply(gel(z2)) @ T["W3"] + T["b3"])
    tl = ((y - torch.from_numpy(yt)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12
    np.testing.assert_allclose(trace["yh"], y.detach().numpy(), rtol=1e-12, atol=1e-14)
    for k in T:
        np.testing.assert_allclose(g[k], T[k].grad.numpy(), rtol=1e-10, atol=1e-13, err_msg=k)
    # the rounding changes the result (it is not a no-op here) but only by bf16 amounts
    _, g0 = S.loss_and_grads(P, xh, yt)
    rel = np.abs(g["W1"][:S.NFEAT] - g0["W1"][:S.NFEAT]).max() / np.abs(g0["W1"]).max()
    assert 1e-5 < rel < 5e-2, rel
