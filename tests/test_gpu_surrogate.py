"""Learned surrogate: GPU kernels against the float64 oracle, and what training gains."""
import numpy as np
import pytest
import torch

from oracle import met as omet
from oracle import surrogate as S
from oracle import transport as tr
from workloads import fourier_modes, fourier_snapshot, grid_global, uniform_particles

from _gpu_common import M, make_ctx  # noqa: F401

pytestmark = pytest.mark.gpu
T6H = 21600.0


@pytest.fixture(scope="module")
def field(M):
    grid = grid_global(120, 61, 30)
    m = fourier_modes(2)
    f0 = fourier_snapshot(grid, m, 0.0)
    f1 = fourier_snapshot(grid, m, T6H)
    ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H])
    return grid, f0, f1, ctx


STORAGES = pytest.mark.parametrize("storage", [0, 1, 2], ids=["fp32", "bf16", "fp16"])


@pytest.fixture(scope="module")
def stored(M, field):
    """Per storage: a context holding the two snapshots in that storage, and the values it holds
    (the oracle's view of the same stored fields, decoded to float64)."""
    grid, f0, f1, _ = field
    cache = {}

    def get(storage):
        if storage not in cache:
            ctx = make_ctx(M, grid, [f0, f1], [0.0, T6H], storage=storage)
            cache[storage] = (ctx, omet.stored_fields(f0, storage), omet.stored_fields(f1, storage))
        return cache[storage]
    return get


@STORAGES
def test_features_match_oracle(M, field, stored, storage):
    """Stencil features from the stored snapshots (16-bit codes decoded with their level scales),
    offsets, time weight and sin/cos of latitude, against the oracle on the same stored values."""
    grid = field[0]
    ctx, f0, f1 = stored(storage)
    st = uniform_particles(20_000, grid.plev, seed=3)
    parts = M.Particles.from_numpy(st)
    t = 5000.0
    X = M.surr_features(ctx, parts, t).cpu().numpy()
    ref = S.features(grid, f0, f1, t, 0.0, T6H, st["lon"], st["lat"], st["p"]).astype(np.float32)
    # the nearest node is chosen in float64 on both sides: identical stencils
    np.testing.assert_array_equal(X[:, :162], ref[:, :162])
    np.testing.assert_allclose(X[:, 162:], ref[:, 162:], rtol=0, atol=2e-7)


def test_targets_match_oracle(M):
    rng = np.random.default_rng(1)
    n = 5000
    a = {"lon": rng.uniform(0, 360, n), "lat": rng.uniform(-80, 80, n), "p": rng.uniform(2e3, 9e4, n),
         "id": np.arange(n, dtype=np.uint32)}
    b = {"lon": np.mod(a["lon"] + rng.uniform(-1, 1, n), 360), "lat": a["lat"] + rng.uniform(-.5, .5, n),
         "p": a["p"] * np.exp(rng.uniform(-.1, .1, n)), "id": a["id"]}
    Y = M.surr_targets(M.Particles.from_numpy(a), M.Particles.from_numpy(b)).cpu().numpy()
    ref = S.targets(a["lon"], a["lat"], a["p"], b["lon"], b["lat"], b["p"])
    np.testing.assert_allclose(Y, ref, rtol=2e-7, atol=1e-6)


KERNELS = pytest.mark.parametrize("kernel", [0, 1], ids=["tcgen05", "mma_sync"])

# Tolerances of the BF16 network against the oracle's BF16 network (oracle.surrogate with
# rnd=bf16_round: the same bf16 weights, inputs and activations, exact float64 sums).
# * The GPU accumulates exact bf16 products in float32: a sum of K products plus a bias is within
#   K 2^-23 sum|terms| of the exact one (truncating adds included).
# * Every other difference comes from an activation or standardised input that lies within
#   float32 error of a bf16 rounding boundary and rounds the other way on the GPU ("flip").  One
#   flip moves output j by at most one bf16 unit of the flipped value times the magnitude of the
#   output's derivative with respect to it (first order).  Rows may hold up to 3 flips.
# * Gradients sum B products each; a flip changes one product by one bf16 unit of an operand,
#   i.e. by at most 2^-8 of that product, far below 2^-8 of the largest gradient element.
ACC = 2.0 ** -23
FLIPS = 3


def _bf16_ulp(v):
    return 2.0 ** (np.floor(np.log2(np.abs(v) + 1e-300)) - 7)


def _flip_bound(Pb, act):
    """Largest first-order change of each output [n, 3] from one bf16 flip of an input or activation."""
    xh, z1, h1, z2, h2 = act
    A = np.einsum("kl,bl,lj->bkj", Pb["W2"], S.gelu_grad(z2), Pb["W3"])    # d y / d h1
    J0 = np.einsum("ik,bk,bkj->bij", Pb["W1"], S.gelu_grad(z1), A)         # d y / d x_hat
    f0 = (_bf16_ulp(xh[:, :S.NFEAT])[:, :, None] * np.abs(J0[:, :S.NFEAT])).max(axis=1)
    f1 = (_bf16_ulp(h1)[:, :, None] * np.abs(A)).max(axis=1)
    f2 = (_bf16_ulp(h2)[:, :, None] * np.abs(Pb["W3"])[None]).max(axis=1)
    return np.maximum(np.maximum(f0, f1), f2)


def _random_model(seed, n):
    rng = np.random.default_rng(seed)
    P = S.init_params(seed)
    P["b1"] = rng.standard_normal(S.HIDDEN) * 0.1
    P["b2"] = rng.standard_normal(S.HIDDEN) * 0.1
    P["b3"] = rng.standard_normal(S.NOUT) * 0.1
    P["W1"][S.NFEAT:] = rng.uniform(-1, 1, (S.KPAD - S.NFEAT, S.HIDDEN))   # padded rows: must not matter
    mu_x = rng.standard_normal(S.KPAD)
    sd_x = rng.uniform(0.5, 2.0, S.KPAD)
    mu_y = rng.standard_normal(S.NOUT)
    sd_y = rng.uniform(0.5, 2.0, S.NOUT)
    X = (mu_x + sd_x * rng.standard_normal((n, S.KPAD))).astype(np.float32)
    X[:, S.NFEAT:] = 0
    Y = (mu_y + sd_y * rng.standard_normal((n, S.NOUT))).astype(np.float32)
    return P, mu_x, sd_x, mu_y, sd_y, X, Y


def _oracle_bf16(P):
    """The GPU's parameters as the oracle sees them: bf16 weights (rounded from float32), float32 biases."""
    return {k: (S.bf16_round(np.float32(v)) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
            for k, v in P.items()}


def _oracle_inputs(mu_x, sd_x, X):
    xh = S.normalise(X, mu_x.astype(np.float32), sd_x.astype(np.float32))
    xh[:, S.NFEAT:] = 0
    return S.bf16_round(xh)


def _gpu_model(M, kernel, P, mu_x, sd_x, mu_y, sd_y, max_batch=8192):
    sur = M.Surrogate(max_batch)
    sur.set_kernel(kernel)
    sur.set_params(S.flatten(P).astype(np.float32))
    sur.set_norm(mu_x, sd_x, mu_y, sd_y)
    return sur


@KERNELS
@pytest.mark.parametrize("n", [4096, 1000])
def test_forward_matches_oracle_per_element(M, kernel, n):
    P, mu_x, sd_x, mu_y, sd_y, X, _ = _random_model(7, n)
    sur = _gpu_model(M, kernel, P, mu_x, sd_x, mu_y, sd_y)
    yh = sur.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    sur.status()
    assert np.all(yh[:, 3:] == 0)
    Pb = _oracle_bf16(P)
    ref, act = S.forward(Pb, _oracle_inputs(mu_x, sd_x, X), rnd=S.bf16_round)
    acc = (S.HIDDEN + 1) * ACC * (S.bf16_round(np.abs(act[4])) @ np.abs(Pb["W3"]) + np.abs(Pb["b3"]))
    d = np.abs(yh[:, :3] - ref)
    exact = np.all(d <= acc, axis=1)
    assert exact.mean() >= 0.99, exact.mean()
    bad = d > acc + FLIPS * _flip_bound(Pb, act)
    assert not bad.any(), (np.argwhere(bad)[:5], d[bad][:5])


@KERNELS
@pytest.mark.parametrize("n", [4096, 1000])
def test_gradients_match_oracle_per_element(M, kernel, n):
    P, mu_x, sd_x, mu_y, sd_y, X, Y = _random_model(8, n)
    sur = _gpu_model(M, kernel, P, mu_x, sd_x, mu_y, sd_y)
    loss = sur.grads(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()).item()
    sur.status()
    g = S.unflatten(sur.get_grads().astype(np.float64))
    Pb = _oracle_bf16(P)
    yt = (Y.astype(np.float64) - mu_y.astype(np.float32)) / sd_y.astype(np.float32)
    rl, rg = S.loss_and_grads(Pb, _oracle_inputs(mu_x, sd_x, X), yt, rnd=S.bf16_round)
    assert abs(loss - rl) <= 2.0 ** -12 * rl, (loss, rl)
    for k in rg:
        ref = rg[k][:S.NFEAT] if k == "W1" else rg[k]
        got = g[k][:S.NFEAT] if k == "W1" else g[k]
        d = np.abs(got - ref)
        scale = np.abs(ref).max()
        assert d.max() <= 2.0 ** -8 * scale, (k, d.max() / scale)
        assert np.median(d) <= 2.0 ** -14 * scale, (k, np.median(d) / scale)
    assert np.all(g["W1"][S.NFEAT:] == 0)      # padded input columns are zero: no gradient


def test_adam_step_matches_oracle(M):
    P, mu_x, sd_x, mu_y, sd_y, X, Y = _random_model(9, 2048)
    sur = M.Surrogate(4096)
    theta0 = S.flatten(P).astype(np.float32)
    sur.set_params(theta0)
    sur.set_norm(mu_x, sd_x, mu_y, sd_y)
    loss = torch.zeros(1, device="cuda")
    sur.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), 1e-3, 1, loss)
    theta1 = sur.get_params()
    grad = sur.get_grads()
    ref, _, _ = S.adam_step(theta0.astype(np.float64), grad.astype(np.float64), np.zeros_like(theta0, np.float64),
                            np.zeros_like(theta0, np.float64), 1, 1e-3)
    np.testing.assert_allclose(theta1, ref, rtol=1e-6, atol=1e-7)


def _dataset(M, grid, ctx, f0, f1, n, seed):
    st = uniform_particles(n, grid.plev, seed=seed, lat_max=75.0)
    parts = M.Particles.from_numpy(st, meso=False, release=False)
    t = 3600.0
    X = M.surr_features(ctx, parts, t)
    p1 = parts.clone()
    ctx.advect(p1, t, 180.0, 10)
    Y = M.surr_targets(parts, p1)
    return st, X, Y, p1


def _compare_with_oracle_pipeline(grid, st, X, got, fbn, P, mu_x, sd_x, mu_y, sd_y):
    """The fused inference's output (positions ``got``, fallback flags ``fbn``) for the particles
    ``st`` with oracle features ``X``, against the oracle's pipeline: standardise -> BF16
    network -> displacement -> position rules (bounds: see the test below)."""
    xh = S.normalise(X, mu_x.astype(np.float32), sd_x.astype(np.float32))
    xh[:, S.NFEAT:] = 0
    env = S.in_envelope(xh, st["lat"])
    Pb = _oracle_bf16(P)
    yh, act = S.forward(Pb, S.bf16_round(xh), rnd=S.bf16_round)
    mu32, sd32 = mu_y.astype(np.float32).astype(np.float64), sd_y.astype(np.float32).astype(np.float64)
    y = yh * sd32 + mu32
    pmin, pmax = grid.plev[-1], grid.plev[0]
    lon1, lat1, p1 = S.apply_displacement(st["lon"], st["lat"], st["p"], y)
    lon1, lat1, p1 = tr.position_bc(lon1, lat1, p1, 0.0, pmin, pmax)

    near = np.any(np.abs(np.abs(X[:, 162:165]) - 0.5) < 1e-4, axis=1)
    near |= np.any(np.abs(np.abs(xh[:, :S.NFEAT]) - 4.0) < 1e-3, axis=1)
    assert near.mean() < 0.01, near.mean()
    np.testing.assert_array_equal(fbn[~near] == 0, env[~near])
    for k in ("lon", "lat", "p"):                      # fallback particles are not moved
        np.testing.assert_array_equal(got[k][fbn == 1], st[k][fbn == 1])

    moved = (fbn == 0) & ~near
    clamped = (p1 <= pmin) | (p1 >= pmax)
    np.testing.assert_array_equal(got["p"][moved & clamped], p1[moved & clamped])
    ygot = S.targets(st["lon"], st["lat"], st["p"], got["lon"], got["lat"], got["p"])
    acc = (S.HIDDEN + 1) * ACC * (S.bf16_round(np.abs(act[4])) @ np.abs(Pb["W3"]) + np.abs(Pb["b3"]))
    conv = 2.0 ** -19 * (np.abs(y) + np.abs(mu32)) + np.array([1e-6, 1e-6, 2.0 ** -20])
    d = np.abs(ygot - y)
    d[:, 2] = np.where(clamped, 0.0, d[:, 2])
    exact = np.all(d <= sd32 * acc + conv, axis=1)[moved]
    assert exact.mean() >= 0.95, exact.mean()
    bad = (d > sd32 * (acc + FLIPS * _flip_bound(Pb, act)) + conv) & moved[:, None]
    assert not bad.any(), (np.argwhere(bad)[:5], d[bad][:5])


@KERNELS
@STORAGES
def test_fused_inference_matches_oracle_pipeline(M, field, stored, kernel, storage):
    """The fused inference (stencil gather, standardisation, three bf16 layers, displacement,
    position rules, fallback flag) against the oracle's pipeline on the same positions:
    oracle features -> standardise -> BF16 network -> displacement -> position rules.

    Rows are left out only where the kernel's float32 choice may differ from the float64 one:
    a position within 1e-4 cells of a half-cell (another nearest node, another stencil), or a
    standardised feature within 1e-3 of the envelope limit 4.  Elsewhere the outputs agree to the
    float32 accumulation bound plus at most three bf16 flips (see above), converted to metres,
    plus the float32 rounding of the conversion itself (2^-19 relative).  In every storage the
    oracle reads the values the context holds (16-bit codes decoded with their level scales)."""
    grid = field[0]
    ctx, f0, f1 = stored(storage)
    n, t = 20_000, 3600.0
    st = uniform_particles(n, grid.plev, seed=21)
    st["lat"][:5] = [85.0, -86.0, 81.0, 10.0, 20.0]
    X = S.features(grid, f0, f1, t, 0.0, T6H, st["lon"], st["lat"], st["p"])
    rng = np.random.default_rng(22)
    P = S.init_params(3)
    for b in ("b1", "b2", "b3"):
        P[b] = rng.standard_normal(P[b].shape) * 0.1
    mu_x, sd_x = X.mean(axis=0), X.std(axis=0)
    sd_x[sd_x < 1e-12] = 1.0
    mu_y, sd_y = np.array([500.0, -300.0, 0.001]), np.array([2.0e4, 1.5e4, 0.05])
    sur = _gpu_model(M, kernel, P, mu_x, sd_x, mu_y, sd_y, max_batch=1024)
    parts = M.Particles.from_numpy(st, meso=False, release=False)
    fb = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sur.advance(ctx, parts, t, 1800.0, fb)
    sur.status()
    got, fbn = parts.to_numpy(), fb.cpu().numpy()

    _compare_with_oracle_pipeline(grid, st, X, got, fbn, P, mu_x, sd_x, mu_y, sd_y)
    assert fbn[0] == 1 and fbn[1] == 1 and fbn[2] == 1
    assert 0.05 < fbn.mean() < 0.5
    # the kernels' own count of fallback particles equals the flags they wrote
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    again = M.Particles.from_numpy(st, meso=False, release=False)
    fb2 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sur.advance(ctx, again, t, 1800.0, fb2, count)
    sur.advance(ctx, M.Particles.from_numpy(st, meso=False, release=False), t, 1800.0, fb2, count)
    torch.cuda.synchronize()
    assert count.item() == 2 * int(fb2.sum().item()) == 2 * int(fbn.sum())
    # the 30-minute window must fit inside the loaded interval, else everything falls back
    sur.advance(ctx, parts, T6H - 900.0, 1800.0, fb)
    torch.cuda.synchronize()
    assert fb.cpu().numpy().all()


def test_training_gains_over_untrained_and_first_order(M, field):
    """A short training run learns the 30-minute displacement far better than the
    untrained network and than a first-order step with the start-point wind."""
    from paper_2211_12616_gb300.learn import evaluate, train
    grid, f0, f1, ctx = field
    st, X, Y, p1 = _dataset(M, grid, ctx, f0, f1, 200_000, 12)
    sur = M.Surrogate(8192)
    sur.set_params(S.flatten(S.init_params(5)).astype(np.float32))
    hist, val = train(sur, X, Y, epochs=20, batch=4096, lr=2e-3, lr_min=1e-4)
    assert hist[-1] < hist[0]
    # untrained network with the same normalisation: loss of order 1
    raw = M.Surrogate(8192)
    raw.set_params(S.flatten(S.init_params(5)).astype(np.float32))
    mu_x, sd_x = M.colstats(X)
    mu_y, sd_y = M.colstats(Y)
    raw.set_norm(mu_x, sd_x, mu_y, sd_y)
    untrained = evaluate(raw, X[:20000], Y[:20000])
    assert val < 0.05 * untrained, (val, untrained)
    # first-order step u(x0, t0) * 1800 s from the stencil's centre node, in the same normalised units
    Xn, Yn = X[:20000].cpu().numpy(), Y[:20000].cpu().numpy()
    yn_true = (Yn - mu_y) / sd_y
    cen = 13                                              # (dk, dj, di) = (0, 0, 0)
    w = Xn[:, 165]
    u = (1 - w) * Xn[:, cen] + w * Xn[:, 81 + cen]
    v = (1 - w) * Xn[:, 27 + cen] + w * Xn[:, 81 + 27 + cen]
    first = np.stack([u * 1800.0, v * 1800.0, Yn[:, 2]], axis=1)   # (dz taken exact: favours the baseline)
    first_loss = np.mean(((first - mu_y) / sd_y - yn_true)[:, :2] ** 2) * 2 / 3
    assert val < first_loss, (val, first_loss)

    # The gain test against the method without the network: the trained surrogate and the plain
    # midpoint method with one 30-minute step (two wind evaluations: the same gather budget as one
    # stencil), both judged against the plain reference of 10 substeps of 180 s, on particles
    # inside the envelope.  Measured: the plain 30-minute step wins by far; this records it.
    from oracle.errors import great_circle_km
    st2 = uniform_particles(20_000, grid.plev, seed=31, lat_max=75.0)
    runs = {}
    for name in ("ref", "mid", "sur"):
        runs[name] = M.Particles.from_numpy(st2, meso=False, release=False)
    ctx.advect(runs["ref"], 3600.0, 180.0, 10)
    ctx.advect(runs["mid"], 3600.0, 1800.0, 1)
    fb = torch.zeros(20_000, dtype=torch.uint8, device="cuda")
    sur.advance(ctx, runs["sur"], 3600.0, 1800.0, fb)
    sur.status()
    out = {k: v.to_numpy() for k, v in runs.items()}
    inside = fb.cpu().numpy() == 0
    assert inside.mean() > 0.8
    err = {k: great_circle_km(out[k]["lon"], out[k]["lat"], out["ref"]["lon"], out["ref"]["lat"])[inside]
           for k in ("mid", "sur")}
    p99 = {k: float(np.percentile(e, 99)) for k, e in err.items()}
    print(f"gain test, 30 min, {inside.sum()} particles: p99 great-circle error surrogate {p99['sur']:.3f} km, "
          f"plain midpoint dt=1800 s {p99['mid']:.4f} km; median {np.median(err['sur']):.3f} / "
          f"{np.median(err['mid']):.4f} km")
    assert p99["sur"] > p99["mid"], p99


def _advance_with(M, sur, ctx, st, kernel, n):
    sur.set_kernel(kernel)
    parts = M.Particles.from_numpy(st, meso=False, release=False)
    fb = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sur.advance(ctx, parts, 3600.0, 1800.0, fb)
    sur.status()
    return parts.to_numpy(), fb.cpu().numpy()


@pytest.mark.parametrize("n", [1, 127, 3000, 20_000])
def test_tcgen05_inference_equals_mma_sync(M, field, n):
    """The tcgen05 kernel (tensor-memory accumulators) and the warp-level mma.sync kernel give the
    same particles: same gather, same bf16 operands, same order of the K = 16 accumulations.
    n spans one partial tile up to several tiles per CTA, with ragged tails."""
    grid, f0, f1, ctx = field
    st, X, Y, _ = _dataset(M, grid, ctx, f0, f1, max(n, 64), 13)
    st = {k: v[:n] for k, v in st.items()}
    sur = M.Surrogate(4096)
    sur.set_params(S.flatten(S.init_params(5)).astype(np.float32))
    mu_x, sd_x = M.colstats(X)
    mu_y, sd_y = M.colstats(Y)
    sur.set_norm(mu_x, sd_x, mu_y, sd_y)
    a, fa = _advance_with(M, sur, ctx, st, M.SURR_KERNEL_MMA_SYNC, n)
    b, fb = _advance_with(M, sur, ctx, st, M.SURR_KERNEL_TCGEN05, n)
    np.testing.assert_array_equal(fb, fa)
    moved = fa == 0
    assert moved.any() or n < 64
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(b[k], a[k], err_msg=k)


def test_bounded_wait_reports_timeout_and_recovers(M, field):
    """The tcgen05 kernel with its MMAs withheld: every wait for the tensor cores runs out
    (about 10 ms), the kernel frees its tensor memory and returns, nothing moves, and
    mptrac_surr_status reports E_TIMEOUT once.  The next launches run normally."""
    grid, f0, f1, ctx = field
    st, X, Y, _ = _dataset(M, grid, ctx, f0, f1, 2000, 17)
    sur = M.Surrogate(4096)
    sur.set_params(S.flatten(S.init_params(7)).astype(np.float32))
    mu_x, sd_x = M.colstats(X)
    mu_y, sd_y = M.colstats(Y)
    sur.set_norm(mu_x, sd_x, mu_y, sd_y)
    sur.set_kernel(M.SURR_KERNEL_WAIT_TEST)
    parts = M.Particles.from_numpy(st, meso=False, release=False)
    fb = torch.zeros(2000, dtype=torch.uint8, device="cuda")
    sur.advance(ctx, parts, 3600.0, 1800.0, fb)
    with pytest.raises(M.MptracError) as e:
        sur.status()
    assert e.value.code == -6
    got = parts.to_numpy()
    for k in ("lon", "lat", "p"):
        np.testing.assert_array_equal(got[k], st[k])
    sur.status()                      # the flag was cleared
    ref, _ = _advance_with(M, sur, ctx, st, M.SURR_KERNEL_MMA_SYNC, 2000)
    again, _ = _advance_with(M, sur, ctx, st, M.SURR_KERNEL_TCGEN05, 2000)
    np.testing.assert_array_equal(again["lon"], ref["lon"])


def test_set_kernel_rejects_unknown(M):
    sur = M.Surrogate(1024)
    with pytest.raises(M.MptracError) as e:
        sur.set_kernel(7)
    assert e.value.code == -1


@pytest.mark.parametrize("batch", [4096, 1000])
def test_training_gemms_tcgen05_match_mma_sync(M, batch):
    """The training GEMMs on tcgen05 (128 x 128 tiles, K chunks of 64 in two shared-memory
    stages) against the warp-level mma.sync GEMMs: the forward outputs agree to float32
    rounding (same bf16 operands, K = 16 products accumulated in the same order), and the
    gradients, whose split-K partial sums are added atomically in another grouping, to 1e-5.
    batch 1000 leaves a ragged 128-row tile and a K range that is not a multiple of 64."""
    P, mu_x, sd_x, mu_y, sd_y, X, Y = _random_model(9, batch)
    out = {}
    for kern in (M.SURR_KERNEL_MMA_SYNC, M.SURR_KERNEL_TCGEN05):
        sur = M.Surrogate(8192)
        sur.set_kernel(kern)
        sur.set_params(S.flatten(P).astype(np.float32))
        sur.set_norm(mu_x, sd_x, mu_y, sd_y)
        yh = sur.forward(torch.from_numpy(X).cuda()).cpu().numpy()
        loss = sur.grads(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()).item()
        sur.status()
        out[kern] = (yh, loss, sur.get_grads())
    a, b = out[M.SURR_KERNEL_MMA_SYNC], out[M.SURR_KERNEL_TCGEN05]
    np.testing.assert_allclose(b[0], a[0], rtol=1e-6, atol=1e-6 * np.abs(a[0]).max())
    assert abs(b[1] - a[1]) <= 1e-5 * abs(a[1])
    np.testing.assert_allclose(b[2], a[2], rtol=1e-5, atol=1e-5 * np.abs(a[2]).max())


def test_train_epoch_equals_step_by_step(M):
    """mptrac_surr_train_epoch makes exactly the Adam steps of single mptrac_surr_train_step calls
    with the cosine learning rates evaluated on the host, bit for bit (rows past the last whole
    batch unused); invalid arguments are rejected before anything runs.  Batches of 64 keep the
    gradients deterministic: every reduction is then done by one block (larger batches split the
    sums across blocks that add their parts with atomics, in any order)."""
    import math
    batch, lr, lr_min, total = 64, 2e-3, 2e-5, 12
    P, mu_x, sd_x, mu_y, sd_y, X, Y = _random_model(10, 5 * batch + 30)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    a = _gpu_model(M, M.SURR_KERNEL_TCGEN05, P, mu_x, sd_x, mu_y, sd_y, max_batch=batch)
    b = _gpu_model(M, M.SURR_KERNEL_TCGEN05, P, mu_x, sd_x, mu_y, sd_y, max_batch=batch)
    la = torch.zeros(1, device="cuda")
    lb = torch.zeros(1, device="cuda")
    a.train_epoch(Xd, Yd, batch, lr, lr_min, 2, total, la)          # steps 3 .. 7 of a 12-step decay
    for k in range(5):
        step = 3 + k
        lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / total))
        b.train_step(Xd[k * batch:(k + 1) * batch], Yd[k * batch:(k + 1) * batch], lr_t, step, lb)
    torch.cuda.synchronize()
    theta = a.get_params()
    np.testing.assert_array_equal(theta, b.get_params())
    assert la.item() == lb.item() and la.item() > 0
    assert not np.array_equal(theta, S.flatten(P).astype(np.float32))
    bad = ((Xd, Yd, 0, lr, lr_min, 0, total),              # empty batch
           (Xd, Yd, batch + 1, lr, lr_min, 0, total),      # above max_batch
           (Xd[:batch - 1], Yd[:batch - 1], batch, lr, lr_min, 0, total),   # no whole batch
           (Xd, Yd, batch, lr, 0.0, 0, total),             # lr_min not > 0
           (Xd, Yd, batch, 1e-5, 2e-5, 0, total),          # lr_max < lr_min
           (Xd, Yd, batch, lr, lr_min, 10, total),         # steps 11 .. 15 past the schedule
           (Xd, Yd, batch, lr, lr_min, -1, total))
    for args in bad:
        with pytest.raises(M.MptracError) as e:
            a.train_epoch(*args, la)
        assert e.value.code == -1
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.get_params(), theta)   # nothing ran


@pytest.fixture(scope="module")
def field_1deg(M):
    from workloads import grid_1deg_60lev
    grid = grid_1deg_60lev()
    m = fourier_modes(2)
    f0, f1 = fourier_snapshot(grid, m, 0.0), fourier_snapshot(grid, m, T6H)
    return grid, f0, f1, make_ctx(M, grid, [f0, f1], [0.0, T6H])


def test_fused_inference_full_size_sampled(M, field_1deg):
    """At the size of the surrogate run: 1e7 + 77 particles (a ragged last tile) on the 1-degree,
    60-level grid, one 30-minute segment of the tcgen05 inference as the run launches it; 3000
    sampled particles (the first and the last 1000, and 1000 drawn between) against the oracle
    pipeline, and the kernel's count of fallback particles against the flags it wrote."""
    grid, f0, f1, ctx = field_1deg
    n, t = 10_000_077, 3600.0
    st = uniform_particles(n, grid.plev, seed=23)
    rng = np.random.default_rng(24)
    idx = np.unique(np.concatenate([np.arange(1000), np.arange(n - 1000, n),
                                    rng.choice(np.arange(1000, n - 1000), 1000, replace=False)]))
    sub = {k: v[idx] for k, v in st.items()}
    X = S.features(grid, f0, f1, t, 0.0, T6H, sub["lon"], sub["lat"], sub["p"])
    P = S.init_params(4)
    for b in ("b1", "b2", "b3"):
        P[b] = rng.standard_normal(P[b].shape) * 0.1
    mu_x, sd_x = X.mean(axis=0), X.std(axis=0)
    sd_x[sd_x < 1e-12] = 1.0
    mu_y, sd_y = np.array([500.0, -300.0, 0.001]), np.array([2.0e4, 1.5e4, 0.05])
    sur = _gpu_model(M, M.SURR_KERNEL_TCGEN05, P, mu_x, sd_x, mu_y, sd_y, max_batch=1024)
    parts = M.Particles.from_numpy(st, meso=False, release=False)
    fb = torch.zeros(n, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    sur.advance(ctx, parts, t, 1800.0, fb, count)
    sur.status()
    it = torch.from_numpy(idx).cuda()
    got = {k: getattr(parts, k)[it].cpu().numpy() for k in ("lon", "lat", "p")}
    fbn = fb[it].cpu().numpy()
    assert count.item() == int(fb.sum().item()) > 0
    _compare_with_oracle_pipeline(grid, sub, X, got, fbn, P, mu_x, sd_x, mu_y, sd_y)
    assert 0.05 < fbn.mean() < 0.5
