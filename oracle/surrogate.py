"""Learned displacement surrogate: features, network, loss and optimiser -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this restates, in float64, the surrogate
the project adds on top of MPTRAC's advection module (Section 3.2): a small MLP
that maps a particle's local wind stencil to its displacement over 10 plain
midpoint substeps (30 min at dt = 180 s), trained on trajectories of the plain
integrator, with the plain integrator as fallback outside the training
envelope.

Features (168, zero-padded to 176), at the segment start (x, t):
* the nearest grid node (i0, j0, k0): x = ((lon - lon0) mod 360)/dlon,
  i0 = floor(x + 1/2) mod nx; y = (lat - lat0)/dlat, j0 = floor(y + 1/2)
  clamped to [1, ny-2]; z = k + fz (the fractional level index of the
  interpolation's cell), k0 = floor(z + 1/2) clamped to [1, nz-2];
* the values of u, v, omega at the 3 x 3 x 3 nodes around it on both
  snapshots, ordered [snapshot][variable][dk][dj][di] (162);
* the offsets x - i0 (folded into [-1/2, 1/2)), y - j0, z - k0 (3);
* the time weight w = (t - t0)/(t1 - t0) (1); sin(lat), cos(lat) (2).
Targets: east and north displacement in metres at the start latitude,
dx = R cos(lat0) dlon_rad, dy = R dlat_rad (dlon folded into [-180, 180)),
and dz = ln(p1/p0).

Network: x_hat = (x - mu_x)/sd_x;  z1 = x_hat W1 + b1, h1 = gelu(z1);
z2 = h1 W2 + b2, h2 = gelu(z2);  y_hat = h2 W3 + b3;  y = y_hat sd_y + mu_y,
with gelu(x) = x/2 (1 + erf(x/sqrt 2)).  Loss: mean over samples and the 3
outputs of (y_hat - (y_target - mu_y)/sd_y)^2.  Optimiser: Adam (Kingma & Ba,
2015) with bias correction.

The network is a BF16 network: every operand of its matrix products is a
bfloat16 value, accumulated exactly (here: in float64).  ``forward`` and
``loss_and_grads`` take that rounding as ``rnd`` (``bf16_round``; None = no
rounding, the real-valued network).  With it, the forward pass rounds the
hidden activations h1, h2 before they enter the next product, and the backward
pass rounds the upstream gradients dy, dz2, dz1 before they enter theirs; each
bias gradient is the column sum of the same rounded gradient that its layer's
weight gradient uses.  The caller rounds the weights and x_hat.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import interp
from .transport import R_EARTH

NFEAT, KPAD, HIDDEN, NOUT = 168, 176, 128, 3
SHAPES = (("W1", (KPAD, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN, NOUT)), ("b3", (NOUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        size = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


# --------------------------------------------------------------------------
# features and targets
# --------------------------------------------------------------------------
def nearest_node(grid, lon, lat, p):
    lon = np.asarray(lon, np.float64)
    lat = np.asarray(lat, np.float64)
    x = np.mod(lon - grid.lon0, 360.0) / grid.dlon
    xr = np.floor(x + 0.5)
    i0 = np.mod(xr.astype(np.int64), grid.nx)
    ox = x - xr
    y = (lat - grid.lat0) / grid.dlat
    j0 = np.clip(np.floor(y + 0.5).astype(np.int64), 1, grid.ny - 2)
    oy = y - j0
    _, _, _, k, _, _, fz = interp.locate(grid, lon, lat, p)
    z = k + fz
    k0 = np.clip(np.floor(z + 0.5).astype(np.int64), 1, grid.nz - 2)
    oz = z - k0
    return i0, j0, k0, ox, oy, oz


def features(grid, f0, f1, t, t0, t1, lon, lat, p):
    """Raw features [n, 176] (float64) at positions (lon, lat, p) and time t.

    f0, f1: dicts u, v, w of the two snapshots (arrays [nz][ny][nx]).
    """
    i0, j0, k0, ox, oy, oz = nearest_node(grid, lon, lat, p)
    n = np.asarray(lon).size
    X = np.zeros((n, KPAD))
    col = 0
    for f in (f0, f1):
        for var in ("u", "v", "w"):
            a = np.asarray(f[var], dtype=np.float64)
            for dk in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    for di in (-1, 0, 1):
                        X[:, col] = a[k0 + dk, j0 + dj, np.mod(i0 + di, grid.nx)]
                        col += 1
    X[:, 162], X[:, 163], X[:, 164] = ox, oy, oz
    X[:, 165] = (t - t0) / (t1 - t0)
    phi = np.radians(np.asarray(lat, np.float64))
    X[:, 166], X[:, 167] = np.sin(phi), np.cos(phi)
    return X


def targets(lon0, lat0, p0, lon1, lat1, p1):
    dlon = np.mod(np.asarray(lon1, float) - lon0 + 180.0, 360.0) - 180.0
    dx = R_EARTH * np.cos(np.radians(lat0)) * np.radians(dlon)
    dy = R_EARTH * np.radians(np.asarray(lat1, float) - lat0)
    dz = np.log(np.asarray(p1, float) / p0)
    return np.stack([dx, dy, dz], axis=1)


def apply_displacement(lon0, lat0, p0, y):
    """Inverse of ``targets`` (before the position rules)."""
    lon1 = lon0 + np.degrees(y[:, 0] / (R_EARTH * np.cos(np.radians(lat0))))
    lat1 = lat0 + np.degrees(y[:, 1] / R_EARTH)
    p1 = p0 * np.exp(y[:, 2])
    return lon1, lat1, p1


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def normalise(X, mu, sd):
    return (np.asarray(X, np.float64) - mu) / sd


def bf16_round(x):
    """Nearest bfloat16 value (8 significant bits), ties to even; finite normal inputs and zero."""
    m, e = np.frexp(np.asarray(x, np.float64))
    return np.ldexp(np.round(np.ldexp(m, 8)), e - 8)


def _identity(a):
    return a


def forward(P, xh, rnd=None):
    """Normalised outputs and the activations (xh, z1, h1, z2, h2), h before rounding."""
    r = rnd or _identity
    z1 = xh @ P["W1"] + P["b1"]
    h1 = gelu(z1)
    z2 = r(h1) @ P["W2"] + P["b2"]
    h2 = gelu(z2)
    yh = r(h2) @ P["W3"] + P["b3"]
    return yh, (xh, z1, h1, z2, h2)


def loss_and_grads(P, xh, yt_hat, rnd=None, trace=None):
    """MSE loss in normalised units and its gradients with respect to every parameter.

    ``trace`` (a dict, optional) receives the forward activations and the
    upstream gradients dy, dz2, dz1 before rounding.
    """
    r = rnd or _identity
    yh, (x, z1, h1, z2, h2) = forward(P, xh, rnd)
    n = xh.shape[0]
    res = yh - yt_hat
    loss = float(np.mean(res * res))
    dy_raw = 2.0 * res / (n * NOUT)
    dy = r(dy_raw)
    g = {"W3": r(h2).T @ dy, "b3": dy.sum(axis=0)}
    dz2_raw = (dy @ P["W3"].T) * gelu_grad(z2)
    dz2 = r(dz2_raw)
    g["W2"], g["b2"] = r(h1).T @ dz2, dz2.sum(axis=0)
    dz1_raw = (dz2 @ P["W2"].T) * gelu_grad(z1)
    dz1 = r(dz1_raw)
    g["W1"], g["b1"] = x.T @ dz1, dz1.sum(axis=0)
    if trace is not None:
        trace.update(yh=yh, z1=z1, h1=h1, z2=z2, h2=h2, dy=dy_raw, dz2=dz2_raw, dz1=dz1_raw)
    return loss, g


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            a = 1.0 / math.sqrt(shp[0])
            P[name] = rng.uniform(-a, a, shp)
        else:
            P[name] = np.zeros(shp)
    P["W1"][NFEAT:] = 0.0
    return P


def in_envelope(xh, lat, lat_max=80.0, zmax=4.0):
    """Inside the training envelope: |lat| <= lat_max and every standardised feature within +-zmax."""
    return (np.abs(lat) <= lat_max) & np.all(np.abs(xh[:, :NFEAT]) <= zmax, axis=1)
