"""Seeded initial weights of the learned surrogate's network (inputs only).

The network has layers 176 -> 128 -> 128 -> 3 (168 features zero-padded to 176).
Its starting point is a draw: weights uniform in +-1/sqrt(fan_in), the rows of
the 8 padding inputs zero, biases zero.  The values are returned in the flat
parameter order W1 [176][128], b1, W2 [128][128], b2, W3 [128][3], b3.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((176, 128, 8), (128, 128, 0), (128, 3, 0))     # fan_in, fan_out, zero padding rows


def initial_weights(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out, pad in LAYERS:
        a = 1.0 / np.sqrt(fan_in)
        w = rng.uniform(-a, a, (fan_in, fan_out))
        if pad:
            w[fan_in - pad:] = 0.0
        parts += [w.ravel(), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)
