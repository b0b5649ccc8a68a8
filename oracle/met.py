"""Met snapshot storage: packing and reduced-precision codes -- TEST INFRASTRUCTURE ONLY.

The paper's ``read_met`` (Section 3.1) fills a ``met_t`` snapshot on the host and
``update device`` copies it to each GPU (Section 4.1).  The method stores each
snapshot on the device as one record per grid point holding (u, v, omega, T),
ordered ``[lat][lon][level]`` with the level index fastest, in one of three
storage precisions:

* float32: the record is the four values (T, or 0 when absent).
* bfloat16 / float16: each value x of level k and variable c is stored as the
  16-bit code q = round_nearest_even(x * 2^-e), with the per-(level, variable)
  power-of-two scale s = 2^e, e = E - 15, where maxabs = m 2^E with m in
  [0.5, 1) is the largest |x| on that level (s = 1 if maxabs = 0).  Scaled
  values then lie in [-2^15, 2^15], inside float16's finite range, and because
  s is a power of two the scaling itself is exact: the only rounding is the
  final one, bounded by half a unit in the last place of the code.

Decoding is x_hat = value(q) * s.
"""
from __future__ import annotations

import numpy as np

FP32, BF16, FP16 = 0, 1, 2
VARS = ("u", "v", "w", "T")


def level_scales(field: np.ndarray) -> np.ndarray:
    """Per-level power-of-two scales of a float32 field [nz][ny][nx]."""
    f = np.asarray(field, dtype=np.float32)
    maxabs = np.abs(f.reshape(f.shape[0], -1)).max(axis=1).astype(np.float64)
    _, E = np.frexp(maxabs)
    s = np.ldexp(1.0, E - 15)
    s = np.where(maxabs == 0.0, 1.0, s)
    return s.astype(np.float32)


def bf16_code(x32: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit pattern, round to nearest, ties to even (finite inputs)."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    return ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)).astype(np.uint16)


def bf16_value(q: np.ndarray) -> np.ndarray:
    return (np.asarray(q, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def fp16_code(x32: np.ndarray) -> np.ndarray:
    return np.asarray(x32, dtype=np.float32).astype(np.float16).view(np.uint16)


def fp16_value(q: np.ndarray) -> np.ndarray:
    return np.asarray(q, dtype=np.uint16).view(np.float16).astype(np.float64)


def quantize(field: np.ndarray, storage: int):
    """Codes (uint16, same shape) and per-level scales (float32 [nz])."""
    s = level_scales(field)
    scaled = (np.asarray(field, dtype=np.float32) * (1.0 / s)[:, None, None]).astype(np.float32)
    q = bf16_code(scaled) if storage == BF16 else fp16_code(scaled)
    return q, s


def dequantize(q: np.ndarray, s: np.ndarray, storage: int) -> np.ndarray:
    val = bf16_value(q) if storage == BF16 else fp16_value(q)
    return val * s.astype(np.float64)[:, None, None]


def stored_fields(fields: dict, storage: int) -> dict:
    """The values the method interpolates (float64), after storage rounding."""
    out = {}
    for name, f in fields.items():
        if storage == FP32:
            out[name] = np.asarray(f, dtype=np.float32).astype(np.float64)
        else:
            q, s = quantize(f, storage)
            out[name] = dequantize(q, s, storage)
    return out


def pack(fields: dict, storage: int):
    """Expected device records and scales of one snapshot.

    Returns ``(records, scales)``: records has shape [ny][nx][nz][4] (float32
    values for FP32 storage, uint16 codes otherwise; a missing T is 0), scales
    has shape [4][nz] float32 (all ones for FP32 storage and for a missing T).
    """
    nz, ny, nx = fields["u"].shape
    dtype = np.float32 if storage == FP32 else np.uint16
    rec = np.zeros((ny, nx, nz, 4), dtype=dtype)
    scales = np.ones((4, nz), dtype=np.float32)
    for c, name in enumerate(VARS):
        if name not in fields or fields[name] is None:
            continue
        f = np.asarray(fields[name], dtype=np.float32)
        if storage == FP32:
            vals = f
        else:
            vals, scales[c] = quantize(f, storage)
        rec[..., c] = np.transpose(vals, (1, 2, 0))
    return rec, scales
