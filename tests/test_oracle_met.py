"""Pins of the oracle's met storage (packing, bf16/fp16 codes, per-level scales)."""
import numpy as np
import pytest
import torch

from oracle import met


def _edge_values():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000).astype(np.float32) * np.float32(1000)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 1 + 2 ** -11, 1 + 3 * 2 ** -11,
                     0.0, -0.0, 2 ** -20, 32768.0, -32768.0, 65504.0 / 2], dtype=np.float32)
    return np.concatenate([x, ties])


def test_bf16_code_matches_torch():
    x = _edge_values()
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(met.bf16_code(x), ref)


def test_fp16_code_matches_torch():
    x = _edge_values()
    ref = torch.from_numpy(x).to(torch.float16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(met.fp16_code(x), ref)


def test_bf16_hand_cases():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.0], dtype=np.float32)
    np.testing.assert_array_equal(met.bf16_code(x), np.array([0x3F80, 0x3F80, 0x3F82, 0xC000], np.uint16))
    np.testing.assert_array_equal(met.bf16_value(met.bf16_code(x)), [1.0, 1.0, 1 + 2 ** -6, -2.0])


def test_level_scales_power_of_two():
    f = np.zeros((3, 2, 2), np.float32)
    f[0, 0, 0] = 20.0        # frexp(20) = 0.625 * 2^5 -> scale 2^-10
    f[1, 1, 1] = -0.5        # 0.5 * 2^0 -> 2^-15
    s = met.level_scales(f)
    np.testing.assert_array_equal(s, np.array([2.0 ** -10, 2.0 ** -15, 1.0], np.float32))
    assert np.all(np.abs(f / s[:, None, None]) <= 2 ** 15)


@pytest.mark.parametrize("storage,u", [(met.BF16, 2.0 ** -8), (met.FP16, 2.0 ** -11)])
def test_quantization_error_bound(storage, u):
    """|x - x_hat| <= u |x| (round to nearest: half an ulp of the code)."""
    rng = np.random.default_rng(1)
    f = (rng.standard_normal((4, 30, 40)) * np.array([20, 0.5, 3e-3, 250])[:, None, None]).astype(np.float32)
    q, s = met.quantize(f, storage)
    xh = met.dequantize(q, s, storage)
    x = f.astype(np.float64)
    # values well inside the normal range of the code: relative bound
    big = np.abs(x / s[:, None, None]) >= 2.0 ** -10
    assert np.all(np.abs(x - xh)[big] <= u * np.abs(x)[big])
    assert np.max(np.abs(x - xh)) <= u * np.max(np.abs(x))


def test_pack_layout():
    rng = np.random.default_rng(2)
    fields = {k: rng.standard_normal((5, 4, 6)).astype(np.float32) for k in ("u", "v", "w")}
    rec, sc = met.pack(fields, met.FP32)
    assert rec.shape == (4, 6, 5, 4)
    for c, k in enumerate(("u", "v", "w")):
        for (kk, j, i) in [(0, 0, 0), (4, 3, 5), (2, 1, 3)]:
            assert rec[j, i, kk, c] == fields[k][kk, j, i]
    assert np.all(rec[..., 3] == 0) and np.all(sc == 1)
    recb, scb = met.pack(fields, met.BF16)
    assert recb.dtype == np.uint16
    q, s = met.quantize(fields["v"], met.BF16)
    np.testing.assert_array_equal(recb[..., 1], np.transpose(q, (1, 2, 0)))
    np.testing.assert_array_equal(scb[1], s)
