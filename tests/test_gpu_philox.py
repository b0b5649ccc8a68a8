"""Philox parity: raw words bit-exact with the oracle; normals within float32 rounding."""
import numpy as np
import pytest
import torch

from oracle import philox as oph

from _gpu_common import M  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 83, 2 ** 40 + 12345, 2 ** 64 - 1])
def test_words_bit_exact(M, seed):
    rng = np.random.default_rng(seed % 1000)
    n = 100_003                        # ragged against the 256-thread blocks
    ctr = rng.integers(0, 2 ** 32, size=(4, n), dtype=np.uint64).astype(np.uint32)
    ctr[:, :3] = [[0, 0xFFFFFFFF, 1]] * 4
    out, z = M.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), seed, with_normals=True)
    got = out.cpu().numpy().view(np.uint32)
    k0, k1 = oph.seed_key(seed)
    ref = np.stack(oph.philox4x32(*ctr, k0, k1))
    np.testing.assert_array_equal(got, ref)
    zr = np.stack(oph.normals4(ctr[0], ctr[1], ctr[2], ctr[3], seed))
    np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-5, atol=5e-6)


def test_empty_and_errors(M):
    ctr = torch.zeros(4, 0, dtype=torch.int32, device="cuda")
    assert M.philox(ctr, 1).numel() == 0
