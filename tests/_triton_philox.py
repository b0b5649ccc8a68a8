"""Helper run in a subprocess: Philox4x32 words from Triton's own implementation.

Triton (a third-party library) ships a Philox4x32 routine; in interpreter mode
(TRITON_INTERPRET=1) it runs on the CPU.  Reads counters/seeds from an .npz
file given on the command line and writes the four output words back.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c0p + offs)
    c1 = tl.load(c1p + offs)
    c2 = tl.load(c2p + offs)
    c3 = tl.load(c3p + offs)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out + offs, a)
    tl.store(out + N + offs, b)
    tl.store(out + 2 * N + offs, c)
    tl.store(out + 3 * N + offs, d)


def main(path_in, path_out):
    d = np.load(path_in)
    ctr = d["ctr"].astype(np.uint32)       # (4, N)
    seeds = d["seeds"].astype(np.uint64)
    N = ctr.shape[1]
    res = []
    for s in seeds:
        out = torch.zeros(4 * N, dtype=torch.uint32)
        cs = [torch.from_numpy(np.ascontiguousarray(ctr[i])) for i in range(4)]
        _philox_kernel[(1,)](out, *cs, int(s), N=N)
        res.append(out.numpy().reshape(4, N))
    np.savez(path_out, words=np.stack(res))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
