"""Independent Philox4x32-10 reference: Triton's `tl.philox`, run by Triton's
CPU interpreter.  Reads counters (uint32 [n][4]) and a 64-bit key from argv
files, writes the four output words.  Used only by the oracle pin tests."""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
    c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
    c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
    c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a, mask=m)
    tl.store(out_ptr + 4 * i + 1, b, mask=m)
    tl.store(out_ptr + 4 * i + 2, c, mask=m)
    tl.store(out_ptr + 4 * i + 3, d, mask=m)


def main():
    ctr = np.load(sys.argv[1]).astype(np.uint32)
    seed = int(sys.argv[2])
    n = ctr.shape[0]
    block = 1 << max(0, (n - 1).bit_length())
    out = torch.zeros(n * 4, dtype=torch.int32)
    _philox_kernel[(1,)](out, torch.from_numpy(ctr.view(np.int32).ravel().copy()), seed, n, BLOCK=block)
    np.save(sys.argv[3], out.numpy().view(np.uint32).reshape(n, 4))


if __name__ == "__main__":
    main()
