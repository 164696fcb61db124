"""Evaluate Triton's own Philox4x32-10 on the CPU (interpreter mode).

Test helper, run as a subprocess by test_oracle_philox.py: it reads
"seed c0 c1 c2 c3" lines from stdin and prints the four output words per line.
Triton's ``tl.philox(seed, c0, c1, c2, c3)`` uses key = (seed mod 2^32,
seed >> 32) and ten rounds by default; it is an implementation independent of
this repository, so agreement pins the oracle's generator.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(out_ptr, seed, c0_ptr, c1_ptr, c2_ptr, c3_ptr, n,
                   BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c0_ptr + offs, mask=m)
    c1 = tl.load(c1_ptr + offs, mask=m)
    c2 = tl.load(c2_ptr + offs, mask=m)
    c3 = tl.load(c3_ptr + offs, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + offs * 4 + 0, a, mask=m)
    tl.store(out_ptr + offs * 4 + 1, b, mask=m)
    tl.store(out_ptr + offs * 4 + 2, c, mask=m)
    tl.store(out_ptr + offs * 4 + 3, d, mask=m)


def main():
    for line in sys.stdin:
        if not line.strip():
            continue
        seed, *ctr = [int(v) for v in line.split()]
        c = [torch.tensor([np.uint32(v).astype(np.int32)], dtype=torch.int32)
             for v in ctr]
        out = torch.zeros(4, dtype=torch.int32)
        _philox_kernel[(1,)](out, seed, *c, 1, BLOCK=1)
        print(" ".join(str(int(v) & 0xFFFFFFFF) for v in out.tolist()))


if __name__ == "__main__":
    main()
