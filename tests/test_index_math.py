"""Host check of the chunk kernel's division-free index split.

The kernel maps a flat index idx < L*S over the L x-line runs of a chunk
(S = p*nc + 1 values each) to (l, kk) with l = trunc((idx + 1/2) * (1/S)) in
FP32 arithmetic.  This test evaluates the same IEEE single-precision
operations for every tile shape the library instantiates (d = 2, 3;
n = 2..7; chunks of R = max(256 / n^(d-1), 1) and R/2 cells; every chunk
length nc) and checks l == idx // S for every idx."""
import numpy as np


def test_fp32_reciprocal_split_is_exact():
    one, half = np.float32(1.0), np.float32(0.5)
    for d in (2, 3):
        for n in range(2, 8):
            L = n ** (d - 1)
            R = max(256 // L, 1)
            for r in sorted({R, max(R // 2, 1)}):
                for nc in range(1, r + 1):
                    S = (n - 1) * nc + 1
                    inv = one / np.float32(S)
                    idx = np.arange(L * S, dtype=np.int64)
                    q = (idx.astype(np.float32) + half) * inv
                    assert q.dtype == np.float32
                    l = np.trunc(q).astype(np.int64)
                    np.testing.assert_array_equal(l, idx // S)
