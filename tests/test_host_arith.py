"""Host-side checks of integer arithmetic the tensor-core epilogue relies on.

The padded-row modes find the row of an output position q as
umulhi(q, floor(2^32 / P) + 1) instead of q / P.  The launch uses this only
when every position of a leaf is below 2^16; pitches P = W + 2 stay within
[6, 258] (maps of 4 to 256 columns).  The identity is checked here for every
such position and pitch.
"""
import numpy as np


def test_multiply_high_row_division_is_exact():
    q = np.arange(1 << 16, dtype=np.uint64)
    for P in range(3, 259):
        magic = np.uint64((1 << 32) // P + 1)
        row = (q * magic) >> np.uint64(32)
        assert np.array_equal(row, q // np.uint64(P)), P
