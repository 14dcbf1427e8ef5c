"""Host-side integer arithmetic the kernels rely on, checked exhaustively on the CPU.

The recompute form's phase-encode roots are roots[(ky iy) mod ny]; the kernel takes the
remainder as a - umulhi(a, magic) ny with magic = ceil(2^32 / ny) (0 for ny = 1), which is
exact only if the quotient umulhi(a, magic) = floor(a / ny) for every product a = ky iy the
kernel forms (0 <= a < ny^2) and every row count the form accepts (ny <= 256)."""
import numpy as np


def test_magic_number_quotient_is_exact_for_every_row_count():
    for n in range(1, 257):
        magic = 0 if n == 1 else (2 ** 32 + n - 1) // n
        a = np.arange(n * n, dtype=np.uint64)
        q = (a * np.uint64(magic)) >> np.uint64(32)
        assert np.array_equal(q, a // np.uint64(n)), n
