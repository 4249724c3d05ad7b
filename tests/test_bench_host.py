"""Host-side pins of the benchmark's units: the sweep's per-n batch sizes
(2^20 systems capped at 6 GiB of A, b, x, ipiv and info), the algorithmic
bytes per system and the algorithmic FP64 flops per system that the
roofline divides by, the latter against an operation count of the
elimination and the two substitutions done step by step."""
import bench


def test_sweep_batch_sizes():
    assert bench.sweep_batch(26) == 1 << 20
    assert bench.sweep_batch(27) == 1010422
    assert bench.sweep_batch(32) == 729113
    for n in range(1, 33):
        S = bench.sweep_batch(n)
        assert S <= 1 << 20 and S * bench.bytes_per_system(n) <= 6 * (1 << 30)
        assert S == 1 << 20 or (S + 1) * bench.bytes_per_system(n) > 6 * (1 << 30)


def test_bytes_per_system():
    # A and b read (8 n^2 + 8 n), x written (8 n), ipiv (4 n) and info (4)
    assert bench.bytes_per_system(8) == 676
    assert bench.bytes_per_system(32) == 8836


def counted_flops(n):
    """FP64 operations of getrf + getrs counted loop by loop (FMA = 2)."""
    flops = 0
    for k in range(n):
        if k < n - 1:
            flops += 1                      # reciprocal of the pivot
        flops += n - k - 1                  # multipliers
        flops += 2 * (n - k - 1) ** 2       # trailing update
    for i in range(n):
        flops += 2 * i                      # forward substitution, row i
    for i in range(n):
        flops += 2 * (n - 1 - i) + 1        # back substitution, row i, and its division
    return flops


def test_flops_per_system_matches_the_count():
    assert bench.flops_per_system(8) == 435
    assert bench.flops_per_system(32) == 23375
    for n in range(1, 33):
        assert bench.flops_per_system(n) == counted_flops(n), n
