"""Host-side arithmetic of the benchmark: the algorithmic work counts behind
every roofline figure, checked by enumerating the operations they count on
small orders (no GPU)."""
import bench


def test_recursion_pairs_by_enumeration():
    """One FMA per (T, S) pair of Eq. recursion: T a proper nonempty subset of S
    holding S's lowest element."""
    for n in range(1, 9):
        pairs = 0
        for S in range(1, 1 << n):
            j = S & -S
            T = (S - 1) & S
            while T:
                if T & j:
                    pairs += 1
                T = (T - 1) & S
        assert bench.sc_flops(n) == 2 * pairs


def test_tree_updates_by_enumeration():
    """Schur updates of the FPM tree: every node at level l has one Schur-
    complemented child of order n - l - 1, one FMA per entry; one reciprocal
    and one minor product per node; a = det^2 one multiply per nonempty set."""
    for n in range(1, 11):
        fma = sum((1 << l) * (n - l - 1) ** 2 for l in range(n - 1))
        nodes = (1 << n) - 1
        assert bench.flops_per_set(n) == 2 * fma + 2 * nodes + bench.sc_flops(n) + nodes


def test_headline_constants():
    assert bench.flops_per_set(12) == 559769
    assert bench.bytes_per_set(12) == 8 * 144 + 16 * 4096 == 66688


def test_permanent_pairs_by_enumeration():
    """One product and one addition per (T subset of S) pair, plus n 2^n row sums."""
    for n in range(1, 8):
        pairs = sum(1 for S in range(1 << n) for T in range(1 << n) if T & ~S == 0)
        assert pairs == 3 ** n
        assert bench.perm_flops(n) == 2 * pairs + n * (1 << n)


def test_fast_subset_convolution_count_and_switch():
    for n in range(1, 17):
        transforms = 2 * n * n * (1 << (n - 1))        # ranked zeta + ranked Mobius, one add per pair
        log = (1 << n) * (n * (n - 1) + 3 * n)          # per mask: k-1 FMAs, a multiply-add and a scaling per k
        assert bench.fsc_flops(n) == transforms + log
        if n < bench.FSC_FROM_N:
            assert bench.cdet_path_flops(n) == bench.flops_per_set(n)
        else:
            assert bench.cdet_path_flops(n) == bench.flops_per_set(n) - bench.sc_flops(n) + bench.fsc_flops(n)


def readable_entries(m):
    """Entries of an m x m node (m even) that a minor keeping at most one row and
    column of each 2 x 2 diagonal block can contain: the diagonal and every
    entry between two different blocks."""
    return sum(1 for r in range(m) for q in range(m) if r == q or r // 2 != q // 2)


def test_keldysh_tree_count():
    """Complex Schur updates of the XOR tree (8 real flops each): every node at
    depth l has two children, each an update of the readable entries of order
    2(n - l - 1)."""
    for n in range(1, 9):
        cfma = sum((1 << l) * 2 * readable_entries(2 * (n - l - 1)) for l in range(n - 1))
        children = sum(1 << (l + 1) for l in range(n))   # a pivot reciprocal and product each (12 flops)
        assert bench.keldysh_flops(n) == 8 * cfma + 12 * children + 2 * (1 << n)


def test_nand_tree_count():
    """The ternary tree: every node at depth l has two kept children of order
    m = 2(n - l - 1), each a rank-1 update of its readable entries (an FMA), m
    row factors and 3 flops for the pivot reciprocal and node product."""
    for n in range(1, 9):
        per_child = [2 * readable_entries(2 * (n - l - 1)) + 2 * (n - l - 1) + 3 for l in range(n)]
        assert bench.nand_flops(n) == sum(3 ** l * 2 * per_child[l] for l in range(n))


def test_throughput_helpers():
    assert bench.job_throughput(1000, 1, 10, 2.0) == 5000.0
    assert bench.job_throughput(1000, 4, 10, 2.0) == 20000.0
    assert bench.max_over_ranks(1.5, 1) == 1.5


def test_minor_set_count_splits_into_tree_and_recursion():
    """A minor set's flops are the tree's (Schur updates, reciprocals and
    products), the squares of the minors, and the recursion's FMAs."""
    for n in range(1, 17):
        assert bench.flops_per_set(n) == bench.minors_flops(n) + (2 ** n - 1) + bench.sc_flops(n)


def test_cpu_rate_sizes_a_bounded_sample():
    """The CPU baselines time a sample sized from a probe: whole multiples of
    the thread count, never more than the workload, at least one per thread."""
    import numpy as np
    A = np.zeros((100, 3, 3))
    calls = []

    def run(sample, threads):
        calls.append(sample.shape[0])
        return np.zeros((sample.shape[0], 8))
    r, threads, count, dt = bench.cpu_rate(run, A, 0.0, 4)
    assert threads == 4 and count % 4 == 0 and 4 <= count <= 100 and r > 0
    assert calls[0] == 2 and calls[1] == 4 and calls[2] == count
