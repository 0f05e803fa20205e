"""Host model of the batched solver's shared-memory arithmetic (smem_for,
vert_bytes, carve_vertex and the migration test in csrc/mst_batched.cu), on
GB300's limits: 228 KB of shared memory per SM, 227 KB per CTA (opt-in),
1 KB reserved per CTA.

Checked for every CTA size and split the autotuner can pick:
- the dynamic shared memory plus the kernel's static shared memory and the
  per-CTA reserve fits both the SM's share and the per-CTA limit;
- arrays moved into shared memory fit the budget, and the merging tail's
  pair table, which starts at the second minimum array, stays inside the
  budget and overlaps none of the arrays the tail reads (the first minimum
  array, parents, new ids, labels);
- the tail's component limit is 0 or between 8 and 128, and the pair table
  holds its triangle of pairs."""
import pytest

PER_SM, PER_BLOCK, RESERVE = 233472, 232448, 1024
STATIC = {128: 1136, 256: 1216, 512: 1376, 1024: 1696}  # ptxas: bytes of static smem
TAIL_MAX_N = 128


def al16(x):
    return (x + 15) & ~15


def smem_for(bps, static):
    share = PER_SM // bps
    s = share - RESERVE - static if share > RESERVE + static else 0
    s = min(s, PER_BLOCK - static if PER_BLOCK > static else 0)
    return s & ~255


def vert_bytes(n):
    return 2 * al16(n * 8) + 3 * al16(n * 4)


def tri_size(n):
    return n * (n - 1) // 2


def carve_vertex(budget, n):
    """Offsets of mA, parent, nid, lab, mB; the pair table's offset and tail_n."""
    off, p = {}, 0
    for name, size in (("mA", n * 8), ("parent", n * 4), ("nid", n * 4), ("lab", n * 4)):
        off[name] = (p, al16(size))
        p += al16(size)
    off["mB"] = (p, al16(n * 8))
    left = budget - p
    tn = TAIL_MAX_N
    while tn >= 8 and tri_size(tn) * 8 > left:
        tn -= 1
    return off, (p if tn >= 8 else None), (tn if tn >= 8 else 0)


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
@pytest.mark.parametrize("bps", [1, 2, 3, 4, 8])
def test_budget_fits_the_sm_and_the_cta(threads, bps):
    s = smem_for(bps, STATIC[threads])
    assert s % 256 == 0 and s > 0
    assert s + STATIC[threads] <= PER_BLOCK
    assert bps * (s + STATIC[threads] + RESERVE) <= PER_SM


@pytest.mark.parametrize("bps", [1, 2, 3, 4])
def test_moved_arrays_and_pair_table_stay_apart(bps):
    budget = smem_for(bps, STATIC[1024])
    n_max = 1
    while vert_bytes(n_max + 1) <= budget:
        n_max += 1
    for n in sorted({2, 3, 7, 64, 127, 128, 129, 1000, n_max // 3, n_max // 2, n_max - 1, n_max}):
        assert vert_bytes(n) <= budget  # the migration test admits it
        off, ptab, tn = carve_vertex(budget, n)
        end_arrays = off["mB"][0] + off["mB"][1]
        assert end_arrays == vert_bytes(n) <= budget
        if tn == 0:
            continue
        assert 8 <= tn <= TAIL_MAX_N
        lo, hi = ptab, ptab + tri_size(tn) * 8
        assert hi <= budget
        for name in ("mA", "parent", "nid", "lab"):  # what the tail reads beside the table
            a, size = off[name]
            assert a + size <= lo or a >= hi, name
        # the tail indexes its arrays below n_t <= min(tail_n, components), and
        # components never exceed the capacity the arrays were carved for
        assert min(tn, n) <= n


def test_second_minimum_array_start_gives_the_tail_more_room():
    budget = smem_for(2, STATIC[1024])  # the default split: 113,920 bytes
    assert budget == 113920
    # a 65,536-vertex graph moves with 3,352 components: its tail may now start
    # at up to 108 components; the table after all five arrays allowed 71
    off, ptab, tn = carve_vertex(budget, 3352)
    assert tn == 108
    left_after_all = budget - vert_bytes(3352)
    old = TAIL_MAX_N
    while old >= 8 and tri_size(old) * 8 > left_after_all:
        old -= 1
    assert old == 71
