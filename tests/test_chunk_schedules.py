"""Index facts behind the FP32 prolongation kernels' chunk schedules (Section 2.2.1, Eqs. 8-11).

A fine node jf of an axis refined by r = 2^lr takes the coarse centre i = floor(jf / r + 1/2) and
the offset s = jf / r - i in [-1/2, 1/2) (the interpolation point of Eqs. 8-11).  The FP32
kernels give each warp chunks of 8 fine nodes that start at multiples of 8 and replace the per-node
centre computation by closed forms:
  r <= 8: node j0 + j has the centre (j0 >> lr) + (j >> lr) + [2 (j mod r) >= r] and the offset
          (j mod r) / r or ((j mod r) - r) / r, and the chunk's last centre is
          (7 >> lr) + [2 (7 mod r) >= r] past its first (the rows loaded up front);
  r >= 16: all 8 nodes share one centre and their offsets step by 1 / r.
Both are checked here against the definition, for every chunk of several axis lengths, and so is
the row range the kernels read ([-2, n + 2], inside the periodic wrap's [-n, 2n) for n >= 3).
The last test checks the two-line stage kernel's traversal of a launch's work items in runs of
consecutive items: every item once.
"""
import math
from fractions import Fraction

import pytest


def centre_offset(jf, r):
    t = Fraction(jf, r)
    i = math.floor(t + Fraction(1, 2))
    return i, t - i


def schedule_small(j0, lr, j):
    r = 1 << lr
    m = j & (r - 1)
    c = (j0 >> lr) + (j >> lr) + (0 if 2 * m < r else 1)
    s = Fraction(m if 2 * m < r else m - r, r)
    return c, s


@pytest.mark.parametrize("lr", [1, 2, 3])
@pytest.mark.parametrize("n", [5, 6, 12, 13, 40])
def test_compile_time_schedule_matches_definition(lr, n):
    r = 1 << lr
    nf = n * r
    nx = (7 >> lr) + (0 if 2 * (7 & (r - 1)) < r else 1)
    for j0 in range(0, nf - 7, 8):  # whole chunks
        c0 = centre_offset(j0, r)[0]
        assert c0 == j0 >> lr  # a chunk starts at a coarse node
        cents = []
        for j in range(8):
            c, s = centre_offset(j0 + j, r)
            assert (c, s) == schedule_small(j0, lr, j)
            cents.append(c)
        assert max(cents) - c0 == nx
        # the centres advance by at most one coarse node from node to node
        assert all(b - a in (0, 1) for a, b in zip(cents, cents[1:]))
        assert -2 <= c0 - 2 and max(cents) + 2 <= n + 2


@pytest.mark.parametrize("lr", [4, 5, 6, 10])
@pytest.mark.parametrize("n", [5, 7, 12])
def test_one_window_for_large_ratios(lr, n):
    r = 1 << lr
    nf = n * r
    for j0 in range(0, nf - 7, 8):
        c0, s0 = centre_offset(j0, r)
        m0 = j0 & (r - 1)
        assert c0 == ((j0 >> lr) if 2 * m0 < r else (j0 >> lr) + 1)
        assert s0 == Fraction(m0 if 2 * m0 < r else m0 - r, r)
        for j in range(8):
            c, s = centre_offset(j0 + j, r)
            assert c == c0 and s == s0 + Fraction(j, r)
        assert -2 <= c0 - 2 and c0 + 2 <= n + 2


def test_ragged_chunks_only_for_small_ratios():
    # N_f = N_r 2^{N_L} is a multiple of 8 once N_L >= 3, so only r <= 4 can leave a last,
    # ragged chunk (the kernels' per-node path)
    for nr in range(5, 40):
        for nl in range(0, 8):
            nf = nr << nl
            if nf % 8:
                assert nl <= 2 and all((1 << lr) <= 4 for lr in range(0, nl + 1))


@pytest.mark.parametrize("run", [1, 2])
@pytest.mark.parametrize("nitems,nblocks", [(1, 760), (759, 760), (1520, 760), (1521, 760), (51101, 760),
                                            (7, 3), (100, 912)])
def test_work_item_runs_visit_every_item_once(nitems, nblocks, run):
    # the two-line stage kernel's traversal: block b takes runs of RUN consecutive items, run
    # c = b, b + nblocks, ...; the host takes RUN = 2 only with at least two items per block
    if run == 2 and nitems < 2 * nblocks:
        pytest.skip("the host launches single items here")
    begin = 3  # a launch covers items [begin, begin + nitems)

    def next_item(i):
        return i + 1 if (i - begin + 1) % run else i + 1 + (nblocks - 1) * run

    seen = []
    for b in range(nblocks):
        it = begin + b * run
        while it < begin + nitems:
            seen.append(it)
            it = next_item(it)
    assert sorted(seen) == list(range(begin, begin + nitems))
