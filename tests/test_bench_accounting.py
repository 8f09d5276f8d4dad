"""The benchmark's work accounting against the oracle (host logic, no GPU).

The bench line's `value` is point-updates per second: the points of every member's grids
(Section 2.2, Eq. 13's grid set) times the steps each took.  `bench._batch_points` enumerates the
grids itself; here its grid counts and point totals are checked against the oracle's grid set
and state sizes for every member shape of the benchmark batch (and two small ones), and the
finest-point count of the combination model against N_f^3.
"""
import pytest

import bench
import oracle as orc
from paper_2007_10196_gb300.inputs import BatchMember, burgers3d_batch

SHAPES = sorted({(m.nr, m.nl) for m in burgers3d_batch(256, seed=2007)} | {(5, 0), (6, 2)})


@pytest.mark.parametrize("nr,nl", SHAPES)
def test_batch_points_match_oracle_grid_set(nr, nl):
    m = BatchMember(nr=nr, nl=nl, a=0.6)
    (grids, points), = bench._batch_points([m])
    lev, co = orc.grid_set(3, nl)
    p = orc.problem(3, nr, nl, pde=orc.BURGERS)
    assert grids == len(lev)
    assert points == sum(orc.state_points(p, lv) for lv in lev)
    fine, _ = bench.combine_work([m])
    assert fine == (nr << nl) ** 3
