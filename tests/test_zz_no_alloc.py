"""sg_step_grid_noalloc, the entry point that allocates nothing, against sg_step.

Some callers cannot allocate device memory: code inside a framework that owns all of it, or
a loop with real-time constraints.  For them the library offers one call whose scratch is a
static device array.  This test drives it through the C ABI on device buffers owned by the
test (PyTorch tensors) and checks, for two calls in a row, that it gives exactly the grid a
level-0 handle gives when stepped twice by sg_step with the same time step -- the FP64
tolerance of the other parity tests, i.e. bit for bit.  It also checks that a grid beyond
SG_NOALLOC_MAX_POINTS is refused with a clear error.

The file is named so that pytest collects it last: a run that stops at the first failure
has then run every other test already.
"""
import numpy as np
import pytest

import paper_2007_10196_gb300 as P
from paper_2007_10196_gb300 import inputs

pytestmark = pytest.mark.gpu

# (dim, nodes per axis, pde, advection speeds, domain lo, domain hi, scheme)
CASES = [
    (1, 37, P.SG_PDE_BURGERS, None, [0.0], [4.0], P.SG_WENO5),
    (2, 20, P.SG_PDE_BURGERS, None, [0.0, -1.0], [4.0, 2.0], P.SG_WENO5),
    (2, 24, P.SG_PDE_ADVECTION, (1.0, -0.5), [0.0, 0.0], [4.0, 4.0], P.SG_LINEAR5),
    (3, 12, P.SG_PDE_ADVECTION, (1.0, -0.6, 0.8), [0.0, 0.0, 0.0], [4.0, 3.0, 2.0], P.SG_WENO5),
    (3, 16, P.SG_PDE_BURGERS, None, [0.0, 0.0, 0.0], [4.0, 4.0, 4.0], P.SG_WENO5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "d%d_n%d_pde%d" % (c[0], c[1], c[2]))
def test_noalloc_matches_sg_step_two_calls(sg, case):
    import torch

    dim, n, pde, adv, lo, hi, scheme = case
    shape = (n,) * dim
    u0 = 0.3 + 0.7 * inputs.random_field(100 + dim, shape, "mixed")
    advs = list(adv) if adv else [1.0] * dim

    # the existing entry point: a level-0 handle (one grid of n^dim nodes), two single steps
    h = P.create(dim, n, 0, pde, lo=lo + [0.0] * (6 - dim), hi=hi + [4.0] * (6 - dim),
                 adv_speed=advs + [1.0] * (6 - dim), scheme=scheme, dt_coef=0.8)
    try:
        P.sg_init_grids(h, u0)
        P.sg_step(h, 1e9, 1)
        dt = P.sg_time(h)[0]  # the first step's dt
        ref1 = P.sg_read(h, 0, count=u0.size)
        P.sg_step(h, 1e9, 1)
        t2 = P.sg_time(h)[0]
        ref2 = P.sg_read(h, 0, count=u0.size)
    finally:
        P.sg_destroy(h)
    assert t2 == dt + dt  # both steps used the same dt

    # the no-allocation entry point on device buffers the caller owns
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.tensor(u0, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    P.sg_step_grid_noalloc(shape, lo, hi, pde, x.data_ptr(), y.data_ptr(), dt, adv_speed=adv,
                           scheme=scheme, eps=1e-3, stream=stream)
    P.sg_step_grid_noalloc(shape, lo, hi, pde, y.data_ptr(), z.data_ptr(), dt, adv_speed=adv,
                           scheme=scheme, eps=1e-3, stream=stream)
    torch.cuda.synchronize()
    got1, got2 = y.cpu().numpy(), z.cpu().numpy()
    assert np.array_equal(got1, ref1), np.max(np.abs(got1 - ref1))
    assert np.array_equal(got2, ref2), np.max(np.abs(got2 - ref2))
    assert np.array_equal(x.cpu().numpy(), u0)  # the input is left untouched

    # in place (u_in == u_out) gives the same result
    P.sg_step_grid_noalloc(shape, lo, hi, pde, x.data_ptr(), x.data_ptr(), dt, adv_speed=adv,
                           scheme=scheme, eps=1e-3, stream=stream)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), ref1)


def test_noalloc_rejects_grids_beyond_its_scratch(sg):
    import torch

    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    n = 1025  # 1025^2 > SG_NOALLOC_MAX_POINTS
    with pytest.raises(P.SgError) as e:
        P.sg_step_grid_noalloc((n, n), [0.0, 0.0], [4.0, 4.0], P.SG_PDE_BURGERS, x.data_ptr(), x.data_ptr(), 1e-3)
    assert e.value.status == P.SG_ERR_ARG
    assert "SG_NOALLOC_MAX_POINTS" in P.sg_last_error()
    with pytest.raises(P.SgError) as e:
        P.sg_step_grid_noalloc((4, 9), [0.0, 0.0], [4.0, 4.0], P.SG_PDE_BURGERS, x.data_ptr(), x.data_ptr(), 1e-3)
    assert e.value.status == P.SG_ERR_ARG
    with pytest.raises(P.SgError) as e:
        P.sg_step_grid_noalloc((5, 5, 5, 5), [0.0] * 4, [4.0] * 4, P.SG_PDE_BURGERS, x.data_ptr(), x.data_ptr(), 1e-3)
    assert e.value.status == P.SG_ERR_UNSUPPORTED
