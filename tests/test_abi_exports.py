"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every function
include/sgweno.h declares; the Python binding wraps each of them.  No GPU compute here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sg_[a-z0-9_]+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    import paper_2007_10196_gb300.build as b
    return b.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sg_create", "sg_init", "sg_step", "sg_prolong_combine", "sg_read", "sg_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, missing
    lib = ctypes.CDLL(built)
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_wraps_every_symbol(built):
    import paper_2007_10196_gb300 as P
    assert set(P.EXPORTED) == _declared()
    L = P.lib()
    for n in P.EXPORTED:
        assert getattr(L, n).argtypes is not None or n == "sg_last_error"


def test_params_struct_layout_and_defaults(built):
    import paper_2007_10196_gb300 as P
    p = P.sg_params_init()
    assert p.struct_size == ctypes.sizeof(P.sg_params)
    assert p.eps == 1e-3 and p.precision == P.SG_F64 and p.cfl == 0.4
    assert list(p.hi) == [4.0] * 6
    assert p.tile_points == 0 and p.stage_kernel == P.SG_STAGE_AUTO and p.combine_budget_gb == 0.0
    assert p.theta == 1.0 and p.tau == 1.0


def test_argument_errors_without_gpu(built):
    """Argument validation happens before any CUDA call."""
    import paper_2007_10196_gb300 as P
    with pytest.raises(P.SgError) as e:
        P.sg_create(7, 10, 3, P.SG_PDE_ADVECTION)
    assert e.value.status == P.SG_ERR_ARG
    with pytest.raises(P.SgError) as e:
        P.sg_create(2, 4, 3, P.SG_PDE_ADVECTION)
    assert e.value.status == P.SG_ERR_ARG
    with pytest.raises(P.SgError) as e:
        P.sg_create(2, 10, 3, P.SG_PDE_ADVECTION, P.sg_params_init(bc=[2] * 6))
    assert e.value.status == P.SG_ERR_ARG and "bc" in P.sg_last_error()
    with pytest.raises(P.SgError) as e:
        P.sg_create(2, 10, 3, P.SG_PDE_ADVECTION, P.sg_params_init(eps=0.0))
    assert e.value.status == P.SG_ERR_ARG
    assert "eps" in P.sg_last_error()
    with pytest.raises(P.SgError) as e:  # the sweep kernel exists for d = 3 only
        P.sg_create(2, 10, 3, P.SG_PDE_ADVECTION, P.sg_params_init(stage_kernel=P.SG_STAGE_SWEEP))
    assert e.value.status == P.SG_ERR_UNSUPPORTED
    with pytest.raises(P.SgError) as e:
        P.sg_create(3, 10, 3, P.SG_PDE_ADVECTION, P.sg_params_init(stage_kernel=4))
    assert e.value.status == P.SG_ERR_ARG
    with pytest.raises(P.SgError) as e:
        P.sg_create(3, 10, 3, P.SG_PDE_ADVECTION, P.sg_params_init(tile_points=300))
    assert e.value.status == P.SG_ERR_ARG
    with pytest.raises(P.SgError) as e:  # 1300^3 > 2^31 points in one grid (32-bit offsets)
        P.sg_create(3, 1300, 0, P.SG_PDE_ADVECTION)
    assert e.value.status == P.SG_ERR_UNSUPPORTED and "2^31" in P.sg_last_error()
    with pytest.raises(P.SgError) as e:  # six axes of 2^20 nodes: the count must not overflow
        P.sg_create(6, 1 << 20, 0, P.SG_PDE_ADVECTION)
    assert e.value.status == P.SG_ERR_UNSUPPORTED
    with pytest.raises(P.SgError) as e:  # the Vlasov-Boltzmann model has d space and d velocity axes
        P.sg_create(3, 10, 1, P.SG_PDE_VLASOV_BOLTZMANN)
    assert e.value.status == P.SG_ERR_ARG
    assert P.lib().sg_destroy(None) == 0


def test_workload_inputs_are_seeded():
    from paper_2007_10196_gb300 import inputs
    a = inputs.burgers3d_batch()
    b = inputs.burgers3d_batch()
    assert [(m.nr, m.nl, m.a) for m in a] == [(m.nr, m.nl, m.a) for m in b]
    assert len(a) == 256 and {m.nr for m in a} == {8, 12, 16} and {m.nl for m in a} == {3, 4, 5}
    assert all(0.5 <= m.a <= 1.0 for m in a)
    f1 = inputs.random_field(3, (5, 7), "mixed")
    f2 = inputs.random_field(3, (5, 7), "mixed")
    assert (f1 == f2).all() and f1.shape == (35,)


def test_noalloc_rejects_partly_overlapping_buffers_without_gpu(built):
    """The no-allocation step takes u_in and u_out as one array or two disjoint ones; a partial
    overlap is refused before any CUDA call (addresses are only compared, never touched)."""
    import paper_2007_10196_gb300 as P
    base = 1 << 20
    with pytest.raises(P.SgError) as e:
        P.sg_step_grid_noalloc((8, 8), 0.0, 1.0, P.SG_PDE_ADVECTION, base, base + 8 * 10, 1e-3)
    assert e.value.status == P.SG_ERR_ARG and "overlap" in P.sg_last_error()
    with pytest.raises(P.SgError) as e:
        P.sg_step_grid_noalloc((8, 8), 0.0, 1.0, P.SG_PDE_ADVECTION, base + 8 * 63, base, 1e-3)
    assert e.value.status == P.SG_ERR_ARG and "overlap" in P.sg_last_error()
