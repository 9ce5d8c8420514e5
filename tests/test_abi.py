"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/ibrd.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ibrd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibrd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_3159_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_paper_boundary():
    names = _declared()
    for want in ["ibrd_grid_create", "ibrd_apply_L", "ibrd_vcycle", "ibrd_spread", "ibrd_interp",
                 "ibrd_solve_reaction", "ibrd_solve_saddle"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_1306_3159_gb300 import EXPORTED
    assert sorted(EXPORTED) == _declared()


def test_default_opts_and_status_strings(lib):
    import paper_1306_3159_gb300 as p
    o = p.ibrd_default_opts()
    assert o.tol == 1e-8 and o.restart == 30 and o.mg_cycles == 1 and o.schur_inner == 5
    assert o.nu1 == 2 and o.nu2 == 2 and o.zeta == 1.0
    lib.ibrd_status_string.restype = ctypes.c_char_p
    assert lib.ibrd_status_string(0) == b"IBRD_OK"
    assert lib.ibrd_status_string(4) == b"IBRD_ERR_NOT_CONVERGED"


def test_create_rejects_bad_arguments_without_touching_gpu(lib):
    # Argument validation happens before any CUDA call.
    import paper_1306_3159_gb300 as p
    for args in [(3, 8, 8, 1.0, 1.0, 0.0), (8, 8, 8, -1.0, 1.0, 0.0), (8, 8, 8, 1.0, 0.0, 0.0),
                 (8, 8, 8, 1.0, 1.0, -0.5), (9, 9, 9, 1.0, 1.0, 0.0)]:
        with pytest.raises(p.IbrdError) as e:
            p.ibrd_grid_create(*args, stream=0)
        assert e.value.status == 1


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1306_3159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_batch_rejects_bad_handles_without_touching_gpu(lib):
    # The batch entry points check count and handles (null, shared) before any
    # handle is dereferenced; the fake addresses below are never followed.
    vp = ctypes.c_void_p
    lib.ibrd_solve_reaction_batch.restype = ctypes.c_int
    ptrs = (vp * 2)(vp(0x1000).value, vp(0x2000).value)
    assert lib.ibrd_solve_reaction_batch(0, None, None, None, None, None, None, 0) == 0
    assert lib.ibrd_solve_reaction_batch(-1, None, None, None, None, None, None, 0) == 1
    for grids in [(vp * 2)(vp(0x1000).value, None), (vp * 2)(vp(0x1000).value, vp(0x1000).value)]:
        assert lib.ibrd_solve_reaction_batch(2, grids, ptrs, ptrs, ptrs, None, None, 4) == 1
        assert lib.ibrd_solve_saddle_batch(2, grids, ptrs, None, ptrs, ptrs, None, None, 4) == 1
    assert lib.ibrd_solve_reaction_batch(2, ptrs, None, ptrs, ptrs, None, None, 0) == 1


def test_solve_many_rejects_bad_items_without_touching_gpu(lib):
    # an unknown kind, a null handle or a shared handle is refused before any
    # handle is dereferenced (the fake addresses are never followed)
    import paper_1306_3159_gb300 as p
    from paper_1306_3159_gb300._abi import SolveItem
    fn = p.load_library().ibrd_solve_many
    assert fn(0, None, 0) == 0 and fn(-1, None, 0) == 1
    for kinds, grids in [((0, 7), (0x1000, 0x2000)), ((0, 1), (0x1000, 0)), ((0, 1), (0x1000, 0x1000))]:
        items = (SolveItem * 2)()
        for k in range(2):
            items[k].kind = kinds[k]
            items[k].grid = grids[k] or None
        assert fn(2, items, 2) == 1


def _ewald_constant(lx, ly, lz, beta_scale, nr, nk):
    """C of G(r) = 1/(4 pi r) + C + ... for the zero-mean periodic Green's
    function of -Laplace: an independent NumPy Ewald sum with its own
    splitting parameter and fixed shells."""
    import numpy as np
    from scipy.special import erfc
    V = lx * ly * lz
    beta = beta_scale / V ** (1 / 3)
    a = np.arange(-nr, nr + 1)
    n = np.stack(np.meshgrid(a * lx, a * ly, a * lz, indexing="ij"), -1).reshape(-1, 3)
    r = np.sqrt((n ** 2).sum(1))
    r = r[r > 0]
    real = np.sum(erfc(beta * r) / (4 * np.pi * r))
    m = np.arange(-nk, nk + 1)
    k = np.stack(np.meshgrid(2 * np.pi * m / lx, 2 * np.pi * m / ly, 2 * np.pi * m / lz, indexing="ij"), -1)
    k2 = (k.reshape(-1, 3) ** 2).sum(1)
    k2 = k2[k2 > 0]
    recip = np.sum(np.exp(-k2 / (4 * beta ** 2)) / k2) / V
    return real + recip - beta / (2 * np.pi ** 1.5) - 1 / (4 * beta ** 2 * V)


def test_periodic_constant(lib):
    """ibrd_periodic_constant (the block preconditioner's model constant and
    the finite-size constant of Sec. IV.A's Eq. a_phi): a cube gives
    -2.837297 / (4 pi L) (the simple cubic lattice constant; the paper prints
    2.84), it scales as 1 / L, and boxes of other shapes agree with an
    independent Ewald sum (another splitting parameter, fixed shells) to
    1e-10; a non-positive side gives NaN."""
    import math
    f = lib.ibrd_periodic_constant
    f.argtypes = [ctypes.c_double] * 3
    f.restype = ctypes.c_double
    for L in (1.0, 64.0, 256.0):
        assert abs(f(L, L, L) * 4 * math.pi * L + 2.837297) < 1e-6
    assert abs(-f(1, 1, 1) * 4 * math.pi - 2.84) < 5e-3
    assert abs(f(3.0, 2.0, 5.0) - 7.0 * f(21.0, 14.0, 35.0)) < 1e-13 * abs(f(3.0, 2.0, 5.0))
    for box in [(2.0, 1.0, 1.0), (1.0, 1.0, 0.5), (64.0, 32.0, 96.0), (40.0, 24.0, 16.0), (128.0, 32.0, 32.0)]:
        want = _ewald_constant(*box, beta_scale=2.2, nr=12, nk=16)
        assert abs(f(*box) - want) < 1e-10 * abs(want), box
    assert math.isnan(f(0.0, 1.0, 1.0)) and math.isnan(f(1.0, -2.0, 1.0))
