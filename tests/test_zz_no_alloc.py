"""ibrd_vcycle_noalloc: the V-cycle for callers that cannot allocate device
memory (no grid handle; workspaces in the library's static device scratch).

Called through the C ABI, it must give what ibrd_vcycle gives on the same
grid, within the 1e-12 the V-cycle parity tests use, on two calls in a row
(the second call runs on the scratch the first one left behind). Grids too
large for the scratch are rejected before any GPU work. This file is named to
be collected last.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import dev, host, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1306_3159_gb300 import build
    lib = ctypes.CDLL(build.build())
    f = lib.ibrd_vcycle_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib


def _noalloc(lib, dims, h, chi, alpha, b, x, zero):
    import torch
    st = lib.ibrd_vcycle_noalloc(dims[0], dims[1], dims[2], h, chi, alpha, ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), int(zero),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("dims,h,chi,alpha,zero", [((64, 64, 64), 1.0, 1.0, 0.0, True),
                                                   ((32, 48, 16), 0.7, 1.3, 0.25, True),
                                                   ((64, 32, 32), 1.0, 1.0, 0.0, False),
                                                   ((16, 16, 16), 1.0, 2.0, 0.0, True),
                                                   ((112, 112, 112), 1.0, 1.0, 0.0, True)])
def test_noalloc_vcycle_matches_vcycle(lib, dims, h, chi, alpha, zero):
    import paper_1306_3159_gb300 as p
    nx, ny, nz = dims
    rng = np.random.default_rng(17)
    b = rng.standard_normal((nz, ny, nx))
    x0 = rng.standard_normal((nz, ny, nx))
    g = p.Grid(*dims, h=h, chi=chi, alpha=alpha)
    ref = dev(x0)
    g.vcycle(dev(b), ref, zero_initial_guess=zero)
    want = host(ref)
    bd = dev(b)
    for _ in range(2):  # two calls in a row on the shared scratch
        x = dev(x0)
        assert _noalloc(lib, dims, h, chi, alpha, bd, x, zero) == 0
        assert rel_max(host(x), want) < 1e-12


@pytest.mark.parametrize("dims", [(128, 128, 128), (120, 120, 120), (128, 128, 96)])
def test_noalloc_rejects_grids_beyond_the_scratch(lib, dims):
    # 112^3 uses about 15.3 MiB of the 16 MiB scratch (its largest case above);
    # these need more: IBRD_ERR_ARG before any GPU work
    st = lib.ibrd_vcycle_noalloc(*dims, 1.0, 1.0, 0.0, None, None, 1, None)
    assert st == 1
