"""fvlbm_mass_noalloc: the total mass computed with no allocation by the call.

Callers that may not allocate while they run (device memory reserved up front
by another allocator, real-time loops, plugins kept off the device heap) use
this entry point instead of fvlbm_mass.  It must give the same numbers, call
after call, even though its scratch is a fixed array shared by every call.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1812_00390_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1812_00390_gb300 import fvlbm
    return fvlbm


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_noalloc_mass_matches_mass_twice(fv, prec):
    parts = [fv.Mesh(mg.cavity(40, 8.0)), fv.Mesh(mg.couette(16, 6)),
             fv.Mesh(mg.cylinder_hybrid(n_rad=20, n_circ=60, first=0.01, growth=1.1, r_far=10.0,
                                        n_tri_rings=30))]
    mesh = fv.Mesh.concat(parts)
    params = [fv.make_params(0.05, scheme="rk2", precision=prec),
              fv.make_params(0.24, scheme="rk2", precision=prec),
              fv.make_params(0.01, scheme="rk2", precision=prec, u0=(0.05, 0.0))]
    s = fv.Solver(mesh, params)
    for call in range(2):            # two calls in a row, the state moving in between
        s.step(7)
        ref = s.mass()
        got = s.mass_noalloc()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        assert got.shape == (3,)
    s.close()


def test_noalloc_mass_rejects_oversized_solver(fv):
    one = fv.Mesh(mg.two_triangles())
    mesh = fv.Mesh.concat([one] * 4097)
    s = fv.Solver(mesh, fv.make_params(0.2, scheme="euler"))
    with pytest.raises(fv.FvlbmError) as e:
        s.mass_noalloc()
    assert e.value.name == "ARG" and "4096" in str(e.value)
    assert s.mass().shape == (4097,)
