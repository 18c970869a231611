"""Unbiased rounding of the 16-bit split storage, through the C ABI.

Every cell is given the same non-equilibrium value v in direction 3 (with
n_1 = v, n_0 = -2 v, so that it carries no mass or momentum), v lying between
two neighbouring values of the 16-bit grid; the cells differ in density,
velocity and a small zero-moment perturbation of directions 5 and 7, so that
each draws its own random number.  After storing (set_f) and reading back
(get_f), the stored non-equilibrium value of direction 3 must be one of the two
grid neighbours of v, and the upper one must come up in the fraction of the
gap that v covers: the mean is v (unbiased).  Round to nearest would store the
same neighbour in every cell.
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


def feq_rows(orc, rho, u):
    return np.array([orc.feq(r, ux, uy) for r, (ux, uy) in zip(rho, u)])


@pytest.mark.parametrize("prec,mant_bits", [("fp16", 10), ("bf16", 7)])
def test_split_storage_rounds_without_bias(fv, orc, prec, mant_bits):
    m = mg.periodic_tri(100, 60, lx=100.0, ly=60.0)
    n = m.n_cell
    rng = np.random.default_rng(7)
    rho = 1.0 + 0.01 * rng.standard_normal(n)
    u = 0.02 * rng.standard_normal((n, 2))
    # v = 2^-6 (1 + 0.3 * 2^-7): 0.3 of a BF16 step above 2^-6, and 0.4 of an
    # FP16 step above its lower FP16 neighbour (the FP16 scale is a power of two)
    v = 2.0 ** -6 * (1.0 + 0.3 * 2.0 ** -7)
    eps = 1e-4 * rng.standard_normal(n)
    f = feq_rows(orc, rho, u)
    f[:, 3] += v
    f[:, 1] += v
    f[:, 0] -= 2 * v
    f[:, 5] += eps
    f[:, 7] += eps
    f[:, 0] -= 2 * eps
    s = fv.Solver(fv.Mesh(m), fv.make_params(0.1, scheme="rk2", precision=prec, u_max=0.1))
    s.set_f(f)
    g = s.get_f()
    stored = g[:, 3] - feq_rows(orc, rho, u)[:, 3]
    # the stored value is one of the two grid neighbours of v (up to the FP32
    # rounding of the moments and of f^eq, far below a grid step)
    step = 2.0 ** -6 * 2.0 ** -mant_bits
    lo = 2.0 ** -6 + np.floor((v - 2.0 ** -6) / step) * step
    hi = lo + step
    near_lo = np.abs(stored - lo) < 1e-3 * step
    near_hi = np.abs(stored - hi) < 1e-3 * step
    assert np.all(near_lo | near_hi), (prec, stored[~(near_lo | near_hi)][:5])
    frac_expected = (v - lo) / step
    frac = near_hi.mean()
    # binomial spread over n cells: sqrt(p (1 - p) / n) ~ 0.006 here
    assert abs(frac - frac_expected) < 0.03, (prec, frac, frac_expected)
    assert abs(stored.mean() - v) < 0.03 * step
