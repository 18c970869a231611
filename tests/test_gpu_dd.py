"""Partitioned solve (domain decomposition) on one GPU, through the C ABI.

Every cell's arithmetic in a part is the same as in the undivided solve (the
same slots, coefficients and upwind writers; ghosts refreshed after every
stage), so the partitioned state must be bitwise equal to the undivided one
for every stage kernel, precision and scheme.  FP64 also matches the oracle to
1e-12, and the mass and residual summed over the parts match the oracle's.
"""
import numpy as np
import pytest

from paper_1812_00390_gb300 import meshgen as mg
from paper_1812_00390_gb300.meshgen import BC, BC_INLET, BC_OUTLET, BC_WALL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1812_00390_gb300 import fvlbm
    return fvlbm


def poiseuille_channel():
    m = mg.channel(nx=20, ny=6, lx=2.0, ly=0.6, u_inf=(0.05, 0.0), top_bottom="inlet", external=0)
    ym = m.xy[m.bedge, 1].mean(1)
    bt = m.btag.copy()
    bt[(np.abs(ym) < 1e-12) | (np.abs(ym - 0.6) < 1e-12)] = 2
    m.btag = bt
    m.bcs = [BC(BC_INLET, external=0, u_inf=(0.05, 0.0)), BC(BC_OUTLET, external=0, rho_inf=1.0), BC(BC_WALL)]
    return m


MESHES = {
    "cavity": lambda: mg.cavity(40, 8.0),
    "couette": lambda: mg.couette(),
    "periodic_tri": lambda: mg.periodic_tri(16, 12, lx=16.0, ly=12.0),
    "cylinder": lambda: mg.cylinder_hybrid(n_rad=12, n_circ=48, first=0.02, growth=1.12, r_far=8.0,
                                           n_tri_rings=12, seed=4),
    "bricks": lambda: mg.bricks(12, 10),
    "internal_io": poiseuille_channel,
    "symmetry": lambda: mg.channel(nx=14, ny=6, top_bottom="symmetry"),
}


def f_random(orc, m, seed, noise=0.02):
    rho, u, dev = mg.random_state(m.n_cell, seed=seed)
    return np.array([orc.feq(r, *v) for r, v in zip(rho, u)]) + noise * dev


def pair(fv, m, n_parts, **kw):
    h = fv.Mesh(m)
    p = fv.make_params(**kw)
    plan = fv.Partition(h, n_parts)
    return fv.Solver(h, p), fv.DDSolver(plan, p), plan


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("n_parts", [2, 4])
@pytest.mark.parametrize("prec,kernel", [("fp64", 1), ("fp64", 128), ("fp32", 1), ("fp32", 128), ("fp32", 256),
                                         ("fp16", 128), ("bf16", 1)])
def test_partitioned_equals_undivided_bitwise(fv, orc, name, n_parts, prec, kernel):
    m = MESHES[name]()
    if kernel == 256 and prec == "fp64":
        pytest.skip("not a combination under test")
    one, dd, plan = pair(fv, m, n_parts, tau=0.1, scheme="rk2", precision=prec, kernel=kernel, u0=(0.02, 0.01))
    assert dd.stage_kernel()[0] == one.stage_kernel() == kernel
    f0 = f_random(orc, m, seed=3)
    one.set_f(f0)
    dd.set_f(f0)
    assert np.array_equal(dd.get_f(), one.get_f())
    for n in (1, 33, 6):
        one.step(n)
        dd.step(n)
    assert np.array_equal(dd.get_f(), one.get_f())
    r1, u1 = one.macros()
    r2, u2 = dd.macros()
    assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
    dd.close()


@pytest.mark.parametrize("scheme", ["euler", "ab2", "rk4"])
@pytest.mark.parametrize("kernel", [1, 128])
@pytest.mark.parametrize("name", ["cylinder", "bricks", "couette"])
def test_partitioned_every_scheme(fv, orc, name, scheme, kernel):
    """Single-stage schemes (alternating state on the fused stage, AB2 history)
    and the 4-stage scheme (three stage buffers on the fused stage)."""
    m = MESHES[name]()
    one, dd, _ = pair(fv, m, 3, tau=0.1, scheme=scheme, precision="fp32", kernel=kernel, u0=(0.02, 0.0))
    f0 = f_random(orc, m, seed=9)
    one.set_f(f0)
    dd.set_f(f0)
    for n in (1, 33, 2):
        one.step(n)
        dd.step(n)
    assert np.array_equal(dd.get_f(), one.get_f())
    dd.close()


@pytest.mark.parametrize("name", ["cavity", "cylinder", "internal_io", "periodic_tri"])
@pytest.mark.parametrize("n_parts", [2, 3, 4])
def test_partitioned_fp64_matches_oracle(fv, orc, name, n_parts):
    m = MESHES[name]()
    tau = 0.1
    o = orc.Oracle(m)
    dt = o.cfl_dt(0.5, 0.1, tau, "rk2")
    plan = fv.Partition(fv.Mesh(m), n_parts)
    dd = fv.DDSolver(plan, fv.make_params(tau, dt=dt, scheme="rk2", precision="fp64", u0=(0.02, 0.01)))
    f0 = f_random(orc, m, seed=11)
    dd.set_f(f0)
    o.set_f(f0)
    dd.residual()                          # snapshot at f0
    _, u_old = o.macros()
    dd.step(30)
    o.run("rk2", tau, dt, 30)
    ref = o.get_f()
    assert np.abs(dd.get_f() - ref).max() / np.abs(ref).max() < 1e-12
    assert abs(dd.mass() - o.mass()) <= 1e-13 * o.mass()
    e_o = o.residual(u_old)
    assert abs(dd.residual() - e_o) <= 1e-12 * e_o
    dd.close()


def test_partitioned_launch_count_and_one_part(fv):
    m = MESHES["cavity"]()
    one, dd, _ = pair(fv, m, 1, tau=0.1, scheme="rk2", precision="fp32", kernel=128)
    k, launches = dd.stage_kernel()
    assert k == 128 and launches == one.launches_per_step()     # one part: no exchange
    one.step(10)
    dd.step(10)
    assert np.array_equal(dd.get_f(), one.get_f())
    _, dd4, _ = pair(fv, m, 4, tau=0.1, scheme="rk2", precision="fp32", kernel=128)
    assert dd4.stage_kernel()[1] == 4 * one.launches_per_step() + 2   # + one exchange per stage
