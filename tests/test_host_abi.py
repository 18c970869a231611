"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/fvlbm.h declares, and its FP64 mesh precompute agrees
with the oracle's independent one (face counts, CFL length, time step)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1812_00390_gb300 import meshgen as mg
from paper_1812_00390_gb300.meshgen import BC, BC_PERIODIC, BC_WALL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1812_00390_gb300 import fvlbm
    return fvlbm


def _declared():
    src = open(os.path.join(ROOT, "include", "fvlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fvlbm_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(fv):
    names = _declared()
    assert len(names) >= 17
    lib = C.CDLL(fv.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fv.EXPORTS) == names


@pytest.mark.parametrize("make", [
    lambda: mg.couette(), lambda: mg.cavity(12, 5.0), lambda: mg.periodic_tri(9, 7),
    lambda: mg.channel(top_bottom="symmetry"), lambda: mg.bricks(),
    lambda: mg.cylinder_hybrid(n_rad=5, n_circ=16, first=0.05, growth=1.2, r_far=5.0, n_tri_rings=4),
    lambda: mg.two_triangles(periodic=True)])
def test_mesh_counts_and_dt_match_oracle(fv, orc, make):
    m = make()
    h = fv.Mesh(m)
    info = h.info()
    o = orc.Oracle(m)
    a, _, l = o.geometry()
    assert info["n_cell"] == m.n_cell
    # every (cell, edge) is one slot: interior/periodic faces are seen twice
    n_slots = o.n_faces()
    assert 2 * (info["n_face"] - info["n_bface"]) + info["n_bface"] == n_slots
    assert abs(info["total_area"] - a.sum()) < 1e-12 * a.sum()
    assert abs(info["min_cfl_length"] - np.min(a / l.sum(1))) < 1e-15
    for scheme in ("euler", "rk2", "ab2", "rk4"):
        for tau in (1e-3, 0.3):
            assert h.suggest_dt(tau, 0.5, 0.1, scheme) == pytest.approx(o.cfl_dt(0.5, 0.1, tau, scheme), rel=1e-15)


def test_concat_instances(fv):
    a, b = fv.Mesh(mg.couette(8, 4)), fv.Mesh(mg.cavity(6, 3.0))
    c = fv.Mesh.concat([a, b, a])
    info = c.info()
    assert info["n_instances"] == 3
    assert info["n_cell"] == 2 * 64 + 36
    assert c.suggest_dt(0.3, instance=1) == pytest.approx(b.suggest_dt(0.3))


def test_mesh_errors(fv):
    m = mg.couette(4, 2)
    with pytest.raises(fv.FvlbmError) as e:
        fv.Mesh(mg.Mesh(m.xy, m.cell_ptr, m.cell_vert, m.bedge[:-1], m.btag[:-1], m.bcs))
    assert e.value.name == "UNTAGGED_BOUNDARY"
    with pytest.raises(fv.FvlbmError) as e:
        fv.Mesh(mg.Mesh(m.xy, m.cell_ptr, m.cell_vert[::-1].copy(), m.bedge, m.btag, m.bcs))
    assert e.value.name in ("DEGENERATE_CELL", "UNTAGGED_BOUNDARY")
    bad = mg.couette(4, 2)
    bad.bcs[1] = BC(BC_PERIODIC, partner=3, shift=(3.0, 0.0))    # wrong period
    with pytest.raises(fv.FvlbmError) as e:
        fv.Mesh(bad)
    assert e.value.name == "MESH_TOPOLOGY"
    bad.bcs[1] = BC(BC_PERIODIC, partner=0, shift=(4.0, 0.0))    # partner is a wall
    with pytest.raises(fv.FvlbmError) as e:
        fv.Mesh(bad)
    assert e.value.name == "ARG"
    # an edge shared by three cells
    tri = mg.Mesh(np.array([[0, 0], [1, 0], [0, 1], [1, 1], [0.5, -1.0]], float),
                  np.array([0, 3, 6, 9]), np.array([0, 1, 2, 1, 3, 2, 0, 4, 1], np.int32),
                  np.zeros((0, 2), np.int32), np.zeros(0, np.int32), [BC(BC_WALL)])
    with pytest.raises(fv.FvlbmError) as e:
        fv.Mesh(tri)
    assert e.value.name in ("MESH_TOPOLOGY", "UNTAGGED_BOUNDARY")


def test_init_without_gpu_fails_loudly(fv):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = fv.Mesh(mg.couette(4, 2))
    with pytest.raises(fv.FvlbmError) as e:
        fv.Solver(h, fv.make_params(0.24), stream=0, use_torch_workspace=False)
    assert e.value.name == "UNSUPPORTED"


def test_stage_kernel_capacity_on_the_host(fv):
    """The layout and the fused stage's tile plan are built on the host: every
    variant that fits a CTA's shared memory gives a workspace; the tile size
    that would not fit (FP64 1024-thread tiles, quads or hexagons) is refused
    with FVLBM_ERR_UNSUPPORTED."""
    def ws(mesh, prec, kernel):
        arr = (fv.ParamsT * 1)(fv.make_params(0.1, scheme="rk2", precision=prec, kernel=kernel))
        n = C.c_size_t()
        rc = fv.lib.fvlbm_workspace_bytes(mesh._h, arr, 1, C.byref(n))
        return fv.ERRORS.get(rc, rc) if rc else "OK", n.value

    quads, hexes = fv.Mesh(mg.cavity(40, 5.0)), fv.Mesh(mg.bricks(20, 16))   # handles kept alive
    for prec in ("fp32", "fp16", "bf16", "fp64"):
        sizes = {}
        for k in (1, 128, 256, 512):
            rc, n = ws(quads, prec, k)
            assert rc == "OK" and n > 0, (prec, k, rc)
            sizes[k] = n
        # the fused stage keeps no face-value table in memory
        assert sizes[512] < sizes[1]
    assert ws(quads, "fp32", 1024)[0] == "OK"
    assert ws(quads, "fp64", 1024)[0] == "UNSUPPORTED"
    assert ws(hexes, "fp64", 512)[0] == "OK"
    assert ws(hexes, "fp64", 1024)[0] == "UNSUPPORTED"
    assert ws(hexes, "fp32", 1024)[0] == "OK"
    assert ws(quads, "fp32", 384)[0] == "ARG"


@pytest.mark.parametrize("name,make", [
    ("cavity", lambda: mg.cavity(96, 20.0)),
    ("cylinder", lambda: mg.cylinder_hybrid(n_rad=25, n_circ=50, n_tri_rings=25, seed=3)),
    ("periodic", lambda: mg.periodic_tri(40, 30, lx=40.0, ly=30.0)),
    ("bricks", lambda: mg.bricks(30, 20)),
    ("couette", lambda: mg.couette()),
])
def test_tile_plan_checks(fv, name, make):
    """The fused stage's tile plan, built and checked on the host: local links,
    one face row per face, one writer per (face, direction), tiles within
    their CTA; the bank-aware face rows keep the modelled face-table
    wavefronts well below those of the neighbour gathers."""
    m = make()
    h = fv.Mesh(m)
    for k in (128, 256, 512, 1024):
        for prec in ("fp32", "fp16", "fp64"):
            p = fv.make_params(0.1, scheme="rk2", precision=prec, kernel=k)
            if prec == "fp64" and k == 1024:
                with pytest.raises(fv.FvlbmError):
                    fv.plan_info(h, p)
                continue
            i = fv.plan_info(h, p)
            assert i["violations"] == 0, (name, k, prec, i.get("first_violation"))
            assert i["stage_kernel"] == k and i["n_tiles"] >= 1
            assert i["n_tiles"] * i["mean_tile_cells"] == pytest.approx(m.n_cell)
            assert i["mean_tile_cells"] + i["mean_ring1_cells"] <= k
            assert i["mean_local_cells"] <= i["max_local_cells"] <= 3 * k // 2 + 64
            assert 1.0 <= i["face_table_waves"] < 1.8
            assert 1.0 <= i["gather_waves"] < 2.6
    two = fv.plan_info(h, fv.make_params(0.1, scheme="rk2", precision="fp64", kernel=1))
    assert two["stage_kernel"] == 1 and two["n_tiles"] == 0 and two["violations"] == 0
