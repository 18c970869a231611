"""Domain decomposition plan (host only, no GPU): recursive coordinate
bisection, the two ghost rings of each part, and the halo messages.

The ghost rings are checked against an adjacency built here from the mesh's
own connectivity (cells sharing an edge), independently of the library's face
matching; the multi-rank test carries the halo messages between processes
over gloo and checks that every ghost ends up with its owner's values.
"""
import math
import os
import socket

import numpy as np
import pytest

from paper_1812_00390_gb300 import meshgen as mg


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1812_00390_gb300 import fvlbm
    return fvlbm


MESHES = {
    "cavity": lambda: mg.cavity(24, 8.0),
    "cavity_tri": lambda: mg.cavity(14, 4.0, triangles=True),
    "cylinder": lambda: mg.cylinder_hybrid(n_rad=8, n_circ=32, first=0.02, growth=1.15, r_far=8.0,
                                           n_tri_rings=8, seed=4),
    "bricks": lambda: mg.bricks(10, 8),
    "couette": lambda: mg.couette(),              # periodic in x
    "periodic_quad": lambda: mg.periodic_quad(10, 8, lx=10.0, ly=8.0),
}
NONPERIODIC = ["cavity", "cavity_tri", "cylinder", "bricks"]


def adjacency(m):
    """Face neighbours of every cell: cells sharing an edge (no periodic pairs)."""
    edges = {}
    for c in range(m.n_cell):
        v = m.cell_vert[m.cell_ptr[c]:m.cell_ptr[c + 1]]
        for k in range(len(v)):
            e = tuple(sorted((int(v[k]), int(v[(k + 1) % len(v)]))))
            edges.setdefault(e, []).append(c)
    nb = [set() for _ in range(m.n_cell)]
    for cs in edges.values():
        if len(cs) == 2:
            nb[cs[0]].add(cs[1])
            nb[cs[1]].add(cs[0])
    return nb


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("n_parts", [1, 2, 3, 4, 7])
def test_every_cell_owned_once_and_balanced(fv, name, n_parts):
    m = MESHES[name]()
    P = fv.Partition(fv.Mesh(m), n_parts)
    owned = [P.cells(p)[:P.info(p)["n_owned"]] for p in range(n_parts)]
    allc = np.concatenate(owned)
    assert np.array_equal(np.sort(allc), np.arange(m.n_cell))
    for o in owned:
        assert np.all(np.diff(o) > 0)                   # ascending, no repeats
    sizes = [len(o) for o in owned]
    # each bisection level puts floor(n * left / parts) on the left: parts differ
    # from the ideal share by less than one cell per level
    levels = max(1, math.ceil(math.log2(n_parts))) if n_parts > 1 else 0
    assert max(sizes) - min(sizes) <= max(1, levels)
    if n_parts == 1:
        i = P.info(0)
        assert i["n_ring1"] == i["n_ring2"] == i["n_send"] == 0


@pytest.mark.parametrize("name", NONPERIODIC)
@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_ghost_rings_match_adjacency(fv, name, n_parts):
    m = MESHES[name]()
    nb = adjacency(m)
    P = fv.Partition(fv.Mesh(m), n_parts)
    for p in range(n_parts):
        i = P.info(p)
        cells = P.cells(p)
        own = set(cells[:i["n_owned"]].tolist())
        r1 = set(cells[i["n_owned"]:i["n_owned"] + i["n_ring1"]].tolist())
        r2 = set(cells[i["n_owned"] + i["n_ring1"]:].tolist())
        want1 = set().union(*[nb[c] for c in own]) - own
        want2 = set().union(*[nb[c] for c in want1]) - own - want1 if want1 else set()
        assert r1 == want1 and r2 == want2, (p, len(r1), len(want1), len(r2), len(want2))
        assert i["n_recv"] == len(r1) + len(r2)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("n_parts", [2, 4, 7])
def test_halo_plan_covers_every_ghost_once(fv, name, n_parts):
    m = MESHES[name]()
    P = fv.Partition(fv.Mesh(m), n_parts)
    cells = [P.cells(p) for p in range(n_parts)]
    info = [P.info(p) for p in range(n_parts)]
    owner = np.full(m.n_cell, -1)
    for p in range(n_parts):
        owner[cells[p][:info[p]["n_owned"]]] = p
    filled = [np.zeros(len(c), int) for c in cells]
    sent = np.zeros(n_parts, int)
    for src in range(n_parts):
        for dst in range(n_parts):
            a, b = P.halo(src, dst)
            if src == dst:
                assert len(a) == 0
                continue
            assert np.all(a < info[src]["n_owned"])            # the sender owns what it sends
            assert np.all(b >= info[dst]["n_owned"])           # into the receiver's ghosts
            assert np.array_equal(cells[src][a], cells[dst][b])
            assert np.all(owner[cells[dst][b]] == src)
            np.add.at(filled[dst], b, 1)
            sent[src] += len(a)
    for p in range(n_parts):
        n_own = info[p]["n_owned"]
        assert np.all(filled[p][:n_own] == 0) and np.all(filled[p][n_own:] == 1)
        assert sent[p] == info[p]["n_send"]


def test_rejects_bad_arguments(fv):
    h = fv.Mesh(mg.two_triangles())
    with pytest.raises(fv.FvlbmError):
        fv.Partition(h, 0)
    with pytest.raises(fv.FvlbmError):
        fv.Partition(h, 3)                                     # more parts than cells
    cat = fv.Mesh.concat([h, h])
    with pytest.raises(fv.FvlbmError) as e:
        fv.Partition(cat, 2)                                   # one instance only
    assert "instances" in str(e.value)


# ----------------------------------------------------------------------------- multi-rank (gloo)
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, out):
    """One rank holding one part: owned rows start as the global values, ghost
    rows as NaN; the plan's messages travel over gloo point-to-point; then every
    local row must equal the global row of its cell.  The FP64 sum of the owned
    rows is all-reduced over the ranks."""
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1812_00390_gb300 import fvlbm as fv
    m = MESHES[name]()
    P = fv.Partition(fv.Mesh(m), world)
    G = np.random.default_rng(5).integers(0, 1 << 20, size=(m.n_cell, 9)).astype(np.float64)
    cells = P.cells(rank)
    n_own = P.info(rank)["n_owned"]
    local = np.full((len(cells), 9), np.nan)
    local[:n_own] = G[cells[:n_own]]
    reqs, bufs = [], []
    for dst in range(world):
        a, _ = P.halo(rank, dst)
        if len(a):
            buf = torch.from_numpy(np.ascontiguousarray(local[a]))
            bufs.append(buf)
            reqs.append(dist.isend(buf, dst))
    for src in range(world):
        _, b = P.halo(src, rank)
        if len(b):
            buf = torch.empty((len(b), 9), dtype=torch.float64)
            dist.recv(buf, src)
            local[b] = buf.numpy()
    for r in reqs:
        r.wait()
    ok = bool(np.array_equal(local, G[cells]))
    s = torch.tensor([local[:n_own].sum()], dtype=torch.float64)
    dist.all_reduce(s)
    out.put((rank, ok, float(s.item()), float(G.sum())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,name", [(2, "cylinder"), (3, "couette")])
def test_halo_exchange_over_gloo(world, name):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, total, want in res:
        assert ok, rank
        assert total == want          # integer-valued rows: the FP64 sums are exact
