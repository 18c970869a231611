// Domain decomposition of one mesh (host only): recursive coordinate
// bisection of the cell centroids into parts, the two ghost rings each part
// needs, and the halo plan that fills them.
//
// A cell's update reads the face values of its faces; the value on a face is
// reconstructed from the gradient of its upwind cell (Eq. lslrflux), which is
// a least-squares fit over that cell's face neighbours (Eq. leastsquare).  So
// a part that updates its own cells needs the state of the cells next to them
// (ring 1: their gradients are recomputed locally) and of the cells next to
// those (ring 2: state only).  After every stage the owners of those cells
// send their new state: one exchange of two rings per stage.  The paper runs
// its solver in Code_Saturne's parallel modules (Sec. 3) and counts one layer
// of ghost cells per partition interface as enough (Conclusions, item 4); with
// one layer the ghosts' gradients would have to be sent as well, a second
// message per stage.  Sending a second ring of state and recomputing the first
// ring's gradients keeps one message per stage.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <numeric>

#include "fvlbm_internal.h"

using namespace fvlbm;

namespace {

// Cells of `ids` (caller numbering) split into `n_parts` parts numbered from
// `first`: cut across the longer extent of their centroids' bounding box, at
// the cell count proportional to the parts on each side (ties broken by cell
// number, so that the result depends only on the mesh).
void rcb(const Mesh& M, std::vector<int64_t>& ids, int32_t first, int32_t n_parts, std::vector<int32_t>& owner) {
    if (n_parts == 1) {
        for (int64_t c : ids) owner[c] = first;
        return;
    }
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int64_t c : ids) {
        x0 = std::min(x0, M.cx[c]); x1 = std::max(x1, M.cx[c]);
        y0 = std::min(y0, M.cy[c]); y1 = std::max(y1, M.cy[c]);
    }
    const bool by_x = x1 - x0 >= y1 - y0;
    const std::vector<double>& key = by_x ? M.cx : M.cy;
    std::sort(ids.begin(), ids.end(), [&](int64_t a, int64_t b) { return key[a] != key[b] ? key[a] < key[b] : a < b; });
    const int32_t nl = n_parts / 2;
    const size_t cut = (size_t)((int64_t)ids.size() * nl / n_parts);
    std::vector<int64_t> lo(ids.begin(), ids.begin() + cut), hi(ids.begin() + cut, ids.end());
    ids.clear();
    ids.shrink_to_fit();
    rcb(M, lo, first, nl, owner);
    rcb(M, hi, first + nl, n_parts - nl, owner);
}

// Interior neighbours (caller numbering) of cell c.
template <typename F>
void for_neighbours(const Mesh& M, int64_t c, F f) {
    for (int k = 0; k < M.nf[c]; k++) {
        const Slot& S = M.slots[(size_t)c * MAXP + k];
        if (S.kind == SK_INTERIOR) f((int64_t)S.nb);
    }
}

// The mesh of one part: its cells in local numbering (owned, ring 1, ring 2),
// geometry copied from the whole mesh, neighbours renumbered; a ring-2 cell's
// faces towards cells outside the part become empty slots (the part never
// computes anything for ring-2 cells but reads their state).  Owned cells keep
// the whole mesh's locality order among themselves; ghosts follow.
int part_mesh(const Mesh& G, const PartPlan& P, const std::vector<int64_t>& local_of_stamp, Mesh& M) {
    const int64_t n = (int64_t)P.cells.size();
    M = Mesh{};
    M.n_cell = n;
    M.n_owned = P.n_owned;
    M.n_grad = P.n_owned + P.n_ring1;
    M.max_faces = G.max_faces;   // same slot count as the whole mesh: the same kernels run
    M.n_inst = 1;
    M.inst_begin = {0, P.n_owned};
    M.inst_bc_begin = {0, (int32_t)G.bcs.size()};
    M.bcs = G.bcs;
    M.inst_cfl_len = G.inst_cfl_len;   // the whole mesh's time step in every part
    M.nf.resize(n);
    M.area.resize(n);
    M.cx.resize(n);
    M.cy.resize(n);
    M.slots.assign((size_t)n * MAXP, Slot());
    for (int64_t l = 0; l < n; l++) {
        const int64_t c = P.cells[l];
        M.nf[l] = G.nf[c];
        M.area[l] = G.area[c];
        M.cx[l] = G.cx[c];
        M.cy[l] = G.cy[c];
        for (int k = 0; k < G.nf[c]; k++) {
            Slot S = G.slots[(size_t)c * MAXP + k];
            if (S.kind == SK_INTERIOR) {
                const int64_t j = local_of_stamp[S.nb];
                if (j >= 0) {
                    S.nb = (int32_t)j;
                } else {   // only ring-2 cells reach outside the part
                    S.kind = SK_NONE;
                    S.nb = -1;
                    S.nb_slot = -1;
                }
            }
            M.slots[(size_t)l * MAXP + k] = S;
        }
    }
    // faces: interior pairs once, every other slot (boundary, or a ring-2
    // slot leading out of the part) once
    for (int64_t l = 0; l < n; l++)
        for (int k = 0; k < M.nf[l]; k++) {
            const Slot& S = M.slots[(size_t)l * MAXP + k];
            if (S.kind != SK_INTERIOR || l < S.nb || (l == S.nb && k < S.nb_slot)) M.n_face++;
            if (l < P.n_owned) {
                if (S.kind > SK_INTERIOR) M.n_bface++;
                if (S.periodic) M.n_periodic++;
            }
        }
    for (int64_t l = 0; l < P.n_owned; l++) M.total_area += M.area[l];
    // internal order: owned cells in the whole mesh's order, then the ghosts
    M.perm.resize(n);
    std::iota(M.perm.begin(), M.perm.end(), 0);
    std::sort(M.perm.begin(), M.perm.begin() + P.n_owned,
              [&](int64_t a, int64_t b) { return G.iperm[P.cells[a]] < G.iperm[P.cells[b]]; });
    M.iperm.resize(n);
    for (int64_t i = 0; i < n; i++) M.iperm[M.perm[i]] = i;
    return FVLBM_OK;
}

int build_partition(const Mesh& G, int32_t n_parts, fvlbm_partition& R) {
    const int64_t N = G.n_cell;
    R.n_parts = n_parts;
    R.n_cell = N;
    R.owner.assign(N, -1);
    {
        std::vector<int64_t> ids(N);
        std::iota(ids.begin(), ids.end(), 0);
        rcb(G, ids, 0, n_parts, R.owner);
    }
    R.parts.resize(n_parts);
    std::vector<std::vector<int64_t>> owned(n_parts);
    for (int64_t c = 0; c < N; c++) owned[R.owner[c]].push_back(c);
    // local index of every cell in the part being built (-1: not in it)
    std::vector<int64_t> local(N, -1);
    std::map<std::pair<int32_t, int32_t>, HaloMsg> msgs;
    for (int32_t p = 0; p < n_parts; p++) {
        PartPlan& P = R.parts[p];
        P.cells = owned[p];
        P.n_owned = (int64_t)P.cells.size();
        for (int64_t l = 0; l < P.n_owned; l++) local[P.cells[l]] = l;
        std::vector<int64_t> r1, r2;
        for (int64_t c : owned[p])
            for_neighbours(G, c, [&](int64_t j) {
                if (local[j] == -1) {
                    local[j] = -2;   // seen
                    r1.push_back(j);
                }
            });
        std::sort(r1.begin(), r1.end());
        for (int64_t j : r1)
            for_neighbours(G, j, [&](int64_t q) {
                if (local[q] == -1) {
                    local[q] = -3;
                    r2.push_back(q);
                }
            });
        std::sort(r2.begin(), r2.end());
        P.n_ring1 = (int64_t)r1.size();
        P.n_ring2 = (int64_t)r2.size();
        P.cells.insert(P.cells.end(), r1.begin(), r1.end());
        P.cells.insert(P.cells.end(), r2.begin(), r2.end());
        for (int64_t l = 0; l < (int64_t)P.cells.size(); l++) local[P.cells[l]] = l;
        fvlbm_mesh* pm = new fvlbm_mesh;
        P.mesh = pm;
        int rc = part_mesh(G, P, local, pm->m);
        if (rc) return rc;
        for (int64_t c : P.cells) local[c] = -1;
    }
    // halo plan: every ghost of part q comes from its owner p
    for (int32_t q = 0; q < n_parts; q++) {
        const PartPlan& P = R.parts[q];
        for (int64_t l = P.n_owned; l < (int64_t)P.cells.size(); l++) {
            const int64_t c = P.cells[l];
            const int32_t p = R.owner[c];
            HaloMsg& m = msgs[{p, q}];
            m.src = p;
            m.dst = q;
            m.src_local.push_back(-1);   // filled below
            m.dst_local.push_back((int32_t)l);
            m.cells.push_back(c);
        }
    }
    // local index of each sent cell in its owner (owned cells of part p are
    // P.cells[0, n_owned) in ascending order)
    for (auto& kv : msgs) {
        HaloMsg& m = kv.second;
        const PartPlan& S = R.parts[m.src];
        for (size_t e = 0; e < m.cells.size(); e++) {
            auto it = std::lower_bound(S.cells.begin(), S.cells.begin() + S.n_owned, m.cells[e]);
            m.src_local[e] = (int32_t)(it - S.cells.begin());
        }
        R.msgs.push_back(std::move(m));
    }
    return FVLBM_OK;
}

}  // namespace

fvlbm_partition::~fvlbm_partition() {
    for (auto& P : parts) delete P.mesh;
}

extern "C" int fvlbm_mesh_partition(const fvlbm_mesh* mesh, int32_t n_parts, fvlbm_partition** out) {
    clear_error();
    if (!mesh || !out) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_partition: null argument");
    *out = nullptr;
    const Mesh& G = mesh->m;
    if (G.n_inst != 1) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_partition: the mesh holds %d instances; one is needed", G.n_inst);
    if (G.n_owned != G.n_cell) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_partition: the mesh is already a part");
    if (n_parts < 1 || n_parts > FVLBM_MAX_PARTS || n_parts > G.n_cell)
        return fail(FVLBM_ERR_ARG, "fvlbm_mesh_partition: n_parts = %d (1..%d and at most the cell count)", n_parts,
                    FVLBM_MAX_PARTS);
    fvlbm_partition* r = new (std::nothrow) fvlbm_partition;
    if (!r) return fail(FVLBM_ERR_OOM, "fvlbm_mesh_partition: out of host memory");
    int rc;
    try {
        rc = build_partition(G, n_parts, *r);
    } catch (const std::bad_alloc&) {
        rc = fail(FVLBM_ERR_OOM, "fvlbm_mesh_partition: out of host memory");
    }
    if (rc) {
        delete r;
        return rc;
    }
    *out = r;
    return FVLBM_OK;
}

extern "C" void fvlbm_partition_destroy(fvlbm_partition* p) { delete p; }

extern "C" int fvlbm_partition_info(const fvlbm_partition* p, int32_t part, fvlbm_part_info_t* info) {
    clear_error();
    if (!p || !info || part < 0 || part >= p->n_parts) return fail(FVLBM_ERR_ARG, "fvlbm_partition_info: bad arguments");
    const PartPlan& P = p->parts[part];
    info->n_owned = P.n_owned;
    info->n_ring1 = P.n_ring1;
    info->n_ring2 = P.n_ring2;
    info->n_recv = P.n_ring1 + P.n_ring2;
    info->n_send = 0;
    info->n_neighbours = 0;
    for (const HaloMsg& m : p->msgs) {
        if (m.src == part) info->n_send += (int64_t)m.src_local.size();
        if (m.dst == part) info->n_neighbours++;
    }
    return FVLBM_OK;
}

extern "C" int fvlbm_partition_cells(const fvlbm_partition* p, int32_t part, int64_t* cells) {
    clear_error();
    if (!p || !cells || part < 0 || part >= p->n_parts) return fail(FVLBM_ERR_ARG, "fvlbm_partition_cells: bad arguments");
    const PartPlan& P = p->parts[part];
    std::copy(P.cells.begin(), P.cells.end(), cells);
    return FVLBM_OK;
}

extern "C" int fvlbm_partition_halo(const fvlbm_partition* p, int32_t src, int32_t dst, int64_t* count,
                                    int32_t* src_local, int32_t* dst_local) {
    clear_error();
    if (!p || !count || src < 0 || src >= p->n_parts || dst < 0 || dst >= p->n_parts)
        return fail(FVLBM_ERR_ARG, "fvlbm_partition_halo: bad arguments");
    *count = 0;
    for (const HaloMsg& m : p->msgs)
        if (m.src == src && m.dst == dst) {
            *count = (int64_t)m.src_local.size();
            if (src_local) std::copy(m.src_local.begin(), m.src_local.end(), src_local);
            if (dst_local) std::copy(m.dst_local.begin(), m.dst_local.end(), dst_local);
        }
    return FVLBM_OK;
}
