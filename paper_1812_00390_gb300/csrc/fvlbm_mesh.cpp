// Mesh construction and FP64 geometry precompute (host only).
//
// From the caller's polygon connectivity this builds, per cell and face slot:
// the outward normal times length and the midpoint of the face (Sec. 2.2,
// Eq. rhs), the neighbour across it (interior or periodic pair) or its
// boundary tag (Sec. 2.4), the least-squares coefficients of the cell's
// gradient (Eq. leastsquare, weights 1/|x_n - x_i|^2), and which side is
// upwind for each direction (Eq. lslrflux).  Cells are then renumbered along a
// Hilbert curve of their centroids so that face neighbours sit close in memory.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "fvlbm_internal.h"

namespace fvlbm {

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

static const int EXI[FVLBM_Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EYI[FVLBM_Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

static uint32_t slot_kind_of(int32_t bc_kind) {
    switch (bc_kind) {
        case FVLBM_BC_WALL: return SK_WALL;
        case FVLBM_BC_INLET: return SK_INLET;
        case FVLBM_BC_OUTLET: return SK_OUTLET;
        case FVLBM_BC_SYMMETRY: return SK_SYMMETRY;
        default: return SK_NONE;
    }
}

// Hilbert index of (x, y) on a 2^16 grid.
static uint64_t hilbert(uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
        d += (uint64_t)s * s * ((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = (s - 1) - (x & (s - 1)) + (x & ~(s - 1));
                y = (s - 1) - (y & (s - 1)) + (y & ~(s - 1));
                x &= 0xFFFF; y &= 0xFFFF;
            }
            std::swap(x, y);
        }
    }
    return d;
}

struct EdgeKey {
    int32_t a, b;
    int64_t cell;
    int32_t k;
};

static int build_single(const double* xy, int64_t n_vert, const int64_t* cell_ptr,
                        const int32_t* cell_vert, int64_t n_cell, const int32_t* bedge,
                        const int32_t* btag, int64_t n_bedge, const fvlbm_bc* bcs,
                        int32_t n_bc, Mesh& M) {
    if (!xy || !cell_ptr || !cell_vert || n_cell <= 0 || n_vert <= 0 || (n_bedge > 0 && (!bedge || !btag)) ||
        n_bc < 0 || (n_bc > 0 && !bcs) || n_bedge < 0)
        return fail(FVLBM_ERR_ARG, "fvlbm_mesh_create: null pointer or bad size");
    if (n_cell > INT32_MAX / 2) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_create: too many cells");
    if (cell_ptr[0] != 0) return fail(FVLBM_ERR_ARG, "cell_ptr[0] must be 0");
    for (int32_t t = 0; t < n_bc; t++) {
        const fvlbm_bc& b = bcs[t];
        if (b.kind < FVLBM_BC_WALL || b.kind > FVLBM_BC_PERIODIC)
            return fail(FVLBM_ERR_ARG, "bc %d: unknown kind %d", t, b.kind);
        if (b.kind == FVLBM_BC_PERIODIC && (b.partner < 0 || b.partner >= n_bc || bcs[b.partner].kind != FVLBM_BC_PERIODIC))
            return fail(FVLBM_ERR_ARG, "bc %d: periodic partner %d is not a periodic tag", t, b.partner);
        if ((b.kind == FVLBM_BC_INLET || b.kind == FVLBM_BC_OUTLET) && !(b.rho_inf > 0))
            return fail(FVLBM_ERR_ARG, "bc %d: rho_inf must be positive", t);
    }
    M.n_cell = M.n_owned = M.n_grad = n_cell;
    M.n_inst = 1;
    M.inst_begin = {0, n_cell};
    M.inst_bc_begin = {0, n_bc};
    M.bcs.assign(bcs, bcs + n_bc);
    M.nf.assign(n_cell, 0);
    M.area.assign(n_cell, 0);
    M.cx.assign(n_cell, 0);
    M.cy.assign(n_cell, 0);
    M.slots.assign((size_t)n_cell * MAXP, Slot());
    std::vector<double> lx(n_cell), ly(n_cell);
    M.max_faces = 0;
    M.total_area = 0;

    // polygon geometry
    for (int64_t c = 0; c < n_cell; c++) {
        int64_t s = cell_ptr[c];
        int64_t nv = cell_ptr[c + 1] - s;
        if (nv < 3 || nv > MAXP)
            return fail(FVLBM_ERR_ARG, "cell %lld has %lld vertices (3..%d allowed)", (long long)c, (long long)nv, MAXP);
        double a2 = 0, sx = 0, sy = 0, x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
        for (int k = 0; k < nv; k++) {
            int32_t va = cell_vert[s + k], vb = cell_vert[s + (k + 1) % nv];
            if (va < 0 || va >= n_vert || vb < 0 || vb >= n_vert)
                return fail(FVLBM_ERR_ARG, "cell %lld: vertex index out of range", (long long)c);
            double xa = xy[2 * va], ya = xy[2 * va + 1], xb = xy[2 * vb], yb = xy[2 * vb + 1];
            double cr = xa * yb - xb * ya;
            a2 += cr;
            sx += (xa + xb) * cr;
            sy += (ya + yb) * cr;
            x0 = std::min(x0, xa); x1 = std::max(x1, xa);
            y0 = std::min(y0, ya); y1 = std::max(y1, ya);
            Slot& S = M.slots[(size_t)c * MAXP + k];
            S.nx = yb - ya;
            S.ny = -(xb - xa);
            S.px = 0.5 * (xa + xb);
            S.py = 0.5 * (ya + yb);
            S.vx = xa;
            S.vy = ya;
        }
        if (!(a2 > 0))
            return fail(FVLBM_ERR_DEGENERATE_CELL, "cell %lld has non-positive area (vertices must be CCW)", (long long)c);
        M.nf[c] = (int32_t)nv;
        M.max_faces = std::max<int32_t>(M.max_faces, (int32_t)nv);
        M.area[c] = 0.5 * a2;
        M.cx[c] = sx / (3.0 * a2);
        M.cy[c] = sy / (3.0 * a2);
        lx[c] = x1 - x0;
        ly[c] = y1 - y0;
        M.total_area += M.area[c];
    }

    // interior faces by edge matching
    std::vector<EdgeKey> E;
    E.reserve((size_t)cell_ptr[n_cell]);
    for (int64_t c = 0; c < n_cell; c++) {
        int64_t s = cell_ptr[c];
        int nv = M.nf[c];
        for (int k = 0; k < nv; k++) {
            int32_t va = cell_vert[s + k], vb = cell_vert[s + (k + 1) % nv];
            E.push_back({std::min(va, vb), std::max(va, vb), c, k});
        }
    }
    auto lessk = [](const EdgeKey& x, const EdgeKey& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        if (x.cell != y.cell) return x.cell < y.cell;
        return x.k < y.k;
    };
    std::sort(E.begin(), E.end(), lessk);
    std::vector<EdgeKey> B((size_t)n_bedge);
    for (int64_t i = 0; i < n_bedge; i++)
        B[i] = {std::min(bedge[2 * i], bedge[2 * i + 1]), std::max(bedge[2 * i], bedge[2 * i + 1]), i, 0};
    std::sort(B.begin(), B.end(), lessk);
    M.n_face = M.n_bface = M.n_periodic = 0;
    std::vector<std::vector<std::pair<int64_t, int>>> per_tag(n_bc);
    for (size_t i = 0; i < E.size();) {
        size_t j = i + 1;
        while (j < E.size() && E[j].a == E[i].a && E[j].b == E[i].b) j++;
        if (j - i == 2) {
            Slot& s0 = M.slots[(size_t)E[i].cell * MAXP + E[i].k];
            Slot& s1 = M.slots[(size_t)E[i + 1].cell * MAXP + E[i + 1].k];
            s0.kind = s1.kind = SK_INTERIOR;
            s0.nb = (int32_t)E[i + 1].cell; s0.nb_slot = E[i + 1].k;
            s1.nb = (int32_t)E[i].cell; s1.nb_slot = E[i].k;
            M.n_face++;
        } else if (j - i == 1) {
            auto it = std::lower_bound(B.begin(), B.end(), EdgeKey{E[i].a, E[i].b, -1, 0}, lessk);
            if (it == B.end() || it->a != E[i].a || it->b != E[i].b)
                return fail(FVLBM_ERR_UNTAGGED_BOUNDARY, "edge (%d, %d) of cell %lld is on the boundary but not tagged",
                            E[i].a, E[i].b, (long long)E[i].cell);
            int32_t tag = btag[it->cell];
            if (tag < 0 || tag >= n_bc) return fail(FVLBM_ERR_ARG, "boundary edge %lld: tag %d out of range", (long long)it->cell, tag);
            Slot& s0 = M.slots[(size_t)E[i].cell * MAXP + E[i].k];
            s0.bc = tag;
            if (bcs[tag].kind == FVLBM_BC_PERIODIC) {
                per_tag[tag].push_back({E[i].cell, E[i].k});
            } else {
                s0.kind = (int32_t)slot_kind_of(bcs[tag].kind);
                M.n_face++;
                M.n_bface++;
            }
        } else {
            return fail(FVLBM_ERR_MESH_TOPOLOGY, "edge (%d, %d) is shared by %zu cells", E[i].a, E[i].b, j - i);
        }
        i = j;
    }

    // periodic pairs: midpoint of the partner edge + shift lands on this edge's midpoint
    for (int32_t t = 0; t < n_bc; t++) {
        if (bcs[t].kind != FVLBM_BC_PERIODIC) continue;
        int32_t p = bcs[t].partner;
        for (auto& ce : per_tag[t]) {
            Slot& s0 = M.slots[(size_t)ce.first * MAXP + ce.second];
            if (s0.kind == SK_INTERIOR) continue;  // paired from the partner side
            double len = std::sqrt(s0.nx * s0.nx + s0.ny * s0.ny);
            bool found = false;
            for (auto& pe : per_tag[p]) {
                Slot& s1 = M.slots[(size_t)pe.first * MAXP + pe.second];
                if (s1.kind == SK_INTERIOR) continue;
                if (pe.first == ce.first && pe.second == ce.second) continue;
                double ex = s1.px + bcs[t].shift[0] - s0.px, ey = s1.py + bcs[t].shift[1] - s0.py;
                if (std::sqrt(ex * ex + ey * ey) <= 1e-9 * len) {
                    s0.kind = s1.kind = SK_INTERIOR;
                    s0.periodic = s1.periodic = 1;
                    s0.nb = (int32_t)pe.first; s0.nb_slot = pe.second;
                    s1.nb = (int32_t)ce.first; s1.nb_slot = ce.second;
                    s0.sx = bcs[t].shift[0]; s0.sy = bcs[t].shift[1];
                    s1.sx = bcs[p].shift[0]; s1.sy = bcs[p].shift[1];
                    found = true;
                    M.n_face++;
                    M.n_periodic++;
                    break;
                }
            }
            if (!found)
                return fail(FVLBM_ERR_MESH_TOPOLOGY, "periodic edge of cell %lld (tag %d) has no partner in tag %d",
                            (long long)ce.first, t, p);
        }
    }

    // upwind masks; periodic pairs must agree on the upwind side of every direction
    for (int64_t c = 0; c < n_cell; c++) {
        for (int k = 0; k < M.nf[c]; k++) {
            Slot& S = M.slots[(size_t)c * MAXP + k];
            S.outmask = 0;
            for (int a = 1; a < FVLBM_Q; a++) {
                double en = EXI[a] * S.nx + EYI[a] * S.ny;
                if (en > 0) S.outmask |= 1u << (a - 1);
            }
        }
    }
    for (int64_t c = 0; c < n_cell; c++) {
        for (int k = 0; k < M.nf[c]; k++) {
            const Slot& S = M.slots[(size_t)c * MAXP + k];
            if (S.kind != SK_INTERIOR) continue;
            const Slot& T = M.slots[(size_t)S.nb * MAXP + S.nb_slot];
            for (int a = 1; a < FVLBM_Q; a++) {
                double e0 = EXI[a] * S.nx + EYI[a] * S.ny, e1 = EXI[a] * T.nx + EYI[a] * T.ny;
                bool o0 = e0 > 0, o1 = e1 > 0;
                if ((e0 != 0 || e1 != 0) && o0 == o1)
                    return fail(FVLBM_ERR_MESH_TOPOLOGY, "cells %lld and %d disagree on the upwind side of a face",
                                (long long)c, S.nb);
            }
        }
    }

    // least-squares coefficients (Eq. leastsquare): grad = sum_k c_k (v_k - f_c),
    // c_k = M^{-1} w_k d_k, M = sum_k w_k d_k d_k^T, w_k = 1 / |d_k|^2
    for (int64_t c = 0; c < n_cell; c++) {
        double dxs[MAXP], dys[MAXP];
        double m11 = 0, m12 = 0, m22 = 0;
        for (int k = 0; k < M.nf[c]; k++) {
            const Slot& S = M.slots[(size_t)c * MAXP + k];
            double xn, yn;
            if (S.kind == SK_INTERIOR) {
                xn = M.cx[S.nb] + S.sx;
                yn = M.cy[S.nb] + S.sy;
            } else if (S.kind == SK_WALL) {
                xn = S.px;
                yn = S.py;
            } else {  // ghost cell: mirror image of the centroid in the face line
                double len = std::sqrt(S.nx * S.nx + S.ny * S.ny);
                double nx = S.nx / len, ny = S.ny / len;
                double dn = (S.px - M.cx[c]) * nx + (S.py - M.cy[c]) * ny;
                xn = M.cx[c] + 2.0 * dn * nx;
                yn = M.cy[c] + 2.0 * dn * ny;
            }
            double dx = xn - M.cx[c], dy = yn - M.cy[c];
            M.slots[(size_t)c * MAXP + k].sdx = dx;
            M.slots[(size_t)c * MAXP + k].sdy = dy;
            double w = 1.0 / (dx * dx + dy * dy);
            dxs[k] = w * dx;
            dys[k] = w * dy;
            m11 += w * dx * dx;
            m12 += w * dx * dy;
            m22 += w * dy * dy;
        }
        double det = m11 * m22 - m12 * m12;
        if (!(det > 1e-12 * (m11 + m22) * (m11 + m22)))
            return fail(FVLBM_ERR_DEGENERATE_CELL, "cell %lld: singular least-squares matrix", (long long)c);
        for (int k = 0; k < M.nf[c]; k++) {
            Slot& S = M.slots[(size_t)c * MAXP + k];
            S.cgx = (m22 * dxs[k] - m12 * dys[k]) / det;
            S.cgy = (m11 * dys[k] - m12 * dxs[k]) / det;
        }
    }

    // CFL length of Eq. (CFL): min over cells of A / (Lx + Ly)
    double lmin = INFINITY;
    for (int64_t c = 0; c < n_cell; c++) lmin = std::min(lmin, M.area[c] / (lx[c] + ly[c]));
    M.inst_cfl_len = {lmin};

    // Hilbert order of centroids
    double bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
    for (int64_t c = 0; c < n_cell; c++) {
        bx0 = std::min(bx0, M.cx[c]); bx1 = std::max(bx1, M.cx[c]);
        by0 = std::min(by0, M.cy[c]); by1 = std::max(by1, M.cy[c]);
    }
    double span = std::max(bx1 - bx0, by1 - by0);
    if (!(span > 0)) span = 1;
    std::vector<uint64_t> key(n_cell);
    for (int64_t c = 0; c < n_cell; c++) {
        uint32_t qx = (uint32_t)std::min(65535.0, std::floor((M.cx[c] - bx0) / span * 65535.0));
        uint32_t qy = (uint32_t)std::min(65535.0, std::floor((M.cy[c] - by0) / span * 65535.0));
        key[c] = hilbert(qx, qy);
    }
    M.perm.resize(n_cell);
    std::iota(M.perm.begin(), M.perm.end(), 0);
    std::stable_sort(M.perm.begin(), M.perm.end(), [&](int64_t x, int64_t y) { return key[x] < key[y]; });
    M.iperm.resize(n_cell);
    for (int64_t i = 0; i < n_cell; i++) M.iperm[M.perm[i]] = i;
    return FVLBM_OK;
}

}  // namespace fvlbm

using namespace fvlbm;

extern "C" int fvlbm_mesh_create(const double* xy, int64_t n_vert, const int64_t* cell_ptr,
                                 const int32_t* cell_vert, int64_t n_cell, const int32_t* bedge,
                                 const int32_t* btag, int64_t n_bedge, const fvlbm_bc* bcs, int32_t n_bc,
                                 fvlbm_mesh** out) {
    clear_error();
    if (!out) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_create: out is null");
    *out = nullptr;
    fvlbm_mesh* m = new (std::nothrow) fvlbm_mesh;
    if (!m) return fail(FVLBM_ERR_OOM, "fvlbm_mesh_create: out of host memory");
    int rc;
    try {
        rc = build_single(xy, n_vert, cell_ptr, cell_vert, n_cell, bedge, btag, n_bedge, bcs, n_bc, m->m);
    } catch (const std::bad_alloc&) {
        rc = fail(FVLBM_ERR_OOM, "fvlbm_mesh_create: out of host memory");
    }
    if (rc != FVLBM_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return FVLBM_OK;
}

extern "C" int fvlbm_mesh_concat(const fvlbm_mesh* const* meshes, int32_t n, fvlbm_mesh** out) {
    clear_error();
    if (!out || !meshes || n <= 0) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_concat: bad arguments");
    *out = nullptr;
    for (int32_t i = 0; i < n; i++)
        if (!meshes[i]) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_concat: mesh %d is null", i);
    fvlbm_mesh* r = new (std::nothrow) fvlbm_mesh;
    if (!r) return fail(FVLBM_ERR_OOM, "fvlbm_mesh_concat: out of host memory");
    try {
        Mesh& R = r->m;
        int64_t nc = 0;
        for (int32_t i = 0; i < n; i++) nc += meshes[i]->m.n_cell;
        if (nc > INT32_MAX / 2) {
            delete r;
            return fail(FVLBM_ERR_ARG, "fvlbm_mesh_concat: too many cells");
        }
        R.n_cell = R.n_owned = R.n_grad = nc;
        R.n_inst = 0;
        R.inst_begin = {0};
        R.inst_bc_begin = {0};
        R.max_faces = 0;
        R.slots.reserve((size_t)nc * MAXP);
        for (int32_t i = 0; i < n; i++) {
            const Mesh& A = meshes[i]->m;
            int64_t c0 = R.inst_begin.back();
            int32_t b0 = R.inst_bc_begin.back();
            for (int32_t k = 0; k < A.n_inst; k++) {
                R.inst_begin.push_back(c0 + A.inst_begin[k + 1]);
                R.inst_bc_begin.push_back(b0 + A.inst_bc_begin[k + 1]);
                R.inst_cfl_len.push_back(A.inst_cfl_len[k]);
                R.n_inst++;
            }
            R.bcs.insert(R.bcs.end(), A.bcs.begin(), A.bcs.end());
            R.nf.insert(R.nf.end(), A.nf.begin(), A.nf.end());
            R.area.insert(R.area.end(), A.area.begin(), A.area.end());
            R.cx.insert(R.cx.end(), A.cx.begin(), A.cx.end());
            R.cy.insert(R.cy.end(), A.cy.begin(), A.cy.end());
            for (const Slot& S : A.slots) {
                Slot T = S;
                if (T.kind == SK_INTERIOR) T.nb += (int32_t)c0;
                if (T.bc >= 0) T.bc += b0;
                R.slots.push_back(T);
            }
            for (int64_t p : A.perm) R.perm.push_back(p + c0);
            R.max_faces = std::max(R.max_faces, A.max_faces);
            R.n_face += A.n_face;
            R.n_bface += A.n_bface;
            R.n_periodic += A.n_periodic;
            R.total_area += A.total_area;
        }
        R.iperm.resize(nc);
        for (int64_t i = 0; i < nc; i++) R.iperm[R.perm[i]] = i;
    } catch (const std::bad_alloc&) {
        delete r;
        return fail(FVLBM_ERR_OOM, "fvlbm_mesh_concat: out of host memory");
    }
    *out = r;
    return FVLBM_OK;
}

extern "C" void fvlbm_mesh_destroy(fvlbm_mesh* mesh) { delete mesh; }

extern "C" int fvlbm_mesh_info(const fvlbm_mesh* mesh, fvlbm_mesh_info_t* info) {
    clear_error();
    if (!mesh || !info) return fail(FVLBM_ERR_ARG, "fvlbm_mesh_info: null argument");
    const Mesh& M = mesh->m;
    info->n_cell = M.n_cell;
    info->n_face = M.n_face;
    info->n_bface = M.n_bface;
    info->n_periodic = M.n_periodic;
    info->max_faces = M.max_faces;
    info->n_instances = M.n_inst;
    info->total_area = M.total_area;
    double l = INFINITY;
    for (double x : M.inst_cfl_len) l = std::min(l, x);
    info->min_cfl_length = l;
    return FVLBM_OK;
}

namespace fvlbm {
// CFL number times the smaller of the advective limit of Eq. (CFL) and the
// collision limit of Eq. (timetau) (tau for AB2).
double suggest_dt(const Mesh& M, int inst, double tau, double cfl, double umax, int scheme) {
    double adv = M.inst_cfl_len[inst] / (std::sqrt(2.0) + umax);
    double col = scheme == FVLBM_AB2 ? tau : 2.0 * tau;
    return cfl * (adv < col ? adv : col);
}
}  // namespace fvlbm

extern "C" int fvlbm_suggest_dt(const fvlbm_mesh* mesh, int32_t instance, double tau, double cfl,
                                double u_max, int32_t scheme, double* dt) {
    clear_error();
    if (!mesh || !dt || instance < 0 || instance >= mesh->m.n_inst || !(tau > 0) || !(cfl > 0) || !(u_max >= 0) ||
        scheme < FVLBM_EULER || scheme > FVLBM_RK4)
        return fail(FVLBM_ERR_ARG, "fvlbm_suggest_dt: bad arguments");
    *dt = suggest_dt(mesh->m, instance, tau, cfl, u_max, scheme);
    return FVLBM_OK;
}

extern "C" const char* fvlbm_last_error(void) { return fvlbm::g_err.c_str(); }
