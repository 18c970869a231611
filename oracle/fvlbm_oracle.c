/*
 * Plain FP64 CPU oracle of the cell-centred finite-volume lattice Boltzmann
 * method (D2Q9) of Wang, Zhong, Cao & Zhuo, "A simplified finite volume
 * lattice Boltzmann method ... Part I" (arXiv:1812.00390).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * library itself never does.  It shares no code, header or table with the
 * CUDA path: it has its own mesh reader, face builder, geometry and solver.
 *
 * What it computes, in the paper's order (Sec. 2, "Step 0" .. "Step 7"):
 *   Step 0  f = f^eq(rho, u)                                  Eq. (feq)
 *   Step 1  wall-face values and ghost values                 Sec. 2.4.1
 *   Step 2  weighted least-squares gradient of every f_alpha  Eq. (leastsquare)
 *   Step 3  inlet / outlet / symmetry face values             Sec. 2.4.2
 *   Step 4  RHS = -(1/A) sum_m (e.n) f_face dl - (f - f^eq)/tau   Eq. (rhs)
 *   Step 5  explicit time scheme (Euler, AB2, multistage RK)  Sec. 2.3
 *   Step 6  macroscopic rho, u                                Sec. 2.1
 * plus the velocity residual of Sec. 3.2 and the total mass sum(A rho).
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *   - tau = nu / c_s^2 with no 1/2 shift (Eq. relaxtime).
 *   - The multistage scheme is f^(k+1) = f^(0) + beta_{k+1} dt RHS(f^(k)), the
 *     printed "- beta RHS" being the residual sign convention of the cited
 *     Jameson-type scheme with dt absorbed; "RK2" is the 2-stage member with
 *     beta = (1/2, 1), "RK4" the 4-stage one with beta = (1/4, 1/3, 1/2, 1).
 *   - The least-squares stencil of a cell holds one point per face: the
 *     neighbour centroid (shifted by the period vector across a periodic
 *     face), the wall-face midpoint P carrying f_P (Eq. wallbc), or, for an
 *     inlet / outlet / symmetry face, the ghost value placed at the mirror
 *     image of the cell centroid in the face line.
 *   - The wall value f_P is the face value for every direction.
 *   - Where e_alpha . n = 0 the flux term is zero whatever face value is taken;
 *     the paper's "<=" branch (neighbour side) is used.
 *   - Cell centre = area centroid of the polygon.
 *   - The velocity residual's denominator is sqrt(sum(u^2 + v^2)).
 *   - A face is periodic when its edge carries a periodic tag; it is matched
 *     with the partner-tag edge whose midpoint, moved by the tag's shift,
 *     lands on its own midpoint.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* D2Q9 velocities and weights, Sec. 2.1 (c = 1, c_s^2 = 1/3). */
static const double EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const double EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

enum { K_WALL = 0, K_INLET = 1, K_OUTLET = 2, K_SYMMETRY = 3, K_PERIODIC = 4 };
enum { F_INTERIOR = 0, F_PERIODIC = 1, F_BOUNDARY = 2 };
enum { S_EULER = 0, S_RK2 = 1, S_AB2 = 2, S_RK4 = 3 };

typedef struct {
    int type;        /* F_INTERIOR, F_PERIODIC or F_BOUNDARY */
    int nb;          /* neighbour cell (interior / periodic) */
    int nb_face;     /* index of the same face inside the neighbour */
    int tag;         /* boundary tag (boundary faces) */
    double sx, sy;   /* periodic: neighbour image = neighbour centroid + (sx, sy) */
    double nx, ny;   /* (e.n) dl = ex*nx + ey*ny: outward normal times length */
    double px, py;   /* face midpoint */
} Face;

typedef struct {
    int64_t n_cell;
    int *nface;        /* faces per cell */
    Face **face;       /* face[c][k]: edge from vertex k to k+1 of cell c */
    double *area, *cx, *cy, *lx, *ly;
    int n_tag;
    int *kind, *ext;
    double *uw, *rinf, *uinf; /* [tag][2], [tag], [tag][2] */
    double *f;         /* [n_cell][Q] current state */
    double *rhs_prev;  /* AB2: previous RHS */
    int have_prev;
    /* work */
    double *grad;      /* [n_cell][Q][2] */
    double *rho, *ux, *uy;
} Oracle;

/* Eq. (feq): f^eq = rho w [1 + e.u/cs2 + (e.u)^2/(2 cs4) - u^2/(2 cs2)]. */
static double feq(int a, double rho, double ux, double uy) {
    const double cs2 = 1.0 / 3.0;
    double eu = EX[a] * ux + EY[a] * uy;
    double uu = ux * ux + uy * uy;
    return rho * W[a] * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
}

/* Sec. 2.1: rho = sum f, rho u = sum f e. */
static void moments(const double *f, double *rho, double *ux, double *uy) {
    double r = 0, mx = 0, my = 0;
    for (int a = 0; a < Q; a++) {
        r += f[a];
        mx += f[a] * EX[a];
        my += f[a] * EY[a];
    }
    *rho = r;
    *ux = mx / r;
    *uy = my / r;
}

typedef struct { int a, b, cell, k; } EdgeRec;

static int cmp_edge(const void *p, const void *q) {
    const EdgeRec *x = (const EdgeRec *)p, *y = (const EdgeRec *)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return x->k < y->k ? -1 : (x->k > y->k);
}

void orc_destroy(void *hv) {
    Oracle *h = (Oracle *)hv;
    if (!h) return;
    if (h->face)
        for (int64_t c = 0; c < h->n_cell; c++) free(h->face[c]);
    free(h->face); free(h->nface);
    free(h->area); free(h->cx); free(h->cy); free(h->lx); free(h->ly);
    free(h->kind); free(h->ext); free(h->uw); free(h->rinf); free(h->uinf);
    free(h->f); free(h->rhs_prev); free(h->grad);
    free(h->rho); free(h->ux); free(h->uy);
    free(h);
}

static void *fail(Oracle *h, char *err, int errlen, const char *msg) {
    if (err && errlen > 0) snprintf(err, (size_t)errlen, "%s", msg);
    orc_destroy(h);
    return NULL;
}

/*
 * Build the oracle's own mesh description: cells, faces, geometry.
 * Cells are CCW polygons (cell_ptr CSR into cell_vert).  Edges seen by two
 * cells are interior faces; an edge seen by one cell must be a tagged
 * boundary edge.  Periodic tags pair edges by midpoint + shift.
 */
void *orc_create(int64_t n_vert, const double *xy, int64_t n_cell, const int64_t *cell_ptr,
                 const int32_t *cell_vert, int64_t n_bedge, const int32_t *bedge,
                 const int32_t *btag, int32_t n_tag, const int32_t *kind,
                 const int32_t *external, const double *uw, const double *rho_inf,
                 const double *uinf, const int32_t *partner, const double *shift,
                 char *err, int errlen) {
    Oracle *h = (Oracle *)calloc(1, sizeof(Oracle));
    if (!h) return NULL;
    h->n_cell = n_cell;
    h->nface = (int *)calloc((size_t)n_cell, sizeof(int));
    h->face = (Face **)calloc((size_t)n_cell, sizeof(Face *));
    h->area = (double *)calloc((size_t)n_cell, sizeof(double));
    h->cx = (double *)calloc((size_t)n_cell, sizeof(double));
    h->cy = (double *)calloc((size_t)n_cell, sizeof(double));
    h->lx = (double *)calloc((size_t)n_cell, sizeof(double));
    h->ly = (double *)calloc((size_t)n_cell, sizeof(double));
    h->f = (double *)calloc((size_t)n_cell * Q, sizeof(double));
    h->rhs_prev = (double *)calloc((size_t)n_cell * Q, sizeof(double));
    h->grad = (double *)calloc((size_t)n_cell * Q * 2, sizeof(double));
    h->rho = (double *)calloc((size_t)n_cell, sizeof(double));
    h->ux = (double *)calloc((size_t)n_cell, sizeof(double));
    h->uy = (double *)calloc((size_t)n_cell, sizeof(double));
    h->n_tag = n_tag;
    h->kind = (int *)calloc((size_t)n_tag + 1, sizeof(int));
    h->ext = (int *)calloc((size_t)n_tag + 1, sizeof(int));
    h->uw = (double *)calloc((size_t)n_tag * 2 + 2, sizeof(double));
    h->rinf = (double *)calloc((size_t)n_tag + 1, sizeof(double));
    h->uinf = (double *)calloc((size_t)n_tag * 2 + 2, sizeof(double));
    for (int t = 0; t < n_tag; t++) {
        h->kind[t] = kind[t];
        h->ext[t] = external[t];
        h->uw[2 * t] = uw[2 * t]; h->uw[2 * t + 1] = uw[2 * t + 1];
        h->rinf[t] = rho_inf[t];
        h->uinf[2 * t] = uinf[2 * t]; h->uinf[2 * t + 1] = uinf[2 * t + 1];
    }

    /* Per-cell polygon geometry: shoelace area, area centroid, bounding box. */
    int64_t n_edge = cell_ptr[n_cell];
    for (int64_t c = 0; c < n_cell; c++) {
        int64_t s = cell_ptr[c];
        int nv = (int)(cell_ptr[c + 1] - s);
        if (nv < 3) return fail(h, err, errlen, "cell with fewer than 3 vertices");
        double A2 = 0, sx = 0, sy = 0;
        double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
        for (int k = 0; k < nv; k++) {
            int va = cell_vert[s + k], vb = cell_vert[s + (k + 1) % nv];
            if (va < 0 || va >= n_vert) return fail(h, err, errlen, "vertex index out of range");
            double xa = xy[2 * va], ya = xy[2 * va + 1], xb = xy[2 * vb], yb = xy[2 * vb + 1];
            double cr = xa * yb - xb * ya;
            A2 += cr;
            sx += (xa + xb) * cr;
            sy += (ya + yb) * cr;
            if (xa < xmin) xmin = xa;
            if (xa > xmax) xmax = xa;
            if (ya < ymin) ymin = ya;
            if (ya > ymax) ymax = ya;
        }
        if (!(A2 > 0)) return fail(h, err, errlen, "cell with non-positive area (not CCW?)");
        h->area[c] = 0.5 * A2;
        h->cx[c] = sx / (3.0 * A2);
        h->cy[c] = sy / (3.0 * A2);
        h->lx[c] = xmax - xmin;
        h->ly[c] = ymax - ymin;
        h->nface[c] = nv;
        h->face[c] = (Face *)calloc((size_t)nv, sizeof(Face));
        for (int k = 0; k < nv; k++) {
            int va = cell_vert[s + k], vb = cell_vert[s + (k + 1) % nv];
            Face *F = &h->face[c][k];
            double dx = xy[2 * vb] - xy[2 * va], dy = xy[2 * vb + 1] - xy[2 * va + 1];
            /* outward normal of a CCW edge, times its length */
            F->nx = dy;
            F->ny = -dx;
            F->px = 0.5 * (xy[2 * va] + xy[2 * vb]);
            F->py = 0.5 * (xy[2 * va + 1] + xy[2 * vb + 1]);
            F->nb = -1;
            F->tag = -1;
        }
    }

    /* Interior faces: the same vertex pair seen from two cells. */
    EdgeRec *E = (EdgeRec *)malloc((size_t)n_edge * sizeof(EdgeRec));
    int64_t ne = 0;
    for (int64_t c = 0; c < n_cell; c++) {
        int64_t s = cell_ptr[c];
        int nv = h->nface[c];
        for (int k = 0; k < nv; k++) {
            int va = cell_vert[s + k], vb = cell_vert[s + (k + 1) % nv];
            E[ne].a = va < vb ? va : vb;
            E[ne].b = va < vb ? vb : va;
            E[ne].cell = (int)c;
            E[ne].k = k;
            ne++;
        }
    }
    qsort(E, (size_t)ne, sizeof(EdgeRec), cmp_edge);
    /* boundary edge lookup table, sorted the same way */
    EdgeRec *B = (EdgeRec *)malloc((size_t)(n_bedge > 0 ? n_bedge : 1) * sizeof(EdgeRec));
    for (int64_t i = 0; i < n_bedge; i++) {
        int va = bedge[2 * i], vb = bedge[2 * i + 1];
        B[i].a = va < vb ? va : vb;
        B[i].b = va < vb ? vb : va;
        B[i].cell = (int)i; /* index of the boundary edge */
        B[i].k = 0;
    }
    qsort(B, (size_t)n_bedge, sizeof(EdgeRec), cmp_edge);
    for (int64_t i = 0; i < ne;) {
        int64_t j = i + 1;
        while (j < ne && E[j].a == E[i].a && E[j].b == E[i].b) j++;
        if (j - i == 2) {
            Face *F0 = &h->face[E[i].cell][E[i].k], *F1 = &h->face[E[i + 1].cell][E[i + 1].k];
            F0->type = F_INTERIOR; F0->nb = E[i + 1].cell; F0->nb_face = E[i + 1].k;
            F1->type = F_INTERIOR; F1->nb = E[i].cell; F1->nb_face = E[i].k;
        } else if (j - i == 1) {
            /* must be a tagged boundary edge: binary search */
            int64_t lo = 0, hi = n_bedge - 1, hit = -1;
            while (lo <= hi) {
                int64_t mid = (lo + hi) / 2;
                if (B[mid].a == E[i].a && B[mid].b == E[i].b) { hit = mid; break; }
                if (B[mid].a < E[i].a || (B[mid].a == E[i].a && B[mid].b < E[i].b)) lo = mid + 1;
                else hi = mid - 1;
            }
            if (hit < 0) { free(E); free(B); return fail(h, err, errlen, "untagged boundary edge"); }
            int tag = btag[B[hit].cell];
            if (tag < 0 || tag >= n_tag) { free(E); free(B); return fail(h, err, errlen, "boundary tag out of range"); }
            Face *F = &h->face[E[i].cell][E[i].k];
            F->type = F_BOUNDARY;
            F->tag = tag;
        } else {
            free(E); free(B);
            return fail(h, err, errlen, "edge shared by more than two cells");
        }
        i = j;
    }
    free(E);
    free(B);

    /* Periodic pairing: edge with tag t pairs with the partner-tag edge whose
       midpoint + shift_t equals its own midpoint (Sec. 3.1 names periodic
       boundaries; the pairing rule is this reading). */
    for (int64_t c = 0; c < n_cell; c++) {
        for (int k = 0; k < h->nface[c]; k++) {
            Face *F = &h->face[c][k];
            if (F->type != F_BOUNDARY || kind[F->tag] != K_PERIODIC) continue;
            int t = F->tag, p = partner[t];
            double sx = shift[2 * t], sy = shift[2 * t + 1];
            double len = sqrt(F->nx * F->nx + F->ny * F->ny);
            int found = 0;
            for (int64_t c2 = 0; c2 < n_cell && !found; c2++) {
                for (int k2 = 0; k2 < h->nface[c2]; k2++) {
                    Face *G = &h->face[c2][k2];
                    if (G->type == F_INTERIOR || G->tag != p) continue;
                    if (G->type == F_PERIODIC && G->nb >= 0 && !(G->nb == c && G->nb_face == k)) continue;
                    double ex = G->px + sx - F->px, ey = G->py + sy - F->py;
                    if (sqrt(ex * ex + ey * ey) <= 1e-9 * len) {
                        F->type = F_PERIODIC; F->nb = (int)c2; F->nb_face = k2;
                        F->sx = sx; F->sy = sy;
                        found = 1;
                        break;
                    }
                }
            }
            if (!found) return fail(h, err, errlen, "periodic edge without a partner");
        }
    }
    for (int64_t c = 0; c < n_cell; c++)
        for (int k = 0; k < h->nface[c]; k++)
            if (h->face[c][k].type == F_BOUNDARY && h->kind[h->face[c][k].tag] == K_PERIODIC)
                return fail(h, err, errlen, "unpaired periodic edge");
    return h;
}

int orc_geometry(void *hv, double *area, double *centroid, double *lxly) {
    Oracle *h = (Oracle *)hv;
    for (int64_t c = 0; c < h->n_cell; c++) {
        if (area) area[c] = h->area[c];
        if (centroid) { centroid[2 * c] = h->cx[c]; centroid[2 * c + 1] = h->cy[c]; }
        if (lxly) { lxly[2 * c] = h->lx[c]; lxly[2 * c + 1] = h->ly[c]; }
    }
    return 0;
}

int64_t orc_n_faces(void *hv) {
    Oracle *h = (Oracle *)hv;
    int64_t n = 0;
    for (int64_t c = 0; c < h->n_cell; c++) n += h->nface[c];
    return n;
}

void orc_feq(double rho, double ux, double uy, double *out) {
    for (int a = 0; a < Q; a++) out[a] = feq(a, rho, ux, uy);
}

int orc_set_f(void *hv, const double *f) {
    Oracle *h = (Oracle *)hv;
    memcpy(h->f, f, (size_t)h->n_cell * Q * sizeof(double));
    h->have_prev = 0;
    return 0;
}

int orc_get_f(void *hv, double *f) {
    Oracle *h = (Oracle *)hv;
    memcpy(f, h->f, (size_t)h->n_cell * Q * sizeof(double));
    return 0;
}

/* Step 0: f = f^eq(rho, u) per cell. */
int orc_set_equilibrium(void *hv, const double *rho, const double *u) {
    Oracle *h = (Oracle *)hv;
    for (int64_t c = 0; c < h->n_cell; c++)
        for (int a = 0; a < Q; a++) h->f[c * Q + a] = feq(a, rho[c], u[2 * c], u[2 * c + 1]);
    h->have_prev = 0;
    return 0;
}

/* Step 6. */
void orc_macros(void *hv, double *rho, double *u) {
    Oracle *h = (Oracle *)hv;
    for (int64_t c = 0; c < h->n_cell; c++) {
        double r, x, y;
        moments(&h->f[c * Q], &r, &x, &y);
        if (rho) rho[c] = r;
        if (u) { u[2 * c] = x; u[2 * c + 1] = y; }
    }
}

double orc_mass(void *hv) {
    Oracle *h = (Oracle *)hv;
    double m = 0;
    for (int64_t c = 0; c < h->n_cell; c++) {
        double r = 0;
        for (int a = 0; a < Q; a++) r += h->f[c * Q + a];
        m += h->area[c] * r;
    }
    return m;
}

/* Velocity residual of Sec. 3.2 between the current state and u_old [n][2]. */
double orc_residual(void *hv, const double *u_old) {
    Oracle *h = (Oracle *)hv;
    double num = 0, den = 0;
    for (int64_t c = 0; c < h->n_cell; c++) {
        double r, x, y;
        moments(&h->f[c * Q], &r, &x, &y);
        double dx = x - u_old[2 * c], dy = y - u_old[2 * c + 1];
        num += dx * dx + dy * dy;
        den += u_old[2 * c] * u_old[2 * c] + u_old[2 * c + 1] * u_old[2 * c + 1];
    }
    if (den == 0) return num == 0 ? 0.0 : INFINITY;
    return sqrt(num) / sqrt(den);
}

/*
 * Ghost / boundary value G_alpha of a boundary face of cell c (Sec. 2.4.1):
 *   wall      f_P  = f^eq(rho_c, u_w) + f_c - f^eq_c            Eq. (wallbc)
 *   inlet     f_GC = f^eq(rho*, u_inf) + f_c - f^eq_c, rho* = rho_inf
 *                    (external flow) or rho_c (internal flow)
 *   outlet    f_GC = f_c (external); f^eq(rho_inf, u_c) + f_c - f^eq_c (internal)
 *   symmetry  f_GC = f^eq(rho_c, u*), u* = u_c mirrored in the face line
 */
static double ghost_value(const Oracle *h, const double *fc, double rho, double ux, double uy,
                          const Face *F, int a) {
    int t = F->tag;
    double fe = feq(a, rho, ux, uy);
    switch (h->kind[t]) {
    case K_WALL:
        return feq(a, rho, h->uw[2 * t], h->uw[2 * t + 1]) + fc[a] - fe;
    case K_INLET: {
        double rs = h->ext[t] ? h->rinf[t] : rho;
        return feq(a, rs, h->uinf[2 * t], h->uinf[2 * t + 1]) + fc[a] - fe;
    }
    case K_OUTLET:
        if (h->ext[t]) return fc[a];
        return feq(a, h->rinf[t], ux, uy) + fc[a] - fe;
    case K_SYMMETRY: {
        double len = sqrt(F->nx * F->nx + F->ny * F->ny);
        double nx = F->nx / len, ny = F->ny / len;
        double un = ux * nx + uy * ny;
        return feq(a, rho, ux - 2.0 * un * nx, uy - 2.0 * un * ny);
    }
    }
    return NAN;
}

/* Position of the least-squares stencil point that face k of cell c provides. */
static void stencil_point(const Oracle *h, int64_t c, const Face *F, double *x, double *y) {
    if (F->type == F_INTERIOR) { *x = h->cx[F->nb]; *y = h->cy[F->nb]; return; }
    if (F->type == F_PERIODIC) { *x = h->cx[F->nb] + F->sx; *y = h->cy[F->nb] + F->sy; return; }
    if (h->kind[F->tag] == K_WALL) { *x = F->px; *y = F->py; return; }
    /* ghost cell centre: mirror image of the cell centre in the face line */
    double len = sqrt(F->nx * F->nx + F->ny * F->ny);
    double nx = F->nx / len, ny = F->ny / len;
    double dn = (F->px - h->cx[c]) * nx + (F->py - h->cy[c]) * ny;
    *x = h->cx[c] + 2.0 * dn * nx;
    *y = h->cy[c] + 2.0 * dn * ny;
}

/* Stencil point of face k of cell c, for tests of the geometry. */
int orc_stencil_point(void *hv, int64_t c, int k, double *xy) {
    Oracle *h = (Oracle *)hv;
    if (c < 0 || c >= h->n_cell || k < 0 || k >= h->nface[c]) return -1;
    stencil_point(h, c, &h->face[c][k], &xy[0], &xy[1]);
    return h->face[c][k].type == F_BOUNDARY ? h->kind[h->face[c][k].tag] : 10 + h->face[c][k].type;
}

/* Value of f_alpha at that stencil point. */
static double stencil_value(const Oracle *h, const double *f, const Face *F, int64_t c, int a) {
    if (F->type != F_BOUNDARY) return f[(int64_t)F->nb * Q + a];
    return ghost_value(h, &f[c * Q], h->rho[c], h->ux[c], h->uy[c], F, a);
}

/*
 * RHS of Eq. (rhs) for state f: Steps 1-4.
 */
int orc_rhs(void *hv, const double *f, double tau, double *rhs) {
    Oracle *h = (Oracle *)hv;
    const int64_t n = h->n_cell;
    /* macros of every cell (needed by ghost values) */
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++) moments(&f[c * Q], &h->rho[c], &h->ux[c], &h->uy[c]);

    /* Step 2: weighted least-squares gradient, Eq. (leastsquare):
       minimise sum_n w_n [f_n - f_c - g.(x_n - x_c)]^2, w_n = 1/|x_n - x_c|^2,
       via its 2x2 normal equations, solved by Cramer's rule. */
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++) {
        double m11 = 0, m12 = 0, m22 = 0;
        double b1[Q] = {0}, b2[Q] = {0};
        for (int k = 0; k < h->nface[c]; k++) {
            const Face *F = &h->face[c][k];
            double xn, yn;
            stencil_point(h, c, F, &xn, &yn);
            double dx = xn - h->cx[c], dy = yn - h->cy[c];
            double w = 1.0 / (dx * dx + dy * dy);
            m11 += w * dx * dx;
            m12 += w * dx * dy;
            m22 += w * dy * dy;
            for (int a = 0; a < Q; a++) {
                double df = stencil_value(h, f, F, c, a) - f[c * Q + a];
                b1[a] += w * dx * df;
                b2[a] += w * dy * df;
            }
        }
        double det = m11 * m22 - m12 * m12;
        for (int a = 0; a < Q; a++) {
            h->grad[(c * Q + a) * 2 + 0] = (b1[a] * m22 - b2[a] * m12) / det;
            h->grad[(c * Q + a) * 2 + 1] = (m11 * b2[a] - m12 * b1[a]) / det;
        }
    }

    /* Steps 3-4: face values (Eq. lslrflux and Sec. 2.4.2), flux sum, collision. */
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++) {
        const double *fc = &f[c * Q];
        double flux[Q] = {0};
        for (int k = 0; k < h->nface[c]; k++) {
            const Face *F = &h->face[c][k];
            for (int a = 0; a < Q; a++) {
                double en = EX[a] * F->nx + EY[a] * F->ny; /* (e.n) dl */
                double own = fc[a] + h->grad[(c * Q + a) * 2] * (F->px - h->cx[c]) +
                             h->grad[(c * Q + a) * 2 + 1] * (F->py - h->cy[c]);
                double fv;
                if (F->type != F_BOUNDARY) {
                    if (en > 0) {
                        fv = own;
                    } else {
                        int64_t j = F->nb;
                        const Face *Fj = &h->face[j][F->nb_face];
                        fv = f[j * Q + a] + h->grad[(j * Q + a) * 2] * (Fj->px - h->cx[j]) +
                             h->grad[(j * Q + a) * 2 + 1] * (Fj->py - h->cy[j]);
                    }
                } else {
                    double G = ghost_value(h, fc, h->rho[c], h->ux[c], h->uy[c], F, a);
                    switch (h->kind[F->tag]) {
                    case K_WALL: fv = G; break;
                    case K_INLET: fv = en > 0 ? own : G; break;
                    case K_OUTLET:
                        if (h->ext[F->tag]) fv = fc[a];
                        else fv = en > 0 ? own : G;
                        break;
                    case K_SYMMETRY: fv = 0.5 * (fc[a] + G); break;
                    default: fv = NAN;
                    }
                }
                flux[a] += en * fv;
            }
        }
        for (int a = 0; a < Q; a++) {
            double fe = feq(a, h->rho[c], h->ux[c], h->uy[c]);
            rhs[c * Q + a] = -flux[a] / h->area[c] - (fc[a] - fe) / tau;
        }
    }
    return 0;
}

/* Step 5: explicit time schemes of Sec. 2.3. */
int orc_run(void *hv, int scheme, double tau, double dt, int64_t nsteps) {
    Oracle *h = (Oracle *)hv;
    const int64_t nq = h->n_cell * Q;
    double *r = (double *)malloc((size_t)nq * sizeof(double));
    double *f0 = (double *)malloc((size_t)nq * sizeof(double));
    double *fk = (double *)malloc((size_t)nq * sizeof(double));
    if (!r || !f0 || !fk) { free(r); free(f0); free(fk); return -1; }
    for (int64_t s = 0; s < nsteps; s++) {
        if (scheme == S_EULER) {                       /* Eq. (euler) */
            orc_rhs(h, h->f, tau, r);
            for (int64_t i = 0; i < nq; i++) h->f[i] += dt * r[i];
        } else if (scheme == S_AB2) {                  /* AB2, first step Euler */
            orc_rhs(h, h->f, tau, r);
            if (!h->have_prev) {
                for (int64_t i = 0; i < nq; i++) h->f[i] += dt * r[i];
            } else {
                for (int64_t i = 0; i < nq; i++) h->f[i] += 0.5 * dt * (3.0 * r[i] - h->rhs_prev[i]);
            }
            memcpy(h->rhs_prev, r, (size_t)nq * sizeof(double));
            h->have_prev = 1;
        } else {                                       /* multistage RK */
            static const double B2[2] = {0.5, 1.0};
            static const double B4[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
            const double *beta = scheme == S_RK2 ? B2 : B4;
            int ns = scheme == S_RK2 ? 2 : 4;
            memcpy(f0, h->f, (size_t)nq * sizeof(double));
            memcpy(fk, h->f, (size_t)nq * sizeof(double));
            for (int k = 0; k < ns; k++) {
                orc_rhs(h, fk, tau, r);
                for (int64_t i = 0; i < nq; i++) fk[i] = f0[i] + beta[k] * dt * r[i];
            }
            memcpy(h->f, fk, (size_t)nq * sizeof(double));
        }
    }
    free(r); free(f0); free(fk);
    return 0;
}

/*
 * Time step of Eqs. (CFL) and (timetau).  Both are stability limits: the
 * advective one dt <= L / (|e|_max + |U|_max), L = min_c A_c/(Lx_c+Ly_c) over
 * all cells (Lx, Ly the cell's projected lengths), and the collision one
 * dt <= 2 tau (tau for AB2, the paper's observed AB2 limit).  The chosen step
 * is the CFL number times the smaller of the two, so that neither limit is
 * met with equality (at dt = 2 tau the relaxation factor of Euler and of the
 * 2-stage scheme has modulus exactly 1).
 */
double orc_cfl_dt(void *hv, double cfl, double umax, double tau, int scheme) {
    Oracle *h = (Oracle *)hv;
    double lmin = INFINITY;
    for (int64_t c = 0; c < h->n_cell; c++) {
        double l = h->area[c] / (h->lx[c] + h->ly[c]);
        if (l < lmin) lmin = l;
    }
    double adv = lmin / (sqrt(2.0) + umax);
    double col = scheme == S_AB2 ? tau : 2.0 * tau;
    return cfl * (adv < col ? adv : col);
}

/*
 * Timing aid (no arithmetic): threads the OpenMP loops above use from now on
 * (n <= 0 leaves the setting); returns the number in effect (1 without OpenMP).
 */
int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
