// Solver lifecycle and the C ABI entry points that touch the GPU.
//
// fvlbm_init packs the FP64 mesh precompute into the device layout of the
// chosen precision (SoA planes [slot][cell] in the locality order), uploads it
// into one workspace, and writes Step 0 (f = f^eq).  fvlbm_step enqueues the
// stages of the time scheme (Sec. 2.3) on the solver's stream.  Everything
// that reads results back (macros, residual, mass, f) synchronises and maps
// cells back to the caller's numbering.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "fvlbm_internal.h"

namespace fvlbm {
double suggest_dt(const Mesh& M, int inst, double tau, double cfl, double umax, int scheme);
}

using namespace fvlbm;

struct fvlbm_solver {
    int device = 0;
    cudaStream_t stream = nullptr;
    int prec = FVLBM_FP64;
    int scheme = FVLBM_EULER;
    int64_t n_cell = 0;
    int32_t n_inst = 1;
    std::vector<int64_t> inst_begin;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    DevView v{};
    std::vector<InstParam> inst;
    bool ab2_started = false;
    // set_f reads the caller's host buffer directly (see fvlbm_host_transfer)
    bool host_can_direct = false;
    bool host_direct = false;
    // single-stage schemes on the fused stage alternate the state between
    // buf[0] and buf[1] (a tile must not overwrite cells other tiles still
    // read); v.fa is always the current state, buf[cur]
    bool pingpong = false;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    // the 4-stage scheme on the fused stage: a third stage buffer, so that no
    // stage writes the buffer it reads (the middle stages alternate fb, fc)
    void* fc = nullptr;
    // CUDA graphs of one step and of GRAPH_CHUNK steps, built lazily, one pair
    // per state buffer the step starts from
    cudaGraphExec_t g1[2] = {nullptr, nullptr}, gk[2] = {nullptr, nullptr};
    bool graphs_ok = true;
    int64_t direct_steps = 0;
};

static constexpr int64_t GRAPH_CHUNK = 32;

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    return fail(FVLBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr size_t ALIGN = 256;
constexpr int64_t CHUNK = 4096;

size_t real_size(int prec) { return prec == FVLBM_FP64 ? 8 : 4; }
// bytes of stored state per cell: 9 values, or for the 16-bit split format
// 3 FP32 moments + 6 16-bit non-equilibrium values
size_t state_bytes(int prec) {
    return prec == FVLBM_FP64 ? 72 : (prec == FVLBM_FP32_DEV ? 36 : 24);
}

// Tile structure of the fused stage kernel.  Tiles are runs of consecutive
// cells (internal order), cut where tile and 1-ring (face neighbours outside
// the tile) would exceed the CTA's `tile` threads, or where the local cells
// (tile, 1-ring, 2-ring = face neighbours of the 1-ring outside tile and
// 1-ring) or the tile's faces would exceed the kernel's shared-memory
// capacity.  Every tile cell slot carries the local
// index of its neighbour and the local index of its face; every 1-ring slot
// the local index of its neighbour and, for faces shared with the tile, the
// local face.
struct TilePlan {
    int tile = 0;
    int64_t n_tiles = 0;
    std::vector<int64_t> begin;     // [n_tiles + 1]
    std::vector<int64_t> halo_ptr;  // [n_tiles + 1]
    std::vector<int32_t> halo;      // 1-ring then 2-ring of each tile
    std::vector<int64_t> r1_ptr;    // [n_tiles + 1]
    std::vector<uint32_t> link;     // [n_cell][maxf] local neighbour | local face << 16
    std::vector<uint32_t> r1link;   // [1-ring entries][maxf] same fields
    int32_t max_local = 0, max_faces = 0;
    int64_t short_tiles = 0;        // tiles cut below `tile` cells by the capacity
    int64_t sum_len = 0, sum_ring1 = 0, sum_local = 0;   // over the tiles
    // filled when the plan is verified (fvlbm_plan_info): modelled
    // shared-memory wavefronts of the warp accesses, and failed invariants
    bool verify = false;
    double face_groups = 0, face_waves = 0, gather_groups = 0, gather_waves = 0;
    int64_t violations = 0;
    std::string first_violation;
};

int64_t internal_nbr(const Mesh& M, int64_t i, int k) {
    const Slot& S = M.slots[(size_t)M.perm[i] * MAXP + k];
    return S.kind == SK_INTERIOR ? M.iperm[S.nb] : -1;
}

// Shared-memory capacity of the fused kernel for a tile size (TileDims).
bool tile_dims(int tile, int maxf, int rsize, int& ls, int& fs, size_t& bytes) {
#define FVLBM_TD(T_)                                                                                         \
    case T_:                                                                                                 \
        ls = TileDims<T_, 4, 4>::LS;                                                                         \
        fs = maxf <= 4 ? TileDims<T_, 4, 4>::FS : TileDims<T_, 8, 4>::FS;                                    \
        bytes = maxf <= 4 ? (rsize == 4 ? TileDims<T_, 4, 4>::BYTES : TileDims<T_, 4, 8>::BYTES)             \
                          : (rsize == 4 ? TileDims<T_, 8, 4>::BYTES : TileDims<T_, 8, 8>::BYTES);            \
        return true;
    switch (tile) {
        FVLBM_TD(128)
        FVLBM_TD(256)
        FVLBM_TD(512)
        FVLBM_TD(1024)
    }
#undef FVLBM_TD
    return false;
}

struct TileScratch {
    std::vector<int64_t> stamp;
    std::vector<int32_t> loc;
    std::vector<int64_t> r1, r2;
    std::vector<int32_t> t_nb, t_f, r_nb, r_f;
    std::vector<int32_t> bank_cnt, face_groups, face_row;   // bank_faces
    int64_t gen = 0;
};

// Face-table rows of a tile chosen for the shared-memory banks (4-byte banks,
// 32 of them: row r lies in bank r mod 32).  A warp reaches, through one
// slot, the faces of its 32 cells at once (phase 2 writes them, phase 3 reads
// them); faces that share a bank there are served one after the other.  Each
// face, in the order numbered, takes the bank that the fewest faces of its
// warps' slot groups already hold (ties: the emptiest bank, room permitting),
// and row bank + 32 * (faces already in that bank); face 0 keeps row 0, which
// unused slots read (with a zero weight: it must hold finite values, and
// every row of a face is written in full).  The rows are only addresses: the
// arithmetic does not change.
void bank_faces(const Mesh& M, int maxf, int64_t c0, int len, int fs, int nf, TileScratch& W) {
    const int n1 = (int)W.r1.size();
    const int depth = fs / BLK;   // rows per bank
    const int n_groups = (len + n1 + BLK - 1) / BLK * maxf;
    W.bank_cnt.assign((size_t)n_groups * BLK, 0);
    W.face_groups.assign((size_t)nf * 2, -1);   // a face is reached through at most two slots
    auto add = [&](int f, int g) {
        int* fg = &W.face_groups[(size_t)f * 2];
        if (fg[0] < 0) fg[0] = g;
        else if (fg[0] != g) fg[1] = g;
    };
    for (int li = 0; li < len; li++) {
        const int nfc = M.nf[M.perm[c0 + li]];
        for (int k = 0; k < maxf; k++) {
            const int g = li / BLK * maxf + k;
            if (k < nfc) add(W.t_f[(size_t)li * maxf + k], g);
            else W.bank_cnt[(size_t)g * BLK] = 1;
        }
    }
    for (int e = 0; e < n1; e++)
        for (int k = 0; k < maxf; k++) {
            const int f = W.r_f[(size_t)e * maxf + k];
            if (f >= 0) add(f, (len + e) / BLK * maxf + k);
        }
    int load[BLK] = {0};
    W.face_row.resize(nf);
    for (int f = 0; f < nf; f++) {
        const int* fg = &W.face_groups[(size_t)f * 2];
        int best = 0, best_cost = -1;
        // face 0 keeps row 0, the row unused slots read: it is written in full
        for (int b = f == 0 ? BLK : 0; b < BLK; b++) {
            if (load[b] >= depth) continue;
            int c = 0;
            for (int q = 0; q < 2; q++)
                if (fg[q] >= 0) c += W.bank_cnt[(size_t)fg[q] * BLK + b];
            c = c * (depth + 1) + load[b];
            if (best_cost < 0 || c < best_cost) {
                best_cost = c;
                best = b;
            }
        }
        for (int q = 0; q < 2; q++)
            if (fg[q] >= 0) W.bank_cnt[(size_t)fg[q] * BLK + best]++;
        W.face_row[f] = best + BLK * load[best]++;
    }
    for (int32_t& x : W.t_f)
        if (x >= 0) x = W.face_row[x];
    for (int32_t& x : W.r_f)
        if (x >= 0) x = W.face_row[x];
}

// Local numbering of the tile [c0, c0 + len): tile cells, 1-ring, 2-ring, and
// the local faces of the tile cells.  False when it exceeds ls / fs, or when
// tile and 1-ring together exceed the CTA's `threads` (the kernel gives every
// thread at most one gradient to compute).
bool try_tile(const Mesh& M, int maxf, int64_t c0, int len, int threads, int ls, int fs, TileScratch& W,
              int& n_local, int& n_faces) {
    const int64_t g = ++W.gen;
    int nl = 0;
    for (int64_t i = c0; i < c0 + len; i++) {
        W.stamp[i] = g;
        W.loc[i] = nl++;
    }
    W.r1.clear();
    W.r2.clear();
    for (int64_t i = c0; i < c0 + len; i++)
        for (int k = 0; k < M.nf[M.perm[i]]; k++) {
            const int64_t j = internal_nbr(M, i, k);
            if (j >= 0 && W.stamp[j] != g) {
                W.stamp[j] = g;
                W.loc[j] = nl++;
                W.r1.push_back(j);
            }
        }
    for (int64_t j : W.r1)
        for (int k = 0; k < M.nf[M.perm[j]]; k++) {
            const int64_t q = internal_nbr(M, j, k);
            if (q >= 0 && W.stamp[q] != g) {
                W.stamp[q] = g;
                W.loc[q] = nl++;
                W.r2.push_back(q);
            }
        }
    const int n1 = (int)W.r1.size();
    if (nl > ls || len + n1 > threads) return false;
    // 1-ring and 2-ring each in global order: the kernel gathers them with
    // consecutive threads, which then share the rows of a 32-cell block
    std::sort(W.r1.begin(), W.r1.end());
    std::sort(W.r2.begin(), W.r2.end());
    int x = len;
    for (int64_t j : W.r1) W.loc[j] = x++;
    for (int64_t q : W.r2) W.loc[q] = x++;
    W.t_nb.assign((size_t)len * maxf, -1);
    W.t_f.assign((size_t)len * maxf, -1);
    W.r_nb.assign((size_t)n1 * maxf, -1);
    W.r_f.assign((size_t)n1 * maxf, -1);
    // faces numbered slot by slot (all cells' slot 0, then slot 1, ...): the
    // cells of a warp then reach their slot-k faces at mostly consecutive
    // indices, which spreads their face-table accesses over the memory banks
    int nf = 0;
    for (int k = 0; k < maxf; k++) {
        for (int li = 0; li < len; li++) {
            const int64_t c = M.perm[c0 + li];
            if (k >= M.nf[c]) continue;
            const Slot& S = M.slots[(size_t)c * MAXP + k];
            const size_t x = (size_t)li * maxf + k;
            if (S.kind == SK_INTERIOR) {
                const int lj = W.loc[M.iperm[S.nb]];
                W.t_nb[x] = lj;
                if (W.t_f[x] < 0) {
                    W.t_f[x] = nf;
                    if (lj < len) W.t_f[(size_t)lj * maxf + S.nb_slot] = nf;
                    else W.r_f[(size_t)(lj - len) * maxf + S.nb_slot] = nf;
                    nf++;
                }
            } else {
                W.t_f[x] = nf++;
            }
        }
    }
    if (nf > fs) return false;
    bank_faces(M, maxf, c0, len, fs, nf, W);
    for (int e = 0; e < n1; e++)
        for (int k = 0; k < M.nf[M.perm[W.r1[e]]]; k++) {
            const int64_t q = internal_nbr(M, W.r1[e], k);
            if (q >= 0) W.r_nb[(size_t)e * maxf + k] = W.loc[q];
        }
    // Slots without a neighbour (boundary faces, unused slots) link to the
    // cell itself, so that the kernel's gradient loop needs no test of the
    // slot kind (the difference to itself is zero); unused slots of tile
    // cells name face row 0, which they never write (their mask is empty) and
    // whose values they weight by a zero face vector.
    for (int li = 0; li < len; li++) {
        const int nfc = M.nf[M.perm[c0 + li]];
        for (int k = 0; k < maxf; k++) {
            const size_t x = (size_t)li * maxf + k;
            if (W.t_nb[x] < 0) W.t_nb[x] = li;
            if (k >= nfc) W.t_f[x] = 0;
        }
    }
    for (int e = 0; e < n1; e++)
        for (int k = 0; k < maxf; k++)
            if (W.r_nb[(size_t)e * maxf + k] < 0) W.r_nb[(size_t)e * maxf + k] = len + e;
    n_local = nl;
    n_faces = nf;
    return true;
}

uint32_t pack_link(int nb, int f) {
    return (uint32_t)(nb < 0 ? LINK_NONE : (uint32_t)nb) | ((uint32_t)(f < 0 ? LINK_NONE : (uint32_t)f) << 16);
}

uint32_t writer_mask(const Slot& S, int64_t i, int k, int64_t j);

// Shared-memory wavefronts of one warp access (4-byte banks, 32 of them):
// the most distinct addresses that fall into one bank.
int bank_waves(const int* idx, int n) {
    int v[BLK];
    for (int q = 0; q < n; q++) v[q] = idx[q];
    std::sort(v, v + n);
    int cnt[BLK] = {0}, m = 0;
    for (int q = 0; q < n; q++)
        if (q == 0 || v[q] != v[q - 1]) m = std::max(m, ++cnt[v[q] & (BLK - 1)]);
    return m;
}

// Checks of one tile's plan (fvlbm_plan_info): every slot links to its
// neighbour's local index (boundary and unused slots to the cell itself, unused
// slots to face row 0), the two sides of a face name one row and no two faces
// share one, every (face, direction) between local cells has exactly one
// writer, and tile + 1-ring and the local cells fit the CTA; then the modelled
// wavefronts of phase 3's face-table reads and phase 2's neighbour gathers.
void verify_tile(const Mesh& M, int maxf, int64_t c0, int len, int threads, int ls, int fs, int nl,
                 const TileScratch& W, TilePlan& P) {
    auto bad = [&](const char* what, int64_t cell) {
        if (P.violations++ == 0) {
            char b[200];
            std::snprintf(b, sizeof b, "tile at cell %lld: %s (cell %lld)", (long long)c0, what, (long long)cell);
            P.first_violation = b;
        }
    };
    const int n1 = (int)W.r1.size();
    if (len + n1 > threads) bad("tile and 1-ring exceed the CTA's threads", c0);
    if (nl > ls) bad("local cells exceed the shared-memory capacity", c0);
    auto slot = [&](int64_t i, int k) -> const Slot& { return M.slots[(size_t)M.perm[i] * MAXP + k]; };
    // a face is named by its side with the lower (cell, slot)
    auto face_key = [&](int64_t i, int k) {
        const Slot& S = slot(i, k);
        if (S.kind == SK_INTERIOR) {
            const int64_t j = M.iperm[S.nb];
            if (j < i || (j == i && S.nb_slot < k)) return std::make_pair(j, S.nb_slot);
        }
        return std::make_pair(i, k);
    };
    std::vector<std::pair<int64_t, int>> owner((size_t)fs, std::make_pair((int64_t)-1, -1));
    for (int li = 0; li < len; li++) {
        const int64_t i = c0 + li;
        const int nfc = M.nf[M.perm[i]];
        for (int k = 0; k < maxf; k++) {
            const size_t x = (size_t)li * maxf + k;
            if (k >= nfc) {
                if (W.t_nb[x] != li || W.t_f[x] != 0) bad("unused slot not linked to itself and row 0", i);
                continue;
            }
            const int row = W.t_f[x];
            if (row < 0 || row >= fs) {
                bad("face row outside the table", i);
                continue;
            }
            const auto key = face_key(i, k);
            if (owner[row].first < 0) owner[row] = key;
            else if (owner[row] != key) bad("two faces share a face row", i);
            const Slot& S = slot(i, k);
            if (S.kind != SK_INTERIOR) {
                if (W.t_nb[x] != li) bad("boundary slot not linked to itself", i);
                continue;
            }
            const int64_t j = M.iperm[S.nb];
            const int lj = W.loc[j];
            if (W.t_nb[x] != lj) bad("slot not linked to its neighbour", i);
            int other = -2;
            if (lj < len) other = W.t_f[(size_t)lj * maxf + S.nb_slot];
            else if (lj < len + n1) other = W.r_f[(size_t)(lj - len) * maxf + S.nb_slot];
            else bad("a tile cell's neighbour is not in the tile or its 1-ring", i);
            if (other != -2 && other != row) bad("the two sides of a face name different rows", i);
            const uint32_t mi = writer_mask(S, i, k, j), mj = writer_mask(slot(j, S.nb_slot), j, S.nb_slot, i);
            if ((mi & mj) != 0 || (mi | mj) != 0xFFu) bad("a (face, direction) without exactly one writer", i);
        }
    }
    for (int e = 0; e < n1; e++) {
        const int64_t j = W.r1[e];
        const int nfc = M.nf[M.perm[j]];
        for (int k = 0; k < maxf; k++) {
            const int64_t q = k < nfc ? internal_nbr(M, j, k) : -1;
            const int want = q >= 0 ? W.loc[q] : len + e;
            if (W.r_nb[(size_t)e * maxf + k] != want) bad("1-ring slot not linked to its neighbour", j);
        }
    }
    // modelled wavefronts of the warp accesses through one slot (used slots only)
    int idx[BLK];
    for (int w = 0; w * BLK < len; w++)
        for (int k = 0; k < maxf; k++) {
            int n = 0;
            bool used = k < 3;
            for (int li = w * BLK; li < std::min(len, (w + 1) * BLK); li++) {
                idx[n++] = W.t_f[(size_t)li * maxf + k];
                used |= k < M.nf[M.perm[c0 + li]];
            }
            if (!used) continue;
            P.face_groups += 1;
            P.face_waves += bank_waves(idx, n);
        }
    for (int w = 0; w * BLK < len + n1; w++)
        for (int k = 0; k < maxf; k++) {
            int n = 0;
            bool used = k < 3;
            for (int l = w * BLK; l < std::min(len + n1, (w + 1) * BLK); l++) {
                const int64_t c = l < len ? c0 + l : W.r1[l - len];
                idx[n++] = l < len ? W.t_nb[(size_t)l * maxf + k] : W.r_nb[(size_t)(l - len) * maxf + k];
                used |= k < M.nf[M.perm[c]];
            }
            if (!used) continue;
            P.gather_groups += 1;
            P.gather_waves += bank_waves(idx, n);
        }
}

int make_tiles(const Mesh& M, int maxf, int tile, TilePlan& P, bool verify) {
    int ls = 0, fs = 0;
    size_t bytes = 0;
    if (!tile_dims(tile, maxf, 4, ls, fs, bytes)) return fail(FVLBM_ERR_ARG, "unsupported tile size %d", tile);
    const int64_t n = M.n_cell;
    P = TilePlan{};
    P.tile = tile;
    P.verify = verify;
    P.begin.push_back(0);
    P.halo_ptr.push_back(0);
    P.r1_ptr.push_back(0);
    P.link.assign((size_t)n * maxf, 0xFFFFFFFFu);
    TileScratch W;
    W.stamp.assign(n, 0);
    W.loc.assign(n, 0);
    // tiles cover the owned cells; ghost cells of a partition only appear in halos
    const int64_t n_own = M.n_owned;
    int64_t c0 = 0;
    int guess = tile;   // neighbouring tiles have similar lengths: start one block above the last
    while (c0 < n_own) {
        int len = (int)std::min<int64_t>(guess, n_own - c0);
        int nl = 0, nf = 0;
        while (!try_tile(M, maxf, c0, len, tile, ls, fs, W, nl, nf)) {
            if (len == 1)
                return fail(FVLBM_ERR_UNSUPPORTED, "cell %lld: its halo exceeds the fused stage's capacity",
                            (long long)c0);
            len = len > BLK ? (len - 1) / BLK * BLK : len / 2;
        }
        guess = std::min(tile, (len + BLK) / BLK * BLK);
        if (len < std::min<int64_t>(tile, n_own - c0)) P.short_tiles++;
        P.sum_len += len;
        P.sum_ring1 += (int64_t)W.r1.size();
        P.sum_local += nl;
        if (verify) verify_tile(M, maxf, c0, len, tile, ls, fs, nl, W, P);
        for (int li = 0; li < len; li++)
            for (int k = 0; k < maxf; k++) {
                const size_t x = (size_t)li * maxf + k;
                if (W.t_f[x] >= 0) P.link[(size_t)(c0 + li) * maxf + k] = pack_link(W.t_nb[x], W.t_f[x]);
            }
        for (int64_t j : W.r1) P.halo.push_back((int32_t)j);
        for (int64_t q : W.r2) P.halo.push_back((int32_t)q);
        for (size_t x = 0; x < W.r_nb.size(); x++) P.r1link.push_back(pack_link(W.r_nb[x], W.r_f[x]));
        c0 += len;
        P.begin.push_back(c0);
        P.halo_ptr.push_back((int64_t)P.halo.size());
        P.r1_ptr.push_back(P.r1_ptr.back() + (int64_t)W.r1.size());
        P.max_local = std::max(P.max_local, nl);
        P.max_faces = std::max(P.max_faces, nf);
    }
    P.n_tiles = (int64_t)P.begin.size() - 1;
    return FVLBM_OK;
}

// Offsets of every array inside the workspace (0 size when a strategy does not use it).
struct Layout {
    int64_t np, n_face, n_chunk;
    int maxf;
    int strategy;
    int block;
    bool pingpong;   // single-stage scheme on the fused stage: the state alternates between fa and fb
    TilePlan tp;
    size_t off_desc, off_geo, off_nbr, off_area, off_grp, off_inst, off_bc, off_fa, off_fb, off_fc, off_rprev, off_fv,
        off_rho, off_ux, off_uy, off_uold, off_part, off_red, off_conv, off_chunk, off_flag, off_tbegin, off_hptr,
        off_halo, off_r1ptr, off_r1link, off_iperm, total;
};

constexpr size_t SMEM_LIMIT = 227 * 1024;

// Streaming multiprocessors of a device (152 on GB300 when no device answers).
int device_sms(int device) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 152;
    }
    return n;
}
constexpr int64_t PLANE_ALIGN = 1024;  // cell arrays hold whole blocks and whole tiles of the largest size

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// kernel: 1 two-kernel, 128/256/512/1024 fused with that tile size, 0
// automatic.  The automatic choice, from measurements on GB300:
//  - FP32 / 16-bit: 512-thread tiles once the mesh gives every SM a tile of
//    512 (the fastest on large batches), 256-thread tiles down to a quarter of
//    the SMs' worth of them (e.g. the 128^2 cavity, the 60k-cell cylinder),
//    128-thread tiles below: a fused stage launches one kernel per stage where
//    the two-kernel stage launches two, which is what small meshes wait on;
//  - FP64: the two-kernel stage (it spends fewer FP64 operations: no 1-ring
//    gradients, and the FP64 mode is bound by GB300's FP64 units) except on
//    meshes of fewer than 32 cells per SM, which are launch-bound: fused 128.
// The two-kernel stage shrinks its blocks (down to 32 threads) so that small
// meshes still spread over the SMs.
int make_layout(const Mesh& M, int prec, int scheme, int kernel, Layout& L, int sms, bool verify = false) {
    L = Layout{};
    L.np = round_up(M.n_cell, PLANE_ALIGN);
    L.n_face = M.n_face;
    L.maxf = M.max_faces <= 4 ? 4 : 8;
    L.n_chunk = 0;
    for (int k = 0; k < M.n_inst; k++) L.n_chunk += (M.inst_begin[k + 1] - M.inst_begin[k] + CHUNK - 1) / CHUNK;
    const size_t R = real_size(prec), S = state_bytes(prec);
    if (kernel != 0 && kernel != 1 && kernel != 128 && kernel != 256 && kernel != 512 && kernel != 1024)
        return fail(FVLBM_ERR_ARG, "params.kernel = %d: use 0, 1, 128, 256, 512 or 1024", kernel);
    int tile = kernel;
    if (kernel == 0) {
        const int64_t n = M.n_owned;
        auto fits = [&](int t) {
            int ls = 0, fs = 0;
            size_t smem = 0;
            tile_dims(t, L.maxf, (int)R, ls, fs, smem);
            return smem <= SMEM_LIMIT;
        };
        if (prec == FVLBM_FP64) tile = n < 32 * (int64_t)sms ? 128 : 1;
        else if (n >= 512 * (int64_t)sms && fits(512)) tile = 512;
        else if (n >= 64 * (int64_t)sms) tile = 256;
        else tile = 128;
    }
    L.strategy = tile == 0 || tile == 1 ? STRATEGY_TWO_KERNEL : STRATEGY_TILE;
    L.block = 256;
    while (L.block > 32 && (M.n_owned + L.block - 1) / L.block < 2 * sms) L.block /= 2;
    if (L.strategy == STRATEGY_TILE) {
        int ls = 0, fs = 0;
        size_t smem = 0;
        tile_dims(tile, L.maxf, (int)R, ls, fs, smem);
        if (smem > SMEM_LIMIT)
            return fail(FVLBM_ERR_UNSUPPORTED, "fused stage with %d-cell tiles needs %zu B of shared memory (limit %zu)",
                        tile, smem, SMEM_LIMIT);
        int rc = make_tiles(M, L.maxf, tile, L.tp, verify);
        if (rc) return rc;
        // the fused kernel indexes its blocked arrays in 32 bits
        const uint64_t lim = (uint64_t)1 << 32;
        if ((uint64_t)L.np * 3 * L.maxf >= lim || (uint64_t)(L.tp.r1_ptr.back() + BLK) * L.maxf >= lim)
            return fail(FVLBM_ERR_UNSUPPORTED, "fused stage: %lld cells exceed its 32-bit indexing; use kernel = 1",
                        (long long)M.n_cell);
    }
    const bool tiled = L.strategy == STRATEGY_TILE, two = !tiled;
    L.pingpong = tiled && (scheme == FVLBM_EULER || scheme == FVLBM_AB2);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += (bytes + ALIGN - 1) / ALIGN * ALIGN;
        return r;
    };
    const size_t plane = (size_t)L.np, slots = plane * L.maxf;
    const size_t n_r1 = tiled ? (size_t)round_up(L.tp.r1_ptr.back(), BLK) : 0;
    L.off_desc = take(8 * slots);
    L.off_geo = take(2 * R * 3 * slots);
    L.off_nbr = take(two ? 4 * slots : 0);
    L.off_area = take(8 * plane);
    L.off_grp = take(4 * plane);
    L.off_iperm = take(4 * plane);
    L.off_inst = take(sizeof(InstParam) * M.n_inst);
    L.off_bc = take(sizeof(BcParam) * std::max<size_t>(1, M.bcs.size()));
    L.off_tbegin = take(tiled ? 8 * (size_t)(L.tp.n_tiles + 1) : 0);
    L.off_hptr = take(tiled ? 8 * (size_t)(L.tp.n_tiles + 1) : 0);
    L.off_halo = take(tiled ? 4 * L.tp.halo.size() : 0);
    L.off_r1ptr = take(tiled ? 8 * (size_t)(L.tp.n_tiles + 1) : 0);
    L.off_r1link = take(tiled ? 4 * n_r1 * L.maxf : 0);
    L.off_fa = take(S * plane);   // everything before this is uploaded once
    L.off_fb = (scheme == FVLBM_RK2 || scheme == FVLBM_RK4 || L.pingpong) ? take(S * plane) : 0;
    L.off_fc = (scheme == FVLBM_RK4 && tiled) ? take(S * plane) : 0;
    L.off_rprev = scheme == FVLBM_AB2 ? take(R * plane * FVLBM_Q) : 0;
    L.off_fv = take(two ? R * (size_t)std::max<int64_t>(1, L.n_face) * (FVLBM_Q - 1) : 0);
    L.off_rho = take(8 * plane);
    L.off_ux = take(8 * plane);
    L.off_uy = take(8 * plane);
    L.off_uold = take(16 * plane);
    L.off_part = take(24 * (size_t)std::max<int64_t>(1, L.n_chunk));
    L.off_red = take(24 * (size_t)M.n_inst);
    L.off_conv = take(8 * plane * FVLBM_Q);
    L.off_chunk = take(24 * (size_t)std::max<int64_t>(1, L.n_chunk));
    L.off_flag = take(16);
    L.total = o;
    return FVLBM_OK;
}

int check_params(const Mesh& M, const fvlbm_params* params, int32_t n_params) {
    if (M.n_cell >= ((int64_t)1 << 31)) return fail(FVLBM_ERR_ARG, "more than 2^31 - 1 cells");
    if (!params || !(n_params == 1 || n_params == M.n_inst))
        return fail(FVLBM_ERR_ARG, "params: need 1 or %d entries, got %d", M.n_inst, n_params);
    for (int32_t k = 0; k < n_params; k++) {
        const fvlbm_params& p = params[k];
        if (!(p.tau > 0) || !(p.dt >= 0) || !(p.cfl >= 0) || !(p.u_max >= 0) || !(p.rho0 > 0))
            return fail(FVLBM_ERR_ARG, "params[%d]: tau, rho0 must be > 0; dt, cfl, u_max >= 0", k);
        if (p.scheme < FVLBM_EULER || p.scheme > FVLBM_RK4) return fail(FVLBM_ERR_ARG, "params[%d]: bad scheme", k);
        if (p.precision < FVLBM_FP64 || p.precision > FVLBM_BF16_DEV)
            return fail(FVLBM_ERR_ARG, "params[%d]: bad precision", k);
        if (p.scheme != params[0].scheme || p.precision != params[0].precision || p.device != params[0].device ||
            p.kernel != params[0].kernel)
            return fail(FVLBM_ERR_ARG, "params[%d]: scheme, precision, device and kernel must match params[0]", k);
    }
    if (M.bcs.size() >= 65536) return fail(FVLBM_ERR_ARG, "too many boundary tags (%zu)", M.bcs.size());
    return FVLBM_OK;
}

// Largest speed the instance is set up with: |U|_max of Eq. (CFL) when not given.
double instance_umax(const Mesh& M, int k, const fvlbm_params& p) {
    if (p.u_max > 0) return p.u_max;
    double u = std::hypot(p.u0[0], p.u0[1]);
    for (int32_t b = M.inst_bc_begin[k]; b < M.inst_bc_begin[k + 1]; b++) {
        const fvlbm_bc& c = M.bcs[b];
        if (c.kind == FVLBM_BC_WALL) u = std::max(u, std::hypot(c.u_w[0], c.u_w[1]));
        if (c.kind == FVLBM_BC_INLET || c.kind == FVLBM_BC_OUTLET) u = std::max(u, std::hypot(c.u_inf[0], c.u_inf[1]));
    }
    return u;
}

// Index of component c of cell i in a blocked array of ncomp components.
inline size_t blk(int64_t i, int c, int ncomp) {
    return (size_t)((i >> BLK_SHIFT) * ((int64_t)ncomp << BLK_SHIFT) + ((int64_t)c << BLK_SHIFT) + (i & (BLK - 1)));
}

// Writer mask of an interior slot: the directions whose face value this side
// computes -- those it is upwind for (e.n > 0) and, for directions parallel
// to the face (e.n = 0, zero flux), the side with the smaller (cell, slot) so
// that every (face, direction) has exactly one finite writer.
uint32_t writer_mask(const Slot& S, int64_t i, int k, int64_t j) {
    static const int EXI[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int EYI[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    uint32_t m = S.outmask;
    const bool first = i < j || (i == j && k < S.nb_slot);
    if (first)
        for (int a = 1; a < FVLBM_Q; a++)
            if (EXI[a] * S.nx + EYI[a] * S.ny == 0.0) m |= 1u << (a - 1);
    return m;
}

template <typename T>
void pack_geometry(const Mesh& M, const Layout& L, std::vector<unsigned char>& host) {
    const int64_t n = M.n_cell;
    const int maxf = L.maxf;
    const bool two = L.strategy == STRATEGY_TWO_KERNEL;
    unsigned char* H = host.data();
    uint32_t* desc = (uint32_t*)(H + L.off_desc);   // pairs (x, y)
    T* geo = (T*)(H + L.off_geo);                   // pairs of T
    double* area = (double*)(H + L.off_area);
    int32_t* grp = (int32_t*)(H + L.off_grp);
    int32_t* iperm = (int32_t*)(H + L.off_iperm);
    for (int64_t c = 0; c < n; c++) iperm[c] = (int32_t)M.iperm[c];
    int32_t* nbr = two ? (int32_t*)(H + L.off_nbr) : nullptr;
    for (size_t x = 0; x < (size_t)maxf * L.np; x++) {
        desc[2 * x] = SK_NONE;
        desc[2 * x + 1] = 0xFFFFFFFFu;
        if (two) nbr[x] = -1;
    }
    // face ids of the two-kernel face table: both slots of an interior face share one
    std::vector<int32_t> fid;
    if (two) fid.assign((size_t)n * maxf, -1);
    int64_t next = 0;
    int32_t g = 0;
    for (int64_t i = 0; i < n; i++) {
        const int64_t c = M.perm[i];
        while (g + 1 < M.n_inst && c >= M.inst_begin[g + 1]) g++;
        grp[i] = g;
        area[i] = M.area[c];
        for (int k = 0; k < M.nf[c]; k++) {
            const Slot& S = M.slots[(size_t)c * MAXP + k];
            const size_t d = blk(i, k, maxf);
            const int64_t j = S.kind == SK_INTERIOR ? M.iperm[S.nb] : -1;
            // the directions this slot writes by reconstruction: on interior
            // faces the upwind ones (writer_mask), on inlet and internal-outlet
            // faces the outflow ones; the other boundary faces take ghost values
            // for every direction, so their mask is empty
            const bool io = S.kind == SK_INLET || (S.kind == SK_OUTLET && !M.bcs[S.bc].external);
            const uint32_t mask = S.kind == SK_INTERIOR ? writer_mask(S, i, k, j) : (io ? S.outmask : 0u);
            desc[2 * d] = (uint32_t)S.kind | (mask << 8) | ((uint32_t)(S.bc < 0 ? 0 : S.bc) << 16);
            if (two) {
                int32_t& f = fid[(size_t)i * maxf + k];
                if (f < 0) {
                    f = (int32_t)next++;
                    if (j >= 0) fid[(size_t)j * maxf + S.nb_slot] = f;
                }
                desc[2 * d + 1] = (uint32_t)f;
                nbr[d] = (int32_t)j;
            }
            const size_t q0 = blk(i, 3 * k, 3 * maxf), q1 = blk(i, 3 * k + 1, 3 * maxf), q2 = blk(i, 3 * k + 2, 3 * maxf);
            geo[2 * q0] = (T)S.cgx;
            geo[2 * q0 + 1] = (T)S.cgy;
            geo[2 * q1] = (T)(S.px - M.cx[c]);
            geo[2 * q1 + 1] = (T)(S.py - M.cy[c]);
            geo[2 * q2] = (T)(S.nx / M.area[c]);
            geo[2 * q2 + 1] = (T)(S.ny / M.area[c]);
        }
        // fused stage: every slot's tile-local links (unused slots included)
        if (!two)
            for (int k = 0; k < maxf; k++) desc[2 * blk(i, k, maxf) + 1] = L.tp.link[(size_t)i * maxf + k];
    }
    if (!two) {
        uint32_t* r1 = (uint32_t*)(H + L.off_r1link);
        const int64_t ne = L.tp.r1_ptr.back();
        for (int64_t e = 0; e < (int64_t)round_up(ne, BLK); e++)
            for (int k = 0; k < maxf; k++)
                r1[blk(e, k, maxf)] = e < ne ? L.tp.r1link[(size_t)e * maxf + k] : 0xFFFFFFFFu;
    }
}

}  // namespace

extern "C" int fvlbm_workspace_bytes(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params,
                                     size_t* bytes) {
    clear_error();
    if (!mesh || !bytes) return fail(FVLBM_ERR_ARG, "fvlbm_workspace_bytes: null argument");
    int rc = check_params(mesh->m, params, n_params);
    if (rc) return rc;
    Layout L;
    try {
        rc = make_layout(mesh->m, params[0].precision, params[0].scheme, params[0].kernel, L, device_sms(params[0].device));
    } catch (const std::bad_alloc&) {
        return fail(FVLBM_ERR_OOM, "fvlbm_workspace_bytes: out of host memory");
    }
    if (rc) return rc;
    *bytes = L.total;
    return FVLBM_OK;
}

extern "C" int fvlbm_plan_info(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params,
                               fvlbm_plan_info_t* info) {
    clear_error();
    if (!mesh || !info) return fail(FVLBM_ERR_ARG, "fvlbm_plan_info: null argument");
    int rc = check_params(mesh->m, params, n_params);
    if (rc) return rc;
    Layout L;
    try {
        rc = make_layout(mesh->m, params[0].precision, params[0].scheme, params[0].kernel, L,
                         device_sms(params[0].device), true);
    } catch (const std::bad_alloc&) {
        return fail(FVLBM_ERR_OOM, "fvlbm_plan_info: out of host memory");
    }
    if (rc) return rc;
    const TilePlan& P = L.tp;
    fvlbm_plan_info_t o{};
    const bool tiled = L.strategy == STRATEGY_TILE;
    o.stage_kernel = tiled ? P.tile : 1;
    o.slots = L.maxf;
    o.n_tiles = tiled ? P.n_tiles : 0;
    o.short_tiles = P.short_tiles;
    o.max_local_cells = P.max_local;
    o.max_faces = P.max_faces;
    if (tiled && P.n_tiles > 0) {
        o.mean_tile_cells = (double)P.sum_len / P.n_tiles;
        o.mean_ring1_cells = (double)P.sum_ring1 / P.n_tiles;
        o.mean_local_cells = (double)P.sum_local / P.n_tiles;
        o.face_table_waves = P.face_groups > 0 ? P.face_waves / P.face_groups : 0;
        o.gather_waves = P.gather_groups > 0 ? P.gather_waves / P.gather_groups : 0;
    }
    o.violations = P.violations;
    *info = o;
    if (P.violations) fail(FVLBM_OK, "%lld failed plan checks; first: %s", (long long)P.violations,
                           P.first_violation.c_str());
    return FVLBM_OK;
}

static int init_impl(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params, void* stream,
                     void* workspace, size_t workspace_bytes, fvlbm_solver* s) {
    const Mesh& M = mesh->m;
    int rc = check_params(M, params, n_params);
    if (rc) return rc;
    const fvlbm_params& p0 = params[0];
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(FVLBM_ERR_UNSUPPORTED, "fvlbm_init: no CUDA device");
    if (p0.device < 0 || p0.device >= ndev) return fail(FVLBM_ERR_ARG, "fvlbm_init: device %d out of range", p0.device);
    DeviceGuard dg(p0.device);
    s->device = p0.device;
    s->stream = (cudaStream_t)stream;
    s->prec = p0.precision;
    s->scheme = p0.scheme;
    s->n_cell = M.n_owned;
    s->n_inst = M.n_inst;
    s->inst_begin = M.inst_begin;
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, p0.device) != cudaSuccess) {
        cudaGetLastError();
        pageable = 0;
    }
    s->host_can_direct = pageable == 1;
    s->host_direct = s->host_can_direct;

    // per-instance constants and the time step of Eqs. (CFL), (timetau)
    s->inst.resize(M.n_inst);
    for (int32_t k = 0; k < M.n_inst; k++) {
        const fvlbm_params& p = params[n_params == 1 ? 0 : k];
        InstParam& I = s->inst[k];
        std::memset(&I, 0, sizeof I);
        const double umax = instance_umax(M, k, p);
        double dt = p.dt > 0 ? p.dt : suggest_dt(M, k, p.tau, p.cfl > 0 ? p.cfl : 0.5, umax, p.scheme);
        const double cap = p.scheme == FVLBM_AB2 ? p.tau : 2.0 * p.tau;
        if (dt > cap * (1 + 1e-12))
            return fail(FVLBM_ERR_UNSTABLE_DT, "instance %d: dt = %g exceeds the collision limit %g", k, dt, cap);
        const double cfl = dt * (std::sqrt(2.0) + umax) / M.inst_cfl_len[k];
        if (cfl > 1.0 + 1e-12)
            return fail(FVLBM_ERR_UNSTABLE_DT, "instance %d: dt = %g gives CFL %g > 1", k, dt, cfl);
        I.tau = p.tau;
        I.inv_tau = 1.0 / p.tau;
        I.dt = dt;
        I.inv_tau_f = (float)I.inv_tau;
        I.dt_f = (float)dt;
        I.rho0 = p.rho0;
        I.u0x = p.u0[0];
        I.u0y = p.u0[1];
        for (int a = 0; a < FVLBM_Q; a++) {
            float sc = 1.0f;
            if (p.precision == FVLBM_FP16_DEV) {
                // power-of-two scale of the stored non-equilibrium part: an
                // estimate of |g_a - g^eq_a| from the size of the equilibrium
                // deviation maps to ~2^5, 2^11 below FP16's largest finite value:
                // the non-equilibrium part grows like tau |e . grad f^eq|, and
                // near the lid corners of a Re 10 cavity it reached 17 times the
                // estimate (with the estimate at ~2^12 such values saturated).
                // FP16 precision is relative down to 2^-14 (6e-5); below, the
                // step stays 2^-24 / scale (~2e-10 of n here)
                const double w = a == 0 ? 4.0 / 9 : (a < 5 ? 1.0 / 9 : 1.0 / 36);
                const double e = a == 0 ? 0.0 : (a < 5 ? 1.0 : std::sqrt(2.0));
                const double U = std::max(umax, 1e-3);
                const double gmax = w * (0.1 + 2.2 * (3 * e * U + 4.5 * e * e * U * U + 1.5 * U * U));
                sc = std::ldexp(1.0f, (int)std::floor(std::log2(32.0 / gmax)));
            }
            I.scale[a] = sc;
            I.inv_scale[a] = 1.0f / sc;
        }
    }

    // layout, workspace
    Layout L;
    try {
        rc = make_layout(M, s->prec, s->scheme, p0.kernel, L, device_sms(p0.device));
    } catch (const std::bad_alloc&) {
        return fail(FVLBM_ERR_OOM, "fvlbm_init: out of host memory");
    }
    if (rc) return rc;
    if (workspace) {
        if (workspace_bytes < L.total)
            return fail(FVLBM_ERR_OOM, "fvlbm_init: workspace of %zu bytes, %zu needed", workspace_bytes, L.total);
        if ((uintptr_t)workspace % ALIGN) return fail(FVLBM_ERR_ARG, "fvlbm_init: workspace not 256-byte aligned");
        s->ws = workspace;
        s->own_ws = false;
    } else {
        cudaError_t e = cudaMalloc(&s->ws, L.total);
        if (e != cudaSuccess) {
            s->ws = nullptr;
            return fail(FVLBM_ERR_OOM, "fvlbm_init: cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e));
        }
        s->own_ws = true;
    }
    s->ws_bytes = L.total;

    // host image of the read-only part (geometry, params, chunk table)
    std::vector<unsigned char> host;
    try {
        host.assign(L.off_fa, 0);
        if (s->prec == FVLBM_FP64) pack_geometry<double>(M, L, host);
        else pack_geometry<float>(M, L, host);
        if (L.strategy == STRATEGY_TILE) {
            std::memcpy(host.data() + L.off_tbegin, L.tp.begin.data(), 8 * L.tp.begin.size());
            std::memcpy(host.data() + L.off_hptr, L.tp.halo_ptr.data(), 8 * L.tp.halo_ptr.size());
            std::memcpy(host.data() + L.off_halo, L.tp.halo.data(), 4 * L.tp.halo.size());
            std::memcpy(host.data() + L.off_r1ptr, L.tp.r1_ptr.data(), 8 * L.tp.r1_ptr.size());
        }
    } catch (const std::bad_alloc&) {
        return fail(FVLBM_ERR_OOM, "fvlbm_init: out of host memory");
    }
    std::memcpy(host.data() + L.off_inst, s->inst.data(), sizeof(InstParam) * M.n_inst);
    BcParam* bcp = (BcParam*)(host.data() + L.off_bc);
    for (size_t b = 0; b < M.bcs.size(); b++) {
        const fvlbm_bc& c = M.bcs[b];
        BcParam& q = bcp[b];
        q.kind = c.kind == FVLBM_BC_WALL ? SK_WALL : c.kind == FVLBM_BC_INLET ? SK_INLET
               : c.kind == FVLBM_BC_OUTLET ? SK_OUTLET : c.kind == FVLBM_BC_SYMMETRY ? SK_SYMMETRY : SK_NONE;
        q.external = c.external;
        q.uwx = c.u_w[0];
        q.uwy = c.u_w[1];
        q.rho_inf = c.rho_inf;
        q.uix = c.u_inf[0];
        q.uiy = c.u_inf[1];
        q.uwx_f = (float)q.uwx;
        q.uwy_f = (float)q.uwy;
        q.rho_f = (float)q.rho_inf;
        q.rdev_f = (float)(q.rho_inf - 1.0);
        q.uix_f = (float)q.uix;
        q.uiy_f = (float)q.uiy;
    }
    std::vector<int64_t> chunks;
    for (int32_t k = 0; k < M.n_inst; k++)
        for (int64_t b = M.inst_begin[k]; b < M.inst_begin[k + 1]; b += CHUNK)
            chunks.insert(chunks.end(), {b, std::min(b + CHUNK, M.inst_begin[k + 1]), (int64_t)k});

    unsigned char* base = (unsigned char*)s->ws;
    CK(cudaMemcpyAsync(base, host.data(), L.off_fa, cudaMemcpyHostToDevice, s->stream), "upload geometry");
    CK(cudaMemcpyAsync(base + L.off_chunk, chunks.data(), chunks.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                       s->stream), "upload chunk table");
    // face values start at zero: directions parallel to a face (e.n = 0) are never written
    if (L.strategy == STRATEGY_TWO_KERNEL)
        CK(cudaMemsetAsync(base + L.off_fv, 0,
                           real_size(s->prec) * (size_t)std::max<int64_t>(1, L.n_face) * (FVLBM_Q - 1), s->stream),
           "clear face values");
    CK(cudaMemsetAsync(base + L.off_flag, 0, 16, s->stream), "clear flag");

    DevView& v = s->v;
    v.n_cell = M.n_owned;
    v.n_grad = M.n_grad;
    v.np = L.np;
    v.n_face = L.n_face;
    v.maxf = L.maxf;
    v.n_inst = M.n_inst;
    v.desc = (const uint2*)(base + L.off_desc);
    v.geo = base + L.off_geo;
    v.nbr = (const int32_t*)(base + L.off_nbr);
    v.area = (const double*)(base + L.off_area);
    v.grp = (const int32_t*)(base + L.off_grp);
    v.iperm = (const int32_t*)(base + L.off_iperm);
    v.inst = (const InstParam*)(base + L.off_inst);
    v.bc = (const BcParam*)(base + L.off_bc);
    v.fa = base + L.off_fa;
    v.fb = L.off_fb ? base + L.off_fb : nullptr;
    v.rprev = L.off_rprev ? base + L.off_rprev : nullptr;
    v.fv = base + L.off_fv;
    v.rho = (double*)(base + L.off_rho);
    v.ux = (double*)(base + L.off_ux);
    v.uy = (double*)(base + L.off_uy);
    v.uold = (double*)(base + L.off_uold);
    v.part = (double*)(base + L.off_part);
    v.red = (double*)(base + L.off_red);
    v.conv = (double*)(base + L.off_conv);
    v.chunk = (const int64_t*)(base + L.off_chunk);
    v.n_chunk = (int64_t)chunks.size() / 3;
    v.flag = (int32_t*)(base + L.off_flag);
    v.strategy = L.strategy;
    v.block = L.block;
    if (L.strategy == STRATEGY_TILE) {
        v.tile = L.tp.tile;
        v.sms = device_sms(p0.device);
        v.n_tiles = L.tp.n_tiles;
        v.tile_begin = (const int64_t*)(base + L.off_tbegin);
        v.halo_ptr = (const int64_t*)(base + L.off_hptr);
        v.halo = (const int32_t*)(base + L.off_halo);
        v.r1_ptr = (const int64_t*)(base + L.off_r1ptr);
        v.r1link = (const uint32_t*)(base + L.off_r1link);
    }
    s->pingpong = L.pingpong;
    s->buf[0] = v.fa;
    s->buf[1] = v.fb;
    s->fc = L.off_fc ? base + L.off_fc : nullptr;
    s->cur = 0;

    // Step 0 and the first residual snapshot
    rc = launch_init_eq(v, s->prec, s->stream);
    if (rc) return rc;
    rc = launch_macros(v, s->prec, s->stream);
    if (rc) return rc;
    CK(cudaMemcpyAsync(v.uold, v.ux, 8 * L.np, cudaMemcpyDeviceToDevice, s->stream), "snapshot u");
    CK(cudaMemcpyAsync(v.uold + L.np, v.uy, 8 * L.np, cudaMemcpyDeviceToDevice, s->stream), "snapshot v");
    CK(cudaStreamSynchronize(s->stream), "fvlbm_init");
    return FVLBM_OK;
}

extern "C" void fvlbm_solver_destroy(fvlbm_solver* s) {
    if (!s) return;
    for (int b = 0; b < 2; b++) {
        if (s->g1[b]) cudaGraphExecDestroy(s->g1[b]);
        if (s->gk[b]) cudaGraphExecDestroy(s->gk[b]);
    }
    if (s->own_ws && s->ws) {
        DeviceGuard dg(s->device);
        cudaStreamSynchronize(s->stream);
        cudaFree(s->ws);
    }
    delete s;
}

extern "C" int fvlbm_init(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params, void* stream,
                          void* workspace, size_t workspace_bytes, fvlbm_solver** out) {
    clear_error();
    if (!mesh || !out) return fail(FVLBM_ERR_ARG, "fvlbm_init: null argument");
    *out = nullptr;
    fvlbm_solver* s = new (std::nothrow) fvlbm_solver;
    if (!s) return fail(FVLBM_ERR_OOM, "fvlbm_init: out of host memory");
    int rc = init_impl(mesh, params, n_params, stream, workspace, workspace_bytes, s);
    if (rc != FVLBM_OK) {
        fvlbm_solver_destroy(s);
        return rc;
    }
    *out = s;
    return FVLBM_OK;
}

// Stages per time step of each scheme.
static int n_stages(int scheme) { return scheme == FVLBM_RK2 ? 2 : scheme == FVLBM_RK4 ? 4 : 1; }

// Make buf[c] the current state (v.fa) and the other buffer v.fb.
static void set_current(fvlbm_solver* s, int c) {
    s->cur = c;
    s->v.fa = s->buf[c];
    s->v.fb = s->buf[c ^ 1];
}

// Enqueue stage k of one time step (0 <= k < n_stages).  ev: null, or 3
// events (see launch_stage).  *out (if not null): the buffer the stage writes.
// The last stage of a single-stage scheme also ends the step (AB2 history,
// alternating state).
static int enqueue_stage(fvlbm_solver* s, int k, void* const* ev, void** out) {
    const DevView& v = s->v;
    void* dst = nullptr;
    int rc = FVLBM_OK;
    switch (s->scheme) {
        case FVLBM_EULER:
        case FVLBM_AB2: {
            const int mode = s->scheme == FVLBM_EULER ? MODE_RK : (s->ab2_started ? MODE_AB2 : MODE_AB2_FIRST);
            // in place on the two-kernel stage (each cell reads only its own state
            // after the face values are written); fa -> fb and swap on the fused stage
            dst = s->pingpong ? v.fb : v.fa;
            rc = launch_stage(v, s->prec, s->stream, v.fa, v.fa, dst, 1.0, mode, ev);
            if (rc) return rc;
            if (s->scheme == FVLBM_AB2) s->ab2_started = true;
            if (s->pingpong) set_current(s, s->cur ^ 1);
            break;
        }
        case FVLBM_RK2:
            dst = k == 0 ? v.fb : v.fa;
            rc = launch_stage(v, s->prec, s->stream, k == 0 ? v.fa : v.fb, v.fa, dst, k == 0 ? 0.5 : 1.0, MODE_RK, ev);
            break;
        case FVLBM_RK4: {
            static const double beta[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
            // fa -> fb -> fb -> fb -> fa, or with a third buffer fa -> fb -> fc -> fb -> fa
            void* const in[4] = {v.fa, v.fb, s->fc ? s->fc : v.fb, v.fb};
            void* const o[4] = {v.fb, s->fc ? s->fc : v.fb, v.fb, v.fa};
            dst = o[k];
            rc = launch_stage(v, s->prec, s->stream, in[k], v.fa, dst, beta[k], MODE_RK, ev);
            break;
        }
        default:
            return fail(FVLBM_ERR_ARG, "bad scheme");
    }
    if (out) *out = dst;
    return rc;
}

// Enqueue one time step.  ev: null, or 3 events per stage (see launch_stage).
static int enqueue_step(fvlbm_solver* s, void* const* ev = nullptr) {
    const int ns = n_stages(s->scheme);
    for (int k = 0; k < ns; k++) {
        int rc = enqueue_stage(s, k, ev ? ev + 3 * k : ev, nullptr);
        if (rc) return rc;
    }
    return FVLBM_OK;
}

extern "C" int fvlbm_profile(fvlbm_solver* s, int64_t n, double* avg_ms, int32_t max_kinds, int32_t* n_kinds,
                             int64_t* launches) {
    clear_error();
    if (!s || n <= 0 || !avg_ms || max_kinds < STAGE_KERNELS || !n_kinds || !launches)
        return fail(FVLBM_ERR_ARG, "fvlbm_profile: bad arguments");
    DeviceGuard dg(s->device);
    const int ns = n_stages(s->scheme);
    std::vector<cudaEvent_t> ev((size_t)3 * ns * n, nullptr);
    int rc = FVLBM_OK;
    for (auto& e : ev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            e = nullptr;
            rc = cuda_fail(ce, "fvlbm_profile: event");
            break;
        }
    }
    for (int64_t k = 0; k < n && rc == FVLBM_OK; k++) rc = enqueue_step(s, (void* const*)&ev[(size_t)3 * ns * k]);
    if (rc == FVLBM_OK) {
        cudaError_t ce = cudaStreamSynchronize(s->stream);
        if (ce != cudaSuccess) rc = cuda_fail(ce, "fvlbm_profile: synchronise");
    }
    if (rc == FVLBM_OK) {
        double t[STAGE_KERNELS] = {0, 0};
        for (size_t q = 0; q < ev.size(); q += 3) {
            float a = 0, b = 0;
            cudaEventElapsedTime(&a, ev[q], ev[q + 1]);
            cudaEventElapsedTime(&b, ev[q + 1], ev[q + 2]);
            t[0] += a;
            t[1] += b;
        }
        const double launches_per_kind = (double)ns * n;
        const int kinds = stage_kernels(s->v);
        for (int q = 0; q < kinds; q++) avg_ms[q] = t[q] / launches_per_kind;
        *n_kinds = kinds;
        *launches = (int64_t)kinds * ns * n;
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    return rc;
}

extern "C" int fvlbm_launches_per_step(const fvlbm_solver* s, int64_t* launches) {
    clear_error();
    if (!s || !launches) return fail(FVLBM_ERR_ARG, "fvlbm_launches_per_step: null argument");
    *launches = (int64_t)stage_kernels(s->v) * n_stages(s->scheme);
    return FVLBM_OK;
}

// Capture `nsteps` steps of the solver's stream into an executable graph.
// Capture only records launches: the host-side state (current buffer, AB2
// start) is put back afterwards.
static bool build_graph(fvlbm_solver* s, int64_t nsteps, cudaGraphExec_t* out) {
    const int cur0 = s->cur;
    const bool ab2 = s->ab2_started;
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int rc = FVLBM_OK;
    for (int64_t k = 0; k < nsteps && rc == FVLBM_OK; k++) rc = enqueue_step(s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    set_current(s, cur0);
    s->ab2_started = ab2;
    bool ok = rc == FVLBM_OK && e == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(out, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        *out = nullptr;
        cudaGetLastError();
        clear_error();
    }
    return ok;
}

// Steps are replayed from CUDA graphs (chunks of GRAPH_CHUNK, then single
// steps) once the solver has run directly at least once (so that kernel
// attributes are set outside capture) and AB2 has its history; the legacy
// default stream cannot be captured and always launches directly.  With a
// ping-pong state there is one pair of graphs per starting buffer (a chunk
// has an even number of steps and ends where it started).
extern "C" int fvlbm_step(fvlbm_solver* s, int64_t n) {
    clear_error();
    if (!s || n < 0) return fail(FVLBM_ERR_ARG, "fvlbm_step: bad arguments");
    DeviceGuard dg(s->device);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s->stream, &cs);
    bool graphs = s->graphs_ok && s->stream != nullptr && cs == cudaStreamCaptureStatusNone &&
                  s->direct_steps > 0 && (s->scheme != FVLBM_AB2 || s->ab2_started);
    auto ready = [&](int b) {
        if (s->g1[b]) return true;
        if (!build_graph(s, 1, &s->g1[b]) || !build_graph(s, GRAPH_CHUNK, &s->gk[b])) {
            s->graphs_ok = false;
            return false;
        }
        return true;
    };
    while (n > 0) {
        if (graphs && !ready(s->cur)) graphs = false;
        int rc = FVLBM_OK;
        if (graphs && n >= GRAPH_CHUNK) {
            cudaError_t e = cudaGraphLaunch(s->gk[s->cur], s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "fvlbm_step: graph launch");
            n -= GRAPH_CHUNK;
            continue;
        }
        if (graphs) {
            cudaError_t e = cudaGraphLaunch(s->g1[s->cur], s->stream);
            rc = e == cudaSuccess ? FVLBM_OK : cuda_fail(e, "fvlbm_step: graph launch");
            if (rc == FVLBM_OK && s->pingpong) set_current(s, s->cur ^ 1);
        } else {
            rc = enqueue_step(s);
            s->direct_steps++;
        }
        if (rc) return rc;
        n--;
    }
    return FVLBM_OK;
}

static int sync_and_check(fvlbm_solver* s) {
    int32_t flag = 0;
    CK(cudaMemcpyAsync(&flag, s->v.flag, sizeof flag, cudaMemcpyDeviceToHost, s->stream), "read flag");
    CK(cudaStreamSynchronize(s->stream), "synchronise");
    if (flag) return fail(FVLBM_ERR_DIVERGED, "a non-finite value appeared in the state");
    return FVLBM_OK;
}

namespace fvlbm {
int solver_ref(fvlbm_solver* s, SolverRef* out) {
    if (!s || !out) return fail(FVLBM_ERR_ARG, "null solver");
    out->view = &s->v;
    out->prec = s->prec;
    out->device = s->device;
    out->stream = s->stream;
    out->n_inst = s->n_inst;
    return FVLBM_OK;
}
int solver_sync_check(fvlbm_solver* s) { return sync_and_check(s); }
}  // namespace fvlbm

extern "C" int fvlbm_sync(fvlbm_solver* s) {
    clear_error();
    if (!s) return fail(FVLBM_ERR_ARG, "fvlbm_sync: null solver");
    DeviceGuard dg(s->device);
    return sync_and_check(s);
}

extern "C" int fvlbm_macros(fvlbm_solver* s, double* rho, double* u) {
    clear_error();
    if (!s) return fail(FVLBM_ERR_ARG, "fvlbm_macros: null solver");
    DeviceGuard dg(s->device);
    // caller order in the device staging buffer, then one copy per output
    // (device -> host always staged; see fvlbm_host_transfer)
    double* d_rho = s->v.conv;
    double* d_u = s->v.conv + s->n_cell;
    int rc = launch_macros_ordered(s->v, s->prec, s->stream, rho ? d_rho : nullptr, u ? d_u : nullptr);
    if (rc) return rc;
    // cudaMemcpyDefault: the caller's buffer may be host (pageable or pinned) or device memory
    if (rho) CK(cudaMemcpyAsync(rho, d_rho, 8 * (size_t)s->n_cell, cudaMemcpyDefault, s->stream), "read rho");
    if (u) CK(cudaMemcpyAsync(u, d_u, 16 * (size_t)s->n_cell, cudaMemcpyDefault, s->stream), "read u");
    return sync_and_check(s);
}

static int reduce(fvlbm_solver* s, int what, std::vector<double>& out) {
    int rc = launch_macros(s->v, s->prec, s->stream);
    if (rc) return rc;
    rc = launch_reduce(s->v, s->stream, what);
    if (rc) return rc;
    out.assign(3 * (size_t)s->n_inst, 0.0);
    CK(cudaMemcpyAsync(out.data(), s->v.red, out.size() * 8, cudaMemcpyDeviceToHost, s->stream), "read sums");
    return sync_and_check(s);
}

namespace fvlbm {
int solver_n_stages(const fvlbm_solver* s) { return n_stages(s->scheme); }
int solver_stage(fvlbm_solver* s, int k, void** out) {
    if (!s || k < 0 || k >= n_stages(s->scheme)) return fail(FVLBM_ERR_ARG, "solver_stage: bad arguments");
    DeviceGuard dg(s->device);
    return enqueue_stage(s, k, nullptr, out);
}
int solver_sums(fvlbm_solver* s, int what, std::vector<double>& out) {
    DeviceGuard dg(s->device);
    return reduce(s, what, out);
}
}  // namespace fvlbm

extern "C" int fvlbm_residual(fvlbm_solver* s, double* e) {
    clear_error();
    if (!s || !e) return fail(FVLBM_ERR_ARG, "fvlbm_residual: null argument");
    DeviceGuard dg(s->device);
    std::vector<double> r;
    int rc = reduce(s, RED_RESIDUAL, r);
    if (rc) return rc;
    for (int32_t k = 0; k < s->n_inst; k++) {
        const double num = r[3 * k], den = r[3 * k + 1];
        e[k] = den == 0 ? (num == 0 ? 0.0 : INFINITY) : std::sqrt(num) / std::sqrt(den);
    }
    return FVLBM_OK;
}

extern "C" int fvlbm_mass(fvlbm_solver* s, double* mass) {
    clear_error();
    if (!s || !mass) return fail(FVLBM_ERR_ARG, "fvlbm_mass: null argument");
    DeviceGuard dg(s->device);
    std::vector<double> r;
    int rc = reduce(s, RED_MASS, r);
    if (rc) return rc;
    for (int32_t k = 0; k < s->n_inst; k++) mass[k] = r[3 * k];
    return FVLBM_OK;
}

extern "C" int fvlbm_get_f(fvlbm_solver* s, double* f) {
    clear_error();
    if (!s || !f) return fail(FVLBM_ERR_ARG, "fvlbm_get_f: null argument");
    DeviceGuard dg(s->device);
    // caller order in the device staging buffer, then one copy (device -> host
    // always staged; see fvlbm_host_transfer)
    int rc = launch_get_f_ordered(s->v, s->prec, s->stream, s->v.conv);
    if (rc) return rc;
    CK(cudaMemcpyAsync(f, s->v.conv, 8 * (size_t)s->n_cell * FVLBM_Q, cudaMemcpyDefault, s->stream), "read f");
    return sync_and_check(s);
}

extern "C" int fvlbm_set_f(fvlbm_solver* s, const double* f) {
    clear_error();
    if (!s || !f) return fail(FVLBM_ERR_ARG, "fvlbm_set_f: null argument");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream), "synchronise");
    int rc;
    if (s->host_direct) {
        rc = launch_set_f_ordered(s->v, s->prec, s->stream, f);
    } else {
        // staged: one copy of the caller's buffer into the device staging buffer
        CK(cudaMemcpyAsync(s->v.conv, f, 8 * (size_t)s->n_cell * FVLBM_Q, cudaMemcpyDefault, s->stream), "write f");
        rc = launch_set_f_ordered(s->v, s->prec, s->stream, s->v.conv);
    }
    if (rc) return rc;
    s->ab2_started = false;
    if (s->scheme == FVLBM_AB2) s->direct_steps = 0;   // the next step is an Euler start, launched directly
    CK(cudaStreamSynchronize(s->stream), "synchronise");
    return FVLBM_OK;
}

extern "C" int fvlbm_stage_kernel(const fvlbm_solver* s, int32_t* kernel) {
    clear_error();
    if (!s || !kernel) return fail(FVLBM_ERR_ARG, "fvlbm_stage_kernel: null argument");
    *kernel = s->v.strategy == STRATEGY_TILE ? s->v.tile : 1;
    return FVLBM_OK;
}

extern "C" int fvlbm_host_transfer(fvlbm_solver* s, int32_t mode, int32_t* direct) {
    clear_error();
    if (!s || (mode != FVLBM_HOST_AUTO && mode != FVLBM_HOST_STAGED))
        return fail(FVLBM_ERR_ARG, "fvlbm_host_transfer: bad arguments");
    s->host_direct = mode == FVLBM_HOST_AUTO && s->host_can_direct;
    if (direct) *direct = s->host_direct ? 1 : 0;
    return FVLBM_OK;
}

extern "C" int fvlbm_get_dt(const fvlbm_solver* s, int32_t instance, double* dt) {
    clear_error();
    if (!s || !dt || instance < 0 || instance >= s->n_inst) return fail(FVLBM_ERR_ARG, "fvlbm_get_dt: bad arguments");
    *dt = s->inst[instance].dt;
    return FVLBM_OK;
}

extern "C" int fvlbm_autotune(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params, void* stream,
                              int32_t steps, int32_t* best_kernel, double* ms_per_step) {
    clear_error();
    if (!mesh || !params || n_params <= 0 || steps <= 0 || !best_kernel)
        return fail(FVLBM_ERR_ARG, "fvlbm_autotune: bad arguments");
    static const int32_t cand[5] = {1, 128, 256, 512, 1024};
    constexpr int REPEATS = 5;
    std::vector<fvlbm_params> p(params, params + n_params);
    double med[5];
    // the automatic choice (params.kernel = 0) for this mesh
    int32_t automatic = 0;
    {
        Layout L;
        if (make_layout(mesh->m, params[0].precision, params[0].scheme, 0, L, device_sms(params[0].device)) == FVLBM_OK)
            automatic = L.strategy == STRATEGY_TILE ? L.tp.tile : 1;
        clear_error();
    }
    for (int c = 0; c < 5; c++) {
        med[c] = INFINITY;
        for (auto& q : p) q.kernel = cand[c];
        fvlbm_solver* sv = nullptr;
        int rc = fvlbm_init(mesh, p.data(), n_params, stream, nullptr, 0, &sv);
        if (rc == FVLBM_ERR_UNSUPPORTED || rc == FVLBM_ERR_OOM) continue;   // variant does not fit
        if (rc) return rc;
        DeviceGuard dg(sv->device);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        rc = fvlbm_step(sv, 3);   // warm-up: direct launches, then the graphs are built
        if (!rc) rc = fvlbm_sync(sv);
        if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
            rc = fail(FVLBM_ERR_CUDA, "fvlbm_autotune: events");
        double t[REPEATS];
        for (int r = 0; r < REPEATS && !rc; r++) {
            float ms = 0;
            cudaEventRecord(e0, sv->stream);
            rc = fvlbm_step(sv, steps);
            cudaEventRecord(e1, sv->stream);
            if (!rc) rc = fvlbm_sync(sv);
            if (!rc) cudaEventElapsedTime(&ms, e0, e1);
            t[r] = ms / steps;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        fvlbm_solver_destroy(sv);
        if (rc) return rc;
        std::sort(t, t + REPEATS);
        med[c] = t[REPEATS / 2];
    }
    int best = -1;
    for (int c = 0; c < 5; c++)
        if (std::isfinite(med[c]) && (best < 0 || med[c] < med[best])) best = c;
    if (best < 0) return fail(FVLBM_ERR_UNSUPPORTED, "fvlbm_autotune: no stage kernel variant fits");
    // timing noise must not flip the choice between variants that are as fast:
    // among those within 3% (or 2 microseconds per step, the launch jitter that
    // small meshes see) of the fastest median, the automatic choice wins, else
    // the first in a fixed order
    static const int32_t pref[5] = {512, 256, 128, 1024, 1};
    const double lim = std::max(1.03 * med[best], med[best] + 0.002);
    int pick = -1;
    for (int c = 0; c < 5; c++)
        if (cand[c] == automatic && med[c] <= lim) pick = c;
    for (int q = 0; q < 5 && pick < 0; q++)
        for (int c = 0; c < 5; c++)
            if (cand[c] == pref[q] && med[c] <= lim) pick = c;
    best = pick;
    if (ms_per_step)
        for (int c = 0; c < 5; c++) ms_per_step[c] = med[c];
    *best_kernel = cand[best];
    return FVLBM_OK;
}
