// Internal declarations shared by the host side (mesh, solver) and the CUDA
// kernels of the library.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include <cuda_runtime_api.h>
#include <vector_types.h>

#include "fvlbm.h"

namespace fvlbm {

// Makes device d current for the guard's scope and restores the caller's
// device afterwards (also when the caller's device could not be read: then the
// device is left as the scope set it, as no previous one is known).
struct DeviceGuard {
    int prev = -1;
    bool ok = true;   // device d is current
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != d && cudaSetDevice(d) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// ---------------------------------------------------------------- errors
// Records a message for fvlbm_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
void clear_error();

// ---------------------------------------------------------------- mesh (host, FP64)
// Face-slot kinds as the kernels see them.
enum SlotKind : uint32_t {
    SK_NONE = 0,      // unused slot (cell has fewer faces)
    SK_INTERIOR = 1,  // interior or periodic face: neighbour cell across it
    SK_WALL = 2,
    SK_INLET = 3,
    SK_OUTLET = 4,
    SK_SYMMETRY = 5,
};

struct Slot {
    int32_t kind = SK_NONE;  // SlotKind
    int32_t nb = -1;         // neighbour cell (caller numbering of the instance-local mesh)
    int32_t nb_slot = -1;    // the same face's slot inside the neighbour
    int32_t bc = -1;         // boundary tag (boundary slots)
    int32_t periodic = 0;    // 1 if the face is a periodic pair
    double nx = 0, ny = 0;   // outward normal times length: (dy, -dx) of the CCW edge
    double px = 0, py = 0;   // face midpoint
    double sx = 0, sy = 0;   // periodic: neighbour image = neighbour centroid + (sx, sy)
    double cgx = 0, cgy = 0; // least-squares coefficient of this slot's stencil point
    double vx = 0, vy = 0;   // start vertex of the edge (the edge runs to the next slot's)
    double sdx = 0, sdy = 0; // stencil point minus cell centroid
    uint32_t outmask = 0;    // bit a-1 set when e_a . n > 0 (a = 1..8): upwind side is this cell
};

constexpr int MAXP = FVLBM_MAX_POLY;

struct Mesh {
    int64_t n_cell = 0;
    // A part of a partitioned mesh also holds ghost cells: cells [0, n_owned)
    // (the same in both numberings) are the part's own and are updated; cells
    // [n_owned, n_grad) are the first ghost ring (their gradient is recomputed
    // from local data), [n_grad, n_cell) the second (state only).  A whole
    // mesh has n_owned = n_grad = n_cell.
    int64_t n_owned = 0, n_grad = 0;
    int32_t max_faces = 0;
    int32_t n_inst = 1;
    std::vector<int64_t> inst_begin;     // [n_inst + 1] cell ranges (same in both numberings)
    std::vector<int32_t> inst_bc_begin;  // [n_inst + 1] ranges of bcs
    std::vector<fvlbm_bc> bcs;           // all boundary tags (global numbering)
    std::vector<double> inst_cfl_len;    // [n_inst] min A/(Lx+Ly)
    std::vector<int32_t> nf;             // [n_cell] faces per cell
    std::vector<double> area, cx, cy;    // [n_cell]
    std::vector<Slot> slots;             // [n_cell * MAXP]; nb is a global caller index
    std::vector<int64_t> perm;           // internal -> caller
    std::vector<int64_t> iperm;          // caller -> internal
    int64_t n_face = 0, n_bface = 0, n_periodic = 0;
    double total_area = 0;
};

// ---------------------------------------------------------------- device view
// Per-instance constants read by the kernels.
struct InstParam {
    double tau, inv_tau, dt;
    float inv_tau_f, dt_f;
    float scale[FVLBM_Q];      // 16-bit split storage: stored = (g_a - g^eq_a) * scale
    float inv_scale[FVLBM_Q];
    double rho0, u0x, u0y;
};

// Per-boundary-tag constants read by the kernels.
struct BcParam {
    int32_t kind;      // SlotKind of the tag
    int32_t external;
    double uwx, uwy, rho_inf, uix, uiy;
    // the same rounded to FP32 on the host (rdev_f = rho_inf - 1 in FP64,
    // then rounded), so that FP32 kernels do no FP64 arithmetic
    float uwx_f, uwy_f, rho_f, rdev_f, uix_f, uiy_f;
};

// Per-cell arrays on the device are blocked: 32 consecutive cells per block,
// each component of the block contiguous (see blk_index in fvlbm_device.cuh).
constexpr int BLK_SHIFT = 5;
constexpr int BLK = 1 << BLK_SHIFT;

// Fused stage: shared-memory capacity of a tile of TILE threads (compile-time
// strides, so that every shared-memory access is a fixed offset from one
// index): LS local cells (tile, 1-ring, 2-ring), FS local faces (the faces of
// the tile's cells) and the instance id of each tile cell; reals of RSIZE
// bytes.  The tile planner ends a tile early when it would not fit.
template <int TILE, int MAXF, int RSIZE> struct TileDims {
    static constexpr int LS = (3 * TILE) / 2 + 64;
    static constexpr int FS = MAXF <= 4 ? 2 * TILE : (7 * TILE) / 2;
    static constexpr size_t BYTES =
        (size_t)RSIZE * ((size_t)FVLBM_Q * LS + (size_t)(FVLBM_Q - 1) * FS) + (size_t)4 * TILE;
};
// "no local face / neighbour" in a 16-bit link field
constexpr uint32_t LINK_NONE = 0xFFFF;

// Device pointers of one solver (all inside one workspace).
struct DevView {
    int64_t n_cell;     // cells updated (internal numbering 0..n_cell-1): the owned cells
    int64_t n_grad;     // cells whose gradient the two-kernel stage computes (owned + first ghost ring)
    int64_t np;         // padded cell count (multiple of the largest tile)
    int64_t n_face;     // face-value table length (two-kernel stage)
    int32_t maxf;       // slots per cell in the packed arrays (4 or 8)
    int32_t n_inst;
    // geometry, blocked per cell, [maxf] (desc) and [3 maxf] (geo) components
    const uint2* desc;  // x: kind | outmask << 8 | bc << 16;  y: link (see below)
    const void* geo;    // T2 [3 maxf]: least-squares coefficients, face midpoint - centroid,
                        //              face vector / area of each slot
    // two-kernel stage: desc.y = face id; nbr = neighbour cell, blocked [maxf]
    const int32_t* nbr;
    const double* area;    // [np]
    const int32_t* grp;    // [np] instance of each cell
    const int32_t* iperm;  // [n_cell] internal index of each cell in the caller's order
    const InstParam* inst; // [n_inst]
    const BcParam* bc;     // [n_bc]
    // state
    void* fa;   // S blocked [9] (or the split format): the state
    void* fb;   // same: stage state (multistage schemes) or the other buffer of a ping-pong pair
    void* rprev;// T [9][np]  AB2 previous RHS
    void* fv;   // T [8][n_face] face values of directions 1..8 (two-kernel stage)
    double* rho;    // [np]
    double* ux;     // [np]
    double* uy;     // [np]
    double* uold;   // [2][np]
    double* part;   // [n_chunk][3] block partial sums
    double* red;    // [n_inst][3]  per-instance sums
    double* conv;   // [9][np] doubles: device staging of get_f / set_f / macros in caller order
    const int64_t* chunk;   // [n_chunk][3] (begin, end, instance)
    int64_t n_chunk;
    int32_t* flag;  // non-finite flag
    // fused stage (one CTA per tile of at most `tile` consecutive cells);
    // desc.y = tile-local neighbour | tile-local face << 16
    int32_t strategy;        // STRATEGY_TWO_KERNEL or STRATEGY_TILE
    int32_t block;           // threads per block of the two-kernel stage
    int32_t tile;            // most cells per tile (threads per CTA)
    int32_t sms;             // streaming multiprocessors of the device
    int64_t n_tiles;
    const int64_t* tile_begin; // [n_tiles + 1] first cell of each tile
    const int64_t* halo_ptr;   // [n_tiles + 1] into halo
    const int32_t* halo;       // 1-ring then 2-ring cells of each tile (global ids)
    const int64_t* r1_ptr;     // [n_tiles + 1] 1-ring entries of each tile (running count)
    const uint32_t* r1link;    // blocked [maxf] over 1-ring entries: local neighbour | local face << 16
};

enum Strategy { STRATEGY_TWO_KERNEL = 0, STRATEGY_TILE = 1 };

// Kernel launchers (fvlbm_kernels.cu).  prec = fvlbm_precision.
int launch_init_eq(const DevView& v, int prec, void* stream);
// ev: null, or 3 cudaEvent_t recorded before the face-value kernel, between
// the two kernels and after the update kernel.
int launch_stage(const DevView& v, int prec, void* stream, const void* fin, const void* fbase,
                 void* fout, double beta, int mode, void* const* ev = nullptr);
// Most kernels launched by one stage (two-kernel strategy).
constexpr int STAGE_KERNELS = 2;
inline int stage_kernels(const DevView& v) { return v.strategy == STRATEGY_TILE ? 1 : 2; }
// One translation unit per state precision.
int stage_fp64(const DevView& v, void* stream, const void* fin, const void* fbase, void* fout, double beta, int mode,
               void* const* ev);
int stage_fp32(const DevView& v, void* stream, const void* fin, const void* fbase, void* fout, double beta, int mode,
               void* const* ev);
int stage_fp16(const DevView& v, void* stream, const void* fin, const void* fbase, void* fout, double beta, int mode,
               void* const* ev);
int stage_bf16(const DevView& v, void* stream, const void* fin, const void* fbase, void* fout, double beta, int mode,
               void* const* ev);
int launch_macros(const DevView& v, int prec, void* stream);
int launch_reduce(const DevView& v, void* stream, int what);
// f and the macros in the caller's cell order, in a buffer the device
// accesses (host memory reachable by the GPU, or device memory).
int launch_get_f_ordered(const DevView& v, int prec, void* stream, double* f);
int launch_set_f_ordered(const DevView& v, int prec, void* stream, const double* f);
int launch_macros_ordered(const DevView& v, int prec, void* stream, double* rho, double* u);

// Solver internals for entry points defined outside the solver's own file.
struct SolverRef {
    const DevView* view;
    int prec;
    int device;
    void* stream;
    int32_t n_inst;
};
int solver_ref(fvlbm_solver* s, SolverRef* out);
// Stages of one time step, and stage k enqueued on the solver's stream (*out:
// the state buffer it writes); the last stage ends the step.
int solver_n_stages(const fvlbm_solver* s);
int solver_stage(fvlbm_solver* s, int k, void** out);
// FP64 sums of a reduction (RED_MASS: [mass, -, -]; RED_RESIDUAL: [numerator,
// denominator, -]) per instance, 3 per instance; synchronises.
int solver_sums(fvlbm_solver* s, int what, std::vector<double>& out);
// Halo exchange of a partitioned solve: entry e = (src part, src internal
// cell, dst part, dst internal cell) copies the stored state of one cell from
// part_state[src] to part_state[dst] (prec = fvlbm_precision of all parts).
int launch_halo_copy(int prec, void* stream, const int4* entries, int64_t n, void* const* part_state, int n_parts);
// Reads the solver's non-finite flag after synchronising its stream.
int solver_sync_check(fvlbm_solver* s);

// Stage modes of launch_stage.
enum StageMode { MODE_RK = 0, MODE_AB2_FIRST = 1, MODE_AB2 = 2 };
// Reductions of launch_reduce.
enum ReduceWhat { RED_MASS = 0, RED_RESIDUAL = 1 };

}  // namespace fvlbm

struct fvlbm_mesh {
    fvlbm::Mesh m;
};

namespace fvlbm {
// One part of a partitioned mesh: its cells (caller numbering of the whole
// mesh) in local order -- owned cells ascending, then ring 1, then ring 2 --
// and its mesh (owned cells followed by the ghosts).
struct PartPlan {
    std::vector<int64_t> cells;
    int64_t n_owned = 0, n_ring1 = 0, n_ring2 = 0;
    fvlbm_mesh* mesh = nullptr;
};
// The cells part `src` sends to part `dst` after every stage: entry e is the
// owned cell src_local[e] of src (local numbering) and the ghost dst_local[e]
// of dst; cells[e] is its number in the whole mesh.
struct HaloMsg {
    int32_t src = -1, dst = -1;
    std::vector<int32_t> src_local, dst_local;
    std::vector<int64_t> cells;
};
}  // namespace fvlbm

struct fvlbm_partition {
    int32_t n_parts = 0;
    int64_t n_cell = 0;
    std::vector<int32_t> owner;            // [n_cell] part owning each cell
    std::vector<fvlbm::PartPlan> parts;
    std::vector<fvlbm::HaloMsg> msgs;      // ordered by (src, dst)
    ~fvlbm_partition();
};
