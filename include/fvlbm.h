/*
 * fvlbm.h -- C ABI of the GB300 finite-volume lattice Boltzmann library.
 *
 * The library advances the D2Q9 discrete Boltzmann-BGK equation on an
 * unstructured 2-D mesh of convex polygons with the cell-centred finite-volume
 * scheme of Wang, Zhong, Cao & Zhuo, "A simplified finite volume lattice
 * Boltzmann method ... Part I" (arXiv:1812.00390):
 *
 *   d f_a / dt = -(1/A) sum_m (e_a . n_m) f_a,m dl_m - (f_a - f_a^eq) / tau
 *                                                         (Sec. 2.2, Eq. rhs)
 *
 * with face values from the least-squares linear upwind reconstruction
 * (Eq. lslrflux, Eq. leastsquare), the boundary treatment of Sec. 2.4
 * (Guo extrapolation at walls, Eq. wallbc; ghost values at inlets, outlets and
 * symmetry planes) and an explicit time scheme (Sec. 2.3).  Every step runs in
 * CUDA kernels for sm_103a; the host side only builds the mesh, packs it and
 * launches.
 *
 * Conventions for every function below:
 *  - Return value: FVLBM_OK (0) or a negative fvlbm_status.  No function
 *    aborts, throws or exits.  fvlbm_last_error() gives a message for the last
 *    failure on the calling thread.
 *  - Pointers marked "host" are plain host memory read (or written) during the
 *    call only; the library copies what it keeps.  The caller keeps ownership.
 *  - Handles are opaque and owned by the library until the matching
 *    *_destroy call.
 *  - Cells are numbered by the caller (0 .. n_cell-1 in the order given to
 *    fvlbm_mesh_create); every array exchanged with the caller uses that order.
 *    Internally the library renumbers cells for locality.
 *  - Distribution functions are indexed a = 0..8 with the D2Q9 velocities of
 *    Sec. 2.1: e_0 = (0,0); e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1);
 *    e_5..e_8 = (1,1),(-1,1),(-1,-1),(1,-1); c = 1, c_s^2 = 1/3.
 */
#ifndef FVLBM_H
#define FVLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FVLBM_Q 9
#define FVLBM_MAX_POLY 8 /* most vertices (and faces) per cell */

typedef enum fvlbm_status {
    FVLBM_OK = 0,
    FVLBM_ERR_ARG = -1,               /* bad argument (null pointer, size, enum) */
    FVLBM_ERR_MESH_TOPOLOGY = -2,     /* edge shared by >2 cells, unmatched periodic edge, ... */
    FVLBM_ERR_DEGENERATE_CELL = -3,   /* non-positive area, or singular least-squares matrix */
    FVLBM_ERR_UNTAGGED_BOUNDARY = -4, /* an edge of one cell only that no boundary edge names */
    FVLBM_ERR_UNSTABLE_DT = -5,       /* dt above 2 tau (Eq. timetau; tau for AB2) or CFL > 1 */
    FVLBM_ERR_OOM = -6,               /* host or device allocation failed, or workspace too small */
    FVLBM_ERR_CUDA = -7,              /* a CUDA runtime call failed */
    FVLBM_ERR_DIVERGED = -8,          /* a non-finite value appeared in the state */
    FVLBM_ERR_TIMEOUT = -9,           /* a bounded wait ran out */
    FVLBM_ERR_UNSUPPORTED = -10       /* combination not built (e.g. no GPU) */
} fvlbm_status;

/* Boundary-condition kinds (Sec. 2.4; periodic as in the Couette case, Sec. 3.1). */
typedef enum fvlbm_bc_kind {
    FVLBM_BC_WALL = 0,     /* no-slip wall moving at u_w, Eq. (wallbc) */
    FVLBM_BC_INLET = 1,    /* ghost f^eq(rho*, u_inf) + f_k - f^eq_k; upwind face value */
    FVLBM_BC_OUTLET = 2,   /* external: f_GC = f_P = f_i; internal: pressure outlet */
    FVLBM_BC_SYMMETRY = 3, /* ghost f^eq(rho_i, u mirrored); face value (f_i + f_GC)/2 */
    FVLBM_BC_PERIODIC = 4  /* edge pairs with the partner tag's edges */
} fvlbm_bc_kind;

typedef enum fvlbm_scheme {
    FVLBM_EULER = 0, /* f^{n+1} = f^n + dt RHS^n, Eq. (euler) */
    FVLBM_RK2 = 1,   /* 2-stage member of the multistage scheme, beta = (1/2, 1) */
    FVLBM_AB2 = 2,   /* Adams-Bashforth, first step Euler (Sec. 2.3) */
    FVLBM_RK4 = 3    /* 4-stage scheme, beta = (1/4, 1/3, 1/2, 1) (Sec. 2.3) */
} fvlbm_scheme;

typedef enum fvlbm_precision {
    FVLBM_FP64 = 0,     /* f stored and computed in FP64 */
    FVLBM_FP32_DEV = 1, /* g = f - w stored and computed in FP32 */
    FVLBM_FP16_DEV = 2, /* split storage: rho - 1 and rho*u in FP32, the non-equilibrium
                           parts n_a = g_a - g_a^eq (a = 3..8) in FP16, each with a power-of-two scale per
                           (instance, a); n_0..n_2 follow from the moment constraints; FP32 math */
    FVLBM_BF16_DEV = 3  /* the same split storage with n_a in BF16; FP32 math */
} fvlbm_precision;

/* One boundary tag.  Boundary edge i uses bcs[btag[i]]. */
typedef struct fvlbm_bc {
    int32_t kind;      /* fvlbm_bc_kind */
    int32_t external;  /* 1: external-flow rules (inlet rho* = rho_inf, outlet f_GC = f_i);
                          0: internal-flow rules (inlet rho* = rho_i, pressure outlet) */
    double u_w[2];     /* wall velocity (FVLBM_BC_WALL); must be tangential to the wall */
    double rho_inf;    /* free-stream density (inlet / outlet) */
    double u_inf[2];   /* free-stream velocity (inlet / outlet) */
    int32_t partner;   /* FVLBM_BC_PERIODIC: tag of the matching boundary */
    int32_t reserved;  /* set to 0 */
    double shift[2];   /* FVLBM_BC_PERIODIC: partner edge points + shift = this edge's points */
} fvlbm_bc;

/* Solver parameters, one set per instance (see fvlbm_init). */
typedef struct fvlbm_params {
    double tau;        /* relaxation time, tau = nu / c_s^2 = 3 nu (Eq. relaxtime, no +1/2) */
    double dt;         /* time step; 0 = choose from Eqs. (CFL) and (timetau) */
    double cfl;        /* CFL number used when dt == 0 (0 = 0.5) */
    double u_max;      /* |U|_max of Eq. (CFL); 0 = largest boundary / initial speed */
    int32_t scheme;    /* fvlbm_scheme; equal for all instances of a solver */
    int32_t precision; /* fvlbm_precision; equal for all instances of a solver */
    double rho0;       /* initial density (Step 0: f = f^eq(rho0, u0)) */
    double u0[2];      /* initial velocity */
    int32_t device;    /* CUDA device ordinal; equal for all instances */
    int32_t kernel;    /* stage kernel: 0 = automatic (FP32 / 16-bit: fused 512-thread tiles
                          from 512 cells per SM, 256-thread tiles from 64, 128-thread tiles
                          below; FP64: two kernels from 32 cells per SM, fused 128-thread
                          tiles below, where one launch per stage matters most);
                          1 = two kernels per stage (face values
                          through memory); 128, 256, 512 or 1024 = one fused kernel per stage
                          with CTAs of that many threads (a tile holds at most that many
                          cells and 1-ring cells together).  Tile sizes whose shared memory
                          exceeds a CTA's (FP64: 1024) give FVLBM_ERR_UNSUPPORTED.  Equal for
                          all instances. */
} fvlbm_params;

typedef struct fvlbm_mesh_info_s {
    int64_t n_cell;        /* cells */
    int64_t n_face;        /* unique faces (interior + periodic pairs + boundary) */
    int64_t n_bface;       /* boundary faces (walls, inlets, outlets, symmetry) */
    int64_t n_periodic;    /* periodic face pairs */
    int32_t max_faces;     /* most faces of one cell */
    int32_t n_instances;   /* independent meshes held (1 unless concatenated) */
    double total_area;     /* sum of cell areas */
    double min_cfl_length; /* min over cells of A / (Lx + Ly), the length of Eq. (CFL) */
} fvlbm_mesh_info_t;

typedef struct fvlbm_mesh fvlbm_mesh;
typedef struct fvlbm_solver fvlbm_solver;

/*
 * Build a mesh (host only, no GPU needed).
 *   xy        host, [n_vert][2] vertex coordinates
 *   cell_ptr  host, [n_cell + 1] offsets into cell_vert (CSR); 3..8 vertices per cell
 *   cell_vert host, vertex indices of each cell, counter-clockwise
 *   bedge     host, [n_bedge][2] boundary edges as vertex pairs (either order)
 *   btag      host, [n_bedge] index into bcs
 *   bcs       host, [n_bc] boundary conditions
 * Interior faces are edges shared by two cells; every edge of one cell only
 * must appear in bedge.  Periodic edges of tag t pair with edges of tag
 * bcs[t].partner whose midpoint plus bcs[t].shift equals their own.
 * Computes in FP64 (Sec. 2.2): areas, centroids, face normals and lengths,
 * least-squares coefficients (Eq. leastsquare), reconstruction vectors
 * (Eq. lslrflux), the upwind side of every face for every direction, and a
 * locality-preserving cell order.
 * Errors: FVLBM_ERR_ARG, _MESH_TOPOLOGY, _DEGENERATE_CELL, _UNTAGGED_BOUNDARY, _OOM.
 */
int fvlbm_mesh_create(const double* xy, int64_t n_vert, const int64_t* cell_ptr,
                      const int32_t* cell_vert, int64_t n_cell, const int32_t* bedge,
                      const int32_t* btag, int64_t n_bedge, const fvlbm_bc* bcs, int32_t n_bc,
                      fvlbm_mesh** out);

/*
 * Concatenate n meshes into one mesh of n independent instances (for a batched
 * solve: one launch advances all of them).  Cells of instance k follow those
 * of instance k-1 in the caller's numbering.  The inputs stay valid and owned
 * by the caller.  Errors: FVLBM_ERR_ARG, _OOM.
 */
int fvlbm_mesh_concat(const fvlbm_mesh* const* meshes, int32_t n, fvlbm_mesh** out);

void fvlbm_mesh_destroy(fvlbm_mesh* mesh);

/* Sizes and CFL length of a mesh.  info: host, written. */
int fvlbm_mesh_info(const fvlbm_mesh* mesh, fvlbm_mesh_info_t* info);

/*
 * Time step of Eqs. (CFL) and (timetau) for instance `instance`:
 *   dt = cfl * min( min_cells(A / (Lx + Ly)) / (sqrt(2) + u_max), 2 tau )
 * (tau in place of 2 tau for AB2, the paper's observed limit).  Lx, Ly are the
 * cell's extents.  The CFL number scales both limits, so neither is met with
 * equality.
 * Writes *dt (host).  Errors: FVLBM_ERR_ARG.
 */
int fvlbm_suggest_dt(const fvlbm_mesh* mesh, int32_t instance, double tau, double cfl,
                     double u_max, int32_t scheme, double* dt);

/*
 * Device bytes fvlbm_init needs when the caller supplies the workspace.
 * params: host, [n_params] as for fvlbm_init.  bytes: host, written.
 */
int fvlbm_workspace_bytes(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params,
                          size_t* bytes);

/*
 * The stage plan fvlbm_init would build (on the host; no GPU needed), checked.
 * The fused stage's tiles are runs of consecutive cells whose state, 1-ring
 * and 2-ring sit in a CTA's shared memory, with a table of the tile's face
 * values (the gradient of Eq. leastsquare and the reconstruction of
 * Eq. lslrflux stay on chip; Sec. 2.4 algorithm Steps 1-5 in one kernel).
 * The check covers what the kernel relies on: every slot names its
 * neighbour's local cell (boundary and unused slots the cell itself, unused
 * slots face row 0), both sides of a face name one face row and no two faces
 * share one, each (face, direction) between local cells has exactly one writer
 * (Sec. 2.4.2: the upwind side), and every tile fits its CTA.  The wavefront
 * figures model the shared-memory bank conflicts of the kernel's warp
 * accesses: the most distinct addresses one of the 32 banks receives, averaged
 * over the accesses (1: conflict-free).
 *   params: host, [n_params] as for fvlbm_init.  info: host, written.
 * A failed check is counted in info->violations and described by
 * fvlbm_last_error(); the call still returns FVLBM_OK.
 * Errors: FVLBM_ERR_ARG, _OOM, _UNSUPPORTED (as fvlbm_workspace_bytes).
 */
typedef struct fvlbm_plan_info_s {
    int32_t stage_kernel;        /* 1: two kernels per stage; else the fused stage's threads per CTA */
    int32_t slots;               /* face slots per cell in the packed arrays (4 or 8) */
    int64_t n_tiles;             /* fused stage: tiles (0 for two kernels) */
    int64_t short_tiles;         /* tiles cut below the CTA size by the shared-memory capacity */
    int32_t max_local_cells;     /* largest tile: its cells, 1-ring and 2-ring */
    int32_t max_faces;           /* largest tile: faces of its cells */
    double mean_tile_cells;      /* cells per tile */
    double mean_ring1_cells;     /* 1-ring cells per tile (gradients recomputed) */
    double mean_local_cells;     /* tile + 1-ring + 2-ring cells per tile */
    double face_table_waves;     /* wavefronts per warp read of the face table (phase 3) */
    double gather_waves;         /* wavefronts per warp gather of neighbour state (phase 2) */
    int64_t violations;          /* failed checks (0) */
} fvlbm_plan_info_t;
int fvlbm_plan_info(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params,
                    fvlbm_plan_info_t* info);

/*
 * Create a solver on params[0].device and set f = f^eq(rho0, u0) (Step 0).
 *   params     host, one entry per instance of the mesh, or one entry for all
 *   n_params   1 or the mesh's instance count
 *   stream     cudaStream_t every kernel and copy of this solver runs on
 *              (NULL = the legacy default stream)
 *   workspace  device memory of at least fvlbm_workspace_bytes bytes, aligned to
 *              256 bytes, owned by the caller and kept alive until
 *              fvlbm_solver_destroy; NULL = the library allocates its own.
 * Uploads the packed geometry (blocking on the stream).
 * Errors: FVLBM_ERR_ARG, _UNSTABLE_DT, _OOM, _CUDA, _UNSUPPORTED.
 */
int fvlbm_init(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params,
               void* stream, void* workspace, size_t workspace_bytes, fvlbm_solver** out);

/*
 * Advance every instance by n time steps (Steps 1-6, Sec. 2.4 algorithm),
 * asynchronously on the solver's stream.  A non-finite value raises a device
 * flag that the next synchronising call reports as FVLBM_ERR_DIVERGED.
 * Errors: FVLBM_ERR_ARG, _CUDA.
 */
int fvlbm_step(fvlbm_solver* s, int64_t n);

/*
 * Macroscopic fields (Step 6): rho = sum f, rho u = sum f e.
 *   rho host [n_cell] (may be NULL), u host [n_cell][2] (may be NULL).
 * Synchronises the stream.  Errors: FVLBM_ERR_ARG, _CUDA, _DIVERGED.
 */
int fvlbm_macros(fvlbm_solver* s, double* rho, double* u);

/*
 * Velocity residual of Sec. 3.2 for each instance,
 *   e = sqrt(sum_i |u_i - u_i^old|^2) / sqrt(sum_i |u_i^old|^2),
 * where u^old is the snapshot taken by the previous call (or by fvlbm_init);
 * then takes a new snapshot.  e = +inf when the snapshot is at rest and the
 * state is not, 0 when both are at rest.  Sums in FP64, in a fixed order.
 *   e host [n_instances].  Synchronises.  Errors: FVLBM_ERR_ARG, _CUDA, _DIVERGED.
 */
int fvlbm_residual(fvlbm_solver* s, double* e);

/* Total mass sum_i A_i rho_i of each instance, FP64.  mass host [n_instances]. */
int fvlbm_mass(fvlbm_solver* s, double* mass);

/*
 * Same result as fvlbm_mass, computed without allocating anything.  The paper
 * has no counterpart; this entry point serves callers that may not allocate
 * memory while they run -- processes whose device memory is reserved up front
 * by another allocator (a framework's caching pool, a fixed serving budget),
 * and real-time loops or plugins that must not touch the device heap.
 *   s     solver (its state and geometry are the inputs)
 *   mass  host [n_instances], written
 * The block partial sums live in a fixed 96 KB array in the library's device
 * memory, not in the solver's workspace.  The array is part of the library's
 * device code: under CUDA's default lazy module loading that code, with the
 * array, is loaded into a device's memory by the first call of this function
 * on that device, which also looks up the array's device address.  The first
 * call on each device may therefore allocate: make it once before the region
 * in which the caller may not allocate, and before any stream capture (with
 * CUDA_MODULE_LOADING=EAGER the array is loaded when the process first uses
 * the device instead).  Every later call allocates nothing.  The array stays
 * on every device it was loaded on until the process exits.
 * Limits: at most 8192 chunks of 4096 cells (33,554,432 cells) and 4096
 * instances per solver; larger solvers get FVLBM_ERR_ARG with the limits in
 * the message.  Every call on a device shares the array, so calls that
 * overlap on the GPU (other threads, other streams) race; serialise them.
 * Nothing carries over from an earlier call.
 * Synchronises the solver's stream.  Errors: FVLBM_ERR_ARG, _CUDA, _DIVERGED.
 */
int fvlbm_mass_noalloc(fvlbm_solver* s, double* mass);

/* Read / write the distribution functions, host [n_cell][9] FP64, caller order.
 * Writing also restarts AB2 history.  Synchronise. */
int fvlbm_get_f(fvlbm_solver* s, double* f);
int fvlbm_set_f(fvlbm_solver* s, const double* f);

/*
 * How fvlbm_set_f reads the caller's buffer.
 *   FVLBM_HOST_AUTO (the default): when the device reports coherent access to
 *     pageable host memory (cudaDevAttrPageableMemoryAccess; GB300 reaches its
 *     Grace host's memory over NVLink-C2C), the kernel reads the caller's
 *     buffer directly, in the caller's cell order, with no staging copy.
 *     Otherwise as FVLBM_HOST_STAGED.
 *   FVLBM_HOST_STAGED: one copy of the caller's buffer into a device staging
 *     buffer in the workspace; the kernel reorders on the device.
 * fvlbm_get_f and fvlbm_macros always write through that staging buffer and
 * one copy: a device write into host pages the process has not touched yet
 * faults each page in over the interconnect (measured ~50x slower into a
 * fresh 480 MB array), and into touched pages the copy is as fast.
 * The buffers passed to those calls may be host memory (malloc, numpy, pinned)
 * or device memory; the calls synchronise before returning, so the caller may
 * reuse them at once.  The results are bitwise the same in both modes.
 * direct: host, optional, written: 1 when fvlbm_set_f reads the caller's
 * buffer directly.  Errors: FVLBM_ERR_ARG.
 */
typedef enum fvlbm_host_mode { FVLBM_HOST_AUTO = 0, FVLBM_HOST_STAGED = 1 } fvlbm_host_mode;
int fvlbm_host_transfer(fvlbm_solver* s, int32_t mode, int32_t* direct);

/* The stage kernel the solver runs (the choice params.kernel = 0 resolved to):
 * 1 for the two-kernel stage, else the fused stage's threads per CTA.
 * kernel: host, written.  Errors: FVLBM_ERR_ARG. */
int fvlbm_stage_kernel(const fvlbm_solver* s, int32_t* kernel);

/* Wait for the solver's stream; reports FVLBM_ERR_DIVERGED if flagged. */
int fvlbm_sync(fvlbm_solver* s);

/* Time step in use for instance k (host, written). */
int fvlbm_get_dt(const fvlbm_solver* s, int32_t instance, double* dt);

/*
 * Measurement aid: run n time steps like fvlbm_step, with a CUDA event pair
 * around every kernel launch, and report the mean device time of each kernel
 * kind in milliseconds.  Fused stage (n_kinds = 1): [0] the stage kernel.
 * Two-kernel stage (n_kinds = 2): [0] face-value kernel (Steps 1-3), [1]
 * update kernel (Steps 4-5).  avg_ms: host [max_kinds] (max_kinds >= 2);
 * n_kinds, launches (kernels launched): host, written.  Synchronises.
 * Errors: FVLBM_ERR_ARG, _CUDA.
 */
int fvlbm_profile(fvlbm_solver* s, int64_t n, double* avg_ms, int32_t max_kinds, int32_t* n_kinds,
                  int64_t* launches);

/*
 * Autotuner: time every stage-kernel variant (params.kernel = 1, 128, 256,
 * 512, 1024; variants that do not fit are skipped) on this mesh and parameters,
 * each in a temporary solver whose workspace the library allocates and frees:
 * 3 warm-up steps, then 5 runs of `steps` steps; a variant's time is the
 * median of the 5.  Reports the fastest, except that among the variants
 * within 3% (or 2 microseconds per step) of the fastest the automatic choice
 * (params.kernel = 0) wins, and else the first of 512, 256, 128, 1024, 1, so
 * that timing noise on small meshes does not flip the pick between equally
 * fast variants.
 *   stream       as for fvlbm_init
 *   best_kernel  host, written: the value to put in fvlbm_params.kernel
 *   ms_per_step  host [5] or NULL: median device ms per step of each variant in
 *                the order above (+inf when skipped)
 * Errors: FVLBM_ERR_ARG, _CUDA, _UNSUPPORTED (no variant fits).
 */
int fvlbm_autotune(const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params, void* stream,
                   int32_t steps, int32_t* best_kernel, double* ms_per_step);

/*
 * Measurement aid: sustained FMA rate of the device, in TFLOP/s (2 flop per
 * FMA), from dependent FMA chains on every SM; fp64 != 0 for FP64, else FP32.
 * Allocates and frees a small buffer.  tflops: host, written.
 */
int fvlbm_fma_peak(int32_t device, int32_t fp64, double* tflops);

/* Kernels one time step launches (host, written). */
int fvlbm_launches_per_step(const fvlbm_solver* s, int64_t* launches);

void fvlbm_solver_destroy(fvlbm_solver* s);

/*
 * Continuous-batching solve server (one GPU).  Requests are queued in arrival
 * order; every fvlbm_server_poll round
 *   1. advances every active request by check_interval time steps (the
 *      residual interval of Sec. 3.2), each request on one of n_streams
 *      streams so that the kernels of different requests overlap;
 *   2. admits queued requests, first fit in arrival order, while fewer than
 *      max_active are active and the device arena (arena_bytes, allocated once
 *      at creation) has a free block for the request's workspace;
 *   3. checks the velocity residual of the requests advanced in step 1 and
 *      retires those with e <= residual_tol or max_steps steps done: rho and u
 *      are copied to host memory and the workspace returns to the arena.
 * A request is an ordinary solver on its own workspace: its result does not
 * depend on the other requests.
 */
typedef struct fvlbm_server fvlbm_server;

typedef struct fvlbm_server_config {
    int32_t device;
    int32_t n_streams;      /* 1..64 */
    size_t arena_bytes;     /* device memory budget for request workspaces */
    int32_t max_active;     /* most requests on the device at once */
    int32_t check_interval; /* time steps between residual checks (the paper uses 1000) */
    double residual_tol;    /* converged when the residual is <= this (e.g. 1e-8) */
    int64_t max_steps;      /* step cap per request */
} fvlbm_server_config;

typedef enum fvlbm_request_state {
    FVLBM_REQ_QUEUED = 0, FVLBM_REQ_ACTIVE = 1, FVLBM_REQ_DONE = 2, FVLBM_REQ_FAILED = 3
} fvlbm_request_state;

typedef struct fvlbm_request_info {
    int32_t state;          /* fvlbm_request_state */
    int32_t status;         /* fvlbm_status of a failed request */
    int64_t steps;          /* time steps done */
    int64_t n_cell;
    double residual;        /* last residual */
    double t_submit, t_admit, t_done;  /* seconds since the server was created */
    size_t workspace_bytes;
} fvlbm_request_info;

typedef struct fvlbm_server_stats_s {
    int32_t queued, active;
    size_t arena_free, arena_free_largest;
    int64_t cell_steps;     /* cell updates done so far */
    double t_now;           /* seconds since creation */
} fvlbm_server_stats_t;

/* Create (allocates the arena and the streams).  Errors: ARG, OOM, CUDA, UNSUPPORTED. */
int fvlbm_server_create(const fvlbm_server_config* cfg, fvlbm_server** out);
/* Queue a request.  mesh must stay valid until the request is done; params
 * host [n_params] as for fvlbm_init, device equal to the server's.  id: host,
 * written.  Errors: ARG, OOM (workspace larger than the whole arena). */
int fvlbm_server_submit(fvlbm_server* s, const fvlbm_mesh* mesh, const fvlbm_params* params, int32_t n_params,
                        int64_t* id);
/* One scheduling round (see above); n_completed: host, written (may be NULL). */
int fvlbm_server_poll(fvlbm_server* s, int32_t* n_completed);
/* State of a request; rho [n_cell] and u [n_cell][2] (host, may be NULL) are
 * written once it is done, in the caller's cell order. */
int fvlbm_server_request(fvlbm_server* s, int64_t id, fvlbm_request_info* info, double* rho, double* u);
int fvlbm_server_stats(const fvlbm_server* s, fvlbm_server_stats_t* stats);
void fvlbm_server_destroy(fvlbm_server* s);

/*
 * Domain decomposition of one mesh (Sec. 3: the paper's solver runs in
 * Code_Saturne's parallel modules; Conclusions, item 4: one ghost layer per
 * partition interface).  The cells are split into parts by recursive
 * coordinate bisection of their centroids.  A part updates its own cells and
 * holds two rings of ghost cells: ring 1, the cells outside the part that share
 * a face with one of its cells (their least-squares gradients, Eq.
 * leastsquare, are recomputed by the part, since the upwind value on a shared
 * face comes from them, Eq. lslrflux), and ring 2, the cells that share a face
 * with ring 1 (their state only).  After every stage the owner of each ghost
 * sends its new state: one halo exchange of two rings per stage.  Every
 * cell's arithmetic is the same as in the undivided solve, so the result is
 * bitwise the same.
 *
 * The plan (host only, no GPU needed):
 */
#define FVLBM_MAX_PARTS 64

typedef struct fvlbm_partition fvlbm_partition;

typedef struct fvlbm_part_info_s {
    int64_t n_owned;      /* cells the part updates */
    int64_t n_ring1;      /* ghost ring 1 */
    int64_t n_ring2;      /* ghost ring 2 */
    int64_t n_recv;       /* ghost cells received per stage (n_ring1 + n_ring2) */
    int64_t n_send;       /* owned cells sent per stage, summed over the receiving parts */
    int32_t n_neighbours; /* parts it receives from */
} fvlbm_part_info_t;

/*
 * Partition a mesh of one instance into n_parts parts (1..FVLBM_MAX_PARTS, at
 * most one per cell).  Cut: across the longer extent of the centroids'
 * bounding box, at the cell count proportional to the parts on each side
 * (ties broken by cell number): part sizes differ by at most one cell per
 * level of bisection.  The plan copies what it keeps; the mesh may be
 * destroyed afterwards.  Errors: FVLBM_ERR_ARG (several instances, n_parts out
 * of range), _OOM.
 */
int fvlbm_mesh_partition(const fvlbm_mesh* mesh, int32_t n_parts, fvlbm_partition** out);
void fvlbm_partition_destroy(fvlbm_partition* p);
/* Sizes of part `part`.  info: host, written.  Errors: FVLBM_ERR_ARG. */
int fvlbm_partition_info(const fvlbm_partition* p, int32_t part, fvlbm_part_info_t* info);
/*
 * The cells of part `part` in its local numbering: cells[l] is the caller's
 * number (in the partitioned mesh) of local cell l; the owned cells come
 * first in ascending order, then ring 1, then ring 2, each ascending.
 * cells: host [n_owned + n_ring1 + n_ring2], written.  Errors: FVLBM_ERR_ARG.
 */
int fvlbm_partition_cells(const fvlbm_partition* p, int32_t part, int64_t* cells);
/*
 * The message part `src` sends part `dst` after every stage: *count entries;
 * entry e is owned local cell src_local[e] of src, stored into ghost local
 * cell dst_local[e] of dst (local numberings of fvlbm_partition_cells).  With
 * src_local / dst_local NULL only *count is written (0 when src sends dst
 * nothing).  Every ghost of every part appears in exactly one message, from
 * the part that owns it.  count: host, written; src_local, dst_local: host
 * [*count] or NULL.  Errors: FVLBM_ERR_ARG.
 */
int fvlbm_partition_halo(const fvlbm_partition* p, int32_t src, int32_t dst, int64_t* count, int32_t* src_local,
                         int32_t* dst_local);

/*
 * A partitioned solve on one GPU: one solver per part (each with its own
 * workspace, allocated by the library); with more than one part each part's
 * stages run on a stream of its own (so that the parts' kernels overlap), and
 * the halo exchange after every stage, a device-to-device copy of the ghost
 * states (one kernel over all messages), runs on the caller's stream after
 * every part's stage and before any part's next (events order them).  Work
 * the caller queued on its stream before fvlbm_dd_step runs first; the
 * caller's stream holds the last exchange of a step.  The FP64 reductions (mass, residual) sum
 * the parts' FP64 partial sums in part order.  A multi-GPU run would place
 * one part per GPU and carry the same messages over the interconnect; this
 * library runs all parts on the device of params->device.
 *   plan     partition (must stay valid until fvlbm_dd_destroy)
 *   params   host, one set for the whole mesh (n_params = 1); params->kernel
 *            is used by every part
 *   stream   as for fvlbm_init
 * Step 0 (f = f^eq) runs in every part, then one exchange fills the ghosts.
 * Errors: as fvlbm_init.
 */
typedef struct fvlbm_dd fvlbm_dd;
int fvlbm_dd_create(const fvlbm_partition* plan, const fvlbm_params* params, int32_t n_params, void* stream,
                    fvlbm_dd** out);
/* Advance n time steps: per stage, the stage kernels of every part, then the
 * exchange.  Asynchronous on the stream.  Errors: FVLBM_ERR_ARG, _CUDA. */
int fvlbm_dd_step(fvlbm_dd* d, int64_t n);
/* As fvlbm_macros / fvlbm_get_f / fvlbm_set_f for the whole mesh, in the
 * caller's numbering of the partitioned mesh (host buffers, synchronise).
 * fvlbm_dd_set_f also refreshes the ghosts. */
int fvlbm_dd_macros(fvlbm_dd* d, double* rho, double* u);
int fvlbm_dd_get_f(fvlbm_dd* d, double* f);
int fvlbm_dd_set_f(fvlbm_dd* d, const double* f);
/* Total mass sum_i A_i rho_i (FP64; the parts' sums added in part order).
 * mass: host [1]. */
int fvlbm_dd_mass(fvlbm_dd* d, double* mass);
/* Velocity residual of Sec. 3.2 over the whole mesh (numerator and
 * denominator summed over the parts in FP64), against the snapshot of the
 * previous call or of creation; then re-snapshots.  e: host [1]. */
int fvlbm_dd_residual(fvlbm_dd* d, double* e);
/* Stage kernel every part runs (as fvlbm_stage_kernel) and launches per step
 * (stage kernels of all parts plus one exchange kernel per stage). */
int fvlbm_dd_stage_kernel(const fvlbm_dd* d, int32_t* kernel, int64_t* launches_per_step);
int fvlbm_dd_sync(fvlbm_dd* d);
void fvlbm_dd_destroy(fvlbm_dd* d);

/* Message of the last failure on this thread ("" if none). */
const char* fvlbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FVLBM_H */
