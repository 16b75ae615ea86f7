/*
 * lbm.h -- C ABI of the GB300 D3Q19 lattice Boltzmann library (liblbm.so).
 *
 * The library advances a D3Q19 BGK lattice with the on-site velocity boundary
 * condition of Hecht & Harting, "Implementation of on-site velocity boundary
 * conditions for D3Q19 lattice Boltzmann" (arXiv:0811.4593), on one CUDA device.
 * One time step is one fused CUDA sweep: pull streaming, the boundary closure on
 * the populations left unknown by streaming, then BGK collision.
 *
 * Conventions used throughout
 *  - Lattice vectors c_1..c_19 are the columns of the paper's matrix M (eq. deffs);
 *    population i is stored at index i-1. Weights follow eq. weights.
 *  - Population arrays are structure-of-arrays [19][nz][ny][nx], x fastest, in the
 *    storage type of the context's precision (see lbm_precision).
 *  - Faces: 0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1, 4: z=0, 5: z=nz-1. The inward
 *    normal of face 2a is +e_a, of face 2a+1 it is -e_a.
 *  - Every function returns an lbm_status; no C++ exception crosses the ABI. On an
 *    error, lbm_last_error() describes it.
 *  - A context belongs to the CUDA device that was current at lbm_create; every
 *    call makes that device current. A context is not thread-safe.
 *  - Work is issued asynchronously on the context's stream (lbm_set_stream) unless a
 *    function says it synchronises.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; created and owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,      /* invalid argument or unsupported boundary specification */
  LBM_ERR_OOM = -2,      /* the allocator returned NULL */
  LBM_ERR_CUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  LBM_ERR_DIVERGED = -4, /* a reduction found a non-finite or non-positive density or
                            a non-finite velocity */
  LBM_ERR_STATE = -5     /* call not valid in the context's current state */
} lbm_status;

/* Storage of the populations and the arithmetic of the sweep.
 *  LBM_F64          f_i stored as double; all arithmetic in double.
 *  LBM_F32          shifted populations h_i = f_i - w_i rho0 stored as float;
 *                   arithmetic in float except the density of a face closure (eq. uin
 *                   and its appendix analogues), which is formed in double, and the
 *                   reductions, which accumulate in double.
 *  LBM_F16_SHIFTED  h_i = f_i - w_i rho0 stored as IEEE binary16 (round to nearest
 *                   even); arithmetic as for LBM_F32. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16_SHIFTED = 2 } lbm_precision;

/* How the populations are streamed between steps (the method, Sec. "Simulation method",
 * is the same; only the memory traffic pattern differs, and both give the same bits).
 *  LBM_SCHEME_AB  two arrays: every step pulls f_i(x - c_i) from one array and writes
 *                 the other (2 x 19 populations per node resident).
 *  LBM_SCHEME_AA  one array, steps in pairs: a gather-scatter step that reads the
 *                 population -i of node x - c_i and writes f*_i back to that slot's
 *                 place, then an in-place step that reads and writes the node's own
 *                 slots with i and -i exchanged (19 populations per node resident; the
 *                 same bytes move per step). An AA lattice is observable (macros,
 *                 residual, population copies) between step pairs only, and lbm_step /
 *                 lbm_step_residual take an even n. */
typedef enum { LBM_SCHEME_AB = 0, LBM_SCHEME_AA = 1 } lbm_scheme;

/* Periodic faces wrap streaming to the opposite face (periodic boundaries of the
 * paper's Sec. "Boundary conditions") and must come in pairs. A velocity face applies
 * the on-site velocity condition; a prescribed velocity of zero is the on-site
 * no-slip wall (Sec. "On-site no-slip boundary condition"). A pressure face applies
 * the density variant (eq. rhoin and its appendix analogues): the density and the
 * tangential velocity are prescribed and the normal velocity follows from the plane's
 * density relation; edges and corners next to it take the buried-link values that give
 * them the prescribed density (eq. buried_rho and the corner variant). */
typedef enum { LBM_FACE_PERIODIC = 0, LBM_FACE_VELOCITY = 1, LBM_FACE_PRESSURE = 2 } lbm_face_kind;

typedef enum { LBM_HOST = 0, LBM_DEVICE = 1 } lbm_memory;

typedef struct {
  int kind;              /* lbm_face_kind */
  double u[3];           /* prescribed velocity (lattice units) on every node of the face,
                            used when u_table is NULL; on a pressure face only its
                            tangential components are used */
  const double* u_table; /* optional HOST array [n2][n1][3] of prescribed velocities, one
                            per node of the face plane, over the face's two tangential
                            axes in increasing axis order (x faces [z][y], y faces [z][x],
                            z faces [y][x]); copied by lbm_create, not retained */
  double rho;            /* pressure face: prescribed density on every node, used when
                            rho_table is NULL */
  const double* rho_table; /* pressure face: optional HOST array [n2][n1] of prescribed
                              densities, laid out like u_table; copied, not retained */
} lbm_face_spec;

/* Device allocator hook: every device buffer the library owns is obtained through
 * alloc(bytes, user) and returned through release(ptr, user). Default: cudaMalloc and
 * cudaFree. Takes effect for allocations made after the call; release is always
 * called with the hook that allocated the pointer. NULL alloc restores the default.
 * alloc must return memory aligned to 256 bytes (as cudaMalloc and PyTorch's caching
 * allocator do): the sweeps read population rows with 16-byte bulk copies and 4-byte
 * pair loads; a pointer with less alignment is returned through release at once and
 * the allocation fails with LBM_ERR_OOM. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void (*lbm_free_fn)(void* ptr, void* user);
LBM_API lbm_status lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* user);

/* Create a lattice of nx x ny x nz nodes.
 *  tau   BGK relaxation time (eq. bgk); kinematic viscosity (tau - 1/2)/3 (eq. visc).
 *  faces six face descriptions (see lbm_face_spec).
 *  rho0  initial density; the initial state is the post-collision state
 *        f_i = f_i^eq(rho0, 0) (eq. feq).
 * Validation (LBM_ERR_ARG): tau > 1/2; every dimension >= 3; 19 * nx*ny*nz < 2^32;
 * periodic faces in pairs; |u.n| < 1 on every velocity face node; finite positive
 * densities on pressure faces, which may lie on one axis only. On edges and corners
 * (nodes on two or three non-periodic faces) the no-slip rules of Sec. "On-site
 * no-slip boundary condition" apply and velocity tables are not read there.
 * Ownership: *out is owned by the library until lbm_destroy. The lattice streams with
 * LBM_SCHEME_AB; lbm_create_scheme chooses the scheme. */
LBM_API lbm_status lbm_create(int nx, int ny, int nz, double tau, const lbm_face_spec faces[6],
                      lbm_precision prec, double rho0, lbm_ctx** out);
LBM_API lbm_status lbm_create_scheme(int nx, int ny, int nz, double tau, const lbm_face_spec faces[6],
                                     lbm_precision prec, double rho0, lbm_scheme scheme, lbm_ctx** out);

/* Release every device buffer of the context (after synchronising its stream) and the
 * context itself. NULL is accepted. */
LBM_API lbm_status lbm_destroy(lbm_ctx* ctx);

/* Use `cuda_stream` (a cudaStream_t; NULL = legacy default stream) for all later work
 * of the context. */
LBM_API lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Advance n >= 0 time steps, asynchronously. Each step is, per node: pull streaming
 * f_i(x) = f*_i(x - c_i) with wrap-around on periodic axes (Sec. "Simulation method",
 * Sec. "Boundary conditions"); on face nodes the density relation eq. uin and the
 * unknown populations eq. f5, eqs. f9-f17 with the corrections eqs. Nx, Ny (and their
 * appendix analogues for the other planes); on edge and corner nodes bounce-back with
 * the edge correction eq. edge, buried links eq. buried and eq. corner; then BGK
 * collision (eq. bgk, eq. feq). Binary16 lattices whose rows are multiples of 8 nodes
 * and at least 256 long take a sweep that stages population rows in shared memory with
 * bulk copies; its waits are bounded, and one that runs out is reported by the next
 * synchronising call as LBM_ERR_CUDA (see lbm_debug_drop_staged_copies). Every sweep
 * variant computes the same bits for a node. */
LBM_API lbm_status lbm_step(lbm_ctx* ctx, int n);

/* Advance n >= 1 steps like lbm_step, the last one also forming, in double, the
 * total mass sum(rho) and the steady-state residual
 *   r = sqrt(sum |u - u_snap|^2) / sqrt(sum |u|^2)
 * where u_snap is the velocity field at the previous residual evaluation (zero
 * before the first one); u_snap is then replaced by the current field. Synchronises.
 * Returns LBM_ERR_DIVERGED (after writing *residual and *mass) when any node has a
 * non-finite or non-positive density or a non-finite velocity. The residual is not
 * part of the paper; it is the library's steady-state criterion. */
LBM_API lbm_status lbm_step_residual(lbm_ctx* ctx, int n, double* residual, double* mass);

/* Same reductions as lbm_step_residual, evaluated on the stored post-collision state
 * without advancing it (density and velocity are collision invariants, so this is the
 * state after the last step's closure). Synchronises. */
LBM_API lbm_status lbm_residual(lbm_ctx* ctx, double* residual, double* mass);

/* Density (eq. rho) into rho[nz][ny][nx] and velocity (eq. vel) into u[3][nz][ny][nx]
 * of the stored state. Both are caller-owned DEVICE buffers of double for LBM_F64,
 * float otherwise. Asynchronous. Either pointer may be NULL. */
LBM_API lbm_status lbm_macros(lbm_ctx* ctx, void* rho, void* u);

/* Copy the planes z0 .. z0+nzs-1 of the stored populations from / to a caller buffer
 * laid out [19][nzs][ny][nx] in the storage type: double holding f_i for LBM_F64,
 * float or binary16 holding h_i = f_i - w_i rho0 for LBM_F32 and LBM_F16_SHIFTED. `where` says whether the caller buffer is host or device
 * memory. Synchronises. The state written by lbm_set_populations counts as
 * post-collision. */
LBM_API lbm_status lbm_set_populations(lbm_ctx* ctx, const void* src, int z0, int nzs, lbm_memory where);
LBM_API lbm_status lbm_get_populations(lbm_ctx* ctx, void* dst, int z0, int nzs, lbm_memory where);

/* Mark solid nodes: `solid` is a HOST array [nz][ny][nx], nonzero for a solid node
 * (copied, not retained). Fluid nodes next to a solid node take the mid-grid
 * bounce-back of Sec. "Boundary conditions" for the populations that would stream in
 * from it: f_i(x) = f*_-i(x), the population the node sent towards the wall, reversed.
 * Solid nodes keep their populations. Costs 4 bytes per node of extra traffic per step.
 * A/B scheme only (LBM_ERR_ARG for AA). Synchronises. */
LBM_API lbm_status lbm_set_solid(lbm_ctx* ctx, const uint8_t* solid);

/* General geometry (Sec. "On-site no-slip boundary condition", complex geometries):
 * `solid` (as for lbm_set_solid, may be NULL) and `code`, a HOST array [nz][ny][nx]
 * of int8 (may be NULL; both copied, not retained) naming the on-site rule of each
 * boundary node by its normal, written as the paper's lattice-vector index i of c_i
 * (the normal points into the fluid; every such wall is at rest):
 *     0          no rule: a bulk node, a face/edge/corner of the box (classified from
 *                the face specs as usual), or a node taking mid-grid bounce-back from
 *                its solid neighbours;
 *     1..6       plane with normal c_i: eq. bbshort with v = 0 (density from the plane's
 *                relation);
 *     7..18      concave edge whose bulk normal is the diagonal c_i = n1 + n2: eq. edge
 *                (bounce-back, along-edge correction, buried links eq. buried);
 *     -7..-18    convex edge with bulk normal c_-code: the population from the solid
 *                side is bounced back, then 1/4 (c_i.e) sum_j f_j (c_j.e) (eq. edge2,
 *                e = n1 x n2) is subtracted from every population with c_i.c_-code > 0;
 *     19..26     corner with normal (sx, sy, sz): code 19 + [sx<0] + 2[sy<0] + 4[sz<0];
 *                eq. corner;
 *     27..50     a convex edge meeting the plane perpendicular to it: code
 *                27 + 4 (p - 1) + j for the plane normal c_p (p = 1..6) and the edge's
 *                bulk normal the j-th (j = 0..3, increasing index) diagonal c_i with
 *                c_i.c_p = 0. The populations coming through the plane or from the edge's
 *                solid side are bounced back and the rest population is set to 12/36 of
 *                the node density (the printed factor taken as a share of the density,
 *                which keeps a resting node at rest).
 * A node with a code must be fluid, and every population it cannot stream (source solid,
 * or outside a walled axis) must be one its rule sets; otherwise LBM_ERR_ARG names the
 * node. Extra traffic: 4 bytes per node per step. A/B scheme only; not while the context
 * is attached to a batch (LBM_ERR_STATE). Synchronises. */
LBM_API lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* solid, const int8_t* code);

/* The populations the rule of a node code overwrites: bit k of *mask set for population
 * k (the paper's f_{k+1}). Host-only, needs no device. LBM_ERR_ARG for a value that is
 * not a code. */
LBM_API lbm_status lbm_rule_unknowns(int code, uint32_t* mask);

/* Uniform body force F (force per volume, lattice units) acting on every fluid node
 * (Sec. "Numerical Results", eq. gravity): the collision relaxes toward the equilibrium
 * at the velocity u + tau F / rho and so adds F to each node's momentum per step. The
 * velocity reported by lbm_macros and the residual is that of the stored post-collision
 * state, u + F / rho. F = 0 switches the force off. Not finite: LBM_ERR_ARG. A/B scheme
 * only; not while attached to a batch (LBM_ERR_STATE). Takes effect with the next step. */
LBM_API lbm_status lbm_set_body_force(lbm_ctx* ctx, const double force[3]);

/* Every device buffer of a context lies between two 256-byte guard regions filled with
 * a fixed pattern at allocation (device_bytes counts the buffers, not the guards). This
 * reads the guards back and returns LBM_ERR_STATE, naming the buffer, if any byte
 * changed -- evidence of a write outside a buffer. Synchronises. */
LBM_API lbm_status lbm_check_guards(lbm_ctx* ctx);

/* Out-of-range indices the sweeps met since the last call, on the current device. The
 * library built with LBM_DEBUG_BOUNDS (build option debug_bounds) checks every
 * population, table and geometry-word index of its sweeps, replaces an index beyond
 * its buffer by 0 and counts it; *enabled says whether this library is such a build
 * (otherwise *count is 0). Synchronises the device. */
LBM_API lbm_status lbm_debug_bounds_errors(int* enabled, uint64_t* count);

/* Failure injection for tests (no counterpart in the paper). The binary16 sweep that
 * stages rows in shared memory waits on its bulk copies with a time limit (about one
 * second); when a wait runs out, the sweep sets the context's device error word and
 * ends, and the next synchronising call (lbm_sync, lbm_step_residual, lbm_residual,
 * lbm_get_populations) returns LBM_ERR_CUDA with a message that says so; the state
 * of the steps since the previous such call is then not valid, but the context stays
 * usable (load a state with lbm_set_populations). With enable != 0, later row-staged
 * sweeps of `ctx` leave the copies of one row group un-issued, so that a wait runs
 * out on purpose (no fault: the sweep ends after about two seconds); enable = 0 turns
 * this off. Other sweep kernels ignore it. */
LBM_API lbm_status lbm_debug_drop_staged_copies(lbm_ctx* ctx, int enable);

/* Block the host until the context's stream is idle; reports asynchronous errors. */
LBM_API lbm_status lbm_sync(lbm_ctx* ctx);

typedef struct {
  int nx, ny, nz;
  int precision;            /* lbm_precision */
  int64_t steps;            /* time steps taken since lbm_create */
  int64_t kernel_launches;  /* CUDA kernels the context has launched */
  int64_t bytes_per_update; /* algorithmic bytes moved per node update: 19 loads + 19
                               stores of the storage type */
  int64_t device_bytes;     /* device memory the context holds */
  int scheme;               /* lbm_scheme */
} lbm_info_t;
LBM_API lbm_status lbm_info(const lbm_ctx* ctx, lbm_info_t* out);

/* ---------------------------------------------------------------------------------
 * Batches: many resident lattices advanced together (continuous-batching serving).
 *
 * A batch advances every attached context by one persistent CUDA launch per time step:
 * the launch's thread blocks draw chunks of the 256-node blocks of all attached
 * lattices from a device counter (chunks shrink toward the end, so the thread blocks
 * finish together) and run, per node, exactly the computation of lbm_step (same
 * device code, same grouping of the residual sums), so an attached lattice evolves to
 * the same bits as when it is stepped alone. The n-step loop is captured once as a
 * CUDA graph per (n, residual) and replayed; the descriptor table it reads is rewritten
 * in device memory before each replay, so lattices can be attached and detached
 * between calls without recapturing.
 * --------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque; owned by the library */

typedef struct {
  int capacity;             /* slots */
  int attached;             /* slots in use */
  int grid;                 /* thread blocks of the persistent launch */
  int64_t nodes;            /* nodes of all attached lattices */
  int64_t steps;            /* batched steps taken */
  int64_t kernel_launches;  /* kernels the batch has launched (sweeps + reductions) */
  int64_t device_bytes;     /* device memory the batch itself holds (its table) */
} lbm_batch_info_t;

/* A batch of `capacity` slots for contexts of precision `prec` on the current device.
 * Work runs on a stream the batch creates (see lbm_batch_set_stream). */
LBM_API lbm_status lbm_batch_create(int capacity, lbm_precision prec, lbm_batch** out);

/* Synchronise, detach every context (the contexts stay valid) and free the batch. */
LBM_API lbm_status lbm_batch_destroy(lbm_batch* b);

/* Issue later batch work on `cuda_stream` (NULL = legacy default stream, on which the
 * steps are launched directly instead of through a CUDA graph). Synchronises the
 * previous stream. */
LBM_API lbm_status lbm_batch_set_stream(lbm_batch* b, void* cuda_stream);

/* Put `ctx` into `slot` (0 <= slot < capacity, empty). The context must have the
 * batch's precision, device and streaming scheme (all attached contexts share one),
 * belong to no other batch and, for AA, stand between step pairs. Waits for the context's
 * own stream and allocates its residual buffers. While attached, the context's own
 * calls (lbm_step, lbm_macros, ...) first wait for the batch's stream; lbm_destroy
 * detaches it. */
LBM_API lbm_status lbm_batch_attach(lbm_batch* b, int slot, lbm_ctx* ctx);

/* Empty `slot` after the batch's queued work has finished (synchronises). */
LBM_API lbm_status lbm_batch_detach(lbm_batch* b, int slot);

/* Advance every attached lattice by n >= 1 time steps (as lbm_step; n even for AA
 * lattices), asynchronously on the batch's stream. With residual != 0 the last step also forms each lattice's
 * residual and mass exactly as lbm_step_residual does (same snapshot semantics); read
 * them with lbm_batch_results. */
LBM_API lbm_status lbm_batch_step(lbm_batch* b, int n, int residual);

/* Per slot (arrays of `capacity`, any may be NULL): residual and mass of the last
 * lbm_batch_step with residual != 0, and a status: LBM_OK, LBM_ERR_DIVERGED (as in
 * lbm_step_residual), or 1 when the slot has no result (empty, or attached after that
 * step). Synchronises. */
LBM_API lbm_status lbm_batch_results(lbm_batch* b, double* residual, double* mass, int* status);

LBM_API lbm_status lbm_batch_info(const lbm_batch* b, lbm_batch_info_t* out);

/* Last error message of a batch (or of the calling thread when b is NULL). */
LBM_API const char* lbm_batch_last_error(const lbm_batch* b);

/* Reduction of a caller-held population array that allocates nothing (the paper has no
 * counterpart; it is the state reduction of lbm_residual without a context).
 *
 * For callers that cannot call cudaMalloc: code that runs while all device memory is
 * owned by another pool or framework, code that must not trigger the device-wide
 * synchronisation cudaMalloc and cudaFree can cause, and code running where new device
 * allocations are forbidden. Every buffer is the caller's; the only scratch, 2 MiB of
 * per-block partial sums, is a static array inside the library that every device
 * which loads the library holds until the process exits.
 *
 *  populations        DEVICE [19][nz][ny][nx] in the storage type of `prec` (double f_i
 *                     for LBM_F64; float / binary16 h_i = f_i - w_i rho0 otherwise)
 *  velocity_snapshot  DEVICE [3][nz][ny][nx], double for LBM_F64 else float: read as
 *                     u_snap, then overwritten with the current velocity
 *  sums               DEVICE double[4], written with {sum rho, sum |u - u_snap|^2,
 *                     sum |u|^2, number of nodes with a non-finite or non-positive
 *                     density or a non-finite velocity}; the residual of lbm_residual is
 *                     sqrt(sums[1]) / sqrt(sums[2])
 *  cuda_stream        stream for the two kernel launches (NULL = legacy default stream)
 * Limit: at most 16,777,216 nodes (256^3); larger lattices get LBM_ERR_ARG with a
 * message naming the limit. Asynchronous; nothing is allocated and nothing is freed.
 * The first call on a device looks up the static array's device address (with that
 * device current); make that first call before any stream capture. All calls share
 * the one array, which keeps the last call's contents (every call overwrites the part
 * it reads, so nothing needs clearing): calls that overlap on the GPU, e.g. on two
 * streams at once, race and give wrong sums. */
LBM_API lbm_status lbm_reduce_state_static(const void* populations, int nx, int ny, int nz,
                                           lbm_precision prec, double rho0, void* velocity_snapshot,
                                           double* sums, void* cuda_stream);

/* Measurement helper (no counterpart in the paper): the current device's rate of FP64
 * fused multiply-adds, from a kernel that keeps every resident warp on eight
 * independent FMA chains per thread for `iters` iterations (after a short warm-up
 * launch), timed with CUDA events on the legacy default stream. Writes thread-level
 * DFMA operations per second to *fma_per_s and the timed launch's duration in
 * milliseconds to *ms (may be NULL). Synchronises. LBM_ERR_ARG for iters < 1 or a NULL
 * fma_per_s; LBM_ERR_CUDA if a launch fails. The FP64 sweep's roofline divides its
 * FP64 instruction rate by this rate. */
LBM_API lbm_status lbm_fp64_fma_rate(int iters, double* fma_per_s, double* ms);

/* Last error message of a context, or of the calling thread's last failed call that
 * had no context (ctx == NULL). Never NULL. */
LBM_API const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
