/*
 * lf.h -- C ABI of the GB300 layered-field library.
 *
 * Layered fields (Zayer, Mlakar, Steinberger, Seidel, "Layered Fields for
 * Natural Tessellations on Surfaces", arXiv 1804.09152) partition a triangle
 * mesh into cells by growing one field per seed concurrently.  The field is a
 * sparse (vertex x layer) matrix F: row i lists the layers present at vertex
 * i with their values in (0, 1].  Layers 0..k-1 belong to the k seeds, layer
 * k is the base layer (Sec. 3.1).  One time-iteration (Algorithm 1) multiplies
 * the mesh Laplacian with F, evaluates the interest skeleton, applies the
 * explicit Euler update with clamping (Eq. 11-13) and normalises every vertex
 * (Sec. 4); this library runs that iteration as one fused CUDA kernel per step.
 *
 * Conventions for every function below.
 *  - Host arrays passed in are owned by the caller and are copied (or fully
 *    consumed) before the call returns.
 *  - Output arrays are allocated by the caller; a call that fills one waits
 *    for the mesh's stream to finish.
 *  - Device memory is owned by the mesh handle.  It is allocated through the
 *    lf_device hooks when given, else with cudaMalloc, and released by
 *    lf_destroy_mesh.
 *  - No C++ exception crosses this interface and nothing aborts the process.
 *    Every function returns an lf_status; lf_last_error() gives a message.
 *  - After LF_ERR_CUDA or LF_ERR_TIMEOUT a handle is poisoned: later calls on
 *    it return LF_ERR_STATE.  Other errors leave the handle usable.
 *  - A handle is not thread-safe.  Distinct handles may be used from distinct
 *    threads on distinct streams.
 *  - Kernels run on the stream given in lf_device (0 = legacy default stream).
 */
#ifndef LF_H
#define LF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LF_OK = 0,
  LF_ERR_INVALID = 1,   /* bad argument; nothing was changed                  */
  LF_ERR_OOM = 2,       /* device allocation failed; state unchanged          */
  LF_ERR_CUDA = 3,      /* a CUDA call failed; the handle is poisoned         */
  LF_ERR_TIMEOUT = 4,   /* a bounded device wait gave up; handle poisoned     */
  LF_ERR_STATE = 5,     /* call not valid in this state (e.g. step before seed,
                           or a poisoned handle)                              */
  LF_ERR_CAPACITY = 6   /* a size limit of the library was exceeded           */
} lf_status;

/* Storage type of the field values.  All arithmetic is FP32. */
typedef enum { LF_F32 = 0, LF_BF16 = 1, LF_F16 = 2 } lf_dtype;

/*
 * Parameters of the update (Algorithm 1; Eq. 2, 11-13; Sec. 7).
 * The coefficient matrices w, a, e of Algorithm 1 are given by two classes of
 * layer pairs: two seed layers ("cell-cell", _cc) and a seed layer with the
 * base layer ("cell-base", _cb).  w and a are symmetric; e is not: e_cb is the
 * entry in a cell's row against the base, e_bc the entry in the base row.
 * A layer has no coefficient with itself.  lf_default_params() fills
 *   dt = 5 (Sec. 7), mu = 1, w_cc = 0.2, a_cc = a_cb = 0.04 (w = 0.2 and a
 *   factor 5 between w and a, Sec. 3.1), w_cb = 0, e_cc = 0, e_cb = 0.5,
 *   e_bc = -0.5 (Eq. 12 is antisymmetric in the pair), iso = 0.25 (Sec. 5.1),
 *   field_dtype = LF_F32, initial_capacity = 0.
 * initial_capacity: entries each field buffer holds before the first growth;
 *   0 picks three entries per vertex (at least 256 per tile of 256 vertices).
 *   Growth is automatic (lf_step), so this only trades memory against re-runs
 *   of a step.
 */
typedef struct {
  double dt;
  double mu;
  double w_cc, w_cb;
  double a_cc, a_cb;
  double e_cc, e_cb, e_bc;
  double iso;
  int32_t field_dtype;   /* lf_dtype */
  int32_t reserved;      /* must be 0 */
  int64_t initial_capacity;
} lf_params;

/*
 * Device context.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  alloc/free, when both non-NULL, replace cudaMalloc/cudaFree for
 * every device buffer of a handle: alloc(bytes, cuda_stream, user) returns a
 * device pointer aligned to 256 bytes or NULL; free(ptr, user) releases it.
 * The struct is copied by lf_create_mesh; the hooks must stay callable until
 * lf_destroy_mesh returns.
 */
typedef struct {
  void* cuda_stream;
  void* (*alloc)(size_t bytes, void* cuda_stream, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} lf_device;

typedef struct lf_mesh_s* lf_mesh;

typedef struct {
  int64_t n_v;            /* vertices                                         */
  int64_t n_layers;       /* k + 1 after lf_seed, else 0                       */
  int64_t steps;          /* time-iterations completed since lf_seed           */
  int64_t nnz;            /* entries of the current field                      */
  int64_t capacity;       /* entries each field buffer can hold                */
  int64_t operator_nnz;   /* off-diagonal entries of L (diagonal is implicit)  */
  uint64_t skeleton_total;/* sum over completed steps of |interest skeleton|    */
  uint64_t nnz_io_total;  /* sum over completed steps of nnz(in) + nnz(out)     */
  int64_t device_bytes;   /* device memory held by the handle                  */
  int32_t retries;        /* steps re-run after a capacity or map overflow     */
  int32_t map_slots;      /* register slots of the step kernel's fast path;
                             larger layer unions take its exact slow path     */
  int32_t field_dtype;    /* lf_dtype                                          */
  int32_t value_bytes;    /* bytes per stored field value                      */
} lf_stats_t;

/* Defaults listed at lf_params. */
void lf_default_params(lf_params* p);

/*
 * Builds the static operator of a triangle mesh: the cotangent Laplacian
 * (precomputed once, Sec. 3.2), L_ij = (cot alpha_ij + cot beta_ij) / 2 over
 * the angles opposite edge ij, L_ii = -sum_j L_ij, no mass matrix; every edge
 * is kept even when its weight is 0.  The mesh is copied to the device once
 * (it stays there for lf_lloyd and lf_extract_dual) and the operator is built
 * there in FP64, summed over the faces in face order, and stored as FP32 CSR
 * without the diagonal (lf_get_operator reads it back).
 *   V: n_v x 3 doubles, row-major.  F: n_f x 3 int32 vertex ids, 0-based.
 *   params: copied; may be NULL for the defaults.
 * Errors: LF_ERR_INVALID for n_v < 3, n_v >= 2^31, n_f < 1, an id out of
 * range, a repeated id in a face or a zero-area face, or invalid params
 * (dt <= 0, mu < 0, unknown dtype); LF_ERR_OOM; LF_ERR_CUDA.  *out is set
 * only on LF_OK.
 */
lf_status lf_create_mesh(const lf_device* dev, const double* V, int64_t n_v,
                         const int32_t* F, int64_t n_f, const lf_params* params,
                         lf_mesh* out);

/*
 * Same with a caller-given symmetric operator instead of the cotangent
 * Laplacian (the paper leaves the discretisation open).  CSR over n_v rows:
 * rowptr (n_v + 1, int64), col (int32, sorted per row), val (double).
 * Diagonal entries are ignored: the library always uses L_ii = -sum_j L_ij.
 * Errors as lf_create_mesh, plus LF_ERR_INVALID for a non-monotone rowptr or
 * a column out of range.
 */
lf_status lf_create_mesh_csr(const lf_device* dev, int64_t n_v, const int64_t* rowptr,
                             const int32_t* col, const double* val,
                             const lf_params* params, lf_mesh* out);

/*
 * Initialisation (Algorithm 1, first line; Sec. 3.1-3.2): seed s (0 <= s < k)
 * gets value 1 in layer s at vertex seed_vertices[s]; every other vertex gets
 * value 1 in the base layer k.  Resets the step counter and statistics.
 * Errors: LF_ERR_INVALID for k < 1, k + 1 > 65536, a vertex out of range or
 * a repeated vertex.
 */
lf_status lf_seed(lf_mesh m, const int32_t* seed_vertices, int32_t k);

/*
 * Region seeds (Sec. 3.2, "Initialization": a vertex and its immediate
 * neighbours set to 1).  rings = 0 is lf_seed; rings = 1 gives layer c to seed
 * vertex seeds[c] and to its neighbours in L.  A vertex reached by several
 * seeds keeps its own seed's layer if it is a seed, else takes the lowest
 * seed id; every other vertex holds the base layer.  Seeds are remembered as
 * for lf_seed.  Errors: as lf_seed, and LF_ERR_INVALID for rings outside [0, 1].
 */
lf_status lf_seed_regions(lf_mesh m, const int32_t* seeds, int32_t k, int32_t rings);

/*
 * General coefficient matrices of Algorithm 1 (Sec. 3.2: the update is
 * written for any w_jl, a_jl, e_jk; Sec. 3.1 gives the uniform values that
 * lf_params holds as two classes).  W, A and E are host pointers, each NULL or an n_layers x n_layers
 * row-major FP32 matrix indexed by layer id (cells 0..k-1, base layer k):
 * W[j * n_layers + l] = w_jl, A[...] = a_jl, E[j * n_layers + k] = e_jk.  A
 * NULL matrix keeps the class rule for that coefficient; all three NULL
 * returns to the class coefficients.  Every entry is used as given, diagonal
 * included, with no symmetry assumed.  The library copies the matrices to
 * the device (n_layers^2 * 4 bytes each) and the call returns after the
 * copy.  They hold until the next call, or until the field takes another
 * layer count (lf_seed or lf_set_field with a different k); seeding again
 * with the same k, as lf_lloyd does, keeps them.  A mesh with matrices runs
 * the general form of the step kernel, which sums the matrices over the
 * skeleton of each vertex.
 * Errors: LF_ERR_STATE before the first lf_seed / lf_set_field;
 * LF_ERR_INVALID if n_layers differs from the field's layer count, exceeds
 * 4096, or an entry is not finite; LF_ERR_OOM.
 */
lf_status lf_set_coefficients(lf_mesh m, int32_t n_layers, const float* W, const float* A, const float* E);

/*
 * Runs n_iters time-iterations of Algorithm 1 (the body of its time loop):
 * L_t = L F (the paper's Phi L^T for a symmetric L), the interest skeleton
 * irows_i = {l : F_il > 0} u {l : F_il = 0, (L F)_il > 0}, the explicit Euler
 * update of Eq. 11-13 over the skeleton with clamping to [0, 1], the
 * normalisation of every vertex to sum 1 and the removal of zero entries
 * (Sec. 4).  Every d uses the values before the step.  Returns after the
 * work is done on the device.  When the output outgrows a field buffer, the
 * library grows it (by at least 20 %, Sec. 4) and re-runs the step; results
 * do not depend on it.  Any number of layers per neighbourhood is handled.
 * Errors: LF_ERR_STATE before lf_seed; LF_ERR_INVALID for n_iters < 0;
 * LF_ERR_OOM when growth fails (the field stays at the last completed step);
 * LF_ERR_CAPACITY when the field would exceed 2^31 entries;
 * LF_ERR_TIMEOUT, LF_ERR_CUDA.
 */
lf_status lf_step(lf_mesh m, int32_t n_iters);

/*
 * Batching form: meshes[a] advances by n_iters[a] time-iterations (as
 * lf_step), for 1 <= n <= 64 meshes, all in shared launches: each step is one
 * kernel launch per storage type present whose CTAs cover the tiles of every
 * mesh of that type, and runs of 128 steps are replayed as one CUDA graph
 * (one independent chain per storage type).  A mesh leaves the launches when
 * its count is reached.  Results are bit-identical to lf_step on each mesh
 * alone.  The batch runs on meshes[0]'s stream after every mesh's earlier work
 * has finished and returns when all steps are done.  A mesh whose field
 * outgrows its buffers is grown and its step re-run while the others go on.
 * meshes and n_iters are caller-owned arrays of n entries, read during the
 * call.  Errors: LF_ERR_INVALID for n outside [1, 64], a null array, a
 * negative count or a repeated mesh; LF_ERR_STATE for an unseeded mesh, or a
 * vertex that sums to zero (that mesh stops where it failed, the others
 * finish); LF_ERR_OOM, LF_ERR_CUDA.
 */
lf_status lf_step_batch(lf_mesh* meshes, int32_t n, const int32_t* n_iters);

/*
 * Sharp labels (Sec. 6: the field of largest value at each vertex).
 * labels[i] = layer of the largest value at vertex i, the lowest layer id on
 * a tie, and -1 when that layer is the base layer.  labels: n_v int32.
 * maxval: NULL or n_v floats receiving that largest value.
 * Errors: LF_ERR_STATE before lf_seed.
 */
lf_status lf_labels(lf_mesh m, int32_t* labels, float* maxval);

/*
 * Copies the mesh's operator to the host as it is stored: the off-diagonal
 * entries L_ij (i != j) as CSR, rowptr (n_v + 1 int64), col (int32,
 * increasing in each row), val (float); L_ii = -sum_j L_ij is implied.  For
 * lf_create_mesh that is the cotangent Laplacian of Sec. 3.2 (half the sum
 * of the cotangents opposite each edge), built on the device in FP64 and
 * rounded to FP32 once.  With col or val NULL, or cap below the entry count,
 * only *nnz and rowptr (if non-NULL) are written: a size query.
 * Errors: LF_ERR_INVALID for a NULL nnz.
 */
lf_status lf_get_operator(lf_mesh m, int64_t* rowptr, int32_t* col, float* val, int64_t cap, int64_t* nnz);

/*
 * Copies the current field to the host as CSR: rowptr (n_v + 1 int64),
 * layer (int32), val (float, widened from the storage type).  With layer or
 * val NULL, or cap smaller than the number of entries, only *nnz and rowptr
 * (if non-NULL) are written and LF_OK is returned: a size query.
 */
lf_status lf_get_field(lf_mesh m, int64_t* rowptr, int32_t* layer, float* val,
                       int64_t cap, int64_t* nnz);

/*
 * Replaces the current field (checkpoint resume, tests).  Same layout as
 * lf_get_field; values are rounded to the storage type.  n_layers = k + 1.
 * Errors: LF_ERR_INVALID for a non-monotone rowptr, a layer out of range or
 * not strictly increasing within a row, a value not in (0, 1] or not finite,
 * n_layers < 2 or > 65536.
 */
lf_status lf_set_field(lf_mesh m, const int64_t* rowptr, const int32_t* layer,
                       const float* val, int64_t nnz, int32_t n_layers);

/* Counters of the handle; see lf_stats_t. */
lf_status lf_stats(lf_mesh m, lf_stats_t* out);

/* Releases the handle and all its device memory (waits for its stream). */
void lf_destroy_mesh(lf_mesh m);

/* Static string for a status code. */
const char* lf_status_string(lf_status s);

/* Message of the last failed call on m (m = NULL: the last failed call made
 * without a handle on this thread: lf_create_mesh*, lf_step_noalloc). */
const char* lf_last_error(lf_mesh m);

/*
 * One time-iteration for callers that cannot allocate device memory.
 *
 * No counterpart in the paper.  Every other entry point here allocates (the
 * handle's buffers and the step's status words).  Callers
 * that own all device memory themselves -- a framework with its own memory
 * pool, a service that allocates only at start-up, code running where an
 * allocation is not allowed -- can call this instead: it runs the same step
 * kernel as lf_step on buffers the caller provides, and calls no cudaMalloc,
 * cudaFree or other allocating routine.  The kernel's scratch (its status and
 * counter words; 1 KiB reserved) lives in a static device array that every
 * GPU loading this library holds until the process exits.
 *
 * All pointers are device pointers on the current device; the call runs on
 * cuda_stream (NULL = legacy default stream) and returns when the step is
 * done.  Layout (FP32 values only):
 *   d_L_rowptr  n_v + 1 int32: row offsets of the operator, off-diagonal entries
 *               only (L_ii = -sum_j L_ij is implied);
 *   d_L_colval  2 int32 per entry: column, then the IEEE-754 bits of L_ij
 *               (8-byte aligned);
 *   field in / out, tile-segmented CSR with T = ceil(n_v / 256) tiles: vertex i
 *   belongs to tile i / 256; d_rows_* hold 2 int32 per vertex (start, count),
 *   8-byte aligned; the rows of tile t lie one after another, layer ids
 *   ascending within a row, inside entries [t * tile_cap, (t + 1) * tile_cap)
 *   of d_ids_* (uint16) and d_vals_* (float); both fields hold T * tile_cap
 *   entries.  d_head_* hold 4 int32 per vertex (16-byte aligned): the row's
 *   count, id0 | id1 << 16, and the IEEE-754 bits of its first two values
 *   (zeros where the row is shorter) -- the input's must match its rows, the
 *   output's is written.  n_layers = k + 1 (the base layer is k).
 *   nnz_out (host, nullable): entries of the output field.
 *   need_tile_cap (host, nullable): on LF_ERR_CAPACITY, the tile_cap needed.
 * Limits: tile_cap a multiple of 16 and >= 256; n_v <= 2^31 - 257;
 * T * tile_cap <= 2^31 - 1.  Larger sizes are rejected (LF_ERR_INVALID or
 * LF_ERR_CAPACITY) with a message in lf_last_error(NULL); so is a field_dtype
 * other than LF_F32.
 * The first call on a device looks up the scratch's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset it no longer names the array, so do not call this entry
 * point again in a process that has reset the device.  Every call shares the
 * scratch and resets it: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  The parameters pass
 * the checks of lf_create_mesh (finite, dt > 0, mu >= 0, reserved = 0) and
 * must also be finite in FP32.
 */
lf_status lf_step_noalloc(void* cuda_stream, int32_t n_v, int32_t n_layers,
                          const int32_t* d_L_rowptr, const int32_t* d_L_colval,
                          const int32_t* d_rows_in, const int32_t* d_head_in, const uint16_t* d_ids_in,
                          const float* d_vals_in, int32_t* d_rows_out, int32_t* d_head_out,
                          uint16_t* d_ids_out, float* d_vals_out, int32_t tile_cap, const lf_params* params,
                          int64_t* nnz_out, int64_t* need_tile_cap);

/*
 * Step-kernel schedules (no counterpart in the paper, which runs one mesh).
 * Schedules 0, 1 and 2 are the step kernel with its registers allocated for
 * 4 (the default), 5 and 3 resident CTAs per SM (the FP32 kernel takes 64,
 * 48 and 80 registers a thread).  Schedule 3 runs a lean register-tier path
 * (every vertex of a tile holding at most five cells and the base layer and
 * seeing at most five cells in its closed neighbourhood; four neighbours'
 * loads in flight a thread, branch-free slot updates) and the full step on
 * any other tile, in the same launch.  Schedule 4 is the step kernel with
 * that lean gather as its register tier and, per vertex, the shared-memory
 * and storage-free tiers beyond it.  All give the same bits.  Which is
 * fastest depends on the job and on its state: more resident warps hide the
 * gather's latency on large meshes, more registers per thread help small
 * ones, schedule 3 pays once the cells have formed but does a tile twice
 * while a vertex of it is outside its shape (fronts meeting, crowded
 * junctions), and schedule 4 sits between.  Measured on GB300 in steady
 * state (us a step under schedules 0 / 3 / 4): a 1024^2 torus with 8192
 * cells 84.5 / 76.3 / 81.7, a 150^2 torus with 500 cells 19.6 / 10.0 / 10.2,
 * a level-7 icosphere with 2000 cells 18.3 / 15.3 / 15.8, and a level-8
 * icosphere with 300 cells, its fronts still meeting, 32.6 / 36.5 / 37.6.  Jobs with
 * coefficient matrices always take the general-coefficient kernel at 4 CTAs.
 * lf_set_schedule fixes a job's schedule; lf_schedule reads it (-1 for
 * NULL).  lf_tune is the autotuner: it runs trial_steps time-iterations under
 * each schedule twice (the second round in reverse order), timed with CUDA
 * events on the mesh's stream, keeps the fastest for the job and returns it
 * in *schedule (nullable).  The trial steps advance the job like lf_step
 * (they count in its steps and statistics).  lf_step and lf_step_batch run
 * each job under its schedule; a batch launches once per step for every
 * storage type and schedule present.
 */
lf_status lf_set_schedule(lf_mesh m, int32_t schedule);
int32_t lf_schedule(lf_mesh m);
lf_status lf_tune(lf_mesh m, int32_t trial_steps, int32_t* schedule);

/*
 * Lloyd-like iterations (Sec. 5): `rounds` times, new seeds from the current
 * field, a fresh field from them (as lf_seed) and steps_per_round steps (as
 * lf_step).  A cell is the set of vertices with an entry of its layer; its
 * centre of mass is the area-weighted mean of the barycentres of the faces
 * with at least one cell vertex, and the line through it along the area-
 * weighted mean normal of those faces is intersected with them (both
 * directions; the hit nearest to the centre wins, ties to the lowest face
 * id).  The new seed is the vertex of the hit face nearest to the hit point
 * (ties to the lowest vertex id); a miss, or a zero mean normal, keeps the
 * seed.  When several cells pick one vertex, the cell whose old seed it is
 * keeps it, else the lowest cell id, and the others return to their old
 * seeds (repeated until the seeds are distinct).  Geometry is FP64 on the
 * device; the per-cell sums are FP64 atomics.  seeds_out (nullable) gets the
 * k final seed vertices.  rounds = 0 only reports the seeds.  Needs a mesh
 * made by lf_create_mesh (the geometry) whose field came from lf_seed (or
 * lf_set_field with the same k after lf_seed): else LF_ERR_STATE.  Errors:
 * LF_ERR_INVALID (negative counts), LF_ERR_OOM, LF_ERR_CUDA, and those of
 * lf_step.
 */
lf_status lf_lloyd(lf_mesh m, int32_t rounds, int32_t steps_per_round, int32_t* seeds_out);

/*
 * Dual mesh (Sec. 5.2) of the current partition, with a vertex at each seed.
 * A cell covers vertex v when F(v, c) >= params.iso (FP32 comparison; iso in
 * [1/16, 1], default 0.25).  Cells are adjacent when they cover a common
 * vertex (A_v), or when they cover vertices of a common face and their
 * isolines (level iso, linear on the face) cross there and they do not
 * already share two A_v neighbours (the manifold check).  Every three
 * mutually adjacent cells form a triangle, except the triangle of the three
 * neighbours of a cell that has exactly three mutually adjacent neighbours
 * (a spurious triangle).  Triangles are oriented consistently, breadth-first
 * over shared edges, starting from the first triangle of each connected part
 * oriented along the mesh normals at its seeds.  The mesh passes run on the
 * device; the graph stage over the k cells runs on the host.
 * tris (nullable) receives *n_tris rows of 3 seed vertex ids, in sorted order
 * of their vertex sets; with tris NULL only *n_tris is set.  The result is
 * kept until the field changes, so a size query followed by the copy costs
 * one extraction.  Errors: LF_ERR_INVALID (null n_tris, iso out of range),
 * LF_ERR_STATE (no field, no geometry, unknown seeds), LF_ERR_CAPACITY (cap
 * smaller than *n_tris, which is still set), LF_ERR_OOM, LF_ERR_CUDA.
 */
lf_status lf_extract_dual(lf_mesh m, int32_t* tris, int64_t cap, int64_t* n_tris);

/* ------------------------------------------------------------------------
 * Serving form: continuous batching of tessellation jobs.
 *
 * A server owns one CUDA stream and one scheduler thread.  lf_server_submit
 * validates a job (mesh, seeds, step count, parameters), builds its cotangent
 * operator on the calling thread and queues it; nothing is put on the device
 * yet.  The scheduler admits queued jobs in arrival order while fewer than
 * max_active jobs run and the estimated device bytes of the admitted jobs
 * stay within hbm_budget_bytes (a job larger than the whole budget fails with
 * LF_ERR_OOM), puts each one on the device (its operator, and its geometry
 * when it asked for Lloyd-like rounds or the dual mesh) and seeds it (as
 * lf_seed), and advances all running jobs together with lf_step_batch in
 * chunks of chunk_steps.  A job asking for Lloyd-like rounds (Sec. 5) gets,
 * each time it has taken its n_iters steps, a seed update and a fresh field,
 * and another n_iters steps in the batches; a job asking for the dual mesh
 * (Sec. 5.2) gets it at the end.  A finished job gets its sharp labels
 * (Sec. 6) copied to the host and its device memory freed; admission then
 * runs again.  A job that fails (e.g. a vertex summing to zero) is retired
 * with its status; the others continue.  The paper runs one mesh at a time;
 * this runtime has no counterpart there.
 * ------------------------------------------------------------------------ */
typedef struct lf_server_s* lf_server;

typedef struct {
  int64_t hbm_budget_bytes;  /* device bytes the running jobs may hold (default 150e9)   */
  int32_t max_active;        /* jobs advanced together, 1..64 (default 64)               */
  int32_t chunk_steps;       /* steps between admission rounds, >= 1 (default 256)      */
} lf_server_params;

typedef enum { LF_JOB_QUEUED = 0, LF_JOB_RUNNING = 1, LF_JOB_DONE = 2, LF_JOB_FAILED = 3 } lf_job_state;

typedef struct {
  int32_t state;             /* lf_job_state                                             */
  int32_t status;            /* LF_OK, or the lf_status a failed job ended with         */
  int64_t n_v;
  int64_t steps;             /* n_iters of the job                                       */
  int64_t steps_done;
  int64_t arrival_ns;        /* CLOCK_MONOTONIC, as given to lf_server_submit            */
  int64_t admit_ns;          /* when the scheduler put the job on the device (0: not yet) */
  int64_t finish_ns;         /* when its labels were on the host (0: not yet)            */
  uint64_t skeleton_total;   /* nnz-updates of the job, all rounds                       */
  int64_t device_bytes;      /* device bytes the job held at the end                     */
  int32_t lloyd_rounds;      /* Lloyd-like rounds asked for                              */
  int32_t lloyd_done;        /* rounds completed                                         */
  int64_t dual_triangles;    /* triangles of the dual mesh (-1: not asked for or not yet) */
} lf_job_info;

typedef struct {
  int64_t submitted, done, failed, queued, running;
  int64_t bytes_in_use, peak_bytes;   /* device bytes of the running jobs                */
  int64_t peak_running;
  int64_t batches;                    /* lf_step_batch calls made                        */
  int64_t busy_ns;                    /* scheduler time spent with running jobs          */
  uint64_t skeleton_total;            /* nnz-updates of the finished jobs                */
} lf_server_stats_t;

void lf_server_default_params(lf_server_params* p);

/* Creates a server on the current CUDA device.  dev may be NULL; its
 * cuda_stream is ignored (the server makes its own) and its allocation hooks
 * are used from the scheduler thread when set.  Errors: LF_ERR_INVALID (bad
 * parameters), LF_ERR_CUDA (no device, stream creation). */
lf_status lf_server_create(const lf_device* dev, const lf_server_params* sp, lf_server* out);

/* Queues one job.  V (n_v x 3 doubles), F (n_f x 3 int32), seeds (k int32),
 * params (NULL: defaults) are caller-owned and copied before the call returns.
 * The job takes n_iters steps, then lloyd_rounds times a seed update and
 * n_iters more steps (as lf_lloyd(m, lloyd_rounds, n_iters)), then, with
 * extract_dual != 0, the dual mesh (as lf_extract_dual).  arrival_ns is the
 * job's arrival time on CLOCK_MONOTONIC (0: now); latency is finish_ns -
 * arrival_ns.  *job_id gets a positive id.  Errors: LF_ERR_INVALID for any
 * input lf_create_mesh or lf_seed would reject, or n_iters or lloyd_rounds
 * < 0; LF_ERR_STATE after lf_server_destroy began. */
lf_status lf_server_submit(lf_server s, const double* V, int64_t n_v, const int32_t* F, int64_t n_f,
                           const int32_t* seeds, int32_t k, int32_t n_iters, int32_t lloyd_rounds,
                           int32_t extract_dual, const lf_params* params, int64_t arrival_ns, int64_t* job_id);

/* Waits up to timeout_s seconds (0: just looks) for the job to finish and
 * fills *info.  When it is done and labels is not NULL, its n_v labels are
 * copied there.  With release != 0 a finished job's record is dropped after
 * the copy (its id becomes unknown).  Returns LF_OK once the job is done,
 * LF_ERR_TIMEOUT while it is queued or running (info filled), the job's own
 * status when it failed, LF_ERR_INVALID for an unknown id. */
lf_status lf_server_wait(lf_server s, int64_t job_id, double timeout_s, lf_job_info* info, int32_t* labels,
                         int32_t release);

/* The dual mesh of a finished job that asked for it, as lf_extract_dual
 * (tris NULL: only *n_tris).  Errors: LF_ERR_INVALID (unknown id), LF_ERR_STATE
 * (not finished, or no dual mesh asked for), LF_ERR_CAPACITY (cap < *n_tris). */
lf_status lf_server_dual_mesh(lf_server s, int64_t job_id, int32_t* tris, int64_t cap, int64_t* n_tris);

/* Waits up to timeout_s seconds until no job is queued or running.  Returns
 * LF_OK or LF_ERR_TIMEOUT. */
lf_status lf_server_drain(lf_server s, double timeout_s);

lf_status lf_server_stats(lf_server s, lf_server_stats_t* out);

/* Stops the scheduler after its current chunk, fails the jobs still queued or
 * running (LF_ERR_STATE), frees all device memory and the handle. */
void lf_server_destroy(lf_server s);

#ifdef __cplusplus
}
#endif

#endif /* LF_H */
