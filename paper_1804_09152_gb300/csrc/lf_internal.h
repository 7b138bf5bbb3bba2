// Internal layout shared by the host code (lf_host.cpp) and the kernels
// (lf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lf.h"

namespace lf {

// NVTX range for the lifetime of a scope (header-only NVTX 3: costs nothing
// unless a profiler is attached), so that a tool can attribute kernels to
// the library call that launched them.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Error bits raised on the device (DevStatus::err).
enum : uint32_t {
  ERR_CAPACITY = 1u,   // a tile's output would exceed its segment of the field buffer
  ERR_ZERO_SUM = 8u,   // a vertex summed to zero before normalisation
  ERR_BOUNDS = 16u,    // an index outside its array (builds with LF_CHECKED only)
};

// Per-mesh device status.  The step kernel reads err and epoch at entry; the
// last CTA of a successful step advances epoch, which selects the buffer that
// holds the current field (buf[epoch & 1]).
struct DevStatus {
  uint32_t err;
  uint32_t epoch;
  uint32_t done;                      // CTAs finished in the running step
  uint32_t pad0;
  unsigned long long need_tile;       // entries asked for by the fullest failing tile
  unsigned long long skeleton_total;  // sum of |skeleton| over completed steps
  unsigned long long skeleton_step;   // running step, summed over tiles
  unsigned long long nnz_io_total;    // sum of nnz(in) + nnz(out), completed steps
  unsigned long long nnz_io_step;     // running step
  unsigned long long nnz_step;        // nnz(out) of the running step
  unsigned long long nnz;             // nnz of the current field
};
static_assert(sizeof(DevStatus) == 72, "DevStatus layout");

// One copy of the field in tile-segmented CSR.  Vertex i belongs to tile
// i / kTile; the rows of a tile are stored one after another, ids ascending
// within a row, in the segment [tile * tile_cap, (tile + 1) * tile_cap) of ids
// and vals.  rows[i] = (start, count) of row i.  head[i] repeats the count
// and the first two entries of row i in one 16-byte record -- (count,
// id0 | id1 << 16, value bits of entry 0, value bits of entry 1), values in
// the storage type's bits, unused parts zero -- so the step kernel reads a
// neighbour's row of one or two entries with a single load.
struct FieldBuf {
  int2* rows;        // n_v
  int4* head;        // n_v
  uint16_t* ids;     // num_tiles * tile_cap
  void* vals;        // num_tiles * tile_cap values of the storage type
};

struct Coefs {
  float dt, mu, w_cc, w_cb, a_cc, a_cb, e_cc, e_cb, e_bc;
};

// One job of a step launch: pointers, sizes and coefficients.  Passed to the
// kernel by value (inside BatchParams), so a launch reads no descriptor from
// memory; the host rebuilds the parameters when anything in it changes.
struct JobDesc {
  int32_t n_v;
  int32_t n_layers;          // k + 1; the base layer is n_layers - 1
  int32_t num_tiles;         // CTAs of this job in one step launch
  int32_t tile_cap;          // entries per tile segment (multiple of 16)
  int32_t parity0;           // the input of launch `step` is buf[(parity0 + step) & 1]
  int32_t steps;             // launches with step >= steps leave this job alone
  const int32_t* L_rowptr;   // n_v + 1, off-diagonal entries only
  const int2* L_colval;      // (column, float bits of L_ij), j != i
  FieldBuf buf[2];
  DevStatus* st;
  // General coefficient matrices (Algorithm 1's w_jl, a_jl, e_jk), dense
  // n_layers x n_layers row-major FP32; null: the class coefficients in c.
  const float* cW;
  const float* cA;
  const float* cE;
  Coefs c;
  int32_t L_nnz;             // entries of L_colval (bounds of the checked build)
};

// Parameters of one step launch: up to kMaxJobs jobs whose tiles are laid
// out one after another in the grid (job j owns CTAs tile_start[j] ..
// tile_start[j + 1] - 1).
constexpr int kMaxJobs = 64;
struct BatchParams {
  int32_t n_jobs;
  int32_t step;
  int32_t tile_start[kMaxJobs + 1];
  int32_t pad;
  JobDesc job[kMaxJobs];
};

constexpr int kTile = 256;   // vertices per tile = threads per step CTA

// Register slots of the step kernel's fast path.
int step_slots();
// Kernel entry of the step for a storage type (0 f32, 1 bf16, 2 f16), in
// the form for general coefficient matrices or not; its only argument is a
// BatchParams.
// Step-kernel schedules: the register allocation of the step kernel for 4,
// 5 or 3 resident CTAs per SM (64, 48 and 80 registers a thread in FP32).  All give
// the same bits; which is fastest depends on the job (its size against the
// GPU, its degree and its cells).
constexpr int kSched4 = 0;      // the default
constexpr int kSched5 = 1;
constexpr int kSched3 = 2;
// The register-tier kernel: a tile whose every vertex holds at most five
// cells and the base layer and sees at most five cells in its closed
// neighbourhood takes a lean path; any other tile takes the full step in the
// same launch.
constexpr int kSchedHot = 3;
// The step kernel with the lean path's gather in its fast tier and, per
// vertex, the other tiers beyond it (at 4 CTAs per SM).
constexpr int kSchedLean = 4;
constexpr int kSchedules = 5;
// A launch kind: the storage type and the schedule of the jobs in one launch.
inline int step_kind(int dtype, int sched) { return dtype + 3 * sched; }
const void* step_kernel(int kind, bool general);
// True when a job of the launch has general coefficient matrices.
bool needs_general(const BatchParams& p);
// One step launch over the jobs in p, with programmatic stream serialisation.
cudaError_t launch_step(const BatchParams& p, int kind, cudaStream_t s);
// The seed and label kernels take one job by value.
cudaError_t launch_seed(const JobDesc& job, int k, const int32_t* d_seeds, int dtype, cudaStream_t s);
cudaError_t launch_labels(const JobDesc& job, int buf, int dtype, int32_t* d_labels, float* d_maxval,
                          cudaStream_t s);
// Region seeds: each seed vertex and its neighbours in L take the seed's
// layer (own seed first, else the lowest seed id); d_owner is n_v scratch.
// Device build of the cotangent operator (lf_cotan.cu).
int64_t cotan_scan_blocks(int64_t n);   // block totals an exclusive scan of n elements needs
// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] = total; block_sum
// holds cotan_scan_blocks(n) entries (at least one).
cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* block_sum, cudaStream_t s);
// Per face: hc[3f + c] = half cotangent of corner c, inc_cnt[v] += 1 per
// corner at v, bad_face = min face index of zero area (left as is if none).
cudaError_t launch_cotan_corners(const double* V, const int32_t* tri, int64_t n_f, double* hc, int32_t* inc_cnt,
                                 unsigned long long* bad_face, cudaStream_t s);
// Per face: inc[inc_start[v] + k] = f for each corner v (fill: zeroed counters).
cudaError_t launch_cotan_incidence(const int32_t* tri, int64_t n_f, const int32_t* inc_start, int32_t* fill,
                                   int32_t* inc, cudaStream_t s);
// Per vertex: pass 0 sorts its face list and writes its neighbour count to
// cnt; pass 1 writes (column, FP32 bits) at rowptr[i] in column order.
cudaError_t launch_cotan_rows(const int32_t* tri, const double* hc, int64_t n_v, const int32_t* inc_start,
                              int32_t* inc, int pass, int32_t* cnt, const int32_t* rowptr, int2* colval,
                              cudaStream_t s);

cudaError_t launch_seed_regions(const JobDesc& job, int k, const int32_t* d_seeds, unsigned* d_owner, int dtype,
                                cudaStream_t s);
// head[] of a field buffer from its rows, ids and vals.
cudaError_t launch_build_head(const FieldBuf& b, int n_v, int dtype, cudaStream_t s);
// Copies the rows of `from` into the segments of `to` (tile_cap may differ).
cudaError_t launch_relayout(const int2* rows_from, const uint16_t* ids_from, const void* vals_from,
                            int cap_from, int2* rows_to, uint16_t* ids_to, void* vals_to, int cap_to,
                            int n_v, int dtype, cudaStream_t s);
// Converts between the storage type and float on the device.
cudaError_t launch_widen(const void* src, float* dst, int64_t n, int dtype, cudaStream_t s);
cudaError_t launch_narrow(const float* src, void* dst, int64_t n, int dtype, cudaStream_t s);

inline int value_bytes(int dtype) { return dtype == 0 ? 4 : 2; }

// Device scratch of one Lloyd-like seed update (k cells, n_v vertices).
struct LloydScratch {
  double* acc;                  // k * 7: area, area * barycentre, area * normal
  double* frame;                // k * 7: centre of mass, unit direction, valid
  unsigned long long* best;     // k * 2: nearest |s| (bits), its lowest face id
  unsigned long long* owner;    // n_v: conflict resolution
  int32_t* rounds;              // 1: rounds the resolution took
};
// New seeds (Sec. 5) from the field in job.buf[buf]: V (n_v x 3 FP64) and tri
// (n_f x 3) are the mesh; old_seed and new_seed hold k vertex ids on the device.
cudaError_t launch_lloyd(const JobDesc& job, int buf, const double* V, const int32_t* tri, int n_f, int k,
                         const int32_t* old_seed, int32_t* new_seed, LloydScratch sc, cudaStream_t s);

// Message returned by lf_last_error(NULL) (thread-local).
void set_last_error(const std::string& msg);

// Device scratch of one dual-mesh extraction (k cells, n_v vertices).
struct DualScratch {
  uint32_t* Hv;         // cap: hash set of the pairs covering a common vertex
  uint32_t* Hc;         // cap: hash set of the face-only pairs whose isolines cross
  uint32_t cap;         // power of two
  uint32_t* out_v;      // cap: compacted Hv
  uint32_t* out_c;      // cap: compacted Hc
  uint32_t* counters;   // 4: overflow, |out_v|, |out_c|, unused
  int32_t* cell_of;     // n_v: cell whose seed a vertex is, or -1
  double* nrm;          // k * 3: mesh normal (area weighted) at each seed vertex
  double* pos;          // k * 3: seed positions
};
// Mesh passes of the dual extraction (Sec. 5.2) on the field in job.buf[buf].
cudaError_t launch_dual(const JobDesc& job, int buf, int dtype, const double* V, const int32_t* tri, int n_f, int k,
                        float iso, const int32_t* d_seeds, DualScratch sc, cudaStream_t s);

// Host helpers shared with the serving runtime (lf_server.cpp).
// Cotangent operator of a triangle mesh as off-diagonal FP64 CSR; false (with
// a reason) on a zero-area face.
bool cotan_offdiag(int64_t n_v, const double* V, int64_t n_f, const int32_t* F, std::vector<int64_t>& rp,
                   std::vector<int32_t>& col, std::vector<double>& val, std::string& why);
// Checks faces (in range, no repeated vertex) and coordinates (finite).
bool mesh_ok(int64_t n_v, const double* V, int64_t n_f, const int32_t* F, std::string& why);
// Checks seeds: 1 <= k <= 65535, in range, no vertex twice.
bool seeds_ok(int64_t n_v, const int32_t* seeds, int32_t k, std::string& why);
// Validates parameters as lf_create_mesh does.
bool params_valid(const lf_params& p, std::string& why);
// lf_create_mesh from a prepared off-diagonal operator.
lf_status create_from_offdiag(const lf_device* dev, int64_t n_v, const std::vector<int64_t>& rp,
                              const std::vector<int32_t>& col, const std::vector<double>& val,
                              const lf_params& prm, lf_mesh* out);
// Uploads a mesh's vertices and faces (the Lloyd-like update and the dual
// mesh need them).
lf_status attach_geometry(lf_mesh m, const double* V, int64_t n_v, const int32_t* F, int64_t n_f);
// Device bytes the geometry, the Lloyd scratch and the dual-mesh scratch add.
int64_t geometry_bytes_estimate(int64_t n_v, int64_t n_f, int64_t k);
// Device bytes lf_create_mesh would allocate for this operator and parameters.
int64_t device_bytes_estimate(int64_t n_v, int64_t nnz_off, const lf_params& prm);

}  // namespace lf
