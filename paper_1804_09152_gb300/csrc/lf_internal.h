// Internal layout shared by the host code (lf_host.cpp) and the kernels
// (lf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace lf {

// Error bits raised on the device (DevStatus::err).
enum : uint32_t {
  ERR_CAPACITY = 1u,   // a tile's output would exceed its segment of the field buffer
  ERR_ZERO_SUM = 8u,   // a vertex summed to zero before normalisation
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
// and vals.  rows[i] = (start, count) of row i.
struct FieldBuf {
  int2* rows;        // n_v
  uint16_t* ids;     // num_tiles * tile_cap
  void* vals;        // num_tiles * tile_cap values of the storage type
};

struct Coefs {
  float dt, mu, w_cc, w_cb, a_cc, a_cb, e_cc, e_cb, e_bc;
};

// Device-resident job descriptor.  Kernels read it every launch, so the host
// can grow buffers without re-capturing a CUDA graph.
struct JobDesc {
  int32_t n_v;
  int32_t n_layers;          // k + 1; the base layer is n_layers - 1
  int32_t num_tiles;         // CTAs of one step launch
  int32_t tile_cap;          // entries per tile segment (multiple of 16)
  const int32_t* L_rowptr;   // n_v + 1, off-diagonal entries only
  const int2* L_colval;      // (column, float bits of L_ij), j != i
  FieldBuf buf[2];
  DevStatus* st;
  Coefs c;
  int32_t pad[3];
};

constexpr int kTile = 256;   // vertices per tile = threads per step CTA

// Register slots of the step kernel's fast path.
int step_slots();
// Kernel entry of the step for a storage type (0 f32, 1 bf16, 2 f16).
const void* step_kernel(int dtype);
// One step launch with programmatic stream serialisation.
cudaError_t launch_step(const JobDesc* d_job, int num_tiles, int dtype, cudaStream_t s);
cudaError_t launch_seed(const JobDesc* d_job, int n_v, int k, const int32_t* d_seeds, int dtype,
                        cudaStream_t s);
cudaError_t launch_labels(const JobDesc* d_job, int n_v, int dtype, int32_t* d_labels, float* d_maxval,
                          cudaStream_t s);
// Copies the rows of `from` into the segments of `to` (tile_cap may differ).
cudaError_t launch_relayout(const int2* rows_from, const uint16_t* ids_from, const void* vals_from,
                            int cap_from, int2* rows_to, uint16_t* ids_to, void* vals_to, int cap_to,
                            int n_v, int dtype, cudaStream_t s);
// Converts between the storage type and float on the device.
cudaError_t launch_widen(const void* src, float* dst, int64_t n, int dtype, cudaStream_t s);
cudaError_t launch_narrow(const float* src, void* dst, int64_t n, int dtype, cudaStream_t s);

inline int value_bytes(int dtype) { return dtype == 0 ? 4 : 2; }

// Message returned by lf_last_error(NULL) (thread-local).
void set_last_error(const std::string& msg);

}  // namespace lf
