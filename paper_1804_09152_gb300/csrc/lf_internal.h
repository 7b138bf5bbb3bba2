// Internal layout shared by the host code (lf_host.cpp) and the kernels
// (lf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lf {

// Error bits raised on the device (DevStatus::err).
enum : uint32_t {
  ERR_CAPACITY = 1u,   // the output field would exceed the buffer capacity
  ERR_MAP = 2u,        // a vertex's layer union exceeded the map slots
  ERR_TIMEOUT = 4u,    // a bounded wait in the decoupled look-back gave up
  ERR_ZERO_SUM = 8u,   // a vertex summed to zero before normalisation
};

// Per-mesh device status.  The step kernel reads err and epoch at entry; the
// last CTA of a successful step advances epoch, which selects the buffer that
// holds the current field (buf[epoch & 1]).
struct DevStatus {
  uint32_t err;
  uint32_t epoch;
  uint32_t ticket;                    // next tile of the running step
  uint32_t done;                      // CTAs finished in the running step
  unsigned long long need_nnz;        // capacity asked for by failing tiles
  uint32_t need_map;                  // nonzero when ERR_MAP was raised
  uint32_t pad0;
  unsigned long long skeleton_total;  // sum of |skeleton| over completed steps
  unsigned long long skeleton_step;   // running step, summed over tiles
  unsigned long long nnz_io_total;    // sum of nnz(in) + nnz(out), completed steps
  unsigned long long pad1;
};
static_assert(sizeof(DevStatus) == 64, "DevStatus layout");

// One CSR copy of the field: rows = vertices, entries sorted by layer id.
struct FieldBuf {
  int32_t* rowptr;   // n_v + 1
  uint16_t* ids;     // capacity
  void* vals;        // capacity values of the storage type
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
  int32_t cap;               // entries per field buffer
  const int32_t* L_rowptr;   // n_v + 1, off-diagonal entries only
  const int2* L_colval;      // (column, float bits of L_ij), j != i
  FieldBuf buf[2];
  DevStatus* st;
  unsigned long long* tile_status;   // num_tiles look-back words
  Coefs c;
  int32_t pad[3];
};

// Step kernel variants: map slots per vertex and threads per CTA.
struct StepTier {
  int map_slots;
  int block;
};
constexpr int kNumTiers = 3;
extern const StepTier kTiers[kNumTiers];

// Returns the kernel entry for (dtype, tier) and its dynamic shared memory.
const void* step_kernel(int dtype, int tier, size_t* smem_bytes);
// Sets the shared-memory attribute of every step kernel variant.
cudaError_t init_kernels();

cudaError_t launch_step(const JobDesc* d_job, int num_tiles, int dtype, int tier, cudaStream_t s);
cudaError_t launch_seed(const JobDesc* d_job, int n_v, int k, const int32_t* d_seeds, int dtype,
                        cudaStream_t s);
cudaError_t launch_labels(const JobDesc* d_job, int n_v, int dtype, int32_t* d_labels, float* d_maxval,
                          cudaStream_t s);
// Converts between the storage type and float on the device.
cudaError_t launch_widen(const void* src, float* dst, int64_t n, int dtype, cudaStream_t s);
cudaError_t launch_narrow(const float* src, void* dst, int64_t n, int dtype, cudaStream_t s);

inline int value_bytes(int dtype) { return dtype == 0 ? 4 : 2; }

}  // namespace lf
