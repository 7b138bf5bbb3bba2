// lf_step_noalloc: one time-iteration for callers that cannot allocate.
//
// The regular entry points allocate the field buffers and the step's status
// words with cudaMalloc (or the lf_device hooks).  Some callers own every byte
// of device memory themselves -- a framework with its own pool, a service that
// allocates only at start-up, code running where allocation is not allowed --
// and pass in all inputs and outputs.  For them the step kernel's scratch (the
// status and counter words it updates) lives in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
// Nothing here calls cudaMalloc, cudaFree or any allocating routine.  The job
// descriptor itself travels in the launch parameters.

#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/lf.h"
#include "lf_internal.h"

namespace {

// Scratch of the step kernel: its status and counter words.
constexpr size_t kScratchBytes = 1024;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct ScratchLayout {
  lf::DevStatus st;
};
static_assert(sizeof(ScratchLayout) <= kScratchBytes, "scratch too small");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
lf_status noalloc_fail(lf_status s, const std::string& msg) {
  lf::set_last_error(msg);      // read back with lf_last_error(NULL)
  return s;
}

// Device address of the scratch on the current device, looked up once per
// device (the host-side name g_scratch is not a device address).
lf_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(LF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LF_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(LF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return LF_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

lf_status lf_step_noalloc(void* cuda_stream, int32_t n_v, int32_t n_layers, const int32_t* d_L_rowptr,
                          const int32_t* d_L_colval, const int32_t* d_rows_in, const int32_t* d_head_in,
                          const uint16_t* d_ids_in, const float* d_vals_in, int32_t* d_rows_out,
                          int32_t* d_head_out, uint16_t* d_ids_out, float* d_vals_out, int32_t tile_cap,
                          const lf_params* params, int64_t* nnz_out, int64_t* need_tile_cap) {
  if (!d_L_rowptr || !d_L_colval || !d_rows_in || !d_head_in || !d_ids_in || !d_vals_in || !d_rows_out ||
      !d_head_out || !d_ids_out || !d_vals_out)
    return noalloc_fail(LF_ERR_INVALID, "null device pointer");
  if (n_v < 1 || n_v > 2147483647 - lf::kTile) return noalloc_fail(LF_ERR_INVALID, "n_v out of range");
  if (n_layers < 2 || n_layers > 65536) return noalloc_fail(LF_ERR_INVALID, "n_layers must be in [2, 65536]");
  if (tile_cap < lf::kTile || tile_cap % 16 != 0)
    return noalloc_fail(LF_ERR_INVALID, "tile_cap must be a multiple of 16 and at least 256");
  const int64_t tiles = (static_cast<int64_t>(n_v) + lf::kTile - 1) / lf::kTile;
  if (tiles * tile_cap > 2147483647LL)
    return noalloc_fail(LF_ERR_CAPACITY, "tiles * tile_cap exceeds 2^31 - 1 entries");
  if (!aligned(d_L_colval, 8) || !aligned(d_rows_in, 8) || !aligned(d_rows_out, 8))
    return noalloc_fail(LF_ERR_INVALID, "L_colval and the row arrays must be 8-byte aligned");
  if (!aligned(d_head_in, 16) || !aligned(d_head_out, 16))
    return noalloc_fail(LF_ERR_INVALID, "the head arrays must be 16-byte aligned");
  lf_params p;
  lf_default_params(&p);
  if (params) p = *params;
  std::string why;
  if (!lf::params_valid(p, why)) return noalloc_fail(LF_ERR_INVALID, "lf_step_noalloc: " + why);
  if (p.field_dtype != LF_F32) return noalloc_fail(LF_ERR_INVALID, "lf_step_noalloc stores FP32 values only");
  // the kernel computes in FP32: every parameter must stay finite there
  const double as_float[] = {p.dt, p.mu, p.w_cc, p.w_cb, p.a_cc, p.a_cb, p.e_cc, p.e_cb, p.e_bc};
  for (double x : as_float)
    if (!std::isfinite(static_cast<float>(x)))
      return noalloc_fail(LF_ERR_INVALID, "lf_step_noalloc: a parameter overflows FP32");

  void* base = nullptr;
  lf_status s = scratch_address(&base);
  if (s != LF_OK) return s;
  auto* d_layout = static_cast<ScratchLayout*>(base);

  lf::BatchParams bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.n_jobs = 1;
  bp.step = 0;
  bp.tile_start[0] = 0;
  bp.tile_start[1] = static_cast<int32_t>(tiles);
  lf::JobDesc& job = bp.job[0];
  job.n_v = n_v;
  job.n_layers = n_layers;
  job.num_tiles = static_cast<int32_t>(tiles);
  job.tile_cap = tile_cap;
  job.parity0 = 0;                                // buf[0] is the input, buf[1] the output
  job.steps = 1;
  job.L_rowptr = d_L_rowptr;
  job.L_colval = reinterpret_cast<const int2*>(d_L_colval);
  job.buf[0] = lf::FieldBuf{const_cast<int2*>(reinterpret_cast<const int2*>(d_rows_in)),
                            const_cast<int4*>(reinterpret_cast<const int4*>(d_head_in)),
                            const_cast<uint16_t*>(d_ids_in), const_cast<float*>(d_vals_in)};
  job.buf[1] = lf::FieldBuf{reinterpret_cast<int2*>(d_rows_out), reinterpret_cast<int4*>(d_head_out), d_ids_out,
                            d_vals_out};
  job.st = &d_layout->st;
  job.L_nnz = INT32_MAX;                          // not known here: no operator bound
  job.c = lf::Coefs{static_cast<float>(p.dt),   static_cast<float>(p.mu),   static_cast<float>(p.w_cc),
                    static_cast<float>(p.w_cb), static_cast<float>(p.a_cc), static_cast<float>(p.a_cb),
                    static_cast<float>(p.e_cc), static_cast<float>(p.e_cb), static_cast<float>(p.e_bc)};
  // the status words start at zero; nnz is the input's (known after the step)
  lf::DevStatus h;
  std::memset(&h, 0, sizeof(h));

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemcpyAsync(&d_layout->st, &h, sizeof(h), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = lf::launch_step(bp, lf::step_kind(LF_F32, lf::kSched4), stream);
  lf::DevStatus st;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, &d_layout->st, sizeof(st), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(LF_ERR_CUDA, std::string("lf_step_noalloc: ") + cudaGetErrorString(e));
  }
  if (need_tile_cap) *need_tile_cap = static_cast<int64_t>(st.need_tile);
  if (st.err & lf::ERR_CAPACITY)
    return noalloc_fail(LF_ERR_CAPACITY, "a tile's output exceeds tile_cap; *need_tile_cap entries are needed");
  if (st.err & lf::ERR_BOUNDS)
    return noalloc_fail(LF_ERR_STATE, "an index left its array (reported by a checked build)");
  if (st.err != 0u) return noalloc_fail(LF_ERR_STATE, "a vertex summed to zero before normalisation");
  if (nnz_out) *nnz_out = static_cast<int64_t>(st.nnz);
  return LF_OK;
}

}  // extern "C"
