// Host side of the layered-field library: mesh validation, the host builder
// of the cotangent operator (used by the serving path; lf_create_mesh builds
// it on the device, lf_cotan.cu), device buffers, the step driver (CUDA
// graphs, overflow recovery), the Lloyd-like and dual-mesh drivers and the C
// ABI of lf.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <deque>
#include <unordered_map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>
#include <atomic>
#include <thread>

#include "../../include/lf.h"
#include "lf_internal.h"

namespace {

thread_local std::string g_create_error;

constexpr int kGraphSteps = 128;     // kernel nodes per captured graph
constexpr int kPollSteps = 512;      // steps between status checks in lf_step
constexpr int64_t kMaxCap = 2147483000LL;
constexpr int kMaxCoefLayers = 4096;  // dense coefficient matrices: at most 64 MiB each

struct Alloc {
  void* p;
  size_t bytes;
};

}  // namespace

struct lf_mesh_s {
  lf_device dev{};
  cudaStream_t stream = nullptr;
  lf_params params{};
  int64_t n_v = 0;
  int64_t L_nnz = 0;
  int dtype = 0;
  int sched = lf::kSched4;       // step-kernel schedule (lf_set_schedule, lf_tune)
  int n_layers = 0;
  int num_tiles = 0;
  int64_t tile_cap = 0;          // entries per tile segment
  int64_t steps = 0;
  int retries = 0;
  bool poisoned = false;
  std::string err;
  int64_t device_bytes = 0;
  std::vector<Alloc> allocs;

  int32_t* d_Lrp = nullptr;
  int2* d_Lcv = nullptr;
  lf::FieldBuf buf[2]{};
  lf::DevStatus* d_st = nullptr;
  lf::JobDesc h_job{};
  lf::DevStatus h_st{};
  int32_t* d_labels = nullptr;
  float* d_scratch_f = nullptr;
  int64_t scratch_f_len = 0;

  cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // step graphs by starting parity
  lf::BatchParams gparams[2]{};                     // the launch parameters each was built with
  int gkind[2] = {-1, -1};                          // and the launch kind

  // general coefficient matrices (lf_set_coefficients): one device block of
  // up to three n_layers x n_layers FP32 matrices for that layer count
  float* d_coef = nullptr;
  int coef_layers = 0;

  // geometry (lf_create_mesh only) and seeds, for the Lloyd-like update
  double* d_V = nullptr;         // n_v x 3
  int32_t* d_tri = nullptr;      // n_f x 3
  int64_t n_f = 0;
  std::vector<int32_t> seeds;    // current seed vertex of each cell (empty: unknown)
  int32_t* d_seed_old = nullptr;
  int32_t* d_seed_new = nullptr;
  lf::LloydScratch lloyd{};
  int64_t lloyd_k = 0;
  // dual-mesh extraction: device scratch and the last result
  lf::DualScratch dual{};
  int64_t dual_k = 0;
  int32_t* d_dual_seeds = nullptr;
  int64_t version = 0;           // bumped whenever the field is replaced (lf_seed, lf_set_field)
  int64_t dual_version = -1, dual_steps = -1;
  std::vector<int32_t> dual_tris;

  ~lf_mesh_s() {
    cudaStreamSynchronize(stream);
    for (auto& g : gexec)
      if (g) cudaGraphExecDestroy(g);
    for (auto& a : allocs) release(a.p);
  }

  int64_t buffer_entries() const { return static_cast<int64_t>(num_tiles) * tile_cap; }

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (dev.alloc && dev.free) {
      p = dev.alloc(bytes, dev.cuda_stream, dev.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) {
      allocs.push_back({p, bytes});
      device_bytes += static_cast<int64_t>(bytes);
    }
    return p;
  }

  void release(void* p) {
    if (!p) return;
    if (dev.alloc && dev.free) dev.free(p, dev.user);
    else cudaFree(p);
  }

  void dfree(void* p) {
    if (!p) return;
    for (size_t i = 0; i < allocs.size(); ++i) {
      if (allocs[i].p == p) {
        device_bytes -= static_cast<int64_t>(allocs[i].bytes);
        allocs.erase(allocs.begin() + static_cast<std::ptrdiff_t>(i));
        break;
      }
    }
    release(p);
  }
};

namespace {

lf_status fail(lf_mesh m, lf_status s, const std::string& msg) {
  if (m) m->err = msg;
  else g_create_error = msg;
  return s;
}

// A failed CUDA call poisons the handle.  The runtime's per-thread error slot
// is cleared so that it does not surface in a later, unrelated call.
lf_status cuda_fail(lf_mesh m, cudaError_t e, const char* where) {
  cudaGetLastError();
  if (m) m->poisoned = true;
  return fail(m, LF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LF_CUDA(m, call)                                    \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((m), e_, #call); \
  } while (0)

bool params_ok(const lf_params& p, std::string& why) {
  if (!(p.dt > 0.0) || !std::isfinite(p.dt)) { why = "dt must be positive"; return false; }
  if (!(p.mu >= 0.0) || !std::isfinite(p.mu)) { why = "mu must be >= 0"; return false; }
  const double cs[] = {p.w_cc, p.w_cb, p.a_cc, p.a_cb, p.e_cc, p.e_cb, p.e_bc, p.iso};
  for (double c : cs)
    if (!std::isfinite(c)) { why = "coefficients must be finite"; return false; }
  if (p.field_dtype < 0 || p.field_dtype > 2) { why = "unknown field_dtype"; return false; }
  if (p.reserved != 0) { why = "reserved must be 0"; return false; }
  if (p.initial_capacity < 0 || p.initial_capacity >= kMaxCap) { why = "initial_capacity out of range"; return false; }
  return true;
}

// Runs fn(lo, hi) over [0, n) split among up to 16 host threads (one thread
// below `grain` items).
template <class Fn>
void parallel_for(int64_t n, int64_t grain, Fn fn) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t nt = std::min<int64_t>({static_cast<int64_t>(std::min(hw, 16u)), (n + grain - 1) / grain});
  if (nt <= 1) {
    fn(int64_t{0}, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(static_cast<size_t>(nt));
  for (int64_t t = 0; t < nt; ++t) th.emplace_back(fn, n * t / nt, n * (t + 1) / nt);
  for (auto& x : th) x.join();
}

// Cotangent weights: for the corner p of triangle (p, q, s), the edge (q, s)
// receives cot(angle at p) / 2.  Returns false on a zero-area face.  The
// per-face and per-vertex passes run on host threads; every sum is taken in
// face order, so the result does not depend on the thread count.
bool cotan_rows(int64_t n_v, const double* V, int64_t n_f, const int32_t* F,
                std::vector<int64_t>& rp, std::vector<int32_t>& col, std::vector<double>& val,
                std::string& why) {
  // half cotangent of each corner
  std::vector<double> hc(3 * static_cast<size_t>(n_f));
  std::atomic<int64_t> first_bad{n_f};
  parallel_for(n_f, 1 << 15, [&](int64_t lo, int64_t hi) {
    for (int64_t f = lo; f < hi; ++f) {
      const int32_t v[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
      for (int c = 0; c < 3; ++c) {
        const double* P = V + 3 * static_cast<int64_t>(v[c]);
        const double* Q = V + 3 * static_cast<int64_t>(v[(c + 1) % 3]);
        const double* S = V + 3 * static_cast<int64_t>(v[(c + 2) % 3]);
        const double ux = Q[0] - P[0], uy = Q[1] - P[1], uz = Q[2] - P[2];
        const double wx = S[0] - P[0], wy = S[1] - P[1], wz = S[2] - P[2];
        const double cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
        const double twice_area = std::sqrt(cx * cx + cy * cy + cz * cz);
        if (!(twice_area > 0.0) || !std::isfinite(twice_area)) {
          int64_t cur = first_bad.load();
          while (f < cur && !first_bad.compare_exchange_weak(cur, f)) {
          }
          hc[3 * static_cast<size_t>(f) + c] = 0.0;
          continue;
        }
        hc[3 * static_cast<size_t>(f) + c] = 0.5 * (ux * wx + uy * wy + uz * wz) / twice_area;
      }
    }
  });
  if (first_bad.load() < n_f) {
    why = "face " + std::to_string(first_bad.load()) + " has zero area";
    return false;
  }
  // contributions per vertex, in face order: corner p of face f adds its
  // half cotangent to the edge between the other two corners, at both ends
  std::vector<int64_t> start(static_cast<size_t>(n_v) + 1, 0);
  for (int64_t f = 0; f < n_f; ++f)
    for (int c = 0; c < 3; ++c) start[static_cast<size_t>(F[3 * f + c]) + 1] += 2;
  for (int64_t i = 0; i < n_v; ++i) start[i + 1] += start[i];
  std::vector<std::pair<int32_t, double>> ent(static_cast<size_t>(start[n_v]));
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t f = 0; f < n_f; ++f) {
      const int32_t v[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
      for (int c = 0; c < 3; ++c) {
        const int32_t q = v[(c + 1) % 3], t = v[(c + 2) % 3];
        const double h = hc[3 * static_cast<size_t>(f) + c];
        ent[static_cast<size_t>(fill[q]++)] = {t, h};
        ent[static_cast<size_t>(fill[t]++)] = {q, h};
      }
    }
  }
  // per vertex: sort by column (stable: equal columns keep face order), sum
  // duplicates; then the offsets and the copy
  std::vector<int64_t> uniq(static_cast<size_t>(n_v), 0);
  parallel_for(n_v, 1 << 14, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      auto b = ent.begin() + start[i], e = ent.begin() + start[i + 1];
      std::stable_sort(b, e, [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
        return x.first < y.first;
      });
      int64_t n = 0;
      for (auto it = b; it != e;) {
        auto jt = it;
        double w = 0.0;
        while (jt != e && jt->first == it->first) { w += jt->second; ++jt; }
        *(b + n) = {it->first, w};       // compacted in place: n never passes it
        ++n;
        it = jt;
      }
      uniq[static_cast<size_t>(i)] = n;
    }
  });
  rp.assign(static_cast<size_t>(n_v) + 1, 0);
  for (int64_t i = 0; i < n_v; ++i) rp[static_cast<size_t>(i) + 1] = rp[static_cast<size_t>(i)] + uniq[static_cast<size_t>(i)];
  col.resize(static_cast<size_t>(rp[static_cast<size_t>(n_v)]));
  val.resize(col.size());
  parallel_for(n_v, 1 << 14, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      for (int64_t k = 0; k < uniq[static_cast<size_t>(i)]; ++k) {
        const auto& x = ent[static_cast<size_t>(start[i] + k)];
        col[static_cast<size_t>(rp[static_cast<size_t>(i)] + k)] = x.first;
        val[static_cast<size_t>(rp[static_cast<size_t>(i)] + k)] = x.second;
      }
  });
  return true;
}


// Launch parameters for `steps` steps of this mesh alone, starting from the
// current buffer.
lf::BatchParams single_job_params(lf_mesh m, int steps) {
  lf::BatchParams p;
  std::memset(&p, 0, sizeof(p));
  p.n_jobs = 1;
  p.step = 0;
  p.tile_start[0] = 0;
  p.tile_start[1] = m->num_tiles;
  p.job[0] = m->h_job;
  p.job[0].parity0 = static_cast<int32_t>(m->h_st.epoch & 1u);
  p.job[0].steps = steps;
  return p;
}

lf_status upload_status(lf_mesh m) {
  LF_CUDA(m, cudaMemcpyAsync(m->d_st, &m->h_st, sizeof(lf::DevStatus), cudaMemcpyHostToDevice, m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  return LF_OK;
}

lf_status read_status(lf_mesh m) {
  LF_CUDA(m, cudaMemcpyAsync(&m->h_st, m->d_st, sizeof(lf::DevStatus), cudaMemcpyDeviceToHost, m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  return LF_OK;
}

// Clears the error state and the per-step counters after a failed step.
lf_status reset_after_failure(lf_mesh m) {
  lf::DevStatus& s = m->h_st;
  s.err = 0;
  s.done = 0;
  s.need_tile = 0;
  s.skeleton_step = 0;
  s.nnz_io_step = 0;
  s.nnz_step = 0;
  return upload_status(m);
}

int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }

// Gives every tile segment new_cap entries.  With keep, the current field is
// moved into the new segments on the device (rows keep their order).
lf_status set_tile_cap(lf_mesh m, int64_t new_cap, bool keep) {
  new_cap = round16(std::max<int64_t>(new_cap, lf::kTile));
  const int64_t entries = static_cast<int64_t>(m->num_tiles) * new_cap;
  if (entries > kMaxCap) return fail(m, LF_ERR_CAPACITY, "field exceeds 2^31 entries");
  const int vb = lf::value_bytes(m->dtype);
  const int cur = static_cast<int>(m->h_st.epoch & 1u);
  void* ids[2] = {nullptr, nullptr};
  void* vals[2] = {nullptr, nullptr};
  for (int b = 0; b < 2; ++b) {
    ids[b] = m->dalloc(sizeof(uint16_t) * static_cast<size_t>(entries));
    vals[b] = m->dalloc(static_cast<size_t>(vb) * static_cast<size_t>(entries));
    if (!ids[b] || !vals[b]) {
      for (int c = 0; c <= b; ++c) { m->dfree(ids[c]); m->dfree(vals[c]); }
      return fail(m, LF_ERR_OOM, "growing the field buffers");
    }
  }
  if (keep && m->buf[cur].ids) {
    LF_CUDA(m, lf::launch_relayout(m->buf[cur].rows, m->buf[cur].ids, m->buf[cur].vals,
                                   static_cast<int>(m->tile_cap), m->buf[cur].rows,
                                   static_cast<uint16_t*>(ids[cur]), vals[cur], static_cast<int>(new_cap),
                                   static_cast<int>(m->n_v), m->dtype, m->stream));
  }
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  for (int b = 0; b < 2; ++b) {
    m->dfree(m->buf[b].ids);
    m->dfree(m->buf[b].vals);
    m->buf[b].ids = static_cast<uint16_t*>(ids[b]);
    m->buf[b].vals = vals[b];
    m->h_job.buf[b] = m->buf[b];
  }
  m->tile_cap = new_cap;
  m->h_job.tile_cap = static_cast<int32_t>(new_cap);
  return LF_OK;
}

// Why a step failed for good (the device error bits other than capacity).
const char* failed_step_message(uint32_t err) {
  if (err & lf::ERR_BOUNDS) return "an index left its array (reported by a checked build)";
  return "a vertex summed to zero before normalisation";
}

// A graph of independent chains, each of kGraphSteps step launches of one
// launch kind -- storage type and schedule -- (chain c launches
// chains[c].second with step = 0, 1, ...).
// Within a chain each launch is joined to the previous one by a programmatic
// edge: it may start its CTAs while the previous one drains, and waits inside
// the kernel (griddepcontrol.wait) before it reads the previous step's output.
cudaError_t make_step_graph(const std::vector<std::pair<int, lf::BatchParams>>& chains, cudaGraphExec_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  std::vector<lf::BatchParams> params;
  params.reserve(chains.size() * kGraphSteps);
  for (size_t c = 0; c < chains.size() && e == cudaSuccess; ++c) {
    const int kind = chains[c].first;
    cudaGraphNode_t prev = nullptr;
    for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) {
      params.push_back(chains[c].second);
      params.back().step = s;
      void* args[1] = {&params.back()};
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void*>(lf::step_kernel(kind, lf::needs_general(chains[c].second)));
      kp.gridDim = dim3(static_cast<unsigned>(chains[c].second.tile_start[chains[c].second.n_jobs]));
      kp.blockDim = dim3(static_cast<unsigned>(lf::kTile));
      kp.sharedMemBytes = 0;
      kp.kernelParams = args;
      cudaGraphNode_t node = nullptr;
      e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);   // copies the parameters
      if (e == cudaSuccess && prev) {
        cudaGraphEdgeData ed{};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.to_port = 0;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        e = cudaGraphAddDependencies(g, &prev, &node, &ed, 1);
      }
      prev = node;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) *out = nullptr;
  return e;
}

// The step graph for the current parity.  A graph is kept while its launch
// parameters stay the same (re-seeding with the same layer count and buffers,
// as every Lloyd-like round and every benchmark job does, reuses it).
lf_status build_graph(lf_mesh m) {
  const int par = static_cast<int>(m->h_st.epoch & 1u);
  const lf::BatchParams p = single_job_params(m, kGraphSteps);
  const int kind = lf::step_kind(m->dtype, m->sched);
  if (m->gexec[par]) {
    if (std::memcmp(&p, &m->gparams[par], sizeof(p)) == 0 && m->gkind[par] == kind) return LF_OK;
    cudaGraphExecDestroy(m->gexec[par]);
    m->gexec[par] = nullptr;
  }
  std::vector<std::pair<int, lf::BatchParams>> chains;
  chains.emplace_back(kind, p);
  cudaError_t e = make_step_graph(chains, &m->gexec[par]);
  if (e != cudaSuccess) return cuda_fail(m, e, "building the step graph");
  m->gparams[par] = p;
  m->gkind[par] = kind;
  return LF_OK;
}

lf_status check_usable(lf_mesh m) {
  if (!m) return fail(nullptr, LF_ERR_INVALID, "null mesh");
  if (m->poisoned) return fail(m, LF_ERR_STATE, "handle is poisoned by an earlier CUDA error or timeout");
  return LF_OK;
}

// Common tail of both create paths: off-diagonal FP64 CSR -> device.
// A mesh handle without operator or field: stream, parameters, tile count.
lf_mesh new_mesh(const lf_device* dev, int64_t n_v, const lf_params& prm) {
  lf_mesh m = new (std::nothrow) lf_mesh_s();
  if (!m) return nullptr;
  if (dev) m->dev = *dev;
  m->stream = static_cast<cudaStream_t>(m->dev.cuda_stream);
  m->params = prm;
  m->n_v = n_v;
  m->dtype = prm.field_dtype;
  m->num_tiles = static_cast<int>((n_v + lf::kTile - 1) / lf::kTile);
  return m;
}

// Off-diagonal FP64 CSR from the host -> the device operator (FP32 values).
lf_status upload_operator(lf_mesh m, const std::vector<int64_t>& rp, const std::vector<int32_t>& col,
                          const std::vector<double>& val) {
  const int64_t n_v = m->n_v;
  const int64_t nnz = static_cast<int64_t>(col.size());
  if (nnz >= kMaxCap) return fail(m, LF_ERR_CAPACITY, "operator exceeds 2^31 entries");
  m->L_nnz = nnz;
  std::vector<int32_t> rp32(static_cast<size_t>(n_v) + 1);
  for (int64_t i = 0; i <= n_v; ++i) rp32[static_cast<size_t>(i)] = static_cast<int32_t>(rp[static_cast<size_t>(i)]);
  std::vector<int2> cv(static_cast<size_t>(std::max<int64_t>(nnz, 1)));
  for (int64_t q = 0; q < nnz; ++q) {
    float w = static_cast<float>(val[static_cast<size_t>(q)]);
    int bits;
    std::memcpy(&bits, &w, 4);
    cv[static_cast<size_t>(q)] = make_int2(col[static_cast<size_t>(q)], bits);
  }
  m->d_Lrp = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * (n_v + 1)));
  m->d_Lcv = static_cast<int2*>(m->dalloc(sizeof(int2) * std::max<int64_t>(nnz, 1)));
  if (!m->d_Lrp || !m->d_Lcv) return fail(m, LF_ERR_OOM, "device allocation");
  LF_CUDA(m, cudaMemcpyAsync(m->d_Lrp, rp32.data(), sizeof(int32_t) * (n_v + 1), cudaMemcpyHostToDevice, m->stream));
  LF_CUDA(m, cudaMemcpyAsync(m->d_Lcv, cv.data(), sizeof(int2) * std::max<int64_t>(nnz, 1), cudaMemcpyHostToDevice,
                             m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));   // the host vectors die on return
  return LF_OK;
}

// The cotangent operator built on the device from the mesh's own geometry
// (d_V, d_tri): the same bits as cotan_rows + upload_operator.
lf_status build_operator_device(lf_mesh m) {
  const int64_t n_v = m->n_v, n_f = m->n_f;
  if (6 * n_f >= kMaxCap) return fail(m, LF_ERR_CAPACITY, "operator exceeds 2^31 entries");
  const int64_t nb = std::max(lf::cotan_scan_blocks(n_v), int64_t{1});
  auto* hc = static_cast<double*>(m->dalloc(sizeof(double) * 3 * static_cast<size_t>(n_f)));
  auto* inc = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * 3 * static_cast<size_t>(n_f)));
  auto* cnt = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * static_cast<size_t>(n_v)));
  auto* inc_start = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * static_cast<size_t>(n_v + 1)));
  auto* bsum = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * static_cast<size_t>(nb)));
  auto* bad = static_cast<unsigned long long*>(m->dalloc(sizeof(unsigned long long)));
  m->d_Lrp = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * static_cast<size_t>(n_v + 1)));
  auto release = [&]() {
    for (void* p : {static_cast<void*>(hc), static_cast<void*>(inc), static_cast<void*>(cnt),
                    static_cast<void*>(inc_start), static_cast<void*>(bsum), static_cast<void*>(bad)})
      m->dfree(p);
  };
  if (!hc || !inc || !cnt || !inc_start || !bsum || !bad || !m->d_Lrp) {
    release();
    return fail(m, LF_ERR_OOM, "operator build scratch");
  }
  cudaStream_t st = m->stream;
  int32_t total = 0;
  unsigned long long first_bad = 0;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n_v, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = lf::launch_cotan_corners(m->d_V, m->d_tri, n_f, hc, cnt, bad, st);
  if (e == cudaSuccess) e = lf::launch_exclusive_scan(cnt, inc_start, n_v, bsum, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n_v, st);
  if (e == cudaSuccess) e = lf::launch_cotan_incidence(m->d_tri, n_f, inc_start, cnt, inc, st);
  if (e == cudaSuccess) e = lf::launch_cotan_rows(m->d_tri, hc, n_v, inc_start, inc, 0, cnt, nullptr, nullptr, st);
  if (e == cudaSuccess) e = lf::launch_exclusive_scan(cnt, m->d_Lrp, n_v, bsum, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, m->d_Lrp + n_v, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&first_bad, bad, sizeof(first_bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && first_bad == ~0ull) {
    m->L_nnz = total;
    m->d_Lcv = static_cast<int2*>(m->dalloc(sizeof(int2) * static_cast<size_t>(std::max<int64_t>(total, 1))));
    if (!m->d_Lcv) {
      release();
      return fail(m, LF_ERR_OOM, "device allocation");
    }
    e = lf::launch_cotan_rows(m->d_tri, hc, n_v, inc_start, inc, 1, nullptr, m->d_Lrp, m->d_Lcv, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  release();
  if (e != cudaSuccess) return cuda_fail(m, e, "building the operator");
  if (first_bad != ~0ull) return fail(m, LF_ERR_INVALID, "face " + std::to_string(first_bad) + " has zero area");
  return LF_OK;
}

// Common tail of both create paths: status word, row arrays, job descriptor,
// tile segments.
lf_status finish_setup(lf_mesh m, const lf_params& prm) {
  const int64_t n_v = m->n_v;
  m->d_st = static_cast<lf::DevStatus*>(m->dalloc(sizeof(lf::DevStatus)));
  for (int b = 0; b < 2; ++b) {
    m->buf[b].rows = static_cast<int2*>(m->dalloc(sizeof(int2) * n_v));
    m->buf[b].head = static_cast<int4*>(m->dalloc(sizeof(int4) * n_v));
  }
  if (!m->d_st || !m->buf[0].rows || !m->buf[1].rows || !m->buf[0].head || !m->buf[1].head)
    return fail(m, LF_ERR_OOM, "device allocation");
  LF_CUDA(m, cudaMemsetAsync(m->d_st, 0, sizeof(lf::DevStatus), m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  lf::JobDesc& j = m->h_job;
  j.n_v = static_cast<int32_t>(n_v);
  j.n_layers = 0;
  j.num_tiles = m->num_tiles;
  j.L_rowptr = m->d_Lrp;
  j.L_colval = m->d_Lcv;
  j.buf[0] = m->buf[0];
  j.buf[1] = m->buf[1];
  j.st = m->d_st;
  j.L_nnz = static_cast<int32_t>(m->L_nnz);
  j.c = lf::Coefs{static_cast<float>(prm.dt),   static_cast<float>(prm.mu),   static_cast<float>(prm.w_cc),
                  static_cast<float>(prm.w_cb), static_cast<float>(prm.a_cc), static_cast<float>(prm.a_cb),
                  static_cast<float>(prm.e_cc), static_cast<float>(prm.e_cb), static_cast<float>(prm.e_bc)};
  // default: three entries per vertex of a tile; the band holds ~1.6 on average
  const int64_t cap = prm.initial_capacity > 0 ? (prm.initial_capacity + m->num_tiles - 1) / m->num_tiles
                                               : 3 * lf::kTile;
  return set_tile_cap(m, cap, false);
}

// Hands a finished mesh out, or deletes a failed one keeping its message.
lf_status hand_out(lf_mesh m, lf_status s, lf_mesh* out) {
  if (s != LF_OK) {
    g_create_error = m->err;
    delete m;
    return s;
  }
  *out = m;
  return LF_OK;
}

// The host-CSR create path (lf_create_mesh_csr, the server).
lf_status finish_create(const lf_device* dev, int64_t n_v, const std::vector<int64_t>& rp,
                        const std::vector<int32_t>& col, const std::vector<double>& val,
                        const lf_params& prm, lf_mesh* out) {
  lf_mesh m = new_mesh(dev, n_v, prm);
  if (!m) return fail(nullptr, LF_ERR_OOM, "host allocation");
  lf_status s = upload_operator(m, rp, col, val);
  if (s == LF_OK) s = finish_setup(m, prm);
  return hand_out(m, s, out);
}

}  // namespace

namespace lf {
void set_last_error(const std::string& msg) { g_create_error = msg; }

bool cotan_offdiag(int64_t n_v, const double* V, int64_t n_f, const int32_t* F, std::vector<int64_t>& rp,
                   std::vector<int32_t>& col, std::vector<double>& val, std::string& why) {
  return cotan_rows(n_v, V, n_f, F, rp, col, val, why);
}

bool mesh_ok(int64_t n_v, const double* V, int64_t n_f, const int32_t* F, std::string& why) {
  if (!V || !F) { why = "null argument"; return false; }
  if (n_v < 3 || n_v >= kMaxCap) { why = "n_v out of range"; return false; }
  if (n_f < 1) { why = "n_f must be >= 1"; return false; }
  std::atomic<int64_t> bad_v{n_v};
  parallel_for(n_v, 1 << 16, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      if (!std::isfinite(V[3 * i]) || !std::isfinite(V[3 * i + 1]) || !std::isfinite(V[3 * i + 2])) {
        int64_t cur = bad_v.load();
        while (i < cur && !bad_v.compare_exchange_weak(cur, i)) {
        }
        break;
      }
  });
  if (bad_v.load() < n_v) { why = "non-finite vertex coordinate"; return false; }
  // per face: ids in range, no repeated id, and a nonzero cross product at
  // the first corner (the first failing face is reported)
  std::atomic<int64_t> bad_f{n_f};
  parallel_for(n_f, 1 << 15, [&](int64_t lo, int64_t hi) {
    for (int64_t f = lo; f < hi && f < bad_f.load(); ++f) {
      const int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
      bool bad = false;
      if (a < 0 || b < 0 || c < 0 || a >= n_v || b >= n_v || c >= n_v || a == b || b == c || a == c) {
        bad = true;
      } else {
        const double* P = V + 3 * static_cast<int64_t>(a);
        const double* Q = V + 3 * static_cast<int64_t>(b);
        const double* S = V + 3 * static_cast<int64_t>(c);
        const double ux = Q[0] - P[0], uy = Q[1] - P[1], uz = Q[2] - P[2];
        const double wx = S[0] - P[0], wy = S[1] - P[1], wz = S[2] - P[2];
        const double cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
        bad = cx == 0.0 && cy == 0.0 && cz == 0.0;
      }
      if (!bad) continue;
      int64_t cur = bad_f.load();
      while (f < cur && !bad_f.compare_exchange_weak(cur, f)) {
      }
      break;
    }
  });
  const int64_t f = bad_f.load();
  if (f < n_f) {
    const int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n_v || b >= n_v || c >= n_v)
      why = "face " + std::to_string(f) + " has a vertex out of range";
    else if (a == b || b == c || a == c)
      why = "face " + std::to_string(f) + " repeats a vertex";
    else
      why = "face " + std::to_string(f) + " has zero area";
    return false;
  }
  return true;
}

bool seeds_ok(int64_t n_v, const int32_t* seeds, int32_t k, std::string& why) {
  if (!seeds || k < 1) { why = "need k >= 1 seeds"; return false; }
  if (static_cast<int64_t>(k) + 1 > 65536) { why = "k + 1 must be <= 65536"; return false; }
  if (k > n_v) { why = "more seeds than vertices"; return false; }
  std::vector<char> used(static_cast<size_t>(n_v), 0);
  for (int32_t i = 0; i < k; ++i) {
    if (seeds[i] < 0 || seeds[i] >= n_v) { why = "seed vertex out of range"; return false; }
    if (used[static_cast<size_t>(seeds[i])]) { why = "repeated seed vertex"; return false; }
    used[static_cast<size_t>(seeds[i])] = 1;
  }
  return true;
}

bool params_valid(const lf_params& p, std::string& why) { return params_ok(p, why); }

lf_status attach_geometry(lf_mesh m, const double* V, int64_t n_v, const int32_t* F, int64_t n_f) {
  if (n_v != m->n_v) return fail(m, LF_ERR_INVALID, "geometry does not match the mesh");
  m->d_V = static_cast<double*>(m->dalloc(sizeof(double) * 3 * static_cast<size_t>(n_v)));
  m->d_tri = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * 3 * static_cast<size_t>(n_f)));
  if (!m->d_V || !m->d_tri) return fail(m, LF_ERR_OOM, "uploading the mesh");
  LF_CUDA(m, cudaMemcpyAsync(m->d_V, V, sizeof(double) * 3 * n_v, cudaMemcpyHostToDevice, m->stream));
  LF_CUDA(m, cudaMemcpyAsync(m->d_tri, F, sizeof(int32_t) * 3 * n_f, cudaMemcpyHostToDevice, m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  m->n_f = n_f;
  return LF_OK;
}

int64_t geometry_bytes_estimate(int64_t n_v, int64_t n_f, int64_t k) {
  auto r = [](int64_t b) { return (std::max<int64_t>(b, 16) + 255) & ~int64_t(255); };
  int64_t tab = 4096;
  while (tab < 16 * k) tab <<= 1;
  return r(24 * n_v) + r(12 * n_f) +                              // V, faces
         r(56 * k) * 2 + r(16 * k) + r(8 * n_v) + 3 * r(4 * k) +  // Lloyd scratch and seeds
         4 * r(4 * tab) + r(4 * n_v) + 2 * r(24 * k);              // dual scratch
}

lf_status create_from_offdiag(const lf_device* dev, int64_t n_v, const std::vector<int64_t>& rp,
                              const std::vector<int32_t>& col, const std::vector<double>& val,
                              const lf_params& prm, lf_mesh* out) {
  return finish_create(dev, n_v, rp, col, val, prm, out);
}

int64_t device_bytes_estimate(int64_t n_v, int64_t nnz_off, const lf_params& prm) {
  auto r = [](int64_t b) { return (std::max<int64_t>(b, 16) + 255) & ~int64_t(255); };
  const int64_t tiles = (n_v + kTile - 1) / kTile;
  const int64_t cap = prm.initial_capacity > 0 ? round16(std::max<int64_t>((prm.initial_capacity + tiles - 1) / tiles, kTile))
                                               : 3 * kTile;
  const int64_t entries = tiles * cap;
  return r(4 * (n_v + 1)) + r(8 * nnz_off) + r(static_cast<int64_t>(sizeof(DevStatus))) + 2 * r(8 * n_v) +
         2 * r(16 * n_v) /* head records */ +
         2 * (r(2 * entries) + r(value_bytes(prm.field_dtype) * entries)) + r(4 * n_v) /* labels */;
}
}  // namespace lf

extern "C" {

void lf_default_params(lf_params* p) {
  if (!p) return;
  p->dt = 5.0;
  p->mu = 1.0;
  p->w_cc = 0.2;
  p->w_cb = 0.0;
  p->a_cc = 0.04;
  p->a_cb = 0.04;
  p->e_cc = 0.0;
  p->e_cb = 0.5;
  p->e_bc = -0.5;
  p->iso = 0.25;
  p->field_dtype = LF_F32;
  p->reserved = 0;
  p->initial_capacity = 0;
}

lf_status lf_create_mesh(const lf_device* dev, const double* V, int64_t n_v, const int32_t* F, int64_t n_f,
                         const lf_params* params, lf_mesh* out) {
  lf::TraceRange trace("lf_create_mesh");
  if (!out) return fail(nullptr, LF_ERR_INVALID, "null argument");
  lf_params prm;
  lf_default_params(&prm);
  if (params) prm = *params;
  std::string why;
  if (!params_ok(prm, why)) return fail(nullptr, LF_ERR_INVALID, why);
  if (!lf::mesh_ok(n_v, V, n_f, F, why)) return fail(nullptr, LF_ERR_INVALID, why);
  // the mesh goes to the device once: the operator is built there from it,
  // and it stays for the Lloyd-like update (Sec. 5) and the dual mesh
  lf_mesh m = new_mesh(dev, n_v, prm);
  if (!m) return fail(nullptr, LF_ERR_OOM, "host allocation");
  lf_status s = lf::attach_geometry(m, V, n_v, F, n_f);
  if (s == LF_OK) s = build_operator_device(m);
  if (s == LF_OK) s = finish_setup(m, prm);
  return hand_out(m, s, out);
}

lf_status lf_create_mesh_csr(const lf_device* dev, int64_t n_v, const int64_t* rowptr, const int32_t* col,
                             const double* val, const lf_params* params, lf_mesh* out) {
  if (!out || !rowptr || (!col && rowptr && n_v > 0 && rowptr[n_v] > 0))
    return fail(nullptr, LF_ERR_INVALID, "null argument");
  if (n_v < 1 || n_v >= kMaxCap) return fail(nullptr, LF_ERR_INVALID, "n_v out of range");
  lf_params prm;
  lf_default_params(&prm);
  if (params) prm = *params;
  std::string why;
  if (!params_ok(prm, why)) return fail(nullptr, LF_ERR_INVALID, why);
  if (rowptr[0] != 0) return fail(nullptr, LF_ERR_INVALID, "rowptr[0] must be 0");
  std::vector<int64_t> rp(static_cast<size_t>(n_v) + 1, 0);
  std::vector<int32_t> c2;
  std::vector<double> v2;
  try {
    for (int64_t i = 0; i < n_v; ++i) {
      if (rowptr[i + 1] < rowptr[i]) return fail(nullptr, LF_ERR_INVALID, "rowptr is not monotone");
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        if (col[q] < 0 || col[q] >= n_v) return fail(nullptr, LF_ERR_INVALID, "column out of range");
        if (!std::isfinite(val[q])) return fail(nullptr, LF_ERR_INVALID, "non-finite operator value");
        if (col[q] == i) continue;                 // the diagonal is implicit
        c2.push_back(col[q]);
        v2.push_back(val[q]);
      }
      rp[static_cast<size_t>(i) + 1] = static_cast<int64_t>(c2.size());
    }
  } catch (const std::bad_alloc&) {
    return fail(nullptr, LF_ERR_OOM, "host allocation");
  }
  return finish_create(dev, n_v, rp, c2, v2, prm, out);
}

}  // extern "C"

namespace {

// Coefficient matrices hold for one layer count: a field with another count
// (new seeds, lf_set_field) returns the mesh to the class coefficients.
void drop_coefficients(lf_mesh m, bool always) {
  if (!m->d_coef || (!always && m->coef_layers == m->n_layers)) return;
  m->dfree(m->d_coef);
  m->d_coef = nullptr;
  m->coef_layers = 0;
  m->h_job.cW = m->h_job.cA = m->h_job.cE = nullptr;
}

// Initial field (Sec. 3.2): point seeds (rings = 0) or a seed vertex with its
// immediate neighbours (rings = 1); every other vertex holds the base layer.
lf_status seed_impl(lf_mesh m, const int32_t* seeds, int32_t k, int32_t rings) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (rings < 0 || rings > 1) return fail(m, LF_ERR_INVALID, "rings must be 0 or 1");
  std::string why;
  if (!lf::seeds_ok(m->n_v, seeds, k, why)) return fail(m, LF_ERR_INVALID, why);
  auto* d_seeds = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * static_cast<size_t>(k)));
  if (!d_seeds) return fail(m, LF_ERR_OOM, "seed upload buffer");
  unsigned* d_owner = nullptr;
  if (rings == 1) {
    d_owner = static_cast<unsigned*>(m->dalloc(sizeof(unsigned) * static_cast<size_t>(m->n_v)));
    if (!d_owner) {
      m->dfree(d_seeds);
      return fail(m, LF_ERR_OOM, "region seed scratch");
    }
  }
  m->n_layers = k + 1;
  m->h_job.n_layers = k + 1;
  drop_coefficients(m, false);
  std::memset(&m->h_st, 0, sizeof(m->h_st));
  m->h_st.nnz = static_cast<unsigned long long>(m->n_v);
  s = upload_status(m);
  if (s != LF_OK) return s;
  LF_CUDA(m, cudaMemcpyAsync(d_seeds, seeds, sizeof(int32_t) * k, cudaMemcpyHostToDevice, m->stream));
  if (rings == 1) {
    LF_CUDA(m, lf::launch_seed_regions(m->h_job, k, d_seeds, d_owner, m->dtype, m->stream));
  } else {
    LF_CUDA(m, lf::launch_seed(m->h_job, k, d_seeds, m->dtype, m->stream));
  }
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  m->dfree(d_seeds);
  m->dfree(d_owner);
  m->steps = 0;
  m->retries = 0;
  m->seeds.assign(seeds, seeds + k);
  ++m->version;
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_seed(lf_mesh m, const int32_t* seeds, int32_t k) { return seed_impl(m, seeds, k, 0); }

lf_status lf_seed_regions(lf_mesh m, const int32_t* seeds, int32_t k, int32_t rings) {
  return seed_impl(m, seeds, k, rings);
}

lf_status lf_set_coefficients(lf_mesh m, int32_t n_layers, const float* W, const float* A, const float* E) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed or lf_set_field must come first");
  if (n_layers != m->n_layers) return fail(m, LF_ERR_INVALID, "n_layers differs from the field's layer count");
  if (n_layers > kMaxCoefLayers) return fail(m, LF_ERR_INVALID, "coefficient matrices take at most 4096 layers");
  const float* src[3] = {W, A, E};
  const int64_t nn = static_cast<int64_t>(n_layers) * n_layers;
  int present = 0;
  for (const float* M : src) {
    if (!M) continue;
    ++present;
    for (int64_t q = 0; q < nn; ++q)
      if (!std::isfinite(M[q])) return fail(m, LF_ERR_INVALID, "coefficient matrices must be finite");
  }
  LF_CUDA(m, cudaStreamSynchronize(m->stream));   // no step in flight reads the old block
  drop_coefficients(m, true);
  if (present == 0) return LF_OK;
  auto* d = static_cast<float*>(m->dalloc(sizeof(float) * static_cast<size_t>(nn * present)));
  if (!d) return fail(m, LF_ERR_OOM, "coefficient matrices");
  const float** dst[3] = {&m->h_job.cW, &m->h_job.cA, &m->h_job.cE};
  int slot = 0;
  for (int x = 0; x < 3; ++x) {
    if (!src[x]) continue;
    float* part = d + static_cast<int64_t>(slot++) * nn;
    LF_CUDA(m, cudaMemcpyAsync(part, src[x], sizeof(float) * static_cast<size_t>(nn), cudaMemcpyHostToDevice,
                               m->stream));
    *dst[x] = part;
  }
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  m->d_coef = d;
  m->coef_layers = n_layers;
  return LF_OK;
}

lf_status lf_step(lf_mesh m, int32_t n_iters) {
  lf::TraceRange trace("lf_step");
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (n_iters < 0) return fail(m, LF_ERR_INVALID, "n_iters must be >= 0");
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed or lf_set_field must come first");
  const int64_t target = m->steps + n_iters;
  while (m->steps < target) {
    const int64_t todo = std::min<int64_t>(target - m->steps, kPollSteps);
    int64_t launched = 0;
    if (todo >= kGraphSteps) {
      s = build_graph(m);
      if (s != LF_OK) return s;
      while (todo - launched >= kGraphSteps) {
        LF_CUDA(m, cudaGraphLaunch(m->gexec[m->h_st.epoch & 1u], m->stream));
        launched += kGraphSteps;
      }
    }
    if (launched < todo) {
      // the graph launches above cover an even number of steps, so the
      // starting parity of the remainder is still that of the current epoch
      lf::BatchParams p = single_job_params(m, static_cast<int>(todo - launched));
      for (int s2 = 0; launched < todo; ++launched, ++s2) {
        p.step = s2;
        LF_CUDA(m, lf::launch_step(p, lf::step_kind(m->dtype, m->sched), m->stream));
      }
    }
    s = read_status(m);
    if (s != LF_OK) return s;
    m->steps = static_cast<int64_t>(m->h_st.epoch);
    if (m->h_st.err == 0u) continue;

    // a step failed: the field is intact in buf[epoch & 1]; fix and re-run
    const uint32_t err = m->h_st.err;
    if (err & (lf::ERR_ZERO_SUM | lf::ERR_BOUNDS)) {
      reset_after_failure(m);
      return fail(m, LF_ERR_STATE, failed_step_message(err));
    }
    if (err & lf::ERR_CAPACITY) {
      const int64_t need = static_cast<int64_t>(m->h_st.need_tile);
      const int64_t grown = std::max<int64_t>(need + need / 4, m->tile_cap + m->tile_cap / 5 + 1);
      s = set_tile_cap(m, grown, true);
      if (s != LF_OK) {
        reset_after_failure(m);
        return s;
      }
    }
    s = reset_after_failure(m);
    if (s != LF_OK) return s;
    ++m->retries;
  }
  return LF_OK;
}

lf_status lf_step_batch(lf_mesh* meshes, int32_t n, const int32_t* n_iters) {
  lf::TraceRange trace("lf_step_batch");
  if (!meshes || n < 1 || n > lf::kMaxJobs)
    return fail(nullptr, LF_ERR_INVALID, "need 1 <= n <= 64 meshes");
  if (!n_iters) return fail(nullptr, LF_ERR_INVALID, "n_iters is null");
  for (int32_t a = 0; a < n; ++a) {
    lf_mesh m = meshes[a];
    lf_status s = check_usable(m);
    if (s != LF_OK) return s;
    if (n_iters[a] < 0) return fail(m, LF_ERR_INVALID, "n_iters must be >= 0");
    if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed or lf_set_field must come first");
    for (int32_t b = 0; b < a; ++b)
      if (meshes[b] == m) return fail(m, LF_ERR_INVALID, "a mesh appears twice in the batch");
  }
  // the batch runs on the first mesh's stream, after every mesh's own work
  lf_mesh m0 = meshes[0];
  std::vector<int64_t> target(static_cast<size_t>(n));
  for (int32_t a = 0; a < n; ++a) {
    lf_status s = read_status(meshes[a]);
    if (s != LF_OK) return s;
    target[static_cast<size_t>(a)] = meshes[a]->steps + n_iters[a];
  }
  // one chain of launches per storage type and schedule present; the graph is rebuilt
  // whenever the parameters of a chain change (members, buffers, parity)
  cudaGraphExec_t gexec = nullptr;
  std::vector<std::pair<int, lf::BatchParams>> gkey;
  auto drop_graph = [&]() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  };
  lf_status result = LF_OK;
  for (;;) {
    // every job still running advances by the same count, so one parameter
    // set holds for the whole chunk and finished jobs leave the launches
    int64_t todo = kPollSteps;
    int active = 0;
    for (int32_t a = 0; a < n; ++a) {
      const int64_t left = target[static_cast<size_t>(a)] - meshes[a]->steps;
      if (left > 0) { todo = std::min(todo, left); ++active; }
    }
    if (active == 0) break;
    std::vector<std::pair<int, lf::BatchParams>> chains;
    for (int kind = 0; kind < 3 * lf::kSchedules; ++kind) {
      lf::BatchParams p;
      std::memset(&p, 0, sizeof(p));
      int tiles = 0;
      for (int32_t a = 0; a < n; ++a) {
        lf_mesh m = meshes[a];
        if (lf::step_kind(m->dtype, m->sched) != kind || target[static_cast<size_t>(a)] == m->steps) continue;
        const int j = p.n_jobs++;
        p.tile_start[j] = tiles;
        tiles += m->num_tiles;
        p.job[j] = m->h_job;
        p.job[j].parity0 = static_cast<int32_t>(m->h_st.epoch & 1u);
        p.job[j].steps = static_cast<int32_t>(todo);
      }
      p.tile_start[p.n_jobs] = tiles;
      if (p.n_jobs > 0) chains.emplace_back(kind, p);
    }
    int64_t launched = 0;
    if (todo >= kGraphSteps) {
      std::vector<std::pair<int, lf::BatchParams>> gc = chains;
      for (auto& c : gc)
        for (int j = 0; j < c.second.n_jobs; ++j) c.second.job[j].steps = kGraphSteps;
      bool same = gexec && gc.size() == gkey.size();
      for (size_t c = 0; same && c < gc.size(); ++c)
        same = gc[c].first == gkey[c].first && std::memcmp(&gc[c].second, &gkey[c].second, sizeof(lf::BatchParams)) == 0;
      if (!same) {
        drop_graph();
        cudaError_t e = make_step_graph(gc, &gexec);
        if (e != cudaSuccess) return cuda_fail(m0, e, "building the batch graph");
        gkey = gc;
      }
      while (todo - launched >= kGraphSteps) {
        cudaError_t e = cudaGraphLaunch(gexec, m0->stream);
        if (e != cudaSuccess) { drop_graph(); return cuda_fail(m0, e, "cudaGraphLaunch"); }
        launched += kGraphSteps;
      }
    }
    for (auto& c : chains)
      for (int j = 0; j < c.second.n_jobs; ++j) {
        c.second.job[j].steps = static_cast<int32_t>(todo - launched);
        c.second.job[j].parity0 = static_cast<int32_t>((c.second.job[j].parity0 + launched) & 1);
      }
    for (int k = 0; launched < todo; ++launched, ++k)
      for (auto& c : chains) {
        c.second.step = k;
        cudaError_t e = lf::launch_step(c.second, c.first, m0->stream);
        if (e != cudaSuccess) { drop_graph(); return cuda_fail(m0, e, "launching a batch step"); }
      }
    cudaError_t e = cudaStreamSynchronize(m0->stream);
    if (e != cudaSuccess) { drop_graph(); return cuda_fail(m0, e, "cudaStreamSynchronize"); }
    // per job: progress, and recovery of the jobs whose step failed
    for (int32_t a = 0; a < n; ++a) {
      lf_mesh m = meshes[a];
      if (target[static_cast<size_t>(a)] == m->steps) continue;
      lf_status s = read_status(m);
      if (s != LF_OK) { drop_graph(); return s; }
      m->steps = static_cast<int64_t>(m->h_st.epoch);
      if (m->h_st.err == 0u) continue;
      if (m->h_st.err & (lf::ERR_ZERO_SUM | lf::ERR_BOUNDS)) {
        const uint32_t err = m->h_st.err;
        reset_after_failure(m);
        target[static_cast<size_t>(a)] = m->steps;          // leave it out of the rest of the batch
        result = fail(m, LF_ERR_STATE, failed_step_message(err));
        continue;
      }
      const int64_t need = static_cast<int64_t>(m->h_st.need_tile);
      s = set_tile_cap(m, std::max<int64_t>(need + need / 4, m->tile_cap + m->tile_cap / 5 + 1), true);
      if (s == LF_OK) s = reset_after_failure(m);
      if (s != LF_OK) { drop_graph(); return s; }
      ++m->retries;
    }
  }
  drop_graph();
  return result;
}

lf_status lf_set_schedule(lf_mesh m, int32_t schedule) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (schedule < 0 || schedule >= lf::kSchedules) return fail(m, LF_ERR_INVALID, "unknown schedule");
  m->sched = schedule;
  return LF_OK;
}

int32_t lf_schedule(lf_mesh m) { return m ? m->sched : -1; }

lf_status lf_tune(lf_mesh m, int32_t trial_steps, int32_t* schedule) {
  lf::TraceRange trace("lf_tune");
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (trial_steps < 1) return fail(m, LF_ERR_INVALID, "trial_steps must be >= 1");
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed or lf_set_field must come first");
  cudaEvent_t ev[2] = {nullptr, nullptr};
  for (auto& e : ev) {
    cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return cuda_fail(m, ce, "cudaEventCreate");
    }
  }
  // two rounds over the schedules, the second in reverse order, so that a
  // trend along the trajectory weighs on every schedule alike; every trial
  // advances the job (the schedules give the same bits)
  float ms[lf::kSchedules] = {};
  for (int r = 0; r < 2 && s == LF_OK; ++r) {
    for (int k = 0; k < lf::kSchedules && s == LF_OK; ++k) {
      const int sc = (r == 0) ? k : lf::kSchedules - 1 - k;
      m->sched = sc;
      s = build_graph(m);                  // outside the timing
      if (s != LF_OK) break;
      cudaError_t ce = cudaEventRecord(ev[0], m->stream);
      if (ce == cudaSuccess) s = lf_step(m, trial_steps);
      if (ce == cudaSuccess && s == LF_OK) ce = cudaEventRecord(ev[1], m->stream);
      if (ce == cudaSuccess && s == LF_OK) ce = cudaEventSynchronize(ev[1]);
      float t = 0.0f;
      if (ce == cudaSuccess && s == LF_OK) ce = cudaEventElapsedTime(&t, ev[0], ev[1]);
      if (ce != cudaSuccess && s == LF_OK) s = cuda_fail(m, ce, "timing a schedule");
      ms[sc] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (s != LF_OK) return s;
  int best = 0;
  for (int k = 1; k < lf::kSchedules; ++k)
    if (ms[k] < ms[best]) best = k;
  m->sched = best;
  if (schedule) *schedule = best;
  return LF_OK;
}

lf_status lf_labels(lf_mesh m, int32_t* labels, float* maxval) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (!labels) return fail(m, LF_ERR_INVALID, "labels must not be NULL");
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed or lf_set_field must come first");
  if (!m->d_labels) {
    m->d_labels = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * m->n_v));
    if (!m->d_labels) return fail(m, LF_ERR_OOM, "label buffer");
  }
  if (maxval && m->scratch_f_len < m->n_v) {
    m->dfree(m->d_scratch_f);
    m->d_scratch_f = static_cast<float*>(m->dalloc(sizeof(float) * m->n_v));
    if (!m->d_scratch_f) { m->scratch_f_len = 0; return fail(m, LF_ERR_OOM, "value buffer"); }
    m->scratch_f_len = m->n_v;
  }
  LF_CUDA(m, lf::launch_labels(m->h_job, static_cast<int>(m->h_st.epoch & 1u), m->dtype, m->d_labels,
                               maxval ? m->d_scratch_f : nullptr, m->stream));
  LF_CUDA(m, cudaMemcpyAsync(labels, m->d_labels, sizeof(int32_t) * m->n_v, cudaMemcpyDeviceToHost, m->stream));
  if (maxval)
    LF_CUDA(m, cudaMemcpyAsync(maxval, m->d_scratch_f, sizeof(float) * m->n_v, cudaMemcpyDeviceToHost, m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  return LF_OK;
}

// The current field in plain CSR on the host: the tile segments are copied
// whole and gathered row by row.
lf_status lf_get_operator(lf_mesh m, int64_t* rowptr, int32_t* col, float* val, int64_t cap, int64_t* nnz) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (!nnz) return fail(m, LF_ERR_INVALID, "nnz must not be NULL");
  *nnz = m->L_nnz;
  if (rowptr) {
    std::vector<int32_t> rp(static_cast<size_t>(m->n_v) + 1);
    LF_CUDA(m, cudaMemcpyAsync(rp.data(), m->d_Lrp, sizeof(int32_t) * (m->n_v + 1), cudaMemcpyDeviceToHost,
                               m->stream));
    LF_CUDA(m, cudaStreamSynchronize(m->stream));
    for (int64_t i = 0; i <= m->n_v; ++i) rowptr[i] = rp[static_cast<size_t>(i)];
  }
  if (!col || !val || cap < m->L_nnz || m->L_nnz == 0) return LF_OK;
  std::vector<int2> cv(static_cast<size_t>(m->L_nnz));
  LF_CUDA(m, cudaMemcpyAsync(cv.data(), m->d_Lcv, sizeof(int2) * m->L_nnz, cudaMemcpyDeviceToHost, m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  for (int64_t q = 0; q < m->L_nnz; ++q) {
    col[q] = cv[static_cast<size_t>(q)].x;
    std::memcpy(&val[q], &cv[static_cast<size_t>(q)].y, 4);
  }
  return LF_OK;
}

lf_status lf_get_field(lf_mesh m, int64_t* rowptr, int32_t* layer, float* val, int64_t cap, int64_t* nnz) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (!nnz) return fail(m, LF_ERR_INVALID, "nnz must not be NULL");
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed or lf_set_field must come first");
  const int cur = static_cast<int>(m->h_st.epoch & 1u);
  std::vector<int2> rows(static_cast<size_t>(m->n_v));
  LF_CUDA(m, cudaMemcpyAsync(rows.data(), m->buf[cur].rows, sizeof(int2) * m->n_v, cudaMemcpyDeviceToHost,
                             m->stream));
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  int64_t total = 0;
  for (int64_t i = 0; i < m->n_v; ++i) {
    if (rowptr) rowptr[i] = total;
    total += rows[static_cast<size_t>(i)].y;
  }
  if (rowptr) rowptr[m->n_v] = total;
  *nnz = total;
  if (!layer || !val || cap < total || total == 0) return LF_OK;
  const int64_t entries = m->buffer_entries();
  std::vector<uint16_t> ids(static_cast<size_t>(entries));
  std::vector<float> vals(static_cast<size_t>(entries));
  LF_CUDA(m, cudaMemcpyAsync(ids.data(), m->buf[cur].ids, sizeof(uint16_t) * entries, cudaMemcpyDeviceToHost,
                             m->stream));
  if (m->dtype == LF_F32) {
    LF_CUDA(m, cudaMemcpyAsync(vals.data(), m->buf[cur].vals, sizeof(float) * entries, cudaMemcpyDeviceToHost,
                               m->stream));
  } else {
    if (m->scratch_f_len < entries) {
      m->dfree(m->d_scratch_f);
      m->d_scratch_f = static_cast<float*>(m->dalloc(sizeof(float) * entries));
      if (!m->d_scratch_f) { m->scratch_f_len = 0; return fail(m, LF_ERR_OOM, "value buffer"); }
      m->scratch_f_len = entries;
    }
    LF_CUDA(m, lf::launch_widen(m->buf[cur].vals, m->d_scratch_f, entries, m->dtype, m->stream));
    LF_CUDA(m, cudaMemcpyAsync(vals.data(), m->d_scratch_f, sizeof(float) * entries, cudaMemcpyDeviceToHost,
                               m->stream));
  }
  LF_CUDA(m, cudaStreamSynchronize(m->stream));
  int64_t o = 0;
  for (int64_t i = 0; i < m->n_v; ++i) {
    const int2 r = rows[static_cast<size_t>(i)];
    for (int p = 0; p < r.y; ++p, ++o) {
      layer[o] = ids[static_cast<size_t>(r.x + p)];
      val[o] = vals[static_cast<size_t>(r.x + p)];
    }
  }
  return LF_OK;
}

lf_status lf_set_field(lf_mesh m, const int64_t* rowptr, const int32_t* layer, const float* val, int64_t nnz,
                       int32_t n_layers) {
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (!rowptr || (nnz > 0 && (!layer || !val))) return fail(m, LF_ERR_INVALID, "null argument");
  if (n_layers < 2 || n_layers > 65536) return fail(m, LF_ERR_INVALID, "n_layers must be in [2, 65536]");
  if (rowptr[0] != 0 || rowptr[m->n_v] != nnz) return fail(m, LF_ERR_INVALID, "rowptr does not match nnz");
  if (nnz >= kMaxCap) return fail(m, LF_ERR_CAPACITY, "field exceeds 2^31 entries");
  int64_t need = 0;
  for (int64_t i = 0; i < m->n_v; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return fail(m, LF_ERR_INVALID, "rowptr is not monotone");
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (layer[p] < 0 || layer[p] >= n_layers) return fail(m, LF_ERR_INVALID, "layer out of range");
      if (p > rowptr[i] && layer[p] <= layer[p - 1]) return fail(m, LF_ERR_INVALID, "layers not increasing in a row");
      if (!(val[p] > 0.0f && val[p] <= 1.0f)) return fail(m, LF_ERR_INVALID, "value not in (0, 1]");
    }
  }
  for (int t = 0; t < m->num_tiles; ++t) {
    const int64_t a = static_cast<int64_t>(t) * lf::kTile;
    const int64_t b = std::min<int64_t>(a + lf::kTile, m->n_v);
    need = std::max(need, rowptr[b] - rowptr[a]);
  }
  if (need > m->tile_cap) {
    s = set_tile_cap(m, need + need / 4 + 1, false);
    if (s != LF_OK) return s;
  }
  // segmented copy: row i of tile t starts at t * tile_cap + (rowptr[i] - rowptr[first row of t])
  const int64_t entries = m->buffer_entries();
  std::vector<int2> rows(static_cast<size_t>(m->n_v));
  std::vector<uint16_t> ids(static_cast<size_t>(entries), 0);
  std::vector<float> vals(static_cast<size_t>(entries), 0.0f);
  for (int64_t i = 0; i < m->n_v; ++i) {
    const int64_t t = i / lf::kTile;
    const int64_t start = t * m->tile_cap + (rowptr[i] - rowptr[t * lf::kTile]);
    rows[static_cast<size_t>(i)] = make_int2(static_cast<int>(start), static_cast<int>(rowptr[i + 1] - rowptr[i]));
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      ids[static_cast<size_t>(start + p - rowptr[i])] = static_cast<uint16_t>(layer[p]);
      vals[static_cast<size_t>(start + p - rowptr[i])] = val[p];
    }
  }
  const int cur = static_cast<int>(m->h_st.epoch & 1u);
  LF_CUDA(m, cudaMemcpyAsync(m->buf[cur].rows, rows.data(), sizeof(int2) * m->n_v, cudaMemcpyHostToDevice,
                             m->stream));
  LF_CUDA(m, cudaMemcpyAsync(m->buf[cur].ids, ids.data(), sizeof(uint16_t) * entries, cudaMemcpyHostToDevice,
                             m->stream));
  if (m->dtype == LF_F32) {
    LF_CUDA(m, cudaMemcpyAsync(m->buf[cur].vals, vals.data(), sizeof(float) * entries, cudaMemcpyHostToDevice,
                               m->stream));
  } else {
    if (m->scratch_f_len < entries) {
      m->dfree(m->d_scratch_f);
      m->d_scratch_f = static_cast<float*>(m->dalloc(sizeof(float) * entries));
      if (!m->d_scratch_f) { m->scratch_f_len = 0; return fail(m, LF_ERR_OOM, "value buffer"); }
      m->scratch_f_len = entries;
    }
    LF_CUDA(m, cudaMemcpyAsync(m->d_scratch_f, vals.data(), sizeof(float) * entries, cudaMemcpyHostToDevice,
                               m->stream));
    LF_CUDA(m, lf::launch_narrow(m->d_scratch_f, m->buf[cur].vals, entries, m->dtype, m->stream));
  }
  LF_CUDA(m, lf::launch_build_head(m->buf[cur], static_cast<int>(m->n_v), m->dtype, m->stream));
  m->n_layers = n_layers;
  m->h_job.n_layers = n_layers;
  drop_coefficients(m, false);
  m->h_st.nnz = static_cast<unsigned long long>(nnz);
  if (static_cast<int64_t>(m->seeds.size()) != n_layers - 1) m->seeds.clear();
  ++m->version;
  s = upload_status(m);
  return s;
}

}  // extern "C"

namespace {

// Graph stage of the dual extraction (Sec. 5.2) on k cells: the manifold check
// (a face-only pair is dropped when its cells share two or more neighbours of
// A_v), the triangles (mutually adjacent triples), the removal of spurious
// triangles (the three neighbours of a cell with exactly three mutually
// adjacent neighbours) and the orientation (breadth-first over shared edges
// from the first triangle of each part, oriented along the mesh normals at
// its seeds).  Returns oriented cell triples in sorted order of their sets.
std::vector<std::array<int32_t, 3>> dual_graph(int k, const std::vector<uint32_t>& av,
                                               const std::vector<uint32_t>& cand, const std::vector<double>& pos,
                                               const std::vector<double>& nrm) {
  std::vector<std::vector<int32_t>> Nv(static_cast<size_t>(k));
  for (uint32_t key : av) {
    const int32_t c = static_cast<int32_t>(key >> 16), d = static_cast<int32_t>(key & 0xffffu);
    Nv[static_cast<size_t>(c)].push_back(d);
    Nv[static_cast<size_t>(d)].push_back(c);
  }
  for (auto& x : Nv) std::sort(x.begin(), x.end());
  auto shared = [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    size_t i = 0, j = 0, n = 0;
    while (i < a.size() && j < b.size()) {
      if (a[i] == b[j]) { ++n; ++i; ++j; }
      else if (a[i] < b[j]) ++i;
      else ++j;
    }
    return n;
  };
  std::vector<std::vector<int32_t>> N = Nv;
  for (uint32_t key : cand) {
    const int32_t c = static_cast<int32_t>(key >> 16), d = static_cast<int32_t>(key & 0xffffu);
    if (shared(Nv[static_cast<size_t>(c)], Nv[static_cast<size_t>(d)]) >= 2) continue;
    N[static_cast<size_t>(c)].push_back(d);
    N[static_cast<size_t>(d)].push_back(c);
  }
  for (auto& x : N) {
    std::sort(x.begin(), x.end());
    x.erase(std::unique(x.begin(), x.end()), x.end());
  }
  std::vector<std::array<int32_t, 3>> tri;
  for (int32_t i = 0; i < k; ++i) {
    const auto& Ni = N[static_cast<size_t>(i)];
    for (int32_t j : Ni) {
      if (j <= i) continue;
      const auto& Nj = N[static_cast<size_t>(j)];
      size_t a = 0, b = 0;
      while (a < Ni.size() && b < Nj.size()) {
        if (Ni[a] == Nj[b]) {
          if (Ni[a] > j) tri.push_back({i, j, Ni[a]});
          ++a;
          ++b;
        } else if (Ni[a] < Nj[b]) {
          ++a;
        } else {
          ++b;
        }
      }
    }
  }
  std::sort(tri.begin(), tri.end());
  std::vector<char> spurious(tri.size(), 0);
  for (int32_t i = 0; i < k; ++i) {
    const auto& Ni = N[static_cast<size_t>(i)];
    if (Ni.size() != 3) continue;
    const std::array<int32_t, 3> t3 = {Ni[0], Ni[1], Ni[2]};
    auto it = std::lower_bound(tri.begin(), tri.end(), t3);
    if (it != tri.end() && *it == t3) spurious[static_cast<size_t>(it - tri.begin())] = 1;
  }
  std::vector<std::array<int32_t, 3>> kept;
  for (size_t t = 0; t < tri.size(); ++t)
    if (!spurious[t]) kept.push_back(tri[t]);
  // orientation
  std::unordered_map<uint64_t, std::vector<int32_t>> edge_tris;
  auto ekey = [](int32_t u, int32_t v) {
    return (static_cast<uint64_t>(std::min(u, v)) << 32) | static_cast<uint32_t>(std::max(u, v));
  };
  for (size_t t = 0; t < kept.size(); ++t) {
    const auto& x = kept[t];
    edge_tris[ekey(x[0], x[1])].push_back(static_cast<int32_t>(t));
    edge_tris[ekey(x[1], x[2])].push_back(static_cast<int32_t>(t));
    edge_tris[ekey(x[0], x[2])].push_back(static_cast<int32_t>(t));
  }
  std::vector<std::array<int32_t, 3>> out(kept.size());
  std::vector<char> done(kept.size(), 0);
  std::deque<int32_t> q;
  for (size_t start = 0; start < kept.size(); ++start) {
    if (done[start]) continue;
    const int32_t a = kept[start][0], b = kept[start][1], c = kept[start][2];
    const double* pa = &pos[3 * static_cast<size_t>(a)];
    const double* pb = &pos[3 * static_cast<size_t>(b)];
    const double* pc = &pos[3 * static_cast<size_t>(c)];
    const double u[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
    const double w[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
    const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double sdot = 0.0;
    for (int j = 0; j < 3; ++j)
      sdot += n[j] * (nrm[3 * static_cast<size_t>(a) + j] + nrm[3 * static_cast<size_t>(b) + j] +
                      nrm[3 * static_cast<size_t>(c) + j]);
    out[start] = sdot >= 0.0 ? std::array<int32_t, 3>{a, b, c} : std::array<int32_t, 3>{a, c, b};
    done[start] = 1;
    q.push_back(static_cast<int32_t>(start));
    while (!q.empty()) {
      const int32_t ti = q.front();
      q.pop_front();
      const auto o = out[static_cast<size_t>(ti)];
      const int32_t de[3][2] = {{o[0], o[1]}, {o[1], o[2]}, {o[2], o[0]}};
      for (const auto& e : de) {
        for (int32_t tj : edge_tris[ekey(e[0], e[1])]) {
          if (done[static_cast<size_t>(tj)]) continue;
          const auto& x = kept[static_cast<size_t>(tj)];
          // the neighbour runs e[1] -> e[0]
          const bool fwd = (x[0] == e[1] && x[1] == e[0]) || (x[1] == e[1] && x[2] == e[0]) ||
                           (x[2] == e[1] && x[0] == e[0]);
          out[static_cast<size_t>(tj)] = fwd ? x : std::array<int32_t, 3>{x[0], x[2], x[1]};
          done[static_cast<size_t>(tj)] = 1;
          q.push_back(tj);
        }
      }
    }
  }
  return out;
}

uint32_t next_pow2(uint64_t x) {
  uint32_t p = 1;
  while (p < x && p < (1u << 31)) p <<= 1;
  return p;
}

lf_status dual_scratch(lf_mesh m, int64_t k, uint32_t cap) {
  if (m->dual_k == k && m->dual.cap >= cap) return LF_OK;
  for (void* p : {static_cast<void*>(m->dual.Hv), static_cast<void*>(m->dual.Hc), static_cast<void*>(m->dual.out_v),
                  static_cast<void*>(m->dual.out_c), static_cast<void*>(m->dual.counters),
                  static_cast<void*>(m->dual.cell_of), static_cast<void*>(m->dual.nrm),
                  static_cast<void*>(m->dual.pos), static_cast<void*>(m->d_dual_seeds)})
    m->dfree(p);
  m->dual = lf::DualScratch{};
  m->d_dual_seeds = nullptr;
  m->dual_k = 0;
  m->dual.cap = cap;
  m->dual.Hv = static_cast<uint32_t*>(m->dalloc(sizeof(uint32_t) * cap));
  m->dual.Hc = static_cast<uint32_t*>(m->dalloc(sizeof(uint32_t) * cap));
  m->dual.out_v = static_cast<uint32_t*>(m->dalloc(sizeof(uint32_t) * cap));
  m->dual.out_c = static_cast<uint32_t*>(m->dalloc(sizeof(uint32_t) * cap));
  m->dual.counters = static_cast<uint32_t*>(m->dalloc(sizeof(uint32_t) * 4));
  m->dual.cell_of = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * m->n_v));
  m->dual.nrm = static_cast<double*>(m->dalloc(sizeof(double) * 3 * k));
  m->dual.pos = static_cast<double*>(m->dalloc(sizeof(double) * 3 * k));
  m->d_dual_seeds = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * k));
  if (!m->dual.Hv || !m->dual.Hc || !m->dual.out_v || !m->dual.out_c || !m->dual.counters || !m->dual.cell_of ||
      !m->dual.nrm || !m->dual.pos || !m->d_dual_seeds)
    return fail(m, LF_ERR_OOM, "dual-mesh scratch");
  m->dual_k = k;
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_extract_dual(lf_mesh m, int32_t* tris, int64_t cap, int64_t* n_tris) {
  lf::TraceRange trace("lf_extract_dual");
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (!n_tris) return fail(m, LF_ERR_INVALID, "n_tris must not be NULL");
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed must come first");
  if (!m->d_V) return fail(m, LF_ERR_STATE, "the dual mesh needs a mesh made by lf_create_mesh");
  const int64_t k = m->n_layers - 1;
  if (static_cast<int64_t>(m->seeds.size()) != k)
    return fail(m, LF_ERR_STATE, "the seeds of the current field are unknown (lf_seed sets them)");
  const double iso = m->params.iso;
  if (!(iso >= 1.0 / 16.0 && iso <= 1.0)) return fail(m, LF_ERR_INVALID, "iso must lie in [1/16, 1]");
  if (m->dual_version != m->version || m->dual_steps != m->steps) {
    s = read_status(m);
    if (s != LF_OK) return s;
    const int cur = static_cast<int>(m->h_st.epoch & 1u);
    uint32_t tab = next_pow2(std::max<uint64_t>(4096, 16 * static_cast<uint64_t>(k)));
    uint32_t counters[4] = {0, 0, 0, 0};
    for (int attempt = 0;; ++attempt) {
      s = dual_scratch(m, k, tab);
      if (s != LF_OK) return s;
      LF_CUDA(m, cudaMemcpyAsync(m->d_dual_seeds, m->seeds.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice,
                                 m->stream));
      LF_CUDA(m, lf::launch_dual(m->h_job, cur, m->dtype, m->d_V, m->d_tri, static_cast<int>(m->n_f),
                                 static_cast<int>(k), static_cast<float>(iso), m->d_dual_seeds, m->dual, m->stream));
      LF_CUDA(m, cudaMemcpyAsync(counters, m->dual.counters, sizeof(counters), cudaMemcpyDeviceToHost, m->stream));
      LF_CUDA(m, cudaStreamSynchronize(m->stream));
      if (counters[0] == 0u) break;
      if (attempt >= 6 || tab >= (1u << 30)) return fail(m, LF_ERR_CAPACITY, "too many cell pairs");
      tab *= 4;                                   // a set ran full: larger tables, again
    }
    std::vector<uint32_t> av(counters[1]), cand(counters[2]);
    std::vector<double> pos(3 * static_cast<size_t>(k)), nrm(3 * static_cast<size_t>(k));
    if (!av.empty())
      LF_CUDA(m, cudaMemcpyAsync(av.data(), m->dual.out_v, sizeof(uint32_t) * av.size(), cudaMemcpyDeviceToHost,
                                 m->stream));
    if (!cand.empty())
      LF_CUDA(m, cudaMemcpyAsync(cand.data(), m->dual.out_c, sizeof(uint32_t) * cand.size(),
                                 cudaMemcpyDeviceToHost, m->stream));
    LF_CUDA(m, cudaMemcpyAsync(pos.data(), m->dual.pos, sizeof(double) * pos.size(), cudaMemcpyDeviceToHost,
                               m->stream));
    LF_CUDA(m, cudaMemcpyAsync(nrm.data(), m->dual.nrm, sizeof(double) * nrm.size(), cudaMemcpyDeviceToHost,
                               m->stream));
    LF_CUDA(m, cudaStreamSynchronize(m->stream));
    std::sort(av.begin(), av.end());
    std::sort(cand.begin(), cand.end());
    const auto t3 = dual_graph(static_cast<int>(k), av, cand, pos, nrm);
    m->dual_tris.resize(3 * t3.size());
    for (size_t t = 0; t < t3.size(); ++t)
      for (int j = 0; j < 3; ++j) m->dual_tris[3 * t + j] = m->seeds[static_cast<size_t>(t3[t][j])];
    m->dual_version = m->version;
    m->dual_steps = m->steps;
  }
  const int64_t n = static_cast<int64_t>(m->dual_tris.size() / 3);
  *n_tris = n;
  if (!tris) return LF_OK;
  if (cap < n) return fail(m, LF_ERR_CAPACITY, "tris holds fewer than *n_tris triangles");
  if (n > 0) std::memcpy(tris, m->dual_tris.data(), sizeof(int32_t) * 3 * n);
  return LF_OK;
}

lf_status lf_lloyd(lf_mesh m, int32_t rounds, int32_t steps_per_round, int32_t* seeds_out) {
  lf::TraceRange trace("lf_lloyd");
  lf_status s = check_usable(m);
  if (s != LF_OK) return s;
  if (rounds < 0 || steps_per_round < 0) return fail(m, LF_ERR_INVALID, "rounds and steps_per_round must be >= 0");
  if (m->n_layers == 0) return fail(m, LF_ERR_STATE, "lf_seed must come first");
  if (!m->d_V) return fail(m, LF_ERR_STATE, "the Lloyd-like update needs a mesh made by lf_create_mesh");
  const int64_t k = m->n_layers - 1;
  if (static_cast<int64_t>(m->seeds.size()) != k)
    return fail(m, LF_ERR_STATE, "the seeds of the current field are unknown (lf_seed sets them)");
  if (m->lloyd_k != k) {
    for (void* p : {static_cast<void*>(m->lloyd.acc), static_cast<void*>(m->lloyd.frame),
                    static_cast<void*>(m->lloyd.best), static_cast<void*>(m->lloyd.owner),
                    static_cast<void*>(m->lloyd.rounds), static_cast<void*>(m->d_seed_old),
                    static_cast<void*>(m->d_seed_new)})
      m->dfree(p);
    m->lloyd.acc = static_cast<double*>(m->dalloc(sizeof(double) * 7 * k));
    m->lloyd.frame = static_cast<double*>(m->dalloc(sizeof(double) * 7 * k));
    m->lloyd.best = static_cast<unsigned long long*>(m->dalloc(sizeof(unsigned long long) * 2 * k));
    m->lloyd.owner = static_cast<unsigned long long*>(m->dalloc(sizeof(unsigned long long) * m->n_v));
    m->lloyd.rounds = static_cast<int32_t*>(m->dalloc(sizeof(int32_t)));
    m->d_seed_old = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * k));
    m->d_seed_new = static_cast<int32_t*>(m->dalloc(sizeof(int32_t) * k));
    if (!m->lloyd.acc || !m->lloyd.frame || !m->lloyd.best || !m->lloyd.owner || !m->lloyd.rounds ||
        !m->d_seed_old || !m->d_seed_new) {
      m->lloyd_k = 0;
      return fail(m, LF_ERR_OOM, "Lloyd scratch");
    }
    m->lloyd_k = k;
  }
  for (int32_t r = 0; r < rounds; ++r) {
    s = read_status(m);
    if (s != LF_OK) return s;
    const int cur = static_cast<int>(m->h_st.epoch & 1u);
    std::vector<int32_t> fresh(static_cast<size_t>(k));
    LF_CUDA(m, cudaMemcpyAsync(m->d_seed_old, m->seeds.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice,
                               m->stream));
    LF_CUDA(m, lf::launch_lloyd(m->h_job, cur, m->d_V, m->d_tri, static_cast<int>(m->n_f), static_cast<int>(k),
                                m->d_seed_old, m->d_seed_new, m->lloyd, m->stream));
    LF_CUDA(m, cudaMemcpyAsync(fresh.data(), m->d_seed_new, sizeof(int32_t) * k, cudaMemcpyDeviceToHost,
                               m->stream));
    LF_CUDA(m, cudaStreamSynchronize(m->stream));
    s = lf_seed(m, fresh.data(), static_cast<int32_t>(k));     // the new partition starts from the new seeds
    if (s == LF_OK) s = lf_step(m, steps_per_round);
    if (s != LF_OK) return s;
  }
  if (seeds_out) std::memcpy(seeds_out, m->seeds.data(), sizeof(int32_t) * k);
  return LF_OK;
}

lf_status lf_stats(lf_mesh m, lf_stats_t* out) {
  if (!m || !out) return fail(m, LF_ERR_INVALID, "null argument");
  if (!m->poisoned) {
    lf_status s = read_status(m);
    if (s != LF_OK) return s;
  }
  std::memset(out, 0, sizeof(*out));
  out->n_v = m->n_v;
  out->n_layers = m->n_layers;
  out->steps = m->steps;
  out->nnz = m->n_layers > 0 ? static_cast<int64_t>(m->h_st.nnz) : 0;
  out->capacity = m->buffer_entries();
  out->operator_nnz = m->L_nnz;
  out->skeleton_total = m->h_st.skeleton_total;
  out->nnz_io_total = m->h_st.nnz_io_total;
  out->device_bytes = m->device_bytes;
  out->retries = m->retries;
  out->map_slots = lf::step_slots();
  out->field_dtype = m->dtype;
  out->value_bytes = lf::value_bytes(m->dtype);
  return LF_OK;
}

void lf_destroy_mesh(lf_mesh m) { delete m; }

const char* lf_status_string(lf_status s) {
  switch (s) {
    case LF_OK: return "LF_OK";
    case LF_ERR_INVALID: return "LF_ERR_INVALID";
    case LF_ERR_OOM: return "LF_ERR_OOM";
    case LF_ERR_CUDA: return "LF_ERR_CUDA";
    case LF_ERR_TIMEOUT: return "LF_ERR_TIMEOUT";
    case LF_ERR_STATE: return "LF_ERR_STATE";
    case LF_ERR_CAPACITY: return "LF_ERR_CAPACITY";
  }
  return "LF_ERR_UNKNOWN";
}

const char* lf_last_error(lf_mesh m) { return m ? m->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
