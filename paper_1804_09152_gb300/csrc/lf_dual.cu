// Dual-mesh extraction (Sec. 5.2), the passes over the mesh: the cell pairs
// that cover a common vertex (A_v), the pairs that only meet on a face and
// whose isolines cross there, the mesh normals at the seed vertices and the
// seed positions.  The graph stage that follows (manifold check, triangles,
// orientation) works on k cells and runs on the host.
//
// A cell c covers vertex v when F(v, c) >= iso.  Pairs are kept in open-
// addressing hash sets of 32-bit keys (c << 16 | d, c < d < 65536).  The
// isoline test uses explicitly rounded FP64 operations in a fixed order, so
// its decisions do not depend on the compiler's contractions.

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lf_internal.h"

namespace lf {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kMaxCover = 16;     // covering cells per vertex (values >= iso sum to <= 1: at most 1 / iso)

template <int DT>
struct ValT;
template <>
struct ValT<0> {
  static __device__ __forceinline__ float load(const void* p, int64_t i) { return static_cast<const float*>(p)[i]; }
};
template <>
struct ValT<1> {
  static __device__ __forceinline__ float load(const void* p, int64_t i) {
    const uint16_t b = static_cast<const uint16_t*>(p)[i];
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
  }
};
template <>
struct ValT<2> {
  static __device__ __forceinline__ float load(const void* p, int64_t i) {
    return __half2float(__ushort_as_half(static_cast<const unsigned short*>(p)[i]));
  }
};

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ void set_insert(uint32_t* tab, uint32_t mask, uint32_t key, uint32_t* overflow) {
  uint32_t h = hash32(key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t prev = atomicCAS(&tab[h], kEmpty, key);
    if (prev == kEmpty || prev == key) return;
    h = (h + 1) & mask;
  }
  atomicOr(overflow, 1u);
}

__device__ __forceinline__ bool set_contains(const uint32_t* tab, uint32_t mask, uint32_t key) {
  uint32_t h = hash32(key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t x = tab[h];
    if (x == key) return true;
    if (x == kEmpty) return false;
    h = (h + 1) & mask;
  }
  return false;
}

// Covering cells of vertex v (ascending, as stored), at most kMaxCover.
template <int DT>
__device__ __forceinline__ int cover(const int2* rows, const uint16_t* ids, const void* vals, int v, int k, float iso,
                                     int* out) {
  const int2 r = rows[v];
  int n = 0;
  for (int p = r.x; p < r.x + r.y; ++p) {
    const int c = ids[p];
    if (c < k && ValT<DT>::load(vals, p) >= iso && n < kMaxCover) out[n++] = c;
  }
  return n;
}

template <int DT>
__device__ __forceinline__ double value_at(const int2* rows, const uint16_t* ids, const void* vals, int v, int c) {
  const int2 r = rows[v];
  for (int p = r.x; p < r.x + r.y; ++p)
    if (ids[p] == c) return static_cast<double>(ValT<DT>::load(vals, p));
  return 0.0;
}

struct P2 {
  double x, y;
};

// Isoline {phi = iso} on the reference triangle (0,0), (1,0), (0,1): two
// points, or false.  Edges in the order (0,1), (1,2), (2,0).
__device__ bool isoline(const double phi[3], double iso, P2& a, P2& b) {
  const P2 B[3] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  int n = 0;
  P2 pts[2];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int i = e, j = (e + 1) % 3;
    const double si = __dsub_rn(phi[i], iso), sj = __dsub_rn(phi[j], iso);
    if ((si >= 0.0) != (sj >= 0.0)) {
      const double t = __ddiv_rn(si, __dsub_rn(si, sj));
      const double u = __dsub_rn(1.0, t);
      if (n < 2) {
        pts[n].x = __dadd_rn(__dmul_rn(u, B[i].x), __dmul_rn(t, B[j].x));
        pts[n].y = __dadd_rn(__dmul_rn(u, B[i].y), __dmul_rn(t, B[j].y));
      }
      ++n;
    }
  }
  if (n != 2) return false;
  a = pts[0];
  b = pts[1];
  return true;
}

__device__ __forceinline__ double orient(P2 a, P2 b, P2 c) {
  return __dsub_rn(__dmul_rn(__dsub_rn(b.x, a.x), __dsub_rn(c.y, a.y)),
                   __dmul_rn(__dsub_rn(b.y, a.y), __dsub_rn(c.x, a.x)));
}

// Closed segments ab and cd.
__device__ bool segments_cross(P2 a, P2 b, P2 c, P2 d) {
  const double o1 = orient(a, b, c), o2 = orient(a, b, d), o3 = orient(c, d, a), o4 = orient(c, d, b);
  if (o1 == 0.0 && o2 == 0.0) {
    const bool ax = fabs(__dsub_rn(b.x, a.x)) >= fabs(__dsub_rn(b.y, a.y));
    const double a0 = ax ? a.x : a.y, a1 = ax ? b.x : b.y, c0 = ax ? c.x : c.y, c1 = ax ? d.x : d.y;
    const double lo1 = fmin(a0, a1), hi1 = fmax(a0, a1), lo2 = fmin(c0, c1), hi2 = fmax(c0, c1);
    return fmax(lo1, lo2) <= fmin(hi1, hi2);
  }
  return __dmul_rn(o1, o2) <= 0.0 && __dmul_rn(o3, o4) <= 0.0;
}

template <int DT>
__global__ void dual_vertex_kernel(const int2* rows, const uint16_t* ids, const void* vals, int n_v, int k, float iso,
                                   uint32_t* Hv, uint32_t mask, uint32_t* overflow) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_v) return;
  int cs[kMaxCover];
  const int n = cover<DT>(rows, ids, vals, v, k, iso, cs);
  for (int x = 0; x < n; ++x)
    for (int y = x + 1; y < n; ++y)
      set_insert(Hv, mask, (static_cast<uint32_t>(cs[x]) << 16) | static_cast<uint32_t>(cs[y]), overflow);
}

template <int DT>
__global__ void dual_face_kernel(const int2* rows, const uint16_t* ids, const void* vals, const int32_t* tri, int n_f,
                                 int k, float iso, const uint32_t* Hv, uint32_t* Hc, uint32_t mask,
                                 uint32_t* overflow) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_f) return;
  const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  int cs[3 * kMaxCover];
  int n = 0;
  for (int a = 0; a < 3; ++a) {
    int loc[kMaxCover];
    const int m = cover<DT>(rows, ids, vals, v[a], k, iso, loc);
    for (int q = 0; q < m; ++q) {
      bool seen = false;
      for (int r = 0; r < n; ++r) seen = seen || cs[r] == loc[q];
      if (!seen) cs[n++] = loc[q];
    }
  }
  // ascending, so every pair is (smaller, larger)
  for (int a = 1; a < n; ++a) {
    const int x = cs[a];
    int b = a - 1;
    for (; b >= 0 && cs[b] > x; --b) cs[b + 1] = cs[b];
    cs[b + 1] = x;
  }
  for (int x = 0; x < n; ++x) {
    for (int y = x + 1; y < n; ++y) {
      const uint32_t key = (static_cast<uint32_t>(cs[x]) << 16) | static_cast<uint32_t>(cs[y]);
      if (set_contains(Hv, mask, key)) continue;
      double pc[3], pd[3];
      for (int a = 0; a < 3; ++a) {
        pc[a] = value_at<DT>(rows, ids, vals, v[a], cs[x]);
        pd[a] = value_at<DT>(rows, ids, vals, v[a], cs[y]);
      }
      P2 a0, a1, b0, b1;
      const double isod = static_cast<double>(iso);
      if (isoline(pc, isod, a0, a1) && isoline(pd, isod, b0, b1) && segments_cross(a0, a1, b0, b1))
        set_insert(Hc, mask, key, overflow);
    }
  }
}

// Area-weighted mesh normals at the seed vertices (cell_of[v] = cell or -1),
// and the seed positions.
__global__ void seed_normal_kernel(const double* V, const int32_t* tri, int n_f, const int32_t* cell_of, double* nrm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_f) return;
  const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  int cells[3];
  bool any = false;
  for (int a = 0; a < 3; ++a) {
    cells[a] = cell_of[v[a]];
    any = any || cells[a] >= 0;
  }
  if (!any) return;
  const double* A = V + 3 * static_cast<int64_t>(v[0]);
  const double* B = V + 3 * static_cast<int64_t>(v[1]);
  const double* C = V + 3 * static_cast<int64_t>(v[2]);
  const double ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
  const double wx = C[0] - A[0], wy = C[1] - A[1], wz = C[2] - A[2];
  const double cx = 0.5 * (uy * wz - uz * wy), cy = 0.5 * (uz * wx - ux * wz), cz = 0.5 * (ux * wy - uy * wx);
  for (int a = 0; a < 3; ++a) {
    if (cells[a] < 0) continue;
    double* n = nrm + 3 * static_cast<int64_t>(cells[a]);
    atomicAdd(n + 0, cx);
    atomicAdd(n + 1, cy);
    atomicAdd(n + 2, cz);
  }
}

__global__ void seed_setup_kernel(const double* V, const int32_t* seeds, int k, int32_t* cell_of, double* pos) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int s = seeds[c];
  cell_of[s] = c;
  for (int j = 0; j < 3; ++j) pos[3 * c + j] = V[3 * static_cast<int64_t>(s) + j];
}

__global__ void compact_kernel(const uint32_t* tab, uint32_t cap, uint32_t* out, uint32_t* count) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cap) return;
  const uint32_t key = tab[s];
  if (key != kEmpty) out[atomicAdd(count, 1u)] = key;
}

inline unsigned blocks(int64_t n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }

template <int DT>
void launch_pairs(const JobDesc& job, int buf, const int32_t* tri, int n_f, int k, float iso, DualScratch sc,
                  cudaStream_t s) {
  const int2* rows = job.buf[buf].rows;
  const uint16_t* ids = job.buf[buf].ids;
  const void* vals = job.buf[buf].vals;
  const uint32_t mask = sc.cap - 1;
  dual_vertex_kernel<DT><<<blocks(job.n_v), kThreads, 0, s>>>(rows, ids, vals, job.n_v, k, iso, sc.Hv, mask,
                                                              sc.counters);
  if (n_f > 0)
    dual_face_kernel<DT><<<blocks(n_f), kThreads, 0, s>>>(rows, ids, vals, tri, n_f, k, iso, sc.Hv, sc.Hc, mask,
                                                          sc.counters);
}

}  // namespace

cudaError_t launch_dual(const JobDesc& job, int buf, int dtype, const double* V, const int32_t* tri, int n_f, int k,
                        float iso, const int32_t* d_seeds, DualScratch sc, cudaStream_t s) {
  // counters: [0] overflow, [1] |A_v|, [2] |candidates|
  cudaError_t e = cudaMemsetAsync(sc.counters, 0, 4 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.Hv, 0xff, sizeof(uint32_t) * sc.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.Hc, 0xff, sizeof(uint32_t) * sc.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.cell_of, 0xff, sizeof(int32_t) * job.n_v, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.nrm, 0, sizeof(double) * 3 * k, s);
  if (e != cudaSuccess) return e;
  switch (dtype) {
    case 0: launch_pairs<0>(job, buf, tri, n_f, k, iso, sc, s); break;
    case 1: launch_pairs<1>(job, buf, tri, n_f, k, iso, sc, s); break;
    default: launch_pairs<2>(job, buf, tri, n_f, k, iso, sc, s); break;
  }
  compact_kernel<<<blocks(sc.cap), kThreads, 0, s>>>(sc.Hv, sc.cap, sc.out_v, sc.counters + 1);
  compact_kernel<<<blocks(sc.cap), kThreads, 0, s>>>(sc.Hc, sc.cap, sc.out_c, sc.counters + 2);
  seed_setup_kernel<<<blocks(k), kThreads, 0, s>>>(V, d_seeds, k, sc.cell_of, sc.pos);
  if (n_f > 0) seed_normal_kernel<<<blocks(n_f), kThreads, 0, s>>>(V, tri, n_f, sc.cell_of, sc.nrm);
  return cudaGetLastError();
}

}  // namespace lf
