// Lloyd-like reseeding (Sec. 5): every cell's centre of mass and normal from
// the current field, the back-projection of the centre onto the cell, the new
// seed, and the separation of cells that pick the same vertex.
//
// Cell c consists of the vertices with an entry of layer c in the field (all
// stored entries are positive) and of the faces with at least one such vertex.
// Geometry is FP64; the per-cell sums use FP64 atomics, so their rounding
// order varies from run to run (a near-tie between two hits or two vertices
// can then go either way).

#include <cuda_runtime.h>
#include <stdint.h>

#include "lf_internal.h"

namespace lf {
namespace {

constexpr int kThreads = 256;
constexpr int kAcc = 7;        // per cell: area, area * barycentre (3), area * unit normal (3)

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 vertex(const double* V, int i) { return {V[3 * i], V[3 * i + 1], V[3 * i + 2]}; }

// Calls fn(c) once for every distinct cell (< k) present at the face's three
// vertices.  Rows are short and sorted, so duplicates are found by scanning
// the earlier rows.
template <class Fn>
__device__ __forceinline__ void for_each_cell(const int2* rows, const uint16_t* ids, const int v[3], int k, Fn fn) {
  int2 r[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = rows[v[a]];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int p = r[a].x; p < r[a].x + r[a].y; ++p) {
      const int c = ids[p];
      if (c >= k) continue;
      bool seen = false;
      for (int b = 0; b < a && !seen; ++b)
        for (int q = r[b].x; q < r[b].x + r[b].y; ++q)
          if (ids[q] == c) { seen = true; break; }
      if (!seen) fn(c);
    }
  }
}

// Moller-Trumbore for the whole line o + s d against the closed triangle.
__device__ bool line_hit(D3 o, D3 d, D3 a, D3 b, D3 c, double& s) {
  const D3 e1 = sub(b, a), e2 = sub(c, a);
  const D3 p = cross(d, e2);
  const double det = dot(e1, p);
  if (det == 0.0) return false;
  const D3 tv = sub(o, a);
  const double u = dot(tv, p) / det;
  const D3 q = cross(tv, e1);
  const double v = dot(d, q) / det;
  s = dot(e2, q) / det;
  return !(u < 0.0 || v < 0.0 || u + v > 1.0);
}

__global__ void cell_accumulate_kernel(const int2* rows, const uint16_t* ids, const double* V, const int32_t* tri,
                                       int n_f, int k, double* acc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_f) return;
  const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  const D3 a = vertex(V, v[0]), b = vertex(V, v[1]), c = vertex(V, v[2]);
  const D3 cr = cross(sub(b, a), sub(c, a));
  const double twice = sqrt(dot(cr, cr));
  const double area = 0.5 * twice;
  const D3 bary = {(a.x + b.x + c.x) / 3.0, (a.y + b.y + c.y) / 3.0, (a.z + b.z + c.z) / 3.0};
  const D3 n = {cr.x / twice, cr.y / twice, cr.z / twice};
  for_each_cell(rows, ids, v, k, [&](int cell) {
    double* s = acc + static_cast<int64_t>(cell) * kAcc;
    atomicAdd(s + 0, area);
    atomicAdd(s + 1, area * bary.x);
    atomicAdd(s + 2, area * bary.y);
    atomicAdd(s + 3, area * bary.z);
    atomicAdd(s + 4, area * n.x);
    atomicAdd(s + 5, area * n.y);
    atomicAdd(s + 6, area * n.z);
  });
}

// acc[c] -> frame[c] = (centre of mass, unit direction, valid); best keys reset.
__global__ void cell_frame_kernel(const double* acc, double* frame, unsigned long long* best, int k) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const double* s = acc + static_cast<int64_t>(c) * kAcc;
  double* f = frame + static_cast<int64_t>(c) * kAcc;
  const double A = s[0];
  const D3 N = {s[4], s[5], s[6]};
  const double nn = sqrt(dot(N, N));
  const bool ok = A > 0.0 && nn > 0.0;
  f[0] = ok ? s[1] / A : 0.0;
  f[1] = ok ? s[2] / A : 0.0;
  f[2] = ok ? s[3] / A : 0.0;
  f[3] = ok ? N.x / nn : 0.0;
  f[4] = ok ? N.y / nn : 0.0;
  f[5] = ok ? N.z / nn : 0.0;
  f[6] = ok ? 1.0 : 0.0;
  best[2 * c] = ~0ull;          // |s| of the nearest hit, as ordered bits
  best[2 * c + 1] = ~0ull;      // lowest face id among hits at that |s|
}

__device__ __forceinline__ bool frame_of(const double* frame, int c, D3& P, D3& d) {
  const double* f = frame + static_cast<int64_t>(c) * kAcc;
  if (f[6] == 0.0) return false;
  P = {f[0], f[1], f[2]};
  d = {f[3], f[4], f[5]};
  return true;
}

// pass 0: nearest |s| per cell; pass 1: lowest face id at that |s|
__global__ void cell_ray_kernel(const int2* rows, const uint16_t* ids, const double* V, const int32_t* tri, int n_f,
                                int k, const double* frame, unsigned long long* best, int pass) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_f) return;
  const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  const D3 a = vertex(V, v[0]), b = vertex(V, v[1]), c = vertex(V, v[2]);
  for_each_cell(rows, ids, v, k, [&](int cell) {
    D3 P, d;
    if (!frame_of(frame, cell, P, d)) return;
    double s;
    if (!line_hit(P, d, a, b, c, s)) return;
    const unsigned long long key = static_cast<unsigned long long>(__double_as_longlong(fabs(s)));
    if (pass == 0) atomicMin(&best[2 * cell], key);
    else if (key == best[2 * cell]) atomicMin(&best[2 * cell + 1], static_cast<unsigned long long>(t));
  });
}

// New seed per cell: the vertex of the winning face nearest to the hit point
// (ties to the lowest vertex id); a miss keeps the old seed.
__global__ void cell_pick_kernel(const double* V, const int32_t* tri, int k, const double* frame,
                                 const unsigned long long* best, const int32_t* old_seed, int32_t* cand) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  int out = old_seed[c];
  D3 P, d;
  const unsigned long long t = best[2 * c + 1];
  if (t != ~0ull && frame_of(frame, c, P, d)) {
    const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    const D3 a = vertex(V, v[0]), b = vertex(V, v[1]), cc = vertex(V, v[2]);
    double s;
    if (line_hit(P, d, a, b, cc, s)) {
      const D3 X = {P.x + s * d.x, P.y + s * d.y, P.z + s * d.z};
      double bd = 0.0;
      int bv = -1;
      const D3 q[3] = {a, b, cc};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const D3 e = sub(q[j], X);
        const double dist = sqrt(dot(e, e));
        if (bv < 0 || dist < bd || (dist == bd && v[j] < bv)) { bd = dist; bv = v[j]; }
      }
      out = bv;
    }
  }
  cand[c] = out;
}

// Distinct seeds, in synchronous rounds: every vertex held by several cells
// goes to the cell that holds it as its old seed, else to the lowest cell id;
// the others return to their old seeds.  Old seeds are distinct, so at most
// k rounds change anything.  One CTA.
__global__ void resolve_kernel(const int32_t* old_seed, int32_t* cur, int k, unsigned long long* owner,
                               int32_t* rounds_out) {
  __shared__ int changed;
  int round = 0;
  for (; round <= k; ++round) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) owner[cur[c]] = ~0ull;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      const unsigned long long key =
          (cur[c] == old_seed[c] ? 0ull : (1ull << 32)) | static_cast<unsigned long long>(c);
      atomicMin(&owner[cur[c]], key);
    }
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      if (static_cast<int>(owner[cur[c]] & 0xffffffffull) != c) {
        cur[c] = old_seed[c];
        changed = 1;
      }
    }
    __syncthreads();
    if (!changed) break;
  }
  if (threadIdx.x == 0) *rounds_out = round;
}

inline unsigned blocks(int64_t n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_lloyd(const JobDesc& job, int buf, const double* V, const int32_t* tri, int n_f, int k,
                         const int32_t* old_seed, int32_t* new_seed, LloydScratch sc, cudaStream_t s) {
  const int2* rows = job.buf[buf].rows;
  const uint16_t* ids = job.buf[buf].ids;
  cudaError_t e = cudaMemsetAsync(sc.acc, 0, sizeof(double) * kAcc * static_cast<size_t>(k), s);
  if (e != cudaSuccess) return e;
  if (n_f > 0) cell_accumulate_kernel<<<blocks(n_f), kThreads, 0, s>>>(rows, ids, V, tri, n_f, k, sc.acc);
  cell_frame_kernel<<<blocks(k), kThreads, 0, s>>>(sc.acc, sc.frame, sc.best, k);
  for (int pass = 0; pass < 2 && n_f > 0; ++pass)
    cell_ray_kernel<<<blocks(n_f), kThreads, 0, s>>>(rows, ids, V, tri, n_f, k, sc.frame, sc.best, pass);
  cell_pick_kernel<<<blocks(k), kThreads, 0, s>>>(V, tri, k, sc.frame, sc.best, old_seed, new_seed);
  resolve_kernel<<<1, 1024, 0, s>>>(old_seed, new_seed, k, sc.owner, sc.rounds);
  return cudaGetLastError();
}

int lloyd_acc_doubles() { return kAcc; }

}  // namespace lf
