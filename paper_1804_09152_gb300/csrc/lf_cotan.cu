// Cotangent Laplacian of a triangle mesh, built on the device (Sec. 3.2: the
// method diffuses with a Laplacian of the surface; the cotangent weights are
// this library's discretisation).
//
// For the corner p of face (p, q, s) the edge (q, s) receives half the
// cotangent of the angle at p; L_ij sums those over the faces around the edge
// (i, j).  Only the off-diagonal entries are stored (L_ii = -sum_j L_ij is
// rebuilt by the step kernel).  Every value is FP64 with explicitly rounded
// operations, and the duplicates of an edge are summed in face order, then
// rounded to FP32 once: the same bits as the host assembly in lf_host.cpp,
// which takes the same operations in the same order.
//
// Passes: corners (per face: half cotangents, incident-face counts), scan,
// incidence (per face: scatter the face id into each corner's list), rows
// (per vertex: sort its faces, then count and later write its distinct
// neighbours in increasing column order), scan, rows again.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "lf_internal.h"

namespace lf {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;   // elements per scan block

__global__ void corner_kernel(const double* __restrict__ V, const int32_t* __restrict__ tri, int64_t n_f,
                              double* __restrict__ hc, int32_t* __restrict__ inc_cnt,
                              unsigned long long* __restrict__ bad_face) {
  const int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= n_f) return;
  const int32_t v[3] = {tri[3 * f], tri[3 * f + 1], tri[3 * f + 2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* P = V + 3 * static_cast<int64_t>(v[c]);
    const double* Q = V + 3 * static_cast<int64_t>(v[(c + 1) % 3]);
    const double* S = V + 3 * static_cast<int64_t>(v[(c + 2) % 3]);
    const double ux = __dsub_rn(Q[0], P[0]), uy = __dsub_rn(Q[1], P[1]), uz = __dsub_rn(Q[2], P[2]);
    const double wx = __dsub_rn(S[0], P[0]), wy = __dsub_rn(S[1], P[1]), wz = __dsub_rn(S[2], P[2]);
    const double cx = __dsub_rn(__dmul_rn(uy, wz), __dmul_rn(uz, wy));
    const double cy = __dsub_rn(__dmul_rn(uz, wx), __dmul_rn(ux, wz));
    const double cz = __dsub_rn(__dmul_rn(ux, wy), __dmul_rn(uy, wx));
    const double twice_area =
        __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz)));
    double h = 0.0;
    if (!(twice_area > 0.0) || !isfinite(twice_area)) {
      atomicMin(bad_face, static_cast<unsigned long long>(f));
    } else {
      const double dot = __dadd_rn(__dadd_rn(__dmul_rn(ux, wx), __dmul_rn(uy, wy)), __dmul_rn(uz, wz));
      h = __ddiv_rn(__dmul_rn(0.5, dot), twice_area);
    }
    hc[3 * f + c] = h;
    atomicAdd(&inc_cnt[v[c]], 1);
  }
}

__global__ void incidence_kernel(const int32_t* __restrict__ tri, int64_t n_f, const int32_t* __restrict__ inc_start,
                                 int32_t* __restrict__ fill, int32_t* __restrict__ inc) {
  const int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= n_f) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int32_t v = tri[3 * f + c];
    inc[inc_start[v] + atomicAdd(&fill[v], 1)] = static_cast<int32_t>(f);
  }
}

// One thread per vertex.  Pass 0 sorts the vertex's face list (ascending face
// id, the host's order) and counts its distinct neighbours into cnt; pass 1
// writes them, each weight summed over the faces in that order.
__global__ void rows_kernel(const int32_t* __restrict__ tri, const double* __restrict__ hc, int64_t n_v,
                            const int32_t* __restrict__ inc_start, int32_t* __restrict__ inc, int pass,
                            int32_t* __restrict__ cnt, const int32_t* __restrict__ rowptr, int2* __restrict__ colval) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const int32_t a = inc_start[i], b = inc_start[i + 1];
  if (pass == 0) {
    for (int32_t x = a + 1; x < b; ++x) {        // insertion sort; lists are short on meshes
      const int32_t fx = inc[x];
      int32_t y = x - 1;
      while (y >= a && inc[y] > fx) {
        inc[y + 1] = inc[y];
        --y;
      }
      inc[y + 1] = fx;
    }
  }
  // the two entries of face f in row i, in corner order: corner c adds the
  // half cotangent hc[3f + c] to the edge between the other two corners
  auto scan = [&](int32_t cur, double& w) {
    int32_t nx = INT_MAX;
    w = 0.0;
    for (int32_t x = a; x < b; ++x) {
      const int64_t f = inc[x];
      const int32_t v[3] = {__ldg(tri + 3 * f), __ldg(tri + 3 * f + 1), __ldg(tri + 3 * f + 2)};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int32_t q = v[(c + 1) % 3], t = v[(c + 2) % 3];
        int32_t col = -1;
        if (q == i) col = t;
        else if (t == i) col = q;
        if (col < 0) continue;
        if (col == cur) w = __dadd_rn(w, __ldg(hc + 3 * f + c));
        else if (col > cur && col < nx) nx = col;
      }
    }
    return nx;
  };
  double w;
  int32_t cur = scan(-1, w);
  int32_t n = 0;
  while (cur != INT_MAX) {
    const int32_t nx = scan(cur, w);
    if (pass == 1) colval[rowptr[i] + n] = make_int2(cur, __float_as_int(__double2float_rn(w)));
    ++n;
    cur = nx;
  }
  if (pass == 0) cnt[i] = n;
}

// Exclusive scan in three launches: block scans with block totals, a scan of
// the totals by one block, the block offsets added back.  out has n + 1
// entries; out[n] is the total.
__device__ __forceinline__ int32_t block_excl_scan(int32_t x, int32_t* s_warp, int32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t y = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t z = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) y += z;
  }
  if (lane == 31) s_warp[warp] = y;
  __syncthreads();
  int32_t off = 0;
  total = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
    if (w < warp) off += s_warp[w];
    total += s_warp[w];
  }
  __syncthreads();
  return off + y - x;
}

__global__ void scan_blocks_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ out,
                                   int32_t* __restrict__ block_sum) {
  __shared__ int32_t s_warp[kScanThreads / 32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanBlock + static_cast<int64_t>(threadIdx.x) * kScanItems;
  int32_t v[kScanItems];
  int32_t sum = 0;
#pragma unroll
  for (int u = 0; u < kScanItems; ++u) {
    v[u] = base + u < n ? in[base + u] : 0;
    sum += v[u];
  }
  int32_t total;
  int32_t run = block_excl_scan(sum, s_warp, total);
#pragma unroll
  for (int u = 0; u < kScanItems; ++u) {
    if (base + u < n) out[base + u] = run;
    run += v[u];
  }
  if (threadIdx.x == 0) block_sum[blockIdx.x] = total;
}

__global__ void scan_totals_kernel(int32_t* __restrict__ block_sum, int64_t n_blocks, int32_t* __restrict__ out_total) {
  __shared__ int32_t s_warp[kScanThreads / 32];
  int32_t carry = 0;
  for (int64_t b0 = 0; b0 < n_blocks; b0 += kScanThreads) {
    const int64_t b = b0 + threadIdx.x;
    const int32_t x = b < n_blocks ? block_sum[b] : 0;
    int32_t total;
    const int32_t e = block_excl_scan(x, s_warp, total);
    if (b < n_blocks) block_sum[b] = carry + e;
    carry += total;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ block_sum) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_sum[i / kScanBlock];
}

unsigned grid_for(int64_t n, int threads) { return static_cast<unsigned>((n + threads - 1) / threads); }

}  // namespace

int64_t cotan_scan_blocks(int64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* block_sum, cudaStream_t s) {
  const int64_t nb = cotan_scan_blocks(n);
  if (nb > 0) scan_blocks_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, out, block_sum);
  scan_totals_kernel<<<1, kScanThreads, 0, s>>>(block_sum, nb, out + n);
  if (n > 0) scan_add_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n, block_sum);
  return cudaGetLastError();
}

cudaError_t launch_cotan_corners(const double* V, const int32_t* tri, int64_t n_f, double* hc, int32_t* inc_cnt,
                                 unsigned long long* bad_face, cudaStream_t s) {
  if (n_f > 0) corner_kernel<<<grid_for(n_f, 256), 256, 0, s>>>(V, tri, n_f, hc, inc_cnt, bad_face);
  return cudaGetLastError();
}

cudaError_t launch_cotan_incidence(const int32_t* tri, int64_t n_f, const int32_t* inc_start, int32_t* fill,
                                   int32_t* inc, cudaStream_t s) {
  if (n_f > 0) incidence_kernel<<<grid_for(n_f, 256), 256, 0, s>>>(tri, n_f, inc_start, fill, inc);
  return cudaGetLastError();
}

cudaError_t launch_cotan_rows(const int32_t* tri, const double* hc, int64_t n_v, const int32_t* inc_start,
                              int32_t* inc, int pass, int32_t* cnt, const int32_t* rowptr, int2* colval,
                              cudaStream_t s) {
  if (n_v > 0)
    rows_kernel<<<grid_for(n_v, 128), 128, 0, s>>>(tri, hc, n_v, inc_start, inc, pass, cnt, rowptr, colval);
  return cudaGetLastError();
}

}  // namespace lf
