// Layered-field step on sm_103a: one fused kernel per time-iteration.
//
// One thread owns one vertex i.  It gathers the closed neighbourhood of i
// from L (CSR, off-diagonal only) and the field F (CSR, layer ids sorted),
// accumulating G = L F (the paper's L_t = Phi L^T, Algorithm 1) per layer in
// a register map of four cell slots and the base layer; applies the
// interest-skeleton test, the explicit Euler update of Eq. 11-13 in closed
// form, the clamp and the normalisation (Sec. 4); and writes the surviving
// entries of row i into the output CSR.  A vertex whose neighbourhood holds
// more layers than the map re-gathers into a map in shared memory, and past
// that takes a path that enumerates the layer union in increasing id order
// by repeated minimum search over the same rows, so any union size is exact
// without extra storage.  Every tier sums in the same order with explicitly
// rounded operations: a vertex's bits do not depend on its tier.
//
// The field is a tile-segmented CSR: the 256 vertices of a tile (one CTA)
// write their rows one after another into the tile's own segment, row
// offsets coming from a block-wide prefix sum of the row lengths.  No CTA
// waits for another, so one launch is one iteration with no host round trip;
// consecutive launches overlap through programmatic dependent launch.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lf_internal.h"

namespace lf {

namespace {

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------
template <int DT> struct Val;
// bits() / from_bits(): a stored value as the 32-bit word kept in a row's head
// record (16-bit types in the low half).
template <> struct Val<0> {
  using T = float;
  static __device__ __forceinline__ float load(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ T round(float v) { return v; }
  static __device__ __forceinline__ float widen(T v) { return v; }
  static __device__ __forceinline__ int bits(T v) { return __float_as_int(v); }
  static __device__ __forceinline__ float from_bits(int b) { return __int_as_float(b); }
};
template <> struct Val<1> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float load(const T* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ T round(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float widen(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ int bits(T v) { return static_cast<int>(__bfloat16_as_ushort(v)); }
  static __device__ __forceinline__ float from_bits(int b) { return __int_as_float(b << 16); }
};
template <> struct Val<2> {
  using T = __half;
  static __device__ __forceinline__ float load(const T* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ T round(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float widen(T v) { return __half2float(v); }
  static __device__ __forceinline__ int bits(T v) { return static_cast<int>(__half_as_ushort(v)); }
  static __device__ __forceinline__ float from_bits(int b) {
    return __half2float(__ushort_as_half(static_cast<unsigned short>(b)));
  }
};

// ---------------------------------------------------------------------------
// device-scope relaxed accesses and dependent-launch control
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Waits until the previous kernel in the stream has completed and its writes
// are visible (no-op when the launch carries no programmatic dependency).
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel in the stream start launching its CTAs.
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr int kBlock = kTile;   // threads (= vertices) per CTA
#ifndef LF_SLOTS
#define LF_SLOTS 5
#endif
constexpr int kSlots = LF_SLOTS; // register map slots of the fast path
constexpr int kChunk = 2;       // neighbours fetched per batch (register-map tier)
#ifndef LF_CHUNK0
#define LF_CHUNK0 4
#endif
constexpr int kChunk0 = LF_CHUNK0;  // neighbours fetched per batch (lean gather)
#ifndef LF_HOT_CELLS
#define LF_HOT_CELLS 5
#endif
constexpr int kHotCells = LF_HOT_CELLS;   // cells in the lean gather's register map
constexpr int kPool = 4;        // medium-path maps per CTA
constexpr int kMed = 32;        // slots of a medium-path map

// Per-vertex quantities of the closed-form update (class coefficients).
struct VertexSums {
  float sG, sF, r, Gb, Fb, sqFb;
  int nC, hasb;
};

// d for one skeleton entry, then the Euler step and the clamp.  With S the
// skeleton, A_j = sum_{l in S} a_jl G_l and W_j = sum_{l in S} w_jl F_l,
// Algorithm 1's double sum is -(mu/n)[1/2 (n A_j - sum A) + (n W_j - sum W)]
// and its band term (mu/n) sqrt(F_j) sum_k e_jk sqrt(F_k).
struct Update {
  // d_j is linear in G_j and F_j once the per-vertex sums are known:
  //   cell: d = (mu/n) (-K + gA G_j + fW F_j + sqrt(F_j) (R0 - e_cc sqrt(F_j)))
  //   base: d = (mu/n) (-Kb + sqrt(F_b) Rb)
  // with K = 1/2 (n a_cc sum_G + n [b] a_cb G_b - sum A) + (n w_cc sum_F + n [b] w_cb F_b - sum W),
  // gA = n a_cc / 2, fW = n w_cc, R0 = e_cc sum_sqrtF + [b] e_cb sqrt(F_b),
  // Kb = 1/2 (n a_cb sum_G - sum A) + (n w_cb sum_F - sum W), Rb = e_bc sum_sqrtF.
  // All roundings are explicit (no contraction left to the compiler), so every
  // tier that inlines this gives bit-identical results.
  float mun, K, gA, fW, R0, eS, Kb, Rb;
  __device__ __forceinline__ Update(const VertexSums& s, const Coefs& c) {
    const int n = s.nC + s.hasb;
    const float fn = static_cast<float>(n);
    const float fnc = static_cast<float>(s.nC);
    const float bA = s.hasb ? __fmul_rn(c.a_cb, __fmaf_rn(fnc, s.Gb, s.sG)) : 0.0f;
    const float bW = s.hasb ? __fmul_rn(c.w_cb, __fmaf_rn(fnc, s.Fb, s.sF)) : 0.0f;
    const float sumA = __fmaf_rn(__fmul_rn(c.a_cc, __fsub_rn(fnc, 1.0f)), s.sG, bA);
    const float sumW = __fmaf_rn(__fmul_rn(c.w_cc, __fsub_rn(fnc, 1.0f)), s.sF, bW);
    const float A0 = __fmaf_rn(c.a_cc, s.sG, s.hasb ? __fmul_rn(c.a_cb, s.Gb) : 0.0f);
    const float W0 = __fmaf_rn(c.w_cc, s.sF, s.hasb ? __fmul_rn(c.w_cb, s.Fb) : 0.0f);
    K = __fmaf_rn(0.5f, __fmaf_rn(fn, A0, -sumA), __fmaf_rn(fn, W0, -sumW));
    gA = __fmul_rn(0.5f, __fmul_rn(fn, c.a_cc));
    fW = __fmul_rn(fn, c.w_cc);
    R0 = __fmaf_rn(c.e_cc, s.r, s.hasb ? __fmul_rn(c.e_cb, s.sqFb) : 0.0f);
    eS = c.e_cc;
    Kb = __fmaf_rn(0.5f, __fmaf_rn(fn, __fmul_rn(c.a_cb, s.sG), -sumA),
                   __fmaf_rn(fn, __fmul_rn(c.w_cb, s.sF), -sumW));
    Rb = __fmul_rn(c.e_bc, s.r);
    mun = c.mu / fn;
  }
  // f, g: F and G of the entry; sqf = root(f), computed once by the caller.
  __device__ __forceinline__ float value(bool is_base, float f, float g, float sqf, const VertexSums&,
                                         const Coefs& c) const {
    const float k = is_base ? Kb : K;
    const float ga = is_base ? 0.0f : gA;
    const float fw = is_base ? 0.0f : fW;
    const float r0 = is_base ? Rb : R0;
    const float es = is_base ? 0.0f : eS;
    float t = __fmaf_rn(ga, g, -k);
    t = __fmaf_rn(fw, f, t);
    t = __fmaf_rn(sqf, __fmaf_rn(-es, sqf, r0), t);
    float v = __fmaf_rn(__fmul_rn(mun, t), c.dt, f);
    if (v > 1.0f) v = 1.0f;
    if (v <= 0.0f) v = 0.0f;
    return v;
  }
};

// Algorithm 1 with general coefficient matrices (w_jl, a_jl, e_jk): with
// A_j = sum_l a_jl G_l, W_j = sum_l w_jl F_l, E_j = sum_k e_jk sqrt(F_k) over
// the skeleton S (n entries), d_j = -(mu/n)[1/2 (n A_j - sum_S A) +
// (n W_j - sum_S W)] + (mu/n) sqrt(F_j) E_j.  A missing matrix falls back to
// the class rule of the coefficients.  Every sum runs in ascending layer
// order with explicit roundings, the same in every tier.
struct GenCoef {
  const float* W;
  const float* A;
  const float* E;
  int K1, base;
  Coefs c;
  __device__ __forceinline__ float w(int j, int l) const {
    if (W) return __ldg(W + static_cast<int64_t>(j) * K1 + l);
    return j == l ? 0.0f : ((j == base || l == base) ? c.w_cb : c.w_cc);
  }
  __device__ __forceinline__ float a(int j, int l) const {
    if (A) return __ldg(A + static_cast<int64_t>(j) * K1 + l);
    return j == l ? 0.0f : ((j == base || l == base) ? c.a_cb : c.a_cc);
  }
  __device__ __forceinline__ float e(int j, int k) const {
    if (E) return __ldg(E + static_cast<int64_t>(j) * K1 + k);
    if (j == k) return 0.0f;
    if (j == base) return c.e_bc;
    return k == base ? c.e_cb : c.e_cc;
  }
  // value of entry j from its A_j, W_j, E_j and the skeleton totals
  __device__ __forceinline__ float value(float f, float sqf, float Aj, float Wj, float Ej, float sumA, float sumW,
                                         float fn) const {
    const float mun = c.mu / fn;
    const float inner = __fmaf_rn(0.5f, __fmaf_rn(fn, Aj, -sumA), __fmaf_rn(fn, Wj, -sumW));
    const float d = __fmaf_rn(-mun, inner, __fmul_rn(__fmul_rn(mun, sqf), Ej));
    float v = __fmaf_rn(d, c.dt, f);
    if (v > 1.0f) v = 1.0f;
    if (v <= 0.0f) v = 0.0f;
    return v;
  }
};

// Square root of a field value for the band term: the hardware's approximate
// root (sqrt.approx.f32, a few ulp), the same instruction in every tier.
__device__ __forceinline__ float root(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ bool in_skeleton(float f, float g) { return f > 0.0f || (f == 0.0f && g > 0.0f); }

__device__ __forceinline__ void add_to_sums(VertexSums& s, bool is_base, float f, float g, float sqf) {
  if (is_base) {
    s.hasb = 1;
    s.Gb = g;
    s.Fb = f;
    s.sqFb = sqf;
  } else {
    s.sG += g;
    s.sF += f;
    s.r += sqf;
    ++s.nC;
  }
}


// Checked builds (-DLF_CHECKED) test every index the step kernel reads or
// writes through against its array; one outside raises ERR_BOUNDS in the
// job's status word and the access goes to element 0 instead, so the kernel
// never leaves its buffers and the host fails the step.  Other builds compile
// the checks away.
#ifdef LF_CHECKED
#define LF_CK(obj, x, hi) (obj).ck((x), (hi))
#else
#define LF_CK(obj, x, hi) (x)
#endif

// The closed neighbourhood of one vertex, read straight from global memory.
// Used by the slow path, which enumerates the layer union in increasing id
// order: next_layer() scans the sorted rows for the smallest id above `cur`,
// sums() accumulates G and F of one layer in the order of the row of L.
template <int DT>
struct Neighbourhood {
  using V = Val<DT>;
  using T = typename V::T;
  const int2* __restrict__ rows;
  const uint16_t* __restrict__ Fid;
  const T* __restrict__ Fval;
  const int2* __restrict__ Lcv;
  int p0, p1, q0, q1;
  float dsum;
#ifdef LF_CHECKED
  DevStatus* st;
  int n_v, L_nnz, entries;
  __device__ int ck(int x, int hi) const {
    if (static_cast<unsigned>(x) >= static_cast<unsigned>(hi)) {
      atomicOr(&st->err, ERR_BOUNDS);
      return 0;
    }
    return x;
  }
#endif

  __device__ int next_layer(int cur) const {
    int nx = 0x7fffffff;
    for (int p = p0; p < p1; ++p) {
      const int l = __ldg(Fid + LF_CK(*this, p, entries));
      if (l > cur) { nx = min(nx, l); break; }
    }
    for (int q = q0; q < q1; ++q) {
      const int2 rj = __ldg(rows + LF_CK(*this, __ldg(&Lcv[LF_CK(*this, q, L_nnz)].x), n_v));
      for (int p = rj.x; p < rj.x + rj.y; ++p) {
        const int l = __ldg(Fid + LF_CK(*this, p, entries));
        if (l > cur) { nx = min(nx, l); break; }
      }
    }
    return nx;
  }

  __device__ void sums(int lay, float& G, float& F) const {
    F = 0.0f;
    G = 0.0f;
    for (int p = p0; p < p1; ++p) {
      const int l = __ldg(Fid + LF_CK(*this, p, entries));
      if (l == lay) { F = V::load(Fval + LF_CK(*this, p, entries)); break; }
      if (l > lay) break;
    }
    for (int q = q0; q < q1; ++q) {
      const int2 cv = __ldg(Lcv + LF_CK(*this, q, L_nnz));
      const float lij = __int_as_float(cv.y);
      const int2 rj = __ldg(rows + LF_CK(*this, cv.x, n_v));
      for (int p = rj.x; p < rj.x + rj.y; ++p) {
        const int l = __ldg(Fid + LF_CK(*this, p, entries));
        if (l == lay) { G = __fadd_rn(G, __fmul_rn(lij, V::load(Fval + LF_CK(*this, p, entries)))); break; }
        if (l > lay) break;
      }
    }
    G = fmaf(-dsum, F, G);        // diagonal: L_ii = -sum_{j != i} L_ij
  }
};

// The general update of layer j on the storage-free tier: A_j, W_j and E_j
// summed over the skeleton of the neighbourhood in ascending layer order,
// the order of the other tiers.
template <int DT>
__device__ float slow_general_value(const Neighbourhood<DT>& nb, const GenCoef& gc, int j, float Fj, float sumA,
                                    float sumW, float fn, float* Aout = nullptr, float* Wout = nullptr) {
  float Aj = 0.0f, Wj = 0.0f, Ej = 0.0f, G, F;
  for (int l = nb.next_layer(-1); l != 0x7fffffff; l = nb.next_layer(l)) {
    nb.sums(l, G, F);
    if (!in_skeleton(F, G)) continue;
    Aj = __fmaf_rn(gc.a(j, l), G, Aj);
    Wj = __fmaf_rn(gc.w(j, l), F, Wj);
    Ej = __fmaf_rn(gc.e(j, l), root(F), Ej);
  }
  if (Aout) {
    *Aout = Aj;
    *Wout = Wj;
    return 0.0f;
  }
  return gc.value(Fj, root(Fj), Aj, Wj, Ej, sumA, sumW, fn);
}

// Register map of K slots: layer id (-1 = empty), G and F per slot.
template <int K>
struct SlotMapT {
  int id[K];
  float g[K];
  float f[K];
  int cnt;

  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int s = 0; s < K; ++s) { id[s] = -1; g[s] = 0.0f; f[s] = 0.0f; }
    cnt = 0;
  }
  // Adds x to the slot of layer l, opening a slot if needed.  False when full.
  __device__ __forceinline__ bool add(int l, float x) {
    bool found = false;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      if (s < cnt && !found && id[s] == l) { g[s] = __fadd_rn(g[s], x); found = true; }
    }
    if (found) return true;
    if (cnt >= K - 1) return false;    // one slot stays for the base layer
#pragma unroll
    for (int s = 0; s < K; ++s) {
      if (s == cnt) { id[s] = l; g[s] = x; }
    }
    ++cnt;
    return true;
  }
  __device__ __forceinline__ void cswap(int a, int b) {
    const bool sw = static_cast<unsigned>(id[a]) > static_cast<unsigned>(id[b]);   // -1 sorts last
    const int ia = id[a], ib = id[b];
    const float ga = g[a], gb = g[b], fa = f[a], fb = f[b];
    id[a] = sw ? ib : ia; id[b] = sw ? ia : ib;
    g[a] = sw ? gb : ga;  g[b] = sw ? ga : gb;
    f[a] = sw ? fb : fa;  f[b] = sw ? fa : fb;
  }
  // The first M slots in ascending id order (ids are distinct; empty slots,
  // -1, sort last).  A warp's lanes use at most M + 1 slots and the base
  // layer, the largest id, is each lane's last live slot, so ordering the
  // first min(M, K - 1) slots orders every live one: optimal networks for
  // two to five slots (one, three, five and nine exchanges), odd-even
  // transposition beyond.
  template <int M>
  __device__ __forceinline__ void sort_first() {
    if constexpr (M == 2) {
      cswap(0, 1);
    } else if constexpr (M == 3) {
      cswap(0, 1); cswap(1, 2); cswap(0, 1);
    } else if constexpr (M == 4) {
      cswap(0, 1); cswap(2, 3); cswap(0, 2); cswap(1, 3); cswap(1, 2);
    } else if constexpr (M == 5) {
      cswap(0, 1); cswap(3, 4); cswap(2, 4); cswap(2, 3); cswap(1, 4);
      cswap(0, 3); cswap(0, 2); cswap(1, 3); cswap(1, 2);
    } else if constexpr (M > 5) {
#pragma unroll
      for (int r = 0; r < M; ++r)
#pragma unroll
        for (int a = r & 1; a + 1 < M; a += 2) cswap(a, a + 1);
    }
  }
};
using SlotMap = SlotMapT<kSlots>;

// Runs fn with the number of register slots a warp's lanes use at most as a
// compile-time constant (1 to K), so that the per-slot loops after the gather
// unroll over the live slots only (n is warp-uniform).
template <int K, int M = 1, class Fn>
__device__ __forceinline__ void with_slots(int n, Fn&& fn) {
  if constexpr (M >= K) {
    fn(std::integral_constant<int, K>{});
  } else {
    if (n <= M) fn(std::integral_constant<int, M>{});
    else with_slots<K, M + 1>(n, fn);
  }
}

// As with_slots with three variants only (2, 4 or K slots): a lane does up
// to one slot more work, and the kernel's warps share less code (the
// register-tier kernel, which also holds the full step, lost issue slots to
// instruction fetch with six variants).
template <int K, class Fn>
__device__ __forceinline__ void with_slots_coarse(int n, Fn&& fn) {
  if (n <= 2) fn(std::integral_constant<int, 2>{});
  else if (n <= 4) fn(std::integral_constant<int, 4>{});
  else fn(std::integral_constant<int, K>{});
}

// Medium path: a map of kMed slots in shared memory, one of kPool per CTA,
// taken by the (rare) threads whose union outgrows the register map.
struct MedMap {
  int* id;
  float* g;
  float* f;
  int cnt;
  __device__ bool add(int l, float x, float fv) {
    for (int s = 0; s < cnt; ++s)
      if (id[s] == l) { g[s] = __fadd_rn(g[s], x); return true; }
    if (cnt == kMed) return false;
    id[cnt] = l;
    g[cnt] = x;
    f[cnt] = fv;
    ++cnt;
    return true;
  }
};


// The update over a register map of N live slots: the diagonal term of the own entries, ascending slot
// order, the skeleton test, the per-vertex sums, Algorithm 1's update (the
// class closed form or the general matrices), the clamp, the normalisation
// and the rounding to the storage type.
template <int DT, bool GEN, int N, int K>
__device__ __forceinline__ void slot_update(SlotMapT<K>& mp, const int own_cells, const int own, const float dsum,
                                            const int base, const Coefs& c, const GenCoef& gc, const bool general,
                                            VertexSums& S, float (&vnew)[K], bool (&keep)[K], int& kept,
                                            float& tot, bool& zero_sum) {
  using V = Val<DT>;
    // diagonal: the own entries (the own cells, then the base layer)
#pragma unroll
    for (int s = 0; s < N; ++s)
      if (s < own_cells || (s == mp.cnt - 1 && own_cells < own)) mp.g[s] = fmaf(-dsum, mp.f[s], mp.g[s]);
    // slots in ascending layer order (empty slots, id -1, last): the sums
    // below then run in the same order as on the other paths, and the row
    // is written in slot order
    mp.template sort_first<(N < K - 1 ? N : K - 1)>();
    float sq[N];
#pragma unroll
    for (int s = 0; s < N; ++s) sq[s] = root(mp.f[s]);
    bool ins[N];
#pragma unroll
    for (int s = 0; s < N; ++s) {
      ins[s] = s < mp.cnt && in_skeleton(mp.f[s], mp.g[s]);
      if (ins[s]) add_to_sums(S, mp.id[s] == base, mp.f[s], mp.g[s], sq[s]);
    }
    if (general) {
      const float fn = static_cast<float>(S.nC + S.hasb);
      float Aj[N], Wj[N], Ej[N];
      float sumA = 0.0f, sumW = 0.0f;
#pragma unroll
      for (int s = 0; s < N; ++s) {
        Aj[s] = Wj[s] = Ej[s] = 0.0f;
        if (ins[s]) {
#pragma unroll
          for (int l = 0; l < N; ++l) {
            if (ins[l]) {
              Aj[s] = __fmaf_rn(gc.a(mp.id[s], mp.id[l]), mp.g[l], Aj[s]);
              Wj[s] = __fmaf_rn(gc.w(mp.id[s], mp.id[l]), mp.f[l], Wj[s]);
              Ej[s] = __fmaf_rn(gc.e(mp.id[s], mp.id[l]), sq[l], Ej[s]);
            }
          }
          sumA = __fadd_rn(sumA, Aj[s]);
          sumW = __fadd_rn(sumW, Wj[s]);
        }
      }
#pragma unroll
      for (int s = 0; s < N; ++s) {
        if (ins[s]) {
          vnew[s] = gc.value(mp.f[s], sq[s], Aj[s], Wj[s], Ej[s], sumA, sumW, fn);
          tot += vnew[s];
        }
      }
    } else {
      const Update U(S, c);
#pragma unroll
      for (int s = 0; s < N; ++s) {
        if (ins[s]) {
          vnew[s] = U.value(mp.id[s] == base, mp.f[s], mp.g[s], sq[s], S, c);
          tot += vnew[s];
        }
      }
    }
    if (!(tot > 0.0f)) zero_sum = true;
    const float rtot = 1.0f / tot;           // normalisation: one division per vertex
#pragma unroll
    for (int s = 0; s < N; ++s) {
      if (ins[s]) {
        const float vs = V::widen(V::round(__fmul_rn(vnew[s], rtot)));
        if (vs != 0.0f) { keep[s] = true; vnew[s] = vs; ++kept; }
      }
    }
}

// Writes the kept entries of a register map of N slots in slot order.
template <int DT, int N, int K, class Put>
__device__ __forceinline__ void slot_write(const SlotMapT<K>& mp, const bool (&keep)[K], const float (&vnew)[K],
                                           int off, Put& put) {
  using V = Val<DT>;
  int o = off;
#pragma unroll
  for (int s = 0; s < N; ++s) {
    if (!keep[s]) continue;
    put(o, mp.id[s], V::round(vnew[s]));
    ++o;
  }
}

// G = sum_j L_ij F(j, .) over the register map, lean form: the neighbours in
// batches of kChunk0 (their L entries, then their head records, loaded before
// any is used), every entry through one compare over the cell slots, a cell
// new to the map opening the first empty slot (the map's cells fill its
// first slots, the rest hold -1), the base layer summed apart in gB.
// Each layer's sum runs in the row order of L, as on every other path.  The
// sum of the row's off-diagonal weights goes to nb.dsum.  False when a cell
// found no free slot (one stays for the base layer); the map is then
// incomplete and only nb.dsum is final.  mp.cnt: the cells in the map (all K
// slots counted).
template <int DT, int K>
__device__ __forceinline__ bool lean_gather(Neighbourhood<DT>& nb, const int4* __restrict__ head, const int base,
                                            SlotMapT<K>& mp, float& gB) {
  using V = Val<DT>;
  bool fit = true;
  // slots fill in order (empty ones hold -1): a cell new to the map opens the
  // first empty slot; every update is a select, no branch
  auto add = [&](int l, float x, bool live) {
    const bool isb = live && l == base;
    gB = isb ? __fadd_rn(gB, x) : gB;
    const int cell = (live && !isb) ? l : -2;
    bool m[K - 1];
    bool fresh = cell >= 0;
#pragma unroll
    for (int s2 = 0; s2 < K - 1; ++s2) {
      m[s2] = cell == mp.id[s2];
      fresh = fresh && !m[s2];
    }
    fit = fit && !(fresh && mp.id[K - 2] >= 0);
    bool o[K - 1];
#pragma unroll
    for (int s2 = 0; s2 < K - 1; ++s2) o[s2] = fresh && mp.id[s2] < 0 && (s2 == 0 || mp.id[s2 - 1] >= 0);
#pragma unroll
    for (int s2 = 0; s2 < K - 1; ++s2) {
      mp.g[s2] = o[s2] ? x : (m[s2] ? __fadd_rn(mp.g[s2], x) : mp.g[s2]);
      mp.id[s2] = o[s2] ? cell : mp.id[s2];
    }
  };
  for (int qb = nb.q0; qb < nb.q1; qb += kChunk0) {
    int2 cv[kChunk0];
#pragma unroll
    for (int k = 0; k < kChunk0; ++k) {
      cv[k] = make_int2(-1, 0);
      if (qb + k < nb.q1) cv[k] = __ldg(nb.Lcv + LF_CK(nb, qb + k, nb.L_nnz));
    }
    int4 hj[kChunk0];
#pragma unroll
    for (int k = 0; k < kChunk0; ++k) {
      hj[k] = make_int4(0, 0, 0, 0);
      if (cv[k].x >= 0) hj[k] = __ldg(head + LF_CK(nb, cv[k].x, nb.n_v));
    }
#pragma unroll
    for (int k = 0; k < kChunk0; ++k) {
      if (cv[k].x < 0) continue;
      const float lij = __int_as_float(cv[k].y);
      nb.dsum += lij;
      if (!fit) continue;
      const int rn = hj[k].x;
      const int e1 = (hj[k].y >> 16) & 0xffff;
      add(hj[k].y & 0xffff, __fmul_rn(lij, V::from_bits(hj[k].z)), rn >= 1);
      if (rn >= 2) {
        const float x1 = __fmul_rn(lij, V::from_bits(hj[k].w));
        if (e1 == base) gB = __fadd_rn(gB, x1);
        else add(e1, x1, true);                // a row of two cells
      }
      if (rn > 2) {                              // rows of three entries or more
        const int rs = __ldg(nb.rows + LF_CK(nb, cv[k].x, nb.n_v)).x;
        for (int p = 2; p < rn; ++p)
          add(__ldg(nb.Fid + LF_CK(nb, rs + p, nb.entries)),
              __fmul_rn(lij, V::load(nb.Fval + LF_CK(nb, rs + p, nb.entries))), true);
      }
    }
  }
  // every slot counts: an own row of K cells and no base entry fills the
  // last slot too, and the caller must see K (no room left for the base)
  int n = 0;
#pragma unroll
  for (int s2 = 0; s2 < K; ++s2) n += mp.id[s2] >= 0;
  mp.cnt = n;
  return fit;
}

// ---------------------------------------------------------------------------
// the step kernel
// ---------------------------------------------------------------------------
enum : int { kFast = 0, kMedium = 1, kSlow = 2 };

// One step of the tile of this CTA with every tier: the body of the step
// kernel, and of the register-tier kernel for a tile outside its shape.
template <int DT, bool GEN, bool LEAN>
__device__ __forceinline__ void step_tile(const BatchParams& P) {
  using V = Val<DT>;
  using T = typename V::T;
  constexpr int kWarps = kBlock / 32;
  constexpr int K = LEAN ? kHotCells + 1 : kSlots;   // register-map slots
  __shared__ uint32_t s_err;
  __shared__ int s_pool;
  __shared__ unsigned s_red[kWarps];
  __shared__ int s_warp_cnt[kWarps];
  __shared__ int s_med_id[kPool][kMed];
  __shared__ float s_med_g[kPool][kMed];
  __shared__ float s_med_f[kPool][kMed];

  // ---- the job of this CTA (uniform): last j with tile_start[j] <= blockIdx.x
  int lo = 0, hi = P.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.tile_start[mid] <= static_cast<int>(blockIdx.x)) lo = mid; else hi = mid - 1;
  }
  const JobDesc& J = P.job[lo];
  if (P.step >= J.steps) return;

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int warp = t >> 5;
  const int tile = static_cast<int>(blockIdx.x) - P.tile_start[lo];
  const int n_v = J.n_v;
  const int base = J.n_layers - 1;
  const int cap = J.tile_cap;
  const int par = (J.parity0 + P.step) & 1;
  const FieldBuf in = J.buf[par];
  const FieldBuf out = J.buf[par ^ 1];
  const Coefs& c = J.c;
  // general coefficient matrices: only in the GEN form, and only for a job
  // that has them (a class-coefficient job runs the class update there too)
  const bool general = GEN && (J.cW != nullptr || J.cA != nullptr || J.cE != nullptr);
  GenCoef gc;
  gc.W = J.cW;
  gc.A = J.cA;
  gc.E = J.cE;
  gc.K1 = J.n_layers;
  gc.base = J.n_layers - 1;
  gc.c = J.c;
  float gsumA = 0.0f, gsumW = 0.0f;        // skeleton totals of the general update (storage-free tier)
  DevStatus* st = J.st;

  Neighbourhood<DT> nb;
  nb.rows = in.rows;
  nb.Fid = in.ids;
  nb.Fval = static_cast<const T*>(in.vals);
  nb.Lcv = J.L_colval;
  nb.dsum = 0.0f;
  nb.p0 = nb.p1 = nb.q0 = nb.q1 = 0;
#ifdef LF_CHECKED
  nb.st = J.st;
  nb.n_v = J.n_v;
  nb.L_nnz = J.L_nnz;
  nb.entries = J.num_tiles * J.tile_cap;
#endif

  // the first loads do not depend on the error word: issue them before the
  // barrier that publishes it
  const int i = tile * kBlock + t;
  int4 h_own = make_int4(0, 0, 0, 0);    // head record of the own row
  if (i < n_v) {
    h_own = __ldg(in.head + i);
    nb.q0 = __ldg(J.L_rowptr + i);
    nb.q1 = __ldg(J.L_rowptr + i + 1);
  }
  // the own row's place in the segment, read only where its entries beyond
  // the head record are needed (rows of three or more, the other tiers)
  bool own_row_read = false;
  auto read_own_row = [&]() {
    if (!own_row_read && i < n_v) {
      const int2 ri = __ldg(nb.rows + i);
      nb.p0 = ri.x;
      nb.p1 = ri.x + ri.y;
    }
    own_row_read = true;
  };
  if (t == 0) {
    s_err = ld_relaxed_u32(&st->err);
    s_pool = 0;
  }
  __syncthreads();
  if (s_err) return;                 // an earlier step of this job failed

  SlotMapT<K> mp;
  mp.clear();
  int mode = kFast;
  bool zero_sum = false;
  int kept = 0, nsk = 0;
  const int own = h_own.x;
  float vnew[K];
  bool keep[K];
#pragma unroll
  for (int s = 0; s < K; ++s) { vnew[s] = 0.0f; keep[s] = false; }
  VertexSums S = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, 0};
  float tot = 0.0f;
  MedMap med;
  med.cnt = 0;
  med.id = nullptr;
  med.g = med.f = nullptr;

  // The base layer is kept apart from the cell slots: its G and F live in
  // gB / fB and it joins the slots (as the largest id) after the gather.  Most
  // rows hold it at round-off level, as their second entry.
  float gB = 0.0f, fB = 0.0f;
  int own_cells = own;              // own entries other than the base layer
  if (i < n_v) {
    if (own > K) {
      mode = kMedium;
    } else if (own <= 2) {
      if (own > 0) {
        mp.id[0] = h_own.y & 0xffff;
        mp.f[0] = V::from_bits(h_own.z);
      }
      if (own > 1) {
        mp.id[1] = (h_own.y >> 16) & 0xffff;
        mp.f[1] = V::from_bits(h_own.w);
      }
    } else {
      read_own_row();
#pragma unroll
      for (int s = 0; s < K; ++s) {
        if (s < own) {
          mp.id[s] = __ldg(nb.Fid + LF_CK(nb, nb.p0 + s, nb.entries));
          mp.f[s] = V::load(nb.Fval + LF_CK(nb, nb.p0 + s, nb.entries));
        }
      }
    }
    if (mode == kFast && own > 0) {
      // ids ascend within a row and the base layer is the largest id, so an
      // own base entry is the last one
      int last = -1;
      float flast = 0.0f;
#pragma unroll
      for (int s = 0; s < K; ++s) {
        last = (s == own - 1) ? mp.id[s] : last;
        flast = (s == own - 1) ? mp.f[s] : flast;
      }
      if (last == base) {
        fB = flast;
        own_cells = own - 1;
#pragma unroll
        for (int s = 0; s < K; ++s)
          if (s == own - 1) { mp.id[s] = -1; mp.f[s] = 0.0f; }
      }
    }
    mp.cnt = own_cells;
    if constexpr (LEAN) {
      // ---- G = sum_j L_ij F(j, .), lean form; a vertex whose cells outgrow
      // the map takes the medium path (the weights' sum is complete either way)
      if (!lean_gather(nb, in.head, base, mp, gB)) mode = kMedium;
    } else {
      // ---- G = sum_j L_ij F(j, .): neighbours in batches of kChunk; the head
      // records of the batch's rows are loaded before any is used
      for (int qb = nb.q0; qb < nb.q1; qb += kChunk) {
        int jj[kChunk], rn[kChunk];
        float lij[kChunk];
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
          jj[k] = -1;
          lij[k] = 0.0f;
          if (qb + k < nb.q1) {
            const int2 cv = __ldg(nb.Lcv + LF_CK(nb, qb + k, nb.L_nnz));
            jj[k] = cv.x;
            lij[k] = __int_as_float(cv.y);
          }
        }
        int4 hj[kChunk];
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
          hj[k] = make_int4(0, 0, 0, 0);
          if (jj[k] >= 0) {
            hj[k] = __ldg(in.head + LF_CK(nb, jj[k], nb.n_v));
            nb.dsum += lij[k];
          }
          rn[k] = hj[k].x;
        }
        if (mode != kFast) continue;
        // the first two entries of each row of the batch; -2 marks "no entry"
        int e0[kChunk], e1[kChunk];
        float x0[kChunk], x1[kChunk];
        bool simple = true;           // every row: at most a cell, then the base layer
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
          e0[k] = e1[k] = -2;
          x0[k] = x1[k] = 0.0f;
          if (rn[k] > 0) {
            e0[k] = hj[k].y & 0xffff;
            x0[k] = __fmul_rn(lij[k], V::from_bits(hj[k].z));
          }
          if (rn[k] > 1) {
            e1[k] = (hj[k].y >> 16) & 0xffff;
            x1[k] = __fmul_rn(lij[k], V::from_bits(hj[k].w));
          }
          simple = simple && rn[k] <= 2 && (rn[k] < 2 || e1[k] == base);
        }
        if (simple) {
          // base contributions, one per row at most, in row order
#pragma unroll
          for (int k = 0; k < kChunk; ++k) {
            gB = (e0[k] == base) ? __fadd_rn(gB, x0[k]) : gB;
            gB = (e1[k] == base) ? __fadd_rn(gB, x1[k]) : gB;
            if (e0[k] == base) e0[k] = -2;
          }
          // cell entries (first entries only): slot x entry compare matrix, each
          // slot summing its entries in row order (empty slots hold -1)
          bool hit[kChunk];
#pragma unroll
          for (int k = 0; k < kChunk; ++k) hit[k] = e0[k] < 0;
          // over the cell slots that the lanes here have opened at most (the
          // slots beyond are empty in every lane)
          auto matrix = [&](auto cells) {
#pragma unroll
            for (int s2 = 0; s2 < decltype(cells)::value; ++s2) {
#pragma unroll
              for (int k = 0; k < kChunk; ++k) {
                const bool m = e0[k] == mp.id[s2];
                mp.g[s2] = m ? __fadd_rn(mp.g[s2], x0[k]) : mp.g[s2];
                hit[k] = hit[k] || m;
              }
            }
          };
          const int open_cells = __reduce_max_sync(__activemask(), mp.cnt);
          if (open_cells <= 1) matrix(std::integral_constant<int, 1>{});
          else if (open_cells == 2) matrix(std::integral_constant<int, 2>{});
          else matrix(std::integral_constant<int, K - 1>{});
          // cells new to the map, in row order: a missed entry opens the next
          // slot (no existing slot can match it: the matrix above compared them
          // all); when both entries of the batch miss with the same layer, one
          // slot opens with their sum taken in row order
          static_assert(kChunk == 2, "the miss handling below is written for batches of two");
          const bool m0 = !hit[0], m1 = !hit[1];
          if (m0 || m1) {
            const bool same = m0 && m1 && e0[0] == e0[1];
            const int la = m0 ? e0[0] : e0[1];
            const float xa = m0 ? (same ? __fadd_rn(x0[0], x0[1]) : x0[0]) : x0[1];
            const bool second = m0 && m1 && !same;
            if (mp.cnt + (second ? 1 : 0) >= K - 1) {
              mode = kMedium;                    // one slot stays for the base layer
            } else {
#pragma unroll
              for (int s2 = 0; s2 < K - 1; ++s2) {
                if (s2 == mp.cnt) { mp.id[s2] = la; mp.g[s2] = xa; }
                if (second && s2 == mp.cnt + 1) { mp.id[s2] = e0[1]; mp.g[s2] = x0[1]; }
              }
              mp.cnt += second ? 2 : 1;
            }
          }
        } else {
          // rows with two cells or more than two entries (transients, band
          // vertices): every entry in row order, strictly sequential
#pragma unroll
          for (int k = 0; k < kChunk; ++k) {
            if (rn[k] <= 0 || mode != kFast) continue;
            const int start = rn[k] > 2 ? __ldg(nb.rows + LF_CK(nb, jj[k], nb.n_v)).x : 0;
            for (int p = 0; p < rn[k] && mode == kFast; ++p) {
              int l;
              float x;
              if (p == 0) { l = e0[k]; x = x0[k]; }
              else if (p == 1) { l = e1[k]; x = x1[k]; }
              else {
                l = __ldg(nb.Fid + LF_CK(nb, start + p, nb.entries));
                x = __fmul_rn(lij[k], V::load(nb.Fval + LF_CK(nb, start + p, nb.entries)));
              }
              if (l == base) gB = __fadd_rn(gB, x);
              else if (!mp.add(l, x)) mode = kMedium;
            }
          }
        }
      }
    }
    // the base layer joins the slots last (largest id); with six cells
    // already there the vertex takes the next tier
    if (mode == kFast) {
      if (mp.cnt >= K) {
        mode = kMedium;
      } else {
#pragma unroll
        for (int s2 = 0; s2 < K; ++s2) {
          if (s2 == mp.cnt) { mp.id[s2] = base; mp.g[s2] = gB; mp.f[s2] = fB; }
        }
        ++mp.cnt;
      }
    }
  }

  // ---- medium path: a shared-memory map for unions beyond the register map
  if (mode != kFast) read_own_row();
  if (mode == kMedium) {
    const int slot = atomicAdd(&s_pool, 1);
    mode = kSlow;
    if (slot < kPool && own <= kMed) {
      med.id = s_med_id[slot];
      med.g = s_med_g[slot];
      med.f = s_med_f[slot];
      bool ok = true;
      for (int p = nb.p0; p < nb.p1; ++p)
        ok = ok && med.add(__ldg(nb.Fid + LF_CK(nb, p, nb.entries)), 0.0f, V::load(nb.Fval + LF_CK(nb, p, nb.entries)));
      for (int q = nb.q0; q < nb.q1 && ok; ++q) {
        const int2 cv = __ldg(nb.Lcv + LF_CK(nb, q, nb.L_nnz));
        const float lij = __int_as_float(cv.y);
        const int2 rj = __ldg(nb.rows + LF_CK(nb, cv.x, nb.n_v));
        for (int p = rj.x; p < rj.x + rj.y && ok; ++p)
          ok = med.add(__ldg(nb.Fid + LF_CK(nb, p, nb.entries)),
                       __fmul_rn(lij, V::load(nb.Fval + LF_CK(nb, p, nb.entries))), 0.0f);
      }
      if (ok) {
        mode = kMedium;
        for (int s = 0; s < own; ++s) med.g[s] = fmaf(-nb.dsum, med.f[s], med.g[s]);
        // ascending layer order (insertion sort), so that every per-vertex sum
        // below runs in the same order as on the other paths
        for (int s = 1; s < med.cnt; ++s) {
          const int li = med.id[s];
          const float gi = med.g[s], fi = med.f[s];
          int u = s - 1;
          for (; u >= 0 && med.id[u] > li; --u) {
            med.id[u + 1] = med.id[u];
            med.g[u + 1] = med.g[u];
            med.f[u + 1] = med.f[u];
          }
          med.id[u + 1] = li;
          med.g[u + 1] = gi;
          med.f[u + 1] = fi;
        }
      }
    }
  }

  if (i < n_v) {
    if (mode == kFast) {
      // ---- fast path: diagonal, skeleton, update over the register map ------
      // over the slots that the lanes here use at most (every lane's own
      // count is within it, whichever lanes run this together)
      // (the general form keeps all slots: its matrix sums are the cost there)
      with_slots<K>(GEN ? K : __reduce_max_sync(__activemask(), mp.cnt), [&](auto slots) {
        slot_update<DT, GEN, decltype(slots)::value>(mp, own_cells, own, nb.dsum, base, c, gc, general, S, vnew, keep,
                                                     kept, tot, zero_sum);
      });
    } else if (mode == kMedium) {
      // ---- medium path: the same update over the shared-memory map ----------
      for (int s = 0; s < med.cnt; ++s)
        if (in_skeleton(med.f[s], med.g[s])) add_to_sums(S, med.id[s] == base, med.f[s], med.g[s], root(med.f[s]));
      if (general) {
        const float fn = static_cast<float>(S.nC + S.hasb);
        float sumA = 0.0f, sumW = 0.0f;
        float vt[kMed];
        for (int pass = 0; pass < 2; ++pass) {
          for (int s = 0; s < med.cnt; ++s) {
            if (!in_skeleton(med.f[s], med.g[s])) continue;
            float Aj = 0.0f, Wj = 0.0f, Ej = 0.0f;
            for (int l = 0; l < med.cnt; ++l) {
              if (!in_skeleton(med.f[l], med.g[l])) continue;
              Aj = __fmaf_rn(gc.a(med.id[s], med.id[l]), med.g[l], Aj);
              Wj = __fmaf_rn(gc.w(med.id[s], med.id[l]), med.f[l], Wj);
              Ej = __fmaf_rn(gc.e(med.id[s], med.id[l]), root(med.f[l]), Ej);
            }
            if (pass == 0) {
              sumA = __fadd_rn(sumA, Aj);
              sumW = __fadd_rn(sumW, Wj);
            } else {
              vt[s] = gc.value(med.f[s], root(med.f[s]), Aj, Wj, Ej, sumA, sumW, fn);
            }
          }
        }
        for (int s = 0; s < med.cnt; ++s) {
          if (in_skeleton(med.f[s], med.g[s])) {
            med.g[s] = vt[s];
            tot += med.g[s];
          } else {
            med.f[s] = -1.0f;                    // not in the skeleton
          }
        }
      } else {
        const Update U(S, c);
        for (int s = 0; s < med.cnt; ++s) {
          if (in_skeleton(med.f[s], med.g[s])) {
            med.g[s] = U.value(med.id[s] == base, med.f[s], med.g[s], root(med.f[s]), S, c);
            tot += med.g[s];
          } else {
            med.f[s] = -1.0f;                    // not in the skeleton
          }
        }
      }
      if (!(tot > 0.0f)) zero_sum = true;
      const float rtot = 1.0f / tot;
      for (int s = 0; s < med.cnt; ++s) {
        if (med.f[s] < 0.0f) continue;
        const float vs = V::widen(V::round(__fmul_rn(med.g[s], rtot)));
        if (vs != 0.0f) { med.g[s] = vs; ++kept; }
        else med.f[s] = -1.0f;
      }
    } else {
      // ---- slow path: the union in increasing id order, three passes -------
      float G, F;
      for (int l = nb.next_layer(-1); l != 0x7fffffff; l = nb.next_layer(l)) {
        nb.sums(l, G, F);
        if (in_skeleton(F, G)) add_to_sums(S, l == base, F, G, root(F));
      }
      const Update U(S, c);
      const float fn = static_cast<float>(S.nC + S.hasb);
      if (general) {
        for (int l = nb.next_layer(-1); l != 0x7fffffff; l = nb.next_layer(l)) {
          nb.sums(l, G, F);
          if (!in_skeleton(F, G)) continue;
          float Aj, Wj;
          slow_general_value(nb, gc, l, F, 0.0f, 0.0f, fn, &Aj, &Wj);
          gsumA = __fadd_rn(gsumA, Aj);
          gsumW = __fadd_rn(gsumW, Wj);
        }
      }
      auto value = [&](int l, float F, float G) {
        return general ? slow_general_value(nb, gc, l, F, gsumA, gsumW, fn) : U.value(l == base, F, G, root(F), S, c);
      };
      for (int l = nb.next_layer(-1); l != 0x7fffffff; l = nb.next_layer(l)) {
        nb.sums(l, G, F);
        if (in_skeleton(F, G)) tot += value(l, F, G);
      }
      if (!(tot > 0.0f)) zero_sum = true;
      for (int l = nb.next_layer(-1); l != 0x7fffffff; l = nb.next_layer(l)) {
        nb.sums(l, G, F);
        if (in_skeleton(F, G) && V::widen(V::round(__fmul_rn(value(l, F, G), 1.0f / tot))) != 0.0f) ++kept;
      }
    }
    nsk = S.nC + S.hasb;
    if (zero_sum) kept = 0;
  }

  // ---- block scan of the output row lengths: offsets inside the segment ----
  int x = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  // the skeleton sizes are reduced per warp alongside, so one barrier serves both
  const unsigned sk = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(nsk));
  if (lane == 31) {
    s_warp_cnt[warp] = x;
    s_red[warp] = sk;
  }
  const bool bad_sum = __syncthreads_or(zero_sum);
  int warp_off = 0, tile_total = 0;
  unsigned tile_sk = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) warp_off += s_warp_cnt[w];
    tile_total += s_warp_cnt[w];
    tile_sk += s_red[w];
  }
  const int local_excl = warp_off + x - kept;

  bool write = !bad_sum;
  if (t == 0 && bad_sum) atomicOr(&st->err, ERR_ZERO_SUM);
  if (write && tile_total > cap) {
    write = false;
    if (t == 0) {
      atomicOr(&st->err, ERR_CAPACITY);
      atomicMax(&st->need_tile, static_cast<unsigned long long>(tile_total));
    }
  }

  // ---- write row i of the output, entries sorted by layer id ---------------
  if (write && i < n_v) {
    const int off = tile * cap + local_excl;
    out.rows[i] = make_int2(off, kept);
    T* ov = static_cast<T*>(out.vals);
    // head record: the count and the first two entries written
    int4 ho = make_int4(kept, 0, 0, 0);
    auto put = [&](int o, int l, T vt) {
#ifdef LF_CHECKED
      const int w = tile * cap + nb.ck(o - tile * cap, cap);   // inside the tile's segment
#else
      const int w = o;
#endif
      out.ids[w] = static_cast<uint16_t>(l);
      ov[w] = vt;
      if (o == off) { ho.y = l; ho.z = V::bits(vt); }
      else if (o == off + 1) { ho.y |= l << 16; ho.w = V::bits(vt); }
    };
    if (mode == kFast) {
      int top = 1;                             // slots up to the last kept one
#pragma unroll
      for (int s = 0; s < K; ++s) top = keep[s] ? s + 1 : top;
      with_slots<K>(GEN ? K : __reduce_max_sync(__activemask(), top), [&](auto slots) {
        slot_write<DT, decltype(slots)::value>(mp, keep, vnew, off, put);
      });
    } else if (mode == kMedium) {
      int o = off;
      for (int s = 0; s < med.cnt; ++s) {
        if (med.f[s] < 0.0f) continue;
        put(o, med.id[s], V::round(med.g[s]));
        ++o;
      }
    } else {
      const Update U(S, c);
      const float fn = static_cast<float>(S.nC + S.hasb);
      float G, F;
      int o = off;
      for (int l = nb.next_layer(-1); l != 0x7fffffff; l = nb.next_layer(l)) {
        nb.sums(l, G, F);
        if (!in_skeleton(F, G)) continue;
        const float v = general ? slow_general_value(nb, gc, l, F, gsumA, gsumW, fn) : U.value(l == base, F, G, root(F), S, c);
        const T vt = V::round(__fmul_rn(v, 1.0f / tot));
        if (V::widen(vt) != 0.0f) {
          put(o, l, vt);
          ++o;
        }
      }
    }
    out.head[i] = ho;
  }

  // ---- end of step: the last CTA of the job commits the step ----------------
  if (t == 0) {
    atomicAdd(&st->skeleton_step, static_cast<unsigned long long>(tile_sk));
    atomicAdd(&st->nnz_step, static_cast<unsigned long long>(tile_total));
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done, 1u);
    if (prev == static_cast<uint32_t>(J.num_tiles) - 1u) {
      __threadfence();
      if (ld_relaxed_u32(&st->err) == 0u) {
        const unsigned long long nin = ld_relaxed(&st->nnz);
        const unsigned long long nout = ld_relaxed(&st->nnz_step);
        st->skeleton_total = ld_relaxed(&st->skeleton_total) + ld_relaxed(&st->skeleton_step);
        st->nnz_io_total = ld_relaxed(&st->nnz_io_total) + nin + nout;
        st->nnz = nout;
        st->epoch = st->epoch + 1u;
      }
      st->skeleton_step = 0ull;
      st->nnz_step = 0ull;
      st->done = 0u;
      __threadfence();
    }
  }
}

// MINB: CTAs per SM the register allocation is made for (the schedule).
// LEAN: the fast tier's gather in its lean form (schedule kSchedLean).
template <int DT, bool GEN, int MINB, bool LEAN = false>
__global__ void __launch_bounds__(kBlock, MINB) step_kernel_impl(const __grid_constant__ BatchParams P) {
  wait_previous_grid();
  allow_next_grid();
  step_tile<DT, GEN, LEAN>(P);
}

// ---------------------------------------------------------------------------
// the register-tier kernel (schedule kSchedHot)
// ---------------------------------------------------------------------------
// The same time-iteration as step_kernel_impl for the tiles whose every vertex
// holds at most kHotCells cells and the base layer itself and sees at most
// kHotCells cells in its closed neighbourhood: the register-map tier alone.  A cell's
// sum opens on the first entry of that cell and every later entry of it adds
// to it, in the order of the row of L, so every layer's sum -- and so the
// result -- is that of the other tiers, bit for bit.  A tile with a vertex
// outside the shape writes nothing here and takes the full step (every tier)
// instead, in the same CTA.  The lean path has fewer instructions a vertex
// and more neighbours' loads in flight; it pays wherever the shape holds on
// nearly every tile, which is the steady state once the cells have formed.
template <int DT>
__global__ void __launch_bounds__(kBlock, 4) step_kernel_hot(const __grid_constant__ BatchParams P) {
  using V = Val<DT>;
  using T = typename V::T;
  constexpr int kWarps = kBlock / 32;
  constexpr int K = kHotCells + 1;                // slots: the cells', then the base layer's
  __shared__ uint32_t s_err;
  __shared__ unsigned s_red[kWarps];
  __shared__ int s_warp_cnt[kWarps];

  wait_previous_grid();
  allow_next_grid();

  int lo = 0, hi = P.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.tile_start[mid] <= static_cast<int>(blockIdx.x)) lo = mid; else hi = mid - 1;
  }
  const JobDesc& J = P.job[lo];
  if (P.step >= J.steps) return;

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int warp = t >> 5;
  const int tile = static_cast<int>(blockIdx.x) - P.tile_start[lo];
  const int n_v = J.n_v;
  const int base = J.n_layers - 1;
  const int cap = J.tile_cap;
  const int par = (J.parity0 + P.step) & 1;
  const FieldBuf in = J.buf[par];
  const FieldBuf out = J.buf[par ^ 1];
  const Coefs& c = J.c;
  DevStatus* st = J.st;

  Neighbourhood<DT> nb;
  nb.rows = in.rows;
  nb.Fid = in.ids;
  nb.Fval = static_cast<const T*>(in.vals);
  nb.Lcv = J.L_colval;
  nb.dsum = 0.0f;
  nb.p0 = nb.p1 = nb.q0 = nb.q1 = 0;
#ifdef LF_CHECKED
  nb.st = J.st;
  nb.n_v = J.n_v;
  nb.L_nnz = J.L_nnz;
  nb.entries = J.num_tiles * J.tile_cap;
#endif

  const int i = tile * kBlock + t;
  int4 h_own = make_int4(0, 0, 0, 0);
  if (i < n_v) {
    h_own = __ldg(in.head + i);
    nb.q0 = __ldg(J.L_rowptr + i);
    nb.q1 = __ldg(J.L_rowptr + i + 1);
  }
  if (t == 0) s_err = ld_relaxed_u32(&st->err);
  __syncthreads();
  if (s_err) return;                 // an earlier step of this job failed

  const int own = h_own.x;
  SlotMapT<K> mp;
  mp.clear();
  int own_cells = 0;
  bool ok = true;
  if (i < n_v) {
    float gb = 0.0f, fb = 0.0f;
    // the own row: the head record's two entries, the rest from the segment;
    // its cells take the first slots (ids ascend, the base layer is last)
    ok = own <= K;
    int start = 0;
    if (ok && own > 2) start = __ldg(nb.rows + i).x;
#pragma unroll
    for (int p = 0; p < K; ++p) {
      if (!ok || p >= own) continue;
      int l;
      float f;
      if (p == 0) { l = h_own.y & 0xffff; f = V::from_bits(h_own.z); }
      else if (p == 1) { l = (h_own.y >> 16) & 0xffff; f = V::from_bits(h_own.w); }
      else { l = __ldg(nb.Fid + LF_CK(nb, start + p, nb.entries)); f = V::load(nb.Fval + LF_CK(nb, start + p, nb.entries)); }
      if (l == base) {
        fb = f;
      } else {
#pragma unroll
        for (int s2 = 0; s2 < K - 1; ++s2)
          if (s2 == own_cells) { mp.id[s2] = l; mp.f[s2] = f; }
        ++own_cells;
      }
    }
    ok = ok && own_cells <= K - 1;
    ok = lean_gather(nb, in.head, base, mp, gb) && ok;
    // the base layer joins the slots last (largest id)
#pragma unroll
    for (int s2 = 0; s2 < K; ++s2) {
      if (s2 == mp.cnt) { mp.id[s2] = base; mp.g[s2] = gb; mp.f[s2] = fb; }
    }
    mp.cnt += 1;
  }
  // a tile with a vertex outside the shape takes the full step
  if (!__syncthreads_and(ok)) {
    step_tile<DT, false, false>(P);
    return;
  }

  bool zero_sum = false;
  int kept = 0, nsk = 0;
  float vnew[K];
  bool keep[K];
#pragma unroll
  for (int s2 = 0; s2 < K; ++s2) { vnew[s2] = 0.0f; keep[s2] = false; }
  VertexSums S = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, 0};
  float tot = 0.0f;
  const GenCoef gc{};                // unused: class coefficients only
  if (i < n_v) {
    with_slots_coarse<K>(__reduce_max_sync(__activemask(), mp.cnt), [&](auto slots) {
      slot_update<DT, false, decltype(slots)::value>(mp, own_cells, own, nb.dsum, base, c, gc, false, S, vnew, keep,
                                                     kept, tot, zero_sum);
    });
    nsk = S.nC + S.hasb;
    if (zero_sum) kept = 0;
  }

  // ---- block scan of the output row lengths: offsets inside the segment ----
  int x = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  const unsigned sk = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(nsk));
  if (lane == 31) {
    s_warp_cnt[warp] = x;
    s_red[warp] = sk;
  }
  const bool bad_sum = __syncthreads_or(zero_sum);
  int warp_off = 0, tile_total = 0;
  unsigned tile_sk = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) warp_off += s_warp_cnt[w];
    tile_total += s_warp_cnt[w];
    tile_sk += s_red[w];
  }
  const int local_excl = warp_off + x - kept;

  bool write = !bad_sum;
  if (t == 0 && bad_sum) atomicOr(&st->err, ERR_ZERO_SUM);
  if (write && tile_total > cap) {
    write = false;
    if (t == 0) {
      atomicOr(&st->err, ERR_CAPACITY);
      atomicMax(&st->need_tile, static_cast<unsigned long long>(tile_total));
    }
  }

  // ---- write row i of the output, entries sorted by layer id ---------------
  if (write && i < n_v) {
    const int off = tile * cap + local_excl;
    out.rows[i] = make_int2(off, kept);
    T* ov = static_cast<T*>(out.vals);
    int4 ho = make_int4(kept, 0, 0, 0);
    auto put = [&](int o, int l, T vt) {
#ifdef LF_CHECKED
      const int w = tile * cap + nb.ck(o - tile * cap, cap);   // inside the tile's segment
#else
      const int w = o;
#endif
      out.ids[w] = static_cast<uint16_t>(l);
      ov[w] = vt;
      if (o == off) { ho.y = l; ho.z = V::bits(vt); }
      else if (o == off + 1) { ho.y |= l << 16; ho.w = V::bits(vt); }
    };
    int top = 1;
#pragma unroll
    for (int s2 = 0; s2 < K; ++s2) top = keep[s2] ? s2 + 1 : top;
    with_slots_coarse<K>(__reduce_max_sync(__activemask(), top), [&](auto slots) {
      slot_write<DT, decltype(slots)::value>(mp, keep, vnew, off, put);
    });
    out.head[i] = ho;
  }

  // ---- end of step: the last CTA of the job commits the step ----------------
  if (t == 0) {
    atomicAdd(&st->skeleton_step, static_cast<unsigned long long>(tile_sk));
    atomicAdd(&st->nnz_step, static_cast<unsigned long long>(tile_total));
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done, 1u);
    if (prev == static_cast<uint32_t>(J.num_tiles) - 1u) {
      __threadfence();
      if (ld_relaxed_u32(&st->err) == 0u) {
        const unsigned long long nin = ld_relaxed(&st->nnz);
        const unsigned long long nout = ld_relaxed(&st->nnz_step);
        st->skeleton_total = ld_relaxed(&st->skeleton_total) + ld_relaxed(&st->skeleton_step);
        st->nnz_io_total = ld_relaxed(&st->nnz_io_total) + nin + nout;
        st->nnz = nout;
        st->epoch = st->epoch + 1u;
      }
      st->skeleton_step = 0ull;
      st->nnz_step = 0ull;
      st->done = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// seeding, labels, relayout, conversions
// ---------------------------------------------------------------------------
template <int DT>
__global__ void seed_fill_kernel(const __grid_constant__ JobDesc job, int base) {
  using V = Val<DT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= job.n_v) return;
  const FieldBuf b = job.buf[0];
  const int tile = i / kTile;
  const int off = tile * job.tile_cap + (i - tile * kTile);
  b.rows[i] = make_int2(off, 1);
  b.ids[off] = static_cast<uint16_t>(base);
  static_cast<typename V::T*>(b.vals)[off] = V::round(1.0f);
}

__global__ void seed_scatter_kernel(const __grid_constant__ JobDesc job, int k, const int32_t* __restrict__ seeds) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= k) return;
  const int v = seeds[s];
  const int tile = v / kTile;
  job.buf[0].ids[tile * job.tile_cap + (v - tile * kTile)] = static_cast<uint16_t>(s);
}

// Region seeds (Sec. 3.2, "Initialization"): the seed vertex and its
// immediate neighbours take the seed's layer.  A vertex claimed by several
// seeds goes to its own seed if it is one, else to the lowest seed id:
// key = (neighbour ? 2^20 : 0) | seed, smallest key wins.
__global__ void region_claim_kernel(const __grid_constant__ JobDesc job, int k, const int32_t* __restrict__ seeds,
                                    unsigned* __restrict__ owner) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= k) return;
  const int v = seeds[s];
  atomicMin(&owner[v], static_cast<unsigned>(s));
  for (int q = job.L_rowptr[v]; q < job.L_rowptr[v + 1]; ++q)
    atomicMin(&owner[job.L_colval[q].x], (1u << 20) | static_cast<unsigned>(s));
}

__global__ void region_scatter_kernel(const __grid_constant__ JobDesc job, const unsigned* __restrict__ owner) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= job.n_v) return;
  const unsigned o = owner[i];
  if (o == ~0u) return;
  const int tile = i / kTile;
  job.buf[0].ids[tile * job.tile_cap + (i - tile * kTile)] = static_cast<uint16_t>(o & 0xfffffu);
}

template <int DT>
__global__ void labels_kernel(const __grid_constant__ JobDesc job, int buf, int32_t* __restrict__ labels,
                              float* __restrict__ maxval) {
  using V = Val<DT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= job.n_v) return;
  const FieldBuf b = job.buf[buf];
  const int base = job.n_layers - 1;
  const int2 r = b.rows[i];
  int best = -1;
  float bv = -1.0f;
  const typename V::T* vals = static_cast<const typename V::T*>(b.vals);
  for (int p = r.x; p < r.x + r.y; ++p) {   // ids ascending: strict > keeps the lowest id on a tie
    const float v = V::widen(vals[p]);
    if (v > bv) { bv = v; best = b.ids[p]; }
  }
  labels[i] = (best == base) ? -1 : best;
  if (maxval) maxval[i] = bv;
}

template <int DT>
__global__ void relayout_kernel(const int2* __restrict__ rows_from, const uint16_t* __restrict__ ids_from,
                                const void* __restrict__ vals_from, int cap_from, int2* __restrict__ rows_to,
                                uint16_t* __restrict__ ids_to, void* __restrict__ vals_to, int cap_to, int n_v) {
  using T = typename Val<DT>::T;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const int tile = i / kTile;
  const int2 r = rows_from[i];
  const int start = r.x - tile * cap_from + tile * cap_to;
  rows_to[i] = make_int2(start, r.y);
  for (int p = 0; p < r.y; ++p) {
    ids_to[start + p] = ids_from[r.x + p];
    static_cast<T*>(vals_to)[start + p] = static_cast<const T*>(vals_from)[r.x + p];
  }
}

template <int DT>
__global__ void build_head_kernel(const FieldBuf b, int n_v) {
  using V = Val<DT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const int2 r = b.rows[i];
  const typename V::T* vals = static_cast<const typename V::T*>(b.vals);
  int4 h = make_int4(r.y, 0, 0, 0);
  if (r.y > 0) {
    h.y = b.ids[r.x];
    h.z = V::bits(vals[r.x]);
  }
  if (r.y > 1) {
    h.y |= static_cast<int>(b.ids[r.x + 1]) << 16;
    h.w = V::bits(vals[r.x + 1]);
  }
  b.head[i] = h;
}

template <int DT>
__global__ void widen_kernel(const void* __restrict__ src, float* __restrict__ dst, int64_t n) {
  using V = Val<DT>;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = V::widen(static_cast<const typename V::T*>(src)[i]);
}

template <int DT>
__global__ void narrow_kernel(const float* __restrict__ src, void* __restrict__ dst, int64_t n) {
  using V = Val<DT>;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) static_cast<typename V::T*>(dst)[i] = V::round(src[i]);
}

using StepFn = void (*)(const BatchParams);
// [schedule][storage type]: the class-coefficient kernel at 4, 5 and 3 CTAs
// per SM, the register-tier kernel, and the kernel with the lean gather; the
// general-coefficient form keeps 4.
const StepFn kClassFns[kSchedules][3] = {
    {&step_kernel_impl<0, false, 4>, &step_kernel_impl<1, false, 4>, &step_kernel_impl<2, false, 4>},
    {&step_kernel_impl<0, false, 5>, &step_kernel_impl<1, false, 5>, &step_kernel_impl<2, false, 5>},
    {&step_kernel_impl<0, false, 3>, &step_kernel_impl<1, false, 3>, &step_kernel_impl<2, false, 3>},
    {&step_kernel_hot<0>, &step_kernel_hot<1>, &step_kernel_hot<2>},
    {&step_kernel_impl<0, false, 4, true>, &step_kernel_impl<1, false, 4, true>, &step_kernel_impl<2, false, 4, true>}};
const StepFn kGeneralFns[3] = {&step_kernel_impl<0, true, 4>, &step_kernel_impl<1, true, 4>,
                               &step_kernel_impl<2, true, 4>};

}  // namespace

int step_slots() { return kSlots; }

// The kernel of a launch kind; a launch with coefficient matrices takes the
// general-coefficient form.
static StepFn step_fn(int kind, bool general) {
  const int dtype = kind % 3;
  const int sched = kind / 3;
  return general ? kGeneralFns[dtype] : kClassFns[sched][dtype];
}

const void* step_kernel(int kind, bool general) { return reinterpret_cast<const void*>(step_fn(kind, general)); }

bool needs_general(const BatchParams& p) {
  for (int j = 0; j < p.n_jobs; ++j)
    if (p.job[j].cW || p.job[j].cA || p.job[j].cE) return true;
  return false;
}

cudaError_t launch_step(const BatchParams& p, int kind, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(p.tile_start[p.n_jobs]));
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_fn(kind, needs_general(p)), p);
}

#define LF_DISPATCH(dtype, KERNEL, GRID, BLOCK, STREAM, ...)                       \
  switch (dtype) {                                                                \
    case 0: KERNEL<0><<<(GRID), (BLOCK), 0, (STREAM)>>>(__VA_ARGS__); break;        \
    case 1: KERNEL<1><<<(GRID), (BLOCK), 0, (STREAM)>>>(__VA_ARGS__); break;        \
    default: KERNEL<2><<<(GRID), (BLOCK), 0, (STREAM)>>>(__VA_ARGS__); break;       \
  }

cudaError_t launch_seed(const JobDesc& job, int k, const int32_t* d_seeds, int dtype, cudaStream_t s) {
  const int blocks = (job.n_v + 255) / 256;
  LF_DISPATCH(dtype, seed_fill_kernel, blocks, 256, s, job, k);
  seed_scatter_kernel<<<(k + 255) / 256, 256, 0, s>>>(job, k, d_seeds);
  LF_DISPATCH(dtype, build_head_kernel, blocks, 256, s, job.buf[0], job.n_v);
  return cudaGetLastError();
}

cudaError_t launch_seed_regions(const JobDesc& job, int k, const int32_t* d_seeds, unsigned* d_owner, int dtype,
                                cudaStream_t s) {
  const int blocks = (job.n_v + 255) / 256;
  cudaError_t e = cudaMemsetAsync(d_owner, 0xff, sizeof(unsigned) * static_cast<size_t>(job.n_v), s);
  if (e != cudaSuccess) return e;
  LF_DISPATCH(dtype, seed_fill_kernel, blocks, 256, s, job, k);
  region_claim_kernel<<<(k + 255) / 256, 256, 0, s>>>(job, k, d_seeds, d_owner);
  region_scatter_kernel<<<blocks, 256, 0, s>>>(job, d_owner);
  LF_DISPATCH(dtype, build_head_kernel, blocks, 256, s, job.buf[0], job.n_v);
  return cudaGetLastError();
}

cudaError_t launch_build_head(const FieldBuf& b, int n_v, int dtype, cudaStream_t s) {
  const int blocks = (n_v + 255) / 256;
  LF_DISPATCH(dtype, build_head_kernel, blocks, 256, s, b, n_v);
  return cudaGetLastError();
}

cudaError_t launch_labels(const JobDesc& job, int buf, int dtype, int32_t* d_labels, float* d_maxval,
                          cudaStream_t s) {
  const int blocks = (job.n_v + 255) / 256;
  LF_DISPATCH(dtype, labels_kernel, blocks, 256, s, job, buf, d_labels, d_maxval);
  return cudaGetLastError();
}

cudaError_t launch_relayout(const int2* rows_from, const uint16_t* ids_from, const void* vals_from,
                            int cap_from, int2* rows_to, uint16_t* ids_to, void* vals_to, int cap_to,
                            int n_v, int dtype, cudaStream_t s) {
  const int blocks = (n_v + 255) / 256;
  LF_DISPATCH(dtype, relayout_kernel, blocks, 256, s, rows_from, ids_from, vals_from, cap_from, rows_to,
              ids_to, vals_to, cap_to, n_v);
  return cudaGetLastError();
}

cudaError_t launch_widen(const void* src, float* dst, int64_t n, int dtype, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  LF_DISPATCH(dtype, widen_kernel, blocks, 256, s, src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_narrow(const float* src, void* dst, int64_t n, int dtype, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  LF_DISPATCH(dtype, narrow_kernel, blocks, 256, s, src, dst, n);
  return cudaGetLastError();
}

}  // namespace lf
