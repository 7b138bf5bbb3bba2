// Layered-field step on sm_103a: one fused kernel per time-iteration.
//
// One thread owns one vertex i.  It gathers the closed neighbourhood of i
// from L (CSR, off-diagonal only) and the field F (CSR, layer ids sorted),
// accumulating G = L F (the paper's L_t = Phi L^T, Algorithm 1) per layer in
// a small per-thread map in shared memory; applies the interest-skeleton
// test, the explicit Euler update of Eq. 11-13 in closed form, the clamp and
// the normalisation (Sec. 4); and writes the surviving entries of row i into
// the output CSR.  Row offsets come from a single-pass scan with decoupled
// look-back (Merrill and Garland, 2016) over tiles of one CTA each, so the
// whole iteration is one launch with no host round trip.
//
// Every wait in this file is bounded by the global timer; a wait that runs
// out raises ERR_TIMEOUT, poisons its tile and lets the kernel finish.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lf_internal.h"

namespace lf {

const StepTier kTiers[kNumTiers] = {{16, 256}, {48, 128}, {160, 32}};

namespace {

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------
template <int DT> struct Val;
template <> struct Val<0> {
  using T = float;
  static __device__ __forceinline__ float load(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ T round(float v) { return v; }
  static __device__ __forceinline__ float widen(T v) { return v; }
};
template <> struct Val<1> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float load(const T* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ T round(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float widen(T v) { return __bfloat162float(v); }
};
template <> struct Val<2> {
  using T = __half;
  static __device__ __forceinline__ float load(const T* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ T round(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float widen(T v) { return __half2float(v); }
};

// ---------------------------------------------------------------------------
// device-scope relaxed atomics and the global timer
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Look-back status word: value in bits 0-31, flag in bits 32-33, tag in 34-63.
constexpr unsigned long long kFlagAgg = 1ull, kFlagPrefix = 2ull, kFlagPoison = 3ull;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long pack_status(uint32_t tag, unsigned long long flag, uint32_t v) {
  return (static_cast<unsigned long long>(tag) << 34) | (flag << 32) | v;
}

// ---------------------------------------------------------------------------
// the step kernel
// ---------------------------------------------------------------------------
template <int DT, int M, int B>
__global__ void __launch_bounds__(B) step_kernel_impl(const JobDesc* __restrict__ job) {
  using V = Val<DT>;
  using T = typename V::T;
  constexpr int kWarps = B / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  float* s_g = reinterpret_cast<float*>(smem);                 // [M][B] G, then new value
  float* s_f = s_g + M * B;                                    // [M][B] F before the step
  uint16_t* s_id = reinterpret_cast<uint16_t*>(s_f + M * B);   // [M][B] layer ids
  __shared__ uint32_t s_tile, s_epoch, s_abort, s_prefix, s_fail;
  __shared__ int s_warp_cnt[kWarps];
  __shared__ int s_warp_sk[kWarps];

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int warp = t >> 5;
  DevStatus* st = job->st;

  if (t == 0) {
    const uint32_t e = ld_relaxed_u32(&st->err);
    s_abort = e;
    if (e == 0u) {
      s_tile = atomicAdd(&st->ticket, 1u);
      s_epoch = ld_relaxed_u32(&st->epoch);
    }
  }
  __syncthreads();
  if (s_abort) return;

  const uint32_t tile = s_tile;
  const uint32_t epoch = s_epoch;
  const int n_v = job->n_v;
  const int base = job->n_layers - 1;
  const FieldBuf in = job->buf[epoch & 1u];
  const FieldBuf out = job->buf[(epoch & 1u) ^ 1u];
  const int32_t* __restrict__ Frp = in.rowptr;
  const uint16_t* __restrict__ Fid = in.ids;
  const T* __restrict__ Fval = static_cast<const T*>(in.vals);
  const Coefs c = job->c;

  const int i = static_cast<int>(tile) * B + t;
  int cnt = 0;      // distinct layers seen in the closed neighbourhood
  int kept = 0;     // entries of the output row
  int nsk = 0;      // |interest skeleton| of the row
  bool map_ovf = false, zero_sum = false;

  if (i < n_v) {
    // ---- own row: F(i, .) -------------------------------------------------
    const int p0 = __ldg(Frp + i), p1 = __ldg(Frp + i + 1);
    for (int p = p0; p < p1; ++p) {
      if (cnt == M) { map_ovf = true; break; }
      s_id[cnt * B + t] = __ldg(Fid + p);
      s_f[cnt * B + t] = V::load(Fval + p);
      s_g[cnt * B + t] = 0.0f;
      ++cnt;
    }
    const int own = cnt;
    // ---- G = sum_j L_ij F(j, .) over the off-diagonal entries of row i ----
    float dsum = 0.0f;
    const int q0 = __ldg(job->L_rowptr + i), q1 = __ldg(job->L_rowptr + i + 1);
    for (int q = q0; q < q1 && !map_ovf; ++q) {
      const int2 cv = __ldg(job->L_colval + q);
      const int j = cv.x;
      const float lij = __int_as_float(cv.y);
      dsum += lij;
      const int r0 = __ldg(Frp + j), r1 = __ldg(Frp + j + 1);
      for (int p = r0; p < r1; ++p) {
        const uint16_t l = __ldg(Fid + p);
        const float x = lij * V::load(Fval + p);
        int s = 0;
        while (s < cnt && s_id[s * B + t] != l) ++s;
        if (s < cnt) {
          s_g[s * B + t] += x;
        } else if (cnt < M) {
          s_id[cnt * B + t] = l;
          s_g[cnt * B + t] = x;
          s_f[cnt * B + t] = 0.0f;
          ++cnt;
        } else {
          map_ovf = true;
          break;
        }
      }
    }
    // diagonal: L_ii = -sum_{j != i} L_ij
    for (int s = 0; s < own; ++s) s_g[s * B + t] = fmaf(-dsum, s_f[s * B + t], s_g[s * B + t]);

    if (!map_ovf) {
      // ---- interest skeleton and per-vertex sums (class coefficients) -----
      float sG = 0.0f, sF = 0.0f, r = 0.0f, Gb = 0.0f, Fb = 0.0f;
      int nC = 0, hasb = 0;
      for (int s = 0; s < cnt; ++s) {
        const float f = s_f[s * B + t], g = s_g[s * B + t];
        const bool in_sk = (f > 0.0f) || (f == 0.0f && g > 0.0f);
        if (!in_sk) { s_f[s * B + t] = -1.0f; continue; }   // marks "not in skeleton"
        if (s_id[s * B + t] == base) { hasb = 1; Gb = g; Fb = f; }
        else { sG += g; sF += f; r += sqrtf(f); ++nC; }
      }
      const int n = nC + hasb;
      nsk = n;
      const float fn = static_cast<float>(n);
      const float fnc = static_cast<float>(nC);
      const float sumA = c.a_cc * (fnc - 1.0f) * sG + (hasb ? c.a_cb * (fnc * Gb + sG) : 0.0f);
      const float sumW = c.w_cc * (fnc - 1.0f) * sF + (hasb ? c.w_cb * (fnc * Fb + sF) : 0.0f);
      const float mun = c.mu / fn;
      const float sqFb = sqrtf(Fb);
      float tot = 0.0f;
      for (int s = 0; s < cnt; ++s) {
        const float f = s_f[s * B + t];
        if (f < 0.0f) continue;
        const float g = s_g[s * B + t];
        float A, W, R;
        if (s_id[s * B + t] == base) {
          A = c.a_cb * sG;
          W = c.w_cb * sF;
          R = c.e_bc * r;
        } else {
          A = c.a_cc * (sG - g) + (hasb ? c.a_cb * Gb : 0.0f);
          W = c.w_cc * (sF - f) + (hasb ? c.w_cb * Fb : 0.0f);
          R = c.e_cc * (r - sqrtf(f)) + (hasb ? c.e_cb * sqFb : 0.0f);
        }
        const float d = -mun * (0.5f * (fn * A - sumA) + (fn * W - sumW)) + mun * sqrtf(f) * R;
        float v = f + d * c.dt;
        if (v > 1.0f) v = 1.0f;
        if (v <= 0.0f) v = 0.0f;
        s_g[s * B + t] = v;
        tot += v;
      }
      if (!(tot > 0.0f)) zero_sum = true;
      // ---- normalise, round to the storage type, drop zeros ----------------
      for (int s = 0; s < cnt; ++s) {
        if (s_f[s * B + t] < 0.0f) continue;
        const float vs = V::widen(V::round(s_g[s * B + t] / tot));
        if (vs != 0.0f) { s_g[s * B + t] = vs; ++kept; }
        else s_f[s * B + t] = -1.0f;
      }
      if (zero_sum) kept = 0;
    }
  }

  // ---- tile scan of the output row lengths ---------------------------------
  int x = map_ovf ? 0 : kept;
  int sk = nsk;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
    sk += __shfl_xor_sync(0xffffffffu, sk, o);
  }
  if (lane == 31) s_warp_cnt[warp] = x;
  if (lane == 0) s_warp_sk[warp] = sk;
  const bool bad_map = __syncthreads_or(map_ovf);
  const bool bad_sum = __syncthreads_or(zero_sum);
  int warp_off = 0, tile_total = 0, tile_sk = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) warp_off += s_warp_cnt[w];
    tile_total += s_warp_cnt[w];
    tile_sk += s_warp_sk[w];
  }
  const int local_excl = warp_off + x - (map_ovf ? 0 : kept);

  // ---- decoupled look-back: exclusive prefix of this tile ------------------
  if (warp == 0) {
    unsigned long long* ts = job->tile_status;
    const uint32_t tag = (epoch + 1u) & 0x3fffffffu;
    uint32_t excl = 0;
    bool fail = false;
    if (tile == 0) {
      if (lane == 0) st_relaxed(ts, pack_status(tag, kFlagPrefix, static_cast<uint32_t>(tile_total)));
    } else {
      if (lane == 0) st_relaxed(ts + tile, pack_status(tag, kFlagAgg, static_cast<uint32_t>(tile_total)));
      int pred = static_cast<int>(tile) - 1 - lane;
      const unsigned long long t0 = global_ns();
      while (true) {
        unsigned long long w = 0ull, flag = kFlagPrefix;
        uint32_t val = 0u;
        bool timed_out = false;
        if (pred >= 0) {
          unsigned int ns = 32;
          while (true) {
            w = ld_relaxed(ts + pred);
            flag = (w >> 32) & 3ull;
            if ((w >> 34) == tag && flag != 0ull) break;
            if (global_ns() - t0 > kWaitLimitNs) { timed_out = true; break; }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
          }
          val = static_cast<uint32_t>(w);
        }
        const bool poisoned = timed_out || flag == kFlagPoison;
        if (__any_sync(0xffffffffu, poisoned)) { fail = true; break; }
        const unsigned pm = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
        const int first = __ffs(pm) - 1;                 // closest tile with a full prefix
        uint32_t contrib = (pm == 0u || lane <= first) ? val : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        excl += contrib;
        if (pm != 0u) break;
        pred -= 32;
      }
      if (lane == 0) {
        if (fail) {
          st_relaxed(ts + tile, pack_status(tag, kFlagPoison, 0u));
          atomicOr(&st->err, ERR_TIMEOUT);
        } else {
          st_relaxed(ts + tile, pack_status(tag, kFlagPrefix, excl + static_cast<uint32_t>(tile_total)));
        }
      }
    }
    if (lane == 0) {
      s_prefix = excl;
      s_fail = fail ? 1u : 0u;
    }
  }
  __syncthreads();

  const unsigned long long row0 = s_prefix;
  const unsigned long long tile_end = row0 + static_cast<unsigned long long>(tile_total);
  bool write = !s_fail && !bad_map && !bad_sum;
  if (t == 0) {
    if (bad_map) { atomicOr(&st->err, ERR_MAP); atomicMax(&st->need_map, 1u); }
    if (bad_sum) atomicOr(&st->err, ERR_ZERO_SUM);
  }
  if (write && tile_end > static_cast<unsigned long long>(job->cap)) {
    write = false;
    if (t == 0) {
      atomicOr(&st->err, ERR_CAPACITY);
      atomicMax(&st->need_nnz, tile_end);
    }
  }

  // ---- write row i of the output, entries sorted by layer id ---------------
  if (write && i < n_v) {
    const int off = static_cast<int>(row0) + local_excl;
    out.rowptr[i] = off;
    if (i == n_v - 1) out.rowptr[n_v] = off + kept;
    T* ov = static_cast<T*>(out.vals);
    for (int s = 0; s < cnt; ++s) {
      if (s_f[s * B + t] < 0.0f) continue;
      const uint16_t l = s_id[s * B + t];
      int rank = 0;
      for (int u = 0; u < cnt; ++u)
        rank += (s_f[u * B + t] >= 0.0f && s_id[u * B + t] < l) ? 1 : 0;
      out.ids[off + rank] = l;
      ov[off + rank] = V::round(s_g[s * B + t]);
    }
  }

  // ---- end of step: the last CTA commits the step ---------------------------
  __syncthreads();
  if (t == 0) {
    atomicAdd(&st->skeleton_step, static_cast<unsigned long long>(tile_sk));
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done, 1u);
    if (prev == gridDim.x - 1u) {
      __threadfence();
      if (ld_relaxed_u32(&st->err) == 0u) {
        const unsigned long long nin = static_cast<unsigned long long>(__ldcg(Frp + n_v));
        const unsigned long long nout = static_cast<unsigned long long>(__ldcg(out.rowptr + n_v));
        st->skeleton_total = ld_relaxed(&st->skeleton_total) + ld_relaxed(&st->skeleton_step);
        st->nnz_io_total = ld_relaxed(&st->nnz_io_total) + nin + nout;
        st->epoch = epoch + 1u;
      }
      st->skeleton_step = 0ull;
      st->ticket = 0u;
      st->done = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// seeding, labels, conversions
// ---------------------------------------------------------------------------
template <int DT>
__global__ void seed_fill_kernel(const JobDesc* __restrict__ job, int n_v, int base) {
  using V = Val<DT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const FieldBuf b = job->buf[0];
  if (i < n_v) {
    b.rowptr[i] = i;
    b.ids[i] = static_cast<uint16_t>(base);
    static_cast<typename V::T*>(b.vals)[i] = V::round(1.0f);
  }
  if (i == 0) b.rowptr[n_v] = n_v;
}

__global__ void seed_scatter_kernel(const JobDesc* __restrict__ job, int k, const int32_t* __restrict__ seeds) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < k) job->buf[0].ids[seeds[s]] = static_cast<uint16_t>(s);
}

template <int DT>
__global__ void labels_kernel(const JobDesc* __restrict__ job, int n_v, int32_t* __restrict__ labels,
                              float* __restrict__ maxval) {
  using V = Val<DT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const uint32_t epoch = job->st->epoch;
  const FieldBuf b = job->buf[epoch & 1u];
  const int base = job->n_layers - 1;
  const int p0 = b.rowptr[i], p1 = b.rowptr[i + 1];
  int best = -1;
  float bv = -1.0f;
  const typename V::T* vals = static_cast<const typename V::T*>(b.vals);
  for (int p = p0; p < p1; ++p) {     // ids ascending: strict > keeps the lowest id on a tie
    const float v = V::widen(vals[p]);
    if (v > bv) { bv = v; best = b.ids[p]; }
  }
  labels[i] = (best == base) ? -1 : best;
  if (maxval) maxval[i] = bv;
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

template <int DT, int TIER>
constexpr auto step_fn() {
  return &step_kernel_impl<DT, (TIER == 0 ? 16 : TIER == 1 ? 48 : 160), (TIER == 0 ? 256 : TIER == 1 ? 128 : 32)>;
}

using StepFn = void (*)(const JobDesc*);
const StepFn kStepFns[3][kNumTiers] = {
    {step_fn<0, 0>(), step_fn<0, 1>(), step_fn<0, 2>()},
    {step_fn<1, 0>(), step_fn<1, 1>(), step_fn<1, 2>()},
    {step_fn<2, 0>(), step_fn<2, 1>(), step_fn<2, 2>()},
};

size_t tier_smem(int tier) {
  const StepTier& s = kTiers[tier];
  return static_cast<size_t>(s.map_slots) * s.block * (4 + 4 + 2);
}

}  // namespace

const void* step_kernel(int dtype, int tier, size_t* smem_bytes) {
  if (smem_bytes) *smem_bytes = tier_smem(tier);
  return reinterpret_cast<const void*>(kStepFns[dtype][tier]);
}

cudaError_t init_kernels() {
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < kNumTiers; ++t) {
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kStepFns[d][t]),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(tier_smem(t)));
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

cudaError_t launch_step(const JobDesc* d_job, int num_tiles, int dtype, int tier, cudaStream_t s) {
  const size_t smem = tier_smem(tier);
  kStepFns[dtype][tier]<<<num_tiles, kTiers[tier].block, smem, s>>>(d_job);
  return cudaGetLastError();
}

cudaError_t launch_seed(const JobDesc* d_job, int n_v, int k, const int32_t* d_seeds, int dtype,
                        cudaStream_t s) {
  const int blocks = (n_v + 255) / 256;
  const int base = k;
  switch (dtype) {
    case 0: seed_fill_kernel<0><<<blocks, 256, 0, s>>>(d_job, n_v, base); break;
    case 1: seed_fill_kernel<1><<<blocks, 256, 0, s>>>(d_job, n_v, base); break;
    default: seed_fill_kernel<2><<<blocks, 256, 0, s>>>(d_job, n_v, base); break;
  }
  seed_scatter_kernel<<<(k + 255) / 256, 256, 0, s>>>(d_job, k, d_seeds);
  return cudaGetLastError();
}

cudaError_t launch_labels(const JobDesc* d_job, int n_v, int dtype, int32_t* d_labels, float* d_maxval,
                          cudaStream_t s) {
  const int blocks = (n_v + 255) / 256;
  switch (dtype) {
    case 0: labels_kernel<0><<<blocks, 256, 0, s>>>(d_job, n_v, d_labels, d_maxval); break;
    case 1: labels_kernel<1><<<blocks, 256, 0, s>>>(d_job, n_v, d_labels, d_maxval); break;
    default: labels_kernel<2><<<blocks, 256, 0, s>>>(d_job, n_v, d_labels, d_maxval); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_widen(const void* src, float* dst, int64_t n, int dtype, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  switch (dtype) {
    case 0: widen_kernel<0><<<blocks, 256, 0, s>>>(src, dst, n); break;
    case 1: widen_kernel<1><<<blocks, 256, 0, s>>>(src, dst, n); break;
    default: widen_kernel<2><<<blocks, 256, 0, s>>>(src, dst, n); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_narrow(const float* src, void* dst, int64_t n, int dtype, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  switch (dtype) {
    case 0: narrow_kernel<0><<<blocks, 256, 0, s>>>(src, dst, n); break;
    case 1: narrow_kernel<1><<<blocks, 256, 0, s>>>(src, dst, n); break;
    default: narrow_kernel<2><<<blocks, 256, 0, s>>>(src, dst, n); break;
  }
  return cudaGetLastError();
}

}  // namespace lf
