// Level barrier and L2 cache-policy helpers of the level sweeps.
//
// The sweeps of Alg. 1 run as one cooperative launch (all blocks resident)
// that walks the depth levels in order.  After writing its share of level l a
// block adds one to count[l] with release semantics; before gathering level
// l+1 it waits until count[l] equals the number of blocks.  Rows of the next
// level do not depend on the field, so blocks load them before the wait.
// Every wait is bounded: after max_spin polls the block sets ERRBIT_TIMEOUT
// and leaves; a block that sees the bit leaves as well, so the launch ends
// and the host reads GRAPHGP_ERR_TIMEOUT from graphgp_sync_status.
#pragma once

#include "common.cuh"

namespace ggp {

__device__ __forceinline__ uint32_t sync_ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct LevelBarrier {
  uint32_t* count;  // [num_levels] arrivals per level
  uint32_t* err;
  int64_t max_spin;

  // Call after __syncthreads(): the block's stores of level l are complete.
  __device__ __forceinline__ void arrive(int l) const {
    if (threadIdx.x == 0)
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count + l) : "memory");
  }

  // Whole block: wait until every block arrived at level l.  Returns nonzero
  // (uniformly) when the block must leave.
  __device__ __forceinline__ int wait(int l, uint32_t nblocks, int* s_flag) const {
    if (threadIdx.x == 0) {
      int abort = 0;
      int64_t spins = 0;
      while (sync_ld_acquire(count + l) < nblocks) {
        if ((++spins & 63) == 0 && (sync_ld_acquire(err) & ERRBIT_TIMEOUT)) {
          abort = 1;
          break;
        }
        if (spins > max_spin) {
          atomicOr(err, ERRBIT_TIMEOUT);
          abort = 1;
          break;
        }
        __nanosleep(32);
      }
      *s_flag = abort;
    }
    __syncthreads();
    return *s_flag;
  }
};

// L2 eviction policies.  Streamed rows are read once; the field vector is
// gathered again by later levels.  GGP_ROW_POLICY / GGP_V_POLICY select the
// priority: 0 evict_normal, 1 evict_first, 2 evict_last.
#ifndef GGP_ROW_POLICY
#define GGP_ROW_POLICY 1
#endif
#ifndef GGP_V_POLICY
#define GGP_V_POLICY 2
#endif

template <int P>
__device__ __forceinline__ uint64_t l2_policy() {
  uint64_t p;
  if (P == 1)
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  else if (P == 2)
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t l2_evict_first() { return l2_policy<GGP_ROW_POLICY>(); }
__device__ __forceinline__ uint64_t l2_evict_last() { return l2_policy<GGP_V_POLICY>(); }

__device__ __forceinline__ int4 ld_stream_i4(const int4* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ float4 ld_stream_f4(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ float ld_stream_f(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(v)
               : "l"(p), "l"(pol));
  return v;
}

// Streamed loads that do not allocate in L1.
__device__ __forceinline__ int4 ld_stream_na_i4(const int4* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ float4 ld_stream_na_f4(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ float ld_stream_na_f(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(v)
               : "l"(p), "l"(pol));
  return v;
}

// read-only input vector, kept in L2
__device__ __forceinline__ float ld_keep_f(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

// field values of earlier levels inside a level sweep: cached in L1.  They
// were written before the level barrier, whose gpu-scope acquire makes them
// visible, and nothing read during a level is written during that level.
__device__ __forceinline__ float ld_level_f(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(v)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}

// vector written by other blocks during the launch: read at L2 (coherent)
__device__ __forceinline__ float ld_coherent_f(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(v)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}

__device__ __forceinline__ void st_keep_f(float* p, float v, uint64_t pol) {
  asm volatile("st.global.cg.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol)
               : "memory");
}

__device__ __forceinline__ void st_stream_f(float* p, float v, uint64_t pol) {
  asm volatile("st.global.cs.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol)
               : "memory");
}

// Threads sharing one position in the sweeps: row slices of a multiple of 4
// entries (KP = padded row length).
__host__ __device__ constexpr int gen_lanes(int kp) { return kp % 16 == 0 ? 4 : (kp % 8 == 0 ? 2 : 1); }

// sum_a b_a v[c_a] of one row whose weights are in registers, in the stored
// sweeps' summation order: the row cut into gen_lanes(K) slices, two
// alternating accumulators per slice, slices combined as the sweeps'
// xor-shuffle tree does.  LEVEL: v is being written level by level in the
// same launch (read through ld_level_f).
template <int K, bool LEVEL>
__device__ __forceinline__ float dot_stored_order(const float (&b)[K], const int32_t* row,
                                                  const float* v, uint64_t pol) {
  constexpr int LANES = gen_lanes(K), HP = K / LANES;
  float part[LANES];
#pragma unroll
  for (int h = 0; h < LANES; h++) {
    float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
    for (int q = 0; q < HP / 4; q++) {
      const int e = h * HP + 4 * q;
      const int4 c = __ldg(reinterpret_cast<const int4*>(row + e));
      float v0, v1, v2, v3;
      if (LEVEL) {
        v0 = ld_level_f(v + c.x, pol); v1 = ld_level_f(v + c.y, pol);
        v2 = ld_level_f(v + c.z, pol); v3 = ld_level_f(v + c.w, pol);
      } else {
        v0 = ld_keep_f(v + c.x, pol); v1 = ld_keep_f(v + c.y, pol);
        v2 = ld_keep_f(v + c.z, pol); v3 = ld_keep_f(v + c.w, pol);
      }
      acc0 = fmaf(b[e], v0, acc0);
      acc1 = fmaf(b[e + 1], v1, acc1);
      acc0 = fmaf(b[e + 2], v2, acc0);
      acc1 = fmaf(b[e + 3], v3, acc1);
    }
    part[h] = acc0 + acc1;
  }
  if (LANES == 4) return (part[0] + part[2]) + (part[1] + part[3]);
  if (LANES == 2) return part[0] + part[1];
  return part[0];
}

// The same sum for the one-warp-per-point form: lane a holds b_a (b_own);
// lane h of the warp forms slice h from the shuffled weights and the row's
// neighbour indices (padding entries included).  Valid on lane 0.
template <int KP, bool LEVEL>
__device__ __forceinline__ float warp_dot_stored_order(float b_own, const int32_t* row,
                                                       const float* v, uint64_t pol) {
  constexpr int LANES = gen_lanes(KP), HP = KP / LANES;
  const int h = (threadIdx.x & 31) % LANES;
  float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
  for (int q = 0; q < HP / 4; q++) {
    const int e = h * HP + 4 * q;
    const int4 c = __ldg(reinterpret_cast<const int4*>(row + e));
    const float w0 = __shfl_sync(0xffffffffu, b_own, (e + 0) & 31);
    const float w1 = __shfl_sync(0xffffffffu, b_own, (e + 1) & 31);
    const float w2 = __shfl_sync(0xffffffffu, b_own, (e + 2) & 31);
    const float w3 = __shfl_sync(0xffffffffu, b_own, (e + 3) & 31);
    float v0, v1, v2, v3;
    if (LEVEL) {
      v0 = ld_level_f(v + c.x, pol); v1 = ld_level_f(v + c.y, pol);
      v2 = ld_level_f(v + c.z, pol); v3 = ld_level_f(v + c.w, pol);
    } else {
      v0 = ld_keep_f(v + c.x, pol); v1 = ld_keep_f(v + c.y, pol);
      v2 = ld_keep_f(v + c.z, pol); v3 = ld_keep_f(v + c.w, pol);
    }
    acc0 = fmaf(w0, v0, acc0);
    acc1 = fmaf(w1, v1, acc1);
    acc0 = fmaf(w2, v2, acc0);
    acc1 = fmaf(w3, v3, acc1);
  }
  float acc = acc0 + acc1;
  if (LANES >= 4) acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (LANES >= 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  return acc;
}

// Largest grid of kernel `fn` (block threads, dyn smem) that is co-resident.
template <class F>
inline int coop_grid(F fn, int threads, size_t smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms();
}

// coop_grid remembered per device in `cache` (one slot per device index).
template <class F>
inline int coop_grid_cached(int (&cache)[kMaxDevices], F fn, int threads, size_t smem = 0) {
  const int d = current_device();
  if (!cache[d]) cache[d] = coop_grid(fn, threads, smem);
  return cache[d];
}

}  // namespace ggp
