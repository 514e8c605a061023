// evd_common.cuh — device helpers shared by the cluster EVD kernels:
// distributed-shared-memory stores and remote mbarrier arrivals, time-bounded
// waits, Newton-refined reciprocal square root / reciprocal, the learned rule's
// dense layer and the thresholding rules in double precision (one warp).
#pragma once
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "../../include/lcf.h"

namespace lcf {

constexpr unsigned long long EP_WAIT_NS = 2000000000ull;   // bound on every mbarrier wait (2 s)

// ---- cluster primitives ----
__device__ __forceinline__ uint32_t ep_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t ep_mapa(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void ep_st_remote_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void ep_arrive_remote(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster_addr) : "memory");
}
// asynchronous 16-byte store into the partner's shared memory; completes 16 bytes of
// the transaction count of the partner's mbarrier (no fence on the issuing thread)
__device__ __forceinline__ void ep_st_async(uint32_t addr, float4 v, uint32_t bar_cluster_addr) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar_cluster_addr)
               : "memory");
}
__device__ __forceinline__ void ep_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ep_smem(b)), "r"(bytes) : "memory");
}
// 1/sqrt(x) and 1/x: hardware approximation plus one Newton-Raphson step
__device__ __forceinline__ float ep_rsqrt(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ float ep_rcp(float x) {
  const float r = __fdividef(1.f, x);
  return fmaf(r, fmaf(-x, r, 1.f), r);
}
__device__ __forceinline__ void ep_bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ep_smem(b)), "r"(count));
}
// Wait with acquire at cluster scope (the arrivals come from the partner CTA),
// for at most EP_WAIT_NS of wall time; false if the limit ran out.
__device__ __forceinline__ bool ep_try(uint64_t* b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred q;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 q, [%1], %2;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(done)
      : "r"(ep_smem(b)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t ep_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool ep_wait(uint64_t* b, uint32_t parity) {
  if (ep_try(b, parity)) return true;
  const uint64_t t0 = ep_now();
  for (;;) {
    if (ep_try(b, parity)) return true;
    if (ep_now() - t0 > EP_WAIT_NS) return false;
  }
}

// ---- learned cutoff rule: one dense layer on all warps of the CTA ----
// out[o] = act(b[o] + sum_k W[o][k] x[k]), W bf16 row-major (K per row), FP32 accumulation
__device__ inline void ep_dense(const float* x, int K, const __nv_bfloat16* __restrict__ W,
                                const float* __restrict__ b, float* out, int N, bool relu, int warp, int lane,
                                int nwarps) {
  for (int o = warp; o < N; o += nwarps) {
    const __nv_bfloat16* w = W + (size_t)o * K;
    float s = 0.f;
    for (int k = lane; k < K; k += 32) s = fmaf(__bfloat162float(w[k]), x[k], s);
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(~0u, s, off);
    if (lane == 0) {
      s += b[o];
      out[o] = relu ? fmaxf(s, 0.f) : s;
    }
  }
}

// ---- warp-parallel thresholding rules (double precision, warp 0) ----
// Same arithmetic per element as the one-thread rule; reductions by shuffles.
__device__ __forceinline__ double ep_floor(const double* lam, int n, int i) {
  const double fl = lam[0] * n * 2.220446049250313e-16;
  return lam[i] > fl ? lam[i] : fl;
}
__device__ inline void ep_norm_log(const double* lam, int n, double beta, int literal, double* y, int lane) {
  for (int i = lane; i < n; i += 32) y[i] = log10(ep_floor(lam, n, i));
  __syncwarp();
  const double y1 = y[0], yn = y[n - 1], span = y1 - yn;
  double v[4];
  int c = 0;
  for (int i = lane; i < n; i += 32, ++c) {
    if (literal) v[c] = (y1 != 0.0) ? beta * y[i] / y1 * n : 0.0;
    else v[c] = (span > 0) ? beta * n * (y[i] - yn) / span : 0.0;
  }
  __syncwarp();
  c = 0;
  for (int i = lane; i < n; i += 32, ++c) y[i] = v[c];
  __syncwarp();
}
__device__ inline void ep_grad(const double* y, double* d, int n, int lane) {
  for (int i = lane; i < n; i += 32) {
    if (n == 1) d[i] = 0.0;
    else if (i == 0) d[i] = y[1] - y[0];
    else if (i == n - 1) d[i] = y[n - 1] - y[n - 2];
    else d[i] = 0.5 * (y[i + 1] - y[i - 1]);
  }
  __syncwarp();
}
// k of a hard rule (FIXED, CURVATURE, SLOPE, MEDIAN); all lanes return it
__device__ inline int ep_rule_k(int mode, const double* lam, int n, double beta, int k_fixed, int literal, double* s0,
                         double* s1, double* s2, int lane) {
  switch (mode) {
    case LCF_T_FIXED: return k_fixed < 0 ? 0 : (k_fixed > n ? n : k_fixed);
    case LCF_T_CURVATURE: {
      if (n < 3) return 0;
      ep_norm_log(lam, n, beta, literal, s0, lane);
      ep_grad(s0, s1, n, lane);
      ep_grad(s1, s2, n, lane);
      double best = -1.0;
      int bi = 0x7fffffff;
      for (int i = 1 + lane; i < n - 1; i += 32) {
        const double q = 1.0 + s1[i] * s1[i];
        const double kap = fabs(s2[i]) / (q * sqrt(q));
        if (kap > best) { best = kap; bi = i; }
      }
      for (int o = 16; o; o >>= 1) {   // max, ties to the smallest index (first maximum)
        const double ob = __shfl_xor_sync(~0u, best, o);
        const int oi = __shfl_xor_sync(~0u, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      return bi == 0x7fffffff ? 2 : bi + 1;
    }
    case LCF_T_SLOPE: {
      if (n < 2) return 0;
      ep_norm_log(lam, n, 1.0, literal, s0, lane);
      ep_grad(s0, s1, n, lane);
      int first = n - 1;
      for (int i = lane; i < n; i += 32)
        if (-s1[i] <= beta && i < first) first = i;
      for (int o = 16; o; o >>= 1) first = min(first, __shfl_xor_sync(~0u, first, o));
      return first;
    }
    case LCF_T_MEDIAN: {
      const double med = (n & 1) ? lam[n / 2] : 0.5 * (lam[n / 2 - 1] + lam[n / 2]);
      const double T = beta * med;
      int cnt = 0;
      for (int i = lane; i < n; i += 32) cnt += lam[i] > T;
      for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(~0u, cnt, o);
      return cnt;
    }
    default: return 0;
  }
}


}  // namespace lcf
