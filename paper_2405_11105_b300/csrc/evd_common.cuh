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


// k of a hard rule (FIXED, CURVATURE, SLOPE, MEDIAN) over the whole CTA: the per-element FP64
// arithmetic of ep_rule_k (log10, the normalisation, the two gradients, the curvature) one element
// per thread, so the FP64 units of all four schedulers share it (warp 0 alone took ~40 us a window
// at Nt = 100); the maximum (ties to the smallest index) and the counts do not depend on the order.
// Every thread calls it and gets k.  Uses y, d1, d2 (n doubles each) and red (one int).
__device__ inline int ep_rule_k_cta(int mode, const double* lam, int n, double beta, int k_fixed, int literal, double* y,
                             double* d1, double* d2, int* red, int tid, int nthr) {
  if (mode == LCF_T_FIXED) return k_fixed < 0 ? 0 : (k_fixed > n ? n : k_fixed);
  if (mode == LCF_T_MEDIAN) {
    const double med = (n & 1) ? lam[n / 2] : 0.5 * (lam[n / 2 - 1] + lam[n / 2]);
    const double T = beta * med;
    if (tid == 0) *red = 0;
    __syncthreads();
    int cnt = 0;
    for (int i = tid; i < n; i += nthr) cnt += lam[i] > T;
    if (cnt) atomicAdd(red, cnt);
    __syncthreads();
    const int r = *red;
    __syncthreads();
    return r;
  }
  if (mode != LCF_T_CURVATURE && mode != LCF_T_SLOPE) return 0;
  if (mode == LCF_T_CURVATURE ? n < 3 : n < 2) return 0;
  const double bt = mode == LCF_T_CURVATURE ? beta : 1.0;
  for (int i = tid; i < n; i += nthr) y[i] = log10(ep_floor(lam, n, i));
  __syncthreads();
  const double y1 = y[0], yn = y[n - 1], span = y1 - yn;
  __syncthreads();
  for (int i = tid; i < n; i += nthr) {
    if (literal) y[i] = (y1 != 0.0) ? bt * y[i] / y1 * n : 0.0;
    else y[i] = (span > 0) ? bt * n * (y[i] - yn) / span : 0.0;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nthr)
    d1[i] = i == 0 ? y[1] - y[0] : (i == n - 1 ? y[n - 1] - y[n - 2] : 0.5 * (y[i + 1] - y[i - 1]));
  __syncthreads();
  if (mode == LCF_T_SLOPE) {
    if (tid == 0) *red = n - 1;
    __syncthreads();
    for (int i = tid; i < n; i += nthr)
      if (-d1[i] <= beta) atomicMin(red, i);
    __syncthreads();
    const int r = *red;
    __syncthreads();
    return r;
  }
  for (int i = tid; i < n; i += nthr)
    d2[i] = i == 0 ? d1[1] - d1[0] : (i == n - 1 ? d1[n - 1] - d1[n - 2] : 0.5 * (d1[i + 1] - d1[i - 1]));
  __syncthreads();
  for (int i = tid; i < n; i += nthr) {   // the curvature, into y
    if (i >= 1 && i < n - 1) {
      const double q = 1.0 + d1[i] * d1[i];
      y[i] = fabs(d2[i]) / (q * sqrt(q));
    }
  }
  __syncthreads();
  if (tid < 32) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = 1 + tid; i < n - 1; i += 32) {
      const double kap = y[i];
      if (kap > best) { best = kap; bi = i; }
    }
    for (int o = 16; o; o >>= 1) {   // max, ties to the smallest index (first maximum)
      const double ob = __shfl_xor_sync(~0u, best, o);
      const int oi = __shfl_xor_sync(~0u, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (tid == 0) *red = bi == 0x7fffffff ? 2 : bi + 1;
  }
  __syncthreads();
  const int r = *red;
  __syncthreads();
  return r;
}

// The weights of the thresholding rule for lam (descending) into wts over the whole CTA (every
// thread calls it); returns the cut k of a hard or sigmoid rule, -1 for the adaptive soft rule
// (whose per-element log and exp run one element per thread, the maximum on warp 0).  Uses y, d1,
// d2 (n doubles each), red and mxs.
__device__ inline int ep_rule_weights_cta(int md, const double* lam, int n, double beta, double beta_src, int k_fixed,
                                          int k_src, int literal, double* wts, double* y, double* d1, double* d2,
                                          int* red, double* mxs, int tid, int nthr) {
  int kk = -1;
  if (md == LCF_T_NONE) {
    for (int i = tid; i < n; i += nthr) wts[i] = 1.0;
    kk = 0;
  } else if (md <= LCF_T_MEDIAN) {
    kk = ep_rule_k_cta(md, lam, n, beta, k_fixed, literal, y, d1, d2, red, tid, nthr);
    for (int i = tid; i < n; i += nthr) wts[i] = (i + 1 > kk) ? 1.0 : 0.0;
  } else if (md == LCF_T_SIGMOID) {
    kk = ep_rule_k_cta(k_src, lam, n, beta_src, k_fixed, literal, y, d1, d2, red, tid, nthr);
    for (int i = tid; i < n; i += nthr) wts[i] = 1.0 / (1.0 + exp(-beta * ((i + 1) - kk)));
  } else {   // LCF_T_ADAPTIVE_SOFT (method 4's rule is applied afterwards by the post kernel)
    for (int i = tid; i < n; i += nthr) {
      const double u = n > 1 ? 2.5 * i / (n - 1) : 0.0;
      wts[i] = -0.5 * u * u - beta * log(ep_floor(lam, n, i));
    }
    __syncthreads();
    if (tid < 32) {
      double mx = -INFINITY;
      for (int i = tid; i < n; i += 32) mx = fmax(mx, wts[i]);
      for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(~0u, mx, o));
      if (tid == 0) *mxs = mx;
    }
    __syncthreads();
    const double mx = *mxs;
    for (int i = tid; i < n; i += nthr) wts[i] = exp(wts[i] - mx);
  }
  __syncthreads();
  return kk;
}

// ---- cyclic round-robin ordering over np (even) indices in h = np/2 pair slots ----
// At step r (0 <= r < np-1) slot i holds ((r + i) mod (np-1), (r - i) mod (np-1)), slot 0 (r, np-1).
// Returns the slot of index x and sets its partner.
__device__ __forceinline__ int ep_slot(int x, int r, int np, int h, int& partner) {
  const int M = np - 1;
  if (x == M) { partner = r; return 0; }
  int i = x - r;
  if (i < 0) i += M;                        // x = (r + i) mod M
  if (i < h) {
    partner = i == 0 ? M : (r - i < 0 ? r - i + M : r - i);
    return i;
  }
  const int i2 = M - i;                     // x = (r - i2) mod M, 1 <= i2 < h
  partner = r + i2 >= M ? r + i2 - M : r + i2;
  return i2;
}

// Complex Jacobi rotation for the Hermitian 2x2 block [[app, b], [conj(b), aqq]] (p < q):
// rotate unless |b| <= tol sqrt(|app aqq|); c real, st = s b/|b|; new diagonal dp, dq.
// 1/sqrt and 1/x by the hardware approximation plus one Newton-Raphson step.
__device__ __forceinline__ void ep_rotation(float app, float aqq, float2 b, float tol, float& c, float2& st,
                                            float& dp, float& dq, int& rot) {
  const float b2 = b.x * b.x + b.y * b.y;
  c = 1.f;
  st = make_float2(0.f, 0.f);
  dp = app;
  dq = aqq;
  rot = 0;
  if (b2 > 0.f && b2 > (tol * tol) * fabsf(app * aqq)) {
    const float ib = ep_rsqrt(b2), ab = b2 * ib;   // 1/|b|, |b|
    const float zeta = 0.5f * (aqq - app) * ib;
    float t;
    if (fabsf(zeta) > 1e18f) {
      t = 0.5f * ep_rcp(zeta);
    } else {
      const float z2 = fmaf(zeta, zeta, 1.f);
      t = copysignf(ep_rcp(fabsf(zeta) + z2 * ep_rsqrt(z2)), zeta);   // 1 / (|zeta| + sqrt(1 + zeta^2))
    }
    c = ep_rsqrt(fmaf(t, t, 1.f));
    const float sib = t * c * ib;
    st = make_float2(sib * b.x, sib * b.y);
    dp = fmaf(-t, ab, app);
    dq = fmaf(t, ab, aqq);
    rot = 1;
  }
}

// The same rotation from two reciprocal square roots: with d = aqq - app and
// x = d^2 + 4|b|^2, cos 2theta = |d| / sqrt(x), c^2 = y = (1 + cos 2theta) / 2,
//   st = sgn(d) b / (sqrt(x) c),   t|b| = sgn(d) |b|^2 / (sqrt(x) y),
// which equals the tangent form's t = sgn(d) / (|zeta| + sqrt(1 + zeta^2)) (zeta = d / 2|b|),
// c = 1 / sqrt(1 + t^2), st = t c b / |b|.  x below 2^-100 takes the tangent form.
__device__ __forceinline__ void ep_rotation2(float app, float aqq, float2 b, float tol, float& c, float2& st,
                                             float& dp, float& dq, int& rot) {
  const float b2 = b.x * b.x + b.y * b.y;
  c = 1.f;
  st = make_float2(0.f, 0.f);
  dp = app;
  dq = aqq;
  rot = 0;
  if (b2 > 0.f && b2 > (tol * tol) * fabsf(app * aqq)) {
    const float d = aqq - app;
    const float x = fmaf(d, d, 4.f * b2);
    if (!(x >= 7.888609052e-31f)) {   // 2^-100
      ep_rotation(app, aqq, b, tol, c, st, dp, dq, rot);
      return;
    }
    const float ir = ep_rsqrt(x);
    const float y = fmaf(0.5f * fabsf(d), ir, 0.5f);
    const float ic = ep_rsqrt(y);
    c = y * ic;
    const float sg = d < 0.f ? -1.f : 1.f;
    const float f = sg * ir * ic;
    st = make_float2(f * b.x, f * b.y);
    const float tb = sg * b2 * ir * (ic * ic);
    dp = app - tb;
    dq = aqq + tb;
    rot = 1;
  }
}

// The rotation of ep_rotation2 for the one-sided kernels (the updated diagonal is not needed:
// column norms are summed again) together with the "calm" test of the stopping rule: a pair is
// calm when it does not rotate, or when its cosine |b| / sqrt(app aqq) is at most clim and its
// sine |st| at most slim.  One rotation of the pair (p, q) with sine s moves the cosine of p or q
// with a third column by at most about s times that column's cosine with the other one, and a
// circle touches each pair 2 (n - 2) times, so after a whole calm circle every cosine is at most
// about 2 n clim slim.  With clim = sqrt(n) tol and slim = 1 / (2 n^(3/2)) that is tol, the
// rotation threshold itself, and the circle that would only confirm convergence is skipped (the
// sweep-level test of one-sided Jacobi SVD codes, which stop once n max|cos| max|sin| is below
// the tolerance).
__device__ __forceinline__ void ep_rotation_os(float app, float aqq, float2 b, float tol, float clim2, float slim2,
                                               float& c, float2& st, int& rot, bool& calm) {
  const float b2 = b.x * b.x + b.y * b.y;
  c = 1.f;
  st = make_float2(0.f, 0.f);
  rot = 0;
  calm = true;
  const float pq = fabsf(app * aqq);
  if (b2 > 0.f && b2 > (tol * tol) * pq) {
    const float d = aqq - app;
    const float x = fmaf(d, d, 4.f * b2);
    if (!(x >= 7.888609052e-31f)) {   // 2^-100
      float dp, dq;
      ep_rotation(app, aqq, b, tol, c, st, dp, dq, rot);
      calm = b2 <= clim2 * pq && st.x * st.x + st.y * st.y <= slim2;
      return;
    }
    const float ir = ep_rsqrt(x);
    const float y = fmaf(0.5f * fabsf(d), ir, 0.5f);
    const float ic = ep_rsqrt(y);
    c = y * ic;
    const float f = (d < 0.f ? -ir : ir) * ic;
    st = make_float2(f * b.x, f * b.y);
    rot = 1;
    calm = b2 <= clim2 * pq && (f * f) * b2 <= slim2;   // |st|^2 = f^2 |b|^2
  }
}

}  // namespace lcf
