// k_subtract.cu — the subtractive reconstruction (Eq. 5) for hard thresholds:
// C-hat = C_w - C_w V_k V_k^H, V_k the k rejected (clutter) eigenvectors, so
//   PD_k(p) = (1/Nt) (||g s_p||^2 - ||g s_p Q||^2),   Q an orthonormal basis of V_k,
// and alpha_k (Eq. 13) from the same per-pixel energies, PD = sum_k alpha_k PD_k.
//
// The difference cancels the clutter against itself (50-60 dB), so every sum is
// double-float (FMA two-products, two-sums) and Q is the rejected columns
// re-orthonormalised in double-float (classical Gram-Schmidt twice): the FP32
// eigenvectors' own orthonormality error (~1e-7) would otherwise leave 1e-7 of the
// clutter energy in the difference.  Cost: k + 1 dot products of length Nt per
// pixel and window (k rejected components), against the PD identity's one GEMM over
// the Nt - k kept columns.
#include <math.h>

#include "lcf_internal.cuh"

namespace lcf {

constexpr int SB_THREADS = 256;

// complex double-float
__device__ __forceinline__ zdf zdf_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ zdf zdf_sub(zdf a, zdf b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }
// conj(a) * b, both complex double-float (double-float products: the low words' cross terms
// at float precision)
__device__ __forceinline__ zdf zdf_cmulc(zdf a, zdf b) {
  auto mul = [](df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return quick_two_sum(p, e);
  };
  const df rr = mul(a.re, b.re), ii = mul(a.im, b.im), ri = mul(a.re, b.im), ir = mul(a.im, b.re);
  return {df_add(rr, ii), df_add(ri, df_neg(ir))};
}
__device__ __forceinline__ zdf zdf_mul(zdf a, zdf b) {   // a * b
  zdf ac = a;
  ac.im = df_neg(ac.im);
  return zdf_cmulc(ac, b);
}

// block sum of a complex double-float (all threads get it); red: [SB_THREADS / 32] zdf
__device__ inline zdf block_sum(zdf v, zdf* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    zdf t;
    t.re.hi = __shfl_xor_sync(~0u, v.re.hi, o); t.re.lo = __shfl_xor_sync(~0u, v.re.lo, o);
    t.im.hi = __shfl_xor_sync(~0u, v.im.hi, o); t.im.lo = __shfl_xor_sync(~0u, v.im.lo, o);
    v = zdf_add(v, t);
  }
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  zdf s = zdf_zero();
  for (int w = 0; w < SB_THREADS / 32; ++w) s = zdf_add(s, red[w]);
  return s;
}

// double-float product with the cross terms of the low words
__device__ __forceinline__ df df_mul_df(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return quick_two_sum(p, e);
}

// Q = the first k columns of V orthonormalised (CGS twice, double-float), one CTA per window;
// q_hi / q_lo: [nd][nt][nt] complex (column j at [j][t]), the high and low words.  The column in
// progress lives in shared memory, the finished ones are read back from q_hi / q_lo.
__global__ void __launch_bounds__(SB_THREADS)
sub_prep_kernel(const float2* __restrict__ V, const int* __restrict__ kcut, int n, float2* __restrict__ q_hi,
                float2* __restrict__ q_lo) {
  extern __shared__ zdf cur[];   // [n]
  __shared__ zdf red[SB_THREADS / 32];
  const int k = blockIdx.x, tid = threadIdx.x;
  const int kk = min(max(kcut[k], 0), n);
  const float2* Vk = V + (size_t)k * n * n;
  float2* Qh = q_hi + (size_t)k * n * n;
  float2* Ql = q_lo + (size_t)k * n * n;
  for (int j = 0; j < kk; ++j) {
    for (int t = tid; t < n; t += SB_THREADS) {
      const float2 v = Vk[(size_t)t * n + j];
      cur[t] = {{v.x, 0.f}, {v.y, 0.f}};
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        zdf c = zdf_zero();
        for (int t = tid; t < n; t += SB_THREADS) {
          const float2 h = Qh[(size_t)i * n + t], l = Ql[(size_t)i * n + t];
          c = zdf_add(c, zdf_cmulc({{h.x, l.x}, {h.y, l.y}}, cur[t]));   // q_i^H cur
        }
        c = block_sum(c, red);
        for (int t = tid; t < n; t += SB_THREADS) {
          const float2 h = Qh[(size_t)i * n + t], l = Ql[(size_t)i * n + t];
          cur[t] = zdf_sub(cur[t], zdf_mul(c, {{h.x, l.x}, {h.y, l.y}}));
        }
        __syncthreads();
      }
    zdf nr = zdf_zero();
    for (int t = tid; t < n; t += SB_THREADS) nr = zdf_add(nr, zdf_cmulc(cur[t], cur[t]));
    nr = block_sum(nr, red);
    const double nn = df_to_double(nr.re);
    const df sc = df_from_double(nn > 0.0 ? 1.0 / sqrt(nn) : 0.0);
    for (int t = tid; t < n; t += SB_THREADS) {
      const zdf v = {df_mul_df(cur[t].re, sc), df_mul_df(cur[t].im, sc)};
      Qh[(size_t)j * n + t] = make_float2(v.re.hi, v.im.hi);
      Ql[(size_t)j * n + t] = make_float2(v.re.lo, v.im.lo);
    }
    __syncthreads();
  }
}

// Per pixel of window k's support (split s of its pixels): PD_k(p) = g^2 (E - sum_j |s_p q_j|^2) / Nt
// (or without 1/Nt for pd_mode 1), all in double-float, written to pdk[off_k + box index]; the
// split's sum of PD_k to part[k][s] (double).  Threads: one pixel each.
__global__ void __launch_bounds__(SB_THREADS)
sub_project_kernel(const float2* __restrict__ iq, int nz, int nx, int n, const Box* __restrict__ boxes,
                   const float* __restrict__ gz, const float* __restrict__ gx, const int* __restrict__ kcut,
                   const float2* __restrict__ q_hi, const float2* __restrict__ q_lo, const long long* __restrict__ pdk_off,
                   int pd_mode, int nsplit, float* __restrict__ pdk, double* __restrict__ part) {
  extern __shared__ float2 qsm[];   // a chunk of columns of Q: [QC][n] hi then [QC][n] lo
  constexpr int QC = 8;   // = SB_QC
  __shared__ double red[SB_THREADS / 32];
  const int k = blockIdx.y, s = blockIdx.x, tid = threadIdx.x;
  const Box b = boxes[k];
  const int W = b.x1 - b.x0;
  const long Pk = (long)(b.z1 - b.z0) * W;
  const long l0 = Pk * s / nsplit, l1 = Pk * (s + 1) / nsplit;
  const int kk = min(max(kcut[k], 0), n);
  const size_t npix = (size_t)nz * nx;
  const float2* Qh = q_hi + (size_t)k * n * n;
  const float2* Ql = q_lo + (size_t)k * n * n;
  double acc_sum = 0.0;
  for (long lb = l0; lb < l1; lb += SB_THREADS) {
    const long l = lb + tid;
    const bool valid = l < l1;
    size_t p = 0;
    float g = 0.f;
    if (valid) {
      const int zr = (int)(l / W), z = b.z0 + zr, x = b.x0 + (int)(l - (long)zr * W);
      p = (size_t)z * nx + x;
      g = gz[(size_t)k * nz + z] * gx[(size_t)k * nx + x];
    }
    df e = {0.f, 0.f};   // ||s_p||^2, exact squares
    if (valid)
      for (int t = 0; t < n; ++t) {
        const float2 v = iq[(size_t)t * npix + p];
        e = df_add(e, df_add(two_prod_df(v.x, v.x), two_prod_df(v.y, v.y)));
      }
    df r = {0.f, 0.f};   // sum_j |s_p q_j|^2
    for (int j0 = 0; j0 < kk; j0 += QC) {
      const int nc = min(QC, kk - j0);
      __syncthreads();
      for (int x = tid; x < nc * n; x += SB_THREADS) {
        qsm[x] = Qh[(size_t)j0 * n + x];
        qsm[QC * n + x] = Ql[(size_t)j0 * n + x];
      }
      __syncthreads();
      if (valid) {
        zdf y[QC];
#pragma unroll
        for (int c = 0; c < QC; ++c) y[c] = zdf_zero();
        for (int t = 0; t < n; ++t) {
          const float2 v = iq[(size_t)t * npix + p];
#pragma unroll
          for (int c = 0; c < QC; ++c) {
            if (c < nc) {   // y_c += s(t) q_c(t) with q = hi + lo, s exact in float
              const float2 h = qsm[c * n + t], lo = qsm[QC * n + c * n + t];
              const zdf q = {{h.x, lo.x}, {h.y, lo.y}};
              y[c].re = df_add(y[c].re, df_add(df_mul_f(q.re, v.x), df_neg(df_mul_f(q.im, v.y))));
              y[c].im = df_add(y[c].im, df_add(df_mul_f(q.im, v.x), df_mul_f(q.re, v.y)));
            }
          }
        }
#pragma unroll
        for (int c = 0; c < QC; ++c)
          if (c < nc) {
            const zdf w = zdf_cmulc(y[c], y[c]);
            r = df_add(r, w.re);
          }
      }
    }
    if (valid) {
      const double g2 = (double)g * (double)g;
      double pdv = g2 * df_to_double(df_add(e, df_neg(r)));   // e - r in double-float, then to double
      if (pdv < 0.0) pdv = 0.0;
      if (pd_mode == 0) pdv /= n;
      pdk[pdk_off[k] + l] = (float)pdv;
      acc_sum += pdv;
    }
  }
  for (int o = 16; o; o >>= 1) acc_sum += __shfl_xor_sync(~0u, acc_sum, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc_sum;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < SB_THREADS / 32; ++w) t += red[w];
    part[(size_t)k * nsplit + s] = t;
  }
}

// alpha_k from the PD sums (Eq. 13, alpha_mode as everywhere), then the blend: one thread per
// pixel, windows in order, PD_k read back from the per-window buffers.
__global__ void sub_alpha_kernel(const double* __restrict__ part, int nsplit, int nd, const Box* __restrict__ boxes,
                                 int nz, int nx, int alpha_mode, float* __restrict__ alpha, int* __restrict__ flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  double S = 0.0;
  for (int s = 0; s < nsplit; ++s) S += part[(size_t)k * nsplit + s];
  int fl = flags[k] & ~LCF_WFLAG_DEGENERATE;
  double al;
  if (alpha_mode == 1) al = 1.0;
  else {
    const Box b = boxes[k];
    const double cnt = alpha_mode == 2 ? (double)(b.z1 - b.z0) * (b.x1 - b.x0) : (double)nz * nx;
    if (S <= 1e-300) { al = 0.0; fl |= LCF_WFLAG_DEGENERATE; }
    else al = cnt / S;
  }
  alpha[k] = (float)al;
  flags[k] = fl;
}

__global__ void sub_blend_kernel(int nz, int nx, int nd, const Box* __restrict__ boxes, const float* __restrict__ alpha,
                                 const long long* __restrict__ pdk_off, const float* __restrict__ pdk,
                                 float* __restrict__ out) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (size_t)nz * nx) return;
  const int z = (int)(p / nx), x = (int)(p - (size_t)z * nx);
  double acc = 0.0;
  for (int k = 0; k < nd; ++k) {
    const Box b = boxes[k];
    if (z < b.z0 || z >= b.z1 || x < b.x0 || x >= b.x1) continue;
    const long l = (long)(z - b.z0) * (b.x1 - b.x0) + (x - b.x0);
    acc += (double)alpha[k] * (double)pdk[pdk_off[k] + l];
  }
  out[p] = (float)acc;
}

size_t sub_prep_smem_bytes(int n) { return (size_t)n * sizeof(zdf); }
constexpr int SB_QC = 8;
size_t sub_project_smem_bytes(int n) { return (size_t)2 * SB_QC * n * sizeof(float2); }

cudaError_t launch_project_subtract(const lcf_plan* P, const float2* iq, float* out, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  const int n = P->nt;
  sub_prep_kernel<<<P->nd, SB_THREADS, sub_prep_smem_bytes(n), st>>>(P->ws.V, P->ws.kcut, n, P->ws.sub_qhi,
                                                                     P->ws.sub_qlo);
  cudaError_t e = counted(P);
  if (e != cudaSuccess) return e;
  sub_project_kernel<<<dim3(P->sub_nsplit, P->nd), SB_THREADS, sub_project_smem_bytes(n), st>>>(
      iq, c.nz, c.nx, n, P->ws.box, P->ws.gz, P->ws.gx, P->ws.kcut, P->ws.sub_qhi, P->ws.sub_qlo, P->ws.sub_off,
      c.pd_mode, P->sub_nsplit, P->ws.sub_pdk, P->ws.sub_part);
  if ((e = counted(P)) != cudaSuccess) return e;
  sub_alpha_kernel<<<(P->nd + 127) / 128, 128, 0, st>>>(P->ws.sub_part, P->sub_nsplit, P->nd, P->ws.box, c.nz, c.nx,
                                                        c.alpha_mode, P->ws.alpha, P->ws.flags);
  if ((e = counted(P)) != cudaSuccess) return e;
  sub_blend_kernel<<<(unsigned)((P->npix + 255) / 256), 256, 0, st>>>(c.nz, c.nx, P->nd, P->ws.box, P->ws.alpha,
                                                                      P->ws.sub_off, P->ws.sub_pdk, out);
  return counted(P);
}

}  // namespace lcf
