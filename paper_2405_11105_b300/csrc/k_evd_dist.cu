// k_evd_dist.cu — batched Hermitian EVD (Eq. 2) for packets longer than one
// SM's shared memory holds (128 < Nt <= kEvdNmax), on a cluster of C CTAs per
// window (C = 4 up to Nt = 224, 8 above).
//
// Same numerical plan as the one-CTA and CTA-pair kernels: FP32 subspace
// iteration for the dominant directions, Householder QR, the double-float
// congruence B = Q^H R Q (compact WY form), cyclic Jacobi in FP32 with the
// relative off-diagonal test, sort / phase fix / rules in double.
//
//  evd_prep_kernel    one CTA per window, R read from global memory: subspace
//                     iteration, QR, T, congruence; writes B (fp32, full
//                     Hermitian), the reflectors Vh, T and the scale.
//  evd_dist_kernel    the Jacobi sweeps and everything after.  The round-robin
//                     ordering puts pair i at step r on indices
//                     ((r + i) mod (Np-1), (r - i) mod (Np-1)) (pair 0: (r, Np-1)),
//                     so from one step to the next the first index of every
//                     pair moves down one pair slot and the second moves up
//                     one.  CTA c owns a contiguous range of pair slots and
//                     holds both full rows (all Np columns, by original index)
//                     of each: the 2x2 block update of A_{pq} rows by J_p^H and
//                     columns by J_t is then local and in place; per step only
//                     two rows cross to the neighbouring CTAs (distributed
//                     shared memory, into a two-row mailbox).  The rotation
//                     records of all pairs are broadcast to every CTA, which
//                     applies them to its own block of V's rows.  Two cluster
//                     barriers per step.
#include <cooperative_groups.h>
#include <math.h>

#include "evd_common.cuh"
#include "lcf_internal.cuh"

namespace cg = cooperative_groups;

namespace lcf {

constexpr int ED_THREADS = 512;
constexpr float ED_TOL = 2.0e-6f;
constexpr int ED_SUBSPACE_ITERS = 6;
constexpr unsigned ED_REC_ROT = 1u << 20;

int evd_dist_cluster(int nt) { return nt <= 224 ? 4 : 8; }

struct EdArgs {
  int nt, nz, nx;
  int thresh_mode;
  double beta, beta_src;
  int k_fixed, k_src;
  int pd_mode, alpha_mode, curv_norm, max_sweeps;
  int ncp;
  int* err;
};

// ----------------------------------------------------------------------------
// evd_prep_kernel: shared memory Ys, Zs (m x ldy, column-major), Yd, Zd (n x m df64)
// + for Nt <= kEvdPairNmax, fp32(R / scale) (n x n) for the subspace iteration
size_t evd_prep_smem_bytes(int n) {
  const int m = n < kEvdHead ? n : kEvdHead, ldy = n + 1;
  return 2 * (size_t)m * ldy * 8 + 2 * (size_t)n * m * 16 + 1024 + (n <= kEvdPairNmax ? (size_t)n * n * 8 : 0);
}

__global__ void __launch_bounds__(ED_THREADS, 1)
evd_prep_kernel(const double2* __restrict__ Rg, int n, int iters, float2* __restrict__ Bg, float2* __restrict__ Vhg,
                float2* __restrict__ Tg, double* __restrict__ scale_g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = n < kEvdHead ? n : kEvdHead, ldy = n + 1;
  const double2* R = Rg + (size_t)k * n * n;
  float2* Ys = reinterpret_cast<float2*>(smem);
  float2* Zs = Ys + (size_t)m * ldy;
  zdf* Yd = reinterpret_cast<zdf*>(Zs + (size_t)m * ldy);
  zdf* Zd = Yd + (size_t)n * m;
  float2* Rf = reinterpret_cast<float2*>(smem + 2 * (size_t)m * ldy * 8 + 2 * (size_t)n * m * 16 + 1024);
  const bool rf = n <= kEvdPairNmax;   // fp32(R / scale) staged once in shared memory
  __shared__ double sh_scale;
  __shared__ float betas[kEvdHead];
  __shared__ float2 Tm[kEvdHead * kEvdHead];
  __shared__ zdf Mm[kEvdHead * kEvdHead], MT[kEvdHead * kEvdHead], W2[kEvdHead * kEvdHead];
  __shared__ float2 cs[kEvdHead];
  __shared__ float sh_nrm;
  if (warp == 0) {
    double mx = 0.0;
    for (int i = lane; i < n; i += 32) mx = fmax(mx, R[(size_t)i * n + i].x);
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(~0u, mx, o));
    if (lane == 0) sh_scale = mx;
  }
  __syncthreads();
  const double dmax = sh_scale;
  if (!(dmax > 0.0) || !isfinite(dmax)) {
    if (tid == 0) scale_g[k] = 0.0;   // degenerate: the cluster kernel writes the empty result
    return;
  }
  int ex;
  frexp(dmax, &ex);
  const double scale = ldexp(1.0, ex);
  const float s_lo = ldexpf(1.f, -ex);
  if (tid == 0) scale_g[k] = scale;
  if (rf) {
    for (int e = tid; e < n * n; e += ED_THREADS) {
      const double2 r = R[e];
      Rf[e] = make_float2(df_from_double_scaled(r.x, ex).hi, df_from_double_scaled(r.y, ex).hi);
    }
  }

  // ---- subspace iteration on fp32(R / scale), R from global memory
  for (int e = tid; e < m * ldy; e += ED_THREADS) {
    const int j = e / ldy, a = e % ldy;
    unsigned hsh = (unsigned)(a * 2654435761u) ^ (unsigned)(j * 40503u + 7u);
    hsh ^= hsh >> 13; hsh *= 0x5bd1e995u; hsh ^= hsh >> 15;
    const float re = (float)(hsh & 0xffff) / 65536.f - 0.5f, im = (float)(hsh >> 16) / 65536.f - 0.5f;
    Ys[e] = (a < n) ? make_float2(re, im) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    if (rf) {   // Z = R Y from the staged fp32 copy, one thread per (row, column)
      for (int e = tid; e < n * m; e += ED_THREADS) {
        const int a = e / m, j = e % m;
        float2 acc = make_float2(0.f, 0.f);
        const float2* yy = Ys + (size_t)j * ldy;
        const float2* rs = Rf + (size_t)a * n;
        for (int b = 0; b < n; ++b) {
          const float2 r = rs[b], y = yy[b];
          acc.x = fmaf(r.x, y.x, fmaf(-r.y, y.y, acc.x));
          acc.y = fmaf(r.x, y.y, fmaf(r.y, y.x, acc.y));
        }
        Zs[(size_t)j * ldy + a] = acc;
      }
    } else {    // from global memory, one thread per row: each double converted once for all columns
      for (int a = tid; a < n; a += ED_THREADS) {
        float2 acc[kEvdHead];
#pragma unroll
        for (int j = 0; j < kEvdHead; ++j) acc[j] = make_float2(0.f, 0.f);
        const double2* rr = R + (size_t)a * n;
        for (int b = 0; b < n; ++b) {
          const double2 rd = rr[b];
          const float2 r = make_float2((float)rd.x * s_lo, (float)rd.y * s_lo);
#pragma unroll
          for (int j = 0; j < kEvdHead; ++j) {
            if (j < m) {
              const float2 y = Ys[(size_t)j * ldy + b];
              acc[j].x = fmaf(r.x, y.x, fmaf(-r.y, y.y, acc[j].x));
              acc[j].y = fmaf(r.x, y.y, fmaf(r.y, y.x, acc[j].y));
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kEvdHead; ++j)
          if (j < m) Zs[(size_t)j * ldy + a] = acc[j];
      }
    }
    __syncthreads();
    if (rf) {   // Nt <= 128: CGS2 of Z's columns into Y by warp 0 in registers (lane: rows lane + 32 i)
      if (warp == 0) {
        float2 z[kEvdHead][4];
#pragma unroll
        for (int j = 0; j < kEvdHead; ++j)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int a = lane + 32 * i;
            z[j][i] = (j < m && a < n) ? Zs[(size_t)j * ldy + a] : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int j = 0; j < kEvdHead; ++j) {
          if (j >= m) break;
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            float2 c[kEvdHead];
#pragma unroll
            for (int l = 0; l < j; ++l) {
              float2 d = make_float2(0.f, 0.f);
#pragma unroll
              for (int i = 0; i < 4; ++i) d = cadd(d, cmulc(z[l][i], z[j][i]));
              for (int o = 16; o; o >>= 1) { d.x += __shfl_xor_sync(~0u, d.x, o); d.y += __shfl_xor_sync(~0u, d.y, o); }
              c[l] = d;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float2 v = z[j][i];
#pragma unroll
              for (int l = 0; l < j; ++l) v = csub(v, cmul(c[l], z[l][i]));
              z[j][i] = v;
            }
          }
          float nr = 0.f;
#pragma unroll
          for (int i = 0; i < 4; ++i) nr += cabs2(z[j][i]);
          for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
          if (nr > 0.f) {   // a vanished column keeps the previous iterate
            const float sc = rsqrtf(nr);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              z[j][i] = cscale(z[j][i], sc);
              const int a = lane + 32 * i;
              if (a < n) Ys[(size_t)j * ldy + a] = z[j][i];
            }
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int a = lane + 32 * i;
              z[j][i] = a < n ? Ys[(size_t)j * ldy + a] : make_float2(0.f, 0.f);
            }
          }
        }
      }
      __syncthreads();
      continue;
    }
    for (int j = 0; j < m; ++j) {   // CGS2 of Z's columns into Y
      float2* zj = Zs + (size_t)j * ldy;
      for (int pass = 0; pass < 2 && j > 0; ++pass) {
        if (warp < j) {
          const float2* yw = Ys + (size_t)warp * ldy;
          float2 c = make_float2(0.f, 0.f);
          for (int a = lane; a < n; a += 32) c = cadd(c, cmulc(yw[a], zj[a]));
          for (int o = 16; o; o >>= 1) { c.x += __shfl_xor_sync(~0u, c.x, o); c.y += __shfl_xor_sync(~0u, c.y, o); }
          if (lane == 0) cs[warp] = c;
        }
        __syncthreads();
        for (int a = tid; a < n; a += ED_THREADS) {
          float2 z = zj[a];
          for (int i = 0; i < j; ++i) z = csub(z, cmul(cs[i], Ys[(size_t)i * ldy + a]));
          zj[a] = z;
        }
        __syncthreads();
      }
      if (warp == 0) {
        float nr = 0.f;
        for (int a = lane; a < n; a += 32) nr += cabs2(zj[a]);
        for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
        if (lane == 0) sh_nrm = nr;
      }
      __syncthreads();
      const float nr = sh_nrm;
      if (nr > 0.f) {
        const float sc = rsqrtf(nr);
        for (int a = tid; a < n; a += ED_THREADS) Ys[(size_t)j * ldy + a] = cscale(zj[a], sc);
      }
      __syncthreads();
    }
  }
  // ---- Householder QR of Y, reflectors -> Zs; compact WY T.  Column j's reflector by warp 0, its
  // application to the later columns by one warp each; T's inner products by all warps.
  for (int j = 0; j < m; ++j) {
    float2* yj = Ys + (size_t)j * ldy;
    float2* vj = Zs + (size_t)j * ldy;
    if (warp == 0) {
      float nr = 0.f;
      for (int a = j + lane; a < n; a += 32) nr += cabs2(yj[a]);
      for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
      const float alpha = sqrtf(nr);
      const float2 x0 = yj[j];
      const float ax0 = sqrtf(cabs2(x0));
      const float2 e = ax0 > 0.f ? cscale(x0, 1.f / ax0) : make_float2(1.f, 0.f);
      const float beta = alpha > 0.f ? 1.f / (alpha * (alpha + ax0)) : 0.f;
      for (int a = lane; a < ldy; a += 32) {
        float2 v = (a < j || a >= n) ? make_float2(0.f, 0.f) : yj[a];
        if (a == j) v = cadd(x0, cscale(e, alpha));
        vj[a] = v;
      }
      if (lane == 0) betas[j] = beta;
    }
    __syncthreads();
    const int c = j + warp;   // warp w > 0 updates column j + w
    if (warp > 0 && c < m) {
      float2* yc = Ys + (size_t)c * ldy;
      float2 t = make_float2(0.f, 0.f);
      for (int a = j + lane; a < n; a += 32) t = cadd(t, cmulc(vj[a], yc[a]));
      for (int o = 16; o; o >>= 1) { t.x += __shfl_xor_sync(~0u, t.x, o); t.y += __shfl_xor_sync(~0u, t.y, o); }
      t = cscale(t, betas[j]);
      for (int a = j + lane; a < n; a += 32) yc[a] = csub(yc[a], cmul(vj[a], t));
    }
    __syncthreads();
  }
  for (int q = warp; q < m * m; q += ED_THREADS / 32) {   // Mm[i m + j].re.hi = v_i^H v_j, i < j
    const int i = q / m, j = q % m;
    if (i >= j) continue;
    float2 c = make_float2(0.f, 0.f);
    for (int a = lane; a < n; a += 32) c = cadd(c, cmulc(Zs[(size_t)i * ldy + a], Zs[(size_t)j * ldy + a]));
    for (int o = 16; o; o >>= 1) { c.x += __shfl_xor_sync(~0u, c.x, o); c.y += __shfl_xor_sync(~0u, c.y, o); }
    if (lane == 0) Mm[q].re.hi = c.x, Mm[q].im.hi = c.y;
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = 0; j < m; ++j) {
      if (lane < j) {
        float2 acc = make_float2(0.f, 0.f);
        for (int l = lane; l < j; ++l) acc = cadd(acc, cmul(Tm[lane * m + l], make_float2(Mm[l * m + j].re.hi, Mm[l * m + j].im.hi)));
        Tm[lane * m + j] = cscale(acc, -betas[j]);
      }
      if (lane == 0) {
        Tm[j * m + j] = make_float2(betas[j], 0.f);
        for (int i = j + 1; i < m; ++i) Tm[i * m + j] = make_float2(0.f, 0.f);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < m * n; e += ED_THREADS) Vhg[(size_t)k * m * n + e] = Zs[(size_t)(e / n) * ldy + e % n];
  for (int e = tid; e < m * m; e += ED_THREADS) Tg[(size_t)k * m * m + e] = Tm[e];

  // ---- B = R/scale - (Vh Z^H + Z Vh^H), double-float
  // Yd = (R / scale) Vh, 4 threads per row; every lane runs every block (the shuffles need the full warp)
  for (int a0 = 0; a0 < n; a0 += ED_THREADS / 4) {
    const int a = a0 + (tid >> 2), sub = tid & 3;
    zdf acc[kEvdHead];
#pragma unroll
    for (int j = 0; j < kEvdHead; ++j) acc[j] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int b = sub; a < n && b < n; b += 4) {
      const double2 r = R[(size_t)a * n + b];
      zdf rz;
      if (rf) {   // integer-pipe split for the short packets; the long ones keep the FP64 conversion
        rz.re = df_from_double_scaled(r.x, ex); rz.im = df_from_double_scaled(r.y, ex);
      } else {
        rz.re = df_from_double(r.x); rz.im = df_from_double(r.y);
        rz.re.hi *= s_lo; rz.re.lo *= s_lo; rz.im.hi *= s_lo; rz.im.lo *= s_lo;
      }
#pragma unroll
      for (int j = 0; j < kEvdHead; ++j)
        if (j < m) acc[j] = zdf_add(acc[j], zdf_mul_c(rz, Zs[(size_t)j * ldy + b]));
    }
#pragma unroll
    for (int j = 0; j < kEvdHead; ++j) {
      zdf v = acc[j];
      for (int o = 1; o < 4; o <<= 1) {
        zdf t;
        t.re.hi = __shfl_xor_sync(~0u, v.re.hi, o); t.re.lo = __shfl_xor_sync(~0u, v.re.lo, o);
        t.im.hi = __shfl_xor_sync(~0u, v.im.hi, o); t.im.lo = __shfl_xor_sync(~0u, v.im.lo, o);
        v = zdf_add(v, t);
      }
      if (sub == 0 && j < m && a < n) Yd[a * m + j] = v;
    }
  }
  __syncthreads();
  for (int q = warp; q < m * m; q += ED_THREADS / 32) {   // M = Vh^H Yd
    const int i = q / m, j = q % m;
    zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
    for (int a = lane; a < n; a += 32) acc = zdf_add(acc, zdf_mul_c(Yd[a * m + j], cconj(Zs[(size_t)i * ldy + a])));
    for (int o = 16; o; o >>= 1) {
      zdf t;
      t.re.hi = __shfl_xor_sync(~0u, acc.re.hi, o); t.re.lo = __shfl_xor_sync(~0u, acc.re.lo, o);
      t.im.hi = __shfl_xor_sync(~0u, acc.im.hi, o); t.im.lo = __shfl_xor_sync(~0u, acc.im.lo, o);
      acc = zdf_add(acc, t);
    }
    if (lane == 0) Mm[q] = acc;
  }
  __syncthreads();
  if (tid < m * m) {
    const int i = tid / m, j = tid % m;
    zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
    for (int l = 0; l <= j; ++l) acc = zdf_add(acc, zdf_mul_c(Mm[i * m + l], Tm[l * m + j]));
    MT[tid] = acc;
  }
  __syncthreads();
  if (tid < m * m) {
    const int i = tid / m, j = tid % m;
    zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
    for (int l = 0; l <= i; ++l) acc = zdf_add(acc, zdf_mul_c(MT[l * m + j], cconj(Tm[l * m + i])));
    W2[tid] = acc;
  }
  __syncthreads();
  for (int e = tid; e < n * m; e += ED_THREADS) {   // Z = Yd T - 1/2 Vh W2
    const int a = e / m, j = e % m;
    zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
    for (int l = 0; l <= j; ++l) acc = zdf_add(acc, zdf_mul_c(Yd[a * m + l], Tm[l * m + j]));
    zdf c2 = {{0.f, 0.f}, {0.f, 0.f}};
    for (int l = 0; l < m; ++l) c2 = zdf_add(c2, zdf_mul_c(W2[l * m + j], Zs[(size_t)l * ldy + a]));
    c2.re.hi *= 0.5f; c2.re.lo *= 0.5f; c2.im.hi *= 0.5f; c2.im.lo *= 0.5f;
    acc.re = df_add(acc.re, df_neg(c2.re));
    acc.im = df_add(acc.im, df_neg(c2.im));
    Zd[e] = acc;
  }
  __syncthreads();
  float2* B = Bg + (size_t)k * n * n;
  for (int e = tid; e < n * n; e += ED_THREADS) {
    const int a = e / n, b = e % n;
    if (a > b) continue;
    const double2 r = R[(size_t)a * n + b];
    zdf x;
    if (rf) {
      x.re = df_from_double_scaled(r.x, ex); x.im = df_from_double_scaled(r.y, ex);
    } else {
      x.re = df_from_double(r.x); x.im = df_from_double(r.y);
      x.re.hi *= s_lo; x.re.lo *= s_lo; x.im.hi *= s_lo; x.im.lo *= s_lo;
    }
    zdf c = {{0.f, 0.f}, {0.f, 0.f}};
    for (int j = 0; j < m; ++j) {
      zdf zb = Zd[b * m + j];
      zb.im = df_neg(zb.im);
      c = zdf_add(c, zdf_mul_c(zb, Zs[(size_t)j * ldy + a]));
      c = zdf_add(c, zdf_mul_c(Zd[a * m + j], cconj(Zs[(size_t)j * ldy + b])));
    }
    x.re = df_add(x.re, df_neg(c.re));
    x.im = df_add(x.im, df_neg(c.im));
    const float2 v = make_float2(x.re.hi + x.re.lo, a == b ? 0.f : x.im.hi + x.im.lo);
    B[(size_t)a * n + b] = v;
    if (a != b) B[(size_t)b * n + a] = cconj(v);
  }
}

// ----------------------------------------------------------------------------
__host__ __device__ inline size_t ed_align(size_t x) { return (x + 15) & ~(size_t)15; }

// evd_dist_kernel shared-memory layout (every CTA of the cluster the same)
struct EdLayout {
  int np, h, C, nsmax, vmax;
  size_t rows, v, rec, dq, tb, bb, ta, dg, fl, end;
};
__host__ __device__ inline EdLayout ed_layout(int n, int C) {
  EdLayout L;
  L.np = n + (n & 1);
  L.h = L.np / 2;
  L.C = C;
  L.nsmax = (L.h + C - 1) / C;
  L.vmax = (n + C - 1) / C;
  size_t o = 0;
  L.rows = o; o = ed_align(o + (size_t)(2 * L.nsmax + 2) * L.np * 8);   // row buffers + 2 mailbox rows
  L.v = o;    o = ed_align(o + (size_t)L.vmax * L.np * 8);               // this CTA's rows of V
  L.rec = o;  o = ed_align(o + (size_t)L.h * 16);                        // rotation records of all pairs
  L.dq = o;   o = ed_align(o + (size_t)L.h * 8);                         // new diagonal of own pairs
  L.tb = o;   o = ed_align(o + (size_t)L.nsmax * 4);                     // buffer of each own pair's top row
  L.bb = o;   o = ed_align(o + (size_t)L.nsmax * 4);                     // ... and bottom row
  L.ta = o;   o = ed_align(o + (size_t)L.nsmax * 4);                     // first index of each own pair
  L.dg = o;   o = ed_align(o + (size_t)L.np * 4);                        // whole diagonal (sweep-start test)
  L.fl = o;   o = ed_align(o + (size_t)16 * 4);                          // per-CTA test flags
  L.end = o;
  return L;
}
size_t evd_dist_smem_bytes(int nt, int C) { return ed_layout(nt, C).end; }

__device__ __forceinline__ void ed_st_remote4(uint32_t addr, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void ed_st_remote2(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

__global__ void __launch_bounds__(ED_THREADS, 1)
evd_dist_kernel(const float2* __restrict__ Bg, const float2* __restrict__ Vhg, const float2* __restrict__ Tg,
                const double* __restrict__ scale_g, const Box* __restrict__ boxes, EdArgs g,
                double* __restrict__ lam_out, float2* __restrict__ V_out, float* __restrict__ wt_out,
                int* __restrict__ kcut_out, float* __restrict__ alpha_out, int* __restrict__ flags_out,
                float2* __restrict__ W_out, int* __restrict__ ncol_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int k = blockIdx.x / C, n = g.nt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const EdLayout L = ed_layout(n, C);
  const int np = L.np, h = L.h, m = n < kEvdHead ? n : kEvdHead;
  const int i0 = (int)((long)h * rank / C), i1 = (int)((long)h * (rank + 1) / C), ns = i1 - i0;
  const int v0 = (int)((long)n * rank / C), v1 = (int)((long)n * (rank + 1) / C), nv = v1 - v0;
  float2* rows = reinterpret_cast<float2*>(smem + L.rows);   // buffer b at rows + b * np
  float2* mb_top = rows + (size_t)(2 * L.nsmax) * np;         // mailbox: incoming top row
  float2* mb_bot = mb_top + np;                                // mailbox: incoming bottom row
  float2* V = reinterpret_cast<float2*>(smem + L.v);          // V[r - v0][c], c by original index
  float4* rec = reinterpret_cast<float4*>(smem + L.rec);
  float2* dq = reinterpret_cast<float2*>(smem + L.dq);
  int* tb = reinterpret_cast<int*>(smem + L.tb);
  int* bb = reinterpret_cast<int*>(smem + L.bb);
  int* ta_s = reinterpret_cast<int*>(smem + L.ta);    // first index of each own pair at this step
  const double scale = scale_g[k];

  if (!(scale > 0.0)) {   // degenerate window (zero Gram): every CTA writes its share of the empty result
    for (int e = tid; e < nv * n; e += ED_THREADS) {
      const int r = v0 + e / n, c = e % n;
      V_out[(size_t)k * n * n + (size_t)r * n + c] = make_float2(r == c, 0.f);
    }
    for (int e = tid; e < nv * g.ncp; e += ED_THREADS)
      W_out[(size_t)k * n * g.ncp + (size_t)v0 * g.ncp + e] = make_float2(0.f, 0.f);
    if (rank == 0) {
      for (int i = tid; i < n; i += ED_THREADS) {
        lam_out[(size_t)k * n + i] = 0.0;
        wt_out[(size_t)k * n + i] = 0.f;
      }
      if (tid == 0) {
        kcut_out[k] = 0; alpha_out[k] = 0.f; ncol_out[k] = 0;
        flags_out[k] = LCF_WFLAG_DEGENERATE;
      }
    }
    return;
  }

  // ---- A rows of the own pair slots at step 0: slot i holds (i, Np-1-i)
  const float2* B = Bg + (size_t)k * n * n;
  for (int ls = tid; ls < ns; ls += ED_THREADS) { tb[ls] = 2 * ls; bb[ls] = 2 * ls + 1; }
  for (int e = tid; e < 2 * ns * np; e += ED_THREADS) {
    const int b = e / np, c = e % np, ls = b >> 1;
    const int idx = (b & 1) ? (np - 1 - (i0 + ls)) : (i0 + ls);
    rows[(size_t)b * np + c] = (idx < n && c < n) ? B[(size_t)idx * n + c] : make_float2(0.f, 0.f);
  }
  // ---- V rows v0..v1 of Q = I - Vh T Vh^H
  {
    const float2* Vh = Vhg + (size_t)k * m * n;   // [j][a]
    const float2* Tm = Tg + (size_t)k * m * m;
    for (int e = tid; e < nv * np; e += ED_THREADS) {
      const int r = v0 + e / np, c = e % np;
      float2 v = make_float2(r == c ? 1.f : 0.f, 0.f);
      if (c < n) {
        for (int j = 0; j < m; ++j) {
          float2 vt = make_float2(0.f, 0.f);   // (Vh T)[r][j]
          for (int l = 0; l <= j; ++l) vt = cadd(vt, cmul(Vh[(size_t)l * n + r], Tm[l * m + j]));
          v = csub(v, cmul(vt, cconj(Vh[(size_t)j * n + c])));
        }
      }
      V[(size_t)(e / np) * np + c] = v;
    }
  }
  cluster.sync();

  const uint32_t rec_l = ep_smem(rec);
  // the bottom row of our last slot goes up (rank + 1's mailbox bottom); the top row of our first slot
  // goes down (rank - 1's mailbox top)
  const uint32_t up_bot = rank + 1 < C ? ep_mapa(ep_smem(mb_bot), rank + 1) : 0u;
  const uint32_t down_top = rank > 0 ? ep_mapa(ep_smem(mb_top), rank - 1) : 0u;
  int sweeps = 0, converged = 0;
  const int maxsw = g.max_sweeps > 0 ? g.max_sweeps : 40;
  float* dgl = reinterpret_cast<float*>(smem + L.dg);
  int* flg = reinterpret_cast<int*>(smem + L.fl);
  for (; sweeps < maxsw; ++sweeps) {
    if (sweeps > 0) {
      // A sweep with no rotation leaves A unchanged: test every pair at once instead (step-0
      // layout here: own slot i holds rows i and Np-1-i).  The diagonal goes to every CTA, each
      // tests its own rows, the flags are exchanged.
      for (int ls = tid; ls < ns; ls += ED_THREADS) {
        const int i = i0 + ls, x0 = i, x1 = np - 1 - i;
        const float d0 = rows[(size_t)tb[ls] * np + x0].x, d1 = rows[(size_t)bb[ls] * np + x1].x;
        for (int dst = 0; dst < C; ++dst) {
          ep_st_remote_u32(ep_mapa(ep_smem(dgl + x0), dst), __float_as_uint(d0));
          ep_st_remote_u32(ep_mapa(ep_smem(dgl + x1), dst), __float_as_uint(d1));
        }
      }
      cluster.sync();
      int big = 0;
      const float tol2 = ED_TOL * ED_TOL;
      for (int e = tid; e < 2 * ns * np; e += ED_THREADS) {
        const int bq = e / np, c = e - bq * np, ls = bq >> 1, i = i0 + ls;
        const int x = (bq & 1) ? np - 1 - i : i;
        if (c == x) continue;
        const float2 v = rows[(size_t)((bq & 1) ? bb[ls] : tb[ls]) * np + c];
        const float v2 = cabs2(v);
        big |= v2 > 0.f && v2 > tol2 * fabsf(dgl[x] * dgl[c]);
      }
      big = __syncthreads_or(big);
      if (tid < C) ep_st_remote_u32(ep_mapa(ep_smem(flg + rank), tid), (unsigned)big);
      cluster.sync();
      int anybig = 0;
      for (int q = 0; q < C; ++q) anybig |= flg[q];
      if (!anybig) { converged = 1; break; }
    }
    int any = 0;
    for (int r = 0; r < np - 1; ++r) {
      // (a) rotations of the own pairs; records to every CTA
      if (tid < ns) {
        const int ls = tid, i = i0 + ls;
        int ta, ba;
        if (i == 0) { ta = r; ba = np - 1; }
        else { ta = (r + i) % (np - 1); ba = (r - i + np - 1) % (np - 1); }
        ta_s[ls] = ta;
        const float2* Rt = rows + (size_t)tb[ls] * np;
        const float2* Rb = rows + (size_t)bb[ls] * np;
        const bool tlow = ta < ba;
        const int p = tlow ? ta : ba, q = tlow ? ba : ta;
        const float2* Rp = tlow ? Rt : Rb;
        const float2* Rq = tlow ? Rb : Rt;
        const float app = Rp[p].x, aqq = Rq[q].x;
        const float2 b = Rp[q];
        const float b2 = cabs2(b);
        float c = 1.f, dp = app, dqq = aqq;
        float2 st = make_float2(0.f, 0.f);
        int rot = 0;
        if (b2 > 0.f && b2 > (ED_TOL * ED_TOL) * fabsf(app * aqq)) {
          const float ib = ep_rsqrt(b2), ab = b2 * ib;
          const float zeta = 0.5f * (aqq - app) * ib;
          float t;
          if (fabsf(zeta) > 1e18f) {
            t = 0.5f * ep_rcp(zeta);
          } else {
            const float z2 = fmaf(zeta, zeta, 1.f);
            t = copysignf(ep_rcp(fabsf(zeta) + z2 * ep_rsqrt(z2)), zeta);
          }
          c = ep_rsqrt(fmaf(t, t, 1.f));
          const float sib = t * c * ib;
          st = make_float2(sib * b.x, sib * b.y);
          dp = fmaf(-t, ab, app);
          dqq = fmaf(t, ab, aqq);
          rot = 1;
        }
        dq[ls] = make_float2(dp, dqq);
        const float4 rc = make_float4(c, st.x, st.y,
                                      __uint_as_float((unsigned)p | ((unsigned)q << 10) | (rot ? ED_REC_ROT : 0u)));
        for (int dst = 0; dst < C; ++dst) ed_st_remote4(ep_mapa(rec_l, dst) + (uint32_t)(i * 16), rc);
      }
      cluster.sync();
      // (b) was anything rotated in this step (same answer in every CTA)?
      int anyr = 0;
      for (int i = tid; i < h; i += ED_THREADS) anyr |= (__float_as_uint(rec[i].w) & ED_REC_ROT) != 0;
      anyr = __syncthreads_or(anyr);
      if (anyr) {
        any = 1;
        // (c) own rows: 2x2 blocks (own pair ls) x (pair t), in place
        for (int e = tid; e < ns * h; e += ED_THREADS) {
          const int ls = e / h, t = e % h, i = i0 + ls;
          const float4 ra = rec[i], rb = rec[t];
          const unsigned ma = __float_as_uint(ra.w), mbits = __float_as_uint(rb.w);
          if (!((ma | mbits) & ED_REC_ROT)) continue;
          const int pa = ma & 1023, qa = (ma >> 10) & 1023, pb = mbits & 1023, qb = (mbits >> 10) & 1023;
          const int ta = ta_s[ls];
          float2* Rp = rows + (size_t)(ta == pa ? tb[ls] : bb[ls]) * np;
          float2* Rq = rows + (size_t)(ta == pa ? bb[ls] : tb[ls]) * np;
          if (t == i) {
            const float2 d = dq[ls];
            Rp[pa] = make_float2(d.x, 0.f);
            Rq[qa] = make_float2(d.y, 0.f);
            Rp[qa] = make_float2(0.f, 0.f);
            Rq[pa] = make_float2(0.f, 0.f);
            continue;
          }
          const float ca = ra.x, cb = rb.x;
          const float2 sa = make_float2(ra.y, ra.z), sb = make_float2(rb.y, rb.z);
          const float2 x00 = Rp[pb], x01 = Rp[qb], x10 = Rq[pb], x11 = Rq[qb];
          const float2 sbc = cconj(sb);
          const float2 y00 = csub(cscale(x00, cb), cmul(sbc, x01)), y01 = cadd(cmul(sb, x00), cscale(x01, cb));
          const float2 y10 = csub(cscale(x10, cb), cmul(sbc, x11)), y11 = cadd(cmul(sb, x10), cscale(x11, cb));
          const float2 sac = cconj(sa);
          Rp[pb] = csub(cscale(y00, ca), cmul(sa, y10));
          Rp[qb] = csub(cscale(y01, ca), cmul(sa, y11));
          Rq[pb] = cadd(cmul(sac, y00), cscale(y10, ca));
          Rq[qb] = cadd(cmul(sac, y01), cscale(y11, ca));
        }
        // V rows: columns (p_t, q_t) of every rotated pair
        for (int e = tid; e < nv * h; e += ED_THREADS) {
          const int rr = e / h, t = e % h;
          const float4 rc = rec[t];
          const unsigned mt = __float_as_uint(rc.w);
          if (!(mt & ED_REC_ROT)) continue;
          const int p = mt & 1023, q = (mt >> 10) & 1023;
          const float c = rc.x;
          const float2 s = make_float2(rc.y, rc.z);
          float2* vr = V + (size_t)rr * np;
          const float2 vp = vr[p], vq = vr[q];
          vr[p] = csub(cscale(vp, c), cmul(cconj(s), vq));
          vr[q] = cadd(cmul(s, vp), cscale(vq, c));
        }
        __syncthreads();
      }
      // (d) rows leaving: top of slot i0 goes down (unless slot 0), bottom of slot i1-1 goes up
      if (rank > 0) {
        const float4* src = reinterpret_cast<const float4*>(rows + (size_t)tb[0] * np);
        for (int e = tid; e < np / 2; e += ED_THREADS) ed_st_remote4(down_top + (uint32_t)(e * 16), src[e]);
      }
      if (rank + 1 < C) {
        const float4* src = reinterpret_cast<const float4*>(rows + (size_t)bb[ns - 1] * np);
        for (int e = tid; e < np / 2; e += ED_THREADS) ed_st_remote4(up_bot + (uint32_t)(e * 16), src[e]);
      }
      cluster.sync();
      // (e) next step's roles: first indices move down one slot, second indices up one slot
      //     (slot 0 keeps Np-1; slot 1 takes slot 0's first index; the last slot's first index is
      //     the old second index of the last slot).  Buffers of rows that left take the arrivals.
      __shared__ int sh_in[2];
      {
        const int T0 = tb[0], Bl = bb[ns - 1], B0 = bb[0];
        // shifted roles, read before any is written
        const int ntb = tid + 1 < ns ? tb[tid + 1] : 0, nbb = (tid >= 1 && tid < ns) ? bb[tid - 1] : 0;
        __syncthreads();
        if (tid + 1 < ns) tb[tid] = ntb;
        if (tid >= 1 && tid < ns && !(rank == 0 && tid == 1)) bb[tid] = nbb;   // rank 0's bb[1] is set below
        if (tid == 0) {
          int in_top = -1, in_bot = -1;
          if (rank == 0) {
            bb[0] = B0;
            bb[1] = T0;
          } else {
            in_bot = (rank + 1 < C) ? Bl : T0;
            bb[0] = in_bot;
          }
          if (rank + 1 < C) {
            in_top = (rank > 0) ? T0 : Bl;
            tb[ns - 1] = in_top;
          } else {
            tb[ns - 1] = Bl;
          }
          sh_in[0] = in_top;
          sh_in[1] = in_bot;
        }
      }
      __syncthreads();
      if (sh_in[0] >= 0) {   // the top row that came from rank + 1
        float4* dst = reinterpret_cast<float4*>(rows + (size_t)sh_in[0] * np);
        const float4* src = reinterpret_cast<const float4*>(mb_top);
        for (int e = tid; e < np / 2; e += ED_THREADS) dst[e] = src[e];
      }
      if (sh_in[1] >= 0) {   // the bottom row that came from rank - 1
        float4* dst = reinterpret_cast<float4*>(rows + (size_t)sh_in[1] * np);
        const float4* src = reinterpret_cast<const float4*>(mb_bot);
        for (int e = tid; e < np / 2; e += ED_THREADS) dst[e] = src[e];
      }
      __syncthreads();
    }
    if (!any) { converged = 1; break; }
  }

  // ---------------- phase E: eigenvalues to rank 0, sort and rule there, results back
  // After the sweeps the own rows are identified by the slot roles of step 0 of the next sweep.
  double* lam0 = reinterpret_cast<double*>(smem + L.rec);   // rank 0: lambda by original index (np doubles)
  // (the record array is no longer needed; it is large enough: h*16 >= np*8)
  cluster.sync();
  {
    const uint32_t lam_r = ep_mapa(ep_smem(lam0), 0);
    for (int ls = tid; ls < ns; ls += ED_THREADS) {
      const int i = i0 + ls;
      const int ta = i, ba = np - 1 - i;   // roles at step 0
      const double lt = (double)rows[(size_t)tb[ls] * np + ta].x, lb = (double)rows[(size_t)bb[ls] * np + ba].x;
      const unsigned long long ut = __double_as_longlong(lt), ub = __double_as_longlong(lb);
      asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(lam_r + (uint32_t)(ta * 8)), "l"(ut) : "memory");
      asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(lam_r + (uint32_t)(ba * 8)), "l"(ub) : "memory");
    }
  }
  cluster.sync();
  // shared scratch after the rows are dead: perm, coef, keep, phase, column maxima
  unsigned char* scr = smem + L.rows;
  size_t so = 0;
  int* perm = reinterpret_cast<int*>(scr + so);     so += (size_t)np * 4;          // sorted -> original index
  float* coef = reinterpret_cast<float*>(scr + so); so += (size_t)np * 4;          // per sorted index
  int* keep = reinterpret_cast<int*>(scr + so);     so = ed_align(so + (size_t)(np + 1) * 4);   // [0] = ncol
  float2* phs = reinterpret_cast<float2*>(scr + so); so = ed_align(so + (size_t)np * 8);
  float4* cmax = reinterpret_cast<float4*>(scr + so); so = ed_align(so + (size_t)C * np * 16);  // [rank][col]
  double* lam_s = reinterpret_cast<double*>(scr + so);
  double* wts = lam_s + np;
  double* s0 = wts + np;
  double* s1 = s0 + np;
  double* s2 = s1 + np;
  __syncthreads();
  if (rank == 0) {
    for (int i = tid; i < n; i += ED_THREADS) {
      const double di = lam0[i];
      int rk = 0;
      for (int j = 0; j < n; ++j) {
        const double dj = lam0[j];
        rk += (dj > di) || (dj == di && j < i);
      }
      perm[rk] = i;
    }
    __syncthreads();
    for (int i = tid; i < n; i += ED_THREADS) lam_s[i] = lam0[perm[i]] * scale;
    __syncthreads();
    if (warp == 0) {
      int kk = -1;
      const int md = g.thresh_mode;
      if (md == LCF_T_NONE) {
        for (int i = lane; i < n; i += 32) wts[i] = 1.0;
        kk = 0;
      } else if (md <= LCF_T_MEDIAN) {
        kk = ep_rule_k(md, lam_s, n, g.beta, g.k_fixed, g.curv_norm, s0, s1, s2, lane);
        for (int i = lane; i < n; i += 32) wts[i] = (i + 1 > kk) ? 1.0 : 0.0;
      } else if (md == LCF_T_SIGMOID) {
        kk = ep_rule_k(g.k_src, lam_s, n, g.beta_src, g.k_fixed, g.curv_norm, s0, s1, s2, lane);
        for (int i = lane; i < n; i += 32) wts[i] = 1.0 / (1.0 + exp(-g.beta * ((i + 1) - kk)));
      } else {   // LCF_T_ADAPTIVE_SOFT
        double mx = -INFINITY;
        for (int i = lane; i < n; i += 32) {
          const double u = n > 1 ? 2.5 * i / (n - 1) : 0.0;
          wts[i] = -0.5 * u * u - g.beta * log(ep_floor(lam_s, n, i));
          mx = fmax(mx, wts[i]);
        }
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(~0u, mx, o));
        for (int i = lane; i < n; i += 32) wts[i] = exp(wts[i] - mx);
        kk = -1;
      }
      __syncwarp();
      double S = 0.0;
      for (int i = lane; i < n; i += 32) S += wts[i] * wts[i] * lam_s[i];
      for (int o = 16; o; o >>= 1) S += __shfl_xor_sync(~0u, S, o);
      double cf = 0.0;
      if (lane == 0) {
        const double pdsum = g.pd_mode == 0 ? S / n : S;
        double al;
        int fl = (converged ? 0 : LCF_WFLAG_NOCONV) | ((sweeps < 255 ? sweeps : 255) << LCF_WFLAG_SWEEP_SHIFT);
        if (g.alpha_mode == 1) al = 1.0;
        else {
          const Box bx = boxes[k];
          const double cnt = g.alpha_mode == 2 ? (double)(bx.z1 - bx.z0) * (bx.x1 - bx.x0) : (double)g.nz * g.nx;
          if (pdsum <= 1e-300) { al = 0.0; fl |= LCF_WFLAG_DEGENERATE; }
          else al = cnt / pdsum;
        }
        kcut_out[k] = kk;
        alpha_out[k] = (float)al;
        flags_out[k] = fl;
        cf = sqrt(al * (g.pd_mode == 0 ? 1.0 / n : 1.0));
      }
      cf = __shfl_sync(~0u, cf, 0);
      int base = 0;
      for (int i0c = 0; i0c < n; i0c += 32) {
        const int i = i0c + lane;
        const bool kp = i < n && wts[i] > 0.0;
        const unsigned bal = __ballot_sync(~0u, kp);
        if (kp) keep[1 + base + __popc(bal & ((1u << lane) - 1u))] = i;
        if (i < n) coef[i] = (float)(wts[i] * cf);
        base += __popc(bal);
      }
      if (lane == 0) { keep[0] = base; ncol_out[k] = base; }
    }
    __syncthreads();
    for (int i = tid; i < n; i += ED_THREADS) {
      lam_out[(size_t)k * n + i] = lam_s[i];
      wt_out[(size_t)k * n + i] = (float)wts[i];
    }
    // perm, coef, keep to the other CTAs
    for (int dst = 1; dst < C; ++dst) {
      const uint32_t base_r = ep_mapa(ep_smem(scr), dst);
      for (int e = tid; e < np * 3 + 1; e += ED_THREADS)   // perm | coef | keep (4-byte words)
        ep_st_remote_u32(base_r + 4u * e, reinterpret_cast<const uint32_t*>(scr)[e]);
    }
  }
  cluster.sync();
  // column maxima of |V|^2 over this CTA's rows -> rank 0
  {
    const uint32_t cm_r = ep_mapa(ep_smem(cmax), 0);
    for (int c = tid; c < n; c += ED_THREADS) {
      float best = -1.f;
      int bi = 0;
      for (int rr = 0; rr < nv; ++rr) {
        const float mg = cabs2(V[(size_t)rr * np + c]);
        if (mg > best) { best = mg; bi = v0 + rr; }
      }
      const float2 v = nv > 0 ? V[(size_t)(bi - v0) * np + c] : make_float2(0.f, 0.f);
      ed_st_remote4(cm_r + (uint32_t)(((size_t)rank * np + c) * 16), make_float4(best, __int_as_float(bi), v.x, v.y));
    }
  }
  cluster.sync();
  if (rank == 0) {
    for (int jj = tid; jj < n; jj += ED_THREADS) {   // largest entry of each sorted eigenvector, ties to the lower row
      const int c = perm[jj];
      float best = -1.f;
      int bi = 0x7fffffff;
      float2 v = make_float2(1.f, 0.f);
      for (int q = 0; q < C; ++q) {
        const float4 cm = cmax[(size_t)q * np + c];
        const int ri = __float_as_int(cm.y);
        if (cm.x > best || (cm.x == best && ri < bi)) { best = cm.x; bi = ri; v = make_float2(cm.z, cm.w); }
      }
      const float mg = sqrtf(cabs2(v));
      phs[jj] = mg > 0.f ? make_float2(v.x / mg, -v.y / mg) : make_float2(1.f, 0.f);
    }
    __syncthreads();
    for (int dst = 1; dst < C; ++dst) {
      const uint32_t pr = ep_mapa(ep_smem(phs), dst);
      for (int e = tid; e < n; e += ED_THREADS) ed_st_remote2(pr + 8u * e, phs[e]);
    }
  }
  cluster.sync();
  for (int e = tid; e < nv * n; e += ED_THREADS) {
    const int rr = e / n, jj = e % n;
    V_out[(size_t)k * n * n + (size_t)(v0 + rr) * n + jj] = cmul(V[(size_t)rr * np + perm[jj]], phs[jj]);
  }
  const int nc = keep[0];
  for (int e = tid; e < nv * g.ncp; e += ED_THREADS) {
    const int rr = e / g.ncp, c = e % g.ncp;
    float2 v = make_float2(0.f, 0.f);
    if (c < nc) {
      const int jj = keep[1 + c];
      v = cscale(cmul(V[(size_t)rr * np + perm[jj]], phs[jj]), coef[jj]);
    }
    W_out[(size_t)k * n * g.ncp + (size_t)(v0 + rr) * g.ncp + c] = v;
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

cudaError_t launch_evd_prep(const lcf_plan* P, cudaStream_t st, int iters) {
  evd_prep_kernel<<<P->nd, ED_THREADS, evd_prep_smem_bytes(P->nt), st>>>(P->ws.R, P->nt, iters, P->ws.evd_B,
                                                                         P->ws.evd_vh, P->ws.evd_t, P->ws.evd_scale);
  return counted(P);
}

cudaError_t launch_evd_dist(const lcf_plan* P, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  cudaError_t e = launch_evd_prep(P, st, ED_SUBSPACE_ITERS);
  if (e != cudaSuccess) return e;
  EdArgs a;
  a.nt = P->nt; a.nz = c.nz; a.nx = c.nx;
  a.thresh_mode = c.thresh_mode; a.beta = c.beta; a.beta_src = c.beta_src;
  a.k_fixed = c.k_fixed; a.k_src = c.k_src; a.pd_mode = c.pd_mode; a.alpha_mode = c.alpha_mode;
  a.curv_norm = c.curv_norm; a.max_sweeps = c.max_sweeps; a.ncp = P->ncp;
  a.err = P->ws.err;
  const int C = P->evd_cluster > 0 ? P->evd_cluster : evd_dist_cluster(P->nt);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * P->nd);
  cfg.blockDim = dim3(ED_THREADS);
  cfg.dynamicSmemBytes = evd_dist_smem_bytes(P->nt, C);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, evd_dist_kernel, (const float2*)P->ws.evd_B, (const float2*)P->ws.evd_vh,
                         (const float2*)P->ws.evd_t, (const double*)P->ws.evd_scale, (const Box*)P->ws.box, a,
                         P->ws.lam, P->ws.V, P->ws.wt, P->ws.kcut, P->ws.alpha, P->ws.flags, P->ws.W, P->ws.ncol);
  if (e != cudaSuccess) return e;
  return counted(P);
}

cudaError_t evd_dist_configure() {
  const size_t pa = evd_prep_smem_bytes(kEvdPairNmax), pb = evd_prep_smem_bytes(kEvdNmax);
  cudaError_t e = cudaFuncSetAttribute(evd_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(pa > pb ? pa : pb));
  size_t mx = 0;
  for (int nt = kEvdPairNmax + 1; nt <= kEvdNmax; ++nt)   // both cluster sizes where they fit
    for (int C = evd_dist_cluster(nt); C <= 8; C += 4) mx = evd_dist_smem_bytes(nt, C) > mx ? evd_dist_smem_bytes(nt, C) : mx;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(evd_dist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  return e;
}

}  // namespace lcf
