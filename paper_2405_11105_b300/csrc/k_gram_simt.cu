// k_gram_simt.cu — packet deflation and the plain FP32 (CUDA-core) windowed
// Gram R_k = C_w^H C_w = sum_p g_k(p)^2 s_p^H s_p  (Eq. 1, Eq. 12).
//
// Numerics.  Each pixel row is split as s_p = c_p + sum_j a_pj phi_j^T, where
// phi_j (j < d, d <= 16) is the per-packet slow-time basis of k_basis.cu (the
// dominant global tissue modes) and a_pj = sum_t conj(phi_j(t)) s_p(t).  With
// the augmented row x_p = [c_p, a_p] (Nt + d entries) and R' = sum_p g^2 x_p^H x_p,
//   R = E^H R' E,  E = [I_Nt ; Phi^T]
//     = R'_cc + U Phi^T + conj(Phi) U^H + conj(Phi) Q Phi^T,
// U = R'[0:Nt, Nt:], Q = R'[Nt:, Nt:], assembled in FP64; the identity holds
// for any basis.  The large same-sign sums end up in Q (d^2 entries, exact
// double-float products) and U (double-float promotion every 4 pixels); the
// Nt x Nt block only sums the small residual c_p (blood and noise) with
// 32-pixel FP32 partial sums.
#include <math.h>

#include "lcf_internal.cuh"

namespace lcf {

// xa[t][p] = c_p(t) = s_p(t) - sum_j a_pj phi_j(t) (t < nt), xa[nt+j][p] = a_pj.
// If xmax_bits is given, the largest |component| written is max-reduced into it
// (non-negative floats order like their bit patterns).
// A CTA is 64 pixels x 4 slow-time phases (t = sub mod 4, one phase per pair of
// warps): a warp reads 32 consecutive pixels of one frame, and four times as many
// loads are in flight as with one thread per pixel.
// DM: the largest deflation depth the instance handles (4 or kDeflateMax); nd_defl <= DM.
template <int DM>
__device__ __forceinline__ void center_body(const float2* __restrict__ iq, const float2* __restrict__ phi, float2* __restrict__ xa, int nt,
                int nd_defl, int npix, unsigned* xmax_bits) {
  __shared__ float2 red[4][DM][64];
  const int pix = threadIdx.x & 63, sub = threadIdx.x >> 6;
  const int p = blockIdx.x * 64 + pix;
  const bool valid = p < npix;
  float2 a[DM];
#pragma unroll
  for (int j = 0; j < DM; ++j) a[j] = make_float2(0.f, 0.f);
  if (valid) {
#pragma unroll 4
    for (int t = sub; t < nt; t += 4) {
      const float2 v = iq[(size_t)t * npix + p];
#pragma unroll
      for (int j = 0; j < DM; ++j)
        if (j < nd_defl) {
          const float2 f = phi[j * nt + t];   // a_j += conj(phi_j(t)) s(t)
          a[j].x = fmaf(f.x, v.x, fmaf(f.y, v.y, a[j].x));
          a[j].y = fmaf(f.x, v.y, fmaf(-f.y, v.x, a[j].y));
        }
    }
  }
#pragma unroll
  for (int j = 0; j < DM; ++j) red[sub][j][pix] = a[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < DM; ++j)
    a[j] = cadd(cadd(red[0][j][pix], red[1][j][pix]), cadd(red[2][j][pix], red[3][j][pix]));
  float mx = 0.f;
  if (valid) {
#pragma unroll 4
    for (int t = sub; t < nt; t += 4) {
      float2 v = iq[(size_t)t * npix + p];
#pragma unroll
      for (int j = 0; j < DM; ++j)
        if (j < nd_defl) {
          const float2 f = phi[j * nt + t];   // c(t) = s(t) - a_j phi_j(t)
          v.x = fmaf(-a[j].x, f.x, fmaf(a[j].y, f.y, v.x));
          v.y = fmaf(-a[j].x, f.y, fmaf(-a[j].y, f.x, v.y));
        }
      xa[(size_t)t * npix + p] = v;
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int j = 0; j < DM; j += 4)   // coefficient rows sub, sub + 4, ...
      if (j + sub < nd_defl) {
        const float2 c = a[j + sub];
        xa[(size_t)(nt + j + sub) * npix + p] = c;
        mx = fmaxf(mx, fmaxf(fabsf(c.x), fabsf(c.y)));
      }
  }
  if (xmax_bits) {
    const unsigned m = __reduce_max_sync(~0u, __float_as_uint(mx));
    if ((threadIdx.x & 31) == 0) atomicMax(xmax_bits, m);
  }
}

template <int DM>
__global__ void __launch_bounds__(256)
center_kernel_t(const float2* __restrict__ iq, const float2* __restrict__ phi, float2* __restrict__ xa, int nt,
                int nd_defl, int npix, unsigned* xmax_bits) {
  center_body<DM>(iq, phi, xa, nt, nd_defl, npix, xmax_bits);
}

cudaError_t launch_center(const lcf_plan* P, const float2* iq, cudaStream_t st) {
  int n = P->npix;
  // the basis kernel, launched before this one, has zeroed the packet maximum
  const bool tc = P->cfg.gram_path == LCF_PATH_TC || P->cfg.project_path == LCF_PATH_TC;
  unsigned* xm = tc ? P->ws.xmax : nullptr;
  if (P->ndefl <= 4)
    center_kernel_t<4><<<(n + 63) / 64, 256, 0, st>>>(iq, P->ws.phi, P->ws.xa, P->nt, P->ndefl, n, xm);
  else
    center_kernel_t<kDeflateMax><<<(n + 63) / 64, 256, 0, st>>>(iq, P->ws.phi, P->ws.xa, P->nt, P->ndefl, n, xm);
  return counted(P);
}

// the depth-4 instance under a plain name, for the allocation-free entry point (default depths)
__global__ void __launch_bounds__(256)
center_kernel(const float2* __restrict__ iq, const float2* __restrict__ phi, float2* __restrict__ xa, int nt,
              int nd_defl, int npix, unsigned* xmax_bits) {
  center_body<4>(iq, phi, xa, nt, nd_defl, npix, xmax_bits);
}

constexpr int GT = 64;   // Gram tile (complex entries per side)
constexpr int GCH = 32;  // pixels per FP32 partial sum

// Residual block R'_cc.  grid: x = upper-triangle tile pair, y = pixel split,
// z = window.  Writes part[k][s][i][j] for the tile's entries (i, j < n1).
__global__ void __launch_bounds__(256, 1)
gram_simt_kernel(const float2* __restrict__ xa, int nz, int nx, int n1, const Box* __restrict__ boxes,
                 const float* __restrict__ gz, const float* __restrict__ gx, int ntile, int nsplit,
                 double2* __restrict__ part) {
  __shared__ float2 As[GCH][GT];   // g^2 conj(x_p(i))
  __shared__ float2 Bs[GCH][GT];   // x_p(j)
  const int k = blockIdx.z, s = blockIdx.y;
  int ti = 0, rem = blockIdx.x;
  while (rem >= ntile - ti) { rem -= ntile - ti; ++ti; }
  const int tj = ti + rem;
  const Box b = boxes[k];
  const int W = b.x1 - b.x0;
  const long Pk = (long)(b.z1 - b.z0) * W;
  const long l0 = Pk * s / nsplit, l1 = Pk * (s + 1) / nsplit;
  const int npix = nz * nx;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float* gzk = gz + (size_t)k * nz;
  const float* gxk = gx + (size_t)k * nx;

  float2 acc[4][4];
  df hr[4][4], hi[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[a][c] = make_float2(0.f, 0.f);
      hr[a][c] = {0.f, 0.f};
      hi[a][c] = {0.f, 0.f};
    }

  __shared__ int gpix[GCH];     // the step's linear pixel indices (-1: past the range)
  __shared__ float gg2[GCH];    // and squared window weights
  for (long l = l0; l < l1; l += GCH) {
    if (threadIdx.x < GCH) {   // (the previous step's tables were read before its closing barrier)
      const int ll = (int)l + threadIdx.x;   // box pixel counts are below 2^31 (plan validation)
      int p = -1;
      float g2 = 0.f;
      if (ll < l1) {
        const int zr = ll / W, xr = ll - zr * W;
        p = (b.z0 + zr) * nx + b.x0 + xr;
        const float g = gzk[b.z0 + zr] * gxk[b.x0 + xr];
        g2 = g * g;
      }
      gpix[threadIdx.x] = p;
      gg2[threadIdx.x] = g2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < GCH * GT; e += 256) {
      int pp = e % GCH, tt = e / GCH;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      const int p = gpix[pp];
      if (p >= 0) {
        const float g2 = gg2[pp];
        int i = ti * GT + tt, j = tj * GT + tt;
        if (i < n1) { float2 v = xa[(size_t)i * npix + p]; va = make_float2(g2 * v.x, -g2 * v.y); }
        if (j < n1) vb = xa[(size_t)j * npix + p];
      }
      As[pp][tt] = va;
      Bs[pp][tt] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int pp = 0; pp < GCH; ++pp) {
      float2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[pp][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[pp][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[a][c].x = fmaf(av[a].x, bv[c].x, fmaf(-av[a].y, bv[c].y, acc[a][c].x));
          acc[a][c].y = fmaf(av[a].x, bv[c].y, fmaf(av[a].y, bv[c].x, acc[a][c].y));
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        hr[a][c] = df_add_f(hr[a][c], acc[a][c].x);
        hi[a][c] = df_add_f(hi[a][c], acc[a][c].y);
        acc[a][c] = make_float2(0.f, 0.f);
      }
  }
  double2* out = part + ((size_t)k * nsplit + s) * n1 * n1;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = ti * GT + ty + 16 * a, j = tj * GT + tx + 16 * c;
      if (i < n1 && j < n1) out[(size_t)i * n1 + j] = make_double2(df_to_double(hr[a][c]), df_to_double(hi[a][c]));
    }
}

cudaError_t launch_gram_simt(const lcf_plan* P, cudaStream_t st) {
  int nt2 = P->gram_tiles * (P->gram_tiles + 1) / 2;
  dim3 grid(nt2, P->gram_nsplit, P->nd);
  gram_simt_kernel<<<grid, 256, 0, st>>>(P->ws.xa, P->cfg.nz, P->cfg.nx, P->nt, P->ws.box, P->ws.gz,
                                          P->ws.gx, P->gram_tiles, P->gram_nsplit, P->ws.gpart);
  return counted(P);
}

constexpr int ACH = 32;  // pixels staged per step of the augmented-column kernel
constexpr int APR = 4;   // pixels per FP32 partial sum there

// Augmented columns Y[i][a] = sum_p g^2 conj(x_p(i)) a_p(a), i < nt + qrows, a < d
// (rows i < nt give U, rows nt.. give Q; qrows = d, or 0 when Q comes from the
// exact coefficient kernel).  grid: x = pixel split, y = window.
// DM: the largest deflation depth of the instance (its accumulators are sized for it).
template <int DM>
__device__ __forceinline__ void gram_aug_body(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl,
                                              const Box* __restrict__ boxes, const float* __restrict__ gz,
                                              const float* __restrict__ gx, int nsplit, int qrows,
                                              double2* __restrict__ aug, float2* Xs) {
  __shared__ float g2s[2][ACH];    // the steps' window weights squared, by step parity
  __shared__ int pix[2][ACH];      // linear pixel index of the steps' pixels (-1: past the range)
  const int k = blockIdx.y, s = blockIdx.x;
  const int na = nt + nd_defl, nout = (nt + qrows) * nd_defl;
  const Box b = boxes[k];
  const int W = b.x1 - b.x0;
  const long Pk = (long)(b.z1 - b.z0) * W;
  const long l0 = Pk * s / nsplit, l1 = Pk * (s + 1) / nsplit;
  const int npix = nz * nx;
  const float* gzk = gz + (size_t)k * nz;
  const float* gxk = gx + (size_t)k * nx;
  // outputs per thread: nout = (nt + d) * d <= (kEvdNmax + DM) * DM over 256 threads
  constexpr int OPT = ((kEvdNmax + DM) * DM + 255) / 256;
  static_assert(OPT * 256 >= (kEvdNmax + DM) * DM, "augmented outputs per thread");
  float2 acc[OPT];
  df hr[OPT], hi[OPT];
#pragma unroll
  for (int u = 0; u < OPT; ++u) { acc[u] = make_float2(0.f, 0.f); hr[u] = {0.f, 0.f}; hi[u] = {0.f, 0.f}; }

  // Steps of ACH pixels, double-buffered: the copies of step t + 1 (cp.async, zero-filled past the
  // range) are in flight while step t is summed.
  auto pixels = [&](long l, int buf) {   // the step's pixels and weights, once per pixel
    if (threadIdx.x < ACH) {
      const int ll = (int)l + threadIdx.x;   // box pixel counts are below 2^31 (plan validation)
      int p = -1;
      float g2 = 0.f;
      if (ll < l1) {
        const int zr = ll / W, xr = ll - zr * W;
        const int z = b.z0 + zr, x = b.x0 + xr;
        p = z * nx + x;
        const float g = gzk[z] * gxk[x];
        g2 = g * g;
      }
      pix[buf][threadIdx.x] = p;
      g2s[buf][threadIdx.x] = g2;
    }
  };
  auto stage = [&](int buf) {
    float2* dst = Xs + (size_t)buf * ACH * na;
    for (int e = threadIdx.x; e < ACH * na; e += blockDim.x) {
      const int pp = e % ACH, i = e / ACH, p = pix[buf][pp];
      const float2* src = p >= 0 ? xa + (size_t)i * npix + p : xa;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst + pp * na + i)),
                   "l"(src), "r"(p >= 0 ? 8 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (l0 < l1) {
    pixels(l0, 0);
    __syncthreads();
    stage(0);
  }
  int buf = 0;
  for (long l = l0; l < l1; l += ACH, buf ^= 1) {
    if (l + ACH < l1) pixels(l + ACH, buf ^ 1);
    __syncthreads();   // the next step's pixels are known; every thread is past step t - 1 (its buffer)
    if (l + ACH < l1) {
      stage(buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();   // step t's rows are in
    const float2* Xb = Xs + (size_t)buf * ACH * na;
    const float* g2b = g2s[buf];
#pragma unroll
    for (int u = 0; u < OPT; ++u) {
      int o = threadIdx.x + u * blockDim.x;
      if (o >= nout) break;
      int i = o / nd_defl, a = o % nd_defl;
      if (i >= nt) {
        // Q block: the largest entries of R', summed with exact products
        // (g^2 * conj(x_i) * x_b in double-float) so that its rounding, which
        // reaches every eigenvalue through Phi, stays at the double-float level
        for (int pp = 0; pp < ACH; ++pp) {
          float g2 = g2b[pp];
          float2 xi = Xb[pp * na + i], xb = Xb[pp * na + nt + a];
          df wr = two_prod_df(g2, xi.x), wi = two_prod_df(-g2, xi.y);      // g^2 conj(x_i)
          df rr = df_mul_f(wr, xb.x), ii = df_mul_f(wi, xb.y);
          df ri = df_mul_f(wr, xb.y), ir = df_mul_f(wi, xb.x);
          hr[u] = df_add(hr[u], df_add(rr, df_neg(ii)));
          hi[u] = df_add(hi[u], df_add(ri, ir));
        }
        continue;
      }
      for (int p0 = 0; p0 < ACH; p0 += APR) {
#pragma unroll
        for (int pp = p0; pp < p0 + APR; ++pp) {
          float g2 = g2b[pp];
          float2 xi = Xb[pp * na + i], xb = Xb[pp * na + nt + a];
          float ar = g2 * xi.x, ai = -g2 * xi.y;          // g^2 conj(x_i)
          acc[u].x = fmaf(ar, xb.x, fmaf(-ai, xb.y, acc[u].x));
          acc[u].y = fmaf(ar, xb.y, fmaf(ai, xb.x, acc[u].y));
        }
        hr[u] = df_add_f(hr[u], acc[u].x);
        hi[u] = df_add_f(hi[u], acc[u].y);
        acc[u] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
  }
  double2* out = aug + ((size_t)k * nsplit + s) * nout;
#pragma unroll
  for (int u = 0; u < OPT; ++u) {
    int o = threadIdx.x + u * blockDim.x;
    if (o < nout) out[o] = make_double2(df_to_double(hr[u]), df_to_double(hi[u]));
  }
}

template <int DM>
__global__ void __launch_bounds__(256, DM > 4 ? 1 : 2)
gram_aug_kernel_t(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl, const Box* __restrict__ boxes,
                  const float* __restrict__ gz, const float* __restrict__ gx, int nsplit, int qrows,
                  double2* __restrict__ aug) {
  extern __shared__ float2 Xs[];   // [2][ACH][nt + d]: x_p, pixel-major, by step parity
  gram_aug_body<DM>(xa, nz, nx, nt, nd_defl, boxes, gz, gx, nsplit, qrows, aug, Xs);
}

// the depth-4 instance under a plain name, for the allocation-free entry point (default depths)
__global__ void __launch_bounds__(256)
gram_aug_kernel(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl, const Box* __restrict__ boxes,
                const float* __restrict__ gz, const float* __restrict__ gx, int nsplit, int qrows,
                double2* __restrict__ aug) {
  extern __shared__ float2 Xs[];
  gram_aug_body<4>(xa, nz, nx, nt, nd_defl, boxes, gz, gx, nsplit, qrows, aug, Xs);
}

size_t gram_aug_smem_bytes(int nt, int nd_defl) { return (size_t)2 * ACH * (nt + nd_defl) * sizeof(float2); }   // two steps

// the augmented-column kernel's staging passes 48 KB beyond Nt = 188
size_t gram_assemble_smem_bytes(int nt, int nd_defl);
__global__ void gram_assemble_kernel(const double2* __restrict__ part, const double2* __restrict__ aug,
                                     const float2* __restrict__ phi, int nsplit, int aug_nsplit, int nt,
                                     int nd_defl, double2* __restrict__ R);
cudaError_t gram_simt_configure() {
  cudaError_t e = cudaFuncSetAttribute(gram_aug_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gram_aug_smem_bytes(kEvdNmax, kDeflateMax));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_aug_kernel_t<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gram_aug_smem_bytes(kEvdNmax, kDeflateMax));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_aug_kernel_t<kDeflateMax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gram_aug_smem_bytes(kEvdNmax, kDeflateMax));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(gram_assemble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gram_assemble_smem_bytes(kEvdNmax, kDeflateMax));
}

cudaError_t launch_gram_aug(const lcf_plan* P, cudaStream_t st, bool with_q) {
  dim3 grid(P->aug_nsplit, P->nd);
  if (P->ndefl <= 4)
    gram_aug_kernel_t<4><<<grid, 256, gram_aug_smem_bytes(P->nt, P->ndefl), st>>>(
        P->ws.xa, P->cfg.nz, P->cfg.nx, P->nt, P->ndefl, P->ws.box, P->ws.gz, P->ws.gx, P->aug_nsplit,
        with_q ? P->ndefl : 0, P->ws.gaug);
  else
    gram_aug_kernel_t<kDeflateMax><<<grid, 256, gram_aug_smem_bytes(P->nt, P->ndefl), st>>>(
        P->ws.xa, P->cfg.nz, P->cfg.nx, P->nt, P->ndefl, P->ws.box, P->ws.gz, P->ws.gx, P->aug_nsplit,
        with_q ? P->ndefl : 0, P->ws.gaug);
  return counted(P);
}

// Residual-block entry summed over splits (entries with a > b from conj of b,a).
__device__ __forceinline__ double2 cc_entry(const double2* __restrict__ pk, int nsplit, int n, int a, int b) {
  bool up = a <= b;
  int r = up ? a : b, c = up ? b : a;
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    double2 v = pk[(size_t)s * n * n + (size_t)r * n + c];
    sx += v.x;
    sy += v.y;
  }
  return up ? make_double2(sx, sy) : make_double2(sx, -sy);
}

// R = R'_cc + U Phi^T + Phi U^H + Phi Q Phi^T  (FP64)
__global__ void gram_assemble_kernel(const double2* __restrict__ part, const double2* __restrict__ aug,
                                     const float2* __restrict__ phi, int nsplit, int aug_nsplit, int nt,
                                     int nd_defl, double2* __restrict__ R) {
  const int k = blockIdx.y;
  const int na = nt + nd_defl, nout = na * nd_defl;
  const double2* pk = part + (size_t)k * nsplit * nt * nt;
  const double2* ak = aug + (size_t)k * aug_nsplit * nout;
  extern __shared__ double2 asm_dyn[];   // U [nt][kDeflateMax], Q [kDeflateMax]^2, ph [d][kEvdNmax]
  double2 (*U)[kDeflateMax] = reinterpret_cast<double2 (*)[kDeflateMax]>(asm_dyn);
  double2 (*Q)[kDeflateMax] = reinterpret_cast<double2 (*)[kDeflateMax]>(asm_dyn + (size_t)nt * kDeflateMax);
  double2 (*ph)[kEvdNmax] =
      reinterpret_cast<double2 (*)[kEvdNmax]>(asm_dyn + (size_t)(nt + kDeflateMax) * kDeflateMax);
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < aug_nsplit; ++s) {
      double2 v = ak[(size_t)s * nout + o];
      sx += v.x;
      sy += v.y;
    }
    int i = o / nd_defl, a = o % nd_defl;
    if (i < nt) U[i][a] = make_double2(sx, sy);
    else Q[i - nt][a] = make_double2(sx, sy);
  }
  for (int e = threadIdx.x; e < nt * nd_defl; e += blockDim.x) {
    float2 f = phi[e];
    ph[e / nt][e % nt] = make_double2((double)f.x, (double)f.y);
  }
  __syncthreads();
  // Q is Hermitian: keep its Hermitian part so that R is exactly Hermitian
  if (threadIdx.x == 0)
    for (int a = 0; a < nd_defl; ++a)
      for (int c = a; c < nd_defl; ++c) {
        double2 x = Q[a][c], y = Q[c][a];
        double2 h = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
        Q[a][c] = h;
        Q[c][a] = make_double2(h.x, -h.y);
      }
  __syncthreads();
  constexpr int WPT = (kEvdNmax * kDeflateMax + 255) / 256;   // W entries per thread (blockDim 256)
  double2 wv[WPT];
  for (int u = 0; u < WPT; ++u) {              // W = U + 1/2 conj(Phi) Q
    int e = threadIdx.x + u * blockDim.x;
    if (e < nt * nd_defl) wv[u] = deflated_w(e / nd_defl, e % nd_defl, nd_defl, U, Q, ph);
  }
  __syncthreads();
  for (int u = 0; u < WPT; ++u) {
    int e = threadIdx.x + u * blockDim.x;
    if (e < nt * nd_defl) U[e / nd_defl][e % nd_defl] = wv[u];
  }
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nt * nt; e += gridDim.x * blockDim.x) {
    int i = e / nt, j = e % nt;
    double2 r = cc_entry(pk, nsplit, nt, i, j);
    add_w_terms(r, i, j, nd_defl, U, ph);
    if (i == j) r.y = 0.0;
    R[(size_t)k * nt * nt + e] = r;
  }
}

// U (nt rows), Q and the basis (d rows) in double precision: the assembly kernels' shared memory
size_t gram_assemble_smem_bytes(int nt, int nd_defl) {
  return ((size_t)(nt + kDeflateMax) * kDeflateMax + (size_t)nd_defl * kEvdNmax) * sizeof(double2);
}

cudaError_t launch_gram_assemble(const lcf_plan* P, cudaStream_t st) {
  dim3 grid((P->nt * P->nt + 255) / 256 < 8 ? (P->nt * P->nt + 255) / 256 : 8, P->nd);
  gram_assemble_kernel<<<grid, 256, gram_assemble_smem_bytes(P->nt, P->ndefl), st>>>(P->ws.gpart, P->ws.gaug, P->ws.phi, P->gram_nsplit, P->aug_nsplit,
                                              P->nt, P->ndefl, P->ws.R);
  return counted(P);
}

}  // namespace lcf
