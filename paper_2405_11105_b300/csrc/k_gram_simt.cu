// k_gram_simt.cu — packet centring and the plain FP32 (CUDA-core) windowed
// Gram R_k = C_w^H C_w = sum_p g_k(p)^2 s_p^H s_p  (Eq. 1, Eq. 12).
//
// Numerics.  Each pixel row is split as s_p = c_p + m_p 1 with m_p its
// slow-time mean.  The Gram of the augmented row [c_p, m_p] (Nt+1 entries)
// gives R_c, u = sum g^2 conj(c) m and q = sum g^2 |m|^2, and
//   R = R_c + u 1^T + 1 u^H + q 1 1^T
// exactly (assembled in FP64).  Removing the static tissue echo first makes
// the FP32 partial sums ~|moving tissue|^2 instead of ~|tissue|^2, which is
// what keeps eigenvalues 1e-6 below the largest accurate to 1e-4.
// Products and 32-pixel partial sums are FP32; partial sums are promoted
// into double-float accumulators.
#include "lcf_internal.cuh"

namespace lcf {

// xa[t][p] = s_p(t) - m_p for t < nt, xa[nt][p] = m_p
__global__ void center_kernel(const float2* __restrict__ iq, float2* __restrict__ xa, int nt,
                              int npix) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  float2 acc = make_float2(0.f, 0.f);
  for (int t = 0; t < nt; ++t) acc = cadd(acc, iq[(size_t)t * npix + p]);
  float2 m = cscale(acc, 1.0f / nt);
  for (int t = 0; t < nt; ++t) xa[(size_t)t * npix + p] = csub(iq[(size_t)t * npix + p], m);
  xa[(size_t)nt * npix + p] = m;
}

cudaError_t launch_center(const lcf_plan* P, const float2* iq, cudaStream_t st) {
  int n = P->npix;
  center_kernel<<<(n + 255) / 256, 256, 0, st>>>(iq, P->ws.xa, P->nt, n);
  return cudaGetLastError();
}

constexpr int GT = 64;   // Gram tile (complex entries per side)
constexpr int GCH = 32;  // pixels per FP32 partial sum

// grid: x = upper-triangle tile pair, y = pixel split, z = window
__global__ void __launch_bounds__(256, 1)
gram_simt_kernel(const float2* __restrict__ xa, int nz, int nx, int n1, const Box* __restrict__ boxes,
                 const float* __restrict__ gz, const float* __restrict__ gx, int ntile, int nsplit,
                 double2* __restrict__ part) {
  __shared__ float2 As[GCH][GT];   // g^2 conj(x_p(i))
  __shared__ float2 Bs[GCH][GT];   // x_p(j)
  const int k = blockIdx.z, s = blockIdx.y;
  // decode the upper-triangle pair (ti <= tj)
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

  for (long l = l0; l < l1; l += GCH) {
    // stage GCH pixels x GT slow-time entries of both tiles
    for (int e = threadIdx.x; e < GCH * GT; e += 256) {
      int pp = e % GCH, tt = e / GCH;
      long ll = l + pp;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (ll < l1) {
        int z = b.z0 + (int)(ll / W), x = b.x0 + (int)(ll % W);
        int p = z * nx + x;
        float g = gzk[z] * gxk[x];
        float g2 = g * g;
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
    // promote the FP32 partial sums
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
  gram_simt_kernel<<<grid, 256, 0, st>>>(P->ws.xa, P->cfg.nz, P->cfg.nx, P->n1, P->ws.box, P->ws.gz,
                                          P->ws.gx, P->gram_tiles, P->gram_nsplit, P->ws.gpart);
  return cudaGetLastError();
}

// R[k][i][j] = f(i,j) + f(i,nt) + f(nt,j) + f(nt,nt), where f(a,b) is the
// augmented Gram summed over splits (entries with a > b from conj of b,a).
__device__ __forceinline__ double2 aug_entry(const double2* __restrict__ pk, int nsplit, int n1, int a,
                                             int b) {
  bool up = a <= b;
  int r = up ? a : b, c = up ? b : a;
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    double2 v = pk[(size_t)s * n1 * n1 + (size_t)r * n1 + c];
    sx += v.x;
    sy += v.y;
  }
  return up ? make_double2(sx, sy) : make_double2(sx, -sy);
}

__global__ void gram_assemble_kernel(const double2* __restrict__ part, int nsplit, int nt,
                                     double2* __restrict__ R) {
  const int k = blockIdx.y;
  const int n1 = nt + 1;
  const double2* pk = part + (size_t)k * nsplit * n1 * n1;
  __shared__ double2 u[kEvdNmax + 1];
  __shared__ double2 q;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) u[i] = aug_entry(pk, nsplit, n1, i, nt);
  if (threadIdx.x == 0) q = aug_entry(pk, nsplit, n1, nt, nt);
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nt * nt; e += gridDim.x * blockDim.x) {
    int i = e / nt, j = e % nt;
    double2 r = aug_entry(pk, nsplit, n1, i, j);
    double2 ui = u[i], uj = u[j];
    r.x += ui.x + uj.x + q.x;          // u_i + conj(u_j) + q
    r.y += ui.y - uj.y;
    if (i == j) r.y = 0.0;
    R[(size_t)k * nt * nt + e] = r;
  }
}

cudaError_t launch_gram_assemble(const lcf_plan* P, cudaStream_t st) {
  dim3 grid((P->nt * P->nt + 255) / 256 < 8 ? (P->nt * P->nt + 255) / 256 : 8, P->nd);
  gram_assemble_kernel<<<grid, 256, 0, st>>>(P->ws.gpart, P->gram_nsplit, P->nt, P->ws.R);
  return cudaGetLastError();
}

}  // namespace lcf
