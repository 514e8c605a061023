// k_basis.cu — per-packet slow-time deflation basis for the Gram stage.
//
// The Gram identity R = E^H R' E (see k_gram_simt.cu) is exact for any basis
// Phi; the basis only decides how much of each pixel's signal is removed
// before the FP32 / tensor-core partial sums.  The tissue's slow-time
// behaviour is shared by the whole field of view (global motion), so the top
// d eigenvectors of a global Gram G = sum_p s_p^H s_p (taken over every
// eighth image row) capture it: after deflation the residual is blood and
// noise, and the rounding of the partial sums (including the tensor core's
// round-toward-zero accumulation) is relative to that small residual.
//
//  global_gram_kernel : FP32 partial Grams of the subsampled packet (64x64
//                       complex tiles, upper triangle), one per pixel split;
//  basis_kernel       : one CTA sums the partials, scales, and runs subspace
//                       iteration from the DCT-II start (CGS2 by one warp),
//                       writing phi[j][t] (complex, orthonormal columns),
//                       and zeroes the packet maximum the centring kernel
//                       accumulates.
#include <math.h>

#include "lcf_internal.cuh"

namespace lcf {

constexpr int BG_T = 64;        // tile side
constexpr int BG_CH = 32;       // pixels staged per step
constexpr int BASIS_ITERS = 4;

__host__ __device__ inline int basis_zstep(int nz) { return nz >= 64 ? 8 : (nz >= 16 ? 4 : 1); }

// grid: x = upper-triangle tile pair, y = pixel split.  Pixels: rows z = 0, zs, 2zs, ...
__global__ void __launch_bounds__(256)
global_gram_kernel(const float2* __restrict__ iq, int nz, int nx, int nt, int zs, int ntile, int nsplit,
                   float2* __restrict__ part) {
  __shared__ float2 As[BG_CH][BG_T];
  __shared__ float2 Bs[BG_CH][BG_T];
  const int s = blockIdx.y;
  int ti = 0, rem = blockIdx.x;
  while (rem >= ntile - ti) { rem -= ntile - ti; ++ti; }
  const int tj = ti + rem;
  const int nzs = (nz + zs - 1) / zs;
  const long Pk = (long)nzs * nx;
  const long l0 = Pk * s / nsplit, l1 = Pk * (s + 1) / nsplit;
  const size_t npix = (size_t)nz * nx;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
  for (long l = l0; l < l1; l += BG_CH) {
    for (int e = threadIdx.x; e < BG_CH * BG_T; e += 256) {
      int pp = e % BG_CH, tt = e / BG_CH;
      long ll = l + pp;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (ll < l1) {
        size_t p = (size_t)(ll / nx) * zs * nx + (size_t)(ll % nx);
        int i = ti * BG_T + tt, j = tj * BG_T + tt;
        if (i < nt) { float2 v = iq[(size_t)i * npix + p]; va = make_float2(v.x, -v.y); }
        if (j < nt) vb = iq[(size_t)j * npix + p];
      }
      As[pp][tt] = va;
      Bs[pp][tt] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int pp = 0; pp < BG_CH; ++pp) {
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
  }
  float2* out = part + (size_t)s * nt * nt;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = ti * BG_T + ty + 16 * a, j = tj * BG_T + tx + 16 * c;
      if (i < nt && j < nt) out[(size_t)i * nt + j] = acc[a][c];
    }
}

// Packets up to this length keep G in shared memory; longer ones read it from
// the (L2-resident) reduced partial sums.
constexpr int kBasisSmemNt = 128;

// One CTA of 256 threads.  smem: G (nt*nt float2, nt <= kBasisSmemNt) + Y, Z (nt*d float2 each).
// part: split 0 holds the full sum (upper triangle) when nsplit == 1.
__global__ void __launch_bounds__(256)
basis_kernel(const float2* __restrict__ part, int nsplit, int nt, int nd_defl, float2* __restrict__ phi,
             unsigned* __restrict__ xmax) {
  extern __shared__ float2 bsm[];
  const bool gsm = nt <= kBasisSmemNt;
  float2* G = bsm;                                   // nt*nt (shared-memory mode)
  float2* Y = gsm ? G + (size_t)nt * nt : bsm;       // nt*d, column j at Y[t*d + j]
  float2* Z = Y + (size_t)nt * nd_defl;
  __shared__ float gmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, d = nd_defl;
  if (tid == 0) *xmax = 0u;   // the centring kernel's atomicMax target for this packet
  // entry (t, u) of the summed global Gram (Hermitian, from its upper triangle)
  auto gsum = [&](int t, int u) {
    const bool up = t <= u;
    const int r = up ? t : u, c = up ? u : t;
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < nsplit; ++s) acc = cadd(acc, part[(size_t)s * nt * nt + (size_t)r * nt + c]);
    return up ? acc : cconj(acc);
  };
  if (gsm) {
    if (nsplit == 1) {   // the upper triangle once (four loads in flight per thread), mirrored
      const int nup = nt * (nt + 1) / 2;
      for (int e0 = tid; e0 < nup; e0 += 4 * blockDim.x) {
        float2 v[4];
        int tt[4], uu[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = e0 + q * blockDim.x;
          int t = 0, u = 0;
          if (e < nup) {
            const float tw = (float)(2 * nt + 1);
            t = (int)floorf(0.5f * (tw - sqrtf(fmaxf(tw * tw - 8.f * (float)e, 0.f))));
            t = t < 0 ? 0 : (t > nt - 1 ? nt - 1 : t);
            while (t > 0 && t * nt - (t * (t - 1)) / 2 > e) --t;
            while (t + 1 < nt && (t + 1) * nt - ((t + 1) * t) / 2 <= e) ++t;
            u = t + (e - (t * nt - (t * (t - 1)) / 2));
            v[q] = part[(size_t)t * nt + u];
          }
          tt[q] = e < nup ? t : -1;
          uu[q] = u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (tt[q] < 0) continue;
          G[tt[q] * nt + uu[q]] = v[q];
          G[uu[q] * nt + tt[q]] = cconj(v[q]);
        }
      }
    } else {
      for (int e = tid; e < nt * nt; e += blockDim.x) G[e] = gsum(e / nt, e % nt);
    }
    __syncthreads();
  }
  if (warp == 0) {   // largest diagonal entry
    float m = 0.f;
    for (int i = lane; i < nt; i += 32) m = fmaxf(m, gsm ? G[i * nt + i].x : gsum(i, i).x);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(~0u, m, o));
    if (lane == 0) gmax = m > 0.f ? m : 1.f;
  }
  __syncthreads();
  const float inv = 1.f / gmax;
  if (gsm) {
    for (int e = tid; e < nt * nt; e += blockDim.x) G[e] = cscale(G[e], inv);
  }
  // DCT-II start
  for (int e = tid; e < nt * d; e += blockDim.x) {
    int t = e / d, j = e % d;
    float v = (j == 0) ? rsqrtf((float)nt) : sqrtf(2.f / nt) * cosf(3.14159265f * j * (t + 0.5f) / nt);
    Y[e] = make_float2(v, 0.f);
  }
  __syncthreads();
  for (int it = 0; it < BASIS_ITERS; ++it) {
    for (int e = tid; e < nt * d; e += blockDim.x) {
      int t = e / d, j = e % d;
      float2 acc = make_float2(0.f, 0.f);
      if (gsm) {   // four interleaved partial sums
        float2 a4[4] = {acc, acc, acc, acc};
        int u = 0;
        for (; u + 4 <= nt; u += 4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) a4[q] = cadd(a4[q], cmul(G[t * nt + u + q], Y[(u + q) * d + j]));
        }
        for (; u < nt; ++u) a4[0] = cadd(a4[0], cmul(G[t * nt + u], Y[u * d + j]));
        acc = cadd(cadd(a4[0], a4[1]), cadd(a4[2], a4[3]));
      } else
        for (int u = 0; u < nt; ++u) acc = cadd(acc, cmul(cscale(gsum(t, u), inv), Y[u * d + j]));
      Z[e] = acc;
    }
    __syncthreads();
    if (warp == 0) {  // CGS2 orthonormalisation of Z -> Y
      for (int j = 0; j < d; ++j) {
        for (int pass = 0; pass < 2; ++pass)
          for (int i = 0; i < j; ++i) {
            float2 c = make_float2(0.f, 0.f);
            for (int t = lane; t < nt; t += 32) c = cadd(c, cmulc(Y[t * d + i], Z[t * d + j]));
            for (int o = 16; o; o >>= 1) { c.x += __shfl_xor_sync(~0u, c.x, o); c.y += __shfl_xor_sync(~0u, c.y, o); }
            for (int t = lane; t < nt; t += 32) Z[t * d + j] = csub(Z[t * d + j], cmul(c, Y[t * d + i]));
            __syncwarp();
          }
        float nr = 0.f;
        for (int t = lane; t < nt; t += 32) nr += cabs2(Z[t * d + j]);
        for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
        if (nr > 0.f) {
          float sc = rsqrtf(nr);
          for (int t = lane; t < nt; t += 32) Y[t * d + j] = cscale(Z[t * d + j], sc);
        }  // a vanishing direction keeps its previous (orthonormal) vector
        __syncwarp();
      }
    }
    __syncthreads();
  }
  // A row signal s_p = a phi^T puts conj(phi) in the column space of G, so the
  // deflation basis is the conjugate of G's top eigenvectors.
  for (int e = tid; e < nt * d; e += blockDim.x) {
    int t = e / d, j = e % d;
    phi[j * nt + t] = cconj(Y[e]);
  }
}

// part[0] += sum_{s>0} part[s] over the upper-triangle entries (fixed order)
__global__ void basis_reduce_kernel(float2* __restrict__ part, int nsplit, int nt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt * nt || (e / nt) > (e % nt)) return;
  float2 acc = part[e];
#pragma unroll 8
  for (int s = 1; s < nsplit; ++s) acc = cadd(acc, part[(size_t)s * nt * nt + e]);
  part[e] = acc;
}

size_t basis_smem_bytes(int nt, int nd_defl) {
  return ((nt <= kBasisSmemNt ? (size_t)nt * nt : 0) + 2 * (size_t)nt * nd_defl) * sizeof(float2);
}

cudaError_t launch_basis(const lcf_plan* P, const float2* iq, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  int ntile = (P->nt + BG_T - 1) / BG_T;
  dim3 grid(ntile * (ntile + 1) / 2, P->basis_nsplit);
  global_gram_kernel<<<grid, 256, 0, st>>>(iq, c.nz, c.nx, P->nt, basis_zstep(c.nz), ntile, P->basis_nsplit,
                                           P->ws.gglob);
  cudaError_t e = counted(P);
  if (e != cudaSuccess) return e;
  if (P->basis_nsplit > 1) {
    basis_reduce_kernel<<<(P->nt * P->nt + 255) / 256, 256, 0, st>>>(P->ws.gglob, P->basis_nsplit, P->nt);
    e = counted(P);
    if (e != cudaSuccess) return e;
  }
  basis_kernel<<<1, 256, basis_smem_bytes(P->nt, P->ndefl), st>>>(P->ws.gglob, 1, P->nt, P->ndefl, P->ws.phi,
                                                                 P->ws.xmax);
  return counted(P);
}

cudaError_t basis_configure() {
  return cudaFuncSetAttribute(basis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)basis_smem_bytes(kBasisSmemNt, kDeflateMax));
}

}  // namespace lcf
