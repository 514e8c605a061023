// k_project_simt.cu — fused projection, |.|^2 slow-time reduction and blend
// on CUDA cores (plain FP32 path), plus the validation-only Eq. 4
// reconstruction of one subset.
//
// Because V is unitary,
//   mean_t |(C_w V diag(wt) V^H)(p,t)|^2 = (1/Nt) sum_i wt_i^2 |(C_w V)(p,i)|^2
// and (C_w V)(p,i) = g_k(p) (s_p V)(p,i).  With W_k = V diag(wt sqrt(alpha/Nt))
// (zero-weight columns dropped) the blended image (Eq. 13) is
//   PD(p) = sum_k g_k(p)^2 sum_c |s_p W_k(:,c)|^2,
// one GEMM per window instead of the two of Eq. 4.  Each CTA owns a
// 64-pixel row segment, loops over the windows whose support covers it and
// writes its pixels once (no atomics, fixed window order).
#include "lcf_internal.cuh"

namespace lcf {

template <int CPT>
__global__ void __launch_bounds__(256)
project_simt_kernel(const float2* __restrict__ iq, int nz, int nx, int nt, int nd,
                    const Box* __restrict__ boxes, const float* __restrict__ gz,
                    const float* __restrict__ gx, const float2* __restrict__ W,
                    const int* __restrict__ ncol, int ncp, float* __restrict__ out) {
  extern __shared__ float2 sm[];
  float2* Ss = sm;              // [nt][64]
  float2* Ws = sm + nt * 64;    // [nt][ncp]
  __shared__ float red[4][64];
  const int z = blockIdx.y, xb = blockIdx.x * 64;
  const int tid = threadIdx.x, pix = tid & 63, cg = tid >> 6;
  const int x = xb + pix;
  const size_t npix = (size_t)nz * nx;
  for (int e = tid; e < nt * 64; e += 256) {
    int t = e >> 6, pp = e & 63, xx = xb + pp;
    Ss[e] = xx < nx ? iq[t * npix + (size_t)z * nx + xx] : make_float2(0.f, 0.f);
  }
  float pd = 0.f;
  for (int k = 0; k < nd; ++k) {
    const Box b = boxes[k];
    if (z < b.z0 || z >= b.z1 || xb + 63 < b.x0 || xb >= b.x1) continue;
    const int nc = ncol[k];
    if (nc == 0) continue;
    __syncthreads();
    const float2* Wk = W + (size_t)k * nt * ncp;
    for (int e = tid; e < nt * ncp; e += 256) Ws[e] = Wk[e];
    __syncthreads();
    float2 y[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) y[c] = make_float2(0.f, 0.f);
    const float2* wcol = Ws + cg * CPT;
    for (int t = 0; t < nt; ++t) {
      float2 s = Ss[t * 64 + pix];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        float2 w = wcol[t * ncp + c];
        y[c].x = fmaf(s.x, w.x, fmaf(-s.y, w.y, y[c].x));
        y[c].y = fmaf(s.x, w.y, fmaf(s.y, w.x, y[c].y));
      }
    }
    float part = 0.f;
#pragma unroll
    for (int c = 0; c < CPT; ++c) part += y[c].x * y[c].x + y[c].y * y[c].y;
    red[cg][pix] = part;
    __syncthreads();
    if (cg == 0) {
      float g = (x < nx) ? gz[(size_t)k * nz + z] * gx[(size_t)k * nx + x] : 0.f;
      pd += g * g * ((red[0][pix] + red[1][pix]) + (red[2][pix] + red[3][pix]));
    }
  }
  if (cg == 0 && x < nx) out[(size_t)z * nx + x] = pd;
}

// Packets longer than 128 frames: 32-pixel row segments, the window's weights
// streamed through shared memory in blocks of 64 rows x 128 columns (eight
// groups of 16 columns per pixel), |.|^2 summed over the column blocks.
// The rows are the deflated packet of the Gram stage, s_p = c_p + sum_j a_pj phi_j,
// so s_p W = [c_p, a_p] [W ; Phi^T W]: the large clutter coefficients a_p meet the
// small Phi^T W (formed with double-float sums) and the residual c_p meets W, so
// the FP32 sums never cancel the clutter against itself.
__global__ void __launch_bounds__(256)
project_simt_long_kernel(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl, int nd,
                         const Box* __restrict__ boxes, const float* __restrict__ gz,
                         const float* __restrict__ gx, const float2* __restrict__ W,
                         const float2* __restrict__ PW, const int* __restrict__ ncol, int ncp,
                         float* __restrict__ out) {
  extern __shared__ float2 sm[];
  const int nk = nt + nd_defl;
  float2* Ss = sm;              // [nk][32]
  float2* Wc = sm + nk * 32;    // [64][128]
  __shared__ float red[8][32];
  const int z = blockIdx.y, xb = blockIdx.x * 32;
  const int tid = threadIdx.x, pix = tid & 31, cg = tid >> 5;
  const int x = xb + pix;
  const size_t npix = (size_t)nz * nx;
  for (int e = tid; e < nk * 32; e += 256) {
    const int t = e >> 5, pp = e & 31, xx = xb + pp;
    Ss[e] = xx < nx ? xa[t * npix + (size_t)z * nx + xx] : make_float2(0.f, 0.f);
  }
  float pd = 0.f;
  for (int k = 0; k < nd; ++k) {
    const Box b = boxes[k];
    if (z < b.z0 || z >= b.z1 || xb + 31 < b.x0 || xb >= b.x1) continue;
    const int nc = ncol[k];
    if (nc == 0) continue;
    const float2* Wk = W + (size_t)k * nt * ncp;
    const float2* PWk = PW + (size_t)k * kDeflateMax * ncp;
    float part = 0.f;
    for (int c0 = 0; c0 < nc; c0 += 128) {
      float2 y[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) y[c] = make_float2(0.f, 0.f);
      for (int t0 = 0; t0 < nk; t0 += 64) {
        __syncthreads();
        for (int e = tid; e < 64 * 128; e += 256) {
          const int tt = t0 + (e >> 7), cc = c0 + (e & 127);
          float2 w = make_float2(0.f, 0.f);
          if (cc < nc) {
            if (tt < nt) w = Wk[(size_t)tt * ncp + cc];
            else if (tt < nk) w = PWk[(size_t)(tt - nt) * ncp + cc];
          }
          Wc[e] = w;
        }
        __syncthreads();
        const int tn = nk - t0 < 64 ? nk - t0 : 64;
        const float2* wrow = Wc + cg * 16;
        for (int tt = 0; tt < tn; ++tt) {
          const float2 sv = Ss[(t0 + tt) * 32 + pix];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const float2 w = wrow[tt * 128 + c];
            y[c].x = fmaf(sv.x, w.x, fmaf(-sv.y, w.y, y[c].x));
            y[c].y = fmaf(sv.x, w.y, fmaf(sv.y, w.x, y[c].y));
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) part += y[c].x * y[c].x + y[c].y * y[c].y;
    }
    __syncthreads();
    red[cg][pix] = part;
    __syncthreads();
    if (cg == 0) {
      const float g = (x < nx) ? gz[(size_t)k * nz + z] * gx[(size_t)k * nx + x] : 0.f;
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) acc += red[q][pix];
      pd += g * g * acc;
    }
  }
  if (cg == 0 && x < nx) out[(size_t)z * nx + x] = pd;
}

size_t project_long_smem_bytes(int nt) { return (size_t)(nt + kDeflateMax) * 32 * 8 + 64 * 128 * 8; }

// Phi^T W of every window for the long-packet projection: PW[k][j][c] = sum_t phi_j(t) W_k(t, c)
// in double-float, one CTA per window.
__global__ void __launch_bounds__(256)
project_pw_kernel(const float2* __restrict__ W, const int* __restrict__ ncol, const float2* __restrict__ phi,
                  int nt, int nd_defl, int ncp, float2* __restrict__ PW) {
  const int k = blockIdx.x, nc = ncol[k];
  const float2* Wk = W + (size_t)k * nt * ncp;
  for (int e = threadIdx.x; e < kDeflateMax * ncp; e += blockDim.x) {
    const int j = e / ncp, c = e % ncp;
    float2 v = make_float2(0.f, 0.f);
    if (j < nd_defl && c < nc) {
      df sr = {0.f, 0.f}, si = {0.f, 0.f};
      for (int t = 0; t < nt; ++t) {
        const float2 f = phi[j * nt + t], w = Wk[(size_t)t * ncp + c];
        sr = df_add(sr, df_add(two_prod_df(f.x, w.x), df_neg(two_prod_df(f.y, w.y))));
        si = df_add(si, df_add(two_prod_df(f.x, w.y), two_prod_df(f.y, w.x)));
      }
      v = make_float2(sr.hi + sr.lo, si.hi + si.lo);
    }
    PW[(size_t)k * kDeflateMax * ncp + e] = v;
  }
}

int project_cpt(int nt) { return nt <= 32 ? 8 : (nt <= 64 ? 16 : (nt <= 112 ? 28 : 32)); }

size_t project_smem_bytes(int nt, int ncp) { return (size_t)nt * 64 * 8 + (size_t)nt * ncp * 8; }

cudaError_t launch_project_simt(const lcf_plan* P, const float2* iq, float* out, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  if (P->nt > kProjectShortNmax) {
    project_pw_kernel<<<P->nd, 256, 0, st>>>(P->ws.W, P->ws.ncol, P->ws.phi, P->nt, P->ndefl, P->ncp, P->ws.pw);
    cudaError_t e = counted(P);
    if (e != cudaSuccess) return e;
    dim3 g2((c.nx + 31) / 32, c.nz);
    project_simt_long_kernel<<<g2, 256, project_long_smem_bytes(P->nt), st>>>(
        P->ws.xa, c.nz, c.nx, P->nt, P->ndefl, P->nd, P->ws.box, P->ws.gz, P->ws.gx, P->ws.W, P->ws.pw,
        P->ws.ncol, P->ncp, out);
    return counted(P);
  }
  dim3 grid((c.nx + 63) / 64, c.nz);
  size_t sm = project_smem_bytes(P->nt, P->ncp);
  int cpt = project_cpt(P->nt);
  if (cpt == 8)
    project_simt_kernel<8><<<grid, 256, sm, st>>>(iq, c.nz, c.nx, P->nt, P->nd, P->ws.box, P->ws.gz,
                                                  P->ws.gx, P->ws.W, P->ws.ncol, P->ncp, out);
  else if (cpt == 16)
    project_simt_kernel<16><<<grid, 256, sm, st>>>(iq, c.nz, c.nx, P->nt, P->nd, P->ws.box, P->ws.gz,
                                                   P->ws.gx, P->ws.W, P->ws.ncol, P->ncp, out);
  else if (cpt == 28)
    project_simt_kernel<28><<<grid, 256, sm, st>>>(iq, c.nz, c.nx, P->nt, P->nd, P->ws.box, P->ws.gz,
                                                   P->ws.gx, P->ws.W, P->ws.ncol, P->ncp, out);
  else
    project_simt_kernel<32><<<grid, 256, sm, st>>>(iq, c.nz, c.nx, P->nt, P->nd, P->ws.box, P->ws.gz,
                                                   P->ws.gx, P->ws.W, P->ws.ncol, P->ncp, out);
  return counted(P);
}

cudaError_t project_configure() {
  size_t mx = project_smem_bytes(kProjectShortNmax, 4 * project_cpt(kProjectShortNmax));
  cudaError_t e = cudaFuncSetAttribute(project_simt_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(project_simt_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(project_simt_kernel<28>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(project_simt_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(project_simt_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)project_long_smem_bytes(kEvdNmax));
  return e;
}

// ---- validation: C-hat = C_w V diag(wt) V^H of one subset (Eq. 4) ----
__global__ void filtered_iq_kernel(const float2* __restrict__ iq, int nz, int nx, int nt, Box b,
                                   const float* __restrict__ gzk, const float* __restrict__ gxk,
                                   const float2* __restrict__ V, const float* __restrict__ wt,
                                   float2* __restrict__ out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  size_t npix = (size_t)nz * nx;
  if (p >= (int)npix) return;
  int z = p / nx, x = p % nx;
  if (z < b.z0 || z >= b.z1 || x < b.x0 || x >= b.x1) {
    for (int t = 0; t < nt; ++t) out[t * npix + p] = make_float2(0.f, 0.f);
    return;
  }
  float g = gzk[z] * gxk[x];
  float2 y[kEvdNmax];
  for (int i = 0; i < nt; ++i) {
    float2 acc = make_float2(0.f, 0.f);
    for (int t = 0; t < nt; ++t) acc = cadd(acc, cmul(iq[t * npix + p], V[t * nt + i]));
    y[i] = cscale(acc, g * wt[i]);
  }
  for (int t = 0; t < nt; ++t) {
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < nt; ++i) acc = cadd(acc, cmul(y[i], cconj(V[t * nt + i])));
    out[t * npix + p] = acc;
  }
}

cudaError_t launch_filtered_iq(const lcf_plan* P, const float2* iq, int k, float2* out, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  int npix = c.nz * c.nx;
  filtered_iq_kernel<<<(npix + 127) / 128, 128, 0, st>>>(
      iq, c.nz, c.nx, P->nt, P->boxes[k], P->ws.gz + (size_t)k * c.nz, P->ws.gx + (size_t)k * c.nx,
      P->ws.V + (size_t)k * P->nt * P->nt, P->ws.wt + (size_t)k * P->nt, out);
  return counted(P);
}

}  // namespace lcf
