// k_post.cu — work that follows the EVD kernels for two options, then the
// thresholding rule, alpha (Eq. 13) and the projection weights W written the
// way the EVD kernels write them:
//
//  * LCF_EP_FP64_POLISH (Eq. 2 in extended precision): every eigenvalue is
//    replaced by the Rayleigh quotient v^H R v / v^H v of its FP32 eigenvector
//    against the FP64 Gram R, formed in double-float on the FP32 pipes; the
//    eigenpairs are re-sorted.  A Rayleigh quotient's error is second order in
//    the eigenvector's error, so eigenvalues far below u * lambda_1 (the FP32
//    Jacobi's absolute resolution) come out with relative accuracy.
//
//  * Method 4 (Eq. 8) and method 5 (Eq. 9) at method 4's cutoff: the cutoff
//    minimising the normalised cross-correlation of the tissue image
//    I_T(k) = sum_{i=k-fn+1..k} |u_i| and the blood image I_B(k) =
//    sum_{i=k+1..k+fn} |u_i|, |u_i(p)| = |(C_w v_i)(p)| / sigma_i.  Every sum the
//    rule needs is a band entry M_ij = sum_p |u_i(p)| |u_j(p)|, |i - j| < 2 fn,
//    of the magnitude Gram, so one pass over the window's pixels (the
//    projection's GEMM with all Nt columns, then band products of the
//    magnitudes) gives NCC(k) for every k.
#include <math.h>

#include "evd_common.cuh"
#include "lcf_internal.cuh"

namespace lcf {

constexpr int PR_ROWS = 16;        // Gram rows per Rayleigh-quotient CTA
constexpr int PS_THREADS = 256;    // post kernel
constexpr int NCC_FN = 5;          // neighbours on each side of the cutoff (the paper's fn)
constexpr int NCC_NB = 2 * NCC_FN; // band width of the magnitude Gram
constexpr int NB_THREADS = 256;    // band kernel: 32 pixels x 8 groups of 16 columns
constexpr int NB_PX = 32;
constexpr int NB_ROWS = 64;        // weight rows staged per step
constexpr int NB_COLS = 128;       // weight columns per chunk

__host__ __device__ inline int ncc_fn(int n) { return n / 2 < NCC_FN ? n / 2 : NCC_FN; }

// a += r * v for a double-float accumulator whose low word collects the rounding errors
// (renormalised once at the end): FMA two-product of the high word, the low word's product,
// a two-sum on the high words
__device__ __forceinline__ void dacc(df& a, const float rh, const float rl, const float v) {
  const float p = rh * v;
  float e = fmaf(rh, v, -p);
  e = fmaf(rl, v, e);
  const float s = a.hi + p;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (p - bb);
  a.hi = s;
  a.lo += err + e;
}

// exponent e of a power-of-two scale 2^-e bringing the window's largest diagonal entry of R
// below 1 (so the double-float words stay inside the FP32 range); 0 for a zero Gram.
// red: one double per warp of the block.
__device__ inline int post_scale_exp(const double2* Rk, int n, double* red) {
  const int tid = threadIdx.x, nw = (blockDim.x + 31) >> 5;
  double mx = 0.0;
  for (int i = tid; i < n; i += blockDim.x) mx = fmax(mx, fabs(Rk[(size_t)i * n + i].x));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(~0u, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);
  return e;
}

// ---------------------------------------------------------------------------
// Rayleigh-quotient partials: q[k][b][i] = sum_{j in rows of block b} conj(V_ji) (R V)_ji,
// thread i = column i; the block's PR_ROWS rows of R (scaled by 2^-e) live in shared memory
// as double-float pairs, V is read from global memory (coalesced along i).
__global__ void __launch_bounds__(320)
polish_rq_kernel(const double2* __restrict__ R, const float2* __restrict__ V, int n, double* __restrict__ part) {
  extern __shared__ float4 rs[];   // [PR_ROWS][n]: (re.hi, re.lo, im.hi, im.lo)
  __shared__ double red[10];
  const int k = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
  const int j0 = b * PR_ROWS, nr = min(PR_ROWS, n - j0);
  const double2* Rk = R + (size_t)k * n * n;
  const float2* Vk = V + (size_t)k * n * n;
  const int e = post_scale_exp(Rk, n, red);
  const double sc = e == 0 ? 0.0 : ldexp(1.0, -e);
  for (int x = tid; x < PR_ROWS * n; x += blockDim.x) {
    const int r = x / n, l = x - r * n;
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < nr) {
      const double2 v = Rk[(size_t)(j0 + r) * n + l];
      const double xr = v.x * sc, xi = v.y * sc;
      const float hr = (float)xr, hi = (float)xi;
      w = make_float4(hr, (float)(xr - (double)hr), hi, (float)(xi - (double)hi));
    }
    rs[x] = w;
  }
  __syncthreads();
  const int i = tid;
  if (i >= n) return;
  df yr[PR_ROWS], yi[PR_ROWS];
#pragma unroll
  for (int r = 0; r < PR_ROWS; ++r) { yr[r] = {0.f, 0.f}; yi[r] = {0.f, 0.f}; }
  for (int l = 0; l < n; ++l) {
    const float2 v = Vk[(size_t)l * n + i];
#pragma unroll
    for (int r = 0; r < PR_ROWS; ++r) {
      const float4 a = rs[r * n + l];   // one address for the whole warp: a broadcast
      dacc(yr[r], a.x, a.y, v.x);
      dacc(yr[r], a.z, a.w, -v.y);
      dacc(yi[r], a.x, a.y, v.y);
      dacc(yi[r], a.z, a.w, v.x);
    }
  }
  df q = {0.f, 0.f};
#pragma unroll
  for (int r = 0; r < PR_ROWS; ++r) {
    if (r < nr) {
      const float2 vj = Vk[(size_t)(j0 + r) * n + i];
      const df a = quick_two_sum(yr[r].hi, yr[r].lo), c = quick_two_sum(yi[r].hi, yi[r].lo);
      dacc(q, a.hi, a.lo, vj.x);   // Re(conj(v_j) y_j) = v_j.x y.re + v_j.y y.im
      dacc(q, c.hi, c.lo, vj.y);
    }
  }
  part[((size_t)k * gridDim.x + b) * n + i] = ldexp((double)q.hi + (double)q.lo, e);
}

// ---------------------------------------------------------------------------
// Method 4 inputs per window: PV = Phi^T V (double-float sums) so that s_p V = c_p V + a_p PV
// for the deflated rows, and 1/sigma_i = 1/sqrt(lambda~_i).
__global__ void __launch_bounds__(256)
ncc_prep_kernel(const float2* __restrict__ V, const double* __restrict__ lam, const float2* __restrict__ phi, int n,
                int nd_defl, float2* __restrict__ pv, float* __restrict__ isig) {
  const int k = blockIdx.x;
  const float2* Vk = V + (size_t)k * n * n;
  const double* lk = lam + (size_t)k * n;
  const double fl = lk[0] * n * 2.220446049250313e-16;
  for (int e = threadIdx.x; e < nd_defl * n; e += blockDim.x) {
    const int j = e / n, c = e - j * n;
    df sr = {0.f, 0.f}, si = {0.f, 0.f};
    for (int t = 0; t < n; ++t) {   // phi_j(t) v_c(t), complex
      const float2 f = phi[(size_t)j * n + t], v = Vk[(size_t)t * n + c];
      sr = df_add(sr, df_add(two_prod_df(f.x, v.x), df_neg(two_prod_df(f.y, v.y))));
      si = df_add(si, df_add(two_prod_df(f.x, v.y), two_prod_df(f.y, v.x)));
    }
    pv[((size_t)k * kDeflateMax + j) * n + c] = make_float2(sr.hi + sr.lo, si.hi + si.lo);
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double l = lk[c] > fl ? lk[c] : fl;
    isig[(size_t)k * n + c] = l > 0.0 ? (float)(1.0 / sqrt(l)) : 0.f;
  }
}

// Band sums of the magnitude Gram of window k over the pixels of split s of its support:
// part[k][s][i][d] = sum_p m_i(p) m_{i+d}(p), d < NCC_NB, m_i(p) = |g(p) (s_p V)_i| / sigma_i.
// Rows of s_p are the deflated packet (residual rows, then coefficient rows) against [V ; PV].
size_t ncc_band_smem_bytes(int n, int nd_defl) {
  return (size_t)(n + nd_defl) * NB_PX * sizeof(float2) + (size_t)NB_ROWS * NB_COLS * sizeof(float2) +
         (size_t)NB_PX * (n + 1) * sizeof(float);
}

__global__ void __launch_bounds__(NB_THREADS, 1)
ncc_band_kernel(const float2* __restrict__ xa, int nz, int nx, int n, int nd_defl, const Box* __restrict__ boxes,
                const float* __restrict__ gz, const float* __restrict__ gx, const float2* __restrict__ V,
                const float2* __restrict__ pv, const float* __restrict__ isig, int nsplit, double* __restrict__ part) {
  extern __shared__ float2 nsm[];
  const int nk = n + nd_defl, ldm = n + 1;
  float2* Ss = nsm;                                   // [nk][NB_PX]
  float2* Wc = Ss + (size_t)nk * NB_PX;               // [NB_ROWS][NB_COLS]
  float* mS = reinterpret_cast<float*>(Wc + NB_ROWS * NB_COLS);   // [NB_PX][n + 1]
  const int k = blockIdx.y, s = blockIdx.x, tid = threadIdx.x;
  const int pix = tid & 31, cg = tid >> 5;
  const Box b = boxes[k];
  const int W = b.x1 - b.x0;
  const long Pk = (long)(b.z1 - b.z0) * W;
  const long l0 = Pk * s / nsplit, l1 = Pk * (s + 1) / nsplit;
  const size_t npix = (size_t)nz * nx;
  const float2* Vk = V + (size_t)k * n * n;
  const float2* PVk = pv + (size_t)k * kDeflateMax * n;
  const float* isk = isig + (size_t)k * n;
  constexpr int BPT = (kEvdNmax * NCC_NB + NB_THREADS - 1) / NB_THREADS;   // band entries per thread
  double bacc[BPT];
#pragma unroll
  for (int u = 0; u < BPT; ++u) bacc[u] = 0.0;
  for (long lb = l0; lb < l1; lb += NB_PX) {
    __syncthreads();
    {   // this batch's deflated rows, weighted by g (zero past the range)
      const long l = lb + pix;
      float g = 0.f;
      size_t p = 0;
      if (l < l1) {
        const int zr = (int)(l / W), z = b.z0 + zr, x = b.x0 + (int)(l - (long)zr * W);
        p = (size_t)z * nx + x;
        g = gz[(size_t)k * nz + z] * gx[(size_t)k * nx + x];
      }
      for (int t = cg; t < nk; t += NB_THREADS / 32) {
        const float2 v = g != 0.f ? xa[(size_t)t * npix + p] : make_float2(0.f, 0.f);
        Ss[t * NB_PX + pix] = make_float2(g * v.x, g * v.y);
      }
    }
    for (int c0 = 0; c0 < n; c0 += NB_COLS) {
      float2 y[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) y[c] = make_float2(0.f, 0.f);
      for (int t0 = 0; t0 < nk; t0 += NB_ROWS) {
        __syncthreads();
        for (int e = tid; e < NB_ROWS * NB_COLS; e += NB_THREADS) {
          const int tt = t0 + e / NB_COLS, cc = c0 + e % NB_COLS;
          float2 w = make_float2(0.f, 0.f);
          if (cc < n) {
            if (tt < n) w = Vk[(size_t)tt * n + cc];
            else if (tt < nk) w = PVk[(size_t)(tt - n) * n + cc];
          }
          Wc[e] = w;
        }
        __syncthreads();
        const int tn = nk - t0 < NB_ROWS ? nk - t0 : NB_ROWS;
        const float2* wrow = Wc + cg * 16;
        for (int tt = 0; tt < tn; ++tt) {
          const float2 sv = Ss[(t0 + tt) * NB_PX + pix];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const float2 w = wrow[tt * NB_COLS + c];
            y[c].x = fmaf(sv.x, w.x, fmaf(-sv.y, w.y, y[c].x));
            y[c].y = fmaf(sv.x, w.y, fmaf(sv.y, w.x, y[c].y));
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = c0 + cg * 16 + c;
        if (col < n) mS[pix * ldm + col] = sqrtf(y[c].x * y[c].x + y[c].y * y[c].y) * isk[col];
      }
    }
    __syncthreads();
    // band products of this batch's magnitudes (FP32 over 32 pixels, then double)
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int e = tid + u * NB_THREADS;
      const int c = e / NCC_NB, d = e - c * NCC_NB;
      if (c + d < n) {
        float acc = 0.f;
        for (int q = 0; q < NB_PX; ++q) acc = fmaf(mS[q * ldm + c], mS[q * ldm + c + d], acc);
        bacc[u] += (double)acc;
      }
    }
  }
  double* out = part + ((size_t)k * nsplit + s) * (size_t)n * NCC_NB;
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int e = tid + u * NB_THREADS;
    if (e < n * NCC_NB) out[e] = bacc[u];
  }
}

// ---------------------------------------------------------------------------
struct PostArgs {
  int nt, nz, nx, ncp;
  int thresh_mode, k_src, k_fixed, pd_mode, alpha_mode, curv_norm;
  double beta, beta_src;
  int do_sort;                 // polished eigenvalues: re-sort the eigenpairs
  int do_rule;                 // rule, alpha and W
  int rq_blocks;               // Rayleigh-quotient partials per window
  const double* rq;            // [nd][rq_blocks][nt]
  int ncc_splits;              // band-sum partials per window (0: the rule needs none)
  const double* band;          // [nd][ncc_splits][nt][NCC_NB]
};

size_t post_smem_bytes(int n) {
  return (size_t)n * 8 * 6 + (size_t)n * NCC_NB * 8 + (size_t)(PS_THREADS / 32) * n * sizeof(float2) +
         (size_t)(n + 1) * 4 * 2 + (size_t)n * 4 + 64;
}

// NCC(k) for a 1-based cutoff from the band sums (sorted order)
__device__ inline double ncc_at(const double* band, int n, int fn, int k) {
  double num = 0.0, dt = 0.0, db = 0.0;
  for (int i = k - fn; i < k; ++i)
    for (int j = k; j < k + fn; ++j) num += band[(size_t)i * NCC_NB + (j - i)];
  for (int i = k - fn; i < k; ++i)
    for (int j = k - fn; j < k; ++j) dt += i <= j ? band[(size_t)i * NCC_NB + (j - i)] : band[(size_t)j * NCC_NB + (i - j)];
  for (int i = k; i < k + fn; ++i)
    for (int j = k; j < k + fn; ++j) db += i <= j ? band[(size_t)i * NCC_NB + (j - i)] : band[(size_t)j * NCC_NB + (i - j)];
  const double den = sqrt(dt) * sqrt(db);
  return den > 0.0 ? num / den : 1.0;
}

__global__ void __launch_bounds__(PS_THREADS)
evd_post_kernel(PostArgs g, const Box* __restrict__ boxes, double* __restrict__ lam, float2* __restrict__ V,
                float* __restrict__ wt_out, int* __restrict__ kcut_out, float* __restrict__ alpha_out,
                int* __restrict__ flags, float2* __restrict__ W_out, int* __restrict__ ncol_out) {
  extern __shared__ double psm[];
  const int n = g.nt, k = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* lam_s = psm;               // [n] sorted eigenvalues
  double* lamn = lam_s + n;          // [n] polished, in the EVD's order
  double* wts = lamn + n;            // [n]
  double* s0 = wts + n;              // rule scratch [n] x 3
  double* s1 = s0 + n;
  double* s2 = s1 + n;
  double* band = s2 + n;             // [n][NCC_NB]
  float2* vrow = reinterpret_cast<float2*>(band + (size_t)n * NCC_NB);   // [8][n]
  int* perm = reinterpret_cast<int*>(vrow + (size_t)(PS_THREADS / 32) * n);   // [n]
  int* keep = perm + n;              // [n + 1]: count, then kept sorted indices
  float* coef = reinterpret_cast<float*>(keep + n + 1);   // [n]
  double* lk = lam + (size_t)k * n;
  float2* Vk = V + (size_t)k * n * n;

  if (g.do_sort) {
    for (int i = tid; i < n; i += PS_THREADS) {
      double q = 0.0, nrm = 0.0;
      for (int b = 0; b < g.rq_blocks; ++b) q += g.rq[((size_t)k * g.rq_blocks + b) * n + i];
      for (int t = 0; t < n; ++t) {
        const float2 v = Vk[(size_t)t * n + i];
        nrm += (double)v.x * v.x + (double)v.y * v.y;
      }
      lamn[i] = nrm > 0.0 ? q / nrm : 0.0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += PS_THREADS) {   // stable descending rank
      const double di = lamn[i];
      int rk = 0;
      for (int j = 0; j < n; ++j) rk += (lamn[j] > di) || (lamn[j] == di && j < i);
      perm[rk] = i;
    }
    __syncthreads();
    for (int i = tid; i < n; i += PS_THREADS) lam_s[i] = lamn[perm[i]];
    // eigenvector columns into the new order, one row per warp
    float2* vr = vrow + (size_t)warp * n;
    for (int t = warp; t < n; t += PS_THREADS / 32) {
      for (int c = lane; c < n; c += 32) vr[c] = Vk[(size_t)t * n + c];
      __syncwarp();
      for (int c = lane; c < n; c += 32) Vk[(size_t)t * n + c] = vr[perm[c]];
      __syncwarp();
    }
    __syncthreads();
    for (int i = tid; i < n; i += PS_THREADS) lk[i] = lam_s[i];
  } else {
    for (int i = tid; i < n; i += PS_THREADS) lam_s[i] = lk[i];
  }
  if (!g.do_rule) return;
  const bool ncc = g.ncc_splits > 0;
  if (ncc) {
    for (int e = tid; e < n * NCC_NB; e += PS_THREADS) {
      double v = 0.0;
      for (int s = 0; s < g.ncc_splits; ++s) v += g.band[((size_t)k * g.ncc_splits + s) * n * NCC_NB + e];
      band[e] = v;
    }
  }
  __syncthreads();
  if (warp == 0) {
    int kk = -1;
    const int md = g.thresh_mode;
    auto ncc_k = [&]() {
      const int fn = ncc_fn(n);
      if (fn < 1) return 0;
      double best = INFINITY;
      int bi = 0x7fffffff;
      for (int kc = fn + lane; kc <= n - fn; kc += 32) {
        const double v = ncc_at(band, n, fn, kc);
        if (v < best) { best = v; bi = kc; }
      }
      for (int o = 16; o; o >>= 1) {   // minimum, ties to the smallest cutoff
        const double ob = __shfl_xor_sync(~0u, best, o);
        const int oi = __shfl_xor_sync(~0u, bi, o);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      return bi == 0x7fffffff ? fn : bi;
    };
    if (md == LCF_T_NONE) {
      for (int i = lane; i < n; i += 32) wts[i] = 1.0;
      kk = 0;
    } else if (md == LCF_T_NCC) {
      kk = ncc_k();
      for (int i = lane; i < n; i += 32) wts[i] = (i + 1 > kk) ? 1.0 : 0.0;
    } else if (md <= LCF_T_MEDIAN) {
      kk = ep_rule_k(md, lam_s, n, g.beta, g.k_fixed, g.curv_norm, s0, s1, s2, lane);
      for (int i = lane; i < n; i += 32) wts[i] = (i + 1 > kk) ? 1.0 : 0.0;
    } else if (md == LCF_T_SIGMOID) {
      kk = g.k_src == LCF_T_NCC ? ncc_k() : ep_rule_k(g.k_src, lam_s, n, g.beta_src, g.k_fixed, g.curv_norm, s0, s1, s2, lane);
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
      int fl = flags[k] & (LCF_WFLAG_NOCONV | (255 << LCF_WFLAG_SWEEP_SHIFT));
      if (g.alpha_mode == 1) al = 1.0;
      else {
        const Box bx = boxes[k];
        const double cnt = g.alpha_mode == 2 ? (double)(bx.z1 - bx.z0) * (bx.x1 - bx.x0) : (double)g.nz * g.nx;
        if (pdsum <= 1e-300) { al = 0.0; fl |= LCF_WFLAG_DEGENERATE; }
        else al = cnt / pdsum;
      }
      kcut_out[k] = kk;
      alpha_out[k] = (float)al;
      flags[k] = fl;
      cf = sqrt(al * (g.pd_mode == 0 ? 1.0 / n : 1.0));
    }
    cf = __shfl_sync(~0u, cf, 0);
    int base = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {   // kept columns in sorted order (ballot prefix)
      const int i = i0 + lane;
      const bool kp = i < n && wts[i] > 0.0;
      const unsigned bal = __ballot_sync(~0u, kp);
      if (kp) keep[1 + base + __popc(bal & ((1u << lane) - 1u))] = i;
      if (i < n) coef[i] = (float)(wts[i] * cf);
      base += __popc(bal);
    }
    if (lane == 0) {
      keep[0] = base;
      ncol_out[k] = base;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += PS_THREADS) wt_out[(size_t)k * n + i] = (float)wts[i];
  const int nc = keep[0];
  for (int e = tid; e < n * g.ncp; e += PS_THREADS) {
    const int t = e / g.ncp, c = e - t * g.ncp;
    float2 v = make_float2(0.f, 0.f);
    if (c < nc) {
      const int j = keep[1 + c];
      v = cscale(Vk[(size_t)t * n + j], coef[j]);
    }
    W_out[(size_t)k * n * g.ncp + e] = v;
  }
}

// ---------------------------------------------------------------------------
bool post_uses_ncc(const lcf_config& c) {
  return c.thresh_mode == LCF_T_NCC || (c.thresh_mode == LCF_T_SIGMOID && c.k_src == LCF_T_NCC);
}

int post_rq_blocks(int nt) { return (nt + PR_ROWS - 1) / PR_ROWS; }
size_t post_band_count(const lcf_plan* P) { return (size_t)P->nd * P->ncc_nsplit * P->nt * NCC_NB; }

cudaError_t post_configure() {
  cudaError_t e = cudaFuncSetAttribute(polish_rq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(PR_ROWS * kEvdNmax * sizeof(float4)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ncc_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ncc_band_smem_bytes(kEvdNmax, kDeflateMax));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(evd_post_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)post_smem_bytes(kEvdNmax));
  return e;
}

// After the EVD kernel: the polish and/or method 4's band sums, then the rule and W.
cudaError_t launch_post(const lcf_plan* P, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  const bool polish = c.evd_precision == LCF_EP_FP64_POLISH, ncc = post_uses_ncc(c);
  if (!polish && !ncc) return cudaSuccess;
  const int n = P->nt;
  PostArgs a;
  a.nt = n; a.nz = c.nz; a.nx = c.nx; a.ncp = P->ncp;
  a.thresh_mode = c.thresh_mode; a.k_src = c.k_src; a.k_fixed = c.k_fixed; a.pd_mode = c.pd_mode;
  a.alpha_mode = c.alpha_mode; a.curv_norm = c.curv_norm; a.beta = c.beta; a.beta_src = c.beta_src;
  a.rq_blocks = post_rq_blocks(n);
  a.rq = P->ws.post_rq;
  a.ncc_splits = 0;
  a.band = P->ws.post_band;
  cudaError_t e;
  if (polish) {
    const int thr = (n + 31) / 32 * 32;
    polish_rq_kernel<<<dim3(a.rq_blocks, P->nd), thr, PR_ROWS * n * sizeof(float4), st>>>(P->ws.R, P->ws.V, n,
                                                                                            P->ws.post_rq);
    if ((e = counted(P)) != cudaSuccess) return e;
    a.do_sort = 1;
    a.do_rule = ncc ? 0 : 1;
    evd_post_kernel<<<P->nd, PS_THREADS, post_smem_bytes(n), st>>>(a, P->ws.box, P->ws.lam, P->ws.V, P->ws.wt,
                                                                   P->ws.kcut, P->ws.alpha, P->ws.flags, P->ws.W,
                                                                   P->ws.ncol);
    if ((e = counted(P)) != cudaSuccess) return e;
  }
  if (ncc) {
    ncc_prep_kernel<<<P->nd, 256, 0, st>>>(P->ws.V, P->ws.lam, P->ws.phi, n, P->ndefl, P->ws.post_pv,
                                           P->ws.post_isig);
    if ((e = counted(P)) != cudaSuccess) return e;
    ncc_band_kernel<<<dim3(P->ncc_nsplit, P->nd), NB_THREADS, ncc_band_smem_bytes(n, P->ndefl), st>>>(
        P->ws.xa, c.nz, c.nx, n, P->ndefl, P->ws.box, P->ws.gz, P->ws.gx, P->ws.V, P->ws.post_pv, P->ws.post_isig,
        P->ncc_nsplit, P->ws.post_band);
    if ((e = counted(P)) != cudaSuccess) return e;
    a.do_sort = 0;
    a.do_rule = 1;
    a.ncc_splits = P->ncc_nsplit;
    evd_post_kernel<<<P->nd, PS_THREADS, post_smem_bytes(n), st>>>(a, P->ws.box, P->ws.lam, P->ws.V, P->ws.wt,
                                                                   P->ws.kcut, P->ws.alpha, P->ws.flags, P->ws.W,
                                                                   P->ws.ncol);
    if ((e = counted(P)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lcf
