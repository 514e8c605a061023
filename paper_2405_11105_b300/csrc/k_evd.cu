// k_evd.cu — batched Hermitian EVD R_k = V Lambda V^H (Eq. 2), eigen-weights
// (thresholding methods 1-3, 5, 6) and the per-window projection weights.
//
// One CTA per window, the whole matrix in shared memory (Nt <= kEvdCtaNmax).
//
// Precision plan (B300 FP64 is ~1/62 of FP32, so FP64 stays out of every
// O(Nt^3) loop):
//  A. subspace iteration in FP32 on R/max(diag R) finds the m dominant
//     (tissue) directions Y;
//  B. Householder reflectors H_0..H_{m-1} from the QR of Y define a unitary
//     Q whose first m columns span Y;
//  C. B = Q^H R Q is formed in double-float (reflectors applied two-sided to
//     R in two-FP32 arithmetic).  Congruence by a near-unitary Q changes every
//     eigenvalue only by a relative O(eps), and B is graded: the tissue
//     eigenvalues sit in the leading diagonal entries, coupled to the rest by
//     ~eps*lambda_tissue;
//  D. cyclic Jacobi in FP32 on B (parallel round-robin ordering, relative
//     test |b_pq| <= tol*sqrt(b_pp*b_qq)), V accumulated starting from Q.
//     Rounding errors are now relative to the small block's own scale, so
//     the eigenvalues far below lambda_1 keep their relative accuracy;
//  E. sort (descending, ties by position), fix each eigenvector's phase,
//     apply the thresholding rule in double precision, and fold wt and
//     alpha into the projection weights W = V diag(wt*sqrt(alpha/Nt)).
#include <math.h>

#include "lcf_internal.cuh"

namespace lcf {

constexpr int EVD_THREADS = 1024;
constexpr float JACOBI_TOL = 2.0e-6f;
constexpr int SUBSPACE_ITERS = 6;

struct EvdArgs {
  int nt, nz, nx;
  int thresh_mode;
  double beta, beta_src;
  int k_fixed, k_src;
  int pd_mode, alpha_mode, curv_norm, max_sweeps;
  int ncp;
  long long* clk;   // [nd][kEvdPhases + 1] phase-boundary SM clocks (stage profiling), or null
};

// thread 0 stamps the SM clock at phase boundary b (right after a block-wide barrier)
#define EVD_STAMP(b)                                                  \
  do {                                                                \
    if (g.clk && tid == 0) g.clk[(size_t)k * (kEvdPhases + 1) + (b)] = clock64(); \
  } while (0)

size_t evd_smem_bytes(int nt) {
  int np = nt + (nt & 1);
  int m = nt < kEvdHead ? nt : kEvdHead;
  size_t region0 = (size_t)np * (np + 1) * 16;                 // df64 B, later A + V^T (fp32, odd stride)
  size_t ys = (size_t)np * m * 8 * 2;                          // Y and Z / reflectors
  size_t small = (size_t)(np / 2) * 32 + (size_t)np * 16 + 1024;
  return region0 + ys + small;
}

// --------------------------------------------------------------------------
// thresholding rules in double precision (run by one thread)
__device__ double floor_lam(const double* lam, int n, int i) {
  double fl = lam[0] * n * 2.220446049250313e-16;
  return lam[i] > fl ? lam[i] : fl;
}
__device__ void norm_log_curve(const double* lam, int n, double beta, int literal, double* y) {
  for (int i = 0; i < n; ++i) y[i] = log10(floor_lam(lam, n, i));
  if (literal) {
    double y1 = y[0];
    for (int i = 0; i < n; ++i) y[i] = (y1 != 0.0) ? beta * y[i] / y1 * n : 0.0;
  } else {
    double y1 = y[0], yn = y[n - 1], span = y1 - yn;
    for (int i = 0; i < n; ++i) y[i] = (span > 0) ? beta * n * (y[i] - yn) / span : 0.0;
  }
}
__device__ void grad(const double* y, double* d, int n) {
  if (n == 1) { d[0] = 0; return; }
  d[0] = y[1] - y[0];
  d[n - 1] = y[n - 1] - y[n - 2];
  for (int i = 1; i < n - 1; ++i) d[i] = 0.5 * (y[i + 1] - y[i - 1]);
}
__device__ int rule_k(int mode, const double* lam, int n, double beta, int k_fixed, int literal,
                      double* s0, double* s1, double* s2) {
  switch (mode) {
    case LCF_T_FIXED: return k_fixed < 0 ? 0 : (k_fixed > n ? n : k_fixed);
    case LCF_T_CURVATURE: {
      if (n < 3) return 0;
      norm_log_curve(lam, n, beta, literal, s0);
      grad(s0, s1, n);
      grad(s1, s2, n);
      int kb = 2; double best = -1.0;
      for (int i = 1; i < n - 1; ++i) {
        double q = 1.0 + s1[i] * s1[i];
        double kap = fabs(s2[i]) / (q * sqrt(q));
        if (kap > best) { best = kap; kb = i + 1; }
      }
      return kb;
    }
    case LCF_T_SLOPE: {
      if (n < 2) return 0;
      norm_log_curve(lam, n, 1.0, literal, s0);
      grad(s0, s1, n);
      for (int i = 0; i < n; ++i) if (-s1[i] <= beta) return i;
      return n - 1;
    }
    case LCF_T_MEDIAN: {
      double med = (n & 1) ? lam[n / 2] : 0.5 * (lam[n / 2 - 1] + lam[n / 2]);
      double T = beta * med;
      int k = 0;
      for (int i = 0; i < n; ++i) k += lam[i] > T;
      return k;
    }
    default: return 0;
  }
}

// --------------------------------------------------------------------------

__global__ void __launch_bounds__(EVD_THREADS, 1)
evd_kernel(const double2* __restrict__ Rg, const Box* __restrict__ boxes, EvdArgs g,
           double* __restrict__ lam_out, float2* __restrict__ V_out, float* __restrict__ wt_out,
           int* __restrict__ kcut_out, float* __restrict__ alpha_out, int* __restrict__ flags_out,
           float2* __restrict__ W_out, int* __restrict__ ncol_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x, n = g.nt, np = n + (n & 1), h = np / 2;
  const int m = n < kEvdHead ? n : kEvdHead;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  zdf* Rdf = reinterpret_cast<zdf*>(smem);                             // np*np (phase C)
  float2* Rh = reinterpret_cast<float2*>(smem);                        // np*np (phase A)
  // phase D: A row-major and V^T (Vt[col][row]) with an odd row stride so that row and
  // column walks of the 2x2 block updates fall on distinct shared-memory banks
  const int ld = np + 1;
  float2* A = reinterpret_cast<float2*>(smem);                             // np*ld
  float2* Vt = reinterpret_cast<float2*>(smem + (size_t)np * ld * 8);      // np*ld
  float2* Ys = reinterpret_cast<float2*>(smem + (size_t)np * ld * 16);
  float2* Zs = Ys + (size_t)np * m;                                    // later: reflectors
  unsigned char* sp = reinterpret_cast<unsigned char*>(Zs + (size_t)np * m);
  int* pr_p = reinterpret_cast<int*>(sp);                sp += h * 4;
  int* pr_q = reinterpret_cast<int*>(sp);                sp += h * 4;
  int* pr_rot = reinterpret_cast<int*>(sp);              sp += h * 4;
  float* pr_c = reinterpret_cast<float*>(sp);            sp += h * 4;
  float2* pr_s = reinterpret_cast<float2*>(sp);          sp += h * 8;
  float* pr_dp = reinterpret_cast<float*>(sp);           sp += h * 4;
  float* pr_dq = reinterpret_cast<float*>(sp);           sp += h * 4;
  double* lam_s = reinterpret_cast<double*>(sp);         sp += np * 8;
  int* perm = reinterpret_cast<int*>(sp);                sp += np * 4;
  float* betas = reinterpret_cast<float*>(sp);           sp += 32 * 4;
  __shared__ double sh_scale;
  __shared__ df sh_kappa;
  __shared__ int sh_flag;
  __shared__ float2 sh_phase[kEvdCtaNmax];

  const double2* R = Rg + (size_t)k * n * n;

  // ---------------- scale and degenerate check
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, R[(size_t)i * n + i].x);
    sh_scale = mx;
    sh_flag = 0;
  }
  __syncthreads();
  const double scale = sh_scale;
  if (!(scale > 0.0) || !isfinite(scale)) {
    for (int i = tid; i < n; i += EVD_THREADS) {
      lam_out[(size_t)k * n + i] = 0.0;
      wt_out[(size_t)k * n + i] = 0.f;
    }
    for (int e = tid; e < n * n; e += EVD_THREADS) V_out[(size_t)k * n * n + e] = make_float2(e / n == e % n, 0.f);
    for (int e = tid; e < n * g.ncp; e += EVD_THREADS) W_out[(size_t)k * n * g.ncp + e] = make_float2(0.f, 0.f);
    if (tid == 0) {
      kcut_out[k] = 0; alpha_out[k] = 0.f; ncol_out[k] = 0;
      flags_out[k] = LCF_WFLAG_DEGENERATE;
    }
    return;
  }
  const double inv = 1.0 / scale;
  EVD_STAMP(0);

  // ---------------- phase A: subspace iteration on Rh = fp32(R/scale)
  for (int e = tid; e < np * np; e += EVD_THREADS) {
    int a = e / np, b = e % np;
    float2 v = make_float2(0.f, 0.f);
    if (a < n && b < n) { double2 r = R[(size_t)a * n + b]; v = make_float2((float)(r.x * inv), (float)(r.y * inv)); }
    Rh[e] = v;
  }
  for (int e = tid; e < np * m; e += EVD_THREADS) {
    int a = e / m, j = e % m;
    // deterministic, well-spread start block
    unsigned hsh = (unsigned)(a * 2654435761u) ^ (unsigned)(j * 40503u + 7u);
    hsh ^= hsh >> 13; hsh *= 0x5bd1e995u; hsh ^= hsh >> 15;
    float re = (float)(hsh & 0xffff) / 65536.f - 0.5f, im = (float)(hsh >> 16) / 65536.f - 0.5f;
    Ys[e] = (a < n) ? make_float2(re, im) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int it = 0; it < SUBSPACE_ITERS; ++it) {
    for (int e = tid; e < np * m; e += EVD_THREADS) {
      int a = e / m, j = e % m;
      float2 acc = make_float2(0.f, 0.f);
      if (a < n)
        for (int b = 0; b < n; ++b) {
          float2 r = Rh[a * np + b], y = Ys[b * m + j];
          acc.x = fmaf(r.x, y.x, fmaf(-r.y, y.y, acc.x));
          acc.y = fmaf(r.x, y.y, fmaf(r.y, y.x, acc.y));
        }
      Zs[e] = acc;
    }
    __syncthreads();
    if (warp == 0) {  // CGS2 orthonormalisation of Z into Y by one warp
      for (int j = 0; j < m; ++j) {
        for (int pass = 0; pass < 2; ++pass) {
          for (int i = 0; i < j; ++i) {
            float2 c = make_float2(0.f, 0.f);
            for (int a = lane; a < n; a += 32) c = cadd(c, cmulc(Ys[a * m + i], Zs[a * m + j]));
            for (int o = 16; o; o >>= 1) { c.x += __shfl_xor_sync(~0u, c.x, o); c.y += __shfl_xor_sync(~0u, c.y, o); }
            for (int a = lane; a < n; a += 32) Zs[a * m + j] = csub(Zs[a * m + j], cmul(c, Ys[a * m + i]));
            __syncwarp();
          }
        }
        float nr = 0.f;
        for (int a = lane; a < n; a += 32) nr += cabs2(Zs[a * m + j]);
        for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
        float s = nr > 0.f ? rsqrtf(nr) : 0.f;
        for (int a = lane; a < n; a += 32) Ys[a * m + j] = cscale(Zs[a * m + j], s);
        __syncwarp();
      }
    }
    __syncthreads();
  }

  EVD_STAMP(1);
  // ---------------- phase B: Householder QR of Y (one warp); reflectors -> Zs
  if (warp == 0) {
    for (int j = 0; j < m; ++j) {
      float nr = 0.f;
      for (int a = j + lane; a < n; a += 32) nr += cabs2(Ys[a * m + j]);
      for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
      float alpha = sqrtf(nr);
      float2 x0 = Ys[j * m + j];
      float ax0 = sqrtf(cabs2(x0));
      float2 e = ax0 > 0.f ? cscale(x0, 1.f / ax0) : make_float2(1.f, 0.f);
      float beta = alpha > 0.f ? 1.f / (alpha * (alpha + ax0)) : 0.f;
      for (int a = lane; a < np; a += 32) {
        float2 v = (a < j || a >= n) ? make_float2(0.f, 0.f) : Ys[a * m + j];
        if (a == j) v = cadd(x0, cscale(e, alpha));
        Zs[a * m + j] = v;
      }
      if (lane == 0) betas[j] = beta;
      __syncwarp();
      for (int c = j + 1; c < m; ++c) {
        float2 t = make_float2(0.f, 0.f);
        for (int a = j + lane; a < n; a += 32) t = cadd(t, cmulc(Zs[a * m + j], Ys[a * m + c]));
        for (int o = 16; o; o >>= 1) { t.x += __shfl_xor_sync(~0u, t.x, o); t.y += __shfl_xor_sync(~0u, t.y, o); }
        t = cscale(t, beta);
        for (int a = j + lane; a < n; a += 32) Ys[a * m + c] = csub(Ys[a * m + c], cmul(Zs[a * m + j], t));
        __syncwarp();
      }
    }
  }
  __syncthreads();

  EVD_STAMP(2);
  // ---------------- phase C: B = Q^H R Q in double-float (upper triangle)
  for (int e = tid; e < np * np; e += EVD_THREADS) {
    int a = e / np, b = e % np;
    zdf v = {{0.f, 0.f}, {0.f, 0.f}};
    if (a < n && b < n && a <= b) {
      double2 r = R[(size_t)a * n + b];
      v.re = df_from_double(r.x * inv);
      v.im = df_from_double(r.y * inv);
    }
    Rdf[e] = v;
  }
  __syncthreads();
  zdf* yv = reinterpret_cast<zdf*>(Ys);  // Y no longer needed: np zdf (16 B) fits in np*m*8 for m >= 2
  for (int j = 0; j < m; ++j) {
    const float bj = betas[j];
    // y = R v (4 threads per row; R read through its upper triangle)
    {
      int a = tid >> 2, sub = tid & 3;
      zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
      if (a < n) {
        for (int b = j + sub; b < n; b += 4) {
          float2 v = Zs[b * m + j];
          zdf r = (a <= b) ? Rdf[a * np + b] : Rdf[b * np + a];
          if (a > b) { r.im = df_neg(r.im); }
          acc = zdf_add(acc, zdf_mul_c(r, v));
        }
      }
      for (int o = 1; o < 4; o <<= 1) {
        zdf t;
        t.re.hi = __shfl_xor_sync(~0u, acc.re.hi, o); t.re.lo = __shfl_xor_sync(~0u, acc.re.lo, o);
        t.im.hi = __shfl_xor_sync(~0u, acc.im.hi, o); t.im.lo = __shfl_xor_sync(~0u, acc.im.lo, o);
        acc = zdf_add(acc, t);
      }
      if (sub == 0 && a < np) yv[a] = acc;
    }
    __syncthreads();
    if (warp == 0) {  // kappa = beta * (v^H y) / 2   (real)
      df gam = {0.f, 0.f};
      for (int a = j + lane; a < n; a += 32) {
        float2 v = Zs[a * m + j];
        zdf y = yv[a];
        // Re(conj(v) y) = v.x*y.re + v.y*y.im
        gam = df_add(gam, df_add(df_mul_f(y.re, v.x), df_mul_f(y.im, v.y)));
      }
      for (int o = 16; o; o >>= 1) {
        df t = {__shfl_xor_sync(~0u, gam.hi, o), __shfl_xor_sync(~0u, gam.lo, o)};
        gam = df_add(gam, t);
      }
      if (lane == 0) sh_kappa = df_mul_f(gam, 0.5f * bj);
    }
    __syncthreads();
    const df kap = sh_kappa;
    for (int a = tid; a < n; a += EVD_THREADS) {  // u = y - kappa v
      float2 v = Zs[a * m + j];
      zdf y = yv[a];
      y.re = df_add(y.re, df_neg(df_mul_f(kap, v.x)));
      y.im = df_add(y.im, df_neg(df_mul_f(kap, v.y)));
      yv[a] = y;
    }
    __syncthreads();
    // R -= beta (u v^H + v u^H), upper triangle
    for (int e = tid; e < n * n; e += EVD_THREADS) {
      int a = e / n, b = e % n;
      if (a > b) continue;
      float2 va = Zs[a * m + j], vb = Zs[b * m + j];
      zdf ua = yv[a], ub = yv[b];
      zdf t1 = zdf_mul_c(ua, cconj(vb));
      // v_a conj(u_b) = conj(u_b conj(v_a))
      zdf t2 = zdf_mul_c(ub, cconj(va));
      t2.im = df_neg(t2.im);
      zdf s = zdf_add(t1, t2);
      s.re = df_mul_f(s.re, bj);
      s.im = df_mul_f(s.im, bj);
      zdf r = Rdf[a * np + b];
      r.re = df_add(r.re, df_neg(s.re));
      r.im = df_add(r.im, df_neg(s.im));
      Rdf[a * np + b] = r;
    }
    __syncthreads();
  }

  EVD_STAMP(3);
  // ---------------- convert B to fp32 A in place: entry e = a*np + b moves to a*ld + b,
  // which only overwrites df64 entries with index <= e, already read in this or an
  // earlier chunk
  for (int base = 0; base < np * np; base += EVD_THREADS) {
    int e = base + tid;
    float2 v = make_float2(0.f, 0.f);
    if (e < np * np) {
      zdf r = Rdf[e];
      v = make_float2(r.re.hi + r.re.lo, r.im.hi + r.im.lo);
    }
    __syncthreads();
    if (e < np * np) A[(e / np) * ld + (e % np)] = v;
    __syncthreads();
  }
  for (int e = tid; e < np * np; e += EVD_THREADS) {  // Hermitian mirror, real diagonal
    int a = e / np, b = e % np;
    if (a > b) A[a * ld + b] = cconj(A[b * ld + a]);
    else if (a == b) A[a * ld + b].y = 0.f;
  }
  // V = Q = H_0 H_1 ... H_{m-1} (applied to I, last reflector first); V^T row c = column c
  for (int e = tid; e < np * ld; e += EVD_THREADS) Vt[e] = make_float2((e / ld) == (e % ld) ? 1.f : 0.f, 0.f);
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    const float bj = betas[j];
    for (int c = tid; c < n; c += EVD_THREADS) {
      float2 t = make_float2(0.f, 0.f);
      for (int a = j; a < n; ++a) t = cadd(t, cmulc(Zs[a * m + j], Vt[c * ld + a]));
      t = cscale(t, bj);
      for (int a = j; a < n; ++a) Vt[c * ld + a] = csub(Vt[c * ld + a], cmul(Zs[a * m + j], t));
    }
    __syncthreads();
  }

  EVD_STAMP(4);
  // ---------------- phase D: cyclic Jacobi (round-robin), relative test
  // Work assignment is fixed for the whole solve: this thread's 2x2 blocks (ia <= ib of the
  // round's pair list) and its (pair, V row) items are decoded once.
  constexpr int MAXB = (56 * 57 / 2 + EVD_THREADS - 1) / EVD_THREADS;   // upper-triangle 2x2 blocks
  constexpr int MAXV = (112 * 56 + EVD_THREADS - 1) / EVD_THREADS;      // (pair, V row) items
  int blk[MAXB], vit[MAXV];
  {
    const int nblk = h * (h + 1) / 2;
    for (int j = 0; j < MAXB; ++j) {
      int e = tid + j * EVD_THREADS;
      int code = -1;
      if (e < nblk) {
        int ia = 0, rem = e;
        while (rem >= h - ia) { rem -= h - ia; ++ia; }
        code = (ia << 8) | (ia + rem);
      }
      blk[j] = code;
    }
    for (int j = 0; j < MAXV; ++j) {
      int e = tid + j * EVD_THREADS;
      vit[j] = (e < n * h) ? (((e / n) << 8) | (e % n)) : -1;
    }
  }
  int sweeps = 0, converged = 0;
  const int maxsw = g.max_sweeps > 0 ? g.max_sweeps : 40;
  for (; sweeps < maxsw; ++sweeps) {
    int any = 0;
    for (int r = 0; r < np - 1; ++r) {
      int rot = 0;
      if (tid < h) {
        int i = tid, pa, pb;
        if (i == 0) { pa = r; pb = np - 1; }
        else { pa = (r + i) % (np - 1); pb = (r - i + np - 1) % (np - 1); }
        int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
        float app = A[p * ld + p].x, aqq = A[q * ld + q].x;
        float2 b = A[p * ld + q];
        float ab = sqrtf(cabs2(b));
        float c = 1.f, dp = app, dq = aqq;
        float2 st = make_float2(0.f, 0.f);
        if (ab > 0.f && ab > JACOBI_TOL * sqrtf(fabsf(app) * fabsf(aqq))) {
          float zeta = (aqq - app) / (2.f * ab);
          float t = fabsf(zeta) > 1e18f ? 0.5f / zeta
                                       : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          c = 1.f / sqrtf(1.f + t * t);
          float s = t * c;
          st = make_float2(s * b.x / ab, s * b.y / ab);
          dp = app - t * ab;
          dq = aqq + t * ab;
          rot = 1;
        }
        pr_p[i] = p; pr_q[i] = q; pr_c[i] = c; pr_s[i] = st; pr_dp[i] = dp; pr_dq[i] = dq; pr_rot[i] = rot;
      }
      int anyr = __syncthreads_or(rot);
      if (!anyr) continue;
      any = 1;
#pragma unroll
      for (int j = 0; j < MAXB; ++j) {
        if (blk[j] < 0) continue;
        const int ia = blk[j] >> 8, ib = blk[j] & 255;
        const int ra = pr_rot[ia], rb = pr_rot[ib];
        if (!ra && !rb) continue;
        const int pa = pr_p[ia], qa = pr_q[ia], pb = pr_p[ib], qb = pr_q[ib];
        if (ia == ib) {
          A[pa * ld + pa] = make_float2(pr_dp[ia], 0.f);
          A[qa * ld + qa] = make_float2(pr_dq[ia], 0.f);
          A[pa * ld + qa] = make_float2(0.f, 0.f);
          A[qa * ld + pa] = make_float2(0.f, 0.f);
          continue;
        }
        const float ca = pr_c[ia], cb = pr_c[ib];
        const float2 sa = pr_s[ia], sb = pr_s[ib];
        float2 x00 = A[pa * ld + pb], x01 = A[pa * ld + qb], x10 = A[qa * ld + pb], x11 = A[qa * ld + qb];
        // Y = X J_b
        float2 sbc = cconj(sb);
        float2 y00 = csub(cscale(x00, cb), cmul(sbc, x01)), y01 = cadd(cmul(sb, x00), cscale(x01, cb));
        float2 y10 = csub(cscale(x10, cb), cmul(sbc, x11)), y11 = cadd(cmul(sb, x10), cscale(x11, cb));
        // X' = J_a^H Y
        float2 sac = cconj(sa);
        float2 z00 = csub(cscale(y00, ca), cmul(sa, y10)), z01 = csub(cscale(y01, ca), cmul(sa, y11));
        float2 z10 = cadd(cmul(sac, y00), cscale(y10, ca)), z11 = cadd(cmul(sac, y01), cscale(y11, ca));
        A[pa * ld + pb] = z00; A[pa * ld + qb] = z01; A[qa * ld + pb] = z10; A[qa * ld + qb] = z11;
        A[pb * ld + pa] = cconj(z00); A[qb * ld + pa] = cconj(z01);
        A[pb * ld + qa] = cconj(z10); A[qb * ld + qa] = cconj(z11);
      }
#pragma unroll
      for (int j = 0; j < MAXV; ++j) {
        if (vit[j] < 0) continue;
        const int ia = vit[j] >> 8, rr = vit[j] & 255;
        if (!pr_rot[ia]) continue;
        const int p = pr_p[ia], q = pr_q[ia];
        const float c = pr_c[ia];
        const float2 s = pr_s[ia];
        float2 vp = Vt[p * ld + rr], vq = Vt[q * ld + rr];
        Vt[p * ld + rr] = csub(cscale(vp, c), cmul(cconj(s), vq));
        Vt[q * ld + rr] = cadd(cmul(s, vp), cscale(vq, c));
      }
      __syncthreads();
    }
    if (!any) { converged = 1; break; }
  }

  __syncthreads();
  EVD_STAMP(5);
  // ---------------- phase E: sort, phase-fix, weights, projection weights
  for (int i = tid; i < n; i += EVD_THREADS) {
    float di = A[i * ld + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      float dj = A[j * ld + j].x;
      rank += (dj > di) || (dj == di && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  for (int i = tid; i < n; i += EVD_THREADS) lam_s[i] = (double)A[perm[i] * ld + perm[i]].x * scale;
  // phase of each (sorted) eigenvector: largest-magnitude entry made real positive
  for (int jj = warp; jj < n; jj += EVD_THREADS / 32) {
    int col = perm[jj];
    float best = -1.f; int bi = 0;
    for (int a = lane; a < n; a += 32) {
      float mg = cabs2(Vt[col * ld + a]);
      if (mg > best) { best = mg; bi = a; }
    }
    for (int o = 16; o; o >>= 1) {
      float ob = __shfl_xor_sync(~0u, best, o);
      int oi = __shfl_xor_sync(~0u, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
      float2 v = Vt[col * ld + bi];
      float mg = sqrtf(cabs2(v));
      sh_phase[jj] = mg > 0.f ? make_float2(v.x / mg, -v.y / mg) : make_float2(1.f, 0.f);
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += EVD_THREADS) {
    int a = e / n, jj = e % n;
    V_out[(size_t)k * n * n + e] = cmul(Vt[perm[jj] * ld + a], sh_phase[jj]);
  }
  // thresholding rule (double precision, one thread)
  double* wts = reinterpret_cast<double*>(Rdf);  // scratch: A's storage is dead after the sort copy
  __syncthreads();
  EVD_STAMP(6);
  if (tid == 0) {
    double* s0 = wts + np;          // scratch curves (A region no longer read)
    double* s1 = s0 + np;
    double* s2 = s1 + np;
    int kk = -1;
    const int md = g.thresh_mode;
    if (md == LCF_T_NONE) {
      for (int i = 0; i < n; ++i) wts[i] = 1.0;
      kk = 0;
    } else if (md <= LCF_T_MEDIAN) {
      kk = rule_k(md, lam_s, n, g.beta, g.k_fixed, g.curv_norm, s0, s1, s2);
      for (int i = 0; i < n; ++i) wts[i] = (i + 1 > kk) ? 1.0 : 0.0;
    } else if (md == LCF_T_SIGMOID) {
      kk = rule_k(g.k_src, lam_s, n, g.beta_src, g.k_fixed, g.curv_norm, s0, s1, s2);
      for (int i = 0; i < n; ++i) wts[i] = 1.0 / (1.0 + exp(-g.beta * ((i + 1) - kk)));
    } else {  // LCF_T_ADAPTIVE_SOFT
      double mx = -INFINITY;
      for (int i = 0; i < n; ++i) {
        double u = n > 1 ? 2.5 * i / (n - 1) : 0.0;
        wts[i] = -0.5 * u * u - g.beta * log(floor_lam(lam_s, n, i));
        mx = fmax(mx, wts[i]);
      }
      for (int i = 0; i < n; ++i) wts[i] = exp(wts[i] - mx);
      kk = -1;
    }
    double S = 0.0;
    for (int i = 0; i < n; ++i) S += wts[i] * wts[i] * lam_s[i];
    double pdsum = g.pd_mode == 0 ? S / n : S;
    double al;
    int fl = (converged ? 0 : LCF_WFLAG_NOCONV) | ((sweeps < 255 ? sweeps : 255) << LCF_WFLAG_SWEEP_SHIFT);
    if (g.alpha_mode == 1) al = 1.0;
    else {
      Box bx = boxes[k];
      double cnt = g.alpha_mode == 2 ? (double)(bx.z1 - bx.z0) * (bx.x1 - bx.x0) : (double)g.nz * g.nx;
      if (pdsum <= 1e-300) { al = 0.0; fl |= LCF_WFLAG_DEGENERATE; }
      else al = cnt / pdsum;
    }
    double cf = sqrt(al * (g.pd_mode == 0 ? 1.0 / n : 1.0));
    int nc = 0;
    for (int i = 0; i < n; ++i) {
      double w = wts[i] * cf;
      s0[i] = w;
      if (wts[i] > 0.0) perm[nc++] = i;       // perm reused: sorted index of column nc
    }
    kcut_out[k] = kk;
    alpha_out[k] = (float)al;
    flags_out[k] = fl;
    ncol_out[k] = nc;
    sh_flag = nc;
  }
  __syncthreads();
  const int nc = sh_flag;
  EVD_STAMP(7);
  for (int i = tid; i < n; i += EVD_THREADS) {
    lam_out[(size_t)k * n + i] = lam_s[i];
    wt_out[(size_t)k * n + i] = (float)wts[i];
  }
  const double* coef = wts + np;
  for (int e = tid; e < n * g.ncp; e += EVD_THREADS) {
    int t = e / g.ncp, c = e % g.ncp;
    float2 v = make_float2(0.f, 0.f);
    if (c < nc) {
      int i = perm[c];
      v = cscale(V_out[(size_t)k * n * n + t * n + i], (float)coef[i]);
    }
    W_out[(size_t)k * n * g.ncp + e] = v;
  }
  __syncthreads();
  EVD_STAMP(8);
}

cudaError_t launch_evd(const lcf_plan* P, cudaStream_t st) {
  EvdArgs a;
  const lcf_config& c = P->cfg;
  a.nt = P->nt; a.nz = c.nz; a.nx = c.nx;
  a.thresh_mode = c.thresh_mode; a.beta = c.beta; a.beta_src = c.beta_src;
  a.k_fixed = c.k_fixed; a.k_src = c.k_src; a.pd_mode = c.pd_mode; a.alpha_mode = c.alpha_mode;
  a.curv_norm = c.curv_norm; a.max_sweeps = c.max_sweeps; a.ncp = P->ncp;
  a.clk = P->profiling ? P->ws.evd_clk : nullptr;
  size_t sm = evd_smem_bytes(P->nt);
  evd_kernel<<<P->nd, EVD_THREADS, sm, st>>>(P->ws.R, P->ws.box, a, P->ws.lam, P->ws.V, P->ws.wt,
                                             P->ws.kcut, P->ws.alpha, P->ws.flags, P->ws.W, P->ws.ncol);
  return counted(P);
}

cudaError_t evd_configure() {
  return cudaFuncSetAttribute(evd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)evd_smem_bytes(kEvdCtaNmax));
}

}  // namespace lcf
