/*
 * lcf_oracle.c — plain FP64 CPU oracle for the localized Gaussian-windowed
 * EVD clutter filter (Huang et al., "Real-time Adaptive and Localized
 * Spatiotemporal Clutter Filtering for Ultrasound Small Vessel Imaging").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every step follows the paper in its own order and notation, in double
 * precision, without blocking, fusion or reordering:
 *   windows g_k                  Eq. 11 and the localized-processing section
 *   R_k = C_w^H C_w              Eq. 1 and Eq. 12 (conjugate transpose: the
 *                                paper writes ^T for complex data; only ^H
 *                                makes R Hermitian PSD with lambda = sigma^2,
 *                                Eq. 3)
 *   R_k = V Lambda V^H           Eq. 2, eigenvalues sorted descending; the
 *                                solver is a hand-written cyclic Jacobi
 *   weights wt (Lambda-hat)      thresholding methods 1-6 (Eq. 6, Eq. 7,
 *                                Eq. 8, Eq. 9, Eq. 10) and a fixed cutoff k
 *   C-hat = C_w (V Lambda-hat V^H)  Eq. 4, literally (the parenthesised
 *                                product is formed first)
 *   PD_k = mean_t |C-hat|^2      power Doppler, mean (or sum) over slow time
 *   PD = sum_k alpha_k PD_k      Eq. 13, alpha_k = 1 / mean flow power
 *
 * Readings of points the paper leaves open, as this oracle takes them:
 *   - centres at cell midpoints, sigma = sigma_scale * spacing, box support
 *     |dz| <= s*sigma_z and |dx| <= s*sigma_x (s = support_sigmas; s <= 0 means
 *     no clipping);
 *   - the windowed data C_w is what gets reconstructed, so PD_k carries g^2;
 *   - alpha_k uses the mean of PD_k over the full image grid (alpha_mode 0),
 *     or over the window support (alpha_mode 2), or alpha = 1 (alpha_mode 1);
 *   - method 1 normalises the log-eigenvalue curve by shifting its minimum
 *     to 0 and scaling it to [0, beta*Nt] (curv_norm 0); curv_norm 1 keeps the
 *     paper's literal beta*y(n)/y(1)*Nt;
 *   - method 2 runs on the same normalised log curve; k is the number of
 *     leading components whose descent -y'(n) is steeper than beta;
 *   - method 3 uses the median of the raw eigenvalues (mean of the two
 *     middle ones for even Nt) and a strict ">" test;
 *   - method 6 uses win(i) = exp(-0.5*(2.5*(i-1)/(Nt-1))^2) (a right
 *     half-Gaussian peaking at i = 1) and normalises wt to a maximum of 1;
 *   - logs and powers of eigenvalues use lambda~ = max(lambda, lambda_1*Nt*2^-52).
 *
 * Build: gcc -O2 -fopenmp -fcx-limited-range -shared -fPIC (see build.py).
 * -fcx-limited-range makes complex products the textbook formula
 * (a+bi)(c+di) = (ac-bd) + (ad+bc)i without NaN/Inf recovery branches.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

/* ---- configuration (mirrors the Python wrapper's ctypes structure) ---- */
typedef struct {
  int nz, nx, nt;          /* packet: iq[nt][nz][nx] complex64, x fastest        */
  int wz, wx;              /* window grid; Nd = wz*wx                             */
  double sigma_scale;      /* sigma = sigma_scale * spacing                       */
  double support_sigmas;   /* support half-width in sigmas; <= 0: whole image     */
  int all_ones_window;     /* 1: g == 1 everywhere (global filter)                */
  int thresh_mode;         /* ORA_T_*                                             */
  double beta;             /* scaling factor of the rule                          */
  int k_fixed;             /* cutoff for ORA_T_FIXED                              */
  int k_src;               /* rule that supplies k to the sigmoid (method 5)      */
  double beta_src;         /* scaling factor of that rule                         */
  int pd_mode;             /* 0: mean over slow time, 1: sum                      */
  int alpha_mode;          /* 0: 1/mean over grid, 1: alpha = 1, 2: 1/mean over support */
  int curv_norm;           /* 0: shifted normalisation, 1: literal beta*y/y1*Nt   */
  int max_sweeps;          /* Jacobi sweep cap (default 60)                       */
} ora_config;

enum { ORA_T_FIXED = 0, ORA_T_CURVATURE = 1, ORA_T_SLOPE = 2, ORA_T_MEDIAN = 3,
       ORA_T_SIGMOID = 4, ORA_T_ADAPTIVE_SOFT = 5, ORA_T_NONE = 6, ORA_T_NCC = 8 };

/* neighbours on each side of the cutoff in method 4 (the paper's fn = 5) */
#define ORA_NCC_FN 5

enum { ORA_FLAG_NOCONV = 1, ORA_FLAG_DEGENERATE = 2 };

/* ------------------------------------------------------------------------
 * Window geometry (Eq. 11; window centres and SD set by the number of
 * subsets).  Window k = iz*wx + ix.  Returns the support box [z0,z1)x[x0,x1)
 * and the centre / sigma so that g can be evaluated at any pixel.
 * ---------------------------------------------------------------------- */
typedef struct { double cz, cx, sz, sx; int z0, z1, x0, x1; int ones; } ora_window;

static ora_window make_window(const ora_config* c, int k) {
  ora_window w;
  int iz = k / c->wx, ix = k % c->wx;
  double dz = (double)c->nz / c->wz, dx = (double)c->nx / c->wx;
  w.cz = (iz + 0.5) * dz - 0.5;
  w.cx = (ix + 0.5) * dx - 0.5;
  w.sz = c->sigma_scale * dz;
  w.sx = c->sigma_scale * dx;
  w.ones = c->all_ones_window;
  w.z0 = 0; w.z1 = c->nz; w.x0 = 0; w.x1 = c->nx;
  if (!w.ones && c->support_sigmas > 0) {
    /* support = { z : |z - cz| <= s*sz } intersected with the image; found
       by testing every row / column (no rounding formula to get wrong). */
    int z0 = c->nz, z1 = 0, x0 = c->nx, x1 = 0;
    for (int z = 0; z < c->nz; ++z)
      if (fabs(z - w.cz) <= c->support_sigmas * w.sz) { if (z < z0) z0 = z; if (z + 1 > z1) z1 = z + 1; }
    for (int x = 0; x < c->nx; ++x)
      if (fabs(x - w.cx) <= c->support_sigmas * w.sx) { if (x < x0) x0 = x; if (x + 1 > x1) x1 = x + 1; }
    if (z1 <= z0 || x1 <= x0) { z0 = z1 = x0 = x1 = 0; }
    w.z0 = z0; w.z1 = z1; w.x0 = x0; w.x1 = x1;
  }
  return w;
}

/* Gaussian weight g_k(z, x); zero outside the support (Eq. 11 weights w_i). */
static double window_weight(const ora_window* w, int z, int x) {
  if (z < w->z0 || z >= w->z1 || x < w->x0 || x >= w->x1) return 0.0;
  if (w->ones) return 1.0;
  double a = (z - w->cz) / w->sz, b = (x - w->cx) / w->sx;
  return exp(-0.5 * a * a - 0.5 * b * b);
}

int ora_window_box(const ora_config* c, int k, int* box /* z0,z1,x0,x1 */, double* geom /* cz,cx,sz,sx */) {
  ora_window w = make_window(c, k);
  box[0] = w.z0; box[1] = w.z1; box[2] = w.x0; box[3] = w.x1;
  geom[0] = w.cz; geom[1] = w.cx; geom[2] = w.sz; geom[3] = w.sx;
  return 0;
}

/* Full-grid weights of window k: g[z*nx + x]. */
void ora_window_weights(const ora_config* c, int k, double* g) {
  ora_window w = make_window(c, k);
  for (int z = 0; z < c->nz; ++z)
    for (int x = 0; x < c->nx; ++x) g[z * c->nx + x] = window_weight(&w, z, x);
}

/* ------------------------------------------------------------------------
 * Casorati rows: s_p(t) = iq[t][z][x] promoted to complex double (the
 * Casorati reshaping of the packet, pixels x Nt).
 * ---------------------------------------------------------------------- */
static zc iq_at(const float* iq, const ora_config* c, int t, int z, int x) {
  size_t o = (((size_t)t * c->nz + z) * c->nx + x) * 2;
  return (double)iq[o] + I * (double)iq[o + 1];
}

/* R = C_w^H C_w = sum_p g_p^2 conj(s_p)^T s_p  (Eq. 12), full Nt x Nt. */
static void gram_window(const float* iq, const ora_config* c, const ora_window* w, zc* R, zc* s) {
  int nt = c->nt;
  memset(R, 0, sizeof(zc) * nt * nt);
  for (int z = w->z0; z < w->z1; ++z)
    for (int x = w->x0; x < w->x1; ++x) {
      double g = window_weight(w, z, x);
      for (int t = 0; t < nt; ++t) s[t] = g * iq_at(iq, c, t, z, x); /* row of C_w */
      for (int i = 0; i < nt; ++i) {
        zc a = conj(s[i]);
        for (int j = 0; j < nt; ++j) R[i * nt + j] += a * s[j];
      }
    }
}

void ora_gram(const float* iq, const ora_config* c, int k, zc* R) {
  ora_window w = make_window(c, k);
  zc* s = (zc*)malloc(sizeof(zc) * c->nt);
  gram_window(iq, c, &w, R, s);
  free(s);
}

/* ------------------------------------------------------------------------
 * Hermitian EVD by cyclic Jacobi (Eq. 2).  A (n x n, row-major) is
 * overwritten; on return lam[] holds the eigenvalues in descending order
 * (ties keep their diagonal position), V's columns the matching unit
 * eigenvectors, each with its largest-magnitude entry real and positive.
 * Returns the number of sweeps, or -1 if max_sweeps was reached first.
 * ---------------------------------------------------------------------- */
int ora_jacobi(int n, zc* A, zc* V, double* lam, int max_sweeps) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro2 = 0.0;
  for (int i = 0; i < n * n; ++i) fro2 += creal(A[i] * conj(A[i]));
  int sweeps = 0, converged = 0;
  for (; sweeps < max_sweeps; ++sweeps) {
    double off2 = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        if (p != q) off2 += creal(A[p * n + q] * conj(A[p * n + q]));
    if (off2 <= 1e-30 * fro2) { converged = 1; break; }
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        zc b = A[p * n + q];
        double ab = cabs(b);
        if (ab == 0.0) continue;
        double a = creal(A[p * n + p]), d = creal(A[q * n + q]);
        /* 2x2 block [[a, b], [conj(b), d]]: with b = |b| e^{i phi} the unitary
           J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] makes J^H B J diagonal when
           t = s/c solves t^2 + 2 zeta t - 1 = 0, zeta = (d - a) / (2|b|);
           the smaller root keeps the rotation angle <= pi/4. */
        double zeta = (d - a) / (2.0 * ab);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        zc e = b / ab;             /* e^{i phi} */
        zc st = sn * e;            /* s e^{i phi} */
        /* A <- J^H A J : columns p, q then rows p, q */
        for (int r = 0; r < n; ++r) {
          zc ap = A[r * n + p], aq = A[r * n + q];
          A[r * n + p] = cs * ap - conj(st) * aq;
          A[r * n + q] = st * ap + cs * aq;
        }
        for (int r = 0; r < n; ++r) {
          zc ap = A[p * n + r], aq = A[q * n + r];
          A[p * n + r] = cs * ap - st * aq;
          A[q * n + r] = conj(st) * ap + cs * aq;
        }
        A[p * n + p] = a - t * ab;
        A[q * n + q] = d + t * ab;
        A[p * n + q] = 0.0;
        A[q * n + p] = 0.0;
        for (int r = 0; r < n; ++r) {
          zc vp = V[r * n + p], vq = V[r * n + q];
          V[r * n + p] = cs * vp - conj(st) * vq;
          V[r * n + q] = st * vp + cs * vq;
        }
      }
  }
  /* sort descending, stable on the diagonal position (insertion sort) */
  int* idx = (int*)malloc(sizeof(int) * n);
  double* dg = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) { idx[i] = i; dg[i] = creal(A[i * n + i]); }
  for (int i = 1; i < n; ++i) {
    int v = idx[i], j = i - 1;
    while (j >= 0 && dg[idx[j]] < dg[v]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = v;
  }
  zc* W = (zc*)malloc(sizeof(zc) * n * n);
  for (int jn = 0; jn < n; ++jn) {
    int jo = idx[jn];
    lam[jn] = dg[jo];
    int imax = 0; double amax = -1.0;
    for (int r = 0; r < n; ++r) { double m = cabs(V[r * n + jo]); if (m > amax) { amax = m; imax = r; } }
    zc ph = (amax > 0) ? conj(V[imax * n + jo]) / amax : 1.0;
    for (int r = 0; r < n; ++r) W[r * n + jn] = V[r * n + jo] * ph;
  }
  memcpy(V, W, sizeof(zc) * n * n);
  free(W); free(dg); free(idx);
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------
 * Eigen-weights (the thresholding section).  lam: descending eigenvalues.
 * wt[i] for i = 0..n-1 corresponds to the paper's i = 1..Nt.  *k_out is the
 * cutoff k (number of rejected components) of the hard rules, or the k fed
 * to the sigmoid; -1 for the adaptive soft rule.
 * ---------------------------------------------------------------------- */
static double floor_lambda(const double* lam, int n, int i) {
  double fl = lam[0] * n * ldexp(1.0, -52);
  return lam[i] > fl ? lam[i] : fl;
}

/* MATLAB-style gradient: one-sided at the ends, central inside. */
static void gradient(const double* y, double* d, int n) {
  if (n == 1) { d[0] = 0; return; }
  d[0] = y[1] - y[0];
  d[n - 1] = y[n - 1] - y[n - 2];
  for (int i = 1; i < n - 1; ++i) d[i] = 0.5 * (y[i + 1] - y[i - 1]);
}

/* normalised log10-eigenvalue curve used by methods 1 and 2 */
static void norm_log_curve(const double* lam, int n, double beta, int literal, double* yh) {
  for (int i = 0; i < n; ++i) yh[i] = log10(floor_lambda(lam, n, i));
  if (literal) {                    /* beta * y(n) / y(1) * Nt, as printed */
    double y1 = yh[0];
    for (int i = 0; i < n; ++i) yh[i] = (y1 != 0.0) ? beta * yh[i] / y1 * n : 0.0;
  } else {                          /* shift min to 0, scale to [0, beta*Nt] */
    double y1 = yh[0], yn = yh[n - 1], span = y1 - yn;
    for (int i = 0; i < n; ++i) yh[i] = (span > 0) ? beta * n * (yh[i] - yn) / span : 0.0;
  }
}

/* method 1, Eq. 6: k = argmax of |y''| / (1 + y'^2)^{3/2} over n = 2..Nt-1 */
static int k_curvature(const double* lam, int n, double beta, int literal) {
  if (n < 3) return 0;
  double* y = (double*)malloc(sizeof(double) * n * 3);
  double *d1 = y + n, *d2 = y + 2 * n;
  norm_log_curve(lam, n, beta, literal, y);
  gradient(y, d1, n);
  gradient(d1, d2, n);
  int kbest = 2; double best = -1.0;
  for (int i = 1; i < n - 1; ++i) {           /* paper index n = i+1 in 2..Nt-1 */
    double kap = fabs(d2[i]) / pow(1.0 + d1[i] * d1[i], 1.5);
    if (kap > best) { best = kap; kbest = i + 1; }
  }
  free(y);
  return kbest;
}

/* method 2: number of leading components whose descent is steeper than beta */
static int k_slope(const double* lam, int n, double beta, int literal) {
  if (n < 2) return 0;
  double* y = (double*)malloc(sizeof(double) * n * 2);
  double* d1 = y + n;
  norm_log_curve(lam, n, 1.0, literal, y);
  gradient(y, d1, n);
  int k = n - 1;
  for (int i = 0; i < n; ++i)
    if (-d1[i] <= beta) { k = i; break; }       /* first flat index (0-based) = k */
  free(y);
  return k;
}

/* method 3, Eq. 7: T = beta * median(lambda); k = #{lambda_i > T} */
static int k_median(const double* lam, int n, double beta) {
  /* lam is sorted descending, so the median is read off the middle */
  double med = (n % 2) ? lam[n / 2] : 0.5 * (lam[n / 2 - 1] + lam[n / 2]);
  double T = beta * med;
  int k = 0;
  for (int i = 0; i < n; ++i) if (lam[i] > T) ++k;
  return k;
}

static int hard_k(int mode, const double* lam, int n, double beta, int k_fixed, int literal) {
  switch (mode) {
    case ORA_T_FIXED: return k_fixed < 0 ? 0 : (k_fixed > n ? n : k_fixed);
    case ORA_T_CURVATURE: return k_curvature(lam, n, beta, literal);
    case ORA_T_SLOPE: return k_slope(lam, n, beta, literal);
    case ORA_T_MEDIAN: return k_median(lam, n, beta);
    default: return 0;
  }
}

int ora_weights(int mode, int n, const double* lam, double beta, int k_fixed, int k_src,
                double beta_src, int curv_norm, double* wt) {
  int k = -1;
  if (mode == ORA_T_NONE) {
    for (int i = 0; i < n; ++i) wt[i] = 1.0;
    return 0;
  }
  if (mode <= ORA_T_MEDIAN) {
    k = hard_k(mode, lam, n, beta, k_fixed, curv_norm);
    for (int i = 0; i < n; ++i) wt[i] = (i + 1 > k) ? 1.0 : 0.0;
  } else if (mode == ORA_T_SIGMOID) {          /* method 5, Eq. 9 */
    k = hard_k(k_src, lam, n, beta_src, k_fixed, curv_norm);
    for (int i = 0; i < n; ++i) wt[i] = 1.0 / (1.0 + exp(-beta * ((i + 1) - k)));
  } else if (mode == ORA_T_ADAPTIVE_SOFT) {    /* method 6, Eq. 10 with a Gaussian taper */
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i) {
      double u = (n > 1) ? 2.5 * i / (n - 1) : 0.0;
      wt[i] = -0.5 * u * u - beta * log(floor_lambda(lam, n, i));   /* log wt */
      if (wt[i] > mx) mx = wt[i];
    }
    for (int i = 0; i < n; ++i) wt[i] = exp(wt[i] - mx);
  }
  return k;
}

/* ------------------------------------------------------------------------
 * Method 4 (Eq. 8): the cutoff k that minimises the normalised spatial
 * cross-correlation of a tissue image and a blood image built from the left
 * singular vectors next to the cutoff.  With C_w V = U D (lambda_i = sigma_i^2),
 * |u_i(p)| = |(C_w v_i)(p)| / sigma_i per pixel p of the window's support;
 * I_T(k) = sum_{i=k-fn+1..k} |u_i|, I_B(k) = sum_{i=k+1..k+fn} |u_i| (weights 1),
 *   NCC(k) = sum_p I_T I_B / (sqrt(sum_p I_T^2) sqrt(sum_p I_B^2)),
 * for the k whose neighbourhoods exist, fn <= k <= Nt - fn (1-based), with
 * fn = min(5, Nt/2).  Readings: sigma_i = sqrt(lambda~_i) (the floored
 * eigenvalue, so a zero eigenvalue gives a zero image, not a division by
 * zero); a k whose I_T or I_B is zero everywhere gets NCC = 1; ties take the
 * smallest k.  curve[k-1] = NCC(k), NaN outside the range (nullable).
 * V: the window's eigenvectors (columns, descending eigenvalues).
 * ---------------------------------------------------------------------- */
static int ncc_fn(int n) { return n / 2 < ORA_NCC_FN ? n / 2 : ORA_NCC_FN; }

static int k_ncc(const float* iq, const ora_config* c, const ora_window* w, const zc* V, const double* lam,
                 double* curve) {
  int n = c->nt, fn = ncc_fn(n);
  if (fn < 1) { if (curve) for (int i = 0; i < n; ++i) curve[i] = NAN; return 0; }
  int nk = n - 2 * fn + 1;                 /* k = fn .. n - fn */
  double* num = (double*)calloc(3 * (size_t)nk, sizeof(double));
  double *dt = num + nk, *db = num + 2 * nk;
  double* sig = (double*)malloc(sizeof(double) * n);
  double* m = (double*)malloc(sizeof(double) * n);
  zc* s = (zc*)malloc(sizeof(zc) * n);
  for (int i = 0; i < n; ++i) sig[i] = sqrt(floor_lambda(lam, n, i));
  for (int z = w->z0; z < w->z1; ++z)
    for (int x = w->x0; x < w->x1; ++x) {
      double g = window_weight(w, z, x);
      for (int t = 0; t < n; ++t) s[t] = g * iq_at(iq, c, t, z, x);      /* row of C_w */
      for (int i = 0; i < n; ++i) {                                        /* |u_i(p)| */
        zc acc = 0;
        for (int t = 0; t < n; ++t) acc += s[t] * V[t * n + i];
        m[i] = cabs(acc) / sig[i];
      }
      for (int j = 0; j < nk; ++j) {
        int k = fn + j;                    /* 1-based cutoff */
        double it = 0.0, ib = 0.0;
        for (int i = k - fn; i < k; ++i) it += m[i];          /* paper i = k-fn+1 .. k */
        for (int i = k; i < k + fn; ++i) ib += m[i];          /* paper i = k+1 .. k+fn */
        num[j] += it * ib;
        dt[j] += it * it;
        db[j] += ib * ib;
      }
    }
  if (curve) for (int i = 0; i < n; ++i) curve[i] = NAN;
  int kbest = fn; double best = INFINITY;
  for (int j = 0; j < nk; ++j) {
    double den = sqrt(dt[j]) * sqrt(db[j]);
    double v = den > 0.0 ? num[j] / den : 1.0;
    if (curve) curve[fn + j - 1] = v;
    if (v < best) { best = v; kbest = fn + j; }
  }
  free(num); free(sig); free(m); free(s);
  return kbest;
}

/* NCC curve of window k (Eq. 8) from the oracle's own Gram and EVD; returns its argmin. */
int ora_ncc_curve(const float* iq, const ora_config* c, int k, double* curve) {
  int nt = c->nt;
  ora_window w = make_window(c, k);
  zc* R = (zc*)malloc(sizeof(zc) * nt * nt);
  zc* V = (zc*)malloc(sizeof(zc) * nt * nt);
  zc* s = (zc*)malloc(sizeof(zc) * nt);
  double* lk = (double*)malloc(sizeof(double) * nt);
  gram_window(iq, c, &w, R, s);
  ora_jacobi(nt, R, V, lk, c->max_sweeps > 0 ? c->max_sweeps : 60);
  int kk = k_ncc(iq, c, &w, V, lk, curve);
  free(R); free(V); free(s); free(lk);
  return kk;
}

/* ------------------------------------------------------------------------
 * Full pipeline.  Outputs (nullable unless stated):
 *   pd       [nz*nx]   PD_final (required)
 *   lam, wt  [nd*nt]   per-window eigenvalues / weights
 *   kk, flags, sweeps [nd]; alpha [nd]
 *   Rout, Vout [nd*nt*nt] complex (row-major per window)
 *   pdk      [nd*nz*nx] per-window PD_k (full grid, 0 outside the support)
 *   dbg_subset >= 0 with filt [nt*nz*nx] complex: C-hat of that subset
 *   k_override [nd] (nullable): where >= 0, the cutoff k of window k is this
 *            value instead of the rule's (hard rules and the sigmoid centre);
 *            used to evaluate a second, equally valid cutoff at a near-tie.
 * ---------------------------------------------------------------------- */
int ora_filter_k(const float* iq, const ora_config* c, double* pd, double* lam, double* wt,
                 int* kk, double* alpha, int* flags, int* sweeps, zc* Rout, zc* Vout,
                 double* pdk, int dbg_subset, zc* filt, int nthreads, const int* k_override);

int ora_filter(const float* iq, const ora_config* c, double* pd, double* lam, double* wt,
               int* kk, double* alpha, int* flags, int* sweeps, zc* Rout, zc* Vout,
               double* pdk, int dbg_subset, zc* filt, int nthreads) {
  return ora_filter_k(iq, c, pd, lam, wt, kk, alpha, flags, sweeps, Rout, Vout, pdk, dbg_subset, filt,
                      nthreads, NULL);
}

int ora_filter_k(const float* iq, const ora_config* c, double* pd, double* lam, double* wt,
                 int* kk, double* alpha, int* flags, int* sweeps, zc* Rout, zc* Vout,
                 double* pdk, int dbg_subset, zc* filt, int nthreads, const int* k_override) {
  int nd = c->wz * c->wx, nt = c->nt, npix = c->nz * c->nx;
  int max_sweeps = c->max_sweeps > 0 ? c->max_sweeps : 60;
  double* pdall = (double*)calloc((size_t)nd * npix, sizeof(double));
  double* alph = (double*)calloc(nd, sizeof(double));
  if (!pdall || !alph) { free(pdall); free(alph); return -1; }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int k = 0; k < nd; ++k) {
    ora_window w = make_window(c, k);
    zc* R = (zc*)malloc(sizeof(zc) * nt * nt);
    zc* V = (zc*)malloc(sizeof(zc) * nt * nt);
    zc* M = (zc*)malloc(sizeof(zc) * nt * nt);
    zc* s = (zc*)malloc(sizeof(zc) * nt);
    zc* ch = (zc*)malloc(sizeof(zc) * nt);
    double* lk = (double*)malloc(sizeof(double) * nt);
    double* wk = (double*)malloc(sizeof(double) * nt);
    int fl = 0;
    gram_window(iq, c, &w, R, s);                                   /* Eq. 12 */
    if (Rout) memcpy(Rout + (size_t)k * nt * nt, R, sizeof(zc) * nt * nt);
    int sw = ora_jacobi(nt, R, V, lk, max_sweeps);                  /* Eq. 2 */
    if (sw < 0) fl |= ORA_FLAG_NOCONV;
    int kc;
    int uses_ncc = c->thresh_mode == ORA_T_NCC || (c->thresh_mode == ORA_T_SIGMOID && c->k_src == ORA_T_NCC);
    if (k_override && k_override[k] >= 0 && (c->thresh_mode <= ORA_T_SIGMOID || c->thresh_mode == ORA_T_NCC)) {
      /* the same weights with the cutoff given: a fixed-k rule, or the sigmoid at k */
      int mode = (c->thresh_mode == ORA_T_SIGMOID) ? ORA_T_SIGMOID : ORA_T_FIXED;
      kc = ora_weights(mode, nt, lk, c->beta, k_override[k], ORA_T_FIXED, 0.0, c->curv_norm, wk);
    } else if (uses_ncc) {
      /* method 4 (Eq. 8) decides k from the data; method 5 (Eq. 9) may take that k */
      int kn = k_ncc(iq, c, &w, V, lk, NULL);
      if (c->thresh_mode == ORA_T_NCC) kc = ora_weights(ORA_T_FIXED, nt, lk, c->beta, kn, ORA_T_FIXED, 0.0, c->curv_norm, wk);
      else kc = ora_weights(ORA_T_SIGMOID, nt, lk, c->beta, kn, ORA_T_FIXED, 0.0, c->curv_norm, wk);
    } else {
      kc = ora_weights(c->thresh_mode, nt, lk, c->beta, c->k_fixed, c->k_src, c->beta_src,
                       c->curv_norm, wk);
    }
    /* M = V diag(wt) V^H : the parenthesised factor of Eq. 4 */
    for (int i = 0; i < nt; ++i)
      for (int j = 0; j < nt; ++j) {
        zc acc = 0;
        for (int m = 0; m < nt; ++m) acc += V[i * nt + m] * wk[m] * conj(V[j * nt + m]);
        M[i * nt + j] = acc;
      }
    /* C-hat = C_w M (Eq. 4), PD_k = mean (or sum) over t of |C-hat|^2 */
    double* pk = pdall + (size_t)k * npix;
    double tot = 0.0;
    for (int z = w.z0; z < w.z1; ++z)
      for (int x = w.x0; x < w.x1; ++x) {
        double g = window_weight(&w, z, x);
        for (int t = 0; t < nt; ++t) s[t] = g * iq_at(iq, c, t, z, x);
        double p = 0.0;
        for (int t = 0; t < nt; ++t) {
          zc acc = 0;
          for (int m = 0; m < nt; ++m) acc += s[m] * M[m * nt + t];
          ch[t] = acc;
          p += creal(acc * conj(acc));
        }
        if (c->pd_mode == 0) p /= nt;
        pk[z * c->nx + x] = p;
        tot += p;
        if (k == dbg_subset && filt)
          for (int t = 0; t < nt; ++t) filt[((size_t)t * c->nz + z) * c->nx + x] = ch[t];
      }
    /* alpha_k: reciprocal of the mean flow power of subset k (Eq. 13) */
    double a;
    if (c->alpha_mode == 1) a = 1.0;
    else {
      double cnt = (c->alpha_mode == 2) ? (double)(w.z1 - w.z0) * (w.x1 - w.x0) : (double)npix;
      if (tot <= 1e-300) { a = 0.0; fl |= ORA_FLAG_DEGENERATE; }
      else a = cnt / tot;
    }
    alph[k] = a;
    if (lam) memcpy(lam + (size_t)k * nt, lk, sizeof(double) * nt);
    if (wt) memcpy(wt + (size_t)k * nt, wk, sizeof(double) * nt);
    if (kk) kk[k] = kc;
    if (alpha) alpha[k] = a;
    if (flags) flags[k] = fl;
    if (sweeps) sweeps[k] = sw;
    if (Vout) memcpy(Vout + (size_t)k * nt * nt, V, sizeof(zc) * nt * nt);
    free(R); free(V); free(M); free(s); free(ch); free(lk); free(wk);
  }
  /* Eq. 13: PD_final = sum_k alpha_k PD_k (fixed window order) */
  for (int p = 0; p < npix; ++p) {
    double acc = 0.0;
    for (int k = 0; k < nd; ++k) acc += alph[k] * pdall[(size_t)k * npix + p];
    pd[p] = acc;
  }
  if (pdk) memcpy(pdk, pdall, sizeof(double) * (size_t)nd * npix);
  free(pdall); free(alph);
  return 0;
}

/* Hermitian EVD entry for tests: A (n x n complex, row-major) is copied. */
int ora_eigh(int n, const zc* A, zc* V, double* lam, int max_sweeps) {
  zc* B = (zc*)malloc(sizeof(zc) * n * n);
  memcpy(B, A, sizeof(zc) * n * n);
  int sw = ora_jacobi(n, B, V, lam, max_sweeps > 0 ? max_sweeps : 60);
  free(B);
  return sw;
}

/* The quantity each hard rule maximises or compares, per index n (0-based):
 * method 1: the curvature K(n) (0 at the excluded ends); method 2: the descent
 * -y'(n) of the normalised curve; method 3: lambda_n / (beta * median).
 * Lets a test tell a near-tie (two cutoffs equally justified) from an error. */
int ora_rule_scores(int mode, int n, const double* lam, double beta, int curv_norm, double* sc) {
  double* y = (double*)malloc(sizeof(double) * n * 3);
  double *d1 = y + n, *d2 = y + 2 * n;
  for (int i = 0; i < n; ++i) sc[i] = 0.0;
  if (mode == ORA_T_CURVATURE && n >= 3) {
    norm_log_curve(lam, n, beta, curv_norm, y);
    gradient(y, d1, n);
    gradient(d1, d2, n);
    for (int i = 1; i < n - 1; ++i) sc[i] = fabs(d2[i]) / pow(1.0 + d1[i] * d1[i], 1.5);
  } else if (mode == ORA_T_SLOPE && n >= 2) {
    norm_log_curve(lam, n, 1.0, curv_norm, y);
    gradient(y, d1, n);
    for (int i = 0; i < n; ++i) sc[i] = -d1[i];
  } else if (mode == ORA_T_MEDIAN) {
    double med = (n % 2) ? lam[n / 2] : 0.5 * (lam[n / 2 - 1] + lam[n / 2]);
    for (int i = 0; i < n; ++i) sc[i] = lam[i] / (beta * med);
  }
  free(y);
  return 0;
}

int ora_abi_version(void) { return 3; }
