// k_evd_os.cu — batched Hermitian EVD (Eq. 2) by one-sided Jacobi on a Cholesky
// factor, one CTA per window (Nt <= 128).
//
// The prep kernel of the distributed EVD (k_evd_dist.cu) forms, per window,
// B = Q^H (R / scale) Q in double-float rounded to fp32, with Q from an FP32
// subspace iteration and its Householder QR, so the dominant (tissue) directions
// are split off before any FP32 rotation.  This kernel then
//   1. factors B = F F^H in FP32 by Cholesky with diagonal pivoting, F = P L with its rows
//      left in the original order (right-looking, every warp; a non-positive pivot ends it and
//      leaves the rest of F zero);
//   2. runs one-sided Jacobi (Hestenes' method) on the columns of F:
//      column pairs are rotated until every pair is orthogonal to a relative
//      tolerance.  B = F F^H = (F J)(F J)^H for every unitary J, so at
//      convergence each column is an eigenvector of B times the square root of
//      its eigenvalue (the scheme Veselic and Hari give for a positive definite
//      matrix; the rotations diagonalise L^H L, which diagonal pivoting makes
//      closer to diagonal than B);
//   3. eigenvalue = squared column norm (double-float sum), eigenvector =
//      column / norm; columns that vanished (numerical rank below Nt) are
//      replaced by a Gram-Schmidt completion;
//   4. V = Q U through the compact WY form, sort, thresholding rule, alpha,
//      phase fix and the projection weights W, as the other EVD kernels.
// Only the factor's columns are rotated: the eigenvectors come out of it, so a
// Jacobi step touches Nt x Nt numbers where the two-sided method updates A and V.
//
// Layout of the sweeps (a block ordering).  The columns, zero-padded to 8 nw for nw warps, form
// 2 nw blocks of four; warp w holds blocks A_w and B_w in registers (lane l rows l, l + 32, l + 64,
// l + 96 as packed pairs of rows, so the 2x2 Grams and the rotations run as packed FP32
// operations).  A round is four steps in which each warp, alone, meets all sixteen pairs of its
// A and B (column s of A with column (s + t) mod 4 of B at step t); the blocks then move one place
// on the circle of the round-robin ordering (A_0 stays, A_1 takes B_0, A_w takes A_(w-1), B_w
// takes B_(w+1), the last B takes its own A) through shared memory.  2 nw - 1 rounds meet every
// pair of blocks once; the first round of a sweep also pairs the columns inside each block (three
// steps), so a sweep meets every pair of columns once, in 8 nw - 1 steps like the circle ordering
// of single columns.  A step sums the four slots' partial Grams over the warp (reduce-scatter),
// forms the rotations (the formulas of the two-sided kernels, ep_rotation_os) and applies them;
// the CTA meets at a barrier once per round (twice where only one exchange buffer fits) instead
// of once per step.
#include <math.h>

#include "evd_common.cuh"
#include "lcf_internal.cuh"

namespace lcf {

constexpr int EO_THREADS = 512;
constexpr float EO_TOL = 2.0e-6f;              // relative orthogonality test (cosine of two columns)
constexpr int EO_SUBSPACE_ITERS = 3;
constexpr int EO_CB = 8;                       // Cholesky columns per trailing update
constexpr size_t EO_SMEM_MAX = 227 * 1024;     // dynamic shared memory a CTA may opt in to

struct EoArgs {
  int nt, nz, nx;
  int thresh_mode;
  double beta, beta_src;
  int k_fixed, k_src;
  int pd_mode, alpha_mode, curv_norm, max_sweeps;
  int ncp;
  long long* clk;   // [nd][kEvdPhases + 1] phase-boundary SM clocks (profiling), or null
};

__host__ __device__ inline size_t eo_align(size_t x) { return (x + 15) & ~(size_t)15; }

struct EoLayout {
  int np, h, lda, m, nw, rp, nbuf;   // nbuf: block-exchange buffers (2: by round parity)
  size_t a, x, colj, lam, sperm, wts, s0, s1, s2, coef, keep, phs, end;
};

// a: the matrix (B, then the Cholesky factor, then the eigenvector columns U, then V), rows by index;
// x: the Cholesky block's columns, the step-parity exchange buffers of the sweeps, later Vh, T,
// X = Vh^H U and Y = T X
__host__ __device__ inline EoLayout eo_layout_b(int n, int nbuf) {
  EoLayout L;
  L.nbuf = nbuf;
  L.nw = (n + 7) / 8;
  L.np = 8 * L.nw;           // column positions: two blocks of four per warp, zero columns past Nt
  L.h = L.np / 2;
  L.lda = L.np + 1;
  L.m = n < kEvdHead ? n : kEvdHead;
  L.rp = (n + 63) / 64;      // row pairs per lane (rows l, l + 32, ...)
  size_t o = 0;
  L.a = o; o = eo_align(o + (size_t)L.np * L.lda * 8);
  {
    // the sweeps' block exchange [buffer][warp][column 0..7][row pair][lane] (float4) overlays a and x
    const size_t xch = (size_t)nbuf * L.nw * 8 * L.rp * 32 * 16;
    const size_t post = ((size_t)L.m * n + (size_t)L.m * L.m + (size_t)2 * L.m * L.np) * 8;
    const size_t chol = (size_t)EO_CB * L.np * 8;   // the Cholesky block's columns
    size_t need = xch > o ? xch - o : 0;
    need = need > post ? need : post;
    need = need > chol ? need : chol;
    L.x = o; o = eo_align(o + need);
  }
  L.colj = o;  o = eo_align(o + (size_t)L.np * 8);
  L.lam = o;   o = eo_align(o + (size_t)L.np * 8);   // squared norm by column position
  L.sperm = o; o = eo_align(o + (size_t)L.np * 4);   // sorted -> column position
  L.wts = o;   o = eo_align(o + (size_t)L.np * 8);   // lambda sorted (scaled), then weights: lam_s | wts
  L.s0 = o;    o = eo_align(o + (size_t)L.np * 8);
  L.s1 = o;    o = eo_align(o + (size_t)L.np * 8);
  L.s2 = o;    o = eo_align(o + (size_t)L.np * 8);
  L.coef = o;  o = eo_align(o + (size_t)L.np * 4);
  L.keep = o;  o = eo_align(o + (size_t)(L.np + 1) * 4);
  L.phs = o;   o = eo_align(o + (size_t)L.np * 8);
  L.end = o;
  return L;
}
// two exchange buffers (one barrier a round) where they fit in shared memory, else one (two barriers)
__host__ __device__ inline EoLayout eo_layout(int n) {
  const EoLayout L = eo_layout_b(n, 2);
  return L.end + (size_t)n * 8 + 4096 <= EO_SMEM_MAX ? L : eo_layout_b(n, 1);
}

size_t evd_os_smem_bytes(int nt) { return eo_layout(nt).end + (size_t)nt * 8; }   // + lam_s

#define EO_STAMP(b)                                                                   \
  do {                                                                                \
    if (g.clk && tid == 0) g.clk[(size_t)k * (kEvdPhases + 1) + (b)] = clock64();      \
  } while (0)

// Row r of column c of the Cholesky factor G (pivot pc = index eliminated at step c), read from
// the in-place storage of the right-looking factorisation
__device__ __forceinline__ float2 eo_factor(const float2* A, int lda, const int* pos, int pc, int c, int r) {
  if (r == pc) return A[(size_t)pc * lda + pc];
  if (pos[r] < c) return make_float2(0.f, 0.f);
  return r > pc ? A[(size_t)r * lda + pc] : cconj(A[(size_t)pc * lda + r]);
}

// ---- the sweeps: warp w holds blocks A_w and B_w of four columns each ----
// Lane l holds rows l, l + 32, l + 64, l + 96 of every column as row pairs (XR = real parts of
// rows (2i) * 32 + l and (2i + 1) * 32 + l, XI the imaginary parts), so the dot products and the
// rotations run as packed FP32 pairs; register set j < 4 is column j of A_w, 4 + j column j of B_w.
// 16 partial sums v[4 s + c] (slot s, component c) summed over the warp; lane l receives the total
// of component ((l >> 1) & 3) of slot (l >> 3)
__device__ __forceinline__ float eo_reduce_scatter(const float (&v)[16], int lane) {
  float w8[8], w4[4], w2[2];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool hi = lane & 16;
    const float send = hi ? v[k] : v[8 + k], keep = hi ? v[8 + k] : v[k];
    w8[k] = keep + __shfl_xor_sync(~0u, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool hi = lane & 8;
    const float send = hi ? w8[k] : w8[4 + k], keep = hi ? w8[4 + k] : w8[k];
    w4[k] = keep + __shfl_xor_sync(~0u, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool hi = lane & 4;
    const float send = hi ? w4[k] : w4[2 + k], keep = hi ? w4[2 + k] : w4[k];
    w2[k] = keep + __shfl_xor_sync(~0u, send, 4);
  }
  const bool hi = lane & 2;
  const float w1 = (hi ? w2[1] : w2[0]) + __shfl_xor_sync(~0u, hi ? w2[0] : w2[1], 2);
  return w1 + __shfl_xor_sync(~0u, w1, 1);
}

// The position (factor column at the start, eigenvector column at the end) of column s of block j
// (A_w: 0, B_w: 1) of warp w: blocks in circle order, shifted so that A_0 holds the last four
__host__ __device__ inline int eo_block_pos(int nw, int w, int j, int s) {
  return 4 * ((2 * w + j + 2 * nw - 1) % (2 * nw)) + s;
}

// The four pairs of step K: K = 0..2 pair the columns inside each block ((0,1)(2,3), (0,2)(1,3),
// (0,3)(1,2) of A in slots 0 and 1, of B in slots 2 and 3); K = 3..6 pair column s of A with
// column (s + K - 3) & 3 of B in slot s, so four such steps meet all sixteen pairs of A and B.
__host__ __device__ constexpr int eo_inner(int k, int pr, int e) {
  constexpr int t[3][2][2] = {{{0, 1}, {2, 3}}, {{0, 2}, {1, 3}}, {{0, 3}, {1, 2}}};
  return t[k][pr][e];
}
template <int K> __host__ __device__ constexpr int eo_px(int s) {
  return K < 3 ? (s < 2 ? 0 : 4) + eo_inner(K, s & 1, 0) : s;
}
template <int K> __host__ __device__ constexpr int eo_py(int s) {
  return K < 3 ? (s < 2 ? 0 : 4) + eo_inner(K, s & 1, 1) : 4 + ((s + K - 3) & 3);
}

// One step of a warp: the 2x2 Gram of each slot's pair summed over the warp, its rotation
// (ep_rotation_os) and the update of both columns.  Returns whether some slot of the warp was not
// calm (warp-uniform).
template <int RP, int K>
__device__ __forceinline__ bool eo_bstep(float2 (&XR)[8][RP], float2 (&XI)[8][RP], int lane, float clim2,
                                         float slim2) {
  // ---- the 2x2 Gram of every slot: |x|^2, |y|^2, conj(x) y
  float v[16];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int t = eo_px<K>(s), b = eo_py<K>(s);
    float2 a2 = make_float2(0.f, 0.f), b2 = a2, gr = a2, gi = a2, gj = a2;
#pragma unroll
    for (int i = 0; i < RP; ++i) {
      a2 = __ffma2_rn(XR[t][i], XR[t][i], a2);
      a2 = __ffma2_rn(XI[t][i], XI[t][i], a2);
      b2 = __ffma2_rn(XR[b][i], XR[b][i], b2);
      b2 = __ffma2_rn(XI[b][i], XI[b][i], b2);
      gr = __ffma2_rn(XR[t][i], XR[b][i], gr);
      gr = __ffma2_rn(XI[t][i], XI[b][i], gr);
      gi = __ffma2_rn(XR[t][i], XI[b][i], gi);
      gj = __ffma2_rn(XI[t][i], XR[b][i], gj);
    }
    v[4 * s] = a2.x + a2.y;
    v[4 * s + 1] = b2.x + b2.y;
    v[4 * s + 2] = gr.x + gr.y;
    v[4 * s + 3] = (gi.x + gi.y) - (gj.x + gj.y);
  }
  const float tot = eo_reduce_scatter(v, lane);
  // ---- each group of 8 lanes forms the rotation of slot lane >> 3, then all four are broadcast
  const int base = lane & 24;
  const float a = __shfl_sync(~0u, tot, base), b = __shfl_sync(~0u, tot, base + 2);
  const float2 gm = make_float2(__shfl_sync(~0u, tot, base + 4), __shfl_sync(~0u, tot, base + 6));
  float c;
  float2 st;
  int rot;
  bool calm;
  ep_rotation_os(a, b, gm, EO_TOL, clim2, slim2, c, st, rot, calm);   // c = 1, st = 0 without a rotation
  const unsigned rmask = __ballot_sync(~0u, rot);
  const unsigned wmask = __ballot_sync(~0u, !calm);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (!((rmask >> (8 * s)) & 1u)) continue;   // warp-uniform
    const float cs = __shfl_sync(~0u, c, 8 * s), sr = __shfl_sync(~0u, st.x, 8 * s), si = __shfl_sync(~0u, st.y, 8 * s);
    const int t = eo_px<K>(s), bb = eo_py<K>(s);
    // [x y] J: x' = c x - conj(st) y, y' = st x + c y
    const float2 C2 = make_float2(cs, cs), SR = make_float2(sr, sr), SI = make_float2(si, si);
    const float2 NSR = make_float2(-sr, -sr), NSI = make_float2(-si, -si);
#pragma unroll
    for (int i = 0; i < RP; ++i) {
      const float2 xr = XR[t][i], xi = XI[t][i], yr = XR[bb][i], yi = XI[bb][i];
      XR[t][i] = __ffma2_rn(NSI, yi, __ffma2_rn(NSR, yr, __fmul2_rn(C2, xr)));
      XI[t][i] = __ffma2_rn(SI, yr, __ffma2_rn(NSR, yi, __fmul2_rn(C2, xi)));
      XR[bb][i] = __ffma2_rn(C2, yr, __ffma2_rn(NSI, xi, __fmul2_rn(SR, xr)));
      XI[bb][i] = __ffma2_rn(C2, yi, __ffma2_rn(SI, xr, __fmul2_rn(SR, xi)));
    }
  }
  return wmask != 0u;
}

template <int RP>
__global__ void __launch_bounds__(EO_THREADS, 1)
evd_os_kernel(const float2* __restrict__ Bg, const float2* __restrict__ Vhg, const float2* __restrict__ Tg,
              const double* __restrict__ scale_g, const Box* __restrict__ boxes, EoArgs g,
              double* __restrict__ lam_out, float2* __restrict__ V_out, float* __restrict__ wt_out,
              int* __restrict__ kcut_out, float* __restrict__ alpha_out, int* __restrict__ flags_out,
              float2* __restrict__ W_out, int* __restrict__ ncol_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x, n = g.nt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x;
  const EoLayout L = eo_layout(n);
  const int np = L.np, lda = L.lda, m = L.m;
  float2* A = reinterpret_cast<float2*>(smem + L.a);
  float2* colj = reinterpret_cast<float2*>(smem + L.colj);
  double* lam = reinterpret_cast<double*>(smem + L.lam);
  int* sperm = reinterpret_cast<int*>(smem + L.sperm);
  double* wts = reinterpret_cast<double*>(smem + L.wts);
  double* s0 = reinterpret_cast<double*>(smem + L.s0);
  double* s1 = reinterpret_cast<double*>(smem + L.s1);
  double* s2 = reinterpret_cast<double*>(smem + L.s2);
  float* coef = reinterpret_cast<float*>(smem + L.coef);
  int* keep = reinterpret_cast<int*>(smem + L.keep);
  float2* phs = reinterpret_cast<float2*>(smem + L.phs);
  double* lam_s = reinterpret_cast<double*>(smem + L.end);
  const double scale = scale_g[k];

  if (!(scale > 0.0)) {   // degenerate window (zero Gram): the empty result
    for (int e = tid; e < n * n; e += nthr) V_out[(size_t)k * n * n + e] = make_float2(e / n == e % n, 0.f);
    for (int e = tid; e < n * g.ncp; e += nthr) W_out[(size_t)k * n * g.ncp + e] = make_float2(0.f, 0.f);
    for (int i = tid; i < n; i += nthr) {
      lam_out[(size_t)k * n + i] = 0.0;
      wt_out[(size_t)k * n + i] = 0.f;
    }
    if (tid == 0) {
      kcut_out[k] = 0; alpha_out[k] = 0.f; ncol_out[k] = 0;
      flags_out[k] = LCF_WFLAG_DEGENERATE;
    }
    return;
  }
  EO_STAMP(3);

  // ---------------- pivoted Cholesky of B in FP32 by every warp, without interchanges: step j
  // takes as pivot p_j the remaining index with the largest diagonal of the Schur complement S and
  // writes column j of the factor, g_r = S(r, p_j) / sqrt(S(p_j, p_j)) for the remaining r, over
  // S's column p_j (lower triangle storage: S(r, c) at A[max][min], conjugated above the diagonal)
  // and sqrt(S(p_j, p_j)) at A[p_j][p_j].  The factor G (column j = step j, rows in the original
  // order) has G G^H = B: row r of column j is zero once r was eliminated before step j.  Columns
  // go in blocks of EO_CB: inside a block a column subtracts the block's earlier columns from the
  // stored S(r, p_j) (one row per thread) and the running diagonal is updated at once, so the next
  // pivot is known after one barrier; the remaining lower triangle then takes the block's rank-EO_CB
  // update in one pass over all its pairs.  A non-positive pivot ends it (numerical rank rk);
  // columns rk .. n - 1 stay zero.  The remaining indices (in increasing order) and their running
  // diagonal are kept by list position, double-buffered by step parity, so every warp searches the
  // pivot itself (n <= 128: at most four list positions per lane).
  float* dgb = reinterpret_cast<float*>(colj);       // running diagonal by list position, [parity][np]
  float2* gv = reinterpret_cast<float2*>(smem + L.x);   // the block's columns by index, [EO_CB][np]
  int* remb = reinterpret_cast<int*>(lam);           // remaining indices, [parity][np]
  int* pos = reinterpret_cast<int*>(s1);             // step that eliminated each index (n: none)
  int* ord = reinterpret_cast<int*>(s2);             // index eliminated at each step
  const int nwarp = nthr / 32;
  {
    const float2* B = Bg + (size_t)k * n * n;
    for (int i = warp; i < n; i += nwarp)
      for (int c = lane; c <= i; c += 32) A[(size_t)i * lda + c] = B[(size_t)i * n + c];
    for (int r = tid; r < np; r += nthr) { remb[r] = r; pos[r] = n; }
    for (int i = tid; i < n; i += nthr) dgb[i] = B[(size_t)i * n + i].x;
  }
  __syncthreads();
  int rk = n;
  {
    float first = 0.f;
    bool stop = false;
    for (int j0 = 0; j0 < n && !stop; j0 += EO_CB) {
      const int j1 = j0 + EO_CB < n ? j0 + EO_CB : n;
      int j = j0;
      for (; j < j1; ++j) {
        const int cnt = n - j, par = j & 1, t = j - j0;
        const int* rin = remb + par * np;
        int* rout = remb + (par ^ 1) * np;
        const float* din = dgb + par * np;
        float* dout = dgb + (par ^ 1) * np;
        float dd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dd[q] = lane + 32 * q < cnt ? din[lane + 32 * q] : -INFINITY;
        float best = -INFINITY;   // the largest remaining diagonal entry, ties to the lower index
        int ba = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (dd[q] > best) { best = dd[q]; ba = lane + 32 * q; }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const float ob = __shfl_xor_sync(~0u, best, o);
          const int oa = __shfl_xor_sync(~0u, ba, o);
          if (ob > best || (ob == best && oa < ba)) { best = ob; ba = oa; }
        }
        if (j == 0) first = best;
        if (!(best > first * 1e-30f) || !isfinite(best)) { rk = j; stop = true; break; }   // in every warp
        const int pa = ba, p = rin[pa];
        const float inv = ep_rsqrt(best);
        for (int a = tid; a < cnt; a += nthr) {
          const int r = rin[a];
          if (a == pa) {
            A[(size_t)p * lda + p] = make_float2(best * inv, 0.f);
            ord[j] = p;
            pos[p] = j;
          } else {
            float2* e = r > p ? &A[(size_t)r * lda + p] : &A[(size_t)p * lda + r];
            float2 v = r > p ? *e : cconj(*e);
            for (int u = 0; u < t; ++u) v = csub(v, cmul(gv[u * np + r], cconj(gv[u * np + p])));
            const float2 g = cscale(v, inv);
            *e = r > p ? g : cconj(g);
            gv[t * np + r] = g;
            const int ao = a - (a > pa);
            dout[ao] = din[a] - cabs2(g);
            rout[ao] = r;
          }
        }
        __syncthreads();
      }
      if (stop) break;
      // the block's update of the remaining lower triangle: pair e = a (a - 1) / 2 + b of list
      // positions b < a; S(r, c) -= sum_u g_u[r] conj(g_u[c]) for the pair's indices r, c
      const int cnt = n - j, nb = j - j0;
      const int* rl = remb + (j & 1) * np;
      const int npair = cnt * (cnt - 1) / 2;
      for (int e = tid; e < npair; e += nthr) {
        int a = (int)(0.5f * (1.f + sqrtf(8.f * (float)e + 1.f)));
        if (a * (a - 1) / 2 > e) --a;
        else if ((a + 1) * a / 2 <= e) ++a;
        const int b = e - a * (a - 1) / 2;
        const int r = rl[a], c = rl[b];
        const int hi = r > c ? r : c, lo = r > c ? c : r;
        float2 acc = A[(size_t)hi * lda + lo];
        for (int u = 0; u < nb; ++u) acc = csub(acc, cmul(gv[u * np + hi], cconj(gv[u * np + lo])));
        A[(size_t)hi * lda + lo] = acc;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  EO_STAMP(4);

  // ---------------- one-sided Jacobi: block j of warp w (A_w: j = 0, B_w: j = 1) starts with
  // columns 4 q .. 4 q + 3, q = (2 w + j - 1) mod 2 nw (eo_block_pos): the last four positions form
  // A_0, which the circle never moves, so with four or more padding columns A_0 is zero and warp 0
  // has no cross pair to rotate (it skips those steps: the other warps then sit three to a
  // scheduler at Nt = 100, where thirteen would put four on one)
  const int nw = L.nw;
  const bool idle0 = warp == 0 && L.np - n >= 4;
  const float ne = (float)(n + (n & 1));   // the calm bounds take the unpadded size
  const float clim2 = ne * EO_TOL * EO_TOL, slim2 = 0.25f / (ne * ne * ne);
  float2 XR[8][RP], XI[8][RP];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int ct = eo_block_pos(nw, warp, 0, s), cb = eo_block_pos(nw, warp, 1, s);
#pragma unroll
    for (int i = 0; i < RP; ++i) {
      float v[2][4];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int r = (2 * i + e) * 32 + lane;
        const float2 t = (r < n && ct < rk) ? eo_factor(A, lda, pos, ord[ct], ct, r) : make_float2(0.f, 0.f);
        const float2 b = (r < n && cb < rk) ? eo_factor(A, lda, pos, ord[cb], cb, r) : make_float2(0.f, 0.f);
        v[e][0] = t.x; v[e][1] = t.y; v[e][2] = b.x; v[e][3] = b.y;
      }
      XR[s][i] = make_float2(v[0][0], v[1][0]);
      XI[s][i] = make_float2(v[0][1], v[1][1]);
      XR[4 + s][i] = make_float2(v[0][2], v[1][2]);
      XI[4 + s][i] = make_float2(v[0][3], v[1][3]);
    }
  }
  __syncthreads();   // the factor is read: a and x hold the block exchange from here on
  // Rounds of four steps; a window has converged once 2 nw - 1 consecutive rounds (a whole sweep:
  // every pair once, the inner pairs included) were calm: no rotation above the cosine and sine
  // bounds of ep_rotation_os.
  int converged = 0, sweeps = 0;
  {
    float4* xq0 = reinterpret_cast<float4*>(smem + L.a);   // [buffer][warp][column 0..7][row pair][lane]
    const size_t xbuf = (size_t)nw * 8 * RP * 32;           // float4 per buffer
    const int per = 2 * nw - 1;
    const int maxrounds = (g.max_sweeps > 0 ? g.max_sweeps : 40) * per;
    int rounds = 0, quiet = 0, last = 0, rr = 0;
    for (;;) {
      bool nc = false;
      if (rr == 0) {   // the pairs inside each block, once per sweep
        nc |= eo_bstep<RP, 0>(XR, XI, lane, clim2, slim2);
        nc |= eo_bstep<RP, 1>(XR, XI, lane, clim2, slim2);
        nc |= eo_bstep<RP, 2>(XR, XI, lane, clim2, slim2);
      }
      if (!idle0) {
        nc |= eo_bstep<RP, 3>(XR, XI, lane, clim2, slim2);
        nc |= eo_bstep<RP, 4>(XR, XI, lane, clim2, slim2);
        nc |= eo_bstep<RP, 5>(XR, XI, lane, clim2, slim2);
        nc |= eo_bstep<RP, 6>(XR, XI, lane, clim2, slim2);
      }
      // ---- the blocks move: A_w goes to warp w + 1 (read by warps 2 .. nw - 1), B_w to warp w - 1
      // (B_0 to warp 1 as its A); A_0 stays and the last warp's A becomes its own B
      float4* xq = xq0 + (L.nbuf == 2 ? (size_t)(rounds & 1) * xbuf : 0);
      if (nw > 1) {
        float4* own = xq + (size_t)warp * 8 * RP * 32 + lane;
        if (warp > 0 && warp < nw - 1) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int i = 0; i < RP; ++i)
              own[(c * RP + i) * 32] = make_float4(XR[c][i].x, XR[c][i].y, XI[c][i].x, XI[c][i].y);
        }
#pragma unroll
        for (int c = 4; c < 8; ++c)
#pragma unroll
          for (int i = 0; i < RP; ++i)
            own[(c * RP + i) * 32] = make_float4(XR[c][i].x, XR[c][i].y, XI[c][i].x, XI[c][i].y);
      }
      const int any = __syncthreads_or(nc);
      if (nw > 1) {
        if (warp == nw - 1) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int i = 0; i < RP; ++i) { XR[4 + c][i] = XR[c][i]; XI[4 + c][i] = XI[c][i]; }
        }
        if (warp > 0) {   // new A: B_0 for warp 1, A_(w-1) for the others
          const float4* src = xq + (size_t)(warp - 1) * 8 * RP * 32 + (warp == 1 ? 4 * RP * 32 : 0) + lane;
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int i = 0; i < RP; ++i) {
              const float4 q = src[(c * RP + i) * 32];
              XR[c][i] = make_float2(q.x, q.y); XI[c][i] = make_float2(q.z, q.w);
            }
        }
        if (warp < nw - 1) {   // new B: B_(w+1)
          const float4* src = xq + (size_t)(warp + 1) * 8 * RP * 32 + lane;
#pragma unroll
          for (int c = 4; c < 8; ++c)
#pragma unroll
            for (int i = 0; i < RP; ++i) {
              const float4 q = src[(c * RP + i) * 32];
              XR[c][i] = make_float2(q.x, q.y); XI[c][i] = make_float2(q.z, q.w);
            }
        }
        // read before the next round writes: with two buffers the next round writes the other one,
        // and the round after it only after the next round's barrier, which follows these reads
        if (L.nbuf == 1) __syncthreads();
      }
      ++rounds;
      if (any) { quiet = 0; last = rounds; }
      else ++quiet;
      if (quiet >= per) { converged = 1; break; }
      if (rounds >= maxrounds) break;
      rr = rr + 1 == per ? 0 : rr + 1;
    }
    sweeps = (last + per - 1) / per;
  }
  EO_STAMP(5);

  // ---------------- columns back to shared memory (column s of block j of warp w at position
  // eo_block_pos(nw, w, j, s)) with their squared norms (double-float sums), then normalised
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int pa = eo_block_pos(nw, warp, 0, s), pb = eo_block_pos(nw, warp, 1, s);
    df na = {0.f, 0.f}, nb = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < RP; ++i) {
      na = df_add_f(na, fmaf(XR[s][i].x, XR[s][i].x, XI[s][i].x * XI[s][i].x));
      na = df_add_f(na, fmaf(XR[s][i].y, XR[s][i].y, XI[s][i].y * XI[s][i].y));
      nb = df_add_f(nb, fmaf(XR[4 + s][i].x, XR[4 + s][i].x, XI[4 + s][i].x * XI[4 + s][i].x));
      nb = df_add_f(nb, fmaf(XR[4 + s][i].y, XR[4 + s][i].y, XI[4 + s][i].y * XI[4 + s][i].y));
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      df t;
      t.hi = __shfl_xor_sync(~0u, na.hi, o); t.lo = __shfl_xor_sync(~0u, na.lo, o); na = df_add(na, t);
      t.hi = __shfl_xor_sync(~0u, nb.hi, o); t.lo = __shfl_xor_sync(~0u, nb.lo, o); nb = df_add(nb, t);
    }
    {
      // squared norms below 2^-100 (the matrix is scaled to a largest diagonal in [1/2, 1)) count as
      // vanished columns
      double la = (double)na.hi + (double)na.lo, lb = (double)nb.hi + (double)nb.lo;
      la = la > 7.888609052210118e-31 ? la : 0.0;
      lb = lb > 7.888609052210118e-31 ? lb : 0.0;
      if (lane == 0) { lam[pa] = la; lam[pb] = lb; }
      const float ia = la > 0.0 ? ep_rsqrt((float)la) : 0.f, ib = lb > 0.0 ? ep_rsqrt((float)lb) : 0.f;
#pragma unroll
      for (int i = 0; i < RP; ++i) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int r = (2 * i + e) * 32 + lane;
          if (r < n) {
            A[(size_t)r * lda + pa] =
                make_float2((e ? XR[s][i].y : XR[s][i].x) * ia, (e ? XI[s][i].y : XI[s][i].x) * ia);
            A[(size_t)r * lda + pb] =
                make_float2((e ? XR[4 + s][i].y : XR[4 + s][i].x) * ib, (e ? XI[4 + s][i].y : XI[4 + s][i].x) * ib);
          }
        }
      }
    }
  }
  __syncthreads();
  // sort positions by squared norm, descending (ties to the lower position); the first n are the
  // eigenpairs (the padding columns past Nt are zero and sort among the zeros)
  // (the squared norms are >= 0, so their bit patterns order as integers: the comparisons run on
  // the integer pipes, not on the few FP64 units)
  const long long* lbits = reinterpret_cast<const long long*>(lam);
  for (int i = tid; i < np; i += nthr) {
    const long long di = lbits[i];
    int r = 0;
    for (int j = 0; j < np; ++j) {
      const long long dj = lbits[j];
      r += (dj > di) || (dj == di && j < i);
    }
    sperm[r] = i;
  }
  __syncthreads();
  // vanished columns: Gram-Schmidt completion (two passes) of unit vectors against the columns before
  // them in sorted order (warp 0; numerical rank below Nt only: the zeros sort last, so none when the
  // n-th norm is positive)
  if (warp == 0 && !(lbits[sperm[n - 1]] > 0)) {
    int cand = 0;
    for (int jj = 0; jj < n; ++jj) {
      const int pos = sperm[jj];
      if (lam[pos] > 0.0) continue;
      for (int tries = 0; tries < n; ++tries, cand = (cand + 1) % n) {
        for (int r = lane; r < n; r += 32) A[(size_t)r * lda + pos] = make_float2(r == cand ? 1.f : 0.f, 0.f);
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int q = 0; q < jj; ++q) {
            const int qp = sperm[q];
            float2 d = make_float2(0.f, 0.f);
            for (int r = lane; r < n; r += 32) d = cadd(d, cmulc(A[(size_t)r * lda + qp], A[(size_t)r * lda + pos]));
            for (int o = 16; o; o >>= 1) { d.x += __shfl_xor_sync(~0u, d.x, o); d.y += __shfl_xor_sync(~0u, d.y, o); }
            for (int r = lane; r < n; r += 32)
              A[(size_t)r * lda + pos] = csub(A[(size_t)r * lda + pos], cmul(d, A[(size_t)r * lda + qp]));
            __syncwarp();
          }
        }
        float nr = 0.f;
        for (int r = lane; r < n; r += 32) nr += cabs2(A[(size_t)r * lda + pos]);
        for (int o = 16; o; o >>= 1) nr += __shfl_xor_sync(~0u, nr, o);
        if (nr > 0.5f / n) {   // some unit vector keeps at least 1/n of its square in the complement
          const float sc = ep_rsqrt(nr);
          for (int r = lane; r < n; r += 32) A[(size_t)r * lda + pos] = cscale(A[(size_t)r * lda + pos], sc);
          __syncwarp();
          cand = (cand + 1) % n;
          break;
        }
      }
      if (lane == 0) lam[pos] = 0.0;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nthr) lam_s[i] = lam[sperm[i]] * scale;
  EO_STAMP(6);

  // ---------------- rule and weights (every thread, double precision), then alpha and the kept
  // columns (warp 0)
  __syncthreads();
  __shared__ int sh_red;
  __shared__ double sh_mx;
  const int kk = ep_rule_weights_cta(g.thresh_mode, lam_s, n, g.beta, g.beta_src, g.k_fixed, g.k_src, g.curv_norm, wts,
                                     s0, s1, s2, &sh_red, &sh_mx, tid, nthr);
  if (warp == 0) {
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
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const bool kp = i < n && wts[i] > 0.0;
      const unsigned bal = __ballot_sync(~0u, kp);
      if (kp) keep[1 + base + __popc(bal & ((1u << lane) - 1u))] = i;
      if (i < n) coef[i] = (float)(wts[i] * cf);
      base += __popc(bal);
    }
    if (lane == 0) { keep[0] = base; ncol_out[k] = base; }
  }
  // ---------------- V = Q U = U - Vh (T (Vh^H U))
  float2* Vh = reinterpret_cast<float2*>(smem + L.x);   // [j][a], a by original index
  float2* Tm = Vh + (size_t)m * n;                      // [i][j]
  float2* X = Tm + (size_t)m * m;                       // [j][pos]
  float2* Y = X + (size_t)m * np;
  for (int e = tid; e < m * n; e += nthr) Vh[e] = Vhg[(size_t)k * m * n + e];
  for (int e = tid; e < m * m; e += nthr) Tm[e] = Tg[(size_t)k * m * m + e];
  __syncthreads();
  for (int e = tid; e < m * np; e += nthr) {
    const int j = e / np, pos = e % np;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < n; ++r) acc = cadd(acc, cmulc(Vh[(size_t)j * n + r], A[(size_t)r * lda + pos]));
    X[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < m * np; e += nthr) {
    const int i = e / np, pos = e % np;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = i; j < m; ++j) acc = cadd(acc, cmul(Tm[i * m + j], X[(size_t)j * np + pos]));
    Y[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < n * np; e += nthr) {
    const int r = e / np, pos = e % np;
    float2 v = A[(size_t)r * lda + pos];
    for (int j = 0; j < m; ++j) v = csub(v, cmul(Vh[(size_t)j * n + r], Y[(size_t)j * np + pos]));
    A[(size_t)r * lda + pos] = v;
  }
  __syncthreads();
  // phase of each sorted eigenvector: its largest-magnitude entry made real positive (ties to the
  // lower row by original index)
  for (int jj = warp; jj < n; jj += (nthr / 32)) {
    const int pos = sperm[jj];
    float best = -1.f;
    int bi = 0x7fffffff;
    for (int a = lane; a < n; a += 32) {
      const float mg = cabs2(A[(size_t)a * lda + pos]);
      if (mg > best) { best = mg; bi = a; }
    }
    for (int o = 16; o; o >>= 1) {
      const float ob = __shfl_xor_sync(~0u, best, o);
      const int oi = __shfl_xor_sync(~0u, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
      const float2 v = A[(size_t)(bi < n ? bi : 0) * lda + pos];   // bi >= n only if every entry is NaN
      const float mg = sqrtf(cabs2(v));
      phs[jj] = mg > 0.f ? make_float2(v.x / mg, -v.y / mg) : make_float2(1.f, 0.f);
    }
  }
  __syncthreads();
  EO_STAMP(7);
  for (int i = tid; i < n; i += nthr) {
    lam_out[(size_t)k * n + i] = lam_s[i];
    wt_out[(size_t)k * n + i] = (float)wts[i];
  }
  for (int e = tid; e < n * n; e += nthr) {
    const int a = e / n, jj = e % n;
    V_out[(size_t)k * n * n + e] = cmul(A[(size_t)a * lda + sperm[jj]], phs[jj]);
  }
  const int nc = keep[0];
  for (int e = tid; e < n * g.ncp; e += nthr) {
    const int a = e / g.ncp, c = e % g.ncp;
    float2 v = make_float2(0.f, 0.f);
    if (c < nc) {
      const int jj = keep[1 + c];
      v = cscale(cmul(A[(size_t)a * lda + sperm[jj]], phs[jj]), coef[jj]);
    }
    W_out[(size_t)k * n * g.ncp + e] = v;
  }
  EO_STAMP(8);
}

template <int RP>
static void eo_launch(const lcf_plan* P, cudaStream_t st, const EoArgs& a) {
  evd_os_kernel<RP><<<P->nd, 32 * eo_layout(P->nt).nw, evd_os_smem_bytes(P->nt), st>>>(
      (const float2*)P->ws.evd_B, (const float2*)P->ws.evd_vh, (const float2*)P->ws.evd_t,
      (const double*)P->ws.evd_scale, (const Box*)P->ws.box, a, P->ws.lam, P->ws.V, P->ws.wt, P->ws.kcut,
      P->ws.alpha, P->ws.flags, P->ws.W, P->ws.ncol);
}

template <int RP>
static cudaError_t eo_configure_one() {
  // the largest request of the packet lengths this instance serves (two exchange buffers make a
  // shorter packet's request the larger one)
  size_t mx = 0;
  for (int n = (RP - 1) * 64 + 1; n <= RP * 64; ++n) mx = evd_os_smem_bytes(n) > mx ? evd_os_smem_bytes(n) : mx;
  return cudaFuncSetAttribute(evd_os_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
}

cudaError_t launch_evd_os(const lcf_plan* P, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  cudaError_t e = launch_evd_prep(P, st, EO_SUBSPACE_ITERS);
  if (e != cudaSuccess) return e;
  EoArgs a;
  a.nt = P->nt; a.nz = c.nz; a.nx = c.nx;
  a.thresh_mode = c.thresh_mode; a.beta = c.beta; a.beta_src = c.beta_src;
  a.k_fixed = c.k_fixed; a.k_src = c.k_src; a.pd_mode = c.pd_mode; a.alpha_mode = c.alpha_mode;
  a.curv_norm = c.curv_norm; a.max_sweeps = c.max_sweeps; a.ncp = P->ncp;
  a.clk = P->profiling ? P->ws.evd_clk : nullptr;
  if (eo_layout(P->nt).rp == 1) eo_launch<1>(P, st, a);
  else eo_launch<2>(P, st, a);
  return counted(P);
}

cudaError_t evd_os_configure() {
  cudaError_t e = eo_configure_one<1>();
  if (e == cudaSuccess) e = eo_configure_one<2>();
  return e;
}

}  // namespace lcf
