// k_evd_pair.cu — batched Hermitian EVD (Eq. 2), eigen-weights and projection
// weights on a CTA pair per window (a thread-block cluster of two).
//
// Same numerical plan as the one-CTA kernel (k_evd.cu): FP32 subspace iteration
// for the dominant (tissue) directions, Householder QR of that block, the
// congruence B = Q^H R Q in double-float, cyclic Jacobi in FP32 with the
// relative test, sort / phase fix / rule in double.  What changes is the
// division of work and the data layout:
//
//  * CTA 0 owns A, CTA 1 owns V.  A Jacobi step's rotations (c, s, p, q) go
//    from CTA 0 into a 16-deep ring in CTA 1's shared memory (st.async with a
//    complete_tx on CTA 1's mbarrier); CTA 1 applies them to V while CTA 0
//    already runs the next steps, and frees ring slots with a remote arrive.
//  * The congruence uses the compact WY form Q = I - Vh T Vh^H:
//      B = R - (Vh Z^H + Z Vh^H),   Z = (R Vh)T - 1/2 Vh(T^H (Vh^H R Vh) T),
//    an identity for any T, so B is exactly Q^H R Q for the Q that seeds the
//    eigenvectors.  The two CTAs split the rows of R Vh and the entries of B.
//  * The Jacobi sweeps keep A's upper triangle in pair-slot storage (by slot and
//    role of the round-robin ordering, see sl_bid / sl_move below): the pairs
//    of a step are the diagonal blocks, and every step rotates and moves the
//    whole triangle into a second buffer with fixed per-thread offsets.  Slot
//    threads form the next step's rotations while the block threads work, so a
//    step has one barrier.
//  * The thresholding rule runs on one warp (log10, gradients and curvature per
//    lane, argmax by shuffles) in double precision.
#include <cooperative_groups.h>
#include <math.h>

#include "evd_common.cuh"
#include "lcf_internal.cuh"

namespace cg = cooperative_groups;

namespace lcf {

constexpr int EP_THREADS = 512;
constexpr int EP_RING = 16;                   // rotation records in flight between the CTAs
constexpr float EP_TOL = 2.0e-6f;             // relative off-diagonal test
constexpr int EP_SUBSPACE_ITERS = 3;
constexpr unsigned EP_REC_ROT = 1u << 16, EP_REC_END = 1u << 17;
constexpr int EP_PLANE = (kEvdPairNmax / 2) * (kEvdPairNmax / 2 + 1) / 2;   // blocks per plane of the slot storage

struct EpArgs {
  int nt, nz, nx;
  int thresh_mode;
  double beta, beta_src;
  int k_fixed, k_src;
  int pd_mode, alpha_mode, curv_norm, max_sweeps;
  int ncp;
  int* err;
  long long* clk;   // [nd][kEvdPhases + 1] phase-boundary SM clocks of CTA 0 (profiling), or null
  int wz, wx;                       // window grid (the learned rule's position input)
  const __nv_bfloat16* mlp_w;       // learned rule: W1 | W2 | W3 | W4 (bf16)
  const float* mlp_b;               //               b1 | b2 | b3 | b4
  int mlp_h;                        // hidden width
  float mlp_pmin;                   // confidence threshold
  float* mlp_dbg;                   // [nd][2 nt + 2]: features, then logits (or null)
};

#define EP_STAMP(b)                                                                  \
  do {                                                                               \
    if (g.clk && tid == 0) g.clk[(size_t)k * (kEvdPhases + 1) + (b)] = clock64();     \
  } while (0)

// ---- shared-memory layout (both CTAs get the larger of the two) ----
struct EpLayout {
  int np, ld, ldy, m, h;
  size_t a, ys, zs, yd, zd, tm, w2, pr, prd, lam, perm, wts, s0, s1, s2, ebar, mlp, sinfo, end_a;   // CTA 0
  size_t vt, ring, vh, tv, vtm, fbar, rperm, rcoef, rkeep, phase, zcp, end_v;            // CTA 1
  size_t total;
};

__host__ __device__ inline size_t ep_align(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline EpLayout ep_layout(int n) {
  EpLayout L;
  L.np = n + (n & 1);
  L.ld = L.np + 1;
  L.ldy = L.np + 1;
  L.m = n < kEvdHead ? n : kEvdHead;
  L.h = L.np / 2;
  size_t o = 0;
  {
    const size_t dense = (size_t)L.np * L.ld * 8, slots = (size_t)2 * 4 * EP_PLANE * 8;
    L.a = o;  o = ep_align(o + (dense > slots ? dense : slots));   // R/scale in fp32, then two slot buffers
  }
  L.ys = o;   o = ep_align(o + (size_t)L.m * L.ldy * 8);      // subspace block, column-major
  L.zs = o;   o = ep_align(o + (size_t)L.m * L.ldy * 8);      // product block, then reflectors Vh
  L.yd = o;   o = ep_align(o + (size_t)n * L.m * 16);         // R Vh (double-float, [a][j])
  L.zd = o;   o = ep_align(o + (size_t)n * L.m * 16);         // Z
  L.tm = o;   o = ep_align(o + (size_t)L.m * L.m * 8);        // T (fp32 complex)
  L.w2 = o;   o = ep_align(o + (size_t)2 * L.m * L.m * 16);   // M T and T^H M T (double-float)
  L.pr = o;   o = ep_align(o + (size_t)2 * L.h * 16);         // rotation records (two steps)
  L.prd = o;  o = ep_align(o + (size_t)2 * L.h * 8);          // new diagonal pairs (two steps)
  L.lam = o;  o = ep_align(o + (size_t)L.np * 8);
  L.perm = o; o = ep_align(o + (size_t)L.np * 4);
  L.wts = o;  o = ep_align(o + (size_t)L.np * 8);
  L.s0 = o;   o = ep_align(o + (size_t)L.np * 8);
  L.s1 = o;   o = ep_align(o + (size_t)L.np * 8);
  L.s2 = o;   o = ep_align(o + (size_t)L.np * 8);
  L.ebar = o; o = ep_align(o + (size_t)EP_RING * 8);
  L.mlp = o;  o = ep_align(o + (size_t)(L.np + 2 + 2 * kMlpHiddenMax) * 4);   // learned rule: input, 2 activations
  L.sinfo = o; o = ep_align(o + (size_t)L.h * 3 * 16);       // per slot: fixed offsets of the Jacobi steps
  L.end_a = o;
  o = 0;
  L.vt = o;    o = ep_align(o + (size_t)L.np * L.ld * 8);     // V^T (row c = column c of V)
  L.ring = o;  o = ep_align(o + (size_t)EP_RING * L.h * 16);
  L.vh = o;    o = ep_align(o + (size_t)L.m * L.ldy * 8);     // reflectors (received)
  L.tv = o;    o = ep_align(o + (size_t)L.m * L.m * 8);       // T (received)
  L.vtm = o;   o = ep_align(o + (size_t)n * L.m * 8);         // Vh T
  L.fbar = o;  o = ep_align(o + (size_t)EP_RING * 8);
  L.rperm = o; o = ep_align(o + (size_t)L.np * 4);            // sorted -> original index
  L.rcoef = o; o = ep_align(o + (size_t)L.np * 4);            // wt * sqrt(alpha/Nt) per sorted index
  L.rkeep = o; o = ep_align(o + (size_t)(L.np + 1) * 4);      // [0] = ncol, then kept sorted indices
  L.phase = o; o = ep_align(o + (size_t)L.np * 8);
  L.zcp = o;   o = ep_align(o + (size_t)n * L.m * 16);        // Z (received for the congruence)
  L.end_v = o;
  L.total = (L.end_a > L.end_v ? L.end_a : L.end_v);
  return L;
}

size_t evd_pair_smem_bytes(int nt) { return ep_layout(nt).total; }

// ---- pair-slot storage of the Hermitian matrix during the Jacobi sweeps ----
// At step r slot i holds (first, second) = ((r + i) mod M, (r - i) mod M), slot 0 (r, M),
// M = np - 1.  Entry A[x][y] with x in slot a (role ra: 0 first, 1 second) and y in slot b
// (role rb) lives in block (a, b) when a < b, or a == b and ra <= rb, in plane 2 ra + rb at
// block index bid(a, b) (upper triangle of slots, row-wise); otherwise its conjugate lives
// in block (b, a), plane 2 rb + ra.  Plane 2 of a diagonal block is unused.  From one step to
// the next every first member moves down one slot and every second member up one (slot 0's
// first becomes slot 1's second, slot h-1's second becomes its first, M stays): the same
// permutation at every step, so each block's destinations are fixed.
__device__ __forceinline__ int sl_bid(int a, int b, int h) { return a * h - (a * (a - 1)) / 2 + (b - a); }
__device__ __forceinline__ void sl_move(int& sl, int& role, int h) {
  if (h == 1) return;
  if (role == 0) {
    if (sl == 0) { sl = 1; role = 1; }
    else --sl;
  } else if (sl == h - 1) {
    role = 0;
  } else if (sl > 0) {
    ++sl;
  }
}
// offset (float2 units within a buffer of 4 planes of nblk entries) of entry (x at (a, ra), y at (b, rb))
__device__ __forceinline__ int sl_off(int a, int ra, int b, int rb, int h, int nblk, bool& cj) {
  if (a < b || (a == b && ra <= rb)) { cj = false; return (2 * ra + rb) * nblk + sl_bid(a, b, h); }
  cj = true;
  return (2 * rb + ra) * nblk + sl_bid(b, a, h);
}
// slot and role of index x at step 0
__device__ __forceinline__ void sl_home(int x, int h, int& sl, int& role) {
  const int M = 2 * h - 1;
  if (x == M) { sl = 0; role = 1; }
  else if (x < h) { sl = x; role = 0; }
  else { sl = M - x; role = 1; }
}

// ---- the congruence B = Q^H R Q, shared by the two CTAs ----
// (h, l) += (ah + al) b: FMA two-product, Knuth two-sum of the high words, the
// rounding errors summed into the low word (renormalised once at the end).
__device__ __forceinline__ void ep_acc(float& h, float& l, float ah, float al, float b) {
  const float p = ah * b;
  const float e = fmaf(al, b, fmaf(ah, b, -p));
  const float s = h + p;
  const float bb = s - h;
  l += ((h - (s - bb)) + (p - bb)) + e;
  h = s;
}
// complex accumulator (re hi, re lo, im hi, im lo) += a * b, a double-float, b float
__device__ __forceinline__ void ep_cmac(float4& c, const zdf& a, float2 b) {
  ep_acc(c.x, c.y, a.re.hi, a.re.lo, b.x);
  ep_acc(c.x, c.y, -a.im.hi, -a.im.lo, b.y);
  ep_acc(c.z, c.w, a.re.hi, a.re.lo, b.y);
  ep_acc(c.z, c.w, a.im.hi, a.im.lo, b.x);
}
__device__ __forceinline__ zdf ep_cacc_zdf(float4 c) { return {quick_two_sum(c.x, c.y), quick_two_sum(c.z, c.w)}; }

// Rows [a0, a1) of Yd = (R / scale) Vh (n x m, double-float, [a][j]); 8 threads per row,
// each an eighth of the columns b, reduced by shuffles.  Vh column-major (stride ldy).
__device__ void ep_yd_rows(const double2* __restrict__ R, int n, int m, int ldy, float s_lo, const float2* Vh,
                           int a0, int a1, zdf* Yd, int tid) {
  for (int base = a0; base < a1; base += EP_THREADS / 8) {
    const int a = base + (tid >> 3), sub = tid & 7;
    float4 acc[kEvdHead];
#pragma unroll
    for (int j = 0; j < kEvdHead; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < a1) {
      double2 rn = sub < n ? R[(size_t)a * n + sub] : make_double2(0.0, 0.0);
      for (int b = sub; b < n; b += 8) {
        const double2 r = rn;
        if (b + 8 < n) rn = R[(size_t)a * n + b + 8];   // next column's entry in flight
        zdf rz;
        rz.re = df_from_double(r.x); rz.im = df_from_double(r.y);
        rz.re.hi *= s_lo; rz.re.lo *= s_lo; rz.im.hi *= s_lo; rz.im.lo *= s_lo;
#pragma unroll
        for (int j = 0; j < kEvdHead; ++j)
          if (j < m) ep_cmac(acc[j], rz, Vh[(size_t)j * ldy + b]);
      }
    }
#pragma unroll
    for (int j = 0; j < kEvdHead; ++j) {
      zdf v = ep_cacc_zdf(acc[j]);
      for (int o = 1; o < 8; o <<= 1) {
        zdf t;
        t.re.hi = __shfl_xor_sync(~0u, v.re.hi, o); t.re.lo = __shfl_xor_sync(~0u, v.re.lo, o);
        t.im.hi = __shfl_xor_sync(~0u, v.im.hi, o); t.im.lo = __shfl_xor_sync(~0u, v.im.lo, o);
        v = zdf_add(v, t);
      }
      if (sub == 0 && a < a1 && j < m) Yd[a * m + j] = v;
    }
  }
}

// Upper-triangle entries [e0, e1) (row-wise over np x np) of B = R - (Vh Z^H + Z Vh^H),
// rounded to fp32 and stored in pair-slot buffer S (step-0 places).
__device__ void ep_bfill(const double2* __restrict__ R, int n, int np, int h, int m, int ldy, float s_lo,
                         const zdf* Zd, const float2* Vh, int e0, int e1, float2* S, int tid) {
  const float two_np1 = (float)(2 * np + 1);
  for (int e = e0 + tid; e < e1; e += EP_THREADS) {
    // row a: the largest a with a np - a (a - 1) / 2 <= e
    int a = (int)floorf(0.5f * (two_np1 - sqrtf(fmaxf(two_np1 * two_np1 - 8.f * (float)e, 0.f))));
    a = a < 0 ? 0 : (a > np - 1 ? np - 1 : a);
    while (a > 0 && a * np - (a * (a - 1)) / 2 > e) --a;
    while (a + 1 < np && (a + 1) * np - ((a + 1) * a) / 2 <= e) ++a;
    const int b = a + (e - (a * np - (a * (a - 1)) / 2));
    float2 v = make_float2(0.f, 0.f);
    if (b < n) {
      const double2 r = R[(size_t)a * n + b];
      float4 c1 = make_float4(0.f, 0.f, 0.f, 0.f), c2 = c1;   // Vh Z^H and Z Vh^H terms
#pragma unroll
      for (int j = 0; j < kEvdHead; ++j) {
        if (j >= m) break;
        zdf zb = Zd[b * m + j];
        zb.im = df_neg(zb.im);
        ep_cmac(c1, zb, Vh[(size_t)j * ldy + a]);                 // Vh_aj conj(Z_bj)
        ep_cmac(c2, Zd[a * m + j], cconj(Vh[(size_t)j * ldy + b]));   // Z_aj conj(Vh_bj)
      }
      zdf x;
      x.re = df_from_double(r.x); x.im = df_from_double(r.y);
      x.re.hi *= s_lo; x.re.lo *= s_lo; x.im.hi *= s_lo; x.im.lo *= s_lo;
      const zdf t1 = ep_cacc_zdf(c1), t2 = ep_cacc_zdf(c2);
      x.re = df_add(x.re, df_neg(df_add(t1.re, t2.re)));
      x.im = df_add(x.im, df_neg(df_add(t1.im, t2.im)));
      v = make_float2(x.re.hi + x.re.lo, a == b ? 0.f : x.im.hi + x.im.lo);
    }
    int sa, ra, sb, rb;
    sl_home(a, h, sa, ra);
    sl_home(b, h, sb, rb);
    bool cj;
    const int o = sl_off(sa, ra, sb, rb, h, EP_PLANE, cj);
    S[o] = cj ? cconj(v) : v;
  }
}

// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(EP_THREADS, 1)
evd_pair_kernel(const double2* __restrict__ Rg, const Box* __restrict__ boxes, EpArgs g,
                double* __restrict__ lam_out, float2* __restrict__ V_out, float* __restrict__ wt_out,
                int* __restrict__ kcut_out, float* __restrict__ alpha_out, int* __restrict__ flags_out,
                float2* __restrict__ W_out, int* __restrict__ ncol_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int k = blockIdx.x >> 1, n = g.nt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const EpLayout L = ep_layout(n);
  const int np = L.np, ldy = L.ldy, m = L.m, h = L.h;
  const double2* R = Rg + (size_t)k * n * n;
  __shared__ double sh_scale;
  __shared__ int sh_ok[2];

  // ---------------- power-of-two scale (max diagonal) and degenerate check, both CTAs
  if (warp == 0) {
    double mx = 0.0;
    for (int i = lane; i < n; i += 32) mx = fmax(mx, R[(size_t)i * n + i].x);
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(~0u, mx, o));
    if (lane == 0) sh_scale = mx;
  }
  __syncthreads();
  const double dmax = sh_scale;
  if (!(dmax > 0.0) || !isfinite(dmax)) {
    if (rank == 0) {
      for (int i = tid; i < n; i += EP_THREADS) {
        lam_out[(size_t)k * n + i] = 0.0;
        wt_out[(size_t)k * n + i] = 0.f;
      }
      if (tid == 0) {
        kcut_out[k] = 0; alpha_out[k] = 0.f; ncol_out[k] = 0;
        flags_out[k] = LCF_WFLAG_DEGENERATE;
      }
    } else {
      for (int e = tid; e < n * n; e += EP_THREADS) V_out[(size_t)k * n * n + e] = make_float2(e / n == e % n, 0.f);
      for (int e = tid; e < n * g.ncp; e += EP_THREADS) W_out[(size_t)k * n * g.ncp + e] = make_float2(0.f, 0.f);
    }
    return;   // both CTAs leave before any cluster-level exchange
  }
  int ex;
  frexp(dmax, &ex);
  const double scale = ldexp(1.0, ex);            // R / scale is exact; its max diagonal is in [1/2, 1)
  const float s_lo = ldexpf(1.f, -ex);            // the same factor for the double-float words

  uint64_t* ebar = reinterpret_cast<uint64_t*>(smem + L.ebar);   // CTA 0: ring slots free
  uint64_t* fbar = reinterpret_cast<uint64_t*>(smem + L.fbar);   // CTA 1: ring slots full
  if (tid == 0) {
    if (rank == 0)
      for (int i = 0; i < EP_RING; ++i) ep_bar_init(&ebar[i], 1);
    else
      for (int i = 0; i < EP_RING; ++i) ep_bar_init(&fbar[i], 1);   // CTA 1's own expect_tx arrive
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster.sync();   // #0: barriers of both CTAs initialised
  const uint32_t peer = (uint32_t)(rank ^ 1);
  bool ok = true;

  if (rank == 0) {
    // =====================================================================
    // CTA 0: subspace, QR, congruence, Jacobi on A, sort and rule
    // =====================================================================
    float2* Rh = reinterpret_cast<float2*>(smem + L.a);    // phase A (np x np)
    float2* Ys = reinterpret_cast<float2*>(smem + L.ys);   // [j][a], stride ldy
    float2* Zs = reinterpret_cast<float2*>(smem + L.zs);
    zdf* Yd = reinterpret_cast<zdf*>(smem + L.yd);          // [a][j]
    zdf* Zd = reinterpret_cast<zdf*>(smem + L.zd);
    float2* Tm = reinterpret_cast<float2*>(smem + L.tm);   // [i][j]
    zdf* MT = reinterpret_cast<zdf*>(smem + L.w2);          // M T
    zdf* W2 = MT + m * m;                                   // T^H M T
    float4* pr = reinterpret_cast<float4*>(smem + L.pr);
    float2* prd = reinterpret_cast<float2*>(smem + L.prd);
    double* lam_s = reinterpret_cast<double*>(smem + L.lam);
    int* perm = reinterpret_cast<int*>(smem + L.perm);
    double* wts = reinterpret_cast<double*>(smem + L.wts);
    double* s0 = reinterpret_cast<double*>(smem + L.s0);
    double* s1 = reinterpret_cast<double*>(smem + L.s1);
    double* s2 = reinterpret_cast<double*>(smem + L.s2);
    __shared__ float betas[kEvdHead];

    EP_STAMP(0);
    // ---------------- phase A: subspace iteration on fp32(R / scale)
    const float inv_s = (float)(1.0 / scale);
    for (int e = tid; e < np * np; e += EP_THREADS) {
      const int a = e / np, b = e % np;
      float2 v = make_float2(0.f, 0.f);
      if (a < n && b < n) {
        const double2 r = R[(size_t)a * n + b];
        v = make_float2((float)r.x * inv_s, (float)r.y * inv_s);
      }
      Rh[e] = v;
    }
    for (int e = tid; e < m * ldy; e += EP_THREADS) {
      const int j = e / ldy, a = e % ldy;
      unsigned hsh = (unsigned)(a * 2654435761u) ^ (unsigned)(j * 40503u + 7u);
      hsh ^= hsh >> 13; hsh *= 0x5bd1e995u; hsh ^= hsh >> 15;
      const float re = (float)(hsh & 0xffff) / 65536.f - 0.5f, im = (float)(hsh >> 16) / 65536.f - 0.5f;
      Ys[e] = (a < n) ? make_float2(re, im) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    __shared__ float2 cs[kEvdHead];
    __shared__ float sh_nrm;
    for (int it = 0; it < EP_SUBSPACE_ITERS; ++it) {
      for (int e = tid; e < n * m; e += EP_THREADS) {   // Z = Rh Y (8 lanes share a row of Rh)
        const int a = e / m, j = e % m;
        float2 acc = make_float2(0.f, 0.f);
        const float2* rr = Rh + (size_t)a * np;
        const float2* yy = Ys + (size_t)j * ldy;
        for (int b = 0; b < n; ++b) {
          const float2 r = rr[b], y = yy[b];
          acc.x = fmaf(r.x, y.x, fmaf(-r.y, y.y, acc.x));
          acc.y = fmaf(r.x, y.y, fmaf(r.y, y.x, acc.y));
        }
        Zs[(size_t)j * ldy + a] = acc;
      }
      __syncthreads();
      // CGS2 of Z's columns into Y: dots on warps 0..j-1, updates on all threads
      for (int j = 0; j < m; ++j) {
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
          for (int a = tid; a < n; a += EP_THREADS) {
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
        if (nr > 0.f) {   // a vanishing direction keeps its previous (orthonormal) vector
          const float sc = rsqrtf(nr);
          for (int a = tid; a < n; a += EP_THREADS) Ys[(size_t)j * ldy + a] = cscale(zj[a], sc);
        }
        __syncthreads();
      }
    }

    EP_STAMP(1);
    // ---------------- phase B: Householder QR of Y (reflectors -> Zs), then T
    // Reflector j on warp 0; the columns after it updated by one warp each.
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
      const int c = j + warp;   // warps 1 .. m - 1 - j
      if (warp >= 1 && c < m) {
        float2* yc = Ys + (size_t)c * ldy;
        float2 t = make_float2(0.f, 0.f);
        for (int a = j + lane; a < n; a += 32) t = cadd(t, cmulc(vj[a], yc[a]));
        for (int o = 16; o; o >>= 1) { t.x += __shfl_xor_sync(~0u, t.x, o); t.y += __shfl_xor_sync(~0u, t.y, o); }
        t = cscale(t, betas[j]);
        for (int a = j + lane; a < n; a += 32) yc[a] = csub(yc[a], cmul(vj[a], t));
      }
      __syncthreads();
    }
    // compact WY: H_0 ... H_{m-1} = I - Vh T Vh^H with T upper triangular,
    // T[j][j] = beta_j, T[0:j, j] = -beta_j T[0:j, 0:j] (Vh[:, 0:j]^H v_j).
    // The products Vh[:, i]^H v_j (i < j) on all warps, then the recurrence on warp 0.
    __shared__ float2 vv[kEvdHead * kEvdHead];
    for (int q = warp; q < m * m; q += EP_THREADS / 32) {
      const int i = q / m, j = q % m;
      if (i >= j) continue;
      float2 cc = make_float2(0.f, 0.f);
      for (int a = lane; a < n; a += 32) cc = cadd(cc, cmulc(Zs[(size_t)i * ldy + a], Zs[(size_t)j * ldy + a]));
      for (int o = 16; o; o >>= 1) { cc.x += __shfl_xor_sync(~0u, cc.x, o); cc.y += __shfl_xor_sync(~0u, cc.y, o); }
      if (lane == 0) vv[q] = cc;
    }
    __syncthreads();
    if (warp == 0) {
      for (int j = 0; j < m; ++j) {
        if (lane < j) {
          float2 acc = make_float2(0.f, 0.f);
          for (int l = lane; l < j; ++l) acc = cadd(acc, cmul(Tm[lane * m + l], vv[l * m + j]));
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
    // send Vh (m x ldy, column-major) and T to CTA 1
    {
      const uint32_t vh_r = ep_mapa(ep_smem(smem + L.vh), peer), tv_r = ep_mapa(ep_smem(smem + L.tv), peer);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(Zs);
      for (int e = tid; e < 2 * m * ldy; e += EP_THREADS) ep_st_remote_u32(vh_r + 4u * e, src[e]);
      const uint32_t* ts = reinterpret_cast<const uint32_t*>(Tm);
      for (int e = tid; e < 2 * m * m; e += EP_THREADS) ep_st_remote_u32(tv_r + 4u * e, ts[e]);
    }
    cluster.sync();   // #1: CTA 1 may build Q
    EP_STAMP(2);

    // ---------------- phase C: B = Q^H R Q = R - (Vh Z^H + Z Vh^H) in double-float
    // Yd = (R / scale) Vh: rows [0, n / 2) here, the rest by CTA 1 into this CTA's Yd
    const int nA = (n + 1) / 2;
    ep_yd_rows(R, n, m, ldy, s_lo, Zs, 0, nA, Yd, tid);
    cluster.sync();   // #1b: every row of Yd is here
    // M = Vh^H Yd (m x m): warp w -> entries w, w + 16, ...
    zdf* Mm = Zd;   // Zd is free until Z is formed; M needs m*m <= n*m entries
    for (int q = warp; q < m * m; q += EP_THREADS / 32) {
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
    if (tid < m * m) {   // MT = M T
      const int i = tid / m, j = tid % m;
      zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
      for (int l = 0; l <= j; ++l) acc = zdf_add(acc, zdf_mul_c(Mm[i * m + l], Tm[l * m + j]));
      MT[tid] = acc;
    }
    __syncthreads();
    if (tid < m * m) {   // W2 = T^H (M T)
      const int i = tid / m, j = tid % m;
      zdf acc = {{0.f, 0.f}, {0.f, 0.f}};
      for (int l = 0; l <= i; ++l) acc = zdf_add(acc, zdf_mul_c(MT[l * m + j], cconj(Tm[l * m + i])));
      W2[tid] = acc;
    }
    __syncthreads();
    // Z = Yd T - 1/2 Vh W2   (n x m)
    for (int e = tid; e < n * m; e += EP_THREADS) {
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
    // Z to CTA 1; B's upper triangle split between the CTAs (fp32 pair-slot buffer 0, real diagonal)
    {
      zdf* zr = cluster.map_shared_rank(reinterpret_cast<zdf*>(smem + L.zcp), (unsigned)peer);
      for (int e = tid; e < n * m; e += EP_THREADS) zr[e] = Zd[e];
    }
    cluster.sync();   // #1c: Z is in CTA 1
    float2* S0 = reinterpret_cast<float2*>(smem + L.a);
    const int ne = np * (np + 1) / 2;
    ep_bfill(R, n, np, h, m, ldy, s_lo, Zd, Zs, 0, ne / 2, S0, tid);
    cluster.sync();   // #1d: CTA 1's half of B is here
    EP_STAMP(3);
    EP_STAMP(4);
    // ---------------- phase D: cyclic Jacobi in pair-slot storage; rotations streamed to CTA 1
    // Step r reads buffer par and writes every entry, rotated and moved to its step-(r+1)
    // place, into buffer par ^ 1.  Thread i < h owns slot i: it writes its diagonal block and,
    // during step r, already forms step r+1's rotation of slot i from the entries that step r
    // moves onto it (its off-diagonal comes from one element of one rotated block).  One
    // barrier per step.  Slot i runs on thread i of the first EP_SLOTW warps, which take no
    // off-diagonal blocks; the blocks (a < b) are spread over the other warps with fixed
    // source and destination offsets.
    constexpr int EP_SLOTW = (kEvdPairNmax / 2 + 31) / 32;     // warps holding the slots
    constexpr int BT = EP_THREADS - 32 * EP_SLOTW;              // threads holding blocks
    constexpr int MAXB = ((kEvdPairNmax / 2) * (kEvdPairNmax / 2 - 1) / 2 + BT - 1) / BT;
    // per block: source block id (bits 0-11, 0xfff: none), slots a (12-17) and b (18-23), conjugation
    // of entry q at bit 31 - q; destinations of entries 0, 1 and 2, 3 (16 bits each)
    unsigned binf[MAXB], bd01[MAXB], bd23[MAXB];
    {
      const int noff = h * (h - 1) / 2;
#pragma unroll
      for (int j = 0; j < MAXB; ++j) {
        const int e = (tid < 32 * EP_SLOTW) ? noff : tid - 32 * EP_SLOTW + j * BT;
        binf[j] = 0xfffu;
        bd01[j] = 0u;
        bd23[j] = 0u;
        if (e < noff) {
          int a = 0, rem = e;
          while (rem >= h - 1 - a) { rem -= h - 1 - a; ++a; }
          const int b = a + 1 + rem;
          binf[j] = (unsigned)sl_bid(a, b, h) | ((unsigned)a << 12) | ((unsigned)b << 18);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int a2 = a, r2 = q >> 1, b2 = b, s2 = q & 1;
            sl_move(a2, r2, h);
            sl_move(b2, s2, h);
            bool cj;
            const unsigned d = (unsigned)sl_off(a2, r2, b2, s2, h, EP_PLANE, cj);
            if (q < 2) bd01[j] |= d << (16 * q);
            else bd23[j] |= d << (16 * (q - 2));
            binf[j] |= (cj ? 0x80000000u : 0u) >> q;   // sign bit of entry q's imaginary part, shifted by q
          }
        }
      }
    }
    // slot thread i: its diagonal block, where the block's entries go, and where slot i's
    // members of the next step come from (slot, role) with the block holding their entry
    const int my_slot = tid;
    const bool is_slot = tid < h;
    int4* sinfo = reinterpret_cast<int4*>(smem + L.sinfo);   // [h][3]
    if (is_slot) {
      const int i = my_slot;
      int a0 = i, r0 = 0, a1 = i, r1 = 1;
      sl_move(a0, r0, h);
      sl_move(a1, r1, h);
      bool cj, dcj;
      const int dsrc = sl_bid(i, i, h);
      const int dd0 = sl_off(a0, r0, a0, r0, h, EP_PLANE, cj);
      const int dd3 = sl_off(a1, r1, a1, r1, h, EP_PLANE, cj);
      const int dd1 = sl_off(a0, r0, a1, r1, h, EP_PLANE, dcj);
      // inverse moves of (i, first) and (i, second)
      int sa = 0, ra = 0, sb = 0, rb = 1;
      if (h > 1) {
        if (i <= h - 2) { sa = i + 1; ra = 0; } else { sa = h - 1; ra = 1; }
        if (i >= 2) { sb = i - 1; rb = 1; } else if (i == 1) { sb = 0; rb = 0; } else { sb = 0; rb = 1; }
      }
      int la_a, la_b, la_el, la_cj;
      if (sa < sb) { la_a = sa; la_b = sb; la_el = 2 * ra + rb; la_cj = 0; }
      else { la_a = sb; la_b = sa; la_el = 2 * rb + ra; la_cj = 1; }
      // (diagonal block, its three destinations), (block with the next off-diagonal, element | flags),
      // (slot | role << 16 of the next first and second member's diagonal value)
      sinfo[3 * i] = make_int4(dsrc, dd0, dd1, dd3);
      sinfo[3 * i + 1] = make_int4(la_a, la_b, sl_bid(la_a, la_b, h), la_el | (dcj ? 4 : 0) | (la_cj << 3));
      sinfo[3 * i + 2] = make_int4(sa | (ra << 16), sb | (rb << 16), 0, 0);
    }
    __syncthreads();
    float4* pr2 = pr;                                     // [2][h] rotation records by step parity
    float2* pd2 = prd;                                    // [2][h] new diagonal pairs by step parity
    const int M = np - 1;
    const uint32_t ring_r = ep_mapa(ep_smem(reinterpret_cast<unsigned char*>(smem) + L.ring), peer);
    const uint32_t fbar_r = ep_mapa(ep_smem(reinterpret_cast<unsigned char*>(smem) + L.fbar), peer);
    constexpr int WT = EP_THREADS - 1;   // the thread that waits for free ring slots (no slot, few blocks)
    const float tol2 = EP_TOL * EP_TOL;
    int sweeps = 0, converged = 0, hand = 0, par = 0;
    const int maxsw = g.max_sweeps > 0 ? g.max_sweeps : 40;
    // slot thread state for the step about to run: rotation, new diagonal, old off-diagonal
    float4 rec = make_float4(1.f, 0.f, 0.f, 0.f);
    float sdp = 0.f, sdq = 0.f;
    float2 sbq = make_float2(0.f, 0.f);
    int srot = 0;
    for (; sweeps < maxsw && ok; ++sweeps) {
      int anyr;
      {
        // Sweep start (step-0 layout).  A sweep with no rotation leaves A unchanged, so it is
        // the same as testing every pair at once: do that instead of the sweep.
        const float2* cur = S0 + (size_t)par * 4 * EP_PLANE;
        if (tid == WT) sh_ok[0] = hand < EP_RING || ep_wait(&ebar[hand % EP_RING], ((hand / EP_RING) - 1) & 1);
        int big = 0;
#pragma unroll
        for (int j = 0; j < MAXB; ++j) {
          if ((binf[j] & 0xfffu) == 0xfffu) continue;
          const int a = (binf[j] >> 12) & 63, b = (binf[j] >> 18) & 63, so = binf[j] & 0xfffu;
          const float da0 = cur[sl_bid(a, a, h)].x, da1 = cur[3 * EP_PLANE + sl_bid(a, a, h)].x;
          const float db0 = cur[sl_bid(b, b, h)].x, db1 = cur[3 * EP_PLANE + sl_bid(b, b, h)].x;
          const float n00 = cabs2(cur[so]), n01 = cabs2(cur[EP_PLANE + so]);
          const float n10 = cabs2(cur[2 * EP_PLANE + so]), n11 = cabs2(cur[3 * EP_PLANE + so]);
          big |= (n00 > 0.f && n00 > tol2 * fabsf(da0 * db0)) | (n01 > 0.f && n01 > tol2 * fabsf(da0 * db1)) |
                 (n10 > 0.f && n10 > tol2 * fabsf(da1 * db0)) | (n11 > 0.f && n11 > tol2 * fabsf(da1 * db1));
        }
        srot = 0;
        if (is_slot) {   // step 0's rotation of slot i
          const int i = my_slot;
          const int dsrc = sinfo[3 * i].x;
          const float app = cur[dsrc].x, aqq = cur[3 * EP_PLANE + dsrc].x;
          sbq = cur[EP_PLANE + dsrc];
          float c;
          float2 st;
          ep_rotation2(app, aqq, sbq, EP_TOL, c, st, sdp, sdq, srot);
          const int f = i == 0 ? 0 : i, sc = i == 0 ? M : M - i;
          rec = make_float4(c, st.x, st.y, __uint_as_float((unsigned)f | ((unsigned)sc << 8) | (srot ? EP_REC_ROT : 0u)));
          pr2[i] = rec;
          pd2[i] = make_float2(sdp, sdq);
          big |= srot;
        }
        if (!__syncthreads_or(big)) { converged = 1; break; }
        anyr = __syncthreads_or(srot);
      }
      for (int r = 0; r < M; ++r) {
        const int pb = r & 1;
        if (!sh_ok[pb]) { ok = false; break; }   // the partner stopped consuming: give up
        const float2* cur = S0 + (size_t)par * 4 * EP_PLANE;
        float2* nxt = S0 + (size_t)(par ^ 1) * 4 * EP_PLANE;
        if (anyr) {
          if (is_slot) {   // hand the step's records to CTA 1
            const int slot = hand % EP_RING;
            ep_st_async(ring_r + (uint32_t)((slot * h + my_slot) * 16), rec, fbar_r + (uint32_t)(slot * 8));
          }
          ++hand;
        }
        // the ring slot of the next hand-off (checked by everyone after the step's barrier)
        if (tid == WT) sh_ok[pb ^ 1] = hand < EP_RING || ep_wait(&ebar[hand % EP_RING], ((hand / EP_RING) - 1) & 1);
        const float4* prc = pr2 + pb * h;
        int nrot = 0;
        if (is_slot) {
          const int i = my_slot;
          const int4 i0 = sinfo[3 * i], i1 = sinfo[3 * i + 1], i2 = sinfo[3 * i + 2];
          const int la_a = i1.x, la_b = i1.y, la_src = i1.z, la_el = i1.w & 3, la_pa = i2.x, la_pb = i2.y;
          const bool dcj = (i1.w & 4) != 0, la_cj = (i1.w & 8) != 0;
          nxt[i0.y] = make_float2(sdp, 0.f);
          nxt[i0.w] = make_float2(sdq, 0.f);
          nxt[i0.z] = srot ? make_float2(0.f, 0.f) : (dcj ? cconj(sbq) : sbq);
          if (r + 1 < M) {
            // step r+1's off-diagonal of slot i: element la_el of block (la_a, la_b) after step r
            float2 z;
            if (h == 1) {
              z = srot ? make_float2(0.f, 0.f) : sbq;
            } else {
              const float4 Ra = prc[la_a], Rb = prc[la_b];
              const int ec = la_el & 1, er = la_el >> 1;
              const float2 xa0 = cur[la_src], xa1 = cur[EP_PLANE + la_src];
              const float2 xb0 = cur[2 * EP_PLANE + la_src], xb1 = cur[3 * EP_PLANE + la_src];
              const float cb = Rb.x, ca = Ra.x;
              const float2 sb = make_float2(Rb.y, Rb.z), sa = make_float2(Ra.y, Ra.z);
              float2 y0, y1;   // column ec of the block after slot la_b's rotation (rows 0, 1)
              if (ec == 0) {
                y0 = csub(cscale(xa0, cb), cmul(cconj(sb), xa1));
                y1 = csub(cscale(xb0, cb), cmul(cconj(sb), xb1));
              } else {
                y0 = cadd(cmul(sb, xa0), cscale(xa1, cb));
                y1 = cadd(cmul(sb, xb0), cscale(xb1, cb));
              }
              z = er == 0 ? csub(cscale(y0, ca), cmul(sa, y1)) : cadd(cmul(cconj(sa), y0), cscale(y1, ca));
              if (la_cj) z = cconj(z);
            }
            const float2 da = pd2[pb * h + (la_pa & 0xffff)], db = pd2[pb * h + (la_pb & 0xffff)];
            const float app = (la_pa >> 16) ? da.y : da.x, aqq = (la_pb >> 16) ? db.y : db.x;
            float c, ndp, ndq;
            float2 st;
            ep_rotation2(app, aqq, z, EP_TOL, c, st, ndp, ndq, nrot);
            int f = r + 1, sc = M;   // original indices of slot i's members at step r+1
            if (i > 0) {
              f = r + 1 + i;
              if (f >= M) f -= M;
              sc = r + 1 - i;
              if (sc < 0) sc += M;
            }
            rec = make_float4(c, st.x, st.y, __uint_as_float((unsigned)f | ((unsigned)sc << 8) | (nrot ? EP_REC_ROT : 0u)));
            pr2[(pb ^ 1) * h + i] = rec;
            pd2[(pb ^ 1) * h + i] = make_float2(ndp, ndq);
            sdp = ndp;
            sdq = ndq;
            sbq = z;
          }
        }
        if (warp >= EP_SLOTW) {
#pragma unroll
          for (int j = 0; j < MAXB; ++j) {
            const unsigned bi = binf[j];
            if ((bi & 0xfffu) == 0xfffu) continue;
            const int so = bi & 0xfffu;
            float2 x00 = cur[so], x01 = cur[EP_PLANE + so], x10 = cur[2 * EP_PLANE + so], x11 = cur[3 * EP_PLANE + so];
            if (anyr) {
              const float4 ra = prc[(bi >> 12) & 63], rb = prc[(bi >> 18) & 63];
              if ((__float_as_uint(ra.w) | __float_as_uint(rb.w)) & EP_REC_ROT) {
                // columns by slot b's rotation, then rows by slot a's
                const float ca = ra.x, cb = rb.x;
                const float2 sa = make_float2(ra.y, ra.z), sb = make_float2(rb.y, rb.z);
                const float2 sbc = cconj(sb), sac = cconj(sa);
                const float2 y00 = csub(cscale(x00, cb), cmul(sbc, x01)), y01 = cadd(cmul(sb, x00), cscale(x01, cb));
                const float2 y10 = csub(cscale(x10, cb), cmul(sbc, x11)), y11 = cadd(cmul(sb, x10), cscale(x11, cb));
                x00 = csub(cscale(y00, ca), cmul(sa, y10));
                x01 = csub(cscale(y01, ca), cmul(sa, y11));
                x10 = cadd(cmul(sac, y00), cscale(y10, ca));
                x11 = cadd(cmul(sac, y01), cscale(y11, ca));
              }
            }
            x00.y = __uint_as_float(__float_as_uint(x00.y) ^ (bi & 0x80000000u));
            x01.y = __uint_as_float(__float_as_uint(x01.y) ^ ((bi << 1) & 0x80000000u));
            x10.y = __uint_as_float(__float_as_uint(x10.y) ^ ((bi << 2) & 0x80000000u));
            x11.y = __uint_as_float(__float_as_uint(x11.y) ^ ((bi << 3) & 0x80000000u));
            nxt[bd01[j] & 0xffffu] = x00;
            nxt[bd01[j] >> 16] = x01;
            nxt[bd23[j] & 0xffffu] = x10;
            nxt[bd23[j] >> 16] = x11;
          }
        }
        srot = nrot;
        anyr = __syncthreads_or(nrot);
        par ^= 1;
      }
      ok = __syncthreads_and(ok);
    }
    // the diagonal by original index: after whole sweeps every index is back at its step-0 place
    float* dg = reinterpret_cast<float*>(prd);   // np floats
    {
      const float2* fin = S0 + (size_t)par * 4 * EP_PLANE;
      for (int x = tid; x < np; x += EP_THREADS) {
        int sl, ro;
        sl_home(x, h, sl, ro);
        dg[x] = fin[3 * ro * EP_PLANE + sl_bid(sl, sl, h)].x;
      }
    }
    __syncthreads();
    // end-of-stream record
    {
      const int slot = hand % EP_RING;
      if (tid == 0 && ok && hand >= EP_RING) ok = ep_wait(&ebar[slot], ((hand / EP_RING) - 1) & 1);
      ok = __syncthreads_and(ok);
      if (ok && tid < h) {
        ep_st_async(ring_r + (uint32_t)((slot * h + tid) * 16), make_float4(0.f, 0.f, 0.f, __uint_as_float(EP_REC_END)),
                    fbar_r + (uint32_t)(slot * 8));
      }
    }

    EP_STAMP(5);
    // ---------------- phase E (CTA 0): sort, rule, alpha; results to CTA 1
    for (int i = tid; i < n; i += EP_THREADS) {
      const float di = dg[i];
      int rk = 0;
      for (int j = 0; j < n; ++j) {
        const float dj = dg[j];
        rk += (dj > di) || (dj == di && j < i);
      }
      perm[rk] = i;
    }
    __syncthreads();
    for (int i = tid; i < n; i += EP_THREADS) lam_s[i] = (double)dg[perm[i]] * scale;
    __syncthreads();
    EP_STAMP(6);
    __shared__ int sh_lk;
    __shared__ float sh_lp;
    if (g.thresh_mode == LCF_T_LEARNED) {
      // learned rule: features (method 1's curve on [0, 1], window centre) -> MLP -> argmax k
      float* xin = reinterpret_cast<float*>(smem + L.mlp);
      float* h1 = xin + np + 2;
      float* h2 = h1 + kMlpHiddenMax;
      const int H = g.mlp_h, nin = n + 2;
      if (warp == 0) {
        const double fl = lam_s[0] * n * 2.220446049250313e-16;
        const double y1 = log10(lam_s[0] > fl ? lam_s[0] : fl), yn = log10(lam_s[n - 1] > fl ? lam_s[n - 1] : fl);
        const double span = y1 - yn;
        for (int i = lane; i < n; i += 32) {
          const double y = log10(lam_s[i] > fl ? lam_s[i] : fl);
          xin[i] = span > 0 ? (float)((y - yn) / span) : 0.f;
        }
        if (lane == 0) {
          xin[n] = (float)(((k / g.wx) + 0.5) / g.wz);
          xin[n + 1] = (float)(((k % g.wx) + 0.5) / g.wx);
        }
      }
      __syncthreads();
      const __nv_bfloat16* W1 = g.mlp_w;
      const __nv_bfloat16* W2 = W1 + (size_t)H * nin;
      const __nv_bfloat16* W3 = W2 + (size_t)H * H;
      const __nv_bfloat16* W4 = W3 + (size_t)H * H;
      ep_dense(xin, nin, W1, g.mlp_b, h1, H, true, warp, lane, EP_THREADS / 32);
      __syncthreads();
      ep_dense(h1, H, W2, g.mlp_b + H, h2, H, true, warp, lane, EP_THREADS / 32);
      __syncthreads();
      ep_dense(h2, H, W3, g.mlp_b + 2 * H, h1, H, true, warp, lane, EP_THREADS / 32);
      __syncthreads();
      ep_dense(h1, H, W4, g.mlp_b + 3 * H, h2, n, false, warp, lane, EP_THREADS / 32);
      __syncthreads();
      if (g.mlp_dbg) {   // the window's network input and logits, for validation
        float* dbo = g.mlp_dbg + (size_t)k * (2 * n + 2);
        for (int i = tid; i < n + 2; i += EP_THREADS) dbo[i] = xin[i];
        for (int i = tid; i < n; i += EP_THREADS) dbo[n + 2 + i] = h2[i];
      }
      if (warp == 0) {   // argmax (first index on ties) and its softmax probability
        float mx = -INFINITY;
        int bi = 0x7fffffff;
        for (int i = lane; i < n; i += 32)
          if (h2[i] > mx) { mx = h2[i]; bi = i; }
        for (int o = 16; o; o >>= 1) {
          const float om = __shfl_xor_sync(~0u, mx, o);
          const int oi = __shfl_xor_sync(~0u, bi, o);
          if (om > mx || (om == mx && oi < bi)) { mx = om; bi = oi; }
        }
        float se = 0.f;
        for (int i = lane; i < n; i += 32) se += expf(h2[i] - mx);
        for (int o = 16; o; o >>= 1) se += __shfl_xor_sync(~0u, se, o);
        if (lane == 0) { sh_lk = bi; sh_lp = 1.f / se; }
      }
      __syncthreads();
    }
    if (warp == 0) {
      int kk = -1, fallback = 0;
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
      } else if (md == LCF_T_LEARNED) {
        if (sh_lp >= g.mlp_pmin) {
          kk = sh_lk;
        } else {
          kk = ep_rule_k(g.k_src, lam_s, n, g.beta_src, g.k_fixed, g.curv_norm, s0, s1, s2, lane);
          fallback = 1;
        }
        for (int i = lane; i < n; i += 32) wts[i] = (i + 1 > kk) ? 1.0 : 0.0;
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
      if (lane == 0) {
        const double pdsum = g.pd_mode == 0 ? S / n : S;
        double al;
        int fl = (converged ? 0 : LCF_WFLAG_NOCONV) | (fallback ? LCF_WFLAG_FALLBACK : 0) |
                 ((sweeps < 255 ? sweeps : 255) << LCF_WFLAG_SWEEP_SHIFT);
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
        s0[0] = sqrt(al * (g.pd_mode == 0 ? 1.0 / n : 1.0));
      }
      __syncwarp();
      // kept columns in sorted order (ballot prefix)
      const double cf = s0[0];
      int base = 0;
      const uint32_t rk_r = ep_mapa(ep_smem(smem + L.rkeep), peer);
      const uint32_t rc_r = ep_mapa(ep_smem(smem + L.rcoef), peer);
      for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool keep = i < n && wts[i] > 0.0;
        const unsigned bal = __ballot_sync(~0u, keep);
        if (keep) ep_st_remote_u32(rk_r + 4u * (1 + base + __popc(bal & ((1u << lane) - 1u))), (uint32_t)i);
        if (i < n) ep_st_remote_u32(rc_r + 4u * i, __float_as_uint((float)(wts[i] * cf)));
        base += __popc(bal);
      }
      if (lane == 0) {
        ep_st_remote_u32(rk_r, (uint32_t)base);
        ncol_out[k] = base;
      }
    }
    {
      const uint32_t rp_r = ep_mapa(ep_smem(smem + L.rperm), peer);
      for (int i = tid; i < n; i += EP_THREADS) ep_st_remote_u32(rp_r + 4u * i, (uint32_t)perm[i]);
    }
    __syncthreads();
    for (int i = tid; i < n; i += EP_THREADS) {
      lam_out[(size_t)k * n + i] = lam_s[i];
      wt_out[(size_t)k * n + i] = (float)wts[i];
    }
    if (!ok && tid == 0) atomicOr(g.err, 1);
    __syncthreads();
    EP_STAMP(7);
    cluster.sync();   // #2: sorted order, coefficients and kept list are in CTA 1
    EP_STAMP(8);
  } else {
    // =====================================================================
    // CTA 1: V = Q, the streamed rotations, phase fix, V and W out
    // =====================================================================
    float2* Vt = reinterpret_cast<float2*>(smem + L.vt);
    const int ldv = np;   // even: entries (rr, rr + 1) of a row of V^T form one 16-byte word
    const float4* ring = reinterpret_cast<const float4*>(smem + L.ring);
    const float2* Vh = reinterpret_cast<const float2*>(smem + L.vh);
    const float2* Tv = reinterpret_cast<const float2*>(smem + L.tv);
    float2* VT = reinterpret_cast<float2*>(smem + L.vtm);
    cluster.sync();   // #1: reflectors and T have arrived
    {   // rows [n / 2, n) of Yd into CTA 0
      zdf* ydr = cluster.map_shared_rank(reinterpret_cast<zdf*>(smem + L.yd), (unsigned)peer);
      ep_yd_rows(R, n, m, ldy, s_lo, Vh, (n + 1) / 2, n, ydr, tid);
    }
    cluster.sync();   // #1b
    for (int e = tid; e < n * m; e += EP_THREADS) {   // VT = Vh T   ([a][j])
      const int a = e / m, j = e % m;
      float2 acc = make_float2(0.f, 0.f);
      for (int l = 0; l <= j; ++l) acc = cadd(acc, cmul(Vh[(size_t)l * ldy + a], Tv[l * m + j]));
      VT[e] = acc;
    }
    __syncthreads();
    // Vt[c][a] = Q[a][c] = delta_ac - sum_j VT[a][j] conj(Vh[c][j])
    for (int e = tid; e < np * ldv; e += EP_THREADS) {
      const int c = e / ldv, a = e % ldv;
      float2 v = make_float2(c == a ? 1.f : 0.f, 0.f);
      if (a < n && c < n)
        for (int j = 0; j < m; ++j) v = csub(v, cmul(VT[a * m + j], cconj(Vh[(size_t)j * ldy + c])));
      Vt[e] = v;
    }
    cluster.sync();   // #1c: Z has arrived
    {   // the second half of B's upper triangle into CTA 0's pair-slot buffer 0
      float2* s0r = cluster.map_shared_rank(reinterpret_cast<float2*>(smem + L.a), (unsigned)peer);
      const int ne = np * (np + 1) / 2;
      ep_bfill(R, n, np, h, m, ldy, s_lo, reinterpret_cast<const zdf*>(smem + L.zcp), Vh, ne / 2, ne, s0r, tid);
    }
    cluster.sync();   // #1d
    // work: warp w takes the pairs w, w + 16, w + 32, w + 48 of every step (one record per
    // pair, read by all lanes), lane l the entries (2l, 2l + 1) and (2l + 64, 2l + 65) of the
    // pair's two rows of V^T
    constexpr int VPW = (kEvdPairNmax / 2 + EP_THREADS / 32 - 1) / (EP_THREADS / 32);   // pairs per warp
    static_assert(2 * 32 * 2 >= kEvdPairNmax, "two 16-byte words per lane cover a row of V^T");
    __shared__ int sh_vok;
    const uint32_t ebar_r = ep_mapa(ep_smem(smem + L.ebar), peer);
    for (int hs = 0;; ++hs) {
      const int slot = hs % EP_RING;
      if (tid == 0) {   // one thread polls; the others acquire the completed phase after the barrier
        ep_arrive_expect_tx(&fbar[slot], (uint32_t)(h * 16));   // the step's h records
        sh_vok = ep_wait(&fbar[slot], (hs / EP_RING) & 1);
      }
      __syncthreads();
      ok = sh_vok != 0;
      if (!ok) break;
      ep_try(&fbar[slot], (hs / EP_RING) & 1);
      const float4* rs = ring + (size_t)slot * h;
      if (__float_as_uint(rs[0].w) & EP_REC_END) break;
      // every record and V entry of the warp's pairs is loaded before any is written
      float4 rc[VPW];
#pragma unroll
      for (int u = 0; u < VPW; ++u) {
        const int ia = warp + u * (EP_THREADS / 32);
        rc[u] = ia < h ? rs[ia] : make_float4(1.f, 0.f, 0.f, 0.f);
      }
      float4 P4[VPW][2], Q4[VPW][2];
      int po[VPW], qo[VPW];
#pragma unroll
      for (int u = 0; u < VPW; ++u) {
        const unsigned mt = __float_as_uint(rc[u].w);
        po[u] = (int)(mt & 255) * ldv + 2 * lane;
        qo[u] = (int)((mt >> 8) & 255) * ldv + 2 * lane;
        if (mt & EP_REC_ROT) {
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            if (lane + 32 * t < h) {
              P4[u][t] = *reinterpret_cast<const float4*>(Vt + po[u] + 64 * t);
              Q4[u][t] = *reinterpret_cast<const float4*>(Vt + qo[u] + 64 * t);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < VPW; ++u) {
        if (!(__float_as_uint(rc[u].w) & EP_REC_ROT)) continue;
        const float c = rc[u].x;
        const float2 s = make_float2(rc[u].y, rc[u].z), sc = cconj(s);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (lane + 32 * t >= h) continue;
          const float2 vp0 = make_float2(P4[u][t].x, P4[u][t].y), vp1 = make_float2(P4[u][t].z, P4[u][t].w);
          const float2 vq0 = make_float2(Q4[u][t].x, Q4[u][t].y), vq1 = make_float2(Q4[u][t].z, Q4[u][t].w);
          const float2 np0 = csub(cscale(vp0, c), cmul(sc, vq0)), np1 = csub(cscale(vp1, c), cmul(sc, vq1));
          const float2 nq0 = cadd(cmul(s, vp0), cscale(vq0, c)), nq1 = cadd(cmul(s, vp1), cscale(vq1, c));
          *reinterpret_cast<float4*>(Vt + po[u] + 64 * t) = make_float4(np0.x, np0.y, np1.x, np1.y);
          *reinterpret_cast<float4*>(Vt + qo[u] + 64 * t) = make_float4(nq0.x, nq0.y, nq1.x, nq1.y);
        }
      }
      __syncthreads();
      if (tid == 0) ep_arrive_remote(ebar_r + (uint32_t)(slot * 8));
    }
    if (!ok && tid == 0) atomicOr(g.err, 1);
    cluster.sync();   // #2: sorted order and coefficients from CTA 0
    const int* rperm = reinterpret_cast<const int*>(smem + L.rperm);
    const float* rcoef = reinterpret_cast<const float*>(smem + L.rcoef);
    const int* rkeep = reinterpret_cast<const int*>(smem + L.rkeep);
    float2* phs = reinterpret_cast<float2*>(smem + L.phase);
    // phase of each sorted eigenvector: largest-magnitude entry made real positive
    for (int jj = warp; jj < n; jj += EP_THREADS / 32) {
      const int col = rperm[jj];
      float best = -1.f;
      int bi = 0;
      for (int a = lane; a < n; a += 32) {
        const float mg = cabs2(Vt[col * ldv + a]);
        if (mg > best) { best = mg; bi = a; }
      }
      for (int o = 16; o; o >>= 1) {
        const float ob = __shfl_xor_sync(~0u, best, o);
        const int oi = __shfl_xor_sync(~0u, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        const float2 v = Vt[col * ldv + bi];
        const float mg = sqrtf(cabs2(v));
        phs[jj] = mg > 0.f ? make_float2(v.x / mg, -v.y / mg) : make_float2(1.f, 0.f);
      }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += EP_THREADS) {
      const int a = e / n, jj = e % n;
      V_out[(size_t)k * n * n + e] = cmul(Vt[rperm[jj] * ldv + a], phs[jj]);
    }
    const int nc = rkeep[0];
    for (int e = tid; e < n * g.ncp; e += EP_THREADS) {
      const int t = e / g.ncp, c = e % g.ncp;
      float2 v = make_float2(0.f, 0.f);
      if (c < nc) {
        const int jj = rkeep[1 + c];
        v = cscale(cmul(Vt[rperm[jj] * ldv + t], phs[jj]), rcoef[jj]);
      }
      W_out[(size_t)k * n * g.ncp + e] = v;
    }
  }
}

cudaError_t launch_evd_pair(const lcf_plan* P, cudaStream_t st) {
  EpArgs a;
  const lcf_config& c = P->cfg;
  a.nt = P->nt; a.nz = c.nz; a.nx = c.nx;
  a.thresh_mode = c.thresh_mode; a.beta = c.beta; a.beta_src = c.beta_src;
  a.k_fixed = c.k_fixed; a.k_src = c.k_src; a.pd_mode = c.pd_mode; a.alpha_mode = c.alpha_mode;
  a.curv_norm = c.curv_norm; a.max_sweeps = c.max_sweeps; a.ncp = P->ncp;
  a.err = P->ws.err;
  a.clk = P->profiling ? P->ws.evd_clk : nullptr;
  a.wz = c.wz; a.wx = c.wx;
  a.mlp_w = P->ws.mlp_w; a.mlp_b = P->ws.mlp_b; a.mlp_h = P->mlp_hidden; a.mlp_pmin = P->mlp_pmin;
  a.mlp_dbg = P->ws.mlp_dbg;
  evd_pair_kernel<<<2 * P->nd, EP_THREADS, evd_pair_smem_bytes(P->nt), st>>>(
      P->ws.R, P->ws.box, a, P->ws.lam, P->ws.V, P->ws.wt, P->ws.kcut, P->ws.alpha, P->ws.flags, P->ws.W,
      P->ws.ncol);
  return counted(P);
}

cudaError_t evd_pair_configure() {
  return cudaFuncSetAttribute(evd_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)evd_pair_smem_bytes(kEvdPairNmax));
}

}  // namespace lcf
