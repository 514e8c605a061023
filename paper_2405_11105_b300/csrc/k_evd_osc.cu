// k_evd_osc.cu — batched Hermitian EVD (Eq. 2) by one-sided Jacobi on a Cholesky
// factor for packets longer than one SM holds (128 < Nt <= 224), on a cluster of
// four CTAs per window.
//
// Same numerical plan as the one-CTA kernel (k_evd_os.cu): B = Q^H (R / scale) Q
// from the distributed EVD's prep kernel (FP32 subspace iteration, Householder QR,
// double-float congruence), its pivoted FP32 Cholesky factor L, one-sided Jacobi
// (Hestenes) on the columns of F = P L until every pair of columns is orthogonal to
// the relative tolerance, eigenvalue = squared column norm, eigenvector = column /
// norm, V = Q U, sort, rules, alpha, phase fix, W.
//
//  evd_chol_kernel   one CTA per window: the packed lower triangle of B in shared
//                    memory, factored right-looking with diagonal pivoting and no
//                    interchanges (every thread on each column, the trailing triangle
//                    updated per block of eight columns); L (pivot row order), the
//                    permutation and the numerical rank to global memory.
//  evd_osc_kernel    the sweeps and everything after, on a cluster of four CTAs.  CTA
//                    c holds rows [c R, (c + 1) R) (R = ceil(Nt / 4)) of every column in
//                    registers, lane l rows l and l + 32 of the CTA's share as one
//                    packed pair; the columns (zero-padded to 16 per warp) form blocks of
//                    eight, two per warp, in a block ordering: a round is eight steps in
//                    which each warp meets all pairs of its two blocks, then the blocks
//                    move one place on the circle through shared memory.  A step sums
//                    each slot's partial 2x2 Gram over the warp (reduce-scatter), sends
//                    that partial to the same warp of the other three CTAs (st.async into
//                    their shared memory, completing the bytes of that warp's
//                    step-parity mbarrier), adds the four partials in rank order (so
//                    every CTA forms the same rotations) and rotates.  Every wait is
//                    bounded (2 s).
#include <cooperative_groups.h>
#include <math.h>

#include "evd_common.cuh"
#include "lcf_internal.cuh"

namespace cg = cooperative_groups;

namespace lcf {

constexpr int EC_THREADS = 1024;               // Cholesky kernel
constexpr int EQ_C = 4;                        // CTAs per window of the sweeps
static_assert((EQ_C & (EQ_C - 1)) == 0, "cluster ranks wrap by masking");
constexpr float EQ_TOL = 2.0e-6f;              // relative orthogonality test
constexpr int EQ_SUBSPACE_ITERS = 6;

// ---------------------------------------------------------------------------------------------
// evd_chol_kernel: packed lower triangle (i, c <= i) at i (i + 1) / 2 + c.  Right-looking
// Cholesky with diagonal pivoting and no interchanges (the one-CTA kernel's scheme): step j takes
// as pivot the remaining index p with the largest diagonal of the Schur complement (every warp
// finds it from the list of remaining indices and their diagonal, double-buffered by step
// parity), writes column j of the factor over p's column of the complement (conjugated where the
// pair lies above the diagonal) and the square root of the pivot on p's diagonal; columns go in
// blocks of EC_CB, each column subtracting the block's earlier columns from its stored entries,
// the remaining triangle taking the block's rank-EC_CB update in one pass over its pairs.  Out: L
// with rows in pivot order (the indices eliminated at steps 0, 1, ..., then the remaining ones)
// and that permutation.
__host__ __device__ inline size_t ec_tri(int n) { return (size_t)n * (n + 1) / 2; }
constexpr int EC_CB = 8;
size_t evd_chol_smem_bytes(int n) {
  return ec_tri(n) * 8 + (size_t)EC_CB * n * 8 + (size_t)2 * n * 4 * 2 + (size_t)2 * n * 4 + 64;
}

__global__ void __launch_bounds__(EC_THREADS, 1)
evd_chol_kernel(float2* __restrict__ Bg, const double* __restrict__ scale_g, int n, int* __restrict__ perm_g,
                int* __restrict__ rank_g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = EC_THREADS;
  float2* A = reinterpret_cast<float2*>(smem);                            // packed lower triangle
  float2* gv = A + ec_tri(n);                                             // the block's columns, [EC_CB][n]
  float* dgb = reinterpret_cast<float*>(gv + (size_t)EC_CB * n);          // diagonal by list position, [2][n]
  int* remb = reinterpret_cast<int*>(dgb + 2 * n);                        // remaining indices, [2][n]
  int* pos = remb + 2 * n;                                                // step that eliminated each index
  int* ord = pos + n;                                                     // index eliminated at each step
  int* perm = perm_g + (size_t)k * n;
  float2* B = Bg + (size_t)k * n * n;
  if (!(scale_g[k] > 0.0)) {   // degenerate window: the sweep kernel writes the empty result
    if (tid == 0) rank_g[k] = 0;
    return;
  }
  for (int i = warp; i < n; i += nthr / 32)
    for (int c = lane; c <= i; c += 32) A[ec_tri(i) + c] = B[(size_t)i * n + c];
  for (int i = tid; i < n; i += nthr) { dgb[i] = B[(size_t)i * n + i].x; remb[i] = i; pos[i] = n; }
  __syncthreads();
  auto S = [&](int r, int c) -> float2* { return r > c ? &A[ec_tri(r) + c] : &A[ec_tri(c) + r]; };
  int rk = n;
  {
    float first = 0.f;
    bool stop = false;
    for (int j0 = 0; j0 < n && !stop; j0 += EC_CB) {
      const int j1 = j0 + EC_CB < n ? j0 + EC_CB : n;
      int j = j0;
      for (; j < j1; ++j) {
        const int cnt = n - j, par = j & 1, t = j - j0;
        const int* rin = remb + par * n;
        int* rout = remb + (par ^ 1) * n;
        const float* din = dgb + par * n;
        float* dout = dgb + (par ^ 1) * n;
        constexpr int NQ = (kEvdOscNmax + 31) / 32;
        float best = -INFINITY;   // the largest remaining diagonal entry, ties to the lower list position
        int ba = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int a = lane + 32 * q;
          const float d = a < cnt ? din[a] : -INFINITY;
          if (d > best) { best = d; ba = a; }
        }
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
            A[ec_tri(p) + p] = make_float2(best * inv, 0.f);
            ord[j] = p;
            pos[p] = j;
          } else {
            float2* e = S(r, p);
            float2 v = r > p ? *e : cconj(*e);
            for (int u = 0; u < t; ++u) v = csub(v, cmul(gv[u * n + r], cconj(gv[u * n + p])));
            const float2 g = cscale(v, inv);
            *e = r > p ? g : cconj(g);
            gv[t * n + r] = g;
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
      const int* rl = remb + (j & 1) * n;
      const int npair = cnt * (cnt - 1) / 2;
      for (int e = tid; e < npair; e += nthr) {
        int a = (int)(0.5f * (1.f + sqrtf(8.f * (float)e + 1.f)));
        if (a * (a - 1) / 2 > e) --a;
        else if ((a + 1) * a / 2 <= e) ++a;
        const int b = e - a * (a - 1) / 2;
        const int r = rl[a], c = rl[b];
        const int hi = r > c ? r : c, lo = r > c ? c : r;
        float2 acc = A[ec_tri(hi) + lo];
        for (int u = 0; u < nb; ++u) acc = csub(acc, cmul(gv[u * n + hi], cconj(gv[u * n + lo])));
        A[ec_tri(hi) + lo] = acc;
      }
      __syncthreads();
    }
  }
  // the permutation: the eliminated indices in step order, then the remaining ones (a stop at step
  // rk leaves them in list parity rk & 1)
  for (int i = tid; i < n; i += nthr) perm[i] = i < rk ? ord[i] : remb[(rk & 1) * n + (i - rk)];
  __syncthreads();
  // L (rows in pivot order) over B: zero above the diagonal and from column rk on; row i of L is
  // row perm[i] of the factor, whose column c (pivot pc) is S(perm[i], pc) below the pivot's step
  for (int e = tid; e < n * n; e += nthr) {
    const int i = e / n, c = e % n;
    float2 v = make_float2(0.f, 0.f);
    if (c <= i && c < rk) {
      const int r = perm[i], pc = ord[c];
      v = r == pc ? A[ec_tri(r) + r] : (r > pc ? A[ec_tri(r) + pc] : cconj(A[ec_tri(pc) + r]));
    }
    B[e] = v;
  }
  if (tid == 0) rank_g[k] = rk;
}



struct EqArgs {
  int nt, nz, nx;
  int thresh_mode;
  double beta, beta_src;
  int k_fixed, k_src;
  int pd_mode, alpha_mode, curv_norm, max_sweeps;
  int ncp;
  int* err;
};

__host__ __device__ inline size_t eq_align(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline size_t eq_xq_bytes(int nw) { return (size_t)nw * 16 * 32 * 16; }

struct EqLayout {
  int np, h, nw, R, lda, m;
  size_t u, x, lamp, lam, sperm, perm, lams, wts, s0, s1, s2, coef, keep, phs, cmax, vh, tm, y, bar, end;
};
// u: this CTA's rows of the columns (then of U, then of V); x: the sweeps' exchange buffers, later
// the partial products Vh^H U of every CTA
__host__ __device__ inline EqLayout eq_layout(int n) {
  EqLayout L;
  // two blocks of eight columns per warp; zero columns past Nt
  L.nw = (n + 15) / 16;
  L.np = 16 * L.nw;
  L.h = L.np / 2;
  L.R = (n + EQ_C - 1) / EQ_C;
  L.lda = L.np + 1;
  L.m = n < kEvdHead ? n : kEvdHead;
  size_t o = 0;
  L.u = o;     o = eq_align(o + (size_t)L.R * L.lda * 8);
  {
    // the sweeps' buffers overlay u and x from u's start: the block exchange [warp][column 0..15]
    // [lane] (float4), then the partial sums [parity][source rank][warp][lane] (float)
    const size_t sweep = eq_xq_bytes(L.nw) + (size_t)2 * EQ_C * L.nw * 32 * 4;
    const size_t post = (size_t)EQ_C * L.m * L.np * 8;
    size_t need = sweep > o ? sweep - o : 0;
    need = need > post ? need : post;
    L.x = o;   o = eq_align(o + need);
  }
  L.lamp = o;  o = eq_align(o + (size_t)EQ_C * L.np * 8);
  L.lam = o;   o = eq_align(o + (size_t)L.np * 8);
  L.sperm = o; o = eq_align(o + (size_t)L.np * 4);
  L.perm = o;  o = eq_align(o + (size_t)L.np * 4);
  L.lams = o;  o = eq_align(o + (size_t)L.np * 8);
  L.wts = o;   o = eq_align(o + (size_t)L.np * 8);
  L.s0 = o;    o = eq_align(o + (size_t)L.np * 8);
  L.s1 = o;    o = eq_align(o + (size_t)L.np * 8);
  L.s2 = o;    o = eq_align(o + (size_t)L.np * 8);
  L.coef = o;  o = eq_align(o + (size_t)L.np * 4);
  L.keep = o;  o = eq_align(o + (size_t)(L.np + 1) * 4);
  L.phs = o;   o = eq_align(o + (size_t)L.np * 8);
  L.cmax = o;  o = eq_align(o + (size_t)EQ_C * L.np * 16);
  L.vh = o;    o = eq_align(o + (size_t)L.m * n * 8);
  L.tm = o;    o = eq_align(o + (size_t)L.m * L.m * 8);
  L.y = o;     o = eq_align(o + (size_t)L.m * L.np * 8);
  L.bar = o;   o = eq_align(o + (size_t)2 * L.nw * 8);   // one mbarrier per step parity and warp
  L.end = o;
  return L;
}
size_t evd_osc_smem_bytes(int nt) { return eq_layout(nt).end; }

// ---------------------------------------------------------------------------------------------
// evd_osc_kernel: the sweeps on a cluster of EQ_C CTAs
struct EqCtx {
  // As few registers as the sweep loop can live with (it keeps every column in registers and
  // runs near the 128-register bound): 32-bit shared addresses, the rest derived.
  uint32_t recv_s;       // float [parity][source rank][warp][lane]: the other CTAs' partial sums
  uint32_t bar_s;        // this CTA's mbarriers [parity][warp]
  int nw, warp, lane, rank;
  float clim2, slim2;    // squared cosine and sine bounds of a calm step (ep_rotation_os)
  __device__ __forceinline__ uint32_t bar(int par) const { return bar_s + (uint32_t)((par * nw + warp) * 8); }
};
// the partial-sum bytes a warp's step brings in: one float per lane from each other CTA
constexpr uint32_t EQ_STEP_BYTES = (EQ_C - 1) * 32 * 4;

// plain (compiler-scheduled) shared-memory accesses by 32-bit shared address
__device__ __forceinline__ void eq_sts4(uint32_t a, float4 v) {
  *reinterpret_cast<float4*>(__cvta_shared_to_generic(a)) = v;
}
__device__ __forceinline__ float4 eq_lds4(uint32_t a) {
  return *reinterpret_cast<const float4*>(__cvta_shared_to_generic(a));
}
__device__ __forceinline__ float eq_lds(uint32_t a) {
  return *reinterpret_cast<const float*>(__cvta_shared_to_generic(a));
}
__device__ __forceinline__ void eq_arrive_expect_tx(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
// wait on this CTA's mbarrier at address b with acquire at cluster scope, for at most EP_WAIT_NS
// of wall time; false if the limit ran out
__device__ __forceinline__ bool eq_try(uint32_t b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred q;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 q, [%1], %2;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(done)
      : "r"(b), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool eq_wait(uint32_t b, uint32_t parity) {
  if (eq_try(b, parity)) return true;
  const uint64_t t0 = ep_now();
  for (;;) {
    if (eq_try(b, parity)) return true;
    if (ep_now() - t0 > EP_WAIT_NS) return false;
  }
}
__device__ __forceinline__ void eq_st_async_f32(uint32_t addr, float v, uint32_t bar_cluster_addr) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(addr), "r"(__float_as_uint(v)), "r"(bar_cluster_addr) : "memory");
}

// this warp's partial sum at byte offset off of CTA q's recv, completing bytes of the mbarrier of
// the same warp and parity in CTA q
__device__ __forceinline__ void eq_send(const EqCtx& x, uint32_t off, int par, int q, float part) {
  eq_st_async_f32(ep_mapa(x.recv_s + off, (uint32_t)q), part, ep_mapa(x.bar(par), (uint32_t)q));
}

// The reduce-scatter of 32 partial sums (value 4 s + c: slot s, component c) after its first level
// (w16[q] = value q + value q + 16 on lanes without bit 4, value q + 16 + value q on the others):
// lane l receives the warp's sum of value l
__device__ __forceinline__ float eq_reduce_scatter_rest(const float (&w16)[16], int lane) {
  float w8[8], w4[4], w2[2];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool hi = lane & 8;
    w8[q] = (hi ? w16[8 + q] : w16[q]) + __shfl_xor_sync(~0u, hi ? w16[q] : w16[8 + q], 8);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool hi = lane & 4;
    w4[q] = (hi ? w8[4 + q] : w8[q]) + __shfl_xor_sync(~0u, hi ? w8[q] : w8[4 + q], 4);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool hi = lane & 2;
    w2[q] = (hi ? w4[2 + q] : w4[q]) + __shfl_xor_sync(~0u, hi ? w4[q] : w4[2 + q], 2);
  }
  const bool hi = lane & 1;
  return (hi ? w2[1] : w2[0]) + __shfl_xor_sync(~0u, hi ? w2[0] : w2[1], 1);
}

// |top|^2, |bottom|^2, Re and Im of conj(top) bottom over the lane's two rows
__device__ __forceinline__ void eq_gram(float2 tr, float2 ti, float2 br, float2 bi, float (&u)[4]) {
  float2 a2 = __fmul2_rn(tr, tr);
  a2 = __ffma2_rn(ti, ti, a2);
  float2 b2 = __fmul2_rn(br, br);
  b2 = __ffma2_rn(bi, bi, b2);
  float2 gr = __fmul2_rn(tr, br);
  gr = __ffma2_rn(ti, bi, gr);
  const float2 gi = __fmul2_rn(tr, bi), gj = __fmul2_rn(ti, br);
  u[0] = a2.x + a2.y;
  u[1] = b2.x + b2.y;
  u[2] = gr.x + gr.y;
  u[3] = (gi.x + gi.y) - (gj.x + gj.y);
}

// The pairs of step K (register set j < 8: column j of block A_w, 8 + j: column j of B_w).
// K = 0..6 pair the columns inside each block by the round-robin of eight (round K: (7, K) and
// (K + i, K - i) mod 7 for i = 1..3), A's four pairs in slots 0..3 and B's in slots 4..7; K = 7..14
// pair column s of A with column (s + K - 7) mod 8 of B in slot s, so eight such steps meet all 64
// pairs of A and B.
__host__ __device__ constexpr int eq_rr(int k, int q, int e) {
  return q == 0 ? (e == 0 ? 7 : k) : (e == 0 ? (k + q) % 7 : (k + 7 - q) % 7);
}
template <int K> __host__ __device__ constexpr int eq_px(int s) {
  return K < 7 ? (s < 4 ? 0 : 8) + eq_rr(K, s & 3, 0) : s;
}
template <int K> __host__ __device__ constexpr int eq_py(int s) {
  return K < 7 ? (s < 4 ? 0 : 8) + eq_rr(K, s & 3, 1) : 8 + ((s + K - 7) & 7);
}

// One step of a warp (the r-th it runs; r's parity picks the buffers and the mbarrier).  The
// eight slots' partial 2x2 Grams over this CTA's rows are reduce-scattered over the warp (lane l
// ends with value l: slot l >> 2, component l & 3), sent to the same warp of the other CTAs and
// summed with theirs in rank order (so every CTA forms the same rotations), and each group of four
// lanes forms its slot's rotation; then both columns of every rotating slot are updated.  Returns
// whether some slot was not calm (warp-uniform); *ok turns false when a wait gives up.
template <int K>
__device__ __forceinline__ bool eq_bstep(float2 (&XR)[16], float2 (&XI)[16], const EqCtx& x, int r, bool* ok) {
  const int lane = x.lane, par = r & 1;
  // slots s and s + 4 together, folded at once into the first level of the reduce-scatter
  float w16[16];
  const bool hi16 = lane & 16;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    float u[4], u2[4];
    eq_gram(XR[eq_px<K>(s)], XI[eq_px<K>(s)], XR[eq_py<K>(s)], XI[eq_py<K>(s)], u);
    eq_gram(XR[eq_px<K>(s + 4)], XI[eq_px<K>(s + 4)], XR[eq_py<K>(s + 4)], XI[eq_py<K>(s + 4)], u2);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      w16[4 * s + c] = (hi16 ? u2[c] : u[c]) + __shfl_xor_sync(~0u, hi16 ? u[c] : u2[c], 16);
  }
  const float part = eq_reduce_scatter_rest(w16, lane);   // this CTA's rows
  // ---- the partial to the other CTAs, then the sum of all four in rank order
  if (lane == 0) eq_arrive_expect_tx(x.bar(par), EQ_STEP_BYTES);
  const uint32_t off = (uint32_t)((((par * EQ_C + x.rank) * x.nw + x.warp) * 32 + lane) * 4);
#pragma unroll
  for (int j = 0; j < EQ_C - 1; ++j) eq_send(x, off, par, (x.rank + 1 + j) & (EQ_C - 1), part);
  if (*ok) *ok = eq_wait(x.bar(par), (r >> 1) & 1);
  float tot = 0.f;
#pragma unroll
  for (int q = 0; q < EQ_C; ++q)
    tot += q == x.rank ? part : eq_lds(x.recv_s + (uint32_t)((((par * EQ_C + q) * x.nw + x.warp) * 32 + lane) * 4));
  // ---- each group of four lanes forms the rotation of slot lane >> 2
  const int base = lane & 28;
  const float a = __shfl_sync(~0u, tot, base), b = __shfl_sync(~0u, tot, base + 1);
  const float2 gm = make_float2(__shfl_sync(~0u, tot, base + 2), __shfl_sync(~0u, tot, base + 3));
  float c;
  float2 st;
  int rot;
  bool calm;
  ep_rotation_os(a, b, gm, EQ_TOL, x.clim2, x.slim2, c, st, rot, calm);
  const unsigned rmask = __ballot_sync(~0u, rot);
  const unsigned wmask = __ballot_sync(~0u, !calm);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    if (!((rmask >> (4 * s)) & 1u)) continue;   // warp-uniform
    const float cs = __shfl_sync(~0u, c, 4 * s), sr = __shfl_sync(~0u, st.x, 4 * s), si = __shfl_sync(~0u, st.y, 4 * s);
    const int t = eq_px<K>(s), bb = eq_py<K>(s);
    const float2 C2 = make_float2(cs, cs), SR = make_float2(sr, sr), SI = make_float2(si, si);
    const float2 NSR = make_float2(-sr, -sr), NSI = make_float2(-si, -si);
    const float2 xr = XR[t], xi = XI[t], yr = XR[bb], yi = XI[bb];
    XR[t] = __ffma2_rn(NSI, yi, __ffma2_rn(NSR, yr, __fmul2_rn(C2, xr)));
    XI[t] = __ffma2_rn(SI, yr, __ffma2_rn(NSR, yi, __fmul2_rn(C2, xi)));
    XR[bb] = __ffma2_rn(C2, yr, __ffma2_rn(NSI, xi, __fmul2_rn(SR, xr)));
    XI[bb] = __ffma2_rn(C2, yi, __ffma2_rn(SI, xr, __fmul2_rn(SR, xi)));
  }
  return wmask != 0u;
}

// The position (column of L at the start, of U at the end) of column s of block j (A_w: 0, B_w: 1)
// of warp w: blocks in circle order, shifted so that A_0 holds the last eight
__host__ __device__ inline int eq_block_pos(int nw, int w, int j, int s) {
  return 8 * ((2 * w + j + 2 * nw - 1) % (2 * nw)) + s;
}


__global__ void __launch_bounds__(32 * ((kEvdOscNmax + 15) / 16), 1)
evd_osc_kernel(const float2* __restrict__ Lg, const int* __restrict__ perm_g,
               const float2* __restrict__ Vhg, const float2* __restrict__ Tg, const double* __restrict__ scale_g,
               const Box* __restrict__ boxes, EqArgs g, double* __restrict__ lam_out, float2* __restrict__ V_out,
               float* __restrict__ wt_out, int* __restrict__ kcut_out, float* __restrict__ alpha_out,
               int* __restrict__ flags_out, float2* __restrict__ W_out, int* __restrict__ ncol_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), k = blockIdx.x / EQ_C, n = g.nt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x;
  const EqLayout L = eq_layout(n);
  const int np = L.np, lda = L.lda, m = L.m;
  const int r0 = rank * L.R, r1 = r0 + L.R < n ? r0 + L.R : n, nr = r1 > r0 ? r1 - r0 : 0;   // own rows (pivot order)
  float2* U = reinterpret_cast<float2*>(smem + L.u);   // [row - r0][pos]
  double* lamp = reinterpret_cast<double*>(smem + L.lamp);
  double* lam = reinterpret_cast<double*>(smem + L.lam);
  int* sperm = reinterpret_cast<int*>(smem + L.sperm);
  int* perm = reinterpret_cast<int*>(smem + L.perm);
  double* lam_s = reinterpret_cast<double*>(smem + L.lams);
  double* wts = reinterpret_cast<double*>(smem + L.wts);
  double* s0 = reinterpret_cast<double*>(smem + L.s0);
  double* s1 = reinterpret_cast<double*>(smem + L.s1);
  double* s2 = reinterpret_cast<double*>(smem + L.s2);
  float* coef = reinterpret_cast<float*>(smem + L.coef);
  int* keep = reinterpret_cast<int*>(smem + L.keep);
  float2* phs = reinterpret_cast<float2*>(smem + L.phs);
  float4* cmax = reinterpret_cast<float4*>(smem + L.cmax);
  float2* Vh = reinterpret_cast<float2*>(smem + L.vh);
  float2* Tm = reinterpret_cast<float2*>(smem + L.tm);
  float2* Y = reinterpret_cast<float2*>(smem + L.y);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  const double scale = scale_g[k];

  if (!(scale > 0.0)) {   // degenerate window (zero Gram): every CTA writes its share of the empty result
    const int v0 = (int)((long)n * rank / EQ_C), v1 = (int)((long)n * (rank + 1) / EQ_C);
    for (int e = tid; e < (v1 - v0) * n; e += nthr) {
      const int a = v0 + e / n, c = e % n;
      V_out[(size_t)k * n * n + (size_t)a * n + c] = make_float2(a == c, 0.f);
    }
    for (int e = tid; e < (v1 - v0) * g.ncp; e += nthr) W_out[(size_t)k * n * g.ncp + (size_t)v0 * g.ncp + e] = make_float2(0.f, 0.f);
    if (rank == 0) {
      for (int i = tid; i < n; i += nthr) { lam_out[(size_t)k * n + i] = 0.0; wt_out[(size_t)k * n + i] = 0.f; }
      if (tid == 0) { kcut_out[k] = 0; alpha_out[k] = 0.f; ncol_out[k] = 0; flags_out[k] = LCF_WFLAG_DEGENERATE; }
    }
    return;   // every CTA of the cluster leaves before any cluster-level exchange
  }
  for (int i = tid; i < n; i += nthr) perm[i] = perm_g[(size_t)k * n + i];
  if (tid < 2 * L.nw) ep_bar_init(&bar[tid], 1);   // [parity][warp]
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  cluster.sync();   // barriers of every CTA initialised

  // ---- blocks: block j of warp w (A_w: j = 0, B_w: j = 1) starts with columns eq_block_pos(nw, w,
  // j, 0..7) of L, this CTA's rows (lane l rows r0 + l and r0 + 32 + l as a packed pair).  The last
  // eight positions form A_0, which the circle never moves: with eight or more zero columns past Nt
  // warp 0 has no cross pair to rotate and skips those steps (at Nt = 200 the other twelve warps
  // then sit three to a scheduler).
  const int nw = L.nw;
  const bool idle0 = warp == 0 && np - n >= 8;
  EqCtx xc;
  xc.recv_s = ep_smem(smem + L.u) + (uint32_t)eq_xq_bytes(nw);
  xc.bar_s = ep_smem(bar);
  xc.nw = nw; xc.warp = warp; xc.lane = lane; xc.rank = rank;
  {
    const float ne = (float)(n + (n & 1));   // the calm bounds take the unpadded size
    xc.clim2 = ne * EQ_TOL * EQ_TOL;
    xc.slim2 = 0.25f / (ne * ne * ne);
  }
  float2 XR[16], XI[16];
  {
    const float2* Lw = Lg + (size_t)k * n * n;
    const int ra = r0 + lane, rb = r0 + 32 + lane;
    const bool va = lane < nr, vb = 32 + lane < nr;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = eq_block_pos(nw, warp, j >> 3, j & 7);
      const float2 z = make_float2(0.f, 0.f);
      const float2 ta = (va && c < n) ? Lw[(size_t)ra * n + c] : z;
      const float2 tb = (vb && c < n) ? Lw[(size_t)rb * n + c] : z;
      XR[j] = make_float2(ta.x, tb.x); XI[j] = make_float2(ta.y, tb.y);
    }
  }
  // ---- sweeps in rounds: eight steps in which each warp meets all pairs of its A and B, then the
  // blocks move one place on the circle (A_0 stays, A_1 takes B_0, A_w takes A_(w-1), B_w takes
  // B_(w+1), the last B takes its own A) through shared memory; the first round of a sweep adds the
  // seven steps of the pairs inside each block.  A warp waits only for the same warp of the other
  // CTAs at each step (its own mbarrier) and for the whole CTA at the round's exchange.  Converged
  // once a whole sweep of rounds (2 nw - 1, which meet every pair once) was calm; every CTA forms the
  // same rotations, so every CTA reaches the same decision.
  __shared__ int sh_fail;
  if (tid == 0) sh_fail = 0;
  __syncthreads();
  bool ok = true;
  int converged = 0, sweeps = 0;
  {
    const uint32_t xq = ep_smem(smem + L.u);   // float4 [warp][column 0..15][lane], overlays u
    const int per = 2 * nw - 1;
    const int maxrounds = (g.max_sweeps > 0 ? g.max_sweeps : 40) * per;
    int rounds = 0, quiet = 0, last = 0, rr = 0, r = 0;
    for (;;) {
      bool nc = false;
      if (rr == 0) {   // the pairs inside each block, once per sweep
        nc |= eq_bstep<0>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<1>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<2>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<3>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<4>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<5>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<6>(XR, XI, xc, r++, &ok);
      }
      if (!idle0) {
        nc |= eq_bstep<7>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<8>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<9>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<10>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<11>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<12>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<13>(XR, XI, xc, r++, &ok);
        nc |= eq_bstep<14>(XR, XI, xc, r++, &ok);
      }
      // ---- the blocks move: A_w to warp w + 1 (read by warps 2 .. nw - 1), B_w to warp w - 1 (B_0
      // to warp 1 as its A)
      if (nw > 1) {
        const uint32_t own = xq + (uint32_t)((warp * 16 * 32 + lane) * 16);
        if (warp > 0 && warp < nw - 1) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            eq_sts4(own + (uint32_t)(j * 32 * 16), make_float4(XR[j].x, XR[j].y, XI[j].x, XI[j].y));
        }
#pragma unroll
        for (int j = 8; j < 16; ++j)
          eq_sts4(own + (uint32_t)(j * 32 * 16), make_float4(XR[j].x, XR[j].y, XI[j].x, XI[j].y));
      }
      const int any = __syncthreads_or(nc);
      if (nw > 1) {
        if (warp == nw - 1) {
#pragma unroll
          for (int j = 0; j < 8; ++j) { XR[8 + j] = XR[j]; XI[8 + j] = XI[j]; }
        }
        if (warp > 0) {   // new A: B_0 for warp 1, A_(w-1) for the others
          const uint32_t src = xq + (uint32_t)((((warp - 1) * 16 + (warp == 1 ? 8 : 0)) * 32 + lane) * 16);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 q = eq_lds4(src + (uint32_t)(j * 32 * 16));
            XR[j] = make_float2(q.x, q.y); XI[j] = make_float2(q.z, q.w);
          }
        }
        if (warp < nw - 1) {   // new B: B_(w+1)
          const uint32_t src = xq + (uint32_t)((((warp + 1) * 16 + 8) * 32 + lane) * 16);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 q = eq_lds4(src + (uint32_t)(j * 32 * 16));
            XR[8 + j] = make_float2(q.x, q.y); XI[8 + j] = make_float2(q.z, q.w);
          }
        }
      }
      // read before the next round writes; and stop exchanging once a wait gave up
      if (__syncthreads_or(!ok)) { sh_fail = 1; break; }
      ++rounds;
      if (any) { quiet = 0; last = rounds; }
      else ++quiet;
      if (quiet >= per) { converged = 1; break; }
      if (rounds >= maxrounds) break;
      rr = rr + 1 == per ? 0 : rr + 1;
    }
    sweeps = (last + per - 1) / per;
  }
  __syncthreads();
  ok = !sh_fail;

  // ---- squared column norms: this CTA's rows (double-float), summed over the cluster in rank order
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int pa = eq_block_pos(nw, warp, 0, s), pb = eq_block_pos(nw, warp, 1, s);
    const float2 tr = XR[s], ti = XI[s], br = XR[8 + s], bi = XI[8 + s];
    df na = {0.f, 0.f}, nb = {0.f, 0.f};
    na = df_add_f(na, fmaf(tr.x, tr.x, ti.x * ti.x));
    na = df_add_f(na, fmaf(tr.y, tr.y, ti.y * ti.y));
    nb = df_add_f(nb, fmaf(br.x, br.x, bi.x * bi.x));
    nb = df_add_f(nb, fmaf(br.y, br.y, bi.y * bi.y));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      df t;
      t.hi = __shfl_xor_sync(~0u, na.hi, o); t.lo = __shfl_xor_sync(~0u, na.lo, o); na = df_add(na, t);
      t.hi = __shfl_xor_sync(~0u, nb.hi, o); t.lo = __shfl_xor_sync(~0u, nb.lo, o); nb = df_add(nb, t);
    }
    if (lane < EQ_C) {   // lane q writes into CTA q
      double* dst = cluster.map_shared_rank(lamp, (unsigned)lane);
      dst[rank * np + pa] = (double)na.hi + (double)na.lo;
      dst[rank * np + pb] = (double)nb.hi + (double)nb.lo;
    }
    // this CTA's rows, unnormalised for now
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int rr = e * 32 + lane;
      if (rr < nr) {
        U[(size_t)rr * lda + pa] = make_float2(e ? tr.y : tr.x, e ? ti.y : ti.x);
        U[(size_t)rr * lda + pb] = make_float2(e ? br.y : br.x, e ? bi.y : bi.x);
      }
    }
  }
  cluster.sync();   // every CTA's partial norms are here
  for (int i = tid; i < np; i += nthr) {
    double t = 0.0;
    for (int q = 0; q < EQ_C; ++q) t += lamp[q * np + i];
    lam[i] = t > 7.888609052210118e-31 ? t : 0.0;   // below 2^-100 (largest diagonal in [1/2, 1)): vanished
  }
  __syncthreads();
  // (the squared norms are >= 0, so their bit patterns order as integers: the comparisons run on
  // the integer pipes, not on the few FP64 units; coef holds each position's scale until the rule)
  const long long* lbits = reinterpret_cast<const long long*>(lam);
  for (int i = tid; i < np; i += nthr) {   // positions by squared norm, descending, ties to the lower one
    const long long di = lbits[i];
    int r = 0;
    for (int j = 0; j < np; ++j) {
      const long long dj = lbits[j];
      r += (dj > di) || (dj == di && j < i);
    }
    sperm[r] = i;
    coef[i] = di > 0 ? ep_rsqrt((float)lam[i]) : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < nr * np; e += nthr) {   // normalise
    const int rr = e / np, pos = e % np;
    U[(size_t)rr * lda + pos] = cscale(U[(size_t)rr * lda + pos], coef[pos]);
  }
  __syncthreads();
  // ---- vanished columns (numerical rank below Nt): Gram-Schmidt completion on CTA 0 over the whole
  // columns, through the scratch buffer [pos][row] in global memory (every CTA decides the same)
  if (!(lbits[sperm[n - 1]] > 0)) {   // the zeros sort last: some among the first n
    float2* S = V_out + (size_t)k * n * n;   // [sorted index][row]: V_out is written last
    for (int e = tid; e < nr * n; e += nthr) {
      const int rr = e / n, jj = e % n;
      S[(size_t)jj * n + r0 + rr] = U[(size_t)rr * lda + sperm[jj]];
    }
    cluster.sync();
    if (rank == 0 && warp == 0) {
      int cand = 0;
      for (int jj = 0; jj < n; ++jj) {
        if (lam[sperm[jj]] > 0.0) continue;
        float2* col = S + (size_t)jj * n;
        for (int tries = 0; tries < n; ++tries, cand = (cand + 1) % n) {
          for (int r = lane; r < n; r += 32) col[r] = make_float2(r == cand ? 1.f : 0.f, 0.f);
          __syncwarp();
          for (int pass = 0; pass < 2; ++pass) {
            for (int q = 0; q < jj; ++q) {
              const float2* cq = S + (size_t)q * n;
              float2 d = make_float2(0.f, 0.f);
              for (int r = lane; r < n; r += 32) d = cadd(d, cmulc(cq[r], col[r]));
              for (int o = 16; o; o >>= 1) { d.x += __shfl_xor_sync(~0u, d.x, o); d.y += __shfl_xor_sync(~0u, d.y, o); }
              for (int r = lane; r < n; r += 32) col[r] = csub(col[r], cmul(d, cq[r]));
              __syncwarp();
            }
          }
          float nrm = 0.f;
          for (int r = lane; r < n; r += 32) nrm += cabs2(col[r]);
          for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(~0u, nrm, o);
          if (nrm > 0.5f / n) {   // some unit vector keeps at least 1/n of its square in the complement
            const float sc = ep_rsqrt(nrm);
            for (int r = lane; r < n; r += 32) col[r] = cscale(col[r], sc);
            __syncwarp();
            cand = (cand + 1) % n;
            break;
          }
        }
      }
      __threadfence();
    }
    cluster.sync();
    for (int e = tid; e < nr * n; e += nthr) {
      const int rr = e / n, jj = e % n;
      U[(size_t)rr * lda + sperm[jj]] = S[(size_t)jj * n + r0 + rr];
    }
    __syncthreads();
  }
  // ---- V = Q U = U - Vh (T (Vh^H U)): Vh^H U summed over the cluster (rank order)
  float2* Xp = reinterpret_cast<float2*>(smem + L.x);   // [source rank][j][pos] (the sweeps are over)
  for (int e = tid; e < m * n; e += nthr) Vh[e] = Vhg[(size_t)k * m * n + e];
  for (int e = tid; e < m * m; e += nthr) Tm[e] = Tg[(size_t)k * m * m + e];
  __syncthreads();
  for (int e = tid; e < m * np; e += nthr) {
    const int j = e / np, pos = e % np;
    float2 acc = make_float2(0.f, 0.f);
    for (int rr = 0; rr < nr; ++rr) acc = cadd(acc, cmulc(Vh[(size_t)j * n + perm[r0 + rr]], U[(size_t)rr * lda + pos]));
    for (int q = 0; q < EQ_C; ++q) cluster.map_shared_rank(Xp, (unsigned)q)[((size_t)rank * m + j) * np + pos] = acc;
  }
  cluster.sync();
  for (int e = tid; e < m * np; e += nthr) {   // Y = T X, T upper triangular
    const int i = e / np, pos = e % np;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = i; j < m; ++j) {
      float2 xs = make_float2(0.f, 0.f);
      for (int q = 0; q < EQ_C; ++q) xs = cadd(xs, Xp[((size_t)q * m + j) * np + pos]);
      acc = cadd(acc, cmul(Tm[i * m + j], xs));
    }
    Y[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < nr * np; e += nthr) {
    const int rr = e / np, pos = e % np, a = perm[r0 + rr];
    float2 v = U[(size_t)rr * lda + pos];
    for (int j = 0; j < m; ++j) v = csub(v, cmul(Vh[(size_t)j * n + a], Y[(size_t)j * np + pos]));
    U[(size_t)rr * lda + pos] = v;
  }
  // ---- sort, rule, alpha, kept columns (every CTA the same; CTA 0 writes the per-window results)
  for (int i = tid; i < n; i += nthr) lam_s[i] = lam[sperm[i]] * scale;
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
      if (rank == 0) {
        kcut_out[k] = kk;
        alpha_out[k] = (float)al;
        flags_out[k] = fl;
      }
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
    if (lane == 0) {
      keep[0] = base;
      if (rank == 0) ncol_out[k] = base;
    }
  }
  __syncthreads();
  if (rank == 0) {
    for (int i = tid; i < n; i += nthr) {
      lam_out[(size_t)k * n + i] = lam_s[i];
      wt_out[(size_t)k * n + i] = (float)wts[i];
    }
  }
  // ---- phase of each sorted eigenvector: its largest-magnitude entry (over the cluster's rows, ties
  // to the lower row by original index) made real positive
  for (int jj = warp; jj < n; jj += nthr / 32) {
    const int pos = sperm[jj];
    float best = -1.f;
    int ba = 0x7fffffff;
    float2 bv = make_float2(0.f, 0.f);
    for (int rr = lane; rr < nr; rr += 32) {
      const float2 v = U[(size_t)rr * lda + pos];
      const float mg = cabs2(v);
      const int a = perm[r0 + rr];
      if (mg > best || (mg == best && a < ba)) { best = mg; ba = a; bv = v; }
    }
    for (int o = 16; o; o >>= 1) {
      const float ob = __shfl_xor_sync(~0u, best, o);
      const int oa = __shfl_xor_sync(~0u, ba, o);
      const float ox = __shfl_xor_sync(~0u, bv.x, o), oy = __shfl_xor_sync(~0u, bv.y, o);
      if (ob > best || (ob == best && oa < ba)) { best = ob; ba = oa; bv = make_float2(ox, oy); }
    }
    if (lane < EQ_C)
      cluster.map_shared_rank(cmax, (unsigned)lane)[(size_t)rank * np + jj] = make_float4(best, __int_as_float(ba), bv.x, bv.y);
  }
  cluster.sync();
  for (int jj = tid; jj < n; jj += nthr) {
    float best = -1.f;
    int ba = 0x7fffffff;
    float2 bv = make_float2(1.f, 0.f);
    for (int q = 0; q < EQ_C; ++q) {
      const float4 c4 = cmax[(size_t)q * np + jj];
      const int a = __float_as_int(c4.y);
      if (c4.x > best || (c4.x == best && a < ba)) { best = c4.x; ba = a; bv = make_float2(c4.z, c4.w); }
    }
    const float mg = sqrtf(cabs2(bv));
    phs[jj] = mg > 0.f ? make_float2(bv.x / mg, -bv.y / mg) : make_float2(1.f, 0.f);
  }
  __syncthreads();
  // ---- V and W rows of this CTA (row a = perm[r] by original index)
  for (int e = tid; e < nr * n; e += nthr) {
    const int rr = e / n, jj = e % n, a = perm[r0 + rr];
    V_out[(size_t)k * n * n + (size_t)a * n + jj] = cmul(U[(size_t)rr * lda + sperm[jj]], phs[jj]);
  }
  const int nc = keep[0];
  for (int e = tid; e < nr * g.ncp; e += nthr) {
    const int rr = e / g.ncp, c = e % g.ncp, a = perm[r0 + rr];
    float2 v = make_float2(0.f, 0.f);
    if (c < nc) {
      const int jj = keep[1 + c];
      v = cscale(cmul(U[(size_t)rr * lda + sperm[jj]], phs[jj]), coef[jj]);
    }
    W_out[(size_t)k * n * g.ncp + (size_t)a * g.ncp + c] = v;
  }
  if (!ok && tid == 0) atomicOr(g.err, 1);
  cluster.sync();   // no CTA leaves while another may still write into its shared memory
}


cudaError_t launch_evd_osc(const lcf_plan* P, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  const int n = P->nt;
  cudaError_t e = launch_evd_prep(P, st, EQ_SUBSPACE_ITERS);
  if (e != cudaSuccess) return e;
  evd_chol_kernel<<<P->nd, EC_THREADS, evd_chol_smem_bytes(n), st>>>(P->ws.evd_B, P->ws.evd_scale, n, P->ws.evd_perm,
                                                                       P->ws.evd_rank);
  if ((e = counted(P)) != cudaSuccess) return e;
  EqArgs a;
  a.nt = n; a.nz = c.nz; a.nx = c.nx;
  a.thresh_mode = c.thresh_mode; a.beta = c.beta; a.beta_src = c.beta_src;
  a.k_fixed = c.k_fixed; a.k_src = c.k_src; a.pd_mode = c.pd_mode; a.alpha_mode = c.alpha_mode;
  a.curv_norm = c.curv_norm; a.max_sweeps = c.max_sweeps; a.ncp = P->ncp;
  a.err = P->ws.err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(EQ_C * P->nd);
  cfg.blockDim = dim3(32 * eq_layout(n).nw);
  cfg.dynamicSmemBytes = evd_osc_smem_bytes(n);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = EQ_C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, evd_osc_kernel, (const float2*)P->ws.evd_B, (const int*)P->ws.evd_perm,
                         (const float2*)P->ws.evd_vh, (const float2*)P->ws.evd_t, (const double*)P->ws.evd_scale,
                         (const Box*)P->ws.box, a, P->ws.lam, P->ws.V, P->ws.wt, P->ws.kcut, P->ws.alpha, P->ws.flags,
                         P->ws.W, P->ws.ncol);
  if (e != cudaSuccess) return e;
  return counted(P);
}

cudaError_t evd_osc_configure() {
  cudaError_t e = cudaFuncSetAttribute(evd_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)evd_chol_smem_bytes(kEvdOscNmax));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(evd_osc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)evd_osc_smem_bytes(kEvdOscNmax));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(evd_osc_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
  return e;
}

}  // namespace lcf
