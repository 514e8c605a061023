// k_gram_tc.cu — windowed Gram on the tcgen05 tensor cores (Eq. 12).
//
// The deflated augmented row x_p = [c_p, a_p] (na = Nt + d entries, see
// k_gram_simt.cu) is weighted, w_p = s g_k(p) x_p, and split per component
// into fp16 halves, w = w_hi + w_lo (22 significant bits; s = 2^e keeps the
// packet below 2^14).  With the complex product written as a real one over
// K = (pixel, re/im),
//   A[i][(p,re)] = Re w_hi(i),  A[i][(p,im)] = Im w_hi(i)
//   B[j][(p,.)]  = (Re w(j), Im w(j))            j <  nbh   -> Re(conj(w_i) w_j)
//   B[nbh+j][.]  = (Im w(j), -Re w(j))           (-i w)      -> Im(conj(w_i) w_j)
// two passes, A B_hi^T + A (2 B_lo)^T, accumulate D' = P_hh + 2 P_hl in TMEM;
// its Hermitian part P_hh + P_hl + P_hl^H equals sum_p g^2 x^H x up to the
// dropped lo*lo term (relative 2^-22 squared).  A aliases the first 128 rows
// of the B_hi buffer (rows past nbh only feed output rows that are unused).
//
// One CTA per (window, range of 32-pixel slabs), warp-specialised: a loader
// warp brings each slab (32 pixels of a box row x all rows) into shared memory
// with one tensor-map load; sixteen producer warps split it into a 3-stage ring
// of MMA operands and signal the stage's `full` mbarrier; one warp issues the
// tcgen05.mma chain and commits `empty` (stage reusable) and the accumulator's
// barrier.  No CTA-wide barrier inside the loop.  The TMEM accumulator holds a
// chain of TG_CPA slabs; the producers promote it into round-to-nearest
// FP32 sums kept in a second TMEM region (load, add, store back) before the next
// chain starts; the range's sum is written as an FP32 partial, added over the
// ranges in double by gram_tc_reduce_kernel.
// The d x d coefficient block (largest entries) comes from gram_q_kernel with
// exact double-float products instead.
//
// Both Gram kernels are templates on the product precision (LCF_GP_*): the
// split above is LCF_GP_F16X3; LCF_GP_BF16X3 splits into bf16 halves (bf16
// MMAs); the one-pass modes keep the hi words only (fp16, bf16, or E4M3 values
// held in fp16) and issue only the A B_hi^T MMAs.
#include <math.h>

#include <cudaTypedefs.h>

#include "lcf_internal.cuh"
#include "tc_util.cuh"

namespace lcf {

constexpr int TG_THREADS = 256;
constexpr int TG_PX = 32;                  // pixels per stage
constexpr int TG_K = 2 * TG_PX;            // K elements per stage
constexpr int TG_STAGES = 3;
// Stages per TMEM accumulation chain before the chain is promoted into the
// round-to-nearest FP32 sums.  The tensor core's FP32 accumulation rounds
// toward zero, which biases long same-sign chains; after deflation the chains
// sum residual (blood + noise) products only, and chains of 16 stages (512
// pixel products) leave the Gram's error against the FP64 oracle where chains
// of 4 had it (1.6e-8 relative at 256x128 px, Nt = 100; 8.9e-9 at 96x64x32;
// unchanged up to 64 stages), far inside the 1e-6 tolerance.
constexpr int TG_CPA = 16;
constexpr int TG_SBO = (TG_K / 8) * 128;   // bytes between 8-row groups
constexpr int TG_NBH_MAX = 128;

__host__ __device__ inline int tc_nbh(int na) { return (na + 7) / 8 * 8; }
__host__ __device__ inline int tc_rows_hi(int nbh) { return 2 * nbh > 128 ? 2 * nbh : 128; }

constexpr int TW_PROD = 16;                      // producer warps: split, promote
constexpr int TW_THREADS = 32 * (TW_PROD + 2);   // + one warp issuing the MMAs, one loading the slabs

// fp32 slab staging, two slots: row r of the slab at r * 272 bytes, filled by one tensor-map load
// of kTcSlabBox pixels x na rows (the 16 bytes past 32 pixels offset the rows' banks, so the
// producers' 16-row reads are free of conflicts), or, for odd Nz Nx, by each producer thread's
// cp.async copies of exactly the 16 bytes per row that it reads
constexpr int TW_ROWB = kTcSlabBox * 8;
__host__ __device__ inline size_t tc_slot_bytes(int na) { return ((size_t)na * TW_ROWB + 1023) / 1024 * 1024; }
__host__ __device__ inline size_t tc_raw_bytes(int na) { return 2 * tc_slot_bytes(na); }
size_t gram_tc_smem_bytes_n(int na, int nstg) {
  int nbh = tc_nbh(na), rh = tc_rows_hi(nbh);
  size_t hi = (size_t)rh * TG_K * 2, lo = (size_t)2 * nbh * TG_K * 2;
  return nstg * (hi + lo) + 1024 + tc_raw_bytes(na);
}
// MMA operand stages: three when they fit beside the fp32 staging (and the kernel's static
// barriers, within the 227 KB a block may hold), else two
int gram_tc_stages(int na) { return gram_tc_smem_bytes_n(na, TG_STAGES) <= 232448 - 1024 ? TG_STAGES : 2; }
size_t gram_tc_smem_bytes(int na) { return gram_tc_smem_bytes_n(na, gram_tc_stages(na)); }

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src, bool valid) {
  // 8-byte asynchronous copy; an invalid source copies nothing and zero-fills
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_u32(dst_smem)), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A slab is 32 consecutive pixels of one box row, starting at xs = x0 - ((z nx + x0) mod 2) + 32 c
// (an even linear index: a tensor-map load must start on a 16-byte boundary); pixels outside
// [x0, x1) take weight 0.  The shift is x0 mod 2 on every row when Nx is even, else 0 or 1, so
// nch = ceil((x1 - x0 + sh) / 32) slabs per box row with sh = x0 mod 2 (Nx even) or 1 (Nx odd).
// Slabs are visited in order: (row zr, chunk cx) advance without divisions.
struct TcSlab {
  int zr, cx;
  __device__ __forceinline__ void start(int t, int nch) {
    zr = t / nch;
    cx = t - zr * nch;
  }
  __device__ __forceinline__ void next(int nch) {
    if (++cx == nch) { cx = 0; ++zr; }
  }
  __device__ __forceinline__ int z(const Box& b) const { return b.z0 + zr; }
  __device__ __forceinline__ int xs(const Box& b, int nx) const {
    return b.x0 - (((b.z0 + zr) * nx + b.x0) & 1) + 32 * cx;
  }
  __device__ __forceinline__ long p0(const Box& b, int nx) const { return (long)(b.z0 + zr) * nx + xs(b, nx); }
};

// barrier among the producer warps (threads 0 .. 32 TW_PROD - 1) only
__device__ __forceinline__ void tc_bar_producers() { asm volatile("bar.sync 1, %0;" ::"n"(32 * TW_PROD) : "memory"); }
// Promotion: the accumulator (columns [0, 2 nbh)) holds one chain of TG_CPA slabs; the FP32
// sums of the chains live in TMEM columns [256, 256 + 2 nbh).  Producer warp w promotes the
// 16-column blocks w / 4, w / 4 + 4, ... of TMEM lane quarter w mod 4.
constexpr uint32_t TW_SUMS = 256;

template <int GP>
__global__ void __launch_bounds__(TW_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmx, int use_map, const float2* __restrict__ xa, int nz, int nx,
               int na, const Box* __restrict__ boxes, const float* __restrict__ gz, const float* __restrict__ gx,
               const unsigned* __restrict__ xmax_bits, int nsplit, int nstg, double* __restrict__ part,
               int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned, derived from the shared array itself (shared-space addressing)
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full_bar[TG_STAGES];    // stage's operands written (one arrive per producer warp)
  __shared__ __align__(8) uint64_t empty_bar[TG_STAGES];   // stage's MMAs done
  __shared__ __align__(8) uint64_t acc_bar;                // the accumulator's chain done
  __shared__ __align__(8) uint64_t accfree_bar;            // the chain promoted (one arrive per producer warp)
  __shared__ __align__(8) uint64_t rfull_bar[2];           // slab slot loaded (tensor-map path)
  __shared__ __align__(8) uint64_t rempty_bar[2];          // slab slot read by every producer warp (tensor-map path)
  __shared__ uint32_t tmem_base;
  __shared__ float wts[2][TG_PX];   // window weights of the slab in slot 0 / 1 (tensor-map path)

  const int k = blockIdx.y, s = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nbh = tc_nbh(na), N = 2 * nbh, rh = tc_rows_hi(nbh);
  const size_t hi_bytes = (size_t)rh * 128, lo_bytes = (size_t)N * 128, st_bytes = hi_bytes + lo_bytes;
  const Box b = boxes[k];
  const int nch = (b.x1 - b.x0 + ((nx & 1) ? 1 : (b.x0 & 1)) + TG_PX - 1) / TG_PX;
  const int S = (b.z1 - b.z0) * nch;
  const int t0 = (int)((long)S * s / nsplit), nst = (int)((long)S * (s + 1) / nsplit) - t0;
  const int nchain = (nst + TG_CPA - 1) / TG_CPA;
  const size_t npix = (size_t)nz * nx;
  const bool bulk = use_map != 0;
  const int rb = (na + 15) / 16;
  const size_t slot_bytes = tc_slot_bytes(na);
  unsigned char* raw = smem + nstg * st_bytes;   // two slab slots

  // zero the stage buffers (padding rows stay zero) and the slab slots
  for (size_t e = tid; e < (nstg * st_bytes + tc_raw_bytes(na)) / 16; e += TW_THREADS)
    reinterpret_cast<uint4*>(smem)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int i = 0; i < nstg; ++i) {
      tc::mbar_init(&full_bar[i], TW_PROD);
      tc::mbar_init(&empty_bar[i], 1);
    }
    tc::mbar_init(&acc_bar, 1);
    tc::mbar_init(&accfree_bar, TW_PROD);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&rfull_bar[i], 1);
      tc::mbar_init(&rempty_bar[i], TW_PROD);
    }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == TW_PROD) {
    // ---- MMA warp: D' = A B_hi^T + A (2 B_lo)^T per stage, chains of TG_CPA stages.  The whole
    // warp runs the loop (warp-uniform counters and descriptors); one elected lane issues.
    {
      const uint32_t idesc = tc::gp_bf16(GP) ? tc::idesc_bf16(128, N) : tc::idesc_f16(128, N);
      const uint32_t sb = tc::smem_u32(smem);
      const uint64_t dh0 = tc::smem_desc(sb, 128, TG_SBO), dl0 = tc::smem_desc(sb + (uint32_t)hi_bytes, 128, TG_SBO);
      bool ok = true;
      for (int i = 0; i < nst; ++i) {
        const int si = i % nstg, c = i / TG_CPA;
        if (ok) ok = tc::mbar_wait(&full_bar[si], (i / nstg) & 1);
        // a chain starts once the previous one has been promoted out of the accumulator
        if (i % TG_CPA == 0 && c > 0 && ok) ok = tc::mbar_wait(&accfree_bar, (c - 1) & 1);
        ok = __all_sync(~0u, ok);
        tc::fence_after();
        // descriptors advance in 16-byte units: a stage, then two core matrices (16 K) per step
        const uint64_t so = (uint64_t)((si * st_bytes) >> 4);
        if (tc::elect_one()) {
#pragma unroll
          for (int ks = 0; ks < TG_K / 16; ++ks) {
            const uint64_t ad = dh0 + so + (uint64_t)(16 * ks), ld = dl0 + so + (uint64_t)(16 * ks);
            tc::mma_f16(tbase, ad, ad, idesc, (i % TG_CPA == 0 && ks == 0) ? 0u : 1u);
            if constexpr (tc::gp_three_products(GP)) tc::mma_f16(tbase, ad, ld, idesc, 1u);
          }
          tc::mma_commit(&empty_bar[si]);
          if (i % TG_CPA == TG_CPA - 1 || i == nst - 1) tc::mma_commit(&acc_bar);
        }
        __syncwarp();
      }
      if (!ok && lane == 0) atomicOr(err, 1);
    }
  } else if (warp == TW_PROD + 1) {
    // ---- loader warp (tensor-map path): slab i into slot i & 1, one load of kTcSlabBox x na
    // (pixels past the image read as zero), and the slab's window weights, one pixel per lane
    if (bulk) {
      bool ok = true;
      const float* gzk = gz + (size_t)k * nz;
      const float* gxk = gx + (size_t)k * nx;
      TcSlab q;
      q.start(t0, nch);
      for (int i = 0; i < nst; ++i, q.next(nch)) {
        if (i >= 2 && ok) ok = tc::mbar_wait(&rempty_bar[i & 1], ((i >> 1) - 1) & 1);
        ok = __all_sync(~0u, ok);
        const int x = q.xs(b, nx) + lane;
        wts[i & 1][lane] = (x >= b.x0 && x < b.x1) ? gzk[q.z(b)] * gxk[x] : 0.f;
        __syncwarp();   // the weights are written before the slab's arrival publishes them
        if (lane == 0) {
          tc::mbar_arrive_expect_tx(&rfull_bar[i & 1], (uint32_t)(na * TW_ROWB));
          tc::tma_load_2d(raw + (size_t)(i & 1) * slot_bytes, &tmx, (int)q.p0(b, nx), 0, &rfull_bar[i & 1]);
        }
      }
      if (!ok && lane == 0) atomicOr(err, 1);
    }
  } else {
    // ---- producer warps: warp w splits pixel slots (ps, ps + 1), ps = 4 (w mod 8) + 2 (lane mod 2),
    // of rows rl + 16 j for j = w / 8, w / 8 + 2, ...
    const int pg = warp & 7, jh = warp >> 3, lgrp = warp & 3, cq = warp >> 2;
    const int ps = 4 * pg + 2 * (lane & 1), rl = lane >> 1;
    const float sc = tc::pow2_scale(__uint_as_float(*xmax_bits));
    const float* gzk = gz + (size_t)k * nz;
    const float* gxk = gx + (size_t)k * nx;
    // this thread's 16 bytes of slab row rl + 16 j: roff + j * 16 * TW_ROWB within a slot
    const int roff = rl * TW_ROWB + ps * 8;
    // its operand entries of row rl + 16 j (K entries 2 ps .. 2 ps + 3): soff + 2048 j within the
    // B_hi / B_lo buffers, rows nbh + r another (nbh / 8) core-row groups further
    const uint32_t soff = (uint32_t)((rl >> 3) * TG_SBO + (2 * ps >> 3) * 128 + (rl & 7) * 16 + (2 * ps & 7) * 2);
    const uint32_t sneg = (uint32_t)(nbh >> 3) * TG_SBO;
    const uint32_t tl = tbase + ((uint32_t)(lgrp * 32) << 16);   // this warp's TMEM lane quarter
    const int nb16 = (N + 15) / 16;
    bool ok = true;

    // cp.async path: this thread's two pixels of slab i (its rows) into slot i & 1
    auto issue = [&](int i, const TcSlab& q) {
      const long pa = q.p0(b, nx) + ps;
      const bool v0 = pa >= 0 && pa < (long)npix, v1 = pa + 1 >= 0 && pa + 1 < (long)npix;
      unsigned char* dst = raw + (size_t)(i & 1) * slot_bytes + roff;
      for (int j = jh; j < rb; j += 2) {
        const int r = rl + 16 * j;
        if (r >= na) break;
        const float2* srow = xa + (size_t)r * npix;
        cp_async8(dst + (size_t)j * 16 * TW_ROWB, srow + (v0 ? pa : 0), v0);
        cp_async8(dst + (size_t)j * 16 * TW_ROWB + 8, srow + (v1 ? pa + 1 : 0), v1);
      }
      cp_async_commit();
    };
    // chain c: sums += accumulator (c == 0: sums = accumulator), this warp's column blocks
    auto promote = [&](int c) {
      if (ok) ok = tc::mbar_wait(&acc_bar, c & 1);   // after a timeout, no further waits
      tc::fence_after();
#pragma unroll
      for (int bq = 0; bq < 4; ++bq) {
        const int blk = cq + 4 * bq;
        if (blk < nb16) {
          uint32_t a[16], t[16];
          tc::tmem_ld16_async(tl + (uint32_t)(16 * blk), a);
          if (c > 0) tc::tmem_ld16_async(tl + TW_SUMS + (uint32_t)(16 * blk), t);
          tc::tmem_wait_ld();
          if (c > 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = __float_as_uint(__uint_as_float(a[j]) + __uint_as_float(t[j]));
          }
          tc::tmem_st16(tl + TW_SUMS + (uint32_t)(16 * blk), a);
        }
      }
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&accfree_bar);
    };

    TcSlab q, qn;
    q.start(t0, nch);
    qn = q;
    qn.next(nch);
    if (!bulk && nst > 0) issue(0, q);
    int next_c = 0;   // first chain still to be promoted
    for (int i = 0; i < nst; ++i, q = qn, qn.next(nch)) {
      const int si = i % nstg;
      // window weights of this thread's two pixels: from the loader (published with the slab)
      // or computed here
      float g0, g1;
      if (bulk) {
        if (ok) ok = tc::mbar_wait(&rfull_bar[i & 1], (i >> 1) & 1);
        g0 = wts[i & 1][ps];
        g1 = wts[i & 1][ps + 1];
      } else {
        const int xa0 = q.xs(b, nx) + ps;
        const float gzz = gzk[q.z(b)];
        g0 = (xa0 >= b.x0 && xa0 < b.x1) ? gzz * gxk[xa0] : 0.f;
        g1 = (xa0 + 1 >= b.x0 && xa0 + 1 < b.x1) ? gzz * gxk[xa0 + 1] : 0.f;
      }
      if (!bulk) {
        if (i + 1 < nst) {   // the next slab's copy overlaps this one's split
          issue(i + 1, qn);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
      }
      if (i >= nstg && ok) ok = tc::mbar_wait(&empty_bar[si], ((i / nstg) - 1) & 1);
      {
        // The pixel pair's four K entries (re, im, re, im) of row r are 8 contiguous bytes of a
        // core-matrix row; a warp's 8-byte stores cover 16 rows x 2 pixel pairs (two wavefronts).
        unsigned char* Bhi = smem + si * st_bytes + soff;
        unsigned char* Blo = Bhi + hi_bytes;
        const unsigned char* src = raw + (size_t)(i & 1) * slot_bytes + roff;
        const float2 gg0 = make_float2(g0 * sc, g0 * sc), gg1 = make_float2(g1 * sc, g1 * sc);
        const float2 gd0 = make_float2(2.f * gg0.x, 2.f * gg0.x), gd1 = make_float2(2.f * gg1.x, 2.f * gg1.x);
#pragma unroll
        for (int jj = 0; jj < kTcGramNaMax / 32; ++jj) {
          const int j = 2 * jj + jh;
          if (rl + 16 * j < na) {
            const float4 v = *reinterpret_cast<const float4*>(src + j * 16 * TW_ROWB);
            uint32_t h0, h1, l0 = 0u, l1 = 0u;
            tc::split2_gp<GP>(make_float2(v.x, v.y), gg0, gd0, h0, l0);
            tc::split2_gp<GP>(make_float2(v.z, v.w), gg1, gd1, h1, l1);
            *reinterpret_cast<uint2*>(Bhi + j * 2 * TG_SBO) = make_uint2(h0, h1);
            *reinterpret_cast<uint2*>(Bhi + sneg + j * 2 * TG_SBO) = make_uint2(tc::neg_i_raw(h0), tc::neg_i_raw(h1));
            if constexpr (tc::gp_three_products(GP)) {
              *reinterpret_cast<uint2*>(Blo + j * 2 * TG_SBO) = make_uint2(l0, l1);
              *reinterpret_cast<uint2*>(Blo + sneg + j * 2 * TG_SBO) = make_uint2(tc::neg_i_raw(l0), tc::neg_i_raw(l1));
            }
          }
        }
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&full_bar[si]);
        if (bulk) tc::mbar_arrive(&rempty_bar[i & 1]);
      }
      // Chain c ends with slab C c + C - 1 (C = TG_CPA); its promotion comes after slab C (c + 1) + 1
      // is split, where the next slab would wait for the same MMAs to free its operand stage.
      if (i % TG_CPA == 1 && i / TG_CPA >= 1) promote(next_c++);
    }
    while (next_c < nchain) promote(next_c++);
    if (!ok && lane == 0) atomicOr(err, 1);

    // partial: plane 0 = Re D', plane 1 = Im D' (rows i < na, columns j < na), written coalesced
    // through shared memory (every MMA has completed and every producer has split its last slab
    // once the last chain was promoted, so the operand and slab buffers are free)
    float* tr = reinterpret_cast<float*>(smem);   // [2][na][ldt], ldt odd: conflict-free column writes
    const int ldt = na + 1 - (na & 1);
    tc_bar_producers();
    const int row = lgrp * 32 + lane;
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) {
      const int blk = cq + 4 * bq;
      if (blk < nb16) {
        uint32_t a[16];
        if (nchain > 0) {
          tc::tmem_ld16_async(tl + TW_SUMS + (uint32_t)(16 * blk), a);
          tc::tmem_wait_ld();
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) a[j] = 0u;
        }
        if (row < na) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = 16 * blk + j, pl = col >= nbh ? 1 : 0, cj = col - pl * nbh;
            if (col < N && cj < na) tr[((size_t)pl * na + row) * ldt + cj] = __uint_as_float(a[j]);
          }
        }
      }
    }
    tc::fence_before();
    tc_bar_producers();
    // FP32 partials (the sums are FP32): gram_tc_reduce_kernel adds the splits in double
    float* out = reinterpret_cast<float*>(part) + ((size_t)k * nsplit + s) * 2 * na * na;
    for (int e = tid; e < 2 * na * na; e += 32 * TW_PROD) {
      const int pl = e / (na * na), rem = e - pl * na * na, r = rem / na, j = rem - r * na;
      out[e] = tr[((size_t)pl * na + r) * ldt + j];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// Long packets (Nt > 128 residual rows): the na x na block (na = Nt + d augmented rows when the
// exact kernel takes the coefficient block, so the tiles give U too; else the Nt residual rows)
// in row tiles of tb rows (T tiles), one CTA per (window, tile pair (a, b)) over the whole
// window support.
// The CTA forms D'(a, b) = A_hi(a) (B_hi(b) + 2 B_lo(b))^T with the operands of the short
// kernel (B(b) = [w ; -i w] of tile b's rows), A from tile a's rows (aliasing B_hi when
// a == b); both orders of every off-diagonal pair are formed, so the assembly takes the
// Hermitian part 1/2 (D'(a, b) + D'(b, a)^H) as before.  This lock-step kernel reads the packet
// directly (no fp32 staging) and is the path for odd pixel counts, where no tensor map can be made;
// otherwise gram_tcp_kernel below runs the same products as a pipeline.
constexpr int TB_STAGES = 3;
__host__ __device__ inline size_t tcb_stage_bytes(int tb, bool same) {
  const int nbh = tc_nbh(tb), rh = same ? tc_rows_hi(nbh) : 2 * nbh;
  return (same ? 0 : (size_t)128 * TG_K * 2) + (size_t)rh * TG_K * 2 + (size_t)2 * nbh * TG_K * 2;
}
size_t gram_tcb_smem_bytes(int tb) {
  const size_t a = tcb_stage_bytes(tb, true), b = tcb_stage_bytes(tb, false);
  return 1024 + TB_STAGES * (a > b ? a : b);
}

template <int GP>
__global__ void __launch_bounds__(TG_THREADS, 1)
gram_tcb_kernel(const float2* __restrict__ xa, int nz, int nx, int nt /* rows tiled */, int tb, int T, const Box* __restrict__ boxes,
                const float* __restrict__ gz, const float* __restrict__ gx, const unsigned* __restrict__ xmax_bits,
                double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mma_bar[TB_STAGES];
  __shared__ __align__(8) uint64_t acc_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int pix_s[TG_PX];
  __shared__ float gg_s[TG_PX];

  const int k = blockIdx.y, ta = blockIdx.x / T, tbk = blockIdx.x % T;
  const bool same = ta == tbk;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ra0 = ta * tb, rna = min(tb, nt - ra0), rb0 = tbk * tb, rnb = min(tb, nt - rb0);
  const int nbh = tc_nbh(rnb), N = 2 * nbh, rh = same ? tc_rows_hi(nbh) : N;
  const size_t a_bytes = same ? 0 : (size_t)128 * TG_K * 2, hi_bytes = (size_t)rh * TG_K * 2;
  const size_t st_bytes = a_bytes + hi_bytes + (size_t)N * TG_K * 2;
  const Box b = boxes[k];
  const int W = b.x1 - b.x0;
  const long Pk = (long)(b.z1 - b.z0) * W;
  const int nst = (int)((Pk + TG_PX - 1) / TG_PX);
  const size_t npix = (size_t)nz * nx;
  const float sc = tc::pow2_scale(__uint_as_float(*xmax_bits));
  const float* gzk = gz + (size_t)k * nz;
  const float* gxk = gx + (size_t)k * nx;
  const int half = warp >> 2, lgrp = warp & 3, row = lgrp * 32 + lane;

  for (size_t e = tid; e < TB_STAGES * st_bytes / 16; e += TG_THREADS)
    reinterpret_cast<uint4*>(smem)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int i = 0; i < TB_STAGES; ++i) tc::mbar_init(&mma_bar[i], 1);
    tc::mbar_init(&acc_bar[0], 1);
    tc::mbar_init(&acc_bar[1], 1);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = tc::gp_bf16(GP) ? tc::idesc_bf16(128, N) : tc::idesc_f16(128, N);

  float sums[TG_NBH_MAX];
#pragma unroll
  for (int j = 0; j < TG_NBH_MAX; ++j) sums[j] = 0.f;
  bool ok = true;
  auto epilogue = [&](int c) {
    if (ok) ok = tc::mbar_wait(&acc_bar[c & 1], (c >> 1) & 1);
    tc::fence_after();
    const uint32_t base = tbase + (uint32_t)((c & 1) * 256) + ((uint32_t)(lgrp * 32) << 16) + (uint32_t)(half * nbh);
#pragma unroll
    for (int cc = 0; cc < TG_NBH_MAX / 16; cc += 2) {
      if (cc * 16 < nbh) {
        uint32_t v0[16], v1[16];
        tc::tmem_ld16_async(base + cc * 16, v0);
        if ((cc + 1) * 16 < nbh) tc::tmem_ld16_async(base + (cc + 1) * 16, v1);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) sums[cc * 16 + j] += __uint_as_float(v0[j]);
        if ((cc + 1) * 16 < nbh) {
#pragma unroll
          for (int j = 0; j < 16; ++j) sums[(cc + 1) * 16 + j] += __uint_as_float(v1[j]);
        }
      }
    }
    tc::fence_before();
  };

  int next_epi = 0;
  for (int i = 0; i < nst; ++i) {
    const int si = i % TB_STAGES;
    unsigned char* Ahi = smem + si * st_bytes;
    unsigned char* Bhi = Ahi + a_bytes;
    unsigned char* Blo = Bhi + hi_bytes;
    if (tid < TG_PX) {
      const long l = (long)i * TG_PX + tid;
      int pp = 0;
      float g = 0.f;
      if (l < Pk) {
        const int zr = (int)l / W, z = b.z0 + zr, x = b.x0 + (int)l - zr * W;   // below 2^31
        pp = z * nx + x;
        g = gzk[z] * gxk[x] * sc;
      }
      pix_s[tid] = pp;
      gg_s[tid] = g;
    }
    if (i >= TB_STAGES && ok) ok = tc::mbar_wait(&mma_bar[si], ((i / TB_STAGES) - 1) & 1);
    __syncthreads();
    {
      // two adjacent pixels of the slab and rows 16 j + lane / 2 per thread (as the short kernel)
      const int pp = 2 * (((tid >> 5) & 7) * 2 + (lane & 1)), rl = lane >> 1;
      const float g0 = gg_s[pp], g1 = gg_s[pp + 1];
      const size_t p0 = pix_s[pp], p1 = pix_s[pp + 1];
      const int kk = 2 * pp;
      const float2 gg0 = make_float2(g0, g0), gg1 = make_float2(g1, g1);
      const float2 gd0 = make_float2(2.f * g0, 2.f * g0), gd1 = make_float2(2.f * g1, 2.f * g1);
      for (int r = rl; r < rnb; r += 16) {
        const float2* src = xa + (size_t)(rb0 + r) * npix;
        uint32_t h0, h1, l0 = 0u, l1 = 0u;
        tc::split2_gp<GP>(src[p0], gg0, gd0, h0, l0);
        tc::split2_gp<GP>(src[p1], gg1, gd1, h1, l1);
        *reinterpret_cast<uint2*>(Bhi + tc::op_off(r, kk, TG_SBO)) = make_uint2(h0, h1);
        *reinterpret_cast<uint2*>(Bhi + tc::op_off(nbh + r, kk, TG_SBO)) =
            make_uint2(tc::neg_i_raw(h0), tc::neg_i_raw(h1));
        if constexpr (tc::gp_three_products(GP)) {
          *reinterpret_cast<uint2*>(Blo + tc::op_off(r, kk, TG_SBO)) = make_uint2(l0, l1);
          *reinterpret_cast<uint2*>(Blo + tc::op_off(nbh + r, kk, TG_SBO)) =
              make_uint2(tc::neg_i_raw(l0), tc::neg_i_raw(l1));
        }
      }
      if (!same) {
        for (int r = rl; r < rna; r += 16) {
          const float2* src = xa + (size_t)(ra0 + r) * npix;
          *reinterpret_cast<uint2*>(Ahi + tc::op_off(r, kk, TG_SBO)) =
              make_uint2(tc::hi2_gp<GP>(src[p0], gg0), tc::hi2_gp<GP>(src[p1], gg1));
        }
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    const int c = i / TG_CPA;
    if (tid == 0) {
      tc::fence_after();
      const uint32_t d = tbase + (uint32_t)((c & 1) * 256);
      const uint32_t ah = tc::smem_u32(same ? Bhi : Ahi), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < TG_K / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(ah + ks * 256, 128, TG_SBO);
        const uint64_t hd = tc::smem_desc(bh + ks * 256, 128, TG_SBO);
        const uint64_t ld = tc::smem_desc(bl + ks * 256, 128, TG_SBO);
        tc::mma_f16(d, ad, hd, idesc, (i % TG_CPA == 0 && ks == 0) ? 0u : 1u);
        if constexpr (tc::gp_three_products(GP)) tc::mma_f16(d, ad, ld, idesc, 1u);
      }
      tc::mma_commit(&mma_bar[si]);
      if (i % TG_CPA == TG_CPA - 1 || i == nst - 1) tc::mma_commit(&acc_bar[c & 1]);
    }
    if (i % TG_CPA == TG_CPA / 2 && c > 0) { epilogue(c - 1); next_epi = c; }
  }
  for (int e = next_epi; nst > 0 && e <= (nst - 1) / TG_CPA; ++e) epilogue(e);
  if (!ok && lane == 0) atomicOr(err, 1);

  // block partial: plane 0 = Re D', plane 1 = Im D' (rows i < rna, columns j < rnb), stride tb
  double* out = part + ((((size_t)k * T + ta) * T + tbk) * 2 + half) * (size_t)tb * tb;
  if (row < rna) {
#pragma unroll
    for (int j = 0; j < TG_NBH_MAX; ++j)
      if (j < rnb) out[(size_t)row * tb + j] = (double)sums[j];
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// Coefficient block Q[a][b] = sum_p g^2 conj(a_pa) a_pb with exact products
// (double-float), one partial per (window, split).  Q is Hermitian: the upper triangle is summed
// and the lower written as its conjugate.
__global__ void __launch_bounds__(256)
gram_q_kernel(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl, const Box* __restrict__ boxes,
              const float* __restrict__ gz, const float* __restrict__ gx, int nsplit, double2* __restrict__ q) {
  const int k = blockIdx.y, s = blockIdx.x, tid = threadIdx.x;
  const Box b = boxes[k];
  const int W = b.x1 - b.x0;
  const long Pk = (long)(b.z1 - b.z0) * W;
  const long l0 = Pk * s / nsplit, l1 = Pk * (s + 1) / nsplit;
  const size_t npix = (size_t)nz * nx;
  df qr[kQExactMax * kQExactMax], qi[kQExactMax * kQExactMax];
#pragma unroll
  for (int e = 0; e < kQExactMax * kQExactMax; ++e) { qr[e] = {0.f, 0.f}; qi[e] = {0.f, 0.f}; }
  for (long l = l0 + tid; l < l1; l += blockDim.x) {
    const int zr = (int)l / W, z = b.z0 + zr, x = b.x0 + (int)l - zr * W;   // box pixel counts are below 2^31
    const size_t p = (size_t)z * nx + x;
    float g = gz[(size_t)k * nz + z] * gx[(size_t)k * nx + x];
    float g2 = g * g;
    float2 a[kQExactMax];
#pragma unroll
    for (int j = 0; j < kQExactMax; ++j) a[j] = j < nd_defl ? xa[(size_t)(nt + j) * npix + p] : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kQExactMax; ++i)
#pragma unroll
      for (int j = i; j < kQExactMax; ++j) {
        if (i >= nd_defl || j >= nd_defl) continue;
        df wr = two_prod_df(g2, a[i].x), wi = two_prod_df(-g2, a[i].y);   // g^2 conj(a_i)
        df rr = df_mul_f(wr, a[j].x), ii = df_mul_f(wi, a[j].y);
        df ri = df_mul_f(wr, a[j].y), ir = df_mul_f(wi, a[j].x);
        qr[i * kQExactMax + j] = df_add(qr[i * kQExactMax + j], df_add(rr, df_neg(ii)));
        qi[i * kQExactMax + j] = df_add(qi[i * kQExactMax + j], df_add(ri, ir));
      }
  }
  // block reduction in double-float
  __shared__ df red_r[8][kQExactMax * kQExactMax], red_i[8][kQExactMax * kQExactMax];
#pragma unroll
  for (int e = 0; e < kQExactMax * kQExactMax; ++e) {
    if (e / kQExactMax > e % kQExactMax) continue;   // the upper triangle only
    df vr = qr[e], vi = qi[e];
    for (int o = 16; o; o >>= 1) {
      df tr = {__shfl_xor_sync(~0u, vr.hi, o), __shfl_xor_sync(~0u, vr.lo, o)};
      df ti = {__shfl_xor_sync(~0u, vi.hi, o), __shfl_xor_sync(~0u, vi.lo, o)};
      vr = df_add(vr, tr);
      vi = df_add(vi, ti);
    }
    if ((tid & 31) == 0) { red_r[tid >> 5][e] = vr; red_i[tid >> 5][e] = vi; }
  }
  __syncthreads();
  if (tid < kQExactMax * kQExactMax) {
    const int i = tid / kQExactMax, j = tid % kQExactMax, e = i <= j ? tid : j * kQExactMax + i;
    df vr = {0.f, 0.f}, vi = {0.f, 0.f};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { vr = df_add(vr, red_r[w][e]); vi = df_add(vi, red_i[w][e]); }
    const double im = df_to_double(vi);
    q[((size_t)k * nsplit + s) * kQExactMax * kQExactMax + tid] = make_double2(df_to_double(vr), i <= j ? im : -im);
  }
}

// R from the tensor-core partials: R' = Herm(sum D') / s^2 for the residual block and U
// (U from the CUDA-core augmented-column partials instead when the tensor-core rows
// nb are the residual rows alone, nb = nt), Q from the exact kernel;
// R = R'_cc + U Phi^T + Phi U^H + Phi Q Phi^T (FP64)
__global__ void gram_assemble_tc_kernel(const double* __restrict__ part, const double2* __restrict__ qpart,
                                        const double2* __restrict__ aug, int aug_nsplit, int aug_qrows,
                                        const float2* __restrict__ phi, const unsigned* __restrict__ xmax_bits,
                                        size_t wstride, int T, int tb, int qsplit, int nt, int nd_defl, int nb,
                                        double2* __restrict__ R) {
  // partials of window k: tile pairs (a, b) of tb rows, [a][b][Re, Im][tb][tb] (T = 1, tb = nb for
  // packets whose augmented rows fit one tile)
  const int k = blockIdx.y;
  const double* pk = part + (size_t)k * wstride;
  extern __shared__ double2 asm_dyn[];   // U [nt][kDeflateMax], Q [kDeflateMax]^2, ph [d][kEvdNmax]
  double2 (*U)[kDeflateMax] = reinterpret_cast<double2 (*)[kDeflateMax]>(asm_dyn);
  double2 (*Q)[kDeflateMax] = reinterpret_cast<double2 (*)[kDeflateMax]>(asm_dyn + (size_t)nt * kDeflateMax);
  double2 (*ph)[kEvdNmax] =
      reinterpret_cast<double2 (*)[kEvdNmax]>(asm_dyn + (size_t)(nt + kDeflateMax) * kDeflateMax);
  __shared__ double inv_s2;
  if (threadIdx.x == 0) {
    float sc = tc::pow2_scale(__uint_as_float(*xmax_bits));
    inv_s2 = 1.0 / ((double)sc * (double)sc);
  }
  __syncthreads();
  const double is2 = inv_s2;
  // Hermitian part of the summed D' at (a, b)
  // (split 0 of each window holds the sum over splits, see gram_tc_reduce_kernel)
  const size_t t2 = (size_t)tb * tb;
  auto dre = [&](int a, int bb, int plane) {   // plane of D' at (a, bb)
    const int ta = a / tb, tbk = bb / tb;
    return pk[((size_t)(ta * T + tbk) * 2 + plane) * t2 + (size_t)(a - ta * tb) * tb + (bb - tbk * tb)];
  };
  auto herm = [&](int a, int bb) {
    const double xr = dre(a, bb, 0) + dre(bb, a, 0);
    const double xi = dre(a, bb, 1) - dre(bb, a, 1);
    return make_double2(0.5 * xr * is2, 0.5 * xi * is2);
  };
  const size_t aout = (size_t)(nt + aug_qrows) * nd_defl;   // augmented-column outputs per split
  const double2* ak = aug + (size_t)k * aug_nsplit * aout;
  for (int e = threadIdx.x; e < nt * nd_defl; e += blockDim.x) {
    int i = e / nd_defl, a = e % nd_defl;
    if (nb > nt) {
      U[i][a] = herm(i, nt + a);
    } else {
      double sx = 0.0, sy = 0.0;
      for (int s = 0; s < aug_nsplit; ++s) {
        const double2 v = ak[(size_t)s * aout + e];
        sx += v.x;
        sy += v.y;
      }
      U[i][a] = make_double2(sx, sy);
    }
    float2 f = phi[a * nt + i];
    ph[a][i] = make_double2((double)f.x, (double)f.y);
  }
  for (int e = threadIdx.x; e < nd_defl * nd_defl; e += blockDim.x) {
    int a = e / nd_defl, c = e % nd_defl;
    double sx = 0.0, sy = 0.0;
    if (aug_qrows > 0) {   // exact-product rows of the augmented-column kernel: Q[a][c] at row nt + a
      for (int s = 0; s < aug_nsplit; ++s) {
        const double2 v1 = ak[(size_t)s * aout + (size_t)(nt + a) * nd_defl + c];
        const double2 v2 = ak[(size_t)s * aout + (size_t)(nt + c) * nd_defl + a];
        sx += 0.5 * (v1.x + v2.x);
        sy += 0.5 * (v1.y - v2.y);
      }
    } else {
      for (int s = 0; s < qsplit; ++s) {
        double2 v1 = qpart[((size_t)k * qsplit + s) * kQExactMax * kQExactMax + a * kQExactMax + c];
        double2 v2 = qpart[((size_t)k * qsplit + s) * kQExactMax * kQExactMax + c * kQExactMax + a];
        sx += 0.5 * (v1.x + v2.x);
        sy += 0.5 * (v1.y - v2.y);
      }
    }
    Q[a][c] = make_double2(sx, sy);
  }
  __syncthreads();
  constexpr int WPT = (kEvdNmax * kDeflateMax + 255) / 256;   // W entries per thread (blockDim 256)
  double2 wv[WPT];
  for (int u = 0; u < WPT; ++u) {              // W = U + 1/2 conj(Phi) Q (nt*d <= 496 < 512)
    int e = threadIdx.x + u * blockDim.x;
    if (e < nt * nd_defl) wv[u] = deflated_w(e / nd_defl, e % nd_defl, nd_defl, U, Q, ph);
  }
  __syncthreads();
  for (int u = 0; u < WPT; ++u) {
    int e = threadIdx.x + u * blockDim.x;
    if (e < nt * nd_defl) U[e / nd_defl][e % nd_defl] = wv[u];
  }
  __syncthreads();
  // upper triangle (row-wise enumeration), each entry written with its mirror
  const int nup = nt * (nt + 1) / 2;
  const float two_n1 = (float)(2 * nt + 1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nup; e += gridDim.x * blockDim.x) {
    int i = (int)floorf(0.5f * (two_n1 - sqrtf(fmaxf(two_n1 * two_n1 - 8.f * (float)e, 0.f))));
    i = i < 0 ? 0 : (i > nt - 1 ? nt - 1 : i);
    while (i > 0 && i * nt - (i * (i - 1)) / 2 > e) --i;
    while (i + 1 < nt && (i + 1) * nt - ((i + 1) * i) / 2 <= e) ++i;
    const int j = i + (e - (i * nt - (i * (i - 1)) / 2));
    double2 r = herm(i, j);
    add_w_terms(r, i, j, nd_defl, U, ph);
    if (i == j) r.y = 0.0;
    R[(size_t)k * nt * nt + (size_t)i * nt + j] = r;
    if (i != j) R[(size_t)k * nt * nt + (size_t)j * nt + i] = make_double2(r.x, -r.y);
  }
}

// ---------------------------------------------------------------------------
// Long packets, pipelined: the one-tile kernel's warp roles over a tile pair (a, b).  One CTA per
// (window, tile pair) over the whole window support; the loader warp brings tile b's rows of each
// slab (and tile a's, off the diagonal) with tensor-map loads of kTcSlabBox x tb; the sixteen
// producer warps take their rows of the slab into registers, hand the slot back, then split tile
// b's rows into B_hi / B_lo ([w ; -i w], as the one-tile kernel) and tile a's into A (hi words
// only; on the diagonal A aliases B_hi); one warp issues D' = A (B_hi + 2 B_lo)^T in chains of
// TG_CPA slabs, promoted by the producers into FP32 sums in tensor memory.  The block partial goes
// out as doubles in the layout of gram_tcb_kernel (both orders of every off-diagonal pair, whose
// Hermitian part the assembly takes).
__host__ __device__ inline size_t tcp_slot_bytes(int tb, bool same) {
  return ((size_t)(same ? 1 : 2) * tb * TW_ROWB + 1023) / 1024 * 1024;
}
static size_t tcp_smem_bytes(int tb, int nstg, int nraw) {
  return 1024 + (size_t)nstg * tcb_stage_bytes(tb, false) + (size_t)nraw * tcp_slot_bytes(tb, false);
}
// stages and slab slots of a launch, sized for an off-diagonal pair: three and two when they fit,
// else fewer (two and one at tb = 104: the producers release a slot before they split it)
static void tcp_shape(int tb, int* nstg, int* nraw) {
  const int cand[4][2] = {{3, 2}, {3, 1}, {2, 2}, {2, 1}};
  for (const auto& c : cand)
    if (tcp_smem_bytes(tb, c[0], c[1]) <= 232448 - 2048) { *nstg = c[0]; *nraw = c[1]; return; }
  *nstg = 0;
  *nraw = 0;
}

template <int GP>
__global__ void __launch_bounds__(TW_THREADS, 1)
gram_tcp_kernel(const __grid_constant__ CUtensorMap tmx, int nz, int nx, int nt /* rows tiled */, int tb, int T,
                const Box* __restrict__ boxes, const float* __restrict__ gz, const float* __restrict__ gx,
                const unsigned* __restrict__ xmax_bits, int nstg, int nraw, double* __restrict__ part,
                int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full_bar[TG_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TG_STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ __align__(8) uint64_t accfree_bar;
  __shared__ __align__(8) uint64_t rfull_bar[2];
  __shared__ __align__(8) uint64_t rempty_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ float wts[2][TG_PX];

  const int k = blockIdx.y, ta = blockIdx.x / T, tbk = blockIdx.x % T;
  const bool same = ta == tbk;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ra0 = ta * tb, rna = min(tb, nt - ra0), rb0 = tbk * tb, rnb = min(tb, nt - rb0);
  const int nbh = tc_nbh(rnb), N = 2 * nbh, rh = same ? tc_rows_hi(nbh) : N;
  const size_t a_bytes = same ? 0 : (size_t)128 * TG_K * 2, hi_bytes = (size_t)rh * TG_K * 2;
  const size_t st_bytes = a_bytes + hi_bytes + (size_t)N * TG_K * 2;
  const size_t slot_bytes = tcp_slot_bytes(tb, same);
  const Box b = boxes[k];
  const int nch = (b.x1 - b.x0 + ((nx & 1) ? 1 : (b.x0 & 1)) + TG_PX - 1) / TG_PX;
  const int nst = (b.z1 - b.z0) * nch;
  const int nchain = (nst + TG_CPA - 1) / TG_CPA;
  unsigned char* raw = smem + nstg * st_bytes;

  for (size_t e = tid; e < (nstg * st_bytes + nraw * slot_bytes) / 16; e += TW_THREADS)
    reinterpret_cast<uint4*>(smem)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int i = 0; i < nstg; ++i) {
      tc::mbar_init(&full_bar[i], TW_PROD);
      tc::mbar_init(&empty_bar[i], 1);
    }
    tc::mbar_init(&acc_bar, 1);
    tc::mbar_init(&accfree_bar, TW_PROD);
    for (int i = 0; i < nraw; ++i) {
      tc::mbar_init(&rfull_bar[i], 1);
      tc::mbar_init(&rempty_bar[i], TW_PROD);
    }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == TW_PROD) {
    // ---- MMA warp (as the one-tile kernel; A is tile a's buffer off the diagonal)
    const uint32_t idesc = tc::gp_bf16(GP) ? tc::idesc_bf16(128, N) : tc::idesc_f16(128, N);
    const uint32_t sb = tc::smem_u32(smem);
    const uint64_t da0 = tc::smem_desc(sb, 128, TG_SBO), dh0 = tc::smem_desc(sb + (uint32_t)a_bytes, 128, TG_SBO);
    const uint64_t dl0 = tc::smem_desc(sb + (uint32_t)(a_bytes + hi_bytes), 128, TG_SBO);
    bool ok = true;
    for (int i = 0; i < nst; ++i) {
      const int si = i % nstg, c = i / TG_CPA;
      if (ok) ok = tc::mbar_wait(&full_bar[si], (i / nstg) & 1);
      if (i % TG_CPA == 0 && c > 0 && ok) ok = tc::mbar_wait(&accfree_bar, (c - 1) & 1);
      ok = __all_sync(~0u, ok);
      tc::fence_after();
      const uint64_t so = (uint64_t)((si * st_bytes) >> 4);
      if (tc::elect_one()) {
#pragma unroll
        for (int ks = 0; ks < TG_K / 16; ++ks) {
          const uint64_t ad = da0 + so + (uint64_t)(16 * ks), hd = dh0 + so + (uint64_t)(16 * ks);
          const uint64_t ld = dl0 + so + (uint64_t)(16 * ks);
          tc::mma_f16(tbase, ad, hd, idesc, (i % TG_CPA == 0 && ks == 0) ? 0u : 1u);
          if constexpr (tc::gp_three_products(GP)) tc::mma_f16(tbase, ad, ld, idesc, 1u);
        }
        tc::mma_commit(&empty_bar[si]);
        if (i % TG_CPA == TG_CPA - 1 || i == nst - 1) tc::mma_commit(&acc_bar);
      }
      __syncwarp();
    }
    if (!ok && lane == 0) atomicOr(err, 1);
  } else if (warp == TW_PROD + 1) {
    // ---- loader warp: slab i into slot i mod nraw: tile b's rows, then tile a's
    bool ok = true;
    const float* gzk = gz + (size_t)k * nz;
    const float* gxk = gx + (size_t)k * nx;
    const uint32_t bytes = (uint32_t)((same ? 1 : 2) * tb * TW_ROWB);
    TcSlab q;
    q.start(0, nch);
    for (int i = 0; i < nst; ++i, q.next(nch)) {
      const int sl = i % nraw;
      if (i >= nraw && ok) ok = tc::mbar_wait(&rempty_bar[sl], ((i / nraw) - 1) & 1);
      ok = __all_sync(~0u, ok);
      const int x = q.xs(b, nx) + lane;
      wts[sl][lane] = (x >= b.x0 && x < b.x1) ? gzk[q.z(b)] * gxk[x] : 0.f;
      __syncwarp();
      if (lane == 0) {
        unsigned char* dst = raw + (size_t)sl * slot_bytes;
        tc::mbar_arrive_expect_tx(&rfull_bar[sl], bytes);
        tc::tma_load_2d(dst, &tmx, (int)q.p0(b, nx), rb0, &rfull_bar[sl]);
        if (!same) tc::tma_load_2d(dst + (size_t)tb * TW_ROWB, &tmx, (int)q.p0(b, nx), ra0, &rfull_bar[sl]);
      }
    }
    if (!ok && lane == 0) atomicOr(err, 1);
  } else {
    // ---- producer warps: pixel slots (ps, ps + 1), rows rl + 16 j of both tiles (as the one-tile
    // kernel's producers)
    const int pg = warp & 7, jh = warp >> 3, lgrp = warp & 3, cq = warp >> 2;
    const int ps = 4 * pg + 2 * (lane & 1), rl = lane >> 1;
    const float sc = tc::pow2_scale(__uint_as_float(*xmax_bits));
    const int roff = rl * TW_ROWB + ps * 8;
    const uint32_t soff = (uint32_t)((rl >> 3) * TG_SBO + (2 * ps >> 3) * 128 + (rl & 7) * 16 + (2 * ps & 7) * 2);
    const uint32_t sneg = (uint32_t)(nbh >> 3) * TG_SBO;
    const uint32_t tl = tbase + ((uint32_t)(lgrp * 32) << 16);
    const int nb16 = (N + 15) / 16;
    bool ok = true;
    auto promote = [&](int c) {
      if (ok) ok = tc::mbar_wait(&acc_bar, c & 1);
      tc::fence_after();
#pragma unroll
      for (int bq = 0; bq < 4; ++bq) {
        const int blk = cq + 4 * bq;
        if (blk < nb16) {
          uint32_t a[16], t[16];
          tc::tmem_ld16_async(tl + (uint32_t)(16 * blk), a);
          if (c > 0) tc::tmem_ld16_async(tl + TW_SUMS + (uint32_t)(16 * blk), t);
          tc::tmem_wait_ld();
          if (c > 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = __float_as_uint(__uint_as_float(a[j]) + __uint_as_float(t[j]));
          }
          tc::tmem_st16(tl + TW_SUMS + (uint32_t)(16 * blk), a);
        }
      }
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&accfree_bar);
    };
    int next_c = 0;
    for (int i = 0; i < nst; ++i) {
      const int si = i % nstg, sl = i % nraw;
      if (ok) ok = tc::mbar_wait(&rfull_bar[sl], (i / nraw) & 1);
      const float g0 = wts[sl][ps], g1 = wts[sl][ps + 1];
      // this thread's rows of both tiles into registers, then the slot goes back to the loader
      float4 vb[kTcGramNaMax / 32], va[kTcGramNaMax / 32];
      {
        const unsigned char* src = raw + (size_t)sl * slot_bytes + roff;
#pragma unroll
        for (int jj = 0; jj < kTcGramNaMax / 32; ++jj) {
          const int j = 2 * jj + jh, r = rl + 16 * j;
          vb[jj] = r < rnb ? *reinterpret_cast<const float4*>(src + j * 16 * TW_ROWB) : make_float4(0.f, 0.f, 0.f, 0.f);
          va[jj] = (!same && r < rna) ? *reinterpret_cast<const float4*>(src + (size_t)tb * TW_ROWB + j * 16 * TW_ROWB)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&rempty_bar[sl]);
      if (i >= nstg && ok) ok = tc::mbar_wait(&empty_bar[si], ((i / nstg) - 1) & 1);
      {
        unsigned char* Ahi = smem + si * st_bytes + soff;
        unsigned char* Bhi = Ahi + a_bytes;
        unsigned char* Blo = Bhi + hi_bytes;
        const float2 gg0 = make_float2(g0 * sc, g0 * sc), gg1 = make_float2(g1 * sc, g1 * sc);
        const float2 gd0 = make_float2(2.f * gg0.x, 2.f * gg0.x), gd1 = make_float2(2.f * gg1.x, 2.f * gg1.x);
#pragma unroll
        for (int jj = 0; jj < kTcGramNaMax / 32; ++jj) {
          const int j = 2 * jj + jh, r = rl + 16 * j;
          if (r < rnb) {
            const float4 v = vb[jj];
            uint32_t h0, h1, l0 = 0u, l1 = 0u;
            tc::split2_gp<GP>(make_float2(v.x, v.y), gg0, gd0, h0, l0);
            tc::split2_gp<GP>(make_float2(v.z, v.w), gg1, gd1, h1, l1);
            *reinterpret_cast<uint2*>(Bhi + j * 2 * TG_SBO) = make_uint2(h0, h1);
            *reinterpret_cast<uint2*>(Bhi + sneg + j * 2 * TG_SBO) = make_uint2(tc::neg_i_raw(h0), tc::neg_i_raw(h1));
            if constexpr (tc::gp_three_products(GP)) {
              *reinterpret_cast<uint2*>(Blo + j * 2 * TG_SBO) = make_uint2(l0, l1);
              *reinterpret_cast<uint2*>(Blo + sneg + j * 2 * TG_SBO) = make_uint2(tc::neg_i_raw(l0), tc::neg_i_raw(l1));
            }
          }
          if (!same && r < rna) {
            const float4 v = va[jj];
            *reinterpret_cast<uint2*>(Ahi + j * 2 * TG_SBO) =
                make_uint2(tc::hi2_gp<GP>(make_float2(v.x, v.y), gg0), tc::hi2_gp<GP>(make_float2(v.z, v.w), gg1));
          }
        }
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full_bar[si]);
      if (i % TG_CPA == 1 && i / TG_CPA >= 1) promote(next_c++);
    }
    while (next_c < nchain) promote(next_c++);
    if (!ok && lane == 0) atomicOr(err, 1);

    // block partial (doubles): plane 0 = Re D', plane 1 = Im D' (rows < rna, columns < rnb), through
    // shared memory for coalesced writes
    float* tr = reinterpret_cast<float*>(smem);   // [2][rna][ldt]
    const int ldt = rnb + 1 - (rnb & 1);
    tc_bar_producers();
    const int row = lgrp * 32 + lane;
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) {
      const int blk = cq + 4 * bq;
      if (blk < nb16) {
        uint32_t a[16];
        if (nchain > 0) {
          tc::tmem_ld16_async(tl + TW_SUMS + (uint32_t)(16 * blk), a);
          tc::tmem_wait_ld();
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) a[j] = 0u;
        }
        if (row < rna) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = 16 * blk + j, pl = col >= nbh ? 1 : 0, cj = col - pl * nbh;
            if (col < N && cj < rnb) tr[((size_t)pl * rna + row) * ldt + cj] = __uint_as_float(a[j]);
          }
        }
      }
    }
    tc::fence_before();
    tc_bar_producers();
    double* out = part + (((size_t)k * T + ta) * T + tbk) * 2 * (size_t)tb * tb;
    for (int e = tid; e < 2 * rna * rnb; e += 32 * TW_PROD) {
      const int pl = e / (rna * rnb), rem = e - pl * rna * rnb, r = rem / rnb, j = rem - r * rnb;
      out[(size_t)pl * tb * tb + (size_t)r * tb + j] = (double)tr[((size_t)pl * rna + r) * ldt + j];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

template <int GP>
static void launch_gram_tc_gp(const lcf_plan* P, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  const int na = P->tc_na;
  int nstg = 0, nraw = 0;
  if (P->tc_T > 1) tcp_shape(P->tc_tb, &nstg, &nraw);
  if (P->tc_T > 1 && P->tm_xa_ok && nstg > 0) {
    dim3 gb(P->tc_T * P->tc_T, P->nd);
    gram_tcp_kernel<GP><<<gb, TW_THREADS, tcp_smem_bytes(P->tc_tb, nstg, nraw), st>>>(
        P->tm_xa, c.nz, c.nx, na, P->tc_tb, P->tc_T, P->ws.box, P->ws.gz, P->ws.gx, P->ws.xmax, nstg, nraw,
        P->ws.gtc, P->ws.err);
  } else if (P->tc_T > 1) {
    dim3 gb(P->tc_T * P->tc_T, P->nd);
    gram_tcb_kernel<GP><<<gb, TG_THREADS, gram_tcb_smem_bytes(P->tc_tb), st>>>(
        P->ws.xa, c.nz, c.nx, na, P->tc_tb, P->tc_T, P->ws.box, P->ws.gz, P->ws.gx, P->ws.xmax, P->ws.gtc,
        P->ws.err);   // na rows: the augmented rows when the tiles give U too, else the residual rows
  } else {
    dim3 grid(P->tc_nsplit, P->nd);
    gram_tc_kernel<GP><<<grid, TW_THREADS, gram_tc_smem_bytes(na), st>>>(
        P->tm_xa, P->tm_xa_ok ? 1 : 0, P->ws.xa, c.nz, c.nx, na, P->ws.box, P->ws.gz, P->ws.gx, P->ws.xmax,
        P->tc_nsplit, gram_tc_stages(na), P->ws.gtc, P->ws.err);
  }
}

cudaError_t launch_gram_tc(const lcf_plan* P, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  const int na = P->tc_na;
  switch (c.gram_precision) {
    case LCF_GP_BF16X3: launch_gram_tc_gp<LCF_GP_BF16X3>(P, st); break;
    case LCF_GP_F16: launch_gram_tc_gp<LCF_GP_F16>(P, st); break;
    case LCF_GP_BF16: launch_gram_tc_gp<LCF_GP_BF16>(P, st); break;
    case LCF_GP_E4M3: launch_gram_tc_gp<LCF_GP_E4M3>(P, st); break;
    default: launch_gram_tc_gp<LCF_GP_F16X3>(P, st); break;
  }
  cudaError_t e = counted(P);
  if (e != cudaSuccess) return e;
  if (P->ndefl > kQExactMax) return launch_gram_aug(P, st, true);   // U and Q (exact products) on CUDA cores
  gram_q_kernel<<<dim3(P->q_nsplit, P->nd), 256, 0, st>>>(P->ws.xa, c.nz, c.nx, P->nt, P->ndefl, P->ws.box,
                                                          P->ws.gz, P->ws.gx, P->q_nsplit, P->ws.gq);
  e = counted(P);
  if (e != cudaSuccess || na > P->nt) return e;
  return launch_gram_aug(P, st, false);   // U for the residual-only tensor-core rows
}

// float -> double on the integer pipes (exact for normal numbers, zero, infinities and NaN;
// subnormal floats become signed zero): the conversion instruction runs on the FP64 units,
// which are few on this part
__device__ __forceinline__ double tc_f2d(float f) {
  const uint32_t u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sign);
  const uint64_t e2 = e == 0xffu ? 0x7ffu : (uint64_t)e + 896u;
  return __longlong_as_double((long long)(sign | (e2 << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}

// sums[k] = sum_s part[k][s], splits in order (coalesced); part holds FP32 partials, added in
// double-float on the FP32 pipes (~2^-48 relative, far below the partials' own rounding) and
// converted once
__global__ void gram_tc_reduce_kernel(const float* __restrict__ part, double* __restrict__ sums, int nsplit,
                                      size_t per_split) {
  const int k = blockIdx.y;
  const float* pk = part + (size_t)k * nsplit * per_split;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_split; e += (size_t)gridDim.x * blockDim.x) {
    df acc = {pk[e], 0.f};
    for (int s = 1; s < nsplit; ++s) acc = df_add_f(acc, pk[(size_t)s * per_split + e]);
    sums[(size_t)k * per_split + e] = tc_f2d(acc.hi) + tc_f2d(acc.lo);
  }
}

// FP32 partials of the one-tile tensor-core Gram at the start of gtc, their double sums after
// them (the buffer holds max(nsplit, 2) splits' worth of doubles)
size_t gram_tc_sums_offset(const lcf_plan* P) {
  const size_t per_split = (size_t)2 * P->tc_na * P->tc_na, nf = (size_t)P->nd * P->tc_nsplit * per_split;
  return (nf + 1) / 2;   // in doubles
}

cudaError_t launch_gram_assemble_tc(const lcf_plan* P, cudaStream_t st) {
  const int na = P->tc_na;
  const size_t per_split = (size_t)2 * na * na;
  double* sums = P->ws.gtc + gram_tc_sums_offset(P);
  if (P->tc_T == 1) {
    dim3 gr((unsigned)((per_split + 255) / 256), P->nd);
    gram_tc_reduce_kernel<<<gr, 256, 0, st>>>(reinterpret_cast<const float*>(P->ws.gtc), sums, P->tc_nsplit,
                                              per_split);
    cudaError_t e = counted(P);
    if (e != cudaSuccess) return e;
  }
  const int nup = P->nt * (P->nt + 1) / 2;
  // four blocks per window: each recomputes the window's W-form columns (FP64), so fewer blocks
  // cost less FP64 work in total, and four still fill the GPU at Nd = 64
  dim3 grid((nup + 255) / 256 < 4 ? (nup + 255) / 256 : 4, P->nd);
  gram_assemble_tc_kernel<<<grid, 256, gram_assemble_smem_bytes(P->nt, P->ndefl), st>>>(
      P->tc_T > 1 ? P->ws.gtc : sums, P->ws.gq, P->ws.gaug, P->aug_nsplit, P->ndefl > kQExactMax ? P->ndefl : 0,
      P->ws.phi, P->ws.xmax,
                                                 P->tc_T > 1 ? (size_t)P->tc_T * P->tc_T * 2 * P->tc_tb * P->tc_tb
                                                             : per_split,
                                                 P->tc_T, P->tc_tb, P->q_nsplit, P->nt, P->ndefl, na,
                                                 P->ws.R);
  return counted(P);
}

// Tensor map of the augmented rows for the slab loads: 8-byte elements, [n1][npix], boxes of
// kTcSlabBox x tc_na, zero fill outside.  Needs the row pitch (npix * 8 bytes) to be a multiple
// of 16; odd pixel counts keep the per-thread copies, and so does a plan whose map cannot be
// made (no driver entry point), with the same results.
cudaError_t gram_tc_make_map(lcf_plan* P) {
  P->tm_xa_ok = false;
  if (P->npix & 1) return cudaSuccess;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();   // not sticky: clear it, keep the per-thread copies
      return cudaSuccess;
    }
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaSuccess;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)P->npix, (cuuint64_t)P->n1};
  const cuuint64_t strides[1] = {(cuuint64_t)P->npix * 8};
  // one tile's rows a box (tile pairs), else all the rows of the one-tile kernel
  const cuuint32_t box[2] = {(cuuint32_t)kTcSlabBox, (cuuint32_t)(P->tc_T > 1 ? P->tc_tb : P->tc_na)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&P->tm_xa, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, P->ws.xa, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  P->tm_xa_ok = r == CUDA_SUCCESS;
  return cudaSuccess;
}

template <int GP>
static cudaError_t gram_tc_configure_gp(size_t mx) {
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<GP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  if (e != cudaSuccess) return e;
  size_t mp = 0;   // the largest tile-pair launch over every tile height
  for (int tb = 8; tb <= kTcTileMax; tb += 8) {
    int nstg = 0, nraw = 0;
    tcp_shape(tb, &nstg, &nraw);
    if (nstg > 0 && tcp_smem_bytes(tb, nstg, nraw) > mp) mp = tcp_smem_bytes(tb, nstg, nraw);
  }
  e = cudaFuncSetAttribute(gram_tcp_kernel<GP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mp);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(gram_tcb_kernel<GP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gram_tcb_smem_bytes(kTcTileMax));
}

cudaError_t gram_tc_configure() {
  size_t mx = 0;   // the largest launch over every augmented row length (three or two stages)
  for (int na = 3; na <= kTcGramNaMax; ++na) mx = gram_tc_smem_bytes(na) > mx ? gram_tc_smem_bytes(na) : mx;
  cudaError_t e = cudaFuncSetAttribute(gram_assemble_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gram_assemble_smem_bytes(kEvdNmax, kDeflateMax));
  if (e == cudaSuccess) e = gram_tc_configure_gp<LCF_GP_F16X3>(mx);
  if (e == cudaSuccess) e = gram_tc_configure_gp<LCF_GP_BF16X3>(mx);
  if (e == cudaSuccess) e = gram_tc_configure_gp<LCF_GP_F16>(mx);
  if (e == cudaSuccess) e = gram_tc_configure_gp<LCF_GP_BF16>(mx);
  if (e == cudaSuccess) e = gram_tc_configure_gp<LCF_GP_E4M3>(mx);
  return e;
}

}  // namespace lcf
