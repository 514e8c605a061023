// k_project_tc.cu — projection, |.|^2 slow-time reduction and blend on the
// 5th-generation tensor cores (tcgen05), Eq. 4 and Eq. 13.
//
// As on the CUDA-core path, V unitary turns the per-window filter into
//   PD(p) = sum_k g_k(p)^2 sum_c |s_p W_k(:,c)|^2,  W_k = V diag(wt sqrt(alpha/Nt)),
// one GEMM per window.  Here the rows come from the deflated packet of the
// Gram stage, s_p = c_p + sum_j a_pj phi_j^T, so
//   s_p W = [c_p, a_p] [W ; Phi^T W]
// and the clutter that the global basis removes never enters the fp16 operands:
// the residual c_p and the coefficients a_p are each split hi + lo (22 bits),
// as are the augmented weights, and three passes (hi.hi, hi.lo, lo.hi) with
// FP32 accumulation in TMEM give the product to ~2^-22.  The complex product
// needs no real embedding: with S = Sr + i Si and W = Wr + i Wi,
//   Yr = Sr Wr - Si Wi,   Yi = Si Wr + Sr Wi,
// four real GEMMs sharing the operands (the minus sign is the MMA's negate-A
// bit), into two TMEM accumulators per window.
//
// Work split: one CTA per 8 x 16-pixel tile (M = 128 rows, one per TMEM lane).
// The tile's [c_p, a_p] rows are staged once in shared memory (fp16 hi/lo,
// K-major); the windows whose support meets the tile are taken in a fixed order,
// each window's pre-split weight image streamed by the TMA engine through a
// 3-stage ring.  Warp 0 issues the copies, warp 1 the MMAs, warps 4-7 read the
// accumulators (double-buffered, so the next window's MMAs overlap the read) and
// keep the blended pixel in a register: every pixel is written once, no atomics.
#include <math.h>

#include "lcf_internal.cuh"
#include "tc_util.cuh"

namespace lcf {

constexpr int PT_THREADS = 256;
constexpr int PT_TX = 16;                // tile: 16 columns x (8 rows, fewer for long packets)
constexpr int PT_KS_MAX = 2;             // k-steps (16 K each) per weight stage, at most
constexpr int PT_STAGES = 3;
constexpr int PT_ACC = 256;              // TMEM columns per accumulator buffer (Yr at +0, Yi at +128)

int pt_k16(int nt, int nd_defl) { return (nt + nd_defl + 15) / 16 * 16; }
__host__ __device__ inline int pt_n16(int ncol) { return (ncol + 15) / 16 * 16; }
// One k-step of a window's weight image: Wr hi, Wr lo, Wi hi, Wi lo, each n16 rows x 16 K (fp16).
__host__ __device__ inline int pt_kstep_bytes(int n16) { return 4 * n16 * 32; }
// offset of (column c, k index kk < 16) inside one n16 x 16 sub-image (K-major, SBO = 256 B)
__device__ __forceinline__ int pt_b_off(int c, int kk) { return (c >> 3) * 256 + (kk >> 3) * 128 + (c & 7) * 16 + (kk & 7) * 2; }

// Long packets (Nt > kProjectShortNmax): the weight columns are taken in chunks of at most
// PT_NCH (one accumulator buffer each), the image is chunk-major with 128-row sub-images
// (PT_LKB bytes per k-step and chunk), and the tile keeps fewer pixel rows resident
// (tile_rows(): 16 x tz pixels, the MMA's remaining rows read past the plane and are ignored).
constexpr int PT_NCH = 128;
constexpr int PT_LKB = 4 * PT_NCH * 32;
constexpr size_t PT_SMEM_MAX = 232448;
__host__ __device__ inline bool pt_long(int nt) { return nt > kProjectShortNmax; }
__host__ __device__ inline int pt_nchunks(int n16) { return (n16 + PT_NCH - 1) / PT_NCH; }

size_t project_tc_image_bytes(int nt, int nd_defl) {
  const int nks = pt_k16(nt, nd_defl) / 16, n16 = pt_n16(nt);
  if (pt_long(nt)) return (size_t)pt_nchunks(n16) * nks * PT_LKB;
  return (size_t)nks * pt_kstep_bytes(n16);
}

static size_t pt_stage_bytes(int nt) { return pt_long(nt) ? (size_t)PT_LKB : (size_t)pt_kstep_bytes(pt_n16(nt)); }
static size_t pt_smem(int nt, int nd_defl, int ksps, int rows) {
  return 1024 + 4 * (size_t)rows * pt_k16(nt, nd_defl) * 2 + (size_t)PT_STAGES * ksps * pt_stage_bytes(nt);
}
// resident pixel rows of a tile: 128 for short packets, else the most that fit beside the ring
int project_tc_tile_rows(int nt, int nd_defl) {
  if (!pt_long(nt)) return 128;
  int tz = 8;
  while (tz > 1 && pt_smem(nt, nd_defl, 1, 16 * tz) > PT_SMEM_MAX) --tz;
  return 16 * tz;
}
// k-steps per ring stage: two unless the stages would not fit beside the resident rows
static int project_tc_ksps(int nt, int nd_defl) {
  if (pt_long(nt)) return 1;
  return pt_smem(nt, nd_defl, PT_KS_MAX, 128) <= PT_SMEM_MAX ? PT_KS_MAX : 1;
}
size_t project_tc_smem_bytes(int nt, int nd_defl, int ksps) {
  return pt_smem(nt, nd_defl, ksps, project_tc_tile_rows(nt, nd_defl));
}

// ---------------------------------------------------------------------------
// Weight images.  One CTA per window: the augmented block [W ; Phi^T W]
// (rows t < Nt: W, rows Nt + j: phi_j^T W, double-float sums), scaled by a power of two
// into fp16 range and split hi/lo, laid out k-step by k-step in the exact
// shared-memory image the MMA reads.
__global__ void __launch_bounds__(512)
project_prep_kernel(const float2* __restrict__ W, const int* __restrict__ ncol, const float2* __restrict__ phi,
                    int nt, int nd_defl, int ncp, int k16, int n16max, unsigned char* __restrict__ bimg,
                    float* __restrict__ bscale) {
  const int k = blockIdx.x, tid = threadIdx.x;
  const int nc = ncol[k], n16 = pt_n16(nc);
  const float2* Wk = W + (size_t)k * nt * ncp;
  __shared__ float2 PW[kDeflateMax][kEvdNmax];   // phi_j^T W(:, c)
  __shared__ float red[16];
  for (int e = tid; e < nd_defl * nc; e += blockDim.x) {   // phi_j^T W(:, c), double-float sums
    const int j = e / nc, c = e % nc;
    df sr = {0.f, 0.f}, si = {0.f, 0.f};
    // unrolled so that the loads run ahead of the (serial) double-float sums
#pragma unroll 10
    for (int t = 0; t < nt; ++t) {
      const float2 f = phi[j * nt + t], w = Wk[(size_t)t * ncp + c];
      sr = df_add(sr, df_add(two_prod_df(f.x, w.x), df_neg(two_prod_df(f.y, w.y))));
      si = df_add(si, df_add(two_prod_df(f.x, w.y), two_prod_df(f.y, w.x)));
    }
    PW[j][c] = make_float2(sr.hi + sr.lo, si.hi + si.lo);
  }
  __syncthreads();
  float m = 0.f;
  for (int e = tid; e < nt * nc; e += blockDim.x) {
    const float2 w = Wk[(size_t)(e / nc) * ncp + e % nc];
    m = fmaxf(m, fmaxf(fabsf(w.x), fabsf(w.y)));
  }
  for (int e = tid; e < nd_defl * nc; e += blockDim.x) {
    const float2 w = PW[e / nc][e % nc];
    m = fmaxf(m, fmaxf(fabsf(w.x), fabsf(w.y)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(~0u, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  if (tid < 32) {
    float v = tid < (int)(blockDim.x >> 5) ? red[tid] : 0.f;
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(~0u, v, o));
    if (tid == 0) red[0] = v;
  }
  __syncthreads();
  const float s = tc::pow2_scale(red[0]);
  if (tid == 0) bscale[k] = s;
  const bool lng = pt_long(nt);
  const int nks = k16 / 16;
  unsigned char* img = bimg + (size_t)k * (lng ? (size_t)pt_nchunks(n16max) * nks * PT_LKB
                                               : (size_t)nks * pt_kstep_bytes(n16max));
  const int kb = lng ? PT_LKB : pt_kstep_bytes(n16), sub = lng ? PT_NCH * 32 : n16 * 32;
  // one item = 8 consecutive rows t of column c: one 16-byte core-matrix row of each sub-image
  for (int e = tid; e < (k16 / 8) * n16; e += blockDim.x) {
    const int o = e / n16, c = e % n16, t0 = 8 * o;
    __align__(16) __half hr[8];
    __align__(16) __half lr[8];
    __align__(16) __half hi[8];
    __align__(16) __half li[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u;
      float2 v = make_float2(0.f, 0.f);
      if (c < nc) {
        if (t < nt) v = Wk[(size_t)t * ncp + c];
        else if (t < nt + nd_defl) v = PW[t - nt][c];
      }
      tc::split_f16(v.x * s, hr[u], lr[u]);
      tc::split_f16(v.y * s, hi[u], li[u]);
    }
    unsigned char* base = lng ? img + ((size_t)(c / PT_NCH) * nks + (t0 >> 4)) * PT_LKB + pt_b_off(c % PT_NCH, t0 & 15)
                              : img + (size_t)(t0 >> 4) * kb + pt_b_off(c, t0 & 15);
    *reinterpret_cast<uint4*>(base) = *reinterpret_cast<const uint4*>(hr);
    *reinterpret_cast<uint4*>(base + sub) = *reinterpret_cast<const uint4*>(lr);
    *reinterpret_cast<uint4*>(base + 2 * sub) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(base + 3 * sub) = *reinterpret_cast<const uint4*>(li);
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PT_THREADS, 1)
project_tc_kernel(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl, int k16, int n16max,
                  int ksps, int rows, int tiles_x, const int* __restrict__ tile_off, const int* __restrict__ tile_win,
                  const float* __restrict__ gz, const float* __restrict__ gx, const unsigned* __restrict__ xmax_bits,
                  const int* __restrict__ ncol, const unsigned char* __restrict__ bimg,
                  const float* __restrict__ bscale, float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[PT_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[PT_STAGES];
  __shared__ __align__(8) uint64_t accf[2];
  __shared__ __align__(8) uint64_t acce[2];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tz = rows / PT_TX;   // tile: tz x 16 pixels (rows pixels), 128 MMA rows
  const int tile = blockIdx.x, z0 = (tile / tiles_x) * tz, x0 = (tile % tiles_x) * PT_TX;
  const int w0 = tile_off[tile], w1 = tile_off[tile + 1];
  const int na = nt + nd_defl, nks = k16 / 16, nstw = (nks + ksps - 1) / ksps;
  const size_t npix = (size_t)nz * nx;
  const int a_sbo = (k16 / 8) * 128;
  const size_t a_bytes = (size_t)rows * k16 * 2;           // one of Sr hi, Sr lo, Si hi, Si lo
  unsigned char* A = smem;
  unsigned char* Bring = smem + 4 * a_bytes;
  const bool lng = pt_long(nt);
  const size_t st_bytes = (size_t)ksps * (lng ? (size_t)PT_LKB : (size_t)pt_kstep_bytes(n16max));
  const size_t img_stride = lng ? (size_t)pt_nchunks(n16max) * nks * PT_LKB : (size_t)nks * pt_kstep_bytes(n16max);
  const float sA = tc::pow2_scale(__uint_as_float(*xmax_bits));

  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int i = 0; i < PT_STAGES; ++i) {
      tc::mbar_init(&full_bar[i], 1);
      tc::mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&accf[i], 1);
      tc::mbar_init(&acce[i], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // ---- stage the tile's rows [c_p, a_p] (scaled, split hi/lo), zero K padding ----
  // item i: lane -> (row%8, k-pair), so a warp's 4-byte stores hit 32 distinct banks;
  // four items per thread at a time, their eight loads issued before any is split
  const int nitems = rows * (k16 / 2), rg = rows / 8;
  for (int i0 = tid; i0 < nitems; i0 += 4 * PT_THREADS) {
    float2 v0[4], v1[4];
    int mm[4], tt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * PT_THREADS;
      const int ln = i & 31, rest = i >> 5;
      mm[u] = (rest % rg) * 8 + (ln & 7);
      tt[u] = (rest / rg) * 8 + (ln >> 3) * 2;
      const int z = z0 + (mm[u] >> 4), x = x0 + (mm[u] & 15);
      v0[u] = make_float2(0.f, 0.f);
      v1[u] = v0[u];
      if (i < nitems && z < nz && x < nx) {
        const size_t p = (size_t)z * nx + x;
        if (tt[u] < na) v0[u] = xa[(size_t)tt[u] * npix + p];
        if (tt[u] + 1 < na) v1[u] = xa[(size_t)(tt[u] + 1) * npix + p];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (i0 + u * PT_THREADS >= nitems) break;
      __half h0r, l0r, h1r, l1r, h0i, l0i, h1i, l1i;
      tc::split_f16(v0[u].x * sA, h0r, l0r);
      tc::split_f16(v1[u].x * sA, h1r, l1r);
      tc::split_f16(v0[u].y * sA, h0i, l0i);
      tc::split_f16(v1[u].y * sA, h1i, l1i);
      const int off = tc::op_off(mm[u], tt[u], a_sbo);
      *reinterpret_cast<__half2*>(A + off) = __halves2half2(h0r, h1r);
      *reinterpret_cast<__half2*>(A + a_bytes + off) = __halves2half2(l0r, l1r);
      *reinterpret_cast<__half2*>(A + 2 * a_bytes + off) = __halves2half2(h0i, h1i);
      *reinterpret_cast<__half2*>(A + 3 * a_bytes + off) = __halves2half2(l0i, l1i);
    }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tmem_base;
  bool ok = true;

  if (warp == 0) {
    // ---------------- producer: weight stages through the ring ----------------
    if (lane == 0) {
      int q = 0;
      for (int wi = w0; wi < w1 && ok; ++wi) {
        const int k = tile_win[wi], nc = ncol[k];
        if (nc == 0) continue;
        const int kb = lng ? PT_LKB : pt_kstep_bytes(pt_n16(nc)), nch = lng ? pt_nchunks(pt_n16(nc)) : 1;
        for (int ch = 0; ch < nch && ok; ++ch) {
          const unsigned char* img = bimg + (size_t)k * img_stride + (size_t)ch * nks * kb;
          for (int s = 0; s < nstw; ++s, ++q) {
            const int slot = q % PT_STAGES;
            if (q >= PT_STAGES && !(ok = tc::mbar_wait(&empty_bar[slot], ((q / PT_STAGES) - 1) & 1))) break;
            const int nk = min(ksps, nks - s * ksps);
            const uint32_t bytes = (uint32_t)(nk * kb);
            tc::mbar_arrive_expect_tx(&full_bar[slot], bytes);
            tc::bulk_g2s(Bring + slot * st_bytes, img + (size_t)s * ksps * kb, bytes, &full_bar[slot]);
          }
        }
      }
      // the copies still in flight land before the CTA exits
      for (int r = 1; r <= PT_STAGES && r <= q; ++r) {
        const int qq = q - r;
        tc::mbar_wait(&full_bar[qq % PT_STAGES], (qq / PT_STAGES) & 1, 200000000ull);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp runs the loop (warp-uniform counters and
    // descriptors), one elected lane issues ----------------
    {
      int q = 0, j = 0;
      // descriptors advance in 16-byte units: a k-step is two core matrices (256 bytes) of A
      const uint64_t d_srh = tc::smem_desc(tc::smem_u32(A), 128, a_sbo);
      const uint64_t d_srl = tc::smem_desc(tc::smem_u32(A + a_bytes), 128, a_sbo);
      const uint64_t d_sih = tc::smem_desc(tc::smem_u32(A + 2 * a_bytes), 128, a_sbo);
      const uint64_t d_sil = tc::smem_desc(tc::smem_u32(A + 3 * a_bytes), 128, a_sbo);
      const uint64_t d_b = tc::smem_desc(tc::smem_u32(Bring), 128, 256);
      for (int wi = w0; wi < w1 && ok; ++wi) {
       const int k = tile_win[wi], nc = ncol[k];
       const int n16w = pt_n16(nc), nch = nc == 0 ? 0 : (lng ? pt_nchunks(n16w) : 1);
       for (int ch = 0; ch < nch && ok; ++ch) {
        const int n16 = lng ? min(PT_NCH, n16w - ch * PT_NCH) : n16w;
        const int kb = lng ? PT_LKB : pt_kstep_bytes(n16), sub = lng ? PT_NCH * 32 : n16 * 32;
        const int buf = j & 1;
        if (j >= 2 && !(ok = __all_sync(~0u, tc::mbar_wait(&acce[buf], ((j >> 1) - 1) & 1)))) break;
        tc::fence_after();
        const uint32_t idesc = tc::idesc_f16(128, n16), idesc_neg = idesc | (1u << 13);   // bit 13: negate A
        const uint32_t dr = tbase + (uint32_t)(buf * PT_ACC), di = dr + 128;
        for (int s = 0; s < nstw; ++s, ++q) {
          const int slot = q % PT_STAGES;
          if (!(ok = __all_sync(~0u, tc::mbar_wait(&full_bar[slot], (q / PT_STAGES) & 1)))) break;
          tc::fence_after();
          const int nk = min(ksps, nks - s * ksps);
          if (tc::elect_one()) {
          for (int kl = 0; kl < nk; ++kl) {
            const int ks = s * ksps + kl;
            const uint64_t ao = (uint64_t)(16 * ks);
            const uint64_t srh = d_srh + ao, srl = d_srl + ao, sih = d_sih + ao, sil = d_sil + ao;
            const uint64_t bo = (uint64_t)((slot * st_bytes + (size_t)kl * kb) >> 4), so = (uint64_t)(sub >> 4);
            const uint64_t wrh = d_b + bo, wrl = wrh + so, wih = wrl + so, wil = wih + so;
            const uint32_t acc = ks == 0 ? 0u : 1u;
            // Yr = Sr Wr - Si Wi
            tc::mma_f16(dr, srh, wrh, idesc, acc);
            tc::mma_f16(dr, srh, wrl, idesc, 1u);
            tc::mma_f16(dr, srl, wrh, idesc, 1u);
            tc::mma_f16(dr, sih, wih, idesc_neg, 1u);
            tc::mma_f16(dr, sih, wil, idesc_neg, 1u);
            tc::mma_f16(dr, sil, wih, idesc_neg, 1u);
            // Yi = Si Wr + Sr Wi
            tc::mma_f16(di, sih, wrh, idesc, acc);
            tc::mma_f16(di, sih, wrl, idesc, 1u);
            tc::mma_f16(di, sil, wrh, idesc, 1u);
            tc::mma_f16(di, srh, wih, idesc, 1u);
            tc::mma_f16(di, srh, wil, idesc, 1u);
            tc::mma_f16(di, srl, wih, idesc, 1u);
          }
          tc::mma_commit(&empty_bar[slot]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (tc::elect_one()) tc::mma_commit(&accf[buf]);
        __syncwarp();
        ++j;
       }
      }
      // every MMA this warp issued has completed before TMEM is released
      if (j > 0) tc::mbar_wait(&accf[(j - 1) & 1], ((j - 1) >> 1) & 1, 200000000ull);
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: |Y|^2 row sums, window weights, blend ----------------
    const int m = (warp - 4) * 32 + lane;
    const int z = z0 + (m >> 4), x = x0 + (m & 15);
    const bool inside = m < rows && z < nz && x < nx;
    float pd = 0.f;
    int j = 0;
    for (int wi = w0; wi < w1 && ok; ++wi) {
     const int k = tile_win[wi], nc = ncol[k];
     const int n16w = pt_n16(nc), nch = nc == 0 ? 0 : (lng ? pt_nchunks(n16w) : 1);
     for (int ch = 0; ch < nch; ++ch) {
      const int n16 = lng ? min(PT_NCH, n16w - ch * PT_NCH) : n16w, buf = j & 1;
      // warp-uniform outcome: the TMEM loads below are .sync.aligned
      if (!(ok = __all_sync(~0u, tc::mbar_wait(&accf[buf], (j >> 1) & 1)))) break;
      tc::fence_after();
      const uint32_t base = tbase + (uint32_t)(buf * PT_ACC) + ((uint32_t)((warp & 3) * 32) << 16);
      float acc = 0.f;
      for (int c = 0; c < n16; c += 16) {   // Yr and Yi columns c..c+15, one wait for both
        uint32_t vr[16], vi[16];
        tc::tmem_ld16_async(base + c, vr);
        tc::tmem_ld16_async(base + 128 + c, vi);
        tc::tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float a = __uint_as_float(vr[u]), b2 = __uint_as_float(vi[u]);
          acc = fmaf(a, a, fmaf(b2, b2, acc));
        }
      }
      tc::fence_before();
      tc::mbar_arrive(&acce[buf]);
      if (inside) {
        const float g = gz[(size_t)k * nz + z] * gx[(size_t)k * nx + x];
        const float inv = 1.f / (sA * bscale[k]);
        pd = fmaf(g * g * inv * inv, acc, pd);
      }
      ++j;
     }
    }
    if (inside) out[(size_t)z * nx + x] = pd;
  }
  if (!ok) atomicOr(err, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

cudaError_t launch_project_tc(const lcf_plan* P, float* out, cudaStream_t st) {
  const lcf_config& c = P->cfg;
  const int k16 = pt_k16(P->nt, P->ndefl), n16max = pt_n16(P->nt);
  project_prep_kernel<<<P->nd, 512, 0, st>>>(P->ws.W, P->ws.ncol, P->ws.phi, P->nt, P->ndefl, P->ncp, k16, n16max,
                                             P->ws.bimg, P->ws.bscale);
  cudaError_t e = counted(P);
  if (e != cudaSuccess) return e;
  const int ksps = project_tc_ksps(P->nt, P->ndefl), rows = project_tc_tile_rows(P->nt, P->ndefl);
  project_tc_kernel<<<P->ptiles_z * P->ptiles_x, PT_THREADS, project_tc_smem_bytes(P->nt, P->ndefl, ksps), st>>>(
      P->ws.xa, c.nz, c.nx, P->nt, P->ndefl, k16, n16max, ksps, rows, P->ptiles_x, P->ws.tile_off, P->ws.tile_win, P->ws.gz,
      P->ws.gx, P->ws.xmax, P->ws.ncol, P->ws.bimg, P->ws.bscale, out, P->ws.err);
  return counted(P);
}

cudaError_t project_tc_configure() {
  size_t mx = 0;   // the largest launch over every packet length and deflation depth
  for (int nt = 2; nt <= kEvdNmax; ++nt)
    for (int d = 1; d <= kDeflateMax && d < nt + (nt == 2); ++d) {
      const size_t b = project_tc_smem_bytes(nt, d, project_tc_ksps(nt, d));
      mx = b > mx ? b : mx;
    }
  return cudaFuncSetAttribute(project_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
}

void project_tc_tiles(const lcf_plan* P, int* tiles_z, int* tiles_x, std::vector<int>& off, std::vector<int>& win) {
  const lcf_config& c = P->cfg;
  const int trz = project_tc_tile_rows(P->nt, P->ndefl) / PT_TX;   // tile rows (z)
  *tiles_z = (c.nz + trz - 1) / trz;
  *tiles_x = (c.nx + PT_TX - 1) / PT_TX;
  off.assign(1, 0);
  win.clear();
  for (int tz = 0; tz < *tiles_z; ++tz)
    for (int tx = 0; tx < *tiles_x; ++tx) {
      const int za = tz * trz, zb = za + trz, xa0 = tx * PT_TX, xb = xa0 + PT_TX;
      for (int k = 0; k < P->nd; ++k) {
        const Box& b = P->boxes[k];
        if (b.z1 <= b.z0 || b.x1 <= b.x0) continue;
        if (b.z0 < zb && za < b.z1 && b.x0 < xb && xa0 < b.x1) win.push_back(k);
      }
      off.push_back((int)win.size());
    }
}

}  // namespace lcf
