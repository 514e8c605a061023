// tc_util.cuh — thin inline-PTX wrappers for the 5th-generation tensor cores
// (tcgen05: TMEM allocation, MMA issue/commit, TMEM loads) and mbarriers,
// used by the tensor-core Gram and projection kernels (sm_103a).
//
// Operand convention: K-major, no swizzle.  A core matrix is 8 rows x 16 bytes
// (8 fp16 along K), stored as 8 consecutive 16-byte rows.  Core (row/8, k/8)
// sits at (row/8)*SBO + (k/8)*LBO; the kernels use LBO = 128 B (cores along K
// contiguous) and SBO = (K_stage/8)*128 B.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/lcf.h"

namespace lcf {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major no-swizzle operand
__device__ __forceinline__ int op_off(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor (tcgen05 format: version 1, SWIZZLE_NONE)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: kind::f16, A/B fp16, D fp32, both K-major, shape M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// the same with A and B bf16 (both operands of one kind::f16 MMA share their type)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return idesc_f16(M, N) | (1u << 7) | (1u << 10);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// one lane of a converged warp (the lowest active one) returns true
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile("{\n.reg .pred p;\nelect.sync _|p, 0xffffffff;\nselp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
  return pred != 0;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}
// the mbarrier arrives once every tcgen05 op issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the completion of the phase with the given parity, for at most
// limit_ns of wall time.  Returns false if the limit ran out (the caller
// reports a timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
  if (mbar_try(mbar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try(mbar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// 32 lanes x 16 consecutive fp32 columns of TMEM, without waiting: the registers are
// valid after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 lanes x 16 consecutive fp32 columns into TMEM; complete after tmem_wait_st()
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 consecutive fp32 columns of TMEM (lane base in taddr bits 31..16)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 2^e with m * 2^e < 2^14 (fp16 headroom for the products' inputs); 1 for m <= 0 or non-finite
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  int e;
  frexpf(m, &e);                 // m < 2^e
  return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// arrive once and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// bulk (untiled) global -> shared copy on the TMA engine; completes `bytes` on mbar.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// tiled tensor-map load of the box at (x, y) into shared memory; completes its bytes on mbar.
// The tensor map must live in kernel-parameter, constant or global memory.
__device__ __forceinline__ void tma_load_2d(void* dst_smem, const void* tmap, int x, int y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst_smem)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(mbar))
      : "memory");
}

// fp16 split of a float: v ~= hi + lo with both halves fp16 (22 significant bits)
__device__ __forceinline__ void split_f16(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}
// Packed split of a complex value x scaled by g: hi = fp16(g x), lo2 = fp16(2 (g x - hi)),
// both components at once (g x and 2 g x are exact scalings of each other, and g x - hi is
// exact, so lo2 is the doubled low half rounded once).
__device__ __forceinline__ void split2_f16(float2 x, float2 gg, float2 gg2, __half2& hi, __half2& lo2) {
  const float2 v = __fmul2_rn(x, gg), v2 = __fmul2_rn(x, gg2);
  hi = __float22half2_rn(v);
  lo2 = __float22half2_rn(__ffma2_rn(__half22float2(hi), make_float2(-2.f, -2.f), v2));
}
// ---- operand splits of the Gram's precision modes (LCF_GP_*), as raw 32-bit pairs ----
// hi: the tensor-core word pair of g x; lo2: the pair of 2 (g x - hi) (the doubled low half),
// written only by the three-product modes.
template <int GP>
__device__ __forceinline__ void split2_gp(float2 x, float2 gg, float2 gg2, uint32_t& hi, uint32_t& lo2) {
  const float2 v = __fmul2_rn(x, gg);
  if constexpr (GP == LCF_GP_F16X3) {
    __half2 h, l;
    split2_f16(x, gg, gg2, h, l);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo2 = *reinterpret_cast<const uint32_t*>(&l);
  } else if constexpr (GP == LCF_GP_BF16X3) {
    const float2 v2 = __fmul2_rn(x, gg2);
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    const __nv_bfloat162 l = __float22bfloat162_rn(__ffma2_rn(__bfloat1622float2(h), make_float2(-2.f, -2.f), v2));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo2 = *reinterpret_cast<const uint32_t*>(&l);
  } else if constexpr (GP == LCF_GP_F16) {
    const __half2 h = __float22half2_rn(v);
    hi = *reinterpret_cast<const uint32_t*>(&h);
  } else if constexpr (GP == LCF_GP_BF16) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    hi = *reinterpret_cast<const uint32_t*>(&h);
  } else {   // LCF_GP_E4M3: the nearest E4M3 value of g x 2^-6 (saturating), times 2^6, held exactly in fp16
    const __nv_fp8x2_storage_t q =
        __nv_cvt_float2_to_fp8x2(make_float2(v.x * 0.015625f, v.y * 0.015625f), __NV_SATFINITE, __NV_E4M3);
    const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3);
    const __half2 h = __hmul2(*reinterpret_cast<const __half2*>(&hr), __float2half2_rn(64.f));
    hi = *reinterpret_cast<const uint32_t*>(&h);
  }
}
// the precision mode's first-pass word pair of g x alone (the A operand of an off-diagonal tile)
template <int GP>
__device__ __forceinline__ uint32_t hi2_gp(float2 x, float2 gg) {
  uint32_t h, l;
  split2_gp<(GP == LCF_GP_F16X3 ? LCF_GP_F16 : GP == LCF_GP_BF16X3 ? LCF_GP_BF16 : GP)>(x, gg, gg, h, l);
  return h;
}
__host__ __device__ constexpr bool gp_three_products(int gp) { return gp == LCF_GP_F16X3 || gp == LCF_GP_BF16X3; }
__host__ __device__ constexpr bool gp_bf16(int gp) { return gp == LCF_GP_BF16X3 || gp == LCF_GP_BF16; }
// (a, b) -> (b, -a) on a raw pair of 16-bit words (fp16 or bf16: the sign is bit 15 of each half)
__device__ __forceinline__ uint32_t neg_i_raw(uint32_t u) { return ((u >> 16) | (u << 16)) ^ 0x80000000u; }

// (a, b) -> (b, -a): the fp16 pair of -i (a + i b)
__device__ __forceinline__ __half2 neg_i(__half2 h) {
  const __half2 sw = __lowhigh2highlow(h);
  uint32_t u = *reinterpret_cast<const uint32_t*>(&sw);
  u ^= 0x80000000u;
  return *reinterpret_cast<const __half2*>(&u);
}

}  // namespace tc
}  // namespace lcf
