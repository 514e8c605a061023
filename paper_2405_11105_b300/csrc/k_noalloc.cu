// k_noalloc.cu — lcf_gram_noalloc: the windowed Gram stage for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: real-time acquisition threads
// that must not block on the allocator, code running under a driver or
// framework that owns all device memory, or embedded pipelines with a fixed
// memory budget.  This entry point computes every R_k of a packet with the
// scratch it needs (window tables, the centred packet, per-split partial
// Grams) in one file-scope static device array of kScratchBytes.  Every GPU
// that loads the library holds that array until the process exits.
//
// The array's host-side name is only a stand-in for the device symbol, so the
// first call on each device looks its device address up with
// cudaGetSymbolAddress (with that device current) and caches it, under a
// mutex so that first calls from several host threads are safe; that first
// call should come before any stream capture.
//
// The arithmetic is the plain path's Gram stage except for the deflation
// basis: a fixed orthonormal DCT-II basis of the slow-time axis instead of the
// plan's data-derived basis (the top eigenvectors of a subsampled global Gram,
// which would need the plan's workspace).  The Gram identity R = E^H R' E is
// exact for any basis; the basis only decides how much tissue energy is left
// in the FP32 residual sums, so the result agrees with a plan's Gram to the
// library's Gram tolerance rather than bit for bit.
//
// All calls share the array and it keeps the previous call's contents: nothing in it needs to start at
// zero (every entry that is read is written earlier in the same call), but
// calls whose work overlaps on the GPU (different streams, no ordering) race
// on it.
#include <math.h>

#include <mutex>

#include "lcf_internal.cuh"

namespace lcf {

constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static void* g_scratch_addr[64];
static bool g_scratch_ready[64];
static std::mutex g_scratch_mutex;   // guards the two tables above

__global__ void center_kernel(const float2* __restrict__ iq, const float2* __restrict__ phi,
                              float2* __restrict__ xa, int nt, int nd_defl, int npix, unsigned* xmax_bits);
__global__ void gram_simt_kernel(const float2* __restrict__ xa, int nz, int nx, int n1,
                                 const Box* __restrict__ boxes, const float* __restrict__ gz,
                                 const float* __restrict__ gx, int ntile, int nsplit,
                                 double2* __restrict__ part);
__global__ void gram_aug_kernel(const float2* __restrict__ xa, int nz, int nx, int nt, int nd_defl,
                                const Box* __restrict__ boxes, const float* __restrict__ gz,
                                const float* __restrict__ gx, int nsplit, int qrows, double2* __restrict__ aug);
__global__ void gram_assemble_kernel(const double2* __restrict__ part, const double2* __restrict__ aug,
                                     const float2* __restrict__ phi, int nsplit, int aug_nsplit, int nt,
                                     int nd_defl, double2* __restrict__ R);

// Orthonormal DCT-II slow-time vectors (the Gram stage's deflation basis)
__global__ void noalloc_basis_kernel(int nt, int nd_defl, float2* phi) {
  for (int e = threadIdx.x; e < nt * nd_defl; e += blockDim.x) {
    int j = e / nt, t = e % nt;
    double v = (j == 0) ? 1.0 / sqrt((double)nt)
                        : sqrt(2.0 / nt) * cos(3.14159265358979323846 * j * (t + 0.5) / nt);
    phi[e] = make_float2((float)v, 0.f);
  }
}

// Window geometry on the device (same definition as plan_create's):
// centres at the cell midpoints, SD = sigma_scale * cell, support clip.
__global__ void noalloc_geometry_kernel(int nz, int nx, int wz, int wx, float sigma_scale,
                                        float support_sigmas, int all_ones, float* gz, float* gx,
                                        Box* boxes) {
  const int k = blockIdx.x;
  const int iz = k / wx, ix = k % wx;
  const double dz = (double)nz / wz, dx = (double)nx / wx;
  const double cz = (iz + 0.5) * dz - 0.5, cx = (ix + 0.5) * dx - 0.5;
  const double sz = sigma_scale * dz, sx = sigma_scale * dx;
  Box b{0, nz, 0, nx};
  if (!all_ones && support_sigmas > 0.f) {
    const double hz = support_sigmas * sz, hx = support_sigmas * sx;
    b.z0 = (int)fmax(0.0, ceil(cz - hz));
    b.z1 = (int)fmin((double)nz, floor(cz + hz) + 1.0);
    b.x0 = (int)fmax(0.0, ceil(cx - hx));
    b.x1 = (int)fmin((double)nx, floor(cx + hx) + 1.0);
    if (b.z1 <= b.z0 || b.x1 <= b.x0) b = Box{0, 0, 0, 0};
  }
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    float v = 0.f;
    if (z >= b.z0 && z < b.z1) {
      double u = (z - cz) / sz;
      v = all_ones ? 1.f : (float)exp(-0.5 * u * u);
    }
    gz[(size_t)k * nz + z] = v;
  }
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    float v = 0.f;
    if (x >= b.x0 && x < b.x1) {
      double u = (x - cx) / sx;
      v = all_ones ? 1.f : (float)exp(-0.5 * u * u);
    }
    gx[(size_t)k * nx + x] = v;
  }
  if (threadIdx.x == 0) boxes[k] = b;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace lcf

using namespace lcf;

extern "C" lcf_status lcf_gram_noalloc(const lcf_config* c, const void* d_iq, void* d_R, cudaStream_t stream) {
  if (!c || !d_iq || !d_R) return LCF_EINVAL;
  if (((uintptr_t)d_iq & 7) || ((uintptr_t)d_R & 15)) return LCF_EINVAL;
  if (c->nz <= 0 || c->nx <= 0 || c->nt < 2 || c->wz <= 0 || c->wx <= 0 || c->wz > c->nz || c->wx > c->nx)
    return LCF_EINVAL;
  if (!(c->sigma_scale > 0.f) || !isfinite(c->sigma_scale) || !isfinite(c->support_sigmas)) return LCF_EINVAL;
  if (c->nt > kEvdNmax) return LCF_EUNSUPPORTED;
  // the kernels index the deflated packet in 32 bits (the bound lcf_plan_create applies), and
  // with it every size_t product below stays far from overflow
  if ((long long)c->nz * c->nx * (c->nt + kDeflateMax) > (1LL << 31)) return LCF_EUNSUPPORTED;
  const int ndefl = deflate_count(c->nt);
  const size_t nd = (size_t)c->wz * c->wx, nt = c->nt, n1 = nt + ndefl, npix = (size_t)c->nz * c->nx;
  const int tiles = (int)((nt + 63) / 64), pairs = tiles * (tiles + 1) / 2;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LCF_ECUDA;
  int sms = 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LCF_ECUDA;

  // scratch layout: gz | gx | boxes | deflation basis | deflated packet |
  //                 augmented-column partials (one per window) | residual-Gram partials
  const size_t off_gx = align256(nd * c->nz * sizeof(float));
  const size_t off_box = off_gx + align256(nd * c->nx * sizeof(float));
  const size_t off_phi = off_box + align256(nd * sizeof(Box));
  const size_t off_xa = off_phi + align256((size_t)ndefl * nt * sizeof(float2));
  const size_t off_aug = off_xa + align256(n1 * npix * sizeof(float2));
  const size_t off_part = off_aug + align256(nd * n1 * ndefl * sizeof(double2));
  const size_t per_split = nd * nt * nt * sizeof(double2);
  if (off_part + per_split > kScratchBytes) return LCF_ESCRATCH;
  int want = (int)((4 * sms + pairs * nd - 1) / (pairs * nd));
  want = want < 1 ? 1 : (want > 64 ? 64 : want);
  int nsplit = (int)((kScratchBytes - off_part) / per_split);
  if (nsplit > want) nsplit = want;

  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ready[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LCF_ECUDA;
      if (gram_simt_configure() != cudaSuccess) return LCF_ECUDA;   // long packets stage > 48 KB
      g_scratch_addr[dev] = p;
      g_scratch_ready[dev] = true;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  float* gz = reinterpret_cast<float*>(base);
  float* gx = reinterpret_cast<float*>(base + off_gx);
  Box* box = reinterpret_cast<Box*>(base + off_box);
  float2* phi = reinterpret_cast<float2*>(base + off_phi);
  float2* xa = reinterpret_cast<float2*>(base + off_xa);
  double2* aug = reinterpret_cast<double2*>(base + off_aug);
  double2* part = reinterpret_cast<double2*>(base + off_part);

  noalloc_geometry_kernel<<<(unsigned)nd, 128, 0, stream>>>(c->nz, c->nx, c->wz, c->wx, c->sigma_scale,
                                                            c->support_sigmas, c->all_ones_window, gz, gx, box);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  noalloc_basis_kernel<<<1, 256, 0, stream>>>((int)nt, ndefl, phi);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  center_kernel<<<(unsigned)((npix + 63) / 64), 256, 0, stream>>>((const float2*)d_iq, phi, xa, (int)nt, ndefl,
                                                                    (int)npix, nullptr);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  gram_aug_kernel<<<dim3(1, (unsigned)nd), 256, gram_aug_smem_bytes((int)nt, ndefl), stream>>>(
      xa, c->nz, c->nx, (int)nt, ndefl, box, gz, gx, 1, ndefl, aug);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  dim3 grid(pairs, nsplit, (unsigned)nd);
  gram_simt_kernel<<<grid, 256, 0, stream>>>(xa, c->nz, c->nx, (int)nt, box, gz, gx, tiles, nsplit, part);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  int bx = (int)((nt * nt + 255) / 256);
  dim3 ga(bx < 8 ? bx : 8, (unsigned)nd);
  gram_assemble_kernel<<<ga, 256, gram_assemble_smem_bytes((int)nt, ndefl), stream>>>(part, aug, phi, nsplit, 1, (int)nt, ndefl,
                                                                       (double2*)d_R);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  return LCF_OK;
}

extern "C" size_t lcf_gram_noalloc_scratch_bytes(void) { return kScratchBytes; }
