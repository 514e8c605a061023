// k_mlp.cu — the learned cutoff rule: training kernels (GEMM forward and
// backward, softmax cross-entropy, AdamW) and the conversion of trained
// parameters into a plan's inference weights (bf16 matrices, FP32 biases).
//
// Network: X (Nt + 2: normalised log spectrum, window centre) -> 3 hidden
// layers of H with ReLU -> Nt logits over the cutoff k.  Flat parameter layout
// W1 (H x nin) b1, W2 (H x H) b2, W3 (H x H) b3, W4 (Nt x H) b4, row-major.
// Training is FP32 throughout (master weights, products, accumulation);
// inference (inside the EVD kernel) reads bf16 weights and accumulates in FP32.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "lcf_internal.cuh"

struct lcf_mlp {
  int device = 0, nt = 0, nin = 0, hidden = 0, nout = 0, max_batch = 0;
  size_t nparams = 0;
  float* p = nullptr;      // parameters
  float* g = nullptr;      // gradients of the last loss_grad call
  float* m = nullptr;      // AdamW first moments
  float* v = nullptr;      // AdamW second moments
  float* a1 = nullptr;     // [max_batch][H] activations
  float* a2 = nullptr;
  float* a3 = nullptr;
  float* z4 = nullptr;     // [max_batch][Nt] logits
  float* dz4 = nullptr;    // [max_batch][Nt]
  float* d1 = nullptr;     // [max_batch][H] back-propagated deltas (ping-pong)
  float* d2 = nullptr;
  float* lossv = nullptr;  // [max_batch] per-sample loss
  long long step = 0;
};

namespace lcf {

struct MlpOff {
  size_t w1, b1, w2, b2, w3, b3, w4, b4, total;
};
__host__ __device__ inline MlpOff mlp_offsets(int nin, int h, int nout) {
  MlpOff o;
  o.w1 = 0;
  o.b1 = o.w1 + (size_t)h * nin;
  o.w2 = o.b1 + h;
  o.b2 = o.w2 + (size_t)h * h;
  o.w3 = o.b2 + h;
  o.b3 = o.w3 + (size_t)h * h;
  o.w4 = o.b3 + h;
  o.b4 = o.w4 + (size_t)nout * h;
  o.total = o.b4 + nout;
  return o;
}

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

// C[i][j] = sum_l opA(i, l) opB(l, j)  (i < M, j < N, l < K), FP32.
//   opA(i, l) = TA ? A[l*lda + i] : A[i*lda + l];  opB(l, j) = TB ? B[j*ldb + l] : B[l*ldb + j]
// Epilogue: + bias[j] (EPI_BIAS), then max(., 0) (EPI_BIAS_RELU), or * (aux[i*ldc + j] > 0) (EPI_MASK).
// 64 x 64 output tile per CTA, 16-deep K slabs in shared memory, 4 x 4 outputs per thread.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256)
mlp_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                float* __restrict__ C, int ldc, const float* __restrict__ bias, const float* __restrict__ aux) {
  __shared__ float As[16][68];
  __shared__ float Bs[16][68];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  for (int l0 = 0; l0 < K; l0 += 16) {
    for (int e = tid; e < 1024; e += 256) {
      int ii, ll;
      if (TA) { ll = e >> 6; ii = e & 63; } else { ii = e >> 4; ll = e & 15; }   // walk the contiguous index
      const int i = i0 + ii, l = l0 + ll;
      float a = 0.f;
      if (i < M && l < K) a = TA ? A[(size_t)l * lda + i] : A[(size_t)i * lda + l];
      As[ll][ii] = a;
      int jj, lb;
      if (TB) { jj = e >> 4; lb = e & 15; } else { lb = e >> 6; jj = e & 63; }
      const int j = j0 + jj, lB = l0 + lb;
      float b = 0.f;
      if (j < N && lB < K) b = TB ? B[(size_t)j * ldb + lB] : B[(size_t)lB * ldb + j];
      Bs[lb][jj] = b;
    }
    __syncthreads();
#pragma unroll
    for (int ll = 0; ll < 16; ++ll) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[ll][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[ll][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i >= M || j >= N) continue;
      float v = acc[r][c];
      if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += bias[j];
      if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
      if (EPI == EPI_MASK) v = aux[(size_t)i * ldc + j] > 0.f ? v : 0.f;
      C[(size_t)i * ldc + j] = v;
    }
}

template <bool TA, bool TB, int EPI>
static cudaError_t gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                        const float* bias, const float* aux, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  mlp_gemm_kernel<TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux);
  return cudaGetLastError();
}

// Softmax cross-entropy, one warp per sample: loss[s] and dZ = (softmax - onehot(k)) / M.
__global__ void mlp_softmax_ce_kernel(const float* __restrict__ z, const int* __restrict__ k, int M, int n,
                                      float* __restrict__ dz, float* __restrict__ loss) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (s >= M) return;
  const float* zs = z + (size_t)s * n;
  float mx = -INFINITY;
  for (int j = lane; j < n; j += 32) mx = fmaxf(mx, zs[j]);
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(~0u, mx, o));
  float sum = 0.f;
  for (int j = lane; j < n; j += 32) sum += expf(zs[j] - mx);
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(~0u, sum, o);
  const int ks = k[s];
  const bool valid = ks >= 0 && ks < n;   // a label outside [0, n) gives a NaN loss and no gradient
  const float inv = 1.f / sum, invm = 1.f / (float)M;
  for (int j = lane; j < n; j += 32)
    dz[(size_t)s * n + j] = valid ? (expf(zs[j] - mx) * inv - (j == ks ? 1.f : 0.f)) * invm : 0.f;
  if (lane == 0) loss[s] = valid ? logf(sum) + mx - zs[ks] : NAN;
}

// db[j] = sum_i dZ[i][j]
__global__ void mlp_colsum_kernel(const float* __restrict__ dz, int M, int N, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int i = 0; i < M; ++i) s += dz[(size_t)i * N + j];
  db[j] = s;
}

__global__ void mlp_adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float wd,
                                 float bc1, float bc2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
  }
}

// plan inference weights: bf16 matrices (W1 | W2 | W3 | W4), FP32 biases (b1 | b2 | b3 | b4)
__global__ void mlp_to_plan_kernel(const float* __restrict__ p, int nin, int h, int nout,
                                   __nv_bfloat16* __restrict__ w, float* __restrict__ b) {
  const MlpOff o = mlp_offsets(nin, h, nout);
  const size_t nw1 = (size_t)h * nin, nw2 = (size_t)h * h, nw4 = (size_t)nout * h;
  const size_t nw = nw1 + 2 * nw2 + nw4, nb = 3 * (size_t)h + nout;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nw + nb; i += (size_t)gridDim.x * blockDim.x) {
    if (i < nw) {
      size_t src;
      if (i < nw1) src = o.w1 + i;
      else if (i < nw1 + nw2) src = o.w2 + (i - nw1);
      else if (i < nw1 + 2 * nw2) src = o.w3 + (i - nw1 - nw2);
      else src = o.w4 + (i - nw1 - 2 * nw2);
      w[i] = __float2bfloat16_rn(p[src]);
    } else {
      const size_t j = i - nw;
      size_t src;
      if (j < (size_t)h) src = o.b1 + j;
      else if (j < 2 * (size_t)h) src = o.b2 + (j - h);
      else if (j < 3 * (size_t)h) src = o.b3 + (j - 2 * h);
      else src = o.b4 + (j - 3 * h);
      b[j] = p[src];
    }
  }
}

static cudaError_t mlp_forward(lcf_mlp* N, const float* x, int batch, cudaStream_t st) {
  const MlpOff o = mlp_offsets(N->nin, N->hidden, N->nout);
  const int H = N->hidden;
  cudaError_t e = gemm<false, true, EPI_BIAS_RELU>(batch, H, N->nin, x, N->nin, N->p + o.w1, N->nin, N->a1, H,
                                                   N->p + o.b1, nullptr, st);
  if (e == cudaSuccess)
    e = gemm<false, true, EPI_BIAS_RELU>(batch, H, H, N->a1, H, N->p + o.w2, H, N->a2, H, N->p + o.b2, nullptr, st);
  if (e == cudaSuccess)
    e = gemm<false, true, EPI_BIAS_RELU>(batch, H, H, N->a2, H, N->p + o.w3, H, N->a3, H, N->p + o.b3, nullptr, st);
  if (e == cudaSuccess)
    e = gemm<false, true, EPI_BIAS>(batch, N->nout, H, N->a3, H, N->p + o.w4, H, N->z4, N->nout, N->p + o.b4,
                                    nullptr, st);
  return e;
}

static cudaError_t mlp_backward(lcf_mlp* N, const float* x, int batch, cudaStream_t st) {
  const MlpOff o = mlp_offsets(N->nin, N->hidden, N->nout);
  const int H = N->hidden, no = N->nout;
  float* g = N->g;
  cudaError_t e = gemm<true, false, EPI_STORE>(no, H, batch, N->dz4, no, N->a3, H, g + o.w4, H, nullptr, nullptr, st);
  if (e == cudaSuccess) { mlp_colsum_kernel<<<(no + 127) / 128, 128, 0, st>>>(N->dz4, batch, no, g + o.b4); e = cudaGetLastError(); }
  if (e == cudaSuccess)   // dZ3 = (dZ4 W4) * (A3 > 0)
    e = gemm<false, false, EPI_MASK>(batch, H, no, N->dz4, no, N->p + o.w4, H, N->d1, H, nullptr, N->a3, st);
  if (e == cudaSuccess) e = gemm<true, false, EPI_STORE>(H, H, batch, N->d1, H, N->a2, H, g + o.w3, H, nullptr, nullptr, st);
  if (e == cudaSuccess) { mlp_colsum_kernel<<<(H + 127) / 128, 128, 0, st>>>(N->d1, batch, H, g + o.b3); e = cudaGetLastError(); }
  if (e == cudaSuccess)   // dZ2 = (dZ3 W3) * (A2 > 0)
    e = gemm<false, false, EPI_MASK>(batch, H, H, N->d1, H, N->p + o.w3, H, N->d2, H, nullptr, N->a2, st);
  if (e == cudaSuccess) e = gemm<true, false, EPI_STORE>(H, H, batch, N->d2, H, N->a1, H, g + o.w2, H, nullptr, nullptr, st);
  if (e == cudaSuccess) { mlp_colsum_kernel<<<(H + 127) / 128, 128, 0, st>>>(N->d2, batch, H, g + o.b2); e = cudaGetLastError(); }
  if (e == cudaSuccess)   // dZ1 = (dZ2 W2) * (A1 > 0)
    e = gemm<false, false, EPI_MASK>(batch, H, H, N->d2, H, N->p + o.w2, H, N->d1, H, nullptr, N->a1, st);
  if (e == cudaSuccess)
    e = gemm<true, false, EPI_STORE>(H, N->nin, batch, N->d1, H, x, N->nin, g + o.w1, N->nin, nullptr, nullptr, st);
  if (e == cudaSuccess) { mlp_colsum_kernel<<<(H + 127) / 128, 128, 0, st>>>(N->d1, batch, H, g + o.b1); e = cudaGetLastError(); }
  return e;
}

cudaError_t mlp_plan_weights(const lcf_mlp* N, __nv_bfloat16* w, float* b, cudaStream_t st) {
  mlp_to_plan_kernel<<<256, 256, 0, st>>>(N->p, N->nin, N->hidden, N->nout, w, b);
  return cudaGetLastError();
}
size_t mlp_plan_weight_count(int nt, int hidden) {
  return (size_t)hidden * (nt + 2) + 2 * (size_t)hidden * hidden + (size_t)nt * hidden;
}
size_t mlp_plan_bias_count(int nt, int hidden) { return 3 * (size_t)hidden + nt; }

}  // namespace lcf

using namespace lcf;

namespace {
struct Dev {
  int prev = -1;
  explicit Dev(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
    else prev = -1;
  }
  ~Dev() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
void mlp_free(lcf_mlp* N) {
  float* ptrs[] = {N->p, N->g, N->m, N->v, N->a1, N->a2, N->a3, N->z4, N->dz4, N->d1, N->d2, N->lossv};
  for (float* q : ptrs)
    if (q) cudaFree(q);
}
}  // namespace

extern "C" lcf_status lcf_mlp_create(int nt, int hidden, int max_batch, int device, lcf_mlp** out) {
  if (!out) return LCF_EINVAL;
  *out = nullptr;
  if (nt < 2 || nt > kEvdNmax || hidden < 1 || hidden > kMlpHiddenMax || max_batch < 1) return LCF_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LCF_EINVAL;
  Dev guard(device);
  lcf_mlp* N = new (std::nothrow) lcf_mlp();
  if (!N) return LCF_ENOMEM;
  N->device = device; N->nt = nt; N->nin = nt + 2; N->hidden = hidden; N->nout = nt; N->max_batch = max_batch;
  N->nparams = mlp_offsets(N->nin, hidden, nt).total;
  const size_t B = (size_t)max_batch;
  cudaError_t e = cudaSuccess;
  float** bufs[] = {&N->p, &N->g, &N->m, &N->v};
  for (float** q : bufs)
    if (e == cudaSuccess) e = cudaMalloc((void**)q, N->nparams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->a1, B * hidden * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->a2, B * hidden * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->a3, B * hidden * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->d1, B * hidden * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->d2, B * hidden * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->z4, B * nt * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->dz4, B * nt * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&N->lossv, B * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(N->p, 0, N->nparams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(N->g, 0, N->nparams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(N->m, 0, N->nparams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(N->v, 0, N->nparams * sizeof(float));
  if (e != cudaSuccess) {
    mlp_free(N);
    delete N;
    return e == cudaErrorMemoryAllocation ? LCF_ENOMEM : LCF_ECUDA;
  }
  *out = N;
  return LCF_OK;
}

extern "C" size_t lcf_mlp_param_count(const lcf_mlp* N) { return N ? N->nparams : 0; }

extern "C" lcf_status lcf_mlp_set_params(lcf_mlp* N, const float* h_params) {
  if (!N || !h_params) return LCF_EINVAL;
  Dev guard(N->device);
  if (cudaMemcpy(N->p, h_params, N->nparams * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return LCF_ECUDA;
  // a new parameter vector starts a new optimisation
  if (cudaMemset(N->m, 0, N->nparams * sizeof(float)) != cudaSuccess) return LCF_ECUDA;
  if (cudaMemset(N->v, 0, N->nparams * sizeof(float)) != cudaSuccess) return LCF_ECUDA;
  N->step = 0;
  return LCF_OK;
}

extern "C" lcf_status lcf_mlp_get_params(const lcf_mlp* N, float* h_params) {
  if (!N || !h_params) return LCF_EINVAL;
  Dev guard(N->device);
  return cudaMemcpy(h_params, N->p, N->nparams * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? LCF_OK
                                                                                                      : LCF_ECUDA;
}

extern "C" lcf_status lcf_mlp_get_grads(const lcf_mlp* N, float* h_grads) {
  if (!N || !h_grads) return LCF_EINVAL;
  Dev guard(N->device);
  return cudaMemcpy(h_grads, N->g, N->nparams * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? LCF_OK
                                                                                                     : LCF_ECUDA;
}

extern "C" lcf_status lcf_mlp_forward(lcf_mlp* N, const float* d_x, int batch, float* d_logits, cudaStream_t st) {
  if (!N || !d_x || !d_logits || batch < 1 || batch > N->max_batch) return LCF_EINVAL;
  Dev guard(N->device);
  if (mlp_forward(N, d_x, batch, st) != cudaSuccess) return LCF_ECUDA;
  if (cudaMemcpyAsync(d_logits, N->z4, (size_t)batch * N->nout * sizeof(float), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return LCF_ECUDA;
  return LCF_OK;
}

extern "C" lcf_status lcf_mlp_loss_grad(lcf_mlp* N, const float* d_x, const int* d_k, int batch, float* h_loss,
                                        cudaStream_t st) {
  if (!N || !d_x || !d_k || batch < 1 || batch > N->max_batch) return LCF_EINVAL;
  Dev guard(N->device);
  if (mlp_forward(N, d_x, batch, st) != cudaSuccess) return LCF_ECUDA;
  mlp_softmax_ce_kernel<<<(batch + 7) / 8, 256, 0, st>>>(N->z4, d_k, batch, N->nout, N->dz4, N->lossv);
  if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  if (mlp_backward(N, d_x, batch, st) != cudaSuccess) return LCF_ECUDA;
  if (h_loss) {
    std::vector<float> l(batch);
    if (cudaMemcpyAsync(l.data(), N->lossv, batch * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return LCF_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LCF_ECUDA;
    double s = 0.0;
    for (float x : l) s += x;
    *h_loss = (float)(s / batch);
  }
  return LCF_OK;
}

extern "C" lcf_status lcf_mlp_adamw(lcf_mlp* N, float lr, float beta1, float beta2, float eps, float wd,
                                    cudaStream_t st) {
  if (!N || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return LCF_EINVAL;
  Dev guard(N->device);
  N->step += 1;
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)N->step));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)N->step));
  const MlpOff o = mlp_offsets(N->nin, N->hidden, N->nout);
  const size_t seg[8][2] = {{o.w1, o.b1}, {o.b1, o.w2}, {o.w2, o.b2}, {o.b2, o.w3},
                            {o.w3, o.b3}, {o.b3, o.w4}, {o.w4, o.b4}, {o.b4, o.total}};
  for (int s = 0; s < 8; ++s) {   // even segments are weight matrices (decayed), odd ones biases
    const size_t n = seg[s][1] - seg[s][0];
    const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    mlp_adamw_kernel<<<blocks, 256, 0, st>>>(N->p + seg[s][0], N->g + seg[s][0], N->m + seg[s][0],
                                             N->v + seg[s][0], n, lr, beta1, beta2, eps, (s & 1) ? 0.f : wd, bc1,
                                             bc2);
    if (cudaGetLastError() != cudaSuccess) return LCF_ECUDA;
  }
  return LCF_OK;
}

extern "C" lcf_status lcf_plan_set_mlp(lcf_plan* P, const lcf_mlp* N, float p_min) {
  if (!P || !N || N->nt != P->nt || N->device != P->device || !(p_min >= 0.f && p_min <= 2.f)) return LCF_EINVAL;
  if (P->cfg.evd_path != LCF_EVD_PAIR) return LCF_EUNSUPPORTED;
  Dev guard(P->device);
  const size_t nw = mlp_plan_weight_count(N->nt, N->hidden), nb = mlp_plan_bias_count(N->nt, N->hidden);
  if (P->mlp_hidden != N->hidden) {
    if (P->ws.mlp_w) cudaFree(P->ws.mlp_w);
    if (P->ws.mlp_b) cudaFree(P->ws.mlp_b);
    P->ws.mlp_w = nullptr;
    P->ws.mlp_b = nullptr;
    P->mlp_hidden = 0;
    if (cudaMalloc((void**)&P->ws.mlp_w, nw * sizeof(__nv_bfloat16)) != cudaSuccess) return LCF_ENOMEM;
    if (cudaMalloc((void**)&P->ws.mlp_b, nb * sizeof(float)) != cudaSuccess) return LCF_ENOMEM;
    P->ws_bytes += nw * sizeof(__nv_bfloat16) + nb * sizeof(float);
  }
  if (!P->ws.mlp_dbg) {
    const size_t nf = (size_t)P->nd * (2 * P->nt + 2);
    if (cudaMalloc((void**)&P->ws.mlp_dbg, nf * sizeof(float)) != cudaSuccess) return LCF_ENOMEM;
    if (cudaMemset(P->ws.mlp_dbg, 0, nf * sizeof(float)) != cudaSuccess) return LCF_ECUDA;
    P->ws_bytes += nf * sizeof(float);
  }
  // the plan's stream may still be reading the previous weights
  if (P->launched && cudaStreamSynchronize(P->last_stream) != cudaSuccess) return LCF_ECUDA;
  plan_drop_graphs(P);   // captured packets may point at the weights just replaced
  if (mlp_plan_weights(N, P->ws.mlp_w, P->ws.mlp_b, 0) != cudaSuccess) return LCF_ECUDA;
  if (cudaStreamSynchronize(0) != cudaSuccess) return LCF_ECUDA;
  P->mlp_hidden = N->hidden;
  P->mlp_pmin = p_min;
  for (size_t l = 1; l < P->lanes.size(); ++l) {   // the in-flight lanes use the same network
    const lcf_status s = lcf_plan_set_mlp(P->lanes[l], N, p_min);
    if (s != LCF_OK) return s;
  }
  return LCF_OK;
}

extern "C" lcf_status lcf_debug_learned(lcf_plan* P, float* features, float* logits) {
  if (!P) return LCF_EINVAL;
  if (!P->ws.mlp_dbg) return LCF_EINVAL;   // no network set
  Dev guard(P->device);
  if (P->launched && cudaStreamSynchronize(P->last_stream) != cudaSuccess) return LCF_ECUDA;
  const int n = P->nt;
  std::vector<float> h((size_t)P->nd * (2 * n + 2));
  if (cudaMemcpy(h.data(), P->ws.mlp_dbg, h.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LCF_ECUDA;
  for (int k = 0; k < P->nd; ++k) {
    const float* r = h.data() + (size_t)k * (2 * n + 2);
    if (features) memcpy(features + (size_t)k * (n + 2), r, (n + 2) * sizeof(float));
    if (logits) memcpy(logits + (size_t)k * n, r + n + 2, n * sizeof(float));
  }
  return LCF_OK;
}

extern "C" lcf_status lcf_mlp_destroy(lcf_mlp* N) {
  if (!N) return LCF_EINVAL;
  Dev guard(N->device);
  mlp_free(N);
  delete N;
  return LCF_OK;
}
