// lcf_internal.cuh — plan layout, double-float helpers and kernel entry
// points shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/lcf.h"

namespace lcf {

// Largest packet length of the library (the distributed EVD spreads A and V
// over a cluster of up to 8 CTAs).
constexpr int kEvdNmax = 320;
// Largest packet length of the CTA-pair EVD (A in one SM's shared memory, V
// in its partner's); longer packets use the distributed EVD.
constexpr int kEvdPairNmax = 128;
// Largest packet length of the one-CTA EVD (A and V in one SM's shared memory).
constexpr int kEvdCtaNmax = 112;
// Longest packet of the shared-memory-resident projections (CUDA-core with the
// whole W_k in shared memory; tensor-core with the tile's rows resident).
constexpr int kProjectShortNmax = 128;
// Largest augmented row (Nt + deflation vectors) of the tensor-core Gram (one M = 128 tile).
constexpr int kTcGramNaMax = 128;
constexpr int kTcTileMax = 112;   // row tile of the long-packet tensor-core Gram (three stages fit)
constexpr int kTcSlabBox = 34;    // pixels per tensor-core Gram slab load (32 used; 272-byte rows)
// Subspace-iteration block of the EVD (head directions isolated exactly).
constexpr int kEvdHead = 8;
// Slow-time vectors (the packet's dominant global modes) deflated from every pixel
// before the Gram: at most kDeflateMax; by default clamp(Nt/4, 1, 4), which leaves
// blood-and-noise-level residuals for sub-pixel tissue motion; strong motion
// (about a pixel and more) needs 8-16 (lcf_config.deflate).
constexpr int kDeflateMax = 16;
constexpr int kDeflateDefaultMax = 4;
// Deflation depths up to this take the coefficient block Q from the register-resident
// exact-product kernel (gram_q_kernel); deeper ones from the augmented-column kernel.
constexpr int kQExactMax = 4;
__host__ __device__ inline int deflate_count(int nt) {
  int d = nt / 4;
  return d < 1 ? 1 : (d > kDeflateDefaultMax ? kDeflateDefaultMax : d);
}
// the plan's deflation depth: cfg->deflate when set, else the default for nt
__host__ __device__ inline int deflate_depth(int nt, int deflate) { return deflate > 0 ? deflate : deflate_count(nt); }
// EVD phases timed by the stage profiler: subspace iteration, QR of the block,
// double-float congruence, fp32 conversion + Q, Jacobi, sort + phase fix,
// thresholding rule, projection weights.
constexpr int kEvdPhases = 8;
// Widest hidden layer of the learned cutoff rule (its activations live in shared memory).
constexpr int kMlpHiddenMax = 256;
// Calls whose stage events are kept between profile reads.
constexpr int kProfCalls = 4096;

struct Box { int z0, z1, x0, x1; };

struct Workspace {
  // geometry
  float* gz = nullptr;        // [nd][nz] Gaussian factor along z (0 outside support)
  float* gx = nullptr;        // [nd][nx]
  Box* box = nullptr;         // [nd]
  // deflated packet: s_p = c_p + sum_j a_pj phi_j
  float2* phi = nullptr;      // [ndefl][nt] per-packet slow-time deflation basis (complex)
  float2* gglob = nullptr;    // [basis_nsplit][nt][nt] partial global Grams (basis estimate)
  float2* gglob_async = nullptr;  // the same for the pipelined host calls' prep stream
  float2* xa = nullptr;       // [nt+ndefl][nz*nx]: residual c_p(t), then coefficients a_pj
  // Gram
  double2* gpart = nullptr;   // [nd][nsplit][nt][nt] partial residual Grams
  double2* gaug = nullptr;    // [nd][aug_nsplit][(nt+ndefl)*ndefl] partial augmented columns
  unsigned* xmax = nullptr;   // [1] max |component| of the deflated packet (float bits)
  float2* phi_alt = nullptr;  // the other staging parity's basis and packet maximum (pipelined
  unsigned* xmax_alt = nullptr;  // host calls swap them with phi / xmax packet by packet)
  double* gtc = nullptr;      // f32 [nd][tc_nsplit][2][na][na] tensor-core partials (Re, Im planes)
                              // then their f64 sums [nd][2][na][na]; or f64 [nd][T][T][2][tb][tb]
                              // tile-pair partials for long packets
  double2* gq = nullptr;      // [nd][q_nsplit][kQExactMax^2] exact coefficient-block partials
  int* err = nullptr;         // [1] device error word (bit 0: a bounded wait gave up)
  double2* R = nullptr;       // [nd][nt][nt] windowed Gram (Eq. 12)
  // EVD + weights
  double* lam = nullptr;      // [nd][nt] descending eigenvalues
  float2* V = nullptr;        // [nd][nt][nt] eigenvectors (columns)
  float* wt = nullptr;        // [nd][nt]
  int* kcut = nullptr;        // [nd]
  float* alpha = nullptr;     // [nd]
  int* flags = nullptr;       // [nd]
  float2* W = nullptr;        // [nd][nt][ncp] projection weights V diag(wt sqrt(alpha/Nt))
  float2* pw = nullptr;       // [nd][kDeflateMax][ncp] Phi^T W (long-packet CUDA-core projection)
  int* ncol = nullptr;        // [nd]
  // tensor-core projection
  int* tile_off = nullptr;    // [ntiles+1] CSR offsets of the windows meeting each 8x16 tile
  int* tile_win = nullptr;    // window indices, ascending per tile
  unsigned char* bimg = nullptr;  // [nd] pre-split weight images (fp16 hi/lo, MMA layout)
  float* bscale = nullptr;    // [nd] power-of-two scale of each weight image
  long long* evd_clk = nullptr;  // [nd][kEvdPhases+1] EVD phase clocks (profiling only)
  // distributed EVD (Nt > kEvdPairNmax)
  float2* evd_B = nullptr;    // [nd][nt][nt] B = Q^H (R/scale) Q, fp32
  float2* evd_vh = nullptr;   // [nd][m][nt] Householder vectors of Q
  float2* evd_t = nullptr;    // [nd][m][m] compact WY factor T
  double* evd_scale = nullptr;// [nd] power-of-two scale (0: degenerate window)
  int* evd_perm = nullptr;     // [nd][nt] pivot order of the Cholesky factor (one-sided EVD, Nt > 128)
  int* evd_rank = nullptr;     // [nd] its numerical rank
  // learned cutoff rule (set by lcf_plan_set_mlp)
  __nv_bfloat16* mlp_w = nullptr;   // W1 | W2 | W3 | W4, bf16
  float* mlp_b = nullptr;           // b1 | b2 | b3 | b4
  float* mlp_dbg = nullptr;         // [nd][2 nt + 2] the last call's network inputs and logits
  // after the EVD: FP64-class polish and method 4 (k_post.cu)
  double* post_rq = nullptr;  // [nd][ceil(nt/16)][nt] Rayleigh-quotient partials
  float2* post_pv = nullptr;  // [nd][kDeflateMax][nt] Phi^T V
  float* post_isig = nullptr; // [nd][nt] 1 / sigma_i
  double* post_band = nullptr;  // [nd][ncc_nsplit][nt][10] magnitude-Gram band partials
  // subtractive reconstruction (Eq. 5, cfg.project_form = LCF_PF_SUBTRACT; k_subtract.cu)
  float2* sub_qhi = nullptr;  // [nd][nt][nt] orthonormalised rejected columns, high words
  float2* sub_qlo = nullptr;  // ... low words
  long long* sub_off = nullptr;  // [nd] offset of each window's box in sub_pdk
  float* sub_pdk = nullptr;   // [sum of box pixels] PD_k of every window's pixels
  double* sub_part = nullptr; // [nd][sub_nsplit] sums of PD_k
  // host-call staging
  float2* iq_stage = nullptr; // [2][nt][nz][nx] device copies for lcf_filter_host(_async)
  float* pd_stage = nullptr;  // [2][nz][nx]
};

}  // namespace lcf

struct lcf_plan {
  lcf_config cfg;
  int device = 0;
  int nd = 0, nt = 0, n1 = 0, npix = 0;
  int ndefl = 1;        // deflated slow-time vectors; the augmented row has nt + ndefl entries
  int aug_nsplit = 1;   // pixel splits of the augmented-column kernel
  int tc_nsplit = 1;    // pixel ranges per window of the tensor-core Gram
  int tc_na = 0;        // rows of the tensor-core Gram: nt + ndefl when that fits one MMA tile, else nt
  int tc_T = 1, tc_tb = 0;  // row tiles of the residual block (T > 1 for Nt > 128) and their size
                        // (the coefficient columns U then come from the CUDA-core kernel)
  int q_nsplit = 1;     // pixel splits of the exact coefficient-block kernel
  int basis_nsplit = 1; // pixel splits of the global Gram behind the deflation basis
  int gram_tiles = 0;   // 64-wide tiles per Gram dimension
  int gram_nsplit = 1;  // pixel splits per window
  int ncp = 0;          // padded projection columns
  int ptiles_z = 0, ptiles_x = 0;   // tensor-core projection tiles (8 x 16 pixels)
  int mlp_hidden = 0;   // hidden width of the plan's learned rule (0: none set)
  float mlp_pmin = 0.f; // confidence below which the learned rule falls back to k_src
  int ncc_nsplit = 1;   // pixel splits per window of method 4's band sums
  int evd_cluster = 0;  // CTAs per window of the distributed EVD (Nt > 128)
  int sub_nsplit = 1;   // pixel splits per window of the subtractive projection
  int sm_count = 0;
  std::vector<lcf::Box> boxes;
  lcf::Workspace ws;
  size_t ws_bytes = 0;
  // xa as a 2-D tensor of 8-byte elements ([n1 rows][npix]), boxes of kTcSlabBox pixels x tc_na
  // rows: the tensor-core Gram's slab loads (valid when npix is even and tc_T == 1)
  CUtensorMap tm_xa{};
  bool tm_xa_ok = false;
  cudaStream_t last_stream = nullptr;       // stream of the latest call (0 = the legacy default stream)
  bool launched = false;                    // some call has put work on last_stream
  cudaStream_t h2d_stream = nullptr;        // copy stream of lcf_filter_host_async
  cudaEvent_t ev_in[2] = {nullptr, nullptr};  // staging buffer b filled
  cudaEvent_t ev_done[2] = {nullptr, nullptr};  // staging buffer b consumed
  long long host_seq = 0;                   // pipelined host calls so far
  cudaStream_t prep_stream = nullptr;       // their basis prep, overlapping the previous packet's kernels
  cudaEvent_t ev_prep[2] = {nullptr, nullptr};  // staging buffer b's basis ready
  int basis_par = 0;                        // parity whose basis / maximum are phi / xmax now
  long long pipe_seq = 0;                   // packets whose basis prep ran on the prep stream
  cudaEvent_t ev_pdone[2] = {nullptr, nullptr};  // end of the last such packet of basis parity p
  cudaEvent_t ev_seq = nullptr;             // end of the latest other filter call on its stream
  bool seq_since_async = false;             // ... not yet waited for by the prep stream
  void* last_iq = nullptr;
  // stage profiling: events[call % kProfCalls][stage boundary]
  // kernels this plan has launched (every launcher adds its own)
  mutable long long launches = 0;
  // the last stream of packets, captured as one CUDA graph (lcf_filter_stream)
  cudaStream_t cap_stream = nullptr;
  // single-packet graphs of lcf_filter (cfg.graph), one per (input, output) pair, oldest replaced
  static constexpr int kPacketGraphs = 16;
  struct PacketGraph {
    const void* iq = nullptr;
    float* out = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    long long used = 0;
  } pg[kPacketGraphs];
  long long pg_clock = 0;
  cudaGraphExec_t sg_exec = nullptr;
  const void* sg_frames = nullptr;
  float* sg_out = nullptr;
  int sg_n = 0, sg_stride = 0;
  long long sg_launches = 0;
  // packets in flight (cfg.inflight > 1): lane 0 is this plan, lanes 1.. are sub-plans with
  // their own workspaces; every lane has a plan-owned stream
  std::vector<lcf_plan*> lanes;
  std::vector<cudaStream_t> lane_st;
  std::vector<cudaEvent_t> lane_ev;
  cudaEvent_t ev_many = nullptr;
  long long lane_seq = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;
  long prof_calls = 0;
};

namespace lcf {

// ----- double-float (two FP32 words) arithmetic on the FP32 pipes -----
// B300's FP64 rate is ~1/62 of FP32, so extended precision is built from
// error-free FP32 transformations (Knuth two-sum, FMA two-product).
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
// a * b with a double-float and b float
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return quick_two_sum(p, e);
}
// exact product of two floats as a double-float
__device__ __forceinline__ df two_prod_df(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_from_double(double d) {
  float h = (float)d;
  return {h, (float)(d - (double)h)};
}
// d * 2^-ex as a double-float, on the integer pipes (the double -> float conversion instruction
// runs on the FP64 units, which are few on this part): hi = the top 24 significand bits, lo = the
// next 29 bits rounded down to 24, renormalised; |error| < 2^-47 |d|.  Zero, subnormal doubles
// and results below the float range give zero; overflow and inf / NaN give inf / NaN in hi.
__device__ __forceinline__ df df_from_double_scaled(double d, int ex) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const int e = (int)((u >> 52) & 0x7ffu);
  const unsigned long long mant = u & 0xfffffffffffffull;
  if (e == 0) return {__uint_as_float(sign), 0.f};
  if (e == 0x7ff) return {__uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u)), 0.f};
  const int E = e - 1023 - ex;   // unbiased exponent of the scaled value
  if (E + 127 >= 255) return {__uint_as_float(sign | 0x7f800000u), 0.f};
  if (E + 127 <= 0) return {__uint_as_float(sign), 0.f};
  const float hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | (unsigned)(mant >> 29));
  const unsigned mr = (unsigned)(mant & 0x1fffffffull);   // remainder: mr * 2^(E - 52)
  float lo = 0.f;
  if (mr) {
    const int hb = 31 - __clz(mr);                      // leading bit of the remainder
    const int fe = hb + E - 52 + 127;
    if (fe > 0) {
      const unsigned m24 = hb >= 23 ? (mr >> (hb - 23)) : (mr << (23 - hb));
      lo = __uint_as_float(sign | ((unsigned)fe << 23) | (m24 & 0x7fffffu));
    }
  }
  return quick_two_sum(hi, lo);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// complex double-float
struct zdf { df re, im; };
__device__ __forceinline__ zdf zdf_add(zdf a, zdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
// (a) * (b) with a complex double-float and b complex float
__device__ __forceinline__ zdf zdf_mul_c(zdf a, float2 b) {
  df rr = df_mul_f(a.re, b.x), ii = df_mul_f(a.im, b.y);
  df ri = df_mul_f(a.re, b.y), ir = df_mul_f(a.im, b.x);
  return {df_add(rr, df_neg(ii)), df_add(ri, ir)};
}

// ----- complex float helpers -----
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// W = U + 1/2 conj(Phi) Q for rows i (one thread per (i, a)); with it the E^H R' E
// terms beyond the residual block are W Phi^T + (W Phi^T)^H (Q Hermitian).
__device__ __forceinline__ double2 deflated_w(int i, int a, int nd_defl, const double2 (*U)[kDeflateMax],
                                              const double2 (*Q)[kDeflateMax], const double2 (*ph)[kEvdNmax]) {
  double2 w = U[i][a];
  for (int c = 0; c < nd_defl; ++c) {          // 1/2 sum_c conj(phi_c(i)) Q[c][a]
    const double2 f = ph[c][i], q = Q[c][a];
    w.x += 0.5 * (f.x * q.x + f.y * q.y);
    w.y += 0.5 * (f.x * q.y - f.y * q.x);
  }
  return w;
}
// r += sum_a W_ia phi_a(j) + conj(sum_a W_ja phi_a(i))
__device__ __forceinline__ void add_w_terms(double2& r, int i, int j, int nd_defl, const double2 (*Wm)[kDeflateMax],
                                            const double2 (*ph)[kEvdNmax]) {
  for (int a = 0; a < nd_defl; ++a) {
    const double2 wi = Wm[i][a], fj = ph[a][j], wj = Wm[j][a], fi = ph[a][i];
    r.x += (wi.x * fj.x - wi.y * fj.y) + (wj.x * fi.x - wj.y * fi.y);
    r.y += (wi.x * fj.y + wi.y * fj.x) - (wj.x * fi.y + wj.y * fi.x);
  }
}

// ----- launchers (each returns cudaGetLastError() after the launch) -----
// Call after each kernel launch of a plan: counts it in P->launches.
inline cudaError_t counted(const lcf_plan* P, int n = 1) {
  P->launches += n;
  return cudaGetLastError();
}
cudaError_t launch_center(const lcf_plan* P, const float2* iq, cudaStream_t st);
cudaError_t launch_gram_aug(const lcf_plan* P, cudaStream_t st, bool with_q = true);
size_t gram_aug_smem_bytes(int nt, int nd_defl);
size_t gram_assemble_smem_bytes(int nt, int nd_defl);
cudaError_t gram_simt_configure();
cudaError_t launch_basis(const lcf_plan* P, const float2* iq, cudaStream_t st);
cudaError_t basis_configure();
cudaError_t launch_gram_simt(const lcf_plan* P, cudaStream_t st);
cudaError_t launch_gram_tc(const lcf_plan* P, cudaStream_t st);
cudaError_t launch_gram_assemble_tc(const lcf_plan* P, cudaStream_t st);
cudaError_t gram_tc_configure();
cudaError_t gram_tc_make_map(lcf_plan* P);
size_t gram_tc_smem_bytes(int na);
cudaError_t launch_gram_assemble(const lcf_plan* P, cudaStream_t st);
cudaError_t launch_evd(const lcf_plan* P, cudaStream_t st);
cudaError_t mlp_plan_weights(const lcf_mlp* N, __nv_bfloat16* w, float* b, cudaStream_t st);
size_t mlp_plan_weight_count(int nt, int hidden);
size_t mlp_plan_bias_count(int nt, int hidden);
cudaError_t launch_evd_pair(const lcf_plan* P, cudaStream_t st);
cudaError_t launch_evd_dist(const lcf_plan* P, cudaStream_t st);
// B = Q^H (R / scale) Q (fp32, full Hermitian), the reflectors, T and the scale of every window,
// from `iters` subspace iterations (the first stage of the distributed and one-sided EVDs)
cudaError_t launch_evd_prep(const lcf_plan* P, cudaStream_t st, int iters);
cudaError_t launch_evd_os(const lcf_plan* P, cudaStream_t st);
// one-sided EVD for 128 < Nt <= kEvdOscNmax: Cholesky kernel, then a cluster of four CTAs per window
constexpr int kEvdOscNmax = 224;
cudaError_t launch_evd_osc(const lcf_plan* P, cudaStream_t st);
cudaError_t evd_osc_configure();
cudaError_t evd_os_configure();
size_t evd_os_smem_bytes(int nt);
cudaError_t evd_dist_configure();
cudaError_t evd_pair_configure();
cudaError_t launch_project_simt(const lcf_plan* P, const float2* iq, float* out, cudaStream_t st);
cudaError_t launch_project_tc(const lcf_plan* P, float* out, cudaStream_t st);
cudaError_t project_tc_configure();
size_t project_tc_image_bytes(int nt, int nd_defl);
void project_tc_tiles(const lcf_plan* P, int* tiles_z, int* tiles_x, std::vector<int>& off, std::vector<int>& win);
cudaError_t launch_filtered_iq(const lcf_plan* P, const float2* iq, int subset, float2* out,
                               cudaStream_t st);
size_t evd_smem_bytes(int nt);
cudaError_t evd_configure();
cudaError_t project_configure();
int project_cpt(int nt);
bool post_uses_ncc(const lcf_config& c);
int post_rq_blocks(int nt);
size_t post_band_count(const lcf_plan* P);
cudaError_t post_configure();
cudaError_t launch_post(const lcf_plan* P, cudaStream_t st);
void plan_drop_graphs(lcf_plan* P);
lcf_status packet_once(lcf_plan* P, const float2* iq, float* out, cudaStream_t st);
cudaError_t launch_project_subtract(const lcf_plan* P, const float2* iq, float* out, cudaStream_t st);
size_t sub_prep_smem_bytes(int n);
int evd_dist_cluster(int nt);
size_t evd_dist_smem_bytes(int nt, int C);

}  // namespace lcf
