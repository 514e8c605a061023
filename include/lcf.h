/*
 * lcf.h — C ABI of the B300 (sm_103a) localized Gaussian-windowed EVD
 * clutter filter (Huang, Lok, Zhang, Liu, Chen: "Real-time Adaptive and
 * Localized Spatiotemporal Clutter Filtering for Ultrasound Small Vessel
 * Imaging").
 *
 * One call turns a packet of complex IQ data S (Nz x Nx pixels x Nt
 * slow-time frames) into one power-Doppler image:
 *
 *   for every 2-D Gaussian window g_k (Eq. 11; centres and SD set by the
 *   number of subsets):
 *     R_k = C_w^H C_w = sum_p g_k(p)^2 s_p^H s_p        (Eq. 1, Eq. 12)
 *     R_k = V_k Lambda_k V_k^H, lambda descending       (Eq. 2)
 *     wt_k from an eigenvalue thresholding rule          (methods 1-3, 5, 6;
 *                                                         Eq. 6, 7, 9, 10)
 *     PD_k(p) = mean_t |(C_w V_k diag(wt_k) V_k^H)(p,t)|^2  (Eq. 4)
 *   PD = sum_k alpha_k PD_k,  alpha_k = 1 / mean_p PD_k  (Eq. 13)
 *
 * Layout: the packet is iq[t][z][x], complex64 (float re, float im
 * interleaved), x fastest, with no padding (pitch = Nx).  The PD image is
 * out_pd[z][x], float32.
 *
 * Ownership: the caller owns every buffer it passes.  A plan owns all device
 * workspace it needs; lcf_filter allocates nothing, never synchronises, and
 * writes every pixel of out_pd (it never accumulates into caller memory).
 * A plan may be used from one stream at a time.
 *
 * Errors: argument errors return synchronously (LCF_EINVAL, nothing is
 * launched).  CUDA launch errors return LCF_ECUDA.  Conditions found on the
 * device (a Jacobi sweep cap hit, a subset with zero flow power) are written
 * to a per-window status word that lcf_plan_status reads.
 */
#ifndef LCF_H_
#define LCF_H_

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lcf_plan lcf_plan;
typedef struct lcf_mlp lcf_mlp;

typedef enum {
  LCF_OK = 0,
  LCF_EINVAL = 1,        /* bad argument or configuration                     */
  LCF_ENOMEM = 2,        /* device or host allocation failed at plan_create    */
  LCF_ECUDA = 3,         /* a CUDA call failed (launch, copy, capture)          */
  LCF_ENOCONV = 4,       /* some window's Jacobi EVD hit its sweep cap          */
  LCF_ETIMEOUT = 5,      /* a bounded device-side wait gave up                  */
  LCF_EDEGENERATE = 6,   /* some window had zero flow power (its alpha set 0)   */
  LCF_EUNSUPPORTED = 7,  /* valid request this build does not implement         */
  LCF_ESCRATCH = 8       /* problem too large for lcf_gram_noalloc's static
                            scratch (see lcf_gram_noalloc_scratch_bytes)        */
} lcf_status;

/* Eigenvalue thresholding rules (the paper's methods; k = number of
 * rejected components, i = 1..Nt in descending eigenvalue order). */
enum {
  LCF_T_FIXED = 0,          /* hard, fixed k = k_fixed                             */
  LCF_T_CURVATURE = 1,      /* method 1, Eq. 6: max curvature of the normalised
                               log10-eigenvalue curve (scaling factor beta)       */
  LCF_T_SLOPE = 2,          /* method 2: leading components whose normalised
                               log-curve descent is steeper than beta             */
  LCF_T_MEDIAN = 3,         /* method 3, Eq. 7: reject lambda > beta * median      */
  LCF_T_SIGMOID = 4,        /* method 5, Eq. 9: wt_i = 1/(1+exp(-beta (i-k))),
                               k from rule k_src with factor beta_src             */
  LCF_T_ADAPTIVE_SOFT = 5,  /* method 6, Eq. 10: wt_i ~ win(i) / lambda_i^beta    */
  LCF_T_NONE = 6,           /* wt = 1 (identity reconstruction, for checks)       */
  LCF_T_LEARNED = 7,        /* hard cutoff k from the plan's learned rule (an MLP
                               set by lcf_plan_set_mlp; no counterpart in the
                               paper); below its confidence threshold the window
                               falls back to rule k_src with factor beta_src     */
  LCF_T_NCC = 8             /* method 4, Eq. 8: the k (fn <= k <= Nt - fn, fn =
                               min(5, Nt/2)) minimising the normalised spatial
                               cross-correlation of the tissue image
                               sum_{i=k-fn+1..k} |u_i| and the blood image
                               sum_{i=k+1..k+fn} |u_i|, u_i = C_w v_i / sigma_i;
                               also a k_src of LCF_T_SIGMOID (method 5 at
                               method 4's k, as the paper evaluates it)          */
};

/* Status bits per window (lcf_plan_status). */
/* Bits 8-15 of a window's status word hold the number of Jacobi sweeps its
 * EVD used (for tuning and convergence monitoring). */
/* LCF_WFLAG_FALLBACK: the learned rule was not confident and k_src decided. */
enum { LCF_WFLAG_NOCONV = 1, LCF_WFLAG_DEGENERATE = 2, LCF_WFLAG_FALLBACK = 4, LCF_WFLAG_SWEEP_SHIFT = 8 };

/* Compute paths.  LCF_PATH_SIMT is the plain FP32 GPU path (CUDA cores,
 * FP32 products, FP32 partial sums promoted to double-float);
 * LCF_PATH_TC runs the Gram and the projection on the tcgen05 tensor cores
 * as split-FP16 (hi + lo, three products) contractions with FP32
 * accumulation promoted to double-float. */
enum { LCF_PATH_SIMT = 0, LCF_PATH_TC = 1 };

/* EVD kernels.  LCF_EVD_CTA: one CTA per window holds A and V (plain path).
 * LCF_EVD_PAIR: a two-CTA cluster per window; one CTA runs the Jacobi
 * rotations on A and streams them through distributed shared memory to the
 * other, which accumulates V.  Same arithmetic and tolerances.
 * LCF_EVD_OS: one-sided Jacobi (Hestenes) on the pivoted FP32 Cholesky factor
 * of the same deflated matrix, the factor's columns in registers: one CTA per
 * window up to Nt = 128, a four-CTA cluster per window (rows split across the
 * CTAs) up to Nt = 224; the eigenvectors are the converged columns, so no V is
 * accumulated.  Longer packets take the distributed two-sided kernel.  Same
 * tolerances; one SM per window at Nt <= 128 (the CTA pair holds two), which
 * leaves room for other packets in flight (cfg.inflight).  The learned rule
 * needs LCF_EVD_PAIR.
 * All three: Eq. 2. */
enum { LCF_EVD_CTA = 0, LCF_EVD_PAIR = 1, LCF_EVD_OS = 2 };

/* Product precision of the tensor-core Gram (gram_path = LCF_PATH_TC; the
 * plain path's products are FP32).  Each weighted component of the deflated
 * packet is scaled by a power of two and split into tensor-core words; the
 * MMAs accumulate in FP32, promoted to double-float across chains.
 *   LCF_GP_F16X3   fp16 hi + lo (22 significant bits); products hi*hi +
 *                  hi*lo + lo*hi (default)
 *   LCF_GP_BF16X3  bf16 hi + lo (16 bits); the same three products on bf16 MMAs
 *   LCF_GP_F16     fp16 hi only (11 bits, TF32's significand; the scaled packet
 *                  lies inside fp16's range, so every product equals the TF32
 *                  product of the same operands), one MMA pass
 *   LCF_GP_BF16    bf16 hi only (8 bits), one pass
 *   LCF_GP_E4M3    FP8 E4M3 operands (4 bits, saturating at 448 after a
 *                  power-of-two scale), one pass on the fp16 MMA, which holds
 *                  E4M3 values and their products exactly: the precision study's
 *                  FP8 case (not an FP8 MMA instruction). */
enum { LCF_GP_F16X3 = 0, LCF_GP_BF16X3 = 1, LCF_GP_F16 = 2, LCF_GP_BF16 = 3, LCF_GP_E4M3 = 4 };

/* Eigen-decomposition precision (Eq. 2 on every path).
 *   LCF_EP_FP32        FP32 Jacobi rotations after a double-float congruence
 *                      that isolates the dominant subspace (default)
 *   LCF_EP_FP64_POLISH the same, then every eigenvalue is replaced by the
 *                      Rayleigh quotient v^H R v / v^H v of its FP32 eigenvector
 *                      against the FP64 Gram, formed in double-float; the
 *                      eigenpairs are re-sorted and the rule, alpha (Eq. 13) and
 *                      the projection weights use the polished values.  For
 *                      packets whose kept eigenvalues lie near the FP32 unit
 *                      roundoff of lambda_1 (60 dB tissue-to-blood, long packets). */
enum { LCF_EP_FP32 = 0, LCF_EP_FP64_POLISH = 1 };

/* How the power Doppler is formed from the eigen-decomposition (both equal Eq. 4
 * for hard weights, Eq. 5 being the paper's subtractive form of it).
 *   LCF_PF_IDENTITY  PD_k(p) = (1/Nt) sum_c wt_c^2 |(C_w V)(p, c)|^2 over the kept
 *                    columns: one GEMM per window (default; every rule)
 *   LCF_PF_SUBTRACT  Eq. 5, C-hat = C_w - C_w V_k V_k^H: PD_k(p) = (1/Nt)(||C_w(p,:)||^2
 *                    - ||C_w(p,:) Q||^2), Q the k rejected eigenvectors
 *                    re-orthonormalised in double-float, every sum double-float,
 *                    alpha (Eq. 13) from the same sums.  Hard rules only (fixed,
 *                    methods 1-4, learned, none); its cost grows with k instead of
 *                    Nt - k. */
enum { LCF_PF_IDENTITY = 0, LCF_PF_SUBTRACT = 1 };

typedef struct {
  int nz, nx, nt;          /* packet size: Nz axial x Nx lateral x Nt frames      */
  int wz, wx;              /* window grid; Nd = wz*wx subsets                     */
  float sigma_scale;       /* window SD = sigma_scale * window spacing (1.0)      */
  float support_sigmas;    /* support clipped to |delta| <= this many SD (3.0);
                              <= 0: no clipping                                    */
  int all_ones_window;     /* 1: g == 1 on the whole image (global filter)       */
  int thresh_mode;         /* LCF_T_*                                             */
  float beta;              /* the rule's scaling factor                           */
  int k_fixed;             /* k of LCF_T_FIXED (and of a FIXED k_src)             */
  int k_src;               /* rule that supplies k to LCF_T_SIGMOID (FIXED..MEDIAN
                              or LCF_T_NCC)                                        */
  float beta_src;          /* scaling factor of that rule                         */
  int pd_mode;             /* 0: PD = mean over slow time, 1: sum                 */
  int alpha_mode;          /* 0: alpha_k = Nz*Nx / sum PD_k (Eq. 13, default);
                              1: alpha_k = 1; 2: mean over the window support     */
  int curv_norm;           /* method 1/2 curve: 0 shifted to [0, beta*Nt];
                              1 literal beta*y(n)/y(1)*Nt                          */
  int gram_path;           /* LCF_PATH_*                                          */
  int project_path;        /* LCF_PATH_*                                          */
  int max_sweeps;          /* Jacobi sweep cap per level (<= 0: 40)               */
  int evd_path;            /* LCF_EVD_*                                           */
  int inputs_ready;        /* 1: every lcf_filter input is complete when the call  */
                           /* is made (e.g. a resident packet ring), so each       */
                           /* packet's basis prep starts on a plan-owned stream    */
                           /* while the previous packet's kernels run; 0 (default):*/
                           /* the input is read in `stream` order                  */
  int gram_precision;      /* LCF_GP_* (tensor-core Gram only; 0 = LCF_GP_F16X3)  */
  int evd_precision;       /* LCF_EP_* (0 = LCF_EP_FP32)                          */
  int graph;               /* 1: lcf_filter runs each packet as one CUDA graph
                              launch (captured on the first call with a given
                              (d_iq, d_out_pd) pair, up to 16 pairs per plan;
                              capturing allocates the graph); 0 (default): the
                              stages are launched one by one.  Not combined
                              with inputs_ready's early basis prep, nor used
                              while stage profiling is on                        */
  int project_form;        /* LCF_PF_*: how PD is formed after the EVD            */
  int deflate;             /* slow-time vectors deflated from every pixel before
                              the Gram and projection products, 1..16 (< Nt);
                              0: clamp(Nt/4, 1, 4).  The deflated part is summed
                              with exact double-float products, so only the
                              residual meets the FP32 / tensor-core products:
                              strong tissue motion (a pixel or more) needs 8-16
                              to bring the residual down to blood and noise     */
  int inflight;            /* packets lcf_filter_many and lcf_filter_host_async
                              keep in progress at once, 1..4 (0: 1).  Each
                              packet beyond the first has its own workspace and
                              plan-owned stream, so the EVD of one packet (which
                              holds one SM per window) runs beside the other
                              stages and EVDs of the next: more images per
                              second, the same time per image.  No counterpart
                              in the paper, which filters one packet at a time */
} lcf_config;

/* Fill *cfg with defaults for an nz x nx x nt packet and a wz x wx grid:
 * sigma_scale 1, support 3 SD, curvature rule beta 1, PD mean, alpha by
 * Eq. 13, the fast path: tensor-core Gram and projection (LCF_PATH_TC) and the
 * cluster EVD (LCF_EVD_PAIR), 40-sweep cap.  The plain FP32 path is
 * gram_path = project_path = LCF_PATH_SIMT with evd_path = LCF_EVD_CTA. */
lcf_status lcf_config_default(lcf_config* cfg, int nz, int nx, int nt, int wz, int wx);

/* Validate cfg, build the window geometry (Eq. 11) and allocate all device
 * workspace on `device`.  Synchronous.  On success *out owns the workspace
 * until lcf_plan_destroy.  Returns LCF_EINVAL (cfg invalid), LCF_ENOMEM,
 * LCF_ECUDA or LCF_EUNSUPPORTED (e.g. nt beyond the EVD kernel's limit). */
lcf_status lcf_plan_create(const lcf_config* cfg, int device, lcf_plan** out);

/* Filter one packet.  d_iq: device pointer to iq[nt][nz][nx] complex64
 * (8-byte aligned).  d_out_pd: device pointer to out_pd[nz][nx] float32.
 * Asynchronous on `stream`; no allocation, no synchronisation.  d_iq is read
 * in `stream` order, except with cfg.inputs_ready set, where the packet's
 * basis prep may read it on a plan-owned stream as soon as the call is made
 * (so d_iq must be complete then); the image is written in `stream` order
 * either way. */
lcf_status lcf_filter(lcf_plan* plan, const void* d_iq, float* d_out_pd, cudaStream_t stream);

/* Same computation with HOST buffers: copies h_iq to the device, filters,
 * copies the image back to h_out_pd and synchronises `stream`.  Pinned host
 * memory makes the copies asynchronous DMA; pageable memory also works. */
lcf_status lcf_filter_host(lcf_plan* plan, const void* h_iq, float* h_out_pd, cudaStream_t stream);

/* Pipelined form of lcf_filter_host for a sequence of packets: returns without
 * synchronising.  The packet's host-to-device copy runs on a plan-owned copy
 * stream into one of two device staging buffers (alternating between calls),
 * so it overlaps the previous packet's kernels on `stream`; so does the
 * packet's deflation-basis prep, on a second plan-owned stream once the copy
 * is in (the basis and packet maximum are kept per staging buffer); the image
 * is copied back to h_out_pd on `stream`.  Other filter calls on the same plan
 * may be interleaved (the next pipelined prep waits for them).  h_iq must stay unchanged and h_out_pd must not
 * be read until lcf_plan_sync returns (pinned host memory required for the
 * overlap).  Calls of one plan must use the same `stream`.  The first call
 * creates the copy stream and its events.  With cfg.inflight > 1 consecutive
 * calls rotate over the plan's lanes: each lane pipelines its own packets on
 * its own plan-owned stream (after the work queued on `stream` before the
 * call), so up to inflight packets compute at once. */
lcf_status lcf_filter_host_async(lcf_plan* plan, const void* h_iq, float* h_out_pd, cudaStream_t stream);

/* Wait for every copy and kernel of the plan's pipelined host calls (every lane). */
lcf_status lcf_plan_sync(lcf_plan* plan);

/* Sliding-packet processing (packets of nt frames every `stride` frames, as
 * the paper's real-time processing does).  d_frames: device frames
 * [n_frames][nz][nx] complex64; d_out_pd: [n_packets][nz][nx] with
 * n_packets = (n_frames - nt) / stride + 1.  Asynchronous.  All packets run
 * as one CUDA graph: the first call with a given (d_frames, n_frames, stride,
 * d_out_pd) captures it on a plan-owned stream (this first call allocates the
 * graph; later calls with the same buffers only launch it on `stream`).  While
 * stage profiling is on, the packets are launched one by one instead. */
lcf_status lcf_filter_stream(lcf_plan* plan, const void* d_frames, int n_frames, int stride,
                             float* d_out_pd, cudaStream_t stream);

/* Synchronise the plan's last stream and read the per-window status words of
 * the last filter call into per_window_flags[Nd] (host, may be NULL).
 * Returns LCF_ENOCONV / LCF_EDEGENERATE if any window raised that flag. */
lcf_status lcf_plan_status(lcf_plan* plan, int* per_window_flags);

/* Copy the last call's intermediates to host memory (synchronises).  Any
 * pointer may be NULL.  eig: [Nd][Nt] eigenvalues, descending; wt: [Nd][Nt]
 * weights; k: [Nd] cutoffs (-1 for soft rules); alpha: [Nd]. */
lcf_status lcf_debug_dump(lcf_plan* plan, double* eig, float* wt, int* k, float* alpha);

/* Copy the last call's windowed Gram matrices R_k (Eq. 12) to host:
 * R: [Nd][Nt][Nt] complex double (re, im interleaved, row-major). */
lcf_status lcf_debug_gram(lcf_plan* plan, double* R);

/* Copy the last call's eigenvectors to host: V: [Nd][Nt][Nt] complex
 * float, column j = eigenvector of eig[j] (row-major, V[i][j]). */
lcf_status lcf_debug_eigvecs(lcf_plan* plan, float* V);

/* Reconstruct the filtered IQ of one subset (Eq. 4, C-hat = C_w V Lambda-hat
 * V^H) from the last call's eigen-decomposition, for validation.  d_iq is
 * the same packet; d_filt: device [nt][nz][nx] complex64, zero outside the
 * subset's support.  Asynchronous. */
lcf_status lcf_debug_filtered_iq(lcf_plan* plan, const void* d_iq, int subset, void* d_filt,
                                 cudaStream_t stream);

/* Number of windows and the support box of window k: box = {z0, z1, x0, x1}
 * (half-open). */
lcf_status lcf_plan_windows(lcf_plan* plan, int* nd, int k, int* box);

/* Pipeline stages, in launch order, for lcf_plan_profile_read. */
enum {
  LCF_STAGE_PREP = 0,      /* packet centring (and split-precision staging)     */
  LCF_STAGE_GRAM = 1,      /* windowed Gram contraction (Eq. 12)                */
  LCF_STAGE_ASSEMBLE = 2,  /* cross-split reduction, Hermitian assembly         */
  LCF_STAGE_EVD = 3,       /* EVD (Eq. 2), thresholding, alpha (Eq. 13)        */
  LCF_STAGE_PROJECT = 4,   /* projection, |.|^2 reduction and blend (Eq. 4, 13) */
  LCF_NSTAGES = 5
};

/* Turn per-stage device timing on (enable != 0) or off.  While on, every
 * filter call records CUDA events between its stages on the call's stream
 * (no synchronisation).  Enabling resets the accumulated times.  Up to 4096
 * calls are kept between reads; older ones are dropped. */
lcf_status lcf_plan_profile(lcf_plan* plan, int enable);

/* Several independent packets (no counterpart in the paper: serving-side
 * batching).  Filters npk packets, d_iq = [npk][Nt][Nz][Nx] complex64 on the
 * device, into d_out_pd = [npk][Nz][Nx] float32 (Eq. 4, 13 per packet), with up
 * to cfg.inflight packets in progress at once: packet p runs on the plan's lane
 * p mod inflight, each lane with its own workspace and plan-owned stream.  All of
 * it starts after the work queued on `stream` before the call, and work queued
 * on `stream` after the call waits for every image.  Images equal lcf_filter's.
 * lcf_plan_status and the debug calls then describe the last packet of lane 0.
 * LCF_EINVAL for null pointers, npk < 0 or misaligned buffers. */
lcf_status lcf_filter_many(lcf_plan* plan, const void* d_iq, int npk, float* d_out_pd, cudaStream_t stream);

/* Synchronise and return the device time of each stage summed over the
 * calls recorded since profiling was enabled: ms[LCF_NSTAGES] (host),
 * *n_calls = number of calls summed.  Either pointer may be NULL. */
lcf_status lcf_plan_profile_read(lcf_plan* plan, double* ms, int* n_calls);

/* EVD phase timing of the most recent filter call made while profiling was
 * on: cycles[8] (host) receives the SM clock cycles of each phase averaged
 * over the windows, in order: subspace iteration, QR of the block,
 * double-float congruence, fp32 conversion and Q, Jacobi sweeps, sort and
 * phase fix, thresholding rule, projection weights.  Synchronises the
 * plan's last stream.  LCF_EINVAL if profiling was never enabled. */
lcf_status lcf_plan_evd_phases(lcf_plan* plan, double* cycles);

/* ---- launch tuning (no counterpart in the paper) ----
 * How a plan spreads its work over the GPU: pixel splits of the Gram stages
 * (more splits = more CTAs and more partial sums to add) and the cluster size
 * of the distributed EVD.  The values change the order of some FP32 partial
 * sums, not the method; every value is within the library's tolerances. */
typedef struct {
  int gram_splits;       /* pixel ranges per window of the one-tile tensor-core Gram */
  int simt_gram_splits;  /* pixel splits per window of the CUDA-core residual Gram  */
  int aug_splits;        /* pixel splits of the CUDA-core coefficient columns (U, Q) */
  int q_splits;          /* pixel splits of the exact coefficient block (depth <= 4) */
  int basis_splits;      /* pixel splits of the global Gram behind the deflation basis */
  int ncc_splits;        /* pixel splits of method 4's band sums                      */
  int evd_cluster;       /* CTAs per window of the distributed EVD (Nt > 128): 4
                            (Nt <= 224) or 8 (Nt >= 200)                            */
} lcf_tuning;

/* The plan's current tuning (host struct).  No synchronisation. */
lcf_status lcf_plan_get_tuning(const lcf_plan* plan, lcf_tuning* t);

/* Apply a tuning: splits in 1..64, evd_cluster 4 or 8 as above.  Synchronous (waits for
 * the plan's work, reallocates the partial-sum buffers, drops captured graphs);
 * LCF_EINVAL for values out of range, LCF_ENOMEM. */
lcf_status lcf_plan_set_tuning(lcf_plan* plan, const lcf_tuning* t);

/* Autotune the plan's launch shapes on one packet (d_iq on the plan's device,
 * read only): each tunable in turn takes the candidate with the shortest packet
 * time (CUDA events on `stream`, best of three after a warm-up), the others held.
 * cache_path (may be NULL): a text file of earlier results, one line per
 * (GPU name, packet and window sizes, paths, precisions, deflation depth, rule
 * family); a line for this plan's key is applied without timing and
 * *from_cache (may be NULL) set to 1, else the result is appended.  Synchronous;
 * allocates (it is a setup call, like lcf_plan_create). */
lcf_status lcf_plan_autotune(lcf_plan* plan, const void* d_iq, cudaStream_t stream, const char* cache_path,
                             int* from_cache);

/* Windowed Gram matrices of one packet without any allocation.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (real-time threads that must not wait on the allocator, hosts
 * that own all device memory, fixed-budget embedded pipelines).
 *
 * Computes R_k = C_w^H C_w for every window of cfg on the CURRENT device with
 * the plain path's Gram kernels (FP32 products, double-float promotion),
 * deflating the packet with a fixed orthonormal DCT-II slow-time basis
 * instead of a plan's data-derived one; the deflation identity is exact for
 * any basis, so R_k agrees with a plan's Gram (and the FP64 oracle) within the
 * library's Gram tolerance (relative Frobenius error 1e-6), not bit for bit.
 * cfg's path, rule and precision fields are ignored.  d_iq: device
 * iq[nt][nz][nx] complex64 (8-byte aligned); d_R: device output [Nd][Nt][Nt]
 * complex double (16-byte aligned), fully written.  Asynchronous on `stream`;
 * calls no allocator of any kind.
 *
 * Scratch: one file-scope static device array of
 * lcf_gram_noalloc_scratch_bytes() bytes (64 MiB) that every GPU loading
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and caches it
 * (safe from several host threads); make that first call before any stream
 * capture.  Calls share the array: calls that overlap on the GPU race.
 * Returns LCF_ESCRATCH when the window tables, the centred packet and one
 * partial Gram per window do not fit (e.g. 256 x 128 x 100 with 8 x 8
 * windows fits; 512 x 256 x 100 does not), LCF_EINVAL for bad arguments,
 * LCF_EUNSUPPORTED for nt > 320 or nz*nx*(nt+4) > 2^31. */
lcf_status lcf_gram_noalloc(const lcf_config* cfg, const void* d_iq, void* d_R, cudaStream_t stream);

/* Size in bytes of lcf_gram_noalloc's static per-device scratch. */
size_t lcf_gram_noalloc_scratch_bytes(void);

/* ---- learned cutoff rule (no counterpart in the paper) ----
 * A multilayer perceptron maps a window's normalised log-eigenvalue spectrum
 * y_i = (log10 l_i - log10 l_Nt) / (log10 l_1 - log10 l_Nt)  (l_i = max(lambda_i,
 * lambda_1 Nt 2^-52), the curve of method 1, Eq. 6) and the window centre
 * ((iz + 1/2)/Wz, (ix + 1/2)/Wx) -- Nt + 2 inputs -- through 3 hidden ReLU
 * layers of H units to Nt logits over the cutoff k = 0 .. Nt-1.  Parameters
 * are one flat FP32 vector: W1 (H x (Nt+2)), b1 (H), W2 (H x H), b2, W3 (H x H),
 * b3, W4 (Nt x H), b4 (Nt), matrices row-major.  Training (FP32) runs on the
 * device with AdamW; inference runs inside the EVD kernel with bf16 weights
 * and FP32 accumulation. */

/* Create a network for packets of nt frames with hidden width H (<= 256) and
 * training batches of up to max_batch samples, on `device`.  Parameters and
 * optimiser moments start at zero.  Synchronous. */
lcf_status lcf_mlp_create(int nt, int hidden, int max_batch, int device, lcf_mlp** out);
/* Number of FP32 parameters (length of the flat vector). */
size_t lcf_mlp_param_count(const lcf_mlp* mlp);
/* Copy the flat parameter vector in from / out to host memory (synchronous).
 * Setting parameters resets the AdamW moments and step count. */
lcf_status lcf_mlp_set_params(lcf_mlp* mlp, const float* h_params);
lcf_status lcf_mlp_get_params(const lcf_mlp* mlp, float* h_params);
/* Gradients of the last lcf_mlp_loss_grad call, flat layout, to host (synchronous). */
lcf_status lcf_mlp_get_grads(const lcf_mlp* mlp, float* h_grads);
/* Logits for a batch: d_x [batch][Nt+2] f32 (device), d_logits [batch][Nt]
 * f32 (device, written).  Asynchronous on `stream`. */
lcf_status lcf_mlp_forward(lcf_mlp* mlp, const float* d_x, int batch, float* d_logits, cudaStream_t stream);
/* Mean softmax cross-entropy of the batch against cutoffs d_k [batch] (int,
 * device, in [0, Nt); a label outside gives a NaN loss and no gradient), and
 * its gradient with respect to every parameter (kept on the device).  If
 * h_loss is not NULL the call synchronises `stream` and writes the loss. */
lcf_status lcf_mlp_loss_grad(lcf_mlp* mlp, const float* d_x, const int* d_k, int batch, float* h_loss,
                             cudaStream_t stream);
/* One AdamW step with the current gradients: bias-corrected moments, decoupled
 * weight decay wd on the weight matrices only.  Asynchronous. */
lcf_status lcf_mlp_adamw(lcf_mlp* mlp, float lr, float beta1, float beta2, float eps, float wd,
                         cudaStream_t stream);
lcf_status lcf_mlp_destroy(lcf_mlp* mlp);

/* Give a plan the learned rule: the network's current parameters are copied
 * (bf16 weights, FP32 biases) into plan-owned device memory; later changes to
 * `mlp` do not affect the plan until this is called again.  p_min: windows whose
 * largest class probability is below it use rule k_src instead (flagged
 * LCF_WFLAG_FALLBACK); 0 <= p_min <= 2, above 1 every window falls back.  A
 * learned plan normally runs with a small max_sweeps, so its status may read
 * LCF_ENOCONV by design.  Requires mlp's Nt = the plan's Nt and the CTA-pair EVD.
 * Synchronous. */
lcf_status lcf_plan_set_mlp(lcf_plan* plan, const lcf_mlp* mlp, float p_min);

/* The learned rule's network input and output of every window of the last
 * LCF_T_LEARNED filter call (for validation; synchronises): features [Nd][Nt+2]
 * (the normalised log-spectrum computed in the EVD kernel, then the window
 * centre) and logits [Nd][Nt], host, either may be NULL.  LCF_EINVAL if no
 * network was set. */
lcf_status lcf_debug_learned(lcf_plan* plan, float* features, float* logits);

/* Self-test of the device-side failure path (no counterpart in the paper):
 * one CTA waits on an mbarrier phase that nothing completes, with the bounded
 * wait every kernel of the library uses, for at most limit_ns (<= 2 s); the
 * kernel records the timeout and returns, the context stays usable.  Returns
 * LCF_ETIMEOUT when the wait ran out (the expected outcome), writes the time
 * waited (seconds, host) to *waited_s if not NULL.  Synchronous. */
lcf_status lcf_selftest_wait_timeout(int device, unsigned long long limit_ns, double* waited_s);

/* Number of kernels the plan has launched since it was created (every
 * filter call adds the launches of its stages; debug dumps add theirs).
 * *n (host) receives the count.  No synchronisation. */
lcf_status lcf_plan_launch_count(const lcf_plan* plan, long long* n);

/* Bytes of device workspace the plan holds. */
size_t lcf_plan_workspace_bytes(const lcf_plan* plan);

lcf_status lcf_plan_destroy(lcf_plan* plan);

const char* lcf_status_string(lcf_status s);

#ifdef __cplusplus
}
#endif
#endif /* LCF_H_ */
