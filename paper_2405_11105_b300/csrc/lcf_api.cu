// lcf_api.cu — the C ABI (include/lcf.h): plan creation with the window
// geometry, workspace management and the per-packet launch sequence.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "lcf_internal.cuh"

using namespace lcf;

#define LCF_CUDA(x)                          \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return LCF_ECUDA; \
  } while (0)

extern "C" const char* lcf_status_string(lcf_status s) {
  switch (s) {
    case LCF_OK: return "ok";
    case LCF_EINVAL: return "invalid argument or configuration";
    case LCF_ENOMEM: return "out of memory";
    case LCF_ECUDA: return "CUDA error";
    case LCF_ENOCONV: return "Jacobi EVD hit its sweep cap in some window";
    case LCF_ETIMEOUT: return "bounded device wait gave up";
    case LCF_EDEGENERATE: return "some window had zero flow power";
    case LCF_EUNSUPPORTED: return "not supported by this build";
    case LCF_ESCRATCH: return "problem too large for the no-allocation entry point's static scratch";
  }
  return "unknown status";
}

extern "C" lcf_status lcf_config_default(lcf_config* c, int nz, int nx, int nt, int wz, int wx) {
  if (!c) return LCF_EINVAL;
  memset(c, 0, sizeof(*c));
  c->nz = nz; c->nx = nx; c->nt = nt; c->wz = wz; c->wx = wx;
  c->sigma_scale = 1.0f;
  c->support_sigmas = 3.0f;
  c->thresh_mode = LCF_T_CURVATURE;
  c->beta = 1.0f;
  c->k_fixed = 0;
  c->k_src = LCF_T_FIXED;
  c->beta_src = 1.0f;
  c->gram_path = LCF_PATH_TC;
  c->project_path = LCF_PATH_TC;
  c->max_sweeps = 40;
  c->evd_path = LCF_EVD_PAIR;
  return LCF_OK;
}

static lcf_status validate(const lcf_config* c) {
  if (!c) return LCF_EINVAL;
  if (c->nz <= 0 || c->nx <= 0 || c->nt < 2 || c->wz <= 0 || c->wx <= 0) return LCF_EINVAL;
  if (c->wz > c->nz || c->wx > c->nx) return LCF_EINVAL;
  if (!(c->sigma_scale > 0.f) || !isfinite(c->sigma_scale) || !isfinite(c->support_sigmas)) return LCF_EINVAL;
  if (c->thresh_mode < LCF_T_FIXED || c->thresh_mode > LCF_T_NCC) return LCF_EINVAL;
  if (c->thresh_mode == LCF_T_LEARNED && (c->k_src < LCF_T_FIXED || c->k_src > LCF_T_MEDIAN)) return LCF_EINVAL;
  if (c->thresh_mode == LCF_T_LEARNED && (c->evd_path != LCF_EVD_PAIR || c->nt > kEvdPairNmax))
    return LCF_EUNSUPPORTED;
  if (c->thresh_mode == LCF_T_SIGMOID && !((c->k_src >= LCF_T_FIXED && c->k_src <= LCF_T_MEDIAN) || c->k_src == LCF_T_NCC))
    return LCF_EINVAL;
  if (c->thresh_mode == LCF_T_LEARNED && c->evd_precision != LCF_EP_FP32) return LCF_EUNSUPPORTED;
  if (!isfinite(c->beta) || !isfinite(c->beta_src)) return LCF_EINVAL;
  if (c->pd_mode < 0 || c->pd_mode > 1 || c->alpha_mode < 0 || c->alpha_mode > 2) return LCF_EINVAL;
  if (c->curv_norm < 0 || c->curv_norm > 1) return LCF_EINVAL;
  if (c->gram_path < LCF_PATH_SIMT || c->gram_path > LCF_PATH_TC) return LCF_EINVAL;
  if (c->project_path < LCF_PATH_SIMT || c->project_path > LCF_PATH_TC) return LCF_EINVAL;
  if (c->evd_path < LCF_EVD_CTA || c->evd_path > LCF_EVD_OS) return LCF_EINVAL;
  if (c->gram_precision < LCF_GP_F16X3 || c->gram_precision > LCF_GP_E4M3) return LCF_EINVAL;
  if (c->gram_path != LCF_PATH_TC && c->gram_precision != LCF_GP_F16X3) return LCF_EINVAL;
  if (c->evd_precision < LCF_EP_FP32 || c->evd_precision > LCF_EP_FP64_POLISH) return LCF_EINVAL;
  if (c->graph < 0 || c->graph > 1) return LCF_EINVAL;
  if (c->project_form < LCF_PF_IDENTITY || c->project_form > LCF_PF_SUBTRACT) return LCF_EINVAL;
  if (c->project_form == LCF_PF_SUBTRACT && (c->thresh_mode == LCF_T_SIGMOID || c->thresh_mode == LCF_T_ADAPTIVE_SOFT))
    return LCF_EINVAL;   // the subtractive form needs 0/1 weights
  if (c->deflate < 0 || c->deflate > kDeflateMax || (c->deflate > 0 && c->deflate >= c->nt)) return LCF_EINVAL;
  if (c->inflight < 0 || c->inflight > 4) return LCF_EINVAL;
  if ((long long)c->nz * c->nx * (c->nt + kDeflateMax) > (1LL << 31)) return LCF_EUNSUPPORTED;
  if (c->nt > kEvdNmax) return LCF_EUNSUPPORTED;
  if (c->evd_path == LCF_EVD_CTA && c->nt > kEvdCtaNmax) return LCF_EUNSUPPORTED;
  return LCF_OK;
}

// Window geometry (Eq. 11): centres at the midpoints of a wz x wx grid of
// cells, SD = sigma_scale * cell size, support |delta| <= support_sigmas*SD.
static void build_geometry(const lcf_config& c, std::vector<Box>& boxes, std::vector<float>& gz,
                           std::vector<float>& gx) {
  const int nd = c.wz * c.wx;
  boxes.resize(nd);
  gz.assign((size_t)nd * c.nz, 0.f);
  gx.assign((size_t)nd * c.nx, 0.f);
  const double dz = (double)c.nz / c.wz, dx = (double)c.nx / c.wx;
  for (int k = 0; k < nd; ++k) {
    const int iz = k / c.wx, ix = k % c.wx;
    Box b{0, c.nz, 0, c.nx};
    if (c.all_ones_window) {
      for (int z = 0; z < c.nz; ++z) gz[(size_t)k * c.nz + z] = 1.f;
      for (int x = 0; x < c.nx; ++x) gx[(size_t)k * c.nx + x] = 1.f;
      boxes[k] = b;
      continue;
    }
    const double cz = (iz + 0.5) * dz - 0.5, cx = (ix + 0.5) * dx - 0.5;
    const double sz = c.sigma_scale * dz, sx = c.sigma_scale * dx;
    if (c.support_sigmas > 0.f) {
      const double hz = c.support_sigmas * sz, hx = c.support_sigmas * sx;
      b.z0 = (int)fmax(0.0, ceil(cz - hz));
      b.z1 = (int)fmin((double)c.nz, floor(cz + hz) + 1.0);
      b.x0 = (int)fmax(0.0, ceil(cx - hx));
      b.x1 = (int)fmin((double)c.nx, floor(cx + hx) + 1.0);
      if (b.z1 <= b.z0 || b.x1 <= b.x0) b = Box{0, 0, 0, 0};
    }
    for (int z = b.z0; z < b.z1; ++z) {
      double u = (z - cz) / sz;
      gz[(size_t)k * c.nz + z] = (float)exp(-0.5 * u * u);
    }
    for (int x = b.x0; x < b.x1; ++x) {
      double u = (x - cx) / sx;
      gx[(size_t)k * c.nx + x] = (float)exp(-0.5 * u * u);
    }
    boxes[k] = b;
  }
}

template <typename T>
static cudaError_t dalloc(T** p, size_t count, size_t* total) {
  *total += count * sizeof(T);
  return cudaMalloc((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
}

static void free_ws(Workspace& w) {
  void* ptrs[] = {w.gz, w.gx, w.box, w.phi, w.gglob, w.xa, w.gpart, w.gaug, w.xmax, w.gtc, w.gq, w.err, w.R, w.lam, w.V, w.wt, w.kcut, w.alpha,
                  w.flags, w.W, w.pw, w.ncol, w.tile_off, w.tile_win, w.bimg, w.bscale, w.evd_clk, w.mlp_w, w.mlp_b, w.mlp_dbg, w.evd_B, w.evd_vh, w.evd_t,
                  w.evd_scale, w.evd_perm, w.evd_rank, w.iq_stage, w.pd_stage, w.phi_alt, w.xmax_alt, w.gglob_async, w.post_rq,
                  w.post_pv, w.post_isig, w.post_band, w.sub_qhi, w.sub_qlo, w.sub_off, w.sub_pdk,
                  w.sub_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w = Workspace();
}

static bool g_configured[64] = {false};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

extern "C" lcf_status lcf_plan_create(const lcf_config* cfg, int device, lcf_plan** out) {
  if (!out) return LCF_EINVAL;
  *out = nullptr;
  lcf_status v = validate(cfg);
  if (v != LCF_OK) return v;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LCF_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return LCF_ECUDA;
  lcf_plan* P = new (std::nothrow) lcf_plan();
  if (!P) { cudaSetDevice(prev); return LCF_ENOMEM; }
  P->cfg = *cfg;
  P->device = device;
  P->nd = cfg->wz * cfg->wx;
  P->nt = cfg->nt;
  P->ndefl = deflate_depth(cfg->nt, cfg->deflate);
  P->n1 = cfg->nt + P->ndefl;
  P->npix = cfg->nz * cfg->nx;
  P->gram_tiles = (P->nt + 63) / 64;
  cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, device);
  {
    int pairs = P->gram_tiles * (P->gram_tiles + 1) / 2;
    int want = (4 * P->sm_count + pairs * P->nd - 1) / (pairs * P->nd);
    P->gram_nsplit = want < 1 ? 1 : (want > 64 ? 64 : want);
    int wa = (4 * P->sm_count + P->nd - 1) / P->nd;   // about four pixel ranges per SM
    P->aug_nsplit = wa < 1 ? 1 : (wa > 64 ? 64 : wa);
    P->q_nsplit = P->aug_nsplit;
    int gt = (P->nt + 63) / 64;
    int gb = (P->sm_count + gt * (gt + 1) / 2 - 1) / (gt * (gt + 1) / 2);
    P->basis_nsplit = gb < 1 ? 1 : (gb > 64 ? 64 : gb);
  }
  {
    long pmax = 0;
    std::vector<Box> bx;
    std::vector<float> tz, tx;
    build_geometry(*cfg, bx, tz, tx);
    for (const Box& b : bx) pmax = std::max(pmax, (long)(b.z1 - b.z0) * (b.x1 - b.x0));
    long ts = (pmax + 2047) / 2048;   // ~2048 pixels per tensor-core CTA
    P->tc_nsplit = (int)(ts < 1 ? 1 : (ts > 64 ? 64 : ts));
  }
  // one tensor-core tile holds the augmented rows when they fit and the exact-product kernel
  // takes the coefficient block; otherwise the residual rows alone, U and Q from CUDA cores.
  // Long packets (Nt > 128) tile the augmented rows when the exact kernel takes Q (d <= 4), so
  // the tile pairs give U too (with more deflated vectors, the residual rows alone).  At
  // 125 <= Nt <= 128 the one-tile kernel with pixel splits plus the CUDA-core columns is faster
  // (384x256x128, 16x16 windows: Gram 2.8 ms against 7.0 ms for tile pairs over the 132 rows).
  P->tc_na = (P->n1 <= kTcGramNaMax && P->ndefl <= kQExactMax) ? P->n1 : P->nt;
  if (P->nt > kTcGramNaMax && P->ndefl <= kQExactMax) P->tc_na = P->n1;
  if (P->tc_na > kTcGramNaMax) {   // long packets: tile pairs of at most kTcTileMax rows, no pixel splits
    P->tc_T = (P->tc_na + kTcTileMax - 1) / kTcTileMax;
    P->tc_tb = ((P->tc_na + P->tc_T - 1) / P->tc_T + 7) / 8 * 8;
    P->tc_nsplit = 1;
  } else {
    P->tc_T = 1;
    P->tc_tb = P->tc_na;
  }
  P->ncp = P->nt <= kProjectShortNmax ? 4 * project_cpt(P->nt) : (P->nt + 15) / 16 * 16;
  P->evd_cluster = evd_dist_cluster(P->nt);
  std::vector<float> gz, gx;
  build_geometry(*cfg, P->boxes, gz, gx);

  Workspace& w = P->ws;
  size_t tot = 0;
  const size_t nd = P->nd, nt = P->nt, n1 = P->n1, npix = P->npix;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&w.gz, nd * cfg->nz, &tot);
  if (e == cudaSuccess) e = dalloc(&w.gx, nd * cfg->nx, &tot);
  if (e == cudaSuccess) e = dalloc(&w.box, nd, &tot);
  if (e == cudaSuccess) e = dalloc(&w.phi, (size_t)P->ndefl * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.phi_alt, (size_t)P->ndefl * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.gglob, (size_t)P->basis_nsplit * nt * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.gglob_async, (size_t)P->basis_nsplit * nt * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.xa, n1 * npix, &tot);
  if (e == cudaSuccess) e = dalloc(&w.gpart, nd * P->gram_nsplit * nt * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.gaug, nd * P->aug_nsplit * n1 * P->ndefl, &tot);
  if (e == cudaSuccess) e = dalloc(&w.xmax, 1, &tot);
  if (e == cudaSuccess) e = dalloc(&w.xmax_alt, 1, &tot);
  if (e == cudaSuccess) e = dalloc(&w.err, 1, &tot);
  if (cfg->gram_path == LCF_PATH_TC) {
    if (e == cudaSuccess)
      e = dalloc(&w.gtc, P->tc_T > 1 ? nd * P->tc_T * P->tc_T * 2 * P->tc_tb * P->tc_tb
                                      : nd * std::max(P->tc_nsplit, 2) * 2 * P->tc_na * P->tc_na, &tot);
    if (e == cudaSuccess) e = dalloc(&w.gq, nd * P->q_nsplit * kQExactMax * kQExactMax, &tot);
    if (e == cudaSuccess) e = gram_tc_make_map(P);
  }
  if (e == cudaSuccess) e = dalloc(&w.R, nd * nt * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.lam, nd * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.V, nd * nt * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.wt, nd * nt, &tot);
  if (e == cudaSuccess) e = dalloc(&w.kcut, nd, &tot);
  if (e == cudaSuccess) e = dalloc(&w.alpha, nd, &tot);
  if (e == cudaSuccess) e = dalloc(&w.flags, nd, &tot);
  if (e == cudaSuccess) e = dalloc(&w.W, nd * nt * P->ncp, &tot);
  if (e == cudaSuccess && nt > (size_t)kProjectShortNmax)
    e = dalloc(&w.pw, nd * kDeflateMax * P->ncp, &tot);
  if (e == cudaSuccess) e = dalloc(&w.ncol, nd, &tot);
  if ((cfg->evd_path == LCF_EVD_PAIR && P->nt > kEvdPairNmax) || cfg->evd_path == LCF_EVD_OS) {
    const size_t m = P->nt < kEvdHead ? P->nt : kEvdHead;
    if (e == cudaSuccess) e = dalloc(&w.evd_B, nd * nt * nt, &tot);
    if (e == cudaSuccess) e = dalloc(&w.evd_vh, nd * m * nt, &tot);
    if (e == cudaSuccess) e = dalloc(&w.evd_t, nd * m * m, &tot);
    if (e == cudaSuccess) e = dalloc(&w.evd_scale, nd, &tot);
    if (e == cudaSuccess && cfg->evd_path == LCF_EVD_OS && P->nt > kEvdPairNmax && P->nt <= kEvdOscNmax) {
      e = dalloc(&w.evd_perm, nd * nt, &tot);
      if (e == cudaSuccess) e = dalloc(&w.evd_rank, nd, &tot);
    }
  }
  if (e == cudaSuccess && cfg->evd_precision == LCF_EP_FP64_POLISH)
    e = dalloc(&w.post_rq, nd * post_rq_blocks(P->nt) * nt, &tot);
  if (post_uses_ncc(*cfg)) {
    const int ns = (3 * P->sm_count + P->nd - 1) / P->nd;   // about three CTAs per SM in all
    P->ncc_nsplit = ns < 1 ? 1 : (ns > 64 ? 64 : ns);
    if (e == cudaSuccess) e = dalloc(&w.post_pv, nd * kDeflateMax * nt, &tot);
    if (e == cudaSuccess) e = dalloc(&w.post_isig, nd * nt, &tot);
    if (e == cudaSuccess) e = dalloc(&w.post_band, post_band_count(P), &tot);
  }
  if (cfg->project_form == LCF_PF_SUBTRACT) {
    std::vector<long long> off(nd);
    long long tot_px = 0;
    for (size_t k = 0; k < nd; ++k) {
      off[k] = tot_px;
      tot_px += (long long)(P->boxes[k].z1 - P->boxes[k].z0) * (P->boxes[k].x1 - P->boxes[k].x0);
    }
    const int ns = (2 * P->sm_count + P->nd - 1) / P->nd;   // about two CTAs per SM in all
    P->sub_nsplit = ns < 1 ? 1 : (ns > 64 ? 64 : ns);
    if (e == cudaSuccess) e = dalloc(&w.sub_qhi, nd * nt * nt, &tot);
    if (e == cudaSuccess) e = dalloc(&w.sub_qlo, nd * nt * nt, &tot);
    if (e == cudaSuccess) e = dalloc(&w.sub_off, nd, &tot);
    if (e == cudaSuccess) e = dalloc(&w.sub_pdk, (size_t)tot_px, &tot);
    if (e == cudaSuccess) e = dalloc(&w.sub_part, nd * P->sub_nsplit, &tot);
    if (e == cudaSuccess) e = cudaMemcpy(w.sub_off, off.data(), nd * sizeof(long long), cudaMemcpyHostToDevice);
  }
  std::vector<int> toff, twin;
  if (cfg->project_path == LCF_PATH_TC) {
    project_tc_tiles(P, &P->ptiles_z, &P->ptiles_x, toff, twin);
    if (e == cudaSuccess) e = dalloc(&w.tile_off, toff.size(), &tot);
    if (e == cudaSuccess) e = dalloc(&w.tile_win, twin.size(), &tot);
    if (e == cudaSuccess) e = dalloc(&w.bimg, nd * project_tc_image_bytes(P->nt, P->ndefl), &tot);
    if (e == cudaSuccess) e = dalloc(&w.bscale, nd, &tot);
  }
  if (e == cudaSuccess) e = dalloc(&w.iq_stage, 2 * nt * npix, &tot);
  if (e == cudaSuccess) e = dalloc(&w.pd_stage, 2 * npix, &tot);
  if (e != cudaSuccess) {
    free_ws(w);
    delete P;
    cudaSetDevice(prev);
    return e == cudaErrorMemoryAllocation ? LCF_ENOMEM : LCF_ECUDA;
  }
  P->ws_bytes = tot;
  e = cudaMemcpy(w.gz, gz.data(), gz.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w.gx, gx.data(), gx.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w.box, P->boxes.data(), nd * sizeof(Box), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(w.flags, 0, nd * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w.err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w.xmax, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(w.xmax_alt, 0, sizeof(unsigned));
  if (e == cudaSuccess && cfg->project_path == LCF_PATH_TC) {
    e = cudaMemcpy(w.tile_off, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !twin.empty())
      e = cudaMemcpy(w.tile_win, twin.data(), twin.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && (device >= 64 || !g_configured[device])) {
    e = evd_configure();
    if (e == cudaSuccess) e = project_configure();
    if (e == cudaSuccess) e = gram_tc_configure();
    if (e == cudaSuccess) e = basis_configure();
    if (e == cudaSuccess) e = project_tc_configure();
    if (e == cudaSuccess) e = evd_pair_configure();
    if (e == cudaSuccess) e = evd_dist_configure();
    if (e == cudaSuccess) e = evd_os_configure();
    if (e == cudaSuccess) e = evd_osc_configure();
    if (e == cudaSuccess) e = gram_simt_configure();
    if (e == cudaSuccess) e = post_configure();
    if (e == cudaSuccess && device < 64) g_configured[device] = true;
  }
  if (e != cudaSuccess) {
    free_ws(w);
    delete P;
    cudaSetDevice(prev);
    return LCF_ECUDA;
  }
  cudaSetDevice(prev);
  *out = P;
  if (cfg->inflight > 1) {   // lanes 1 .. inflight-1: sub-plans with their own workspaces
    lcf_status ls = LCF_OK;
    lcf_config c1 = *cfg;
    c1.inflight = 1;
    P->lanes.assign(cfg->inflight, nullptr);
    for (int l = 1; l < cfg->inflight && ls == LCF_OK; ++l) ls = lcf_plan_create(&c1, device, &P->lanes[l]);
    if (ls == LCF_OK) {
      DeviceGuard dg(device);
      P->lane_st.assign(cfg->inflight, nullptr);
      P->lane_ev.assign(cfg->inflight, nullptr);
      cudaError_t le = cudaEventCreateWithFlags(&P->ev_many, cudaEventDisableTiming);
      for (int l = 0; l < cfg->inflight && le == cudaSuccess; ++l) {
        le = cudaStreamCreateWithFlags(&P->lane_st[l], cudaStreamNonBlocking);
        if (le == cudaSuccess) le = cudaEventCreateWithFlags(&P->lane_ev[l], cudaEventDisableTiming);
      }
      if (le != cudaSuccess) ls = LCF_ECUDA;
    }
    if (ls != LCF_OK) {
      lcf_plan_destroy(P);
      *out = nullptr;
      return ls;
    }
  }
  return LCF_OK;
}


// Event for stage boundary b (0..LCF_NSTAGES) of the current call, or null.
static cudaEvent_t prof_event(lcf_plan* P, int b) {
  if (!P->profiling) return nullptr;
  size_t slot = (size_t)(P->prof_calls % kProfCalls) * (LCF_NSTAGES + 1) + b;
  return P->prof_ev[slot];
}

#define LCF_MARK(b)                                              \
  do {                                                           \
    cudaEvent_t ev_ = prof_event(P, (b));                        \
    if (ev_) LCF_CUDA(cudaEventRecord(ev_, st));                 \
  } while (0)

// with_basis false: the packet's basis (phi, xmax) was prepared on another stream already
static lcf_status run_packet(lcf_plan* P, const float2* iq, float* out, cudaStream_t st, bool with_basis = true) {
  const lcf_config& c = P->cfg;
  const bool tc = c.gram_path == LCF_PATH_TC;
  if (c.thresh_mode == LCF_T_LEARNED && P->mlp_hidden == 0) return LCF_EINVAL;   // no network set
  LCF_MARK(LCF_STAGE_PREP);
  if (with_basis) LCF_CUDA(launch_basis(P, iq, st));
  LCF_CUDA(launch_center(P, iq, st));
  LCF_MARK(LCF_STAGE_GRAM);
  if (tc) {
    LCF_CUDA(launch_gram_tc(P, st));
  } else {
    LCF_CUDA(launch_gram_aug(P, st));
    LCF_CUDA(launch_gram_simt(P, st));
  }
  LCF_MARK(LCF_STAGE_ASSEMBLE);
  if (tc) LCF_CUDA(launch_gram_assemble_tc(P, st));
  else LCF_CUDA(launch_gram_assemble(P, st));
  LCF_MARK(LCF_STAGE_EVD);
  if (c.evd_path == LCF_EVD_OS && P->nt > kEvdPairNmax && P->nt <= kEvdOscNmax) LCF_CUDA(launch_evd_osc(P, st));
  else if (c.evd_path != LCF_EVD_CTA && P->nt > kEvdPairNmax) LCF_CUDA(launch_evd_dist(P, st));
  else if (c.evd_path == LCF_EVD_PAIR) LCF_CUDA(launch_evd_pair(P, st));
  else if (c.evd_path == LCF_EVD_OS) LCF_CUDA(launch_evd_os(P, st));
  else LCF_CUDA(launch_evd(P, st));
  LCF_CUDA(launch_post(P, st));   // FP64-class polish, method 4 (no launch otherwise)
  LCF_MARK(LCF_STAGE_PROJECT);
  if (c.project_form == LCF_PF_SUBTRACT) LCF_CUDA(launch_project_subtract(P, iq, out, st));
  else if (c.project_path == LCF_PATH_TC) LCF_CUDA(launch_project_tc(P, out, st));
  else LCF_CUDA(launch_project_simt(P, iq, out, st));
  LCF_MARK(LCF_NSTAGES);
  if (P->profiling) ++P->prof_calls;
  return LCF_OK;
}

lcf_status lcf::packet_once(lcf_plan* P, const float2* iq, float* out, cudaStream_t st) {
  return run_packet(P, iq, out, st);
}

extern "C" lcf_status lcf_plan_profile(lcf_plan* P, int enable) {
  if (!P) return LCF_EINVAL;
  DeviceGuard g(P->device);
  if (enable && P->prof_ev.empty()) {
    P->prof_ev.resize((size_t)kProfCalls * (LCF_NSTAGES + 1));
    for (auto& e : P->prof_ev) LCF_CUDA(cudaEventCreate(&e));
  }
  if (enable && !P->ws.evd_clk) {
    LCF_CUDA(cudaMalloc((void**)&P->ws.evd_clk, (size_t)P->nd * (kEvdPhases + 1) * sizeof(long long)));
    LCF_CUDA(cudaMemset(P->ws.evd_clk, 0, (size_t)P->nd * (kEvdPhases + 1) * sizeof(long long)));
  }
  P->profiling = enable != 0;
  P->prof_calls = 0;
  return LCF_OK;
}

extern "C" lcf_status lcf_plan_profile_read(lcf_plan* P, double* ms, int* n_calls) {
  if (!P) return LCF_EINVAL;
  DeviceGuard g(P->device);
  double acc[LCF_NSTAGES] = {0};
  long n = P->prof_calls < kProfCalls ? P->prof_calls : kProfCalls;
  if (n > 0) LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  for (long i = P->prof_calls - n; i < P->prof_calls; ++i) {
    size_t base = (size_t)(i % kProfCalls) * (LCF_NSTAGES + 1);
    for (int s = 0; s < LCF_NSTAGES; ++s) {
      float t = 0.f;
      LCF_CUDA(cudaEventElapsedTime(&t, P->prof_ev[base + s], P->prof_ev[base + s + 1]));
      acc[s] += t;
    }
  }
  if (ms) memcpy(ms, acc, sizeof(acc));
  if (n_calls) *n_calls = (int)n;
  return LCF_OK;
}

extern "C" lcf_status lcf_plan_evd_phases(lcf_plan* P, double* cycles) {
  if (!P || !cycles) return LCF_EINVAL;
  if (!P->ws.evd_clk) return LCF_EINVAL;
  DeviceGuard g(P->device);
  LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  std::vector<long long> c((size_t)P->nd * (kEvdPhases + 1));
  LCF_CUDA(cudaMemcpy(c.data(), P->ws.evd_clk, c.size() * sizeof(long long), cudaMemcpyDeviceToHost));
  for (int j = 0; j < kEvdPhases; ++j) {
    double acc = 0.0;
    int cnt = 0;
    for (int k = 0; k < P->nd; ++k) {
      const long long a = c[(size_t)k * (kEvdPhases + 1) + j], b = c[(size_t)k * (kEvdPhases + 1) + j + 1];
      if (a != 0 && b >= a) { acc += (double)(b - a); ++cnt; }
    }
    cycles[j] = cnt ? acc / cnt : 0.0;
  }
  return LCF_OK;
}

// A filter call other than the pipelined one: the next pipelined packet's basis prep (on its own
// stream) must not overwrite the basis buffers this call reads, so it waits for this event once.
static lcf_status note_seq(lcf_plan* P, cudaStream_t stream) {
  if (!P->ev_seq) LCF_CUDA(cudaEventCreateWithFlags(&P->ev_seq, cudaEventDisableTiming));
  LCF_CUDA(cudaEventRecord(P->ev_seq, stream));
  P->seq_since_async = true;
  return LCF_OK;
}

// The pipelined basis prep (lcf_filter_host_async, and lcf_filter when cfg.inputs_ready):
// packet q's basis and maximum live in buffer pair q mod 2, written on the plan's prep stream
// once the packet two back (same pair) is done with them and any other filter call since the
// last prep has finished; `after` orders the prep after the packet's own input.
static lcf_status pipe_streams(lcf_plan* P) {
  if (P->prep_stream) return LCF_OK;
  LCF_CUDA(cudaStreamCreateWithFlags(&P->prep_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b) {
    LCF_CUDA(cudaEventCreateWithFlags(&P->ev_prep[b], cudaEventDisableTiming));
    LCF_CUDA(cudaEventCreateWithFlags(&P->ev_pdone[b], cudaEventDisableTiming));
  }
  return LCF_OK;
}
static lcf_status pipe_packet(lcf_plan* P, const float2* iq, float* out, cudaStream_t stream, cudaEvent_t after) {
  lcf_status s = pipe_streams(P);
  if (s != LCF_OK) return s;
  const int p = (int)(P->pipe_seq & 1);
  if (P->basis_par != p) {
    std::swap(P->ws.phi, P->ws.phi_alt);
    std::swap(P->ws.xmax, P->ws.xmax_alt);
    P->basis_par = p;
  }
  if (after) LCF_CUDA(cudaStreamWaitEvent(P->prep_stream, after, 0));
  if (P->pipe_seq >= 2) LCF_CUDA(cudaStreamWaitEvent(P->prep_stream, P->ev_pdone[p], 0));
  if (P->seq_since_async) {   // another filter call since the last prep may still read phi
    LCF_CUDA(cudaStreamWaitEvent(P->prep_stream, P->ev_seq, 0));
    P->seq_since_async = false;
  }
  // its own global-Gram scratch: a synchronous call on `stream` may be running its basis
  std::swap(P->ws.gglob, P->ws.gglob_async);
  const cudaError_t eb = launch_basis(P, iq, P->prep_stream);
  std::swap(P->ws.gglob, P->ws.gglob_async);
  LCF_CUDA(eb);
  LCF_CUDA(cudaEventRecord(P->ev_prep[p], P->prep_stream));
  LCF_CUDA(cudaStreamWaitEvent(stream, P->ev_prep[p], 0));
  s = run_packet(P, iq, out, stream, false);
  if (s != LCF_OK) return s;
  LCF_CUDA(cudaEventRecord(P->ev_pdone[p], stream));
  ++P->pipe_seq;
  return LCF_OK;
}

// Drop the captured single-packet graphs (their buffer pointers may be stale after a
// setup call that reallocates plan memory).
void lcf::plan_drop_graphs(lcf_plan* P) {
  for (auto& e : P->pg) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    e = lcf_plan::PacketGraph();
  }
}

// One packet as one CUDA graph launch: the stage launches of run_packet captured once per
// (input, output) pair on the plan's capture stream and replayed on `stream`.
static lcf_status graph_packet(lcf_plan* P, const float2* iq, float* out, cudaStream_t stream) {
  int slot = -1, oldest = 0;
  for (int i = 0; i < lcf_plan::kPacketGraphs; ++i) {
    if (P->pg[i].exec && P->pg[i].iq == iq && P->pg[i].out == out) { slot = i; break; }
    if (P->pg[i].used < P->pg[oldest].used) oldest = i;
  }
  if (slot < 0) {
    slot = oldest;
    lcf_plan::PacketGraph& e = P->pg[slot];
    if (e.exec) {
      cudaGraphExecDestroy(e.exec);
      e.exec = nullptr;
    }
    if (!P->cap_stream) LCF_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
    const long long l0 = P->launches;
    LCF_CUDA(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
    lcf_status s = run_packet(P, iq, out, P->cap_stream);
    cudaGraph_t gr = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &gr);
    e.launches = P->launches - l0;
    P->launches = l0;
    if (s != LCF_OK || ce != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return s != LCF_OK ? s : LCF_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) {
      e.exec = nullptr;
      return LCF_ECUDA;
    }
    e.iq = iq;
    e.out = out;
  }
  lcf_plan::PacketGraph& e = P->pg[slot];
  e.used = ++P->pg_clock;
  LCF_CUDA(cudaGraphLaunch(e.exec, stream));
  P->launches += e.launches;
  return LCF_OK;
}

extern "C" lcf_status lcf_filter(lcf_plan* P, const void* d_iq, float* d_out_pd, cudaStream_t stream) {
  if (!P || !d_iq || !d_out_pd) return LCF_EINVAL;
  if (((uintptr_t)d_iq & 7) || ((uintptr_t)d_out_pd & 3)) return LCF_EINVAL;
  DeviceGuard g(P->device);
  const bool pipe = P->cfg.inputs_ready && !P->profiling && !P->cfg.graph;
  const bool graph = P->cfg.graph && !P->profiling;
  lcf_status s = pipe ? pipe_packet(P, (const float2*)d_iq, d_out_pd, stream, nullptr)
                      : graph ? graph_packet(P, (const float2*)d_iq, d_out_pd, stream)
                              : run_packet(P, (const float2*)d_iq, d_out_pd, stream);
  P->last_stream = stream;
  P->launched = true;
  P->last_iq = (void*)d_iq;
  if (s == LCF_OK && !pipe) s = note_seq(P, stream);
  return s;
}

extern "C" lcf_status lcf_filter_many(lcf_plan* P, const void* d_iq, int npk, float* d_out_pd, cudaStream_t stream) {
  if (!P || npk < 0 || (npk > 0 && (!d_iq || !d_out_pd))) return LCF_EINVAL;
  if (((uintptr_t)d_iq & 7) || ((uintptr_t)d_out_pd & 3)) return LCF_EINVAL;
  const size_t in_elems = (size_t)P->nt * P->npix, out_elems = (size_t)P->npix;
  const float2* iq = (const float2*)d_iq;
  const int K = (int)P->lanes.size() > 1 ? (int)P->lanes.size() : 1;
  if (K == 1 || npk <= 1) {
    for (int p = 0; p < npk; ++p) {
      const lcf_status s = lcf_filter(P, iq + p * in_elems, d_out_pd + p * out_elems, stream);
      if (s != LCF_OK) return s;
    }
    return LCF_OK;
  }
  DeviceGuard g(P->device);
  const int nl = npk < K ? npk : K;
  LCF_CUDA(cudaEventRecord(P->ev_many, stream));
  for (int l = 0; l < nl; ++l) LCF_CUDA(cudaStreamWaitEvent(P->lane_st[l], P->ev_many, 0));
  for (int p = 0; p < npk; ++p) {
    const int l = p % K;
    const lcf_status s = lcf_filter(l ? P->lanes[l] : P, iq + p * in_elems, d_out_pd + p * out_elems, P->lane_st[l]);
    if (s != LCF_OK) return s;
  }
  for (int l = 0; l < nl; ++l) {
    LCF_CUDA(cudaEventRecord(P->lane_ev[l], P->lane_st[l]));
    LCF_CUDA(cudaStreamWaitEvent(stream, P->lane_ev[l], 0));
  }
  P->last_stream = stream;
  P->launched = true;
  return LCF_OK;
}

extern "C" lcf_status lcf_filter_host(lcf_plan* P, const void* h_iq, float* h_out_pd, cudaStream_t stream) {
  if (!P || !h_iq || !h_out_pd) return LCF_EINVAL;
  DeviceGuard g(P->device);
  const size_t in_bytes = (size_t)P->nt * P->npix * sizeof(float2);
  LCF_CUDA(cudaMemcpyAsync(P->ws.iq_stage, h_iq, in_bytes, cudaMemcpyHostToDevice, stream));
  lcf_status s = run_packet(P, P->ws.iq_stage, P->ws.pd_stage, stream);
  if (s != LCF_OK) return s;
  s = note_seq(P, stream);
  if (s != LCF_OK) return s;
  LCF_CUDA(cudaMemcpyAsync(h_out_pd, P->ws.pd_stage, (size_t)P->npix * sizeof(float), cudaMemcpyDeviceToHost,
                           stream));
  P->last_stream = stream;
  P->launched = true;
  P->last_iq = P->ws.iq_stage;
  LCF_CUDA(cudaStreamSynchronize(stream));
  return LCF_OK;
}

static lcf_status host_async_one(lcf_plan* P, const void* h_iq, float* h_out_pd, cudaStream_t stream);

extern "C" lcf_status lcf_filter_host_async(lcf_plan* P, const void* h_iq, float* h_out_pd, cudaStream_t stream) {
  if (!P || !h_iq || !h_out_pd) return LCF_EINVAL;
  if (P->lanes.size() > 1) {   // consecutive calls rotate over the lanes
    DeviceGuard g(P->device);
    const int l = (int)(P->lane_seq++ % (long long)P->lanes.size());
    LCF_CUDA(cudaEventRecord(P->ev_many, stream));
    LCF_CUDA(cudaStreamWaitEvent(P->lane_st[l], P->ev_many, 0));
    return host_async_one(l ? P->lanes[l] : P, h_iq, h_out_pd, P->lane_st[l]);
  }
  return host_async_one(P, h_iq, h_out_pd, stream);
}

static lcf_status host_async_one(lcf_plan* P, const void* h_iq, float* h_out_pd, cudaStream_t stream) {
  DeviceGuard g(P->device);
  if (!P->h2d_stream) {
    LCF_CUDA(cudaStreamCreateWithFlags(&P->h2d_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      LCF_CUDA(cudaEventCreateWithFlags(&P->ev_in[b], cudaEventDisableTiming));
      LCF_CUDA(cudaEventCreateWithFlags(&P->ev_done[b], cudaEventDisableTiming));
    }
  }
  const int b = (int)(P->host_seq & 1);
  const size_t in_elems = (size_t)P->nt * P->npix;
  float2* iq = P->ws.iq_stage + (size_t)b * in_elems;
  float* pd = P->ws.pd_stage + (size_t)b * P->npix;
  // the buffer's previous packet has finished with it before the copy overwrites it
  if (P->host_seq >= 2) LCF_CUDA(cudaStreamWaitEvent(P->h2d_stream, P->ev_done[b], 0));
  LCF_CUDA(cudaMemcpyAsync(iq, h_iq, in_elems * sizeof(float2), cudaMemcpyHostToDevice, P->h2d_stream));
  LCF_CUDA(cudaEventRecord(P->ev_in[b], P->h2d_stream));
  lcf_status s;
  if (P->profiling) {   // stage events want every stage on `stream`
    LCF_CUDA(cudaStreamWaitEvent(stream, P->ev_in[b], 0));
    s = run_packet(P, iq, pd, stream);
    if (s == LCF_OK) s = note_seq(P, stream);
  } else {   // basis prep on the prep stream once the input is in, overlapping the previous packet
    s = pipe_packet(P, iq, pd, stream, P->ev_in[b]);
  }
  if (s != LCF_OK) return s;
  LCF_CUDA(cudaMemcpyAsync(h_out_pd, pd, (size_t)P->npix * sizeof(float), cudaMemcpyDeviceToHost, stream));
  LCF_CUDA(cudaEventRecord(P->ev_done[b], stream));
  P->host_seq++;
  P->last_stream = stream;
  P->launched = true;
  P->last_iq = iq;
  return LCF_OK;
}

extern "C" lcf_status lcf_plan_sync(lcf_plan* P) {
  if (!P) return LCF_EINVAL;
  for (size_t l = 1; l < P->lanes.size(); ++l) {
    const lcf_status s = lcf_plan_sync(P->lanes[l]);
    if (s != LCF_OK) return s;
  }
  DeviceGuard g(P->device);
  for (cudaStream_t ls : P->lane_st) LCF_CUDA(cudaStreamSynchronize(ls));
  if (P->h2d_stream) LCF_CUDA(cudaStreamSynchronize(P->h2d_stream));
  if (P->prep_stream) LCF_CUDA(cudaStreamSynchronize(P->prep_stream));
  // the last pipelined packet of each staging buffer, whichever stream it ran on; earlier
  // packets of a buffer finished before its next input copy began
  for (int b = 0; b < 2; ++b)
    if (P->host_seq > b) LCF_CUDA(cudaEventSynchronize(P->ev_done[b]));
  if (P->launched) LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  return LCF_OK;
}

extern "C" lcf_status lcf_filter_stream(lcf_plan* P, const void* d_frames, int n_frames, int stride,
                                        float* d_out_pd, cudaStream_t stream) {
  if (!P || !d_frames || !d_out_pd || stride <= 0 || n_frames < P->nt) return LCF_EINVAL;
  if (((uintptr_t)d_frames & 7) || ((uintptr_t)d_out_pd & 3)) return LCF_EINVAL;
  DeviceGuard g(P->device);
  const int npk = (n_frames - P->nt) / stride + 1;
  const float2* fr = (const float2*)d_frames;
  auto stream_packet = [&](int i, cudaStream_t s_) {
    return run_packet(P, fr + (size_t)i * stride * P->npix, d_out_pd + (size_t)i * P->npix, s_);
  };
  if (P->profiling) {   // stage events need the packets launched one by one
    for (int i = 0; i < npk; ++i) {
      lcf_status s = stream_packet(i, stream);
      if (s != LCF_OK) return s;
    }
  } else {
    // every packet of the stream in one CUDA graph, captured on the plan's own stream the first
    // time these buffers are seen and replayed on `stream` afterwards
    const bool hit = P->sg_exec && P->sg_frames == d_frames && P->sg_out == d_out_pd && P->sg_n == n_frames &&
                     P->sg_stride == stride;
    if (!hit) {
      if (P->sg_exec) {
        cudaGraphExecDestroy(P->sg_exec);
        P->sg_exec = nullptr;
      }
      if (!P->cap_stream) LCF_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
      const long long l0 = P->launches;
      LCF_CUDA(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
      lcf_status s = LCF_OK;
      for (int i = 0; i < npk && s == LCF_OK; ++i) s = stream_packet(i, P->cap_stream);
      cudaGraph_t gr = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &gr);
      P->sg_launches = P->launches - l0;
      P->launches = l0;
      if (s != LCF_OK || ce != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return s != LCF_OK ? s : LCF_ECUDA;
      }
      const cudaError_t ie = cudaGraphInstantiate(&P->sg_exec, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) {
        P->sg_exec = nullptr;
        return LCF_ECUDA;
      }
      P->sg_frames = d_frames;
      P->sg_out = d_out_pd;
      P->sg_n = n_frames;
      P->sg_stride = stride;
    }
    LCF_CUDA(cudaGraphLaunch(P->sg_exec, stream));
    P->launches += P->sg_launches;
  }
  P->last_stream = stream;
  P->launched = true;
  P->last_iq = (void*)(fr + (size_t)(npk - 1) * stride * P->npix);
  return note_seq(P, stream);
}

extern "C" lcf_status lcf_plan_status(lcf_plan* P, int* per_window_flags) {
  if (!P) return LCF_EINVAL;
  DeviceGuard g(P->device);
  LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  std::vector<int> f(P->nd);
  LCF_CUDA(cudaMemcpy(f.data(), P->ws.flags, P->nd * sizeof(int), cudaMemcpyDeviceToHost));
  if (per_window_flags) memcpy(per_window_flags, f.data(), P->nd * sizeof(int));
  int any = 0;
  for (int v : f) any |= v;
  int derr = 0;
  LCF_CUDA(cudaMemcpy(&derr, P->ws.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr) return LCF_ETIMEOUT;
  if (any & LCF_WFLAG_NOCONV) return LCF_ENOCONV;
  if (any & LCF_WFLAG_DEGENERATE) return LCF_EDEGENERATE;
  return LCF_OK;
}

extern "C" lcf_status lcf_debug_dump(lcf_plan* P, double* eig, float* wt, int* k, float* alpha) {
  if (!P) return LCF_EINVAL;
  DeviceGuard g(P->device);
  LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  const size_t nd = P->nd, nt = P->nt;
  if (eig) LCF_CUDA(cudaMemcpy(eig, P->ws.lam, nd * nt * sizeof(double), cudaMemcpyDeviceToHost));
  if (wt) LCF_CUDA(cudaMemcpy(wt, P->ws.wt, nd * nt * sizeof(float), cudaMemcpyDeviceToHost));
  if (k) LCF_CUDA(cudaMemcpy(k, P->ws.kcut, nd * sizeof(int), cudaMemcpyDeviceToHost));
  if (alpha) LCF_CUDA(cudaMemcpy(alpha, P->ws.alpha, nd * sizeof(float), cudaMemcpyDeviceToHost));
  return LCF_OK;
}

extern "C" lcf_status lcf_debug_gram(lcf_plan* P, double* R) {
  if (!P || !R) return LCF_EINVAL;
  DeviceGuard g(P->device);
  LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  LCF_CUDA(cudaMemcpy(R, P->ws.R, (size_t)P->nd * P->nt * P->nt * sizeof(double2), cudaMemcpyDeviceToHost));
  return LCF_OK;
}

extern "C" lcf_status lcf_debug_eigvecs(lcf_plan* P, float* V) {
  if (!P || !V) return LCF_EINVAL;
  DeviceGuard g(P->device);
  LCF_CUDA(cudaStreamSynchronize(P->last_stream));
  LCF_CUDA(cudaMemcpy(V, P->ws.V, (size_t)P->nd * P->nt * P->nt * sizeof(float2), cudaMemcpyDeviceToHost));
  return LCF_OK;
}

extern "C" lcf_status lcf_debug_filtered_iq(lcf_plan* P, const void* d_iq, int subset, void* d_filt,
                                            cudaStream_t stream) {
  if (!P || !d_iq || !d_filt || subset < 0 || subset >= P->nd) return LCF_EINVAL;
  DeviceGuard g(P->device);
  LCF_CUDA(launch_filtered_iq(P, (const float2*)d_iq, subset, (float2*)d_filt, stream));
  return LCF_OK;
}

extern "C" lcf_status lcf_plan_windows(lcf_plan* P, int* nd, int k, int* box) {
  if (!P) return LCF_EINVAL;
  if (nd) *nd = P->nd;
  if (box) {
    if (k < 0 || k >= P->nd) return LCF_EINVAL;
    const Box& b = P->boxes[k];
    box[0] = b.z0; box[1] = b.z1; box[2] = b.x0; box[3] = b.x1;
  }
  return LCF_OK;
}

extern "C" lcf_status lcf_plan_launch_count(const lcf_plan* P, long long* n) {
  if (!P || !n) return LCF_EINVAL;
  *n = P->launches;
  for (size_t l = 1; l < P->lanes.size(); ++l) {
    long long m = 0;
    lcf_plan_launch_count(P->lanes[l], &m);
    *n += m;
  }
  return LCF_OK;
}

extern "C" size_t lcf_plan_workspace_bytes(const lcf_plan* P) {
  if (!P) return 0;
  size_t b = P->ws_bytes;
  for (size_t l = 1; l < P->lanes.size(); ++l) b += lcf_plan_workspace_bytes(P->lanes[l]);
  return b;
}

extern "C" lcf_status lcf_plan_destroy(lcf_plan* P) {
  if (!P) return LCF_EINVAL;
  for (size_t l = 1; l < P->lanes.size(); ++l)
    if (P->lanes[l]) lcf_plan_destroy(P->lanes[l]);
  DeviceGuard g(P->device);
  for (cudaStream_t ls : P->lane_st)
    if (ls) cudaStreamSynchronize(ls);
  if (P->h2d_stream) cudaStreamSynchronize(P->h2d_stream);   // pipelined host calls still in flight
  if (P->prep_stream) cudaStreamSynchronize(P->prep_stream);
  if (P->launched) cudaStreamSynchronize(P->last_stream);
  free_ws(P->ws);
  for (auto& e : P->prof_ev) cudaEventDestroy(e);
  if (P->sg_exec) cudaGraphExecDestroy(P->sg_exec);
  for (auto& e : P->pg)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  if (P->h2d_stream) cudaStreamDestroy(P->h2d_stream);
  if (P->prep_stream) cudaStreamDestroy(P->prep_stream);
  for (int b = 0; b < 2; ++b) {
    if (P->ev_in[b]) cudaEventDestroy(P->ev_in[b]);
    if (P->ev_done[b]) cudaEventDestroy(P->ev_done[b]);
    if (P->ev_prep[b]) cudaEventDestroy(P->ev_prep[b]);
    if (P->ev_pdone[b]) cudaEventDestroy(P->ev_pdone[b]);
  }
  if (P->ev_seq) cudaEventDestroy(P->ev_seq);
  // the lane streams last: last_stream may be one of them
  for (cudaStream_t ls : P->lane_st)
    if (ls) cudaStreamDestroy(ls);
  for (cudaEvent_t le : P->lane_ev)
    if (le) cudaEventDestroy(le);
  if (P->ev_many) cudaEventDestroy(P->ev_many);
  delete P;
  return LCF_OK;
}
