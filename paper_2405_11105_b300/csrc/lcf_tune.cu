// lcf_tune.cu — launch tuning of a plan (include/lcf.h: lcf_plan_get_tuning,
// lcf_plan_set_tuning, lcf_plan_autotune).
//
// The tunables decide how each stage's work is spread over the 148 SMs: the
// pixel splits of the Gram stages (each split is one more CTA per window and one
// more partial sum for the reduction to add) and the cluster size of the
// distributed EVD.  The autotuner times whole packets (CUDA events on the
// caller's stream) and takes the tunables one at a time, the rest held, in the
// order of the stages; results are cached in a text file keyed by the GPU's name
// and everything that shapes the launches.
#include <stdio.h>
#include <string.h>

#include <string>

#include "lcf_internal.cuh"

using namespace lcf;

namespace {

bool uses_tc_one_tile(const lcf_plan* P) { return P->cfg.gram_path == LCF_PATH_TC && P->tc_T == 1; }
bool uses_aug(const lcf_plan* P) { return P->cfg.gram_path == LCF_PATH_SIMT || P->tc_na == P->nt; }
bool uses_q(const lcf_plan* P) { return P->cfg.gram_path == LCF_PATH_TC && P->ndefl <= kQExactMax; }
bool uses_dist(const lcf_plan* P) {
  return P->cfg.evd_path != LCF_EVD_CTA && P->nt > kEvdPairNmax && !(P->cfg.evd_path == LCF_EVD_OS && P->nt <= kEvdOscNmax);
}

// the split-dependent buffers, in the sizes their current splits need (elements)
struct SplitSizes {
  size_t gglob, gpart, gaug, gtc, gq, band;
};
SplitSizes split_sizes(const lcf_plan* P) {
  const size_t nd = P->nd, nt = P->nt;
  SplitSizes z{};
  z.gglob = (size_t)P->basis_nsplit * nt * nt;
  z.gpart = nd * P->gram_nsplit * nt * nt;
  z.gaug = nd * P->aug_nsplit * (size_t)P->n1 * P->ndefl;
  if (P->cfg.gram_path == LCF_PATH_TC) {
    z.gtc = P->tc_T > 1 ? nd * P->tc_T * P->tc_T * 2 * (size_t)P->tc_tb * P->tc_tb
                        : nd * (size_t)(P->tc_nsplit > 2 ? P->tc_nsplit : 2) * 2 * P->tc_na * P->tc_na;
    z.gq = nd * P->q_nsplit * kQExactMax * kQExactMax;
  }
  if (post_uses_ncc(P->cfg)) z.band = post_band_count(P);
  return z;
}

template <typename T>
cudaError_t regrow(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  return cudaMalloc((void**)p, (count > 0 ? count : 1) * sizeof(T));
}

bool in_range(int v) { return v >= 1 && v <= 64; }

std::string tune_key(const lcf_plan* P) {
  cudaDeviceProp prop;
  char name[256] = "gpu";
  if (cudaGetDeviceProperties(&prop, P->device) == cudaSuccess) snprintf(name, sizeof(name), "%s", prop.name);
  for (char* c = name; *c; ++c)
    if (*c == ' ' || *c == '|') *c = '_';
  const lcf_config& c = P->cfg;
  char key[512];
  snprintf(key, sizeof(key), "%s|%d|%d|%d|%d|%d|g%d|p%d|e%d|gp%d|ep%d|d%d|ncc%d", name, c.nz, c.nx, c.nt, c.wz, c.wx,
           c.gram_path, c.project_path, c.evd_path, c.gram_precision, c.evd_precision, P->ndefl,
           post_uses_ncc(c) ? 1 : 0);
  return key;
}

// packet time (ms): one warm-up, then the best of three
lcf_status time_packet(lcf_plan* P, const float2* iq, float* out, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                       float* ms) {
  float best = 1e30f;
  for (int r = 0; r < 4; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return LCF_ECUDA;
    lcf_status s = packet_once(P, iq, out, st);
    if (s != LCF_OK) return s;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return LCF_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return LCF_ECUDA;
    if (r > 0 && t < best) best = t;
  }
  *ms = best;
  return LCF_OK;
}

}  // namespace

extern "C" lcf_status lcf_plan_get_tuning(const lcf_plan* P, lcf_tuning* t) {
  if (!P || !t) return LCF_EINVAL;
  t->gram_splits = P->tc_nsplit;
  t->simt_gram_splits = P->gram_nsplit;
  t->aug_splits = P->aug_nsplit;
  t->q_splits = P->q_nsplit;
  t->basis_splits = P->basis_nsplit;
  t->ncc_splits = P->ncc_nsplit;
  t->evd_cluster = P->evd_cluster;
  return LCF_OK;
}

static lcf_status set_tuning_one(lcf_plan* P, const lcf_tuning* t) {
  if (!P || !t) return LCF_EINVAL;
  if (!in_range(t->gram_splits) || !in_range(t->simt_gram_splits) || !in_range(t->aug_splits) ||
      !in_range(t->q_splits) || !in_range(t->basis_splits) || !in_range(t->ncc_splits))
    return LCF_EINVAL;
  // clusters of 8 for the shorter long packets: checked against the oracle from Nt = 200 up; at
  // Nt = 129 they gave NaN eigenvalues, so 8 is refused below 200
  if (!(t->evd_cluster == 4 && P->nt <= 224) && !(t->evd_cluster == 8 && P->nt >= 200)) return LCF_EINVAL;
  if (P->tc_T > 1 && t->gram_splits != 1) return LCF_EINVAL;   // tile pairs take whole windows
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(P->device) != cudaSuccess) return LCF_ECUDA;
  lcf_status st = LCF_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) st = LCF_ECUDA;
  const SplitSizes old = split_sizes(P);
  if (st == LCF_OK) {
    P->tc_nsplit = t->gram_splits;
    P->gram_nsplit = t->simt_gram_splits;
    P->aug_nsplit = t->aug_splits;
    P->q_nsplit = t->q_splits;
    P->basis_nsplit = t->basis_splits;
    P->ncc_nsplit = t->ncc_splits;
    P->evd_cluster = t->evd_cluster;
    const SplitSizes z = split_sizes(P);
    cudaError_t e = cudaSuccess;
    Workspace& w = P->ws;
    if (e == cudaSuccess && z.gglob != old.gglob) e = regrow(&w.gglob, z.gglob);
    if (e == cudaSuccess && z.gglob != old.gglob) e = regrow(&w.gglob_async, z.gglob);
    if (e == cudaSuccess && z.gpart != old.gpart) e = regrow(&w.gpart, z.gpart);
    if (e == cudaSuccess && z.gaug != old.gaug) e = regrow(&w.gaug, z.gaug);
    if (e == cudaSuccess && z.gtc != old.gtc) e = regrow(&w.gtc, z.gtc);
    if (e == cudaSuccess && z.gq != old.gq) e = regrow(&w.gq, z.gq);
    if (e == cudaSuccess && z.band != old.band) e = regrow(&w.post_band, z.band);
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? LCF_ENOMEM : LCF_ECUDA;
    P->ws_bytes += (2 * (z.gglob - old.gglob)) * sizeof(float2) + (z.gpart - old.gpart + z.gaug - old.gaug +
                                                                  z.gq - old.gq) * sizeof(double2) +
                   (z.gtc - old.gtc + z.band - old.band) * sizeof(double);
    plan_drop_graphs(P);
    if (P->sg_exec) {   // the captured stream graph holds the old launch shapes
      cudaGraphExecDestroy(P->sg_exec);
      P->sg_exec = nullptr;
    }
  }
  cudaSetDevice(prev);
  return st;
}

// the plan and its in-flight lanes take the same launch shapes
extern "C" lcf_status lcf_plan_set_tuning(lcf_plan* P, const lcf_tuning* t) {
  lcf_status st = set_tuning_one(P, t);
  for (size_t l = 1; st == LCF_OK && P && l < P->lanes.size(); ++l) st = set_tuning_one(P->lanes[l], t);
  return st;
}

extern "C" lcf_status lcf_plan_autotune(lcf_plan* P, const void* d_iq, cudaStream_t stream, const char* cache_path,
                                        int* from_cache) {
  if (!P || !d_iq || ((uintptr_t)d_iq & 7)) return LCF_EINVAL;
  if (from_cache) *from_cache = 0;
  if (P->cfg.thresh_mode == LCF_T_LEARNED && P->mlp_hidden == 0) return LCF_EINVAL;
  const std::string key = tune_key(P);
  lcf_tuning cur;
  lcf_plan_get_tuning(P, &cur);
  if (cache_path) {   // the last line for this key wins
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[1024];
      bool hit = false;
      lcf_tuning got = cur;
      while (fgets(line, sizeof(line), f)) {
        char k[600];
        lcf_tuning t;
        if (sscanf(line, "%599s %d %d %d %d %d %d %d", k, &t.gram_splits, &t.simt_gram_splits, &t.aug_splits,
                   &t.q_splits, &t.basis_splits, &t.ncc_splits, &t.evd_cluster) == 8 &&
            key == k) {
          got = t;
          hit = true;
        }
      }
      fclose(f);
      if (hit) {
        lcf_status s = lcf_plan_set_tuning(P, &got);   // a cached result: the lanes too
        if (s == LCF_OK && from_cache) *from_cache = 1;
        return s;
      }
    }
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(P->device) != cudaSuccess) return LCF_ECUDA;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lcf_status st = LCF_OK;
  if (cudaMalloc((void**)&out, (size_t)P->npix * sizeof(float)) != cudaSuccess) st = LCF_ENOMEM;
  if (st == LCF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = LCF_ECUDA;
  const bool prof = P->profiling;
  P->profiling = false;
  struct Knob {
    int lcf_tuning::*field;
    bool active;
    std::vector<int> cand;
  };
  const std::vector<Knob> knobs = {
      {&lcf_tuning::basis_splits, true, {1, 2, 4, 8, 16}},
      {&lcf_tuning::gram_splits, uses_tc_one_tile(P), {1, 2, 3, 4, 5, 6, 8, 10, 12, 16}},
      {&lcf_tuning::simt_gram_splits, P->cfg.gram_path == LCF_PATH_SIMT, {1, 2, 3, 4, 6, 8, 12, 16}},
      {&lcf_tuning::aug_splits, uses_aug(P), {1, 2, 4, 6, 8, 12, 16, 24, 32}},
      {&lcf_tuning::q_splits, uses_q(P), {1, 2, 4, 6, 8, 12, 16, 24, 32}},
      {&lcf_tuning::ncc_splits, post_uses_ncc(P->cfg), {1, 2, 3, 4, 6, 8, 12}},
      {&lcf_tuning::evd_cluster, uses_dist(P) && P->nt >= 200 && P->nt <= 224, {4, 8}},
  };
  for (const Knob& kb : knobs) {
    if (st != LCF_OK) break;
    if (!kb.active) continue;
    int best_v = cur.*kb.field;
    float best_t = 1e30f;
    for (int v : kb.cand) {
      lcf_tuning t = cur;
      t.*kb.field = v;
      if (set_tuning_one(P, &t) != LCF_OK) continue;   // candidates on the plan alone
      float ms = 0.f;
      st = time_packet(P, (const float2*)d_iq, out, stream, e0, e1, &ms);
      if (st != LCF_OK) break;
      if (ms < best_t) {
        best_t = ms;
        best_v = v;
      }
    }
    cur.*kb.field = best_v;
  }
  if (st == LCF_OK) st = lcf_plan_set_tuning(P, &cur);   // the result on every lane
  P->profiling = prof;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaSetDevice(prev);
  if (st == LCF_OK && cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "%s %d %d %d %d %d %d %d\n", key.c_str(), cur.gram_splits, cur.simt_gram_splits, cur.aug_splits,
              cur.q_splits, cur.basis_splits, cur.ncc_splits, cur.evd_cluster);
      fclose(f);
    }
  }
  P->last_stream = stream;
  P->launched = true;
  return st;
}
