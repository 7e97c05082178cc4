// fs1_capi.cu -- host runtime of the FS-1 library: the C ABI of include/fs1.h.
//
// Responsibilities: argument validation (a device-side mass check per pair),
// the choice of team size (CTAs per pair) and number of teams, the handle's
// device workspace (descriptors, results, team exchange slots, barrier
// counters), staging of host-located problems, launches on the handle's
// stream, and the per-problem status / info reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fs1.h"
#include "fs1_internal.h"

using namespace fs1;

struct fs1_handle {
  fs1_config cfg;
  void* stage = nullptr;       // device staging for host-located problems
  size_t stage_bytes = 0;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;          // device workspace
  size_t ws_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

constexpr const char* kVersion = "fs1-gb300 0.1";
std::atomic<long long> g_launches{0};

fs1_status cuda_fail(cudaError_t e, const char* what) {
  fprintf(stderr, "fs1: %s: %s\n", what, cudaGetErrorString(e));
  return FS1_ECUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

fs1_status ensure_ws(fs1_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return FS1_OK;
  if (h->cfg.hbm_budget && bytes > h->cfg.hbm_budget) return FS1_ENOMEM;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  size_t want = std::max(bytes, (size_t)1 << 20);
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return FS1_ENOMEM;
  }
  h->ws_bytes = want;
  return FS1_OK;
}

// ---- validation: per pair, sums of a and b, any negative / non-finite ----
struct ValOut {
  double sa, sb;
  int bad;
  int pad;
};

__global__ void validate_kernel(const PairDesc* pairs, int in_f32, ValOut* out) {
  const PairDesc P = pairs[blockIdx.x];
  double sa = 0.0, sb = 0.0;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < P.n; i += blockDim.x) {
    double va = in_f32 ? (double)((const float*)P.a)[i] : ((const double*)P.a)[i];
    double vb = in_f32 ? (double)((const float*)P.b)[i] : ((const double*)P.b)[i];
    if (!(va >= 0.0) || !(vb >= 0.0) || !isfinite(va) || !isfinite(vb)) bad = 1;
    sa += va;
    sb += vb;
  }
  __shared__ double ssa[32], ssb[32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  __syncthreads();
  if (bad) atomicOr(&sbad, 1);
  if ((threadIdx.x & 31) == 0) {
    ssa[threadIdx.x >> 5] = sa;
    ssb[threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += ssa[w];
      tb += ssb[w];
    }
    out[blockIdx.x] = ValOut{ta, tb, sbad, 0};
  }
}

int kind_of(const fs1_config& c) {
  if (c.variant == FS1_VARIANT_PLAIN) return c.precision == FS1_FP64 ? KK_PLAIN_F64 : KK_PLAIN_F32;
  return KK_LOG_F32;
}

fs1_status check_problem(const fs1_problem& p) {
  if (p.ndim != 1 && p.ndim != 2) return FS1_EINVAL;
  if (p.dtype != FS1_FP64 && p.dtype != FS1_FP32) return FS1_EINVAL;
  if (p.location != FS1_MEM_DEVICE && p.location != FS1_MEM_HOST) return FS1_EINVAL;
  if (p.n[0] < 1 || (p.ndim == 2 && p.n[1] < 1)) return FS1_EINVAL;
  if (!(p.h[0] > 0.0) || !std::isfinite(p.h[0])) return FS1_EINVAL;
  if (p.ndim == 2 && (!(p.h[1] > 0.0) || !std::isfinite(p.h[1]))) return FS1_EINVAL;
  if (!(p.eps > 0.0) || !std::isfinite(p.eps)) return FS1_EINVAL;
  if (!(p.tol >= 0.0) || std::isnan(p.tol)) return FS1_EINVAL;
  if (p.itr_max < 0) return FS1_EINVAL;
  if (!p.a || !p.b) return FS1_EINVAL;
  if ((p.f_init == nullptr) != (p.g_init == nullptr)) return FS1_EINVAL;
  return FS1_OK;
}

int64_t npoints(const fs1_problem& p) { return p.n[0] * (p.ndim == 2 ? p.n[1] : 1); }

// team geometry for a group of problems of one kind
struct Geometry {
  int team_size;
  int num_teams;
};

fs1_status choose_geometry(fs1_handle* h, int kind, const std::vector<const fs1_problem*>& ps, Geometry* g) {
  const int thr = team_threads();
  const int maxc = max_coresident_ctas(kind);
  if (maxc <= 0) return FS1_ECUDA;
  int tmin = 1, tuse = 1;
  for (auto* p : ps) {
    const double c = p->h[0] / p->eps;
    const int64_t cap = elems_cap_for(kind, c);
    const int64_t n = npoints(*p);
    const int64_t t = (n + thr * cap - 1) / (thr * cap);
    const int64_t tu = (n + thr - 1) / thr;
    if (t > maxc) return FS1_EUNSUPPORTED;   // does not fit on chip
    tmin = std::max<int>(tmin, (int)t);
    tuse = std::max<int>(tuse, (int)std::min<int64_t>(tu, maxc));
  }
  int T;
  if (h->cfg.team_size > 0) {
    T = std::max(tmin, h->cfg.team_size);
    if (T > maxc) return FS1_EINVAL;
  } else {
    int teams = std::max(1, std::min((int)ps.size(), maxc / tmin));
    T = std::max(tmin, std::min(tuse, maxc / teams));
  }
  int teams = std::max(1, std::min((int)ps.size(), maxc / T));
  g->team_size = T;
  g->num_teams = teams;
  return FS1_OK;
}

// Heterogeneous team plan for a batch of 1D problems: problems are put in
// classes by the fewest CTAs that hold them on chip (rounded up to a power of
// two); CTAs are split over the classes in proportion to their estimated work
// (N * itr_max); every class is a queue of its problems in decreasing cost
// (longest-processing-time first) served by its teams.
struct Plan {
  std::vector<int> cta_team, cta_rank, team_T, team_slot, team_class, class_off, order, class_T;
  std::vector<int> prob_T;   // team size of each problem
  int num_teams = 0, grid = 0, max_T = 1, slots = 0;
};

fs1_status plan_teams(fs1_handle* h, int kind, const std::vector<const fs1_problem*>& ps, Plan* P) {
  const int thr = team_threads();
  const int maxc = max_coresident_ctas(kind);
  if (maxc <= 0) return FS1_ECUDA;
  const int n = (int)ps.size();
  std::vector<int> tmin(n);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    const double c = ps[i]->h[0] / ps[i]->eps;
    const int64_t cap = elems_cap_for(kind, c);
    const int64_t np = npoints(*ps[i]);
    const int64_t t = (np + thr * cap - 1) / (thr * cap);
    if (t > maxc) return FS1_EUNSUPPORTED;
    int p2 = 1;
    while (p2 < t) p2 <<= 1;
    tmin[i] = std::min<int>(p2, maxc);
    if (h->cfg.team_size > 0) {
      if (h->cfg.team_size > maxc) return FS1_EINVAL;
      tmin[i] = std::max<int>((int)t, h->cfg.team_size);
    }
    cost[i] = (double)np * (double)std::max<int64_t>(1, ps[i]->itr_max);
  }
  // classes by team size
  std::vector<int> keys(tmin);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int nc = (int)keys.size();
  std::vector<double> W(nc, 0.0);
  std::vector<int> cnt(nc, 0), cls(n);
  for (int i = 0; i < n; ++i) {
    cls[i] = (int)(std::lower_bound(keys.begin(), keys.end(), tmin[i]) - keys.begin());
    W[cls[i]] += cost[i];
    cnt[cls[i]] += 1;
  }
  double Wt = 0.0;
  for (double w : W) Wt += w;
  std::vector<int> T(keys), teams(nc, 1);
  int base = 0;
  for (int k = 0; k < nc; ++k) base += T[k];
  if (base > maxc) return FS1_EUNSUPPORTED;   // caller splits by class
  if (nc == 1) {
    teams[0] = std::max(1, std::min(cnt[0], maxc / T[0]));
    if (h->cfg.team_size <= 0) {
      int tuse = 1;
      for (int i = 0; i < n; ++i)
        tuse = std::max<int>(tuse, (int)std::min<int64_t>((npoints(*ps[i]) + thr - 1) / thr, maxc));
      T[0] = std::max(T[0], std::min(tuse, maxc / teams[0]));
    }
  } else {
    for (int k = 0; k < nc; ++k) {
      const int want = (int)std::floor(maxc * W[k] / Wt);
      teams[k] = std::max(1, std::min(cnt[k], want / T[k]));
    }
    auto used = [&]() {
      int u = 0;
      for (int k = 0; k < nc; ++k) u += teams[k] * T[k];
      return u;
    };
    while (used() > maxc) {
      int kk = -1;
      for (int k = 0; k < nc; ++k)
        if (teams[k] > 1 && (kk < 0 || teams[k] * T[k] > teams[kk] * T[kk])) kk = k;
      if (kk < 0) break;
      --teams[kk];
    }
    // leftover CTAs: more teams where the work per team is largest
    for (;;) {
      int kk = -1;
      double best = 0.0;
      for (int k = 0; k < nc; ++k)
        if (teams[k] < cnt[k] && used() + T[k] <= maxc && W[k] / teams[k] > best) {
          best = W[k] / teams[k];
          kk = k;
        }
      if (kk < 0) break;
      ++teams[kk];
    }
  }
  // queues in decreasing cost
  P->class_off.assign(nc + 1, 0);
  for (int k = 0; k < nc; ++k) P->class_off[k + 1] = P->class_off[k] + cnt[k];
  P->order.assign(n, 0);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    if (cls[x] != cls[y]) return cls[x] < cls[y];
    return cost[x] > cost[y];
  });
  for (int i = 0; i < n; ++i) P->order[i] = idx[i];
  // teams and CTAs
  P->cta_team.clear();
  P->cta_rank.clear();
  P->team_T.clear();
  P->team_slot.clear();
  P->team_class.clear();
  P->class_T = T;
  int slot = 0;
  for (int k = 0; k < nc; ++k)
    for (int t = 0; t < teams[k]; ++t) {
      const int team = (int)P->team_T.size();
      P->team_T.push_back(T[k]);
      P->team_slot.push_back(slot);
      P->team_class.push_back(k);
      slot += 2 * T[k];
      for (int r = 0; r < T[k]; ++r) {
        P->cta_team.push_back(team);
        P->cta_rank.push_back(r);
      }
      P->max_T = std::max(P->max_T, T[k]);
    }
  P->num_teams = (int)P->team_T.size();
  P->grid = (int)P->cta_team.size();
  P->slots = slot;
  P->prob_T.assign(n, 0);
  for (int i = 0; i < n; ++i) P->prob_T[i] = T[cls[i]];
  return FS1_OK;
}

// run one group (same kind, all 1D, device-located) in one launch
fs1_status run_group(fs1_handle* h, int kind, int mode, const std::vector<const fs1_problem*>& ps,
                     std::vector<PairResult>& res, Geometry& geo, float* ms, bool validate) {
  const int count = (int)ps.size();
  const bool two_d = ps[0]->ndim == 2;
  fs1_status st = FS1_OK;
  if (two_d) {
    if (kind != KK_LOG_F32) return FS1_EUNSUPPORTED;   // 2D runs the stabilised FP32 variant
    geo.team_size = 0;
    geo.num_teams = 0;
  } else if ((st = choose_geometry(h, kind, ps, &geo)) != FS1_OK) {
    return st;
  }
  Plan plan;
  const bool planned = !two_d && mode == 0;
  if (planned && (st = plan_teams(h, kind, ps, &plan)) != FS1_OK) return st;
  const int T = two_d ? 1 : (planned ? plan.max_T : geo.team_size);
  const int teams = two_d ? 1 : (planned ? plan.num_teams : geo.num_teams);
  const size_t nslots = planned ? (size_t)plan.slots : (size_t)teams * 2 * T;
  const int in_f32 = ps[0]->dtype == FS1_FP32;
  size_t off = 0;
  const size_t o_desc = off; off = align_up(off + sizeof(PairDesc) * count, 256);
  const size_t o_res = off;  off = align_up(off + sizeof(PairResult) * count, 256);
  const size_t o_val = off;  off = align_up(off + sizeof(ValOut) * count, 256);
  const size_t o_slot = off; off = align_up(off + sizeof(Slot) * nslots, 256);
  const size_t o_cslot = off; off = align_up(off + 128 * nslots, 256);
  const size_t o_ctr = off;  off = align_up(off + sizeof(unsigned long long) * teams, 256);
  const size_t o_abt = off;  off = align_up(off + sizeof(int) * teams, 256);
  // plan arrays: cta_team, cta_rank [grid]; team_T, team_slot, team_class
  // [teams]; class_off [nc + 1]; order [count]; class_next [nc]
  const int nclass = planned ? (int)plan.class_T.size() : 0;
  const int pgrid = planned ? plan.grid : 0;
  const size_t plan_ints = planned ? (size_t)2 * pgrid + 3 * teams + (nclass + 1) + count + nclass : 0;
  const size_t o_plan = off; off = align_up(off + sizeof(int) * plan_ints, 256);
  const size_t o_tick = off; off = align_up(off + sizeof(unsigned long long) * (planned ? teams : 0), 256);
  std::vector<PairDesc> desc(count);
  for (int i = 0; i < count; ++i) {
    const fs1_problem& p = *ps[i];
    PairDesc d{};
    d.a = p.a;
    d.b = p.b;
    d.n = npoints(p);
    d.n_fast = p.n[0];
    d.n_slow = p.ndim == 2 ? p.n[1] : 1;
    d.h_fast = p.h[0];
    d.h_slow = p.ndim == 2 ? p.h[1] : 0.0;
    d.eps = p.eps;
    d.tol = p.tol;
    d.itr_max = p.itr_max;
    d.f_out = p.f_out;
    d.g_out = p.g_out;
    d.f_init = p.f_init;
    d.g_init = p.g_init;
    desc[i] = d;
  }
  const size_t o_2d = off;
  if (two_d) off = align_up(off + solve2d_workspace(desc.data(), count), 256);
  if ((st = ensure_ws(h, off)) != FS1_OK) return st;
  char* ws = (char*)h->ws;

  std::vector<PairResult> init(count, PairResult{NAN, NAN, 0, FS1_ETIMEOUT, 0});
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ws + o_desc, desc.data(), sizeof(PairDesc) * count, cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess)
    return cuda_fail(e, "descriptor copy");
  if ((e = cudaMemcpyAsync(ws + o_res, init.data(), sizeof(PairResult) * count, cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess)
    return cuda_fail(e, "result init");
  cudaMemsetAsync(ws + o_slot, 0, sizeof(Slot) * nslots, h->stream);
  cudaMemsetAsync(ws + o_cslot, 0, 128 * nslots, h->stream);
  std::vector<int> pints;
  if (planned) {
    pints.reserve(plan_ints);
    pints.insert(pints.end(), plan.cta_team.begin(), plan.cta_team.end());
    pints.insert(pints.end(), plan.cta_rank.begin(), plan.cta_rank.end());
    pints.insert(pints.end(), plan.team_T.begin(), plan.team_T.end());
    pints.insert(pints.end(), plan.team_slot.begin(), plan.team_slot.end());
    pints.insert(pints.end(), plan.team_class.begin(), plan.team_class.end());
    pints.insert(pints.end(), plan.class_off.begin(), plan.class_off.end());
    pints.insert(pints.end(), plan.order.begin(), plan.order.end());
    pints.insert(pints.end(), (size_t)nclass, 0);   // class_next
    if ((e = cudaMemcpyAsync(ws + o_plan, pints.data(), sizeof(int) * pints.size(), cudaMemcpyHostToDevice,
                             h->stream)) != cudaSuccess)
      return cuda_fail(e, "plan copy");
    cudaMemsetAsync(ws + o_tick, 0, sizeof(unsigned long long) * teams, h->stream);
  }
  cudaMemsetAsync(ws + o_ctr, 0, sizeof(unsigned long long) * teams, h->stream);
  cudaMemsetAsync(ws + o_abt, 0, sizeof(int) * teams, h->stream);

  std::vector<int> bad(count, 0);
  if (validate) {
    validate_kernel<<<count, 256, 0, h->stream>>>((const PairDesc*)(ws + o_desc), in_f32,
                                                  (ValOut*)(ws + o_val));
    g_launches.fetch_add(1);
    std::vector<ValOut> vo(count);
    if ((e = cudaMemcpyAsync(vo.data(), ws + o_val, sizeof(ValOut) * count, cudaMemcpyDeviceToHost,
                             h->stream)) != cudaSuccess)
      return cuda_fail(e, "validation copy");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "validation");
    bool anybad = false;
    for (int i = 0; i < count; ++i) {
      const double sa = vo[i].sa, sb = vo[i].sb;
      if (vo[i].bad || !(sa > 0.0) || !(sb > 0.0) || std::fabs(sa - sb) > 1e-6 * std::max(sa, sb)) {
        bad[i] = 1;
        anybad = true;
      }
    }
    if (anybad) {
      // solve only the valid ones
      std::vector<const fs1_problem*> good;
      std::vector<int> idx;
      for (int i = 0; i < count; ++i)
        if (!bad[i]) { good.push_back(ps[i]); idx.push_back(i); }
      res.assign(count, PairResult{NAN, NAN, 0, FS1_EINVAL, 0});
      if (good.empty()) return FS1_OK;
      std::vector<PairResult> sub;
      fs1_status s2 = run_group(h, kind, mode, good, sub, geo, ms, false);
      if (s2 != FS1_OK) return s2;
      for (size_t j = 0; j < idx.size(); ++j) res[idx[j]] = sub[j];
      return FS1_OK;
    }
  }

  TeamLaunch L{};
  L.pairs = (const PairDesc*)(ws + o_desc);
  L.results = (PairResult*)(ws + o_res);
  L.order = nullptr;
  L.num_pairs = count;
  L.team_size = T;
  L.num_teams = teams;
  L.in_f32 = in_f32;
  L.slots = (Slot*)(ws + o_slot);
  L.cslots = (unsigned long long*)(ws + o_cslot);
  L.counters = (unsigned long long*)(ws + o_ctr);
  L.abort_flags = (int*)(ws + o_abt);
  if (planned) {
    int* pi = (int*)(ws + o_plan);
    L.grid = pgrid;
    L.cta_team = pi;
    L.cta_rank = pi + pgrid;
    L.team_T = pi + 2 * pgrid;
    L.team_slot = pi + 2 * pgrid + teams;
    L.team_class = pi + 2 * pgrid + 2 * teams;
    L.class_off = pi + 2 * pgrid + 3 * teams;
    L.order = pi + 2 * pgrid + 3 * teams + nclass + 1;
    L.class_next = pi + 2 * pgrid + 3 * teams + nclass + 1 + count;
    L.tickets = (unsigned long long*)(ws + o_tick);
  }
  L.spin_cap = h->cfg.spin_cap;
  cudaEventRecord(h->ev0, h->stream);
  int ls;
  if (two_d)
    ls = launch_solve_2d(desc.data(), count, in_f32, (PairResult*)(ws + o_res), ws + o_2d, h->ws_bytes - o_2d,
                         h->cfg.spin_cap, h->stream);
  else
    ls = launch_team_1d(kind | (mode << 8), L, h->stream);
  if (ls != FS1_OK) return (fs1_status)ls;
  g_launches.fetch_add(1);
  cudaEventRecord(h->ev1, h->stream);
  res.resize(count);
  if ((e = cudaMemcpyAsync(res.data(), ws + o_res, sizeof(PairResult) * count, cudaMemcpyDeviceToHost,
                           h->stream)) != cudaSuccess)
    return cuda_fail(e, "result copy");
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "solve");
  cudaEventElapsedTime(ms, h->ev0, h->ev1);
  if (planned) geo.team_size = plan.max_T;
  return FS1_OK;
}

fs1_status worst(fs1_status a, fs1_status b) {
  auto rank = [](fs1_status s) {
    switch (s) {
      case FS1_OK: return 0;
      case FS1_ENOTCONV: return 1;
      default: return 2 + (int)s;
    }
  };
  return rank(b) > rank(a) ? b : a;
}

}  // namespace

extern "C" {

fs1_status fs1_config_default(fs1_config* cfg) {
  if (!cfg) return FS1_EINVAL;
  memset(cfg, 0, sizeof *cfg);
  cfg->variant = FS1_VARIANT_LOG;
  cfg->precision = FS1_FP32;
  cfg->check_every = 1;
  cfg->team_size = 0;
  cfg->spin_cap = 1ll << 22;
  cfg->hbm_budget = 0;
  cfg->stream = nullptr;
  return FS1_OK;
}

fs1_status fs1_create(const fs1_config* cfg, fs1_handle** out) {
  if (!out) return FS1_EINVAL;
  *out = nullptr;
  fs1_config c;
  if (cfg) c = *cfg; else fs1_config_default(&c);
  if (c.variant != FS1_VARIANT_PLAIN && c.variant != FS1_VARIANT_LOG) return FS1_EINVAL;
  if (c.precision != FS1_FP64 && c.precision != FS1_FP32) return FS1_EINVAL;
  if (c.variant == FS1_VARIANT_LOG && c.precision != FS1_FP32) return FS1_EUNSUPPORTED;
  if (c.check_every != 1) return FS1_EUNSUPPORTED;
  if (c.spin_cap <= 0) c.spin_cap = 1ll << 22;
  fs1_handle* h = new (std::nothrow) fs1_handle;
  if (!h) return FS1_ENOMEM;
  h->cfg = c;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  h->stream = (cudaStream_t)c.stream;
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    delete h;
    return FS1_ECUDA;
  }
  *out = h;
  return FS1_OK;
}

void fs1_destroy(fs1_handle* h) {
  if (!h) return;
  if (h->ws || h->stage) {
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->stage) cudaFree(h->stage);
  }
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

fs1_status fs1_solve_batch(fs1_handle* h, const fs1_problem* probs, int64_t count, double* w1_out,
                           fs1_info* infos) {
  if (!h || (count > 0 && !probs) || count < 0) return FS1_EINVAL;
  if (count == 0) return FS1_OK;
  const int kind = kind_of(h->cfg);
  fs1_status overall = FS1_OK;
  std::vector<fs1_status> pst(count, FS1_OK);
  std::vector<PairResult> res(count, PairResult{NAN, NAN, 0, FS1_EINVAL, 0});
  std::vector<int> team(count, 0);
  std::vector<float> ms(count, 0.f);

  // host-located problems are staged into one grow-only device buffer
  std::vector<fs1_problem> staged(probs, probs + count);
  size_t need = 0;
  for (int64_t i = 0; i < count; ++i) {
    pst[i] = check_problem(probs[i]);
    if (pst[i] != FS1_OK || probs[i].location != FS1_MEM_HOST) continue;
    const int64_t n = npoints(probs[i]);
    const size_t in_b = align_up((probs[i].dtype == FS1_FP32 ? 4 : 8) * (size_t)n, 256);
    const size_t d_b = align_up(8 * (size_t)n, 256);
    need += 2 * in_b + (probs[i].f_out ? d_b : 0) + (probs[i].g_out ? d_b : 0) +
            (probs[i].f_init ? 2 * d_b : 0);
  }
  if (need > h->stage_bytes) {
    if (h->stage) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->stage);
      h->stage = nullptr;
      h->stage_bytes = 0;
    }
    if ((h->cfg.hbm_budget && need + h->ws_bytes > h->cfg.hbm_budget) ||
        cudaMalloc(&h->stage, need) != cudaSuccess) {
      cudaGetLastError();
      h->stage = nullptr;
      for (int64_t i = 0; i < count; ++i)
        if (pst[i] == FS1_OK && probs[i].location == FS1_MEM_HOST) pst[i] = FS1_ENOMEM;
    } else {
      h->stage_bytes = need;
    }
  }
  {
    char* cur = (char*)h->stage;
    for (int64_t i = 0; i < count && h->stage; ++i) {
      if (pst[i] != FS1_OK || probs[i].location != FS1_MEM_HOST) continue;
      const int64_t n = npoints(probs[i]);
      const size_t raw_b = (probs[i].dtype == FS1_FP32 ? 4 : 8) * (size_t)n;
      const size_t in_b = align_up(raw_b, 256);
      const size_t d_b = align_up(8 * (size_t)n, 256);
      fs1_problem& s = staged[i];
      s.a = cur; cur += in_b;
      s.b = cur; cur += in_b;
      cudaMemcpyAsync((void*)s.a, probs[i].a, raw_b, cudaMemcpyHostToDevice, h->stream);
      cudaMemcpyAsync((void*)s.b, probs[i].b, raw_b, cudaMemcpyHostToDevice, h->stream);
      s.f_out = probs[i].f_out ? (double*)cur : nullptr; cur += probs[i].f_out ? d_b : 0;
      s.g_out = probs[i].g_out ? (double*)cur : nullptr; cur += probs[i].g_out ? d_b : 0;
      if (probs[i].f_init) {
        s.f_init = (const double*)cur; cur += d_b;
        s.g_init = (const double*)cur; cur += d_b;
        cudaMemcpyAsync((void*)s.f_init, probs[i].f_init, 8 * n, cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync((void*)s.g_init, probs[i].g_init, 8 * n, cudaMemcpyHostToDevice, h->stream);
      }
      s.location = FS1_MEM_DEVICE;
    }
  }
  // group by dimension and input dtype (a launch reads one dtype); 2D groups
  // are cut into launches of at most kMaxImg2D images
  std::vector<std::pair<std::vector<const fs1_problem*>, std::vector<int64_t>>> groups;
  for (int nd = 1; nd <= 2; ++nd)
    for (int dt = 0; dt < 2; ++dt) {
      std::vector<const fs1_problem*> grp;
      std::vector<int64_t> idx;
      for (int64_t i = 0; i < count; ++i)
        if (pst[i] == FS1_OK && staged[i].dtype == dt && staged[i].ndim == nd) {
          grp.push_back(&staged[i]);
          idx.push_back(i);
          if (nd == 2 && (int)grp.size() == kMaxImg2D) {
            groups.emplace_back(grp, idx);
            grp.clear();
            idx.clear();
          }
        }
      if (!grp.empty()) groups.emplace_back(grp, idx);
    }
  for (auto& gi : groups) {
    std::vector<const fs1_problem*>& grp = gi.first;
    std::vector<int64_t>& idx = gi.second;
    std::vector<PairResult> r;
    Geometry geo{0, 0};
    float gms = 0.f;
    fs1_status s = run_group(h, kind, 0, grp, r, geo, &gms, true);
    if (s != FS1_OK) {
      for (int64_t j : idx) pst[j] = s;
      continue;
    }
    for (size_t j = 0; j < idx.size(); ++j) {
      res[idx[j]] = r[j];
      pst[idx[j]] = (fs1_status)r[j].status;
      team[idx[j]] = geo.team_size;
      ms[idx[j]] = gms;
    }
  }
  // copy host-located outputs back
  for (int64_t i = 0; i < count; ++i) {
    if (probs[i].location != FS1_MEM_HOST || staged[i].location != FS1_MEM_DEVICE) continue;
    const int64_t n = npoints(probs[i]);
    if (probs[i].f_out && staged[i].f_out)
      cudaMemcpyAsync(probs[i].f_out, staged[i].f_out, 8 * n, cudaMemcpyDeviceToHost, h->stream);
    if (probs[i].g_out && staged[i].g_out)
      cudaMemcpyAsync(probs[i].g_out, staged[i].g_out, 8 * n, cudaMemcpyDeviceToHost, h->stream);
  }
  cudaStreamSynchronize(h->stream);
  for (int64_t i = 0; i < count; ++i) {
    if (w1_out) w1_out[i] = res[i].w;
    if (infos) {
      fs1_info& f = infos[i];
      f.status = pst[i];
      f.variant = h->cfg.variant;
      f.precision = h->cfg.precision;
      f.team_size = team[i];
      f.iters = res[i].iters;
      f.marginal_err = res[i].err;
      f.w1 = res[i].w;
      f.ms = ms[i];
      f.reserved = 0.f;
    }
    overall = worst(overall, pst[i]);
  }
  return overall;
}

fs1_status fs1_w1(fs1_handle* h, const fs1_problem* prob, double* w1_out, fs1_info* info_out) {
  if (!h || !prob) return FS1_EINVAL;
  fs1_info info;
  double w = NAN;
  fs1_status s = fs1_solve_batch(h, prob, 1, &w, &info);
  if (w1_out) *w1_out = w;
  if (info_out) *info_out = info;
  return s;
}

fs1_status fs1_kernel_apply_log(fs1_handle* h, const double* in, double* out, int64_t n, double hx,
                                double eps) {
  if (!h || !in || !out || n < 1 || !(hx > 0.0) || !(eps > 0.0)) return FS1_EINVAL;
  fs1_problem p{};
  p.ndim = 1;
  p.dtype = FS1_FP64;
  p.location = FS1_MEM_DEVICE;
  p.n[0] = n;
  p.n[1] = 1;
  p.h[0] = hx;
  p.eps = eps;
  p.tol = 0.0;
  p.itr_max = 0;
  p.a = in;   // not read in this mode
  p.b = in;
  p.f_init = in;
  p.g_out = out;
  std::vector<const fs1_problem*> ps{&p};
  std::vector<PairResult> r;
  Geometry geo;
  float ms;
  return run_group(h, kind_of(h->cfg), 1, ps, r, geo, &ms, false);
}

const char* fs1_status_string(fs1_status s) {
  switch (s) {
    case FS1_OK: return "FS1_OK";
    case FS1_EINVAL: return "FS1_EINVAL";
    case FS1_ENOMEM: return "FS1_ENOMEM";
    case FS1_ENUMERIC: return "FS1_ENUMERIC";
    case FS1_ETIMEOUT: return "FS1_ETIMEOUT";
    case FS1_ENOTCONV: return "FS1_ENOTCONV";
    case FS1_ECUDA: return "FS1_ECUDA";
    case FS1_EUNSUPPORTED: return "FS1_EUNSUPPORTED";
  }
  return "FS1_UNKNOWN";
}

const char* fs1_version(void) { return kVersion; }

int64_t fs1_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
