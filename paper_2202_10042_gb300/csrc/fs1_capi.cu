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
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fs1.h"
#include "fs1_internal.h"
#include "fs1_cluster3d.h"

using namespace fs1;

struct GraphEntry {
  std::string key;             // launch signature the graph was captured for
  cudaGraphExec_t exec = nullptr;
};

struct fs1_handle {
  fs1_config cfg;
  void* stage = nullptr;       // device staging for host-located problems
  size_t stage_bytes = 0;
  int device = 0;
  int sms = 0;
  int cc = 0;                  // compute capability, 10 * major + minor
  cudaStream_t stream = nullptr;
  void* ws = nullptr;          // device workspace
  size_t ws_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // pinned host mirrors: the launch header (descriptors, initial results,
  // plan, zeroed counters) copied in one transfer, and the results
  void* hdr = nullptr;
  size_t hdr_bytes = 0;
  void* hres = nullptr;
  size_t hres_bytes = 0;
  // team-size autotuner: single-class batch signature -> team size
  std::map<std::string, int> tuned;
  bool tuning = false;         // inside trial solves
  int force_T = 0;             // team size a trial imposes
  // graphs of the 1D batch call, most recent first
  cudaStream_t cap = nullptr;  // private stream that captures
  std::vector<GraphEntry> graphs;
  std::string pending;         // last signature seen but not captured yet
  bool graphs_off = false;     // capture failed once: stay eager
  int64_t replays = 0, captures = 0, trial_launches = 0;
  int64_t exact_launches = 0, last_E = 0;   // team launches of an exact instantiation
};

namespace {

constexpr const char* kVersion = "fs1-gb300 0.1";
std::atomic<long long> g_launches{0};

fs1_status cuda_fail(cudaError_t e, const char* what) {
  fprintf(stderr, "fs1: %s: %s\n", what, cudaGetErrorString(e));
  return FS1_ECUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void drop_graphs(fs1_handle* h);

fs1_status ensure_ws(fs1_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return FS1_OK;
  if (h->cfg.hbm_budget && bytes > h->cfg.hbm_budget) return FS1_ENOMEM;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  drop_graphs(h);   // graphs hold addresses in the old workspace
  size_t want = std::max(bytes, (size_t)1 << 20);
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return FS1_ENOMEM;
  }
  h->ws_bytes = want;
  return FS1_OK;
}

void drop_graphs(fs1_handle* h) {
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  h->pending.clear();
}

fs1_status ensure_pinned(fs1_handle* h, void** buf, size_t* have, size_t bytes) {
  if (bytes <= *have) return FS1_OK;
  if (*buf) {
    cudaStreamSynchronize(h->stream);
    cudaFreeHost(*buf);
    *buf = nullptr;
    *have = 0;
  }
  drop_graphs(h);   // graphs hold the old host addresses
  const size_t want = std::max(bytes, (size_t)64 << 10);
  if (cudaHostAlloc(buf, want, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return FS1_ENOMEM;
  }
  *have = want;
  return FS1_OK;
}

// ---- validation: per pair, sums of a and b, any negative / non-finite ----
// One block per pair.  The sums are compensated FP32 pairs (Knuth's two-sum
// per addition), so the relative accuracy is about 2^-44 whatever N is, which
// is far inside the 1e-6 mass-balance tolerance; FP64 inputs enter as the
// pair (float(v), float(v - float(v))).  The block writes valid[pair] = 1
// when a, b are finite, non-negative, of positive mass and of equal mass to
// 1e-6 relative.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

__global__ void validate_kernel(const PairDesc* pairs, int in_f32, int* valid) {
  const PairDesc P = pairs[blockIdx.x];
  float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < P.n; i += blockDim.x) {
    float a0, a1 = 0.f, b0, b1 = 0.f;
    if (in_f32) {
      a0 = ((const float*)P.a)[i];
      b0 = ((const float*)P.b)[i];
    } else {
      const double va = ((const double*)P.a)[i], vb = ((const double*)P.b)[i];
      if (!(va >= 0.0) || !(vb >= 0.0) || !isfinite(va) || !isfinite(vb)) bad = 1;
      a0 = (float)va;
      a1 = (float)(va - (double)a0);
      b0 = (float)vb;
      b1 = (float)(vb - (double)b0);
    }
    if (!(a0 >= 0.f) || !(b0 >= 0.f) || !isfinite(a0) || !isfinite(b0)) bad = 1;
    two_sum_acc(ah, al, a0);
    two_sum_acc(bh, bl, b0);
    al += a1;
    bl += b1;
  }
  bad = __syncthreads_or(bad);
  __shared__ double ss[2][32];
  double sa = (double)ah + (double)al, sb = (double)bh + (double)bl;
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ss[0][threadIdx.x >> 5] = sa;
    ss[1][threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += ss[0][w];
      tb += ss[1][w];
    }
    const bool ok = !bad && ta > 0.0 && tb > 0.0 && fabs(ta - tb) <= 1e-6 * fmax(ta, tb);
    valid[blockIdx.x] = ok ? 1 : 0;
  }
}

// The same check for one large pair, in blocks of kCheckBlock points: each
// block writes its compensated sums (as FP64) and a flag; one warp then sums
// the blocks in a fixed order and applies the test of validate_kernel.
constexpr int64_t kCheckBlock = 1 << 16;

__global__ void check_range_kernel(const PairDesc* pd, int in_f32, double* part) {
  const PairDesc P = *pd;
  const int64_t lo = (int64_t)blockIdx.x * kCheckBlock;
  const int64_t hi = lo + kCheckBlock < P.n ? lo + kCheckBlock : P.n;
  float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
  int bad = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    float a0, a1 = 0.f, b0, b1 = 0.f;
    if (in_f32) {
      a0 = ((const float*)P.a)[i];
      b0 = ((const float*)P.b)[i];
    } else {
      const double va = ((const double*)P.a)[i], vb = ((const double*)P.b)[i];
      if (!(va >= 0.0) || !(vb >= 0.0) || !isfinite(va) || !isfinite(vb)) bad = 1;
      a0 = (float)va;
      a1 = (float)(va - (double)a0);
      b0 = (float)vb;
      b1 = (float)(vb - (double)b0);
    }
    if (!(a0 >= 0.f) || !(b0 >= 0.f) || !isfinite(a0) || !isfinite(b0)) bad = 1;
    two_sum_acc(ah, al, a0);
    two_sum_acc(bh, bl, b0);
    al += a1;
    bl += b1;
  }
  bad = __syncthreads_or(bad);
  __shared__ double ss[2][32];
  double sa = (double)ah + (double)al, sb = (double)bh + (double)bl;
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ss[0][threadIdx.x >> 5] = sa;
    ss[1][threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += ss[0][w];
      tb += ss[1][w];
    }
    part[3 * blockIdx.x] = ta;
    part[3 * blockIdx.x + 1] = tb;
    part[3 * blockIdx.x + 2] = bad ? 1.0 : 0.0;
  }
}

__global__ void check_final_kernel(const double* part, int nblk, int* valid) {
  const int lane = threadIdx.x & 31;
  double ta = 0, tb = 0, bad = 0;
  for (int k = lane; k < nblk; k += 32) {
    ta += part[3 * k];
    tb += part[3 * k + 1];
    bad += part[3 * k + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ta += __shfl_xor_sync(0xffffffffu, ta, o);
    tb += __shfl_xor_sync(0xffffffffu, tb, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) valid[0] = (bad == 0.0 && ta > 0.0 && tb > 0.0 && fabs(ta - tb) <= 1e-6 * fmax(ta, tb)) ? 1 : 0;
}

int kind_of(const fs1_config& c) {
  if (c.variant == FS1_VARIANT_PLAIN) return c.precision == FS1_FP64 ? KK_PLAIN_F64 : KK_PLAIN_F32;
  if (c.variant == FS1_VARIANT_PAPER) return KK_PAPER_F64;
  return KK_LOG_F32;
}

fs1_status check_problem(const fs1_problem& p) {
  if (p.ndim < 1 || p.ndim > 3) return FS1_EINVAL;
  if (p.dtype != FS1_FP64 && p.dtype != FS1_FP32) return FS1_EINVAL;
  if (p.location != FS1_MEM_DEVICE && p.location != FS1_MEM_HOST) return FS1_EINVAL;
  for (int a = 0; a < p.ndim; ++a) {
    if (p.n[a] < 1) return FS1_EINVAL;
    if (!(p.h[a] > 0.0) || !std::isfinite(p.h[a])) return FS1_EINVAL;
  }
  if (!(p.eps > 0.0) || !std::isfinite(p.eps)) return FS1_EINVAL;
  if (!(p.tol >= 0.0) || std::isnan(p.tol)) return FS1_EINVAL;
  if (p.itr_max < 0) return FS1_EINVAL;
  if (!p.a || !p.b) return FS1_EINVAL;
  if ((p.f_init == nullptr) != (p.g_init == nullptr)) return FS1_EINVAL;
  for (int a = 0; p.ndim >= 2 && a < p.ndim; ++a)
    if (p.n[a] > kMaxLine2D) return FS1_EUNSUPPORTED;
  return FS1_OK;
}

int64_t npoints(const fs1_problem& p) {
  return p.n[0] * (p.ndim >= 2 ? p.n[1] : 1) * (p.ndim == 3 ? p.n[2] : 1);
}

// team geometry for a group of problems of one kind
struct Geometry {
  int team_size;
  int num_teams;
};

fs1_status choose_geometry(fs1_handle* h, int kind, const std::vector<const fs1_problem*>& ps, Geometry* g) {
  const int thr = team_threads();
  const int maxc = max_coresident_ctas(kind);
  if (maxc <= 0) return FS1_ECUDA;
  const int tcap = std::min(maxc, kMaxTeamCtas);
  int tmin = 1, tuse = 1;
  for (auto* p : ps) {
    const double c = p->h[0] / p->eps;
    const int64_t cap = elems_cap_for(kind, c);
    const int64_t n = npoints(*p);
    const int64_t t = (n + thr * cap - 1) / (thr * cap);
    const int64_t tu = (n + thr - 1) / thr;
    if (t > tcap) return FS1_EUNSUPPORTED;   // does not fit on chip
    tmin = std::max<int>(tmin, (int)t);
    tuse = std::max<int>(tuse, (int)std::min<int64_t>(tu, tcap));
  }
  int T;
  if (h->cfg.team_size > 0) {
    T = std::max(tmin, h->cfg.team_size);
    if (T > tcap) return FS1_EINVAL;
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
// two), and every class is a queue of its problems in decreasing cost
// (longest-processing-time first).  With several classes the launch runs a
// level schedule: all CTAs start in teams of the largest class's size on its
// queue, and a team that finds its queue empty splits into teams of the next
// size down, so that the batch's work runs largest first and no CTA waits
// while another class still has problems (the iteration counts, and so the
// work per class, are not known before the solve).  Team sizes that do not
// divide each other (a class capped at the device's CTA count) fall back to a
// static split of the CTAs over the classes in proportion to N * itr_max.
//
// Small stabilised pairs (at most 32 points per thread on 8 warps) go to the
// kernel's units instead: after the teams' queues, every CTA runs 2 units of
// 8 warps on one queue, then 4 of 4 warps on another and 16 single warps on a
// third, a pair per unit (classes nc, nc + 1 and nc + 2 after the nc team
// classes); such a plan is always a level schedule over all the device's CTAs.
struct Plan {
  std::vector<int> cta_team, cta_rank, team_T, team_slot, team_class, class_off, order, class_T;
  std::vector<int> prob_T;    // team size of each problem (CTAs; 1 for a unit)
  std::vector<int> level_T;   // level schedule: team size per level (empty: static teams)
  int num_teams = 0, grid = 0, max_T = 1, slots = 0, tickets = 0;
  int unit_class = -1;        // class of the 8-warp units' queue (-1: no units)
};

// Warps of the unit that solves problem p (1, 4 or 8), or 0 for a team of
// CTAs: the fewest warps holding it at <= 32 points per thread within the
// frame cap
int unit_warps(int kind, const fs1_problem& p) {
  if (kind != KK_LOG_F32 || p.ndim != 1) return 0;
  const int64_t cap = std::min(32, elems_cap_for(kind, p.h[0] / p.eps));
  const int64_t n = npoints(p);
  return n <= 32 * cap ? 1 : (n <= 128 * cap ? 4 : (n <= 256 * cap ? 8 : 0));
}

// fewest CTAs that hold problem p on chip (0: more than fit)
int64_t min_ctas(int kind, const fs1_problem& p) {
  const int thr = team_threads();
  const int64_t cap = elems_cap_for(kind, p.h[0] / p.eps);
  return (npoints(p) + thr * cap - 1) / (thr * cap);
}

int pow2_at_least(int64_t t) {
  int p2 = 1;
  while (p2 < t) p2 <<= 1;
  return p2;
}

// Signature of a batch whose problems all fall in one size class, for the
// team-size tuning cache: device, kernel kind, the class's minimum team, the
// size octave of the largest problem and the octave of the batch size.  Empty
// when the batch spans several classes (those keep the proportional split).
std::string tune_key(fs1_handle* h, int kind, const std::vector<const fs1_problem*>& ps, int maxc) {
  int t0 = -1;
  int64_t nmax = 1;
  for (auto* p : ps) {
    const int t = std::min(pow2_at_least(min_ctas(kind, *p)), std::min(maxc, kMaxTeamCtas));
    if (t0 >= 0 && t != t0) return std::string();
    t0 = t;
    nmax = std::max<int64_t>(nmax, npoints(*p));
  }
  int nlog = 0, blog = 0;
  while (((int64_t)1 << nlog) < nmax) ++nlog;
  while (((size_t)2 << blog) <= ps.size()) ++blog;
  char buf[96];
  snprintf(buf, sizeof buf, "cc%d.sm%d.k%d.t%d.n%d.b%d", h->cc, h->sms, kind, t0, nlog, blog);
  return buf;
}

fs1_status plan_teams(fs1_handle* h, int kind, const std::vector<const fs1_problem*>& ps, Plan* P, bool units) {
  const int thr = team_threads();
  const int maxc = max_coresident_ctas(kind);
  if (maxc <= 0) return FS1_ECUDA;
  const int tcap = std::min(maxc, kMaxTeamCtas);
  const int n = (int)ps.size();
  std::vector<int> tmin(n), uw(n, 0);
  std::vector<double> cost(n);
  bool any_unit = false;
  for (int i = 0; i < n; ++i) {
    const int64_t np = npoints(*ps[i]);
    cost[i] = (double)np * (double)std::max<int64_t>(1, ps[i]->itr_max);
    if (units && (uw[i] = unit_warps(kind, *ps[i])) > 0) {
      any_unit = true;
      continue;
    }
    const int64_t t = min_ctas(kind, *ps[i]);
    if (t > tcap) return FS1_EUNSUPPORTED;
    tmin[i] = std::min<int>(pow2_at_least(t), tcap);
    if (h->cfg.team_size > 0) {
      if (h->cfg.team_size > tcap) return FS1_EINVAL;
      tmin[i] = std::max<int>((int)t, h->cfg.team_size);
    }
  }
  // classes by team size (a batch of unit pairs only keeps one empty class of
  // teams of one CTA), then the units' three classes
  std::vector<int> keys;
  for (int i = 0; i < n; ++i)
    if (uw[i] == 0) keys.push_back(tmin[i]);
  if (keys.empty()) keys.push_back(1);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int nc = (int)keys.size();
  const int nq = nc + (any_unit ? 3 : 0);   // queues
  std::vector<double> W(nq, 0.0);
  std::vector<int> cnt(nq, 0), cls(n);
  for (int i = 0; i < n; ++i) {
    cls[i] = uw[i] == 8   ? nc
             : uw[i] == 4 ? nc + 1
             : uw[i] == 1 ? nc + 2
                          : (int)(std::lower_bound(keys.begin(), keys.end(), tmin[i]) - keys.begin());
    W[cls[i]] += cost[i];
    cnt[cls[i]] += 1;
  }
  double Wt = 0.0;
  for (double w : W) Wt += w;
  std::vector<int> T(keys), teams(nc, 1);
  int base = 0;
  for (int k = 0; k < nc; ++k) base += T[k];
  if (base > maxc) return FS1_EUNSUPPORTED;   // caller splits by class
  int force = h->force_T;
  if (nc == 1 && force <= 0 && h->cfg.autotune && h->cfg.team_size <= 0 && !h->tuning) {
    auto it = h->tuned.find(tune_key(h, kind, ps, maxc));
    if (it != h->tuned.end()) force = it->second;
  }
  bool levels = (nc > 1 || any_unit) && h->cfg.team_size <= 0;
  for (int k = 1; k < nc && levels; ++k) levels = T[k] % T[k - 1] == 0;
  if (any_unit && !levels) return FS1_EINVAL;   // the caller plans again without units
  if (levels) {
    teams.assign(nc, 0);
    teams[nc - 1] = maxc / T[nc - 1];
  } else if (nc == 1 && force > 0) {
    T[0] = std::min(tcap, std::max(T[0], force));
    teams[0] = std::max(1, std::min(cnt[0], maxc / T[0]));
  } else if (nc == 1) {
    teams[0] = std::max(1, std::min(cnt[0], maxc / T[0]));
    if (h->cfg.team_size <= 0) {
      int tuse = 1;
      for (int i = 0; i < n; ++i)
        tuse = std::max<int>(tuse, (int)std::min<int64_t>((npoints(*ps[i]) + thr - 1) / thr, tcap));
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
  P->level_T.clear();
  if (levels)
    for (int k = nc - 1; k >= 0; --k) P->level_T.push_back(T[k]);
  P->unit_class = any_unit ? nc : -1;
  P->class_off.assign(nq + 1, 0);
  for (int k = 0; k < nq; ++k) P->class_off[k + 1] = P->class_off[k] + cnt[k];
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
  P->slots = levels ? nc * 2 * P->grid : slot;
  P->tickets = levels ? nc * P->grid : P->num_teams;
  P->prob_T.assign(n, 0);
  for (int i = 0; i < n; ++i) P->prob_T[i] = uw[i] > 0 ? 1 : T[cls[i]];
  return FS1_OK;
}

fs1_status run_group(fs1_handle* h, int kind, int mode, const std::vector<const fs1_problem*>& ps,
                     std::vector<PairResult>& res, Geometry& geo, float* ms, bool validate);

// Team-size autotuner for a batch whose problems share one size class.  Trial
// solves of the class's costliest problems (as many as the smallest team runs
// at once), `trial_iters` iterations each with tol = 0 and no outputs, are
// timed for each candidate team size; the size with the most N * iterations
// per second is kept under the batch signature (and appended to the cache
// file named by FS1_AUTOTUNE_CACHE).
fs1_status autotune(fs1_handle* h, int kind, const std::vector<const fs1_problem*>& ps, const std::string& key,
                    int maxc) {
  const int thr = team_threads();
  const int tcap = std::min(maxc, kMaxTeamCtas);
  int tmin = 1;
  int64_t tuse = 1;
  for (auto* p : ps) {
    tmin = std::max(tmin, std::min(pow2_at_least(min_ctas(kind, *p)), tcap));
    tuse = std::max<int64_t>(tuse, std::min<int64_t>((npoints(*p) + thr - 1) / thr, tcap));
  }
  // candidates: powers of two from tmin, and for 1, 2, 3, 4, 6, 8, 12, ...
  // concurrent teams the team size that fills the GPU; none beyond the
  // CTAs that still give every thread a grid point
  std::vector<int> cand;
  auto add = [&](int64_t T) {
    T = std::min<int64_t>(std::max<int64_t>(T, tmin), std::max<int64_t>(tmin, tuse));
    if (T <= tcap && std::find(cand.begin(), cand.end(), (int)T) == cand.end()) cand.push_back((int)T);
  };
  for (int64_t T = tmin; T <= tcap; T *= 2) add(T);
  for (int t = 1; t <= maxc / tmin; t = t < 4 ? t + 1 : t + t / 2) add(maxc / t);
  std::sort(cand.begin(), cand.end());
  std::vector<const fs1_problem*> srt(ps);
  auto cost = [](const fs1_problem* p) { return (double)npoints(*p) * (double)std::max<int64_t>(1, p->itr_max); };
  std::stable_sort(srt.begin(), srt.end(), [&](const fs1_problem* x, const fs1_problem* y) { return cost(x) > cost(y); });
  const size_t m = std::min(srt.size(), (size_t)std::max(1, maxc / tmin));
  std::vector<fs1_problem> trial(m);
  std::vector<const fs1_problem*> tp(m);
  for (size_t i = 0; i < m; ++i) {
    trial[i] = *srt[i];
    trial[i].itr_max = std::max<int64_t>(1, std::min<int64_t>(srt[i]->itr_max, h->cfg.trial_iters));
    trial[i].tol = 0.0;
    trial[i].f_out = nullptr;
    trial[i].g_out = nullptr;
    tp[i] = &trial[i];
  }
  int best_T = 0;
  double best_rate = 0.0;
  h->tuning = true;
  fs1_status st = FS1_OK;
  for (const int T : cand) {
    h->force_T = T;
    std::vector<PairResult> r;
    Geometry g{0, 0};
    float tms = 0.f, t2 = 0.f;
    // two runs, the faster one counts (the first also warms caches and clocks)
    if ((st = run_group(h, kind, 0, tp, r, g, &tms, true)) != FS1_OK) break;
    if ((st = run_group(h, kind, 0, tp, r, g, &t2, true)) != FS1_OK) break;
    tms = std::min(tms, t2);
    double work = 0.0;
    for (size_t i = 0; i < m; ++i)
      if (r[i].status == FS1_OK || r[i].status == FS1_ENOTCONV) work += (double)npoints(*tp[i]) * (double)r[i].iters;
    const double rate = tms > 0.f ? work / tms : 0.0;
    if (rate > best_rate) {
      best_rate = rate;
      best_T = T;
    }
  }
  h->tuning = false;
  h->force_T = 0;
  if (st != FS1_OK) return st;
  h->tuned[key] = best_T;   // 0: no trial ran; the fixed heuristic stays
  if (const char* path = getenv("FS1_AUTOTUNE_CACHE")) {
    if (FILE* f = fopen(path, "a")) {
      fprintf(f, "%s %d\n", key.c_str(), best_T);
      fclose(f);
    }
  }
  return FS1_OK;
}

// Launch signature of a 1D call: the sizes, workspace offsets and kernel
// arguments a captured graph bakes in.  The header's contents (descriptors,
// plan) are data copied from pinned memory on every replay.
std::string graph_key(int kind, int mode, int in_f32, int count, int grid, int T, int teams, int nclass,
                      int nlevel, int unit_class, size_t nslots, size_t hdr, bool validate, long long spin_cap,
                      int exact_E) {
  char buf[192];
  snprintf(buf, sizeof buf, "%d.%d.%d.%d.%d.%d.%d.%d.%d.%d.%zu.%zu.%d.%lld.%d", kind, mode, in_f32, count, grid, T,
           teams, nclass, nlevel, unit_class, nslots, hdr, (int)validate, spin_cap, exact_E);
  return buf;
}

// The point count per thread shared by every pair of a team launch (each pair
// of N points on a team of T CTAs gives every thread ceil(N / (512 T))
// points), or 0 when the pairs differ; the launch then takes the exact
// instantiation of that count when one is built.
int common_points_per_thread(const std::vector<const fs1_problem*>& ps, const std::vector<int>& team_of) {
  const int64_t thr = team_threads();
  int64_t e0 = -1;
  for (size_t i = 0; i < ps.size(); ++i) {
    const int64_t t = team_of[i];
    const int64_t e = (npoints(*ps[i]) + thr * t - 1) / (thr * t);
    if (e0 >= 0 && e != e0) return 0;
    e0 = e;
  }
  return e0 > 0 && e0 <= 32 ? (int)e0 : 0;
}

// Run one group (same kind and input dtype; all 1D or all 2D; device-located).
//
// Workspace layout:
//   header   descriptors | initial results | plan | tickets | counters | aborts
//            (one host-to-device copy from its pinned mirror)
//   valid    per-pair input-check flags (written by the check kernel)
//   slots    generic | compact exchange slots (one memset)
//   2D       per-image state of the 2D solver
// A 1D call is: header copy, slot memset, input check, team kernel, result
// copy, and one stream synchronisation; the team kernel skips (and reports
// FS1_EINVAL for) pairs whose check failed.  From the second call with the
// same launch signature on, that sequence is a replayed CUDA graph.
fs1_status run_group(fs1_handle* h, int kind, int mode, const std::vector<const fs1_problem*>& ps,
                     std::vector<PairResult>& res, Geometry& geo, float* ms, bool validate) {
  const int count = (int)ps.size();
  const bool two_d = ps[0]->ndim >= 2;   // 2D and 3D grids share the grid kernel
  fs1_status st = FS1_OK;
  const bool paper = kind == KK_PAPER_F64;   // one CTA per pair, no teams
  if (two_d) {
    if (kind != KK_LOG_F32) return FS1_EUNSUPPORTED;   // 2D runs the stabilised FP32 variant
    geo.team_size = 0;
    geo.num_teams = 0;
  } else if (paper) {
    if (mode != 0) return FS1_EUNSUPPORTED;
    geo.team_size = 1;
    geo.num_teams = count;
  } else if ((st = choose_geometry(h, kind, ps, &geo)) != FS1_OK) {
    return st;
  }
  const bool planned = !two_d && !paper && mode == 0;
  // small stabilised pairs of a batch on the kernel's units (no team-size
  // tuning then), when they outnumber the co-resident CTAs: with fewer, a
  // whole CTA each leaves no SM idle and runs each pair with shorter serial
  // chains (100 pairs of 8000 points: 1.17e11 N*it/s on whole CTAs, 8.4e10
  // on units of 8 warps that used a third of the SMs).  A lone pair keeps
  // whole CTAs too, so that fs1_w1 stays the computation fs1_w1_noalloc
  // repeats.
  bool units = planned && count > 1 && kind == KK_LOG_F32 && h->cfg.units && h->cfg.team_size <= 0 && !h->tuning;
  if (units) {
    int nu = 0;
    for (auto* p : ps) nu += unit_warps(kind, *p) > 0 ? 1 : 0;
    units = nu > max_coresident_ctas(kind);
  }
  if (planned && !units && h->cfg.autotune && h->cfg.team_size <= 0 && !h->tuning) {
    const int maxc = max_coresident_ctas(kind);
    const std::string key = tune_key(h, kind, ps, maxc);
    if (!key.empty() && !h->tuned.count(key) && (st = autotune(h, kind, ps, key, maxc)) != FS1_OK) return st;
  }
  Plan plan;
  if (planned) {
    st = plan_teams(h, kind, ps, &plan, units);
    if (st == FS1_EINVAL && units) {   // no level schedule for these team sizes: teams only
      units = false;
      st = plan_teams(h, kind, ps, &plan, false);
    }
    if (st != FS1_OK) return st;
  }
  const int T = two_d ? 1 : (planned ? plan.max_T : geo.team_size);
  const int teams = two_d ? 1 : (planned ? plan.num_teams : geo.num_teams);
  const size_t nslots = (two_d || paper) ? 0 : (planned ? (size_t)plan.slots : (size_t)teams * 2 * T);
  const int in_f32 = ps[0]->dtype == FS1_FP32;
  const int nclass = planned ? (int)plan.class_off.size() - 1 : 0;   // queues
  const int pgrid = planned ? plan.grid : 0;
  const int nlevel = planned ? (int)plan.level_T.size() : 0;
  // plan arrays: cta_team, cta_rank [grid]; team_T, team_slot, team_class
  // [teams]; class_off [nc + 1]; order [count]; class_next [nc]; level_T [nlevel]
  const size_t plan_ints =
      planned ? (size_t)2 * pgrid + 3 * teams + (nclass + 1) + count + nclass + nlevel : 0;
  size_t off = 0;
  const size_t o_desc = off; off = align_up(off + sizeof(PairDesc) * count, 256);
  const size_t o_res = off;  off = align_up(off + sizeof(PairResult) * count, 256);
  const size_t o_plan = off; off = align_up(off + sizeof(int) * plan_ints, 256);
  const size_t o_tick = off; off = align_up(off + sizeof(unsigned long long) * (planned ? plan.tickets : 0), 256);
  const size_t o_ctr = off;  off = align_up(off + sizeof(unsigned long long) * teams, 256);
  const size_t o_abt = off;  off = align_up(off + sizeof(int) * teams, 256);
  const size_t o_poff = off; off = align_up(off + sizeof(int64_t) * (paper ? count : 0), 256);
  const size_t hdr = off;
  const size_t o_val = off;  off = align_up(off + sizeof(int) * count, 256);
  const size_t o_slot = off; off = align_up(off + sizeof(Slot) * nslots, 256);
  off = align_up(off + 128 * nslots, 256);
  const size_t slot_end = off;
  std::vector<PairDesc> desc(count);
  for (int i = 0; i < count; ++i) {
    const fs1_problem& p = *ps[i];
    PairDesc d{};
    d.a = p.a;
    d.b = p.b;
    d.n = npoints(p);
    d.n_fast = p.n[0];
    d.n_mid = p.ndim == 3 ? p.n[1] : 1;
    d.n_slow = p.ndim == 3 ? p.n[2] : (p.ndim == 2 ? p.n[1] : 1);
    d.h_fast = p.h[0];
    d.h_mid = p.ndim == 3 ? p.h[1] : 0.0;
    d.h_slow = p.ndim == 3 ? p.h[2] : (p.ndim == 2 ? p.h[1] : 0.0);
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
  // (the grid kernel may take three launches: room for the others' tables)
  if (two_d)
    off = align_up(off + solve2d_workspace(desc.data(), count) + 2 * solve2d_workspace(nullptr, 0) + 2048, 256);
  // 2D images the cluster-resident kernel holds (first in `perm`), 3D grids
  // its 3D variant holds (next), then the rest for the grid kernel by launch
  // class (solve2d_class), one launch each.  The 3D grids' transport cost is
  // one more grid-kernel launch (no iterations, warm-started from the final
  // iterate) with its own workspace and results.
  std::vector<int> perm;
  int ncl = 0, ncl3 = 0;
  int gb[4] = {0, 0, 0, 0};   // [gb[q], gb[q + 1]) of perm: grid launch q
  const size_t o_c2d = off;
  size_t o_c3d = off, o_cost = off, o_cres = off;
  if (two_d) {
    auto on_cluster = [&](int i) { return !h->cfg.grid2d && cluster2d_inst(desc[i]) >= 0; };
    auto on_cluster3 = [&](int i) { return !h->cfg.grid2d && desc[i].n_mid > 1 && cluster3d_ok(desc[i]); };
    for (int i = 0; i < count; ++i)
      if (on_cluster(i)) perm.push_back(i);
    ncl = (int)perm.size();
    for (int i = 0; i < count; ++i)
      if (on_cluster3(i)) perm.push_back(i);
    ncl3 = (int)perm.size() - ncl;
    gb[0] = ncl + ncl3;
    for (int q = 0; q < 3; ++q) {
      for (int i = 0; i < count; ++i)
        if (!on_cluster(i) && !on_cluster3(i) && solve2d_class(desc[i]) == q) perm.push_back(i);
      gb[q + 1] = (int)perm.size();
    }
    std::vector<PairDesc> dcl(ncl), d3(ncl3);
    for (int k = 0; k < ncl; ++k) dcl[k] = desc[perm[k]];
    for (int k = 0; k < ncl3; ++k) d3[k] = desc[perm[ncl + k]];
    if (ncl) off = align_up(off + cluster2d_workspace(dcl.data(), ncl), 256);
    o_c3d = off;
    if (ncl3) {
      off = align_up(off + cluster3d_workspace(d3.data(), ncl3), 256);
      o_cost = off;
      off = align_up(off + solve2d_workspace(d3.data(), ncl3) + 2048, 256);
      o_cres = off;
      off = align_up(off + sizeof(PairResult) * ncl3, 256);
    }
  }
  // paper form: kPaperArrays FP64 arrays of N per pair
  std::vector<int64_t> poff(paper ? count : 0);
  const size_t o_paper = off;
  if (paper) {
    int64_t acc = 0;
    for (int i = 0; i < count; ++i) {
      if (desc[i].n > kMaxPaperN) return FS1_EUNSUPPORTED;
      poff[i] = acc;
      acc += (int64_t)kPaperArrays * desc[i].n;
    }
    off = align_up(off + sizeof(double) * (size_t)acc, 256);
  }
  if ((st = ensure_ws(h, off)) != FS1_OK) return st;
  if ((st = ensure_pinned(h, &h->hdr, &h->hdr_bytes, hdr)) != FS1_OK) return st;
  // pinned results: [count] results, [count] input-check flags, [ncl3] 3D costs
  const size_t o_hcost = sizeof(PairResult) * count + align_up(sizeof(int) * count, 16);
  if ((st = ensure_pinned(h, &h->hres, &h->hres_bytes, o_hcost + sizeof(PairResult) * ncl3)) != FS1_OK) return st;
  char* ws = (char*)h->ws;

  // header image (nothing of ours is in flight: every call ends synchronised)
  char* hb = (char*)h->hdr;
  memset(hb, 0, hdr);
  memcpy(hb + o_desc, desc.data(), sizeof(PairDesc) * count);
  PairResult* r0 = (PairResult*)(hb + o_res);
  for (int i = 0; i < count; ++i) r0[i] = PairResult{NAN, NAN, 0, FS1_ETIMEOUT, 0};
  if (planned) {
    int* pi = (int*)(hb + o_plan);
    for (const std::vector<int>* v : {&plan.cta_team, &plan.cta_rank, &plan.team_T, &plan.team_slot,
                                      &plan.team_class, &plan.class_off, &plan.order}) {
      std::copy(v->begin(), v->end(), pi);
      pi += v->size();
    }
    // class_next stays zero
    std::copy(plan.level_T.begin(), plan.level_T.end(), pi + nclass);
  }
  if (paper) memcpy(hb + o_poff, poff.data(), sizeof(int64_t) * count);
  PairResult* hres = (PairResult*)h->hres;
  cudaError_t e;

  if (two_d) {
    if ((e = cudaMemcpyAsync(ws, hb, hdr, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
      return cuda_fail(e, "header copy");
    if (validate) {
      int* hval = (int*)(hres + count);
      validate_kernel<<<count, 256, 0, h->stream>>>((const PairDesc*)(ws + o_desc), in_f32, (int*)(ws + o_val));
      g_launches.fetch_add(1);
      if ((e = cudaMemcpyAsync(hval, ws + o_val, sizeof(int) * count, cudaMemcpyDeviceToHost, h->stream)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(e, "input check");
      std::vector<const fs1_problem*> good;
      std::vector<int> idx;
      for (int i = 0; i < count; ++i)
        if (hval[i]) {
          good.push_back(ps[i]);
          idx.push_back(i);
        }
      if ((int)good.size() < count) {
        res.assign(count, PairResult{NAN, NAN, 0, FS1_EINVAL, 0});
        if (good.empty()) return FS1_OK;
        std::vector<PairResult> sub;
        if ((st = run_group(h, kind, mode, good, sub, geo, ms, false)) != FS1_OK) return st;
        for (size_t j = 0; j < idx.size(); ++j) res[idx[j]] = sub[j];
        return FS1_OK;
      }
    }
    std::vector<PairDesc> dp(count);
    for (int k = 0; k < count; ++k) dp[k] = desc[perm[k]];
    PairResult* d_res = (PairResult*)(ws + o_res);   // in the order of perm
    cudaEventRecord(h->ev0, h->stream);
    long long nl = 0;
    if (ncl) {
      const int ls = launch_cluster_2d(dp.data(), ncl, in_f32, d_res, nullptr, ws + o_c2d, h->ws_bytes - o_c2d,
                                       h->stream, &nl);
      if (ls != FS1_OK) return (fs1_status)ls;
    }
    if (ncl3) {
      std::vector<PairDesc> cost3(ncl3);
      int ls = launch_cluster_3d(dp.data() + ncl, ncl3, in_f32, d_res + ncl, ws + o_c3d, o_cost - o_c3d, h->stream,
                                 &nl, cost3.data());
      if (ls != FS1_OK) return (fs1_status)ls;
      ls = launch_solve_2d(cost3.data(), ncl3, in_f32, (PairResult*)(ws + o_cres), ws + o_cost, o_cres - o_cost,
                           h->cfg.spin_cap, h->stream);
      if (ls != FS1_OK) return (fs1_status)ls;
      ++nl;
    }
    // the grid kernel: one launch per class (each launch's workspace follows
    // the previous one's)
    size_t o_g = o_2d;
    for (int q = 0; q < 3; ++q) {
      const int k0 = gb[q], k1 = gb[q + 1];
      if (k1 <= k0) continue;
      const size_t wsz = solve2d_workspace(dp.data() + k0, k1 - k0);
      const int ls = launch_solve_2d(dp.data() + k0, k1 - k0, in_f32, d_res + k0, ws + o_g, wsz, h->cfg.spin_cap,
                                     h->stream);
      if (ls != FS1_OK) return (fs1_status)ls;
      o_g += wsz;
      ++nl;
    }
    g_launches.fetch_add(nl);
    cudaEventRecord(h->ev1, h->stream);
    if ((e = cudaMemcpyAsync(hres, ws + o_res, sizeof(PairResult) * count, cudaMemcpyDeviceToHost, h->stream)) !=
        cudaSuccess)
      return cuda_fail(e, "result copy");
    if (ncl3 && (e = cudaMemcpyAsync((char*)hres + o_hcost, ws + o_cres, sizeof(PairResult) * ncl3,
                                     cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
      return cuda_fail(e, "result copy");
  } else {
    TeamLaunch L{};
    L.pairs = (const PairDesc*)(ws + o_desc);
    L.results = (PairResult*)(ws + o_res);
    L.order = nullptr;
    L.num_pairs = count;
    L.team_size = T;
    L.num_teams = teams;
    L.in_f32 = in_f32;
    L.slots = (Slot*)(ws + o_slot);
    L.cslots = (unsigned long long*)(ws + o_slot + align_up(sizeof(Slot) * nslots, 256));
    L.counters = (unsigned long long*)(ws + o_ctr);
    L.abort_flags = (int*)(ws + o_abt);
    L.valid = validate ? (const int*)(ws + o_val) : nullptr;
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
      L.nlevel = nlevel;
      L.level_T = nlevel ? L.class_next + nclass : nullptr;
      L.unit_queues = plan.unit_class >= 0 ? 1 : 0;
      L.unit_class = plan.unit_class;
    }
    L.spin_cap = h->cfg.spin_cap;
    // level schedules run on the generic instantiation
    const int exact_E = (paper || nlevel > 0)
                            ? 0
                            : common_points_per_thread(ps, planned ? plan.prob_T : std::vector<int>(count, T));
    // the call's stream work, issued on s (captured when s is the capture stream)
    auto issue = [&](cudaStream_t s, bool capturing) -> fs1_status {
      cudaError_t ee;
      if ((ee = cudaMemcpyAsync(ws, hb, hdr, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(ee, "header copy");
      if (nslots && (ee = cudaMemsetAsync(ws + o_slot, 0, slot_end - o_slot, s)) != cudaSuccess)
        return cuda_fail(ee, "slot reset");
      if (validate)
        validate_kernel<<<count, 256, 0, s>>>((const PairDesc*)(ws + o_desc), in_f32, (int*)(ws + o_val));
      if (capturing)
        cudaEventRecordWithFlags(h->ev0, s, cudaEventRecordExternal);
      else
        cudaEventRecord(h->ev0, s);
      const int ls = paper ? launch_paper_1d(L.pairs, count, L.results, (double*)(ws + o_paper),
                                             (const int64_t*)(ws + o_poff), in_f32, h->cfg.tau, L.valid, s)
                           : launch_team_1d(kind | (mode << 8), L, s, exact_E);
      if (ls != FS1_OK) return (fs1_status)ls;
      if (capturing)
        cudaEventRecordWithFlags(h->ev1, s, cudaEventRecordExternal);
      else
        cudaEventRecord(h->ev1, s);
      if ((ee = cudaMemcpyAsync(hres, ws + o_res, sizeof(PairResult) * count, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess)
        return cuda_fail(ee, "result copy");
      return FS1_OK;
    };
    const bool graphs = h->cfg.use_graph && !h->graphs_off && !h->tuning;
    const std::string gkey =
        graphs ? graph_key(kind, mode, in_f32, count, planned ? pgrid : teams * T, T, teams, nclass, nlevel,
                           planned ? plan.unit_class : -1, nslots, hdr, validate, h->cfg.spin_cap, exact_E)
               : std::string();
    cudaGraphExec_t exec = nullptr;
    for (size_t k = 0; graphs && k < h->graphs.size(); ++k)
      if (h->graphs[k].key == gkey) {
        exec = h->graphs[k].exec;
        std::rotate(h->graphs.begin(), h->graphs.begin() + k, h->graphs.begin() + k + 1);   // to the front
        break;
      }
    if (!exec && graphs && h->pending == gkey) {
      // second call with this signature: capture it
      cudaGraph_t g = nullptr;
      fs1_status cs = FS1_OK;
      if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cs = issue(h->cap, true);
        const cudaError_t ce = cudaStreamEndCapture(h->cap, &g);
        if (cs == FS1_OK && ce == cudaSuccess && g &&
            cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
          h->graphs.insert(h->graphs.begin(), GraphEntry{gkey, exec});
          if (h->graphs.size() > 4) {
            cudaGraphExecDestroy(h->graphs.back().exec);
            h->graphs.pop_back();
          }
        } else {
          exec = nullptr;
        }
        if (g) cudaGraphDestroy(g);
      }
      if (!exec) {
        cudaGetLastError();
        h->graphs_off = true;   // stay eager on this handle
        fprintf(stderr, "fs1: graph capture unavailable, launching directly\n");
      }
      h->pending.clear();
      if (exec) ++h->captures;
    }
    if (exec) {
      if ((e = cudaGraphLaunch(exec, h->stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
      ++h->replays;
    } else {
      if ((st = issue(h->stream, false)) != FS1_OK) return st;
      if (graphs) h->pending = gkey;
    }
    g_launches.fetch_add(validate ? 2 : 1);
    if (h->tuning) h->trial_launches += 1;
    if (!paper) {
      h->last_E = team_exact_built(kind, exact_E) ? exact_E : 0;
      if (h->last_E) ++h->exact_launches;
    }
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "solve");
  if (cudaEventElapsedTime(ms, h->ev0, h->ev1) != cudaSuccess) {
    cudaGetLastError();
    *ms = NAN;
  }
  if (two_d) {
    res.assign(count, PairResult{});
    for (int k = 0; k < count; ++k) res[perm[k]] = hres[k];
    // the 3D cluster kernel's grids take their cost from the cost launch
    const PairResult* hcost = (const PairResult*)((const char*)hres + o_hcost);
    for (int k = ncl; k < ncl + ncl3; ++k) {
      PairResult& r = res[perm[k]];
      if (r.status != FS1_OK && r.status != FS1_ENOTCONV) continue;
      if (hcost[k - ncl].status == FS1_ETIMEOUT)
        r.status = FS1_ETIMEOUT;
      else
        r.w = hcost[k - ncl].w;
    }
    // an image whose scalings left a cluster kernel's exponent range is
    // solved again by the grid kernel
    std::vector<int> again;
    for (int k = 0; k < ncl + ncl3; ++k)
      if (hres[k].status == FS1_EUNSUPPORTED) again.push_back(perm[k]);
    if (!again.empty()) {
      std::vector<PairDesc> dg(again.size());
      for (size_t k = 0; k < again.size(); ++k) dg[k] = desc[again[k]];
      PairResult* d_res = (PairResult*)(ws + o_res);
      float ms2 = 0.f;
      cudaEventRecord(h->ev0, h->stream);
      const int ls = launch_solve_2d(dg.data(), (int)dg.size(), in_f32, d_res, ws + o_2d, o_c2d - o_2d,
                                     h->cfg.spin_cap, h->stream);
      if (ls != FS1_OK) return (fs1_status)ls;
      g_launches.fetch_add(1);
      cudaEventRecord(h->ev1, h->stream);
      if ((e = cudaMemcpyAsync(hres, d_res, sizeof(PairResult) * dg.size(), cudaMemcpyDeviceToHost, h->stream)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(e, "grid-kernel solve");
      if (cudaEventElapsedTime(&ms2, h->ev0, h->ev1) == cudaSuccess) *ms += ms2;
      for (size_t k = 0; k < again.size(); ++k) res[again[k]] = hres[k];
    }
    return FS1_OK;
  }
  res.assign(hres, hres + count);
  if (planned) geo.team_size = plan.max_T;
  return FS1_OK;
}

// The call's stabilised 1D pairs beyond the on-chip capacity: input checks,
// then the solves with the state in device memory (fs1_stream.cu), up to 8
// pairs sharing each half-step launch.  The workspace holds a head (results |
// check flags | descriptors | check partials per pair) and the pairs' arrays;
// when the HBM budget cannot hold all of them at once they go one by one.
fs1_status run_stream_batch(fs1_handle* h, const std::vector<const fs1_problem*>& ps, std::vector<PairResult>& rs,
                            float* ms) {
  const int count = (int)ps.size();
  std::vector<int64_t> n(count);
  std::vector<int> nblk(count);
  std::vector<size_t> poff(count);
  size_t head = align_up(sizeof(PairResult) * count, 256) + align_up(sizeof(int) * count, 256) +
                align_up(sizeof(PairDesc) * count, 256);
  for (int i = 0; i < count; ++i) {
    n[i] = npoints(*ps[i]);
    nblk[i] = (int)((n[i] + kCheckBlock - 1) / kCheckBlock);
    poff[i] = head;
    head += align_up(sizeof(double) * 3 * (size_t)nblk[i], 256);
  }
  fs1_status s = ensure_ws(h, head + stream_workspace(n.data(), count));
  if (s == FS1_ENOMEM && count > 1) {
    rs.assign(count, PairResult{NAN, NAN, 0, FS1_ENOMEM, 0});
    *ms = 0.f;
    for (int i = 0; i < count; ++i) {
      std::vector<PairResult> one;
      float m = 0.f;
      if ((s = run_stream_batch(h, {ps[i]}, one, &m)) != FS1_OK) return s;
      rs[i] = one[0];
      *ms += m;
    }
    return FS1_OK;
  }
  if (s != FS1_OK) return s;
  if ((s = ensure_pinned(h, &h->hdr, &h->hdr_bytes, sizeof(PairDesc) * count)) != FS1_OK) return s;
  if ((s = ensure_pinned(h, &h->hres, &h->hres_bytes, (sizeof(PairResult) + sizeof(int)) * count)) != FS1_OK)
    return s;
  char* ws = (char*)h->ws;
  PairResult* d_res = (PairResult*)ws;
  int* d_valid = (int*)(ws + align_up(sizeof(PairResult) * count, 256));
  PairDesc* d_desc = (PairDesc*)((char*)d_valid + align_up(sizeof(int) * count, 256));
  std::vector<PairDesc> desc(count);
  std::vector<int> f32(count);
  for (int i = 0; i < count; ++i) {
    const fs1_problem& p = *ps[i];
    PairDesc d{};
    d.a = p.a;
    d.b = p.b;
    d.n = n[i];
    d.n_fast = n[i];
    d.n_mid = 1;
    d.n_slow = 1;
    d.h_fast = p.h[0];
    d.eps = p.eps;
    d.tol = p.tol;
    d.itr_max = p.itr_max;
    d.f_out = p.f_out;
    d.g_out = p.g_out;
    d.f_init = p.f_init;
    d.g_init = p.g_init;
    desc[i] = d;
    f32[i] = p.dtype == FS1_FP32;
  }
  memcpy(h->hdr, desc.data(), sizeof(PairDesc) * count);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_desc, h->hdr, sizeof(PairDesc) * count, cudaMemcpyHostToDevice, h->stream)) !=
      cudaSuccess)
    return cuda_fail(e, "descriptor copy");
  for (int i = 0; i < count; ++i) {
    check_range_kernel<<<nblk[i], 256, 0, h->stream>>>(d_desc + i, f32[i], (double*)(ws + poff[i]));
    check_final_kernel<<<1, 32, 0, h->stream>>>((const double*)(ws + poff[i]), nblk[i], d_valid + i);
  }
  g_launches.fetch_add(2 * count);
  int* hval = (int*)((char*)h->hres + sizeof(PairResult) * count);
  if ((e = cudaMemcpyAsync(hval, d_valid, sizeof(int) * count, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return cuda_fail(e, "input check");
  rs.assign(count, PairResult{NAN, NAN, 0, FS1_EINVAL, 0});
  *ms = 0.f;
  std::vector<PairDesc> dv;
  std::vector<int> fv, idx;
  for (int i = 0; i < count; ++i)
    if (hval[i]) {
      dv.push_back(desc[i]);
      fv.push_back(f32[i]);
      idx.push_back(i);
    }
  if (dv.empty()) return FS1_OK;
  const int nv = (int)dv.size();
  cudaEventRecord(h->ev0, h->stream);
  long long nl = 0;
  const int ls = solve_stream_batch(dv.data(), fv.data(), nv, d_res, ws + head, h->ws_bytes - head, h->stream, &nl);
  g_launches.fetch_add(nl);
  if (ls != FS1_OK) return (fs1_status)ls;
  cudaEventRecord(h->ev1, h->stream);
  PairResult* hr = (PairResult*)h->hres;
  if ((e = cudaMemcpyAsync(hr, d_res, sizeof(PairResult) * nv, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return cuda_fail(e, "streaming solve");
  for (int k = 0; k < nv; ++k) rs[idx[k]] = hr[k];
  if (cudaEventElapsedTime(ms, h->ev0, h->ev1) != cudaSuccess) {
    cudaGetLastError();
    *ms = NAN;
  }
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
  cfg->autotune = 1;
  cfg->trial_iters = 48;
  cfg->use_graph = 1;
  cfg->tau = 1e10;
  cfg->grid2d = 0;
  cfg->units = 1;
  return FS1_OK;
}

fs1_status fs1_create(const fs1_config* cfg, fs1_handle** out) {
  if (!out) return FS1_EINVAL;
  *out = nullptr;
  fs1_config c;
  if (cfg) c = *cfg; else fs1_config_default(&c);
  if (c.variant != FS1_VARIANT_PLAIN && c.variant != FS1_VARIANT_LOG && c.variant != FS1_VARIANT_PAPER)
    return FS1_EINVAL;
  if (c.precision != FS1_FP64 && c.precision != FS1_FP32) return FS1_EINVAL;
  if (c.variant == FS1_VARIANT_LOG && c.precision != FS1_FP32) return FS1_EUNSUPPORTED;
  if (c.variant == FS1_VARIANT_PAPER && c.precision != FS1_FP64) return FS1_EUNSUPPORTED;
  if (c.variant == FS1_VARIANT_PAPER && !(c.tau > 0.0)) return FS1_EINVAL;
  if (c.check_every != 1) return FS1_EUNSUPPORTED;
  if (c.spin_cap <= 0) c.spin_cap = 1ll << 22;
  if (c.trial_iters <= 0) c.trial_iters = 48;
  fs1_handle* h = new (std::nothrow) fs1_handle;
  if (!h) return FS1_ENOMEM;
  h->cfg = c;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  int ccmaj = 0, ccmin = 0;
  cudaDeviceGetAttribute(&ccmaj, cudaDevAttrComputeCapabilityMajor, h->device);
  cudaDeviceGetAttribute(&ccmin, cudaDevAttrComputeCapabilityMinor, h->device);
  h->cc = 10 * ccmaj + ccmin;
  h->stream = (cudaStream_t)c.stream;
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    fs1_destroy(h);
    return FS1_ECUDA;
  }
  if (c.autotune) {
    if (const char* path = getenv("FS1_AUTOTUNE_CACHE")) {
      if (FILE* f = fopen(path, "r")) {
        char key[128];
        int t = 0;
        while (fscanf(f, "%127s %d", key, &t) == 2) h->tuned[key] = t;
        fclose(f);
      }
    }
  }
  *out = h;
  return FS1_OK;
}

void fs1_destroy(fs1_handle* h) {
  if (!h) return;
  if (h->ws || h->stage || h->hdr || h->hres) {
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->stage) cudaFree(h->stage);
    if (h->hdr) cudaFreeHost(h->hdr);
    if (h->hres) cudaFreeHost(h->hres);
  }
  drop_graphs(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

fs1_status fs1_handle_stats(const fs1_handle* h, int64_t* out) {
  if (!h || !out) return FS1_EINVAL;
  out[0] = h->replays;
  out[1] = h->captures;
  out[2] = (int64_t)h->tuned.size();
  out[3] = h->trial_launches;
  return FS1_OK;
}

fs1_status fs1_handle_launch_stats(const fs1_handle* h, int64_t* out) {
  if (!h || !out) return FS1_EINVAL;
  out[0] = h->exact_launches;
  out[1] = h->last_E;
  return FS1_OK;
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
    // the paper form solves 1D pairs of up to kMaxPaperN points (one CTA each)
    if (pst[i] == FS1_OK && kind == KK_PAPER_F64 && (probs[i].ndim != 1 || npoints(probs[i]) > kMaxPaperN))
      pst[i] = FS1_EUNSUPPORTED;
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
  // 1D pairs beyond the team kernel's on-chip capacity: the stabilised
  // variant solves them with the state in device memory after the launches
  // below (h / eps at most kStreamMaxC); the plain variants and larger h / eps
  // report FS1_EUNSUPPORTED for them
  std::vector<char> streamed(count, 0);
  if (kind != KK_PAPER_F64) {
    int maxc = -1;
    for (int64_t i = 0; i < count; ++i) {
      if (pst[i] != FS1_OK || staged[i].ndim != 1) continue;
      if (maxc < 0) maxc = max_coresident_ctas(kind);
      if (maxc <= 0) break;
      if (min_ctas(kind, staged[i]) > std::min(maxc, kMaxTeamCtas)) {
        if (kind == KK_LOG_F32 && staged[i].h[0] / staged[i].eps <= kStreamMaxC)
          streamed[i] = 1;
        else
          pst[i] = FS1_EUNSUPPORTED;
      }
    }
  }
  // group by kernel (1D or grid) and input dtype (a launch reads one dtype);
  // grid groups are cut into launches of at most kMaxImg2D grids
  std::vector<std::pair<std::vector<const fs1_problem*>, std::vector<int64_t>>> groups;
  for (int nd = 1; nd <= 2; ++nd)
    for (int dt = 0; dt < 2; ++dt) {
      std::vector<const fs1_problem*> grp;
      std::vector<int64_t> idx;
      for (int64_t i = 0; i < count; ++i)
        if (pst[i] == FS1_OK && !streamed[i] && staged[i].dtype == dt && (staged[i].ndim >= 2 ? 2 : 1) == nd) {
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
      team[idx[j]] = r[j].pad > 0 ? r[j].pad : geo.team_size;   // the 1D team or the image's cluster
      ms[idx[j]] = gms;
    }
  }
  {
    std::vector<const fs1_problem*> sp;
    std::vector<int64_t> si;
    for (int64_t i = 0; i < count; ++i)
      if (streamed[i]) {
        sp.push_back(&staged[i]);
        si.push_back(i);
      }
    if (!sp.empty()) {
      std::vector<PairResult> r;
      float sms = 0.f;
      const fs1_status s = run_stream_batch(h, sp, r, &sms);
      for (size_t k = 0; k < si.size(); ++k) {
        const int64_t i = si[k];
        if (s != FS1_OK) {
          pst[i] = s;
          continue;
        }
        res[i] = r[k];
        pst[i] = (fs1_status)r[k].status;
        team[i] = 0;
        ms[i] = sms;
      }
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

fs1_status fs1_test_missing_partner(fs1_handle* h, const double* a, const double* b, int64_t n, double hx,
                                    double eps, long long spin_cap, fs1_status* pair_status) {
  const int thr = team_threads();
  if (!h || !a || !b || !pair_status || n < 2 * thr || n > 2 * (int64_t)thr * team_elems_max(KK_LOG_F32) ||
      !(hx > 0.0) || !(eps > 0.0) || spin_cap < 1 || h->cfg.variant != FS1_VARIANT_LOG)
    return FS1_EINVAL;
  // workspace: descriptor | result | [2 parities][2 ranks] generic slots |
  // the same compact slots (one 128-byte line each) | counter | abort flag
  const size_t o_desc = 0, o_res = 256, o_slot = 512;
  const size_t o_cslot = o_slot + align_up(sizeof(Slot) * 4, 256);
  const size_t o_ctr = o_cslot + 128 * 4, o_abt = o_ctr + 256, bytes = o_abt + 256;
  fs1_status st;
  if ((st = ensure_ws(h, bytes)) != FS1_OK) return st;
  char* ws = (char*)h->ws;
  PairDesc d{};
  d.a = a;
  d.b = b;
  d.n = n;
  d.n_fast = n;
  d.n_mid = 1;
  d.n_slow = 1;
  d.h_fast = hx;
  d.eps = eps;
  d.tol = 0.0;
  d.itr_max = 1;
  const PairResult r0{NAN, NAN, 0, FS1_EINVAL, 0};
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, bytes, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ws + o_desc, &d, sizeof d, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ws + o_res, &r0, sizeof r0, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
    return cuda_fail(e, "missing-partner setup");
  TeamLaunch L{};
  L.pairs = (const PairDesc*)(ws + o_desc);
  L.results = (PairResult*)(ws + o_res);
  L.num_pairs = 1;
  L.team_size = 2;   // a team of two CTAs ...
  L.num_teams = 1;
  L.grid = 1;        // ... of which one is launched: its partner never publishes
  L.in_f32 = 0;
  L.slots = (Slot*)(ws + o_slot);
  L.cslots = (unsigned long long*)(ws + o_cslot);
  L.counters = (unsigned long long*)(ws + o_ctr);
  L.abort_flags = (int*)(ws + o_abt);
  L.spin_cap = spin_cap;
  const int ls = launch_team_1d(KK_LOG_F32, L, h->stream, 0);
  g_launches.fetch_add(1);
  if (ls != FS1_OK) return (fs1_status)ls;
  PairResult r;
  if ((e = cudaMemcpyAsync(&r, ws + o_res, sizeof r, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return cuda_fail(e, "missing-partner result");
  *pair_status = (fs1_status)r.status;
  return FS1_OK;
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

void fs1::note_launches(long long k) { g_launches.fetch_add(k); }
