// fs1_noalloc.cu -- fs1_w1_noalloc: a one-problem solve that allocates nothing.
//
// Some callers cannot call cudaMalloc: a process whose memory manager has
// already reserved the device's memory for itself, an embedding that forbids
// the library from owning device memory, or a latency-critical path that must
// not pay for an allocation (which may synchronise the device).  For them this
// entry point runs the same 1D team kernel as fs1_w1, but every byte of device
// scratch it needs (the pair descriptor, the result record, the mass-check
// partials, the two sets of team exchange slots, the counter and the abort flag)
// lives in one file-scope __device__ array of fixed size.  The caller passes
// device-resident inputs and host outputs; nothing is allocated on the device
// or the host.
//
// Notes for users
//   - The array (kScratchBytes, about 84 KiB) is part of the library image:
//     every GPU that loads the library holds it until the process exits.
//   - Host code may not use the array's name as a device address (on the host
//     it names a host-side stand-in).  Every call, with the problem's device
//     current, looks the device address up with cudaGetSymbolAddress (which
//     allocates nothing), so the address stays right across a device reset
//     that reloads the library's module at another address.
//   - The call is synchronous: it synchronises its stream twice (after the
//     mass check and after the solve), so it may not be called on a stream
//     that is being captured.
//   - Every call shares the one array and finds the previous call's contents:
//     the counter, the abort flag and the exchange slots are cleared at the
//     start of each call.  Calls that overlap on the GPU (two host threads, or
//     two streams) race on the array; serialise them.
//   - Problems whose team would exceed kMaxTeam CTAs are rejected with
//     FS1_EINVAL and a message on stderr; pairs beyond the on-chip capacity
//     (no co-resident team holds them) with FS1_EUNSUPPORTED.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "fs1.h"
#include "fs1_internal.h"

namespace fs1 {
namespace {

constexpr int kMaxTeam = 160;          // CTAs per team the static scratch can serve

struct NaValOut {
  double sa, sb;
  int bad;
  int pad;
};

constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffRes = kOffDesc + al(sizeof(PairDesc));
constexpr size_t kOffCtr = kOffRes + al(sizeof(PairResult));
constexpr size_t kOffAbort = kOffCtr + al(sizeof(unsigned long long));
constexpr size_t kOffSlots = kOffAbort + al(sizeof(int));
constexpr size_t kOffCSlots = kOffSlots + al(sizeof(Slot) * 2 * (size_t)kMaxTeam);
constexpr int kCheckBlocks = 128;      // CTAs of the mass check, one partial each
constexpr size_t kOffVal = kOffCSlots + al(128 * 2 * (size_t)kMaxTeam);
constexpr size_t kScratchBytes = kOffVal + al(sizeof(NaValOut) * (size_t)kCheckBlocks);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of g_scratch on the current device.  Looked up on every call:
// cudaGetSymbolAddress allocates nothing, and a cached address would go stale
// if a device reset reloaded the module elsewhere.
fs1_status scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || p == nullptr) {
    fprintf(stderr, "fs1_w1_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  *out = p;
  return FS1_OK;
}

// Input check of the pair: CTA k sums a and b over a grid-stride share of the
// points and flags negative or non-finite entries; its partial goes to out[k]
// and the host adds the partials in CTA order.
__global__ void noalloc_mass_check(const PairDesc* pd, int in_f32, NaValOut* out) {
  const PairDesc P = *pd;
  double sa = 0.0, sb = 0.0;
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    const double va = in_f32 ? (double)((const float*)P.a)[i] : ((const double*)P.a)[i];
    const double vb = in_f32 ? (double)((const float*)P.b)[i] : ((const double*)P.b)[i];
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
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += ssa[w];
      tb += ssb[w];
    }
    out[blockIdx.x] = NaValOut{ta, tb, sbad, 0};
  }
}

}  // namespace
}  // namespace fs1

using namespace fs1;

extern "C" fs1_status fs1_w1_noalloc(const fs1_config* cfg_in, const fs1_problem* prob, double* w1_out,
                                     fs1_info* info_out) {
  if (!prob) return FS1_EINVAL;
  fs1_config cfg;
  if (cfg_in) cfg = *cfg_in; else fs1_config_default(&cfg);
  const fs1_problem& p = *prob;
  if (cfg.variant == FS1_VARIANT_PAPER) return FS1_EUNSUPPORTED;   // the team kernel only
  if (cfg.variant != FS1_VARIANT_PLAIN && cfg.variant != FS1_VARIANT_LOG) return FS1_EINVAL;
  if (cfg.variant == FS1_VARIANT_LOG && cfg.precision != FS1_FP32) return FS1_EUNSUPPORTED;
  if (cfg.check_every != 1) return FS1_EUNSUPPORTED;
  if (p.ndim != 1 || p.location != FS1_MEM_DEVICE) return FS1_EINVAL;   // no staging here
  if (p.dtype != FS1_FP64 && p.dtype != FS1_FP32) return FS1_EINVAL;
  if (p.n[0] < 1 || !(p.h[0] > 0.0) || !std::isfinite(p.h[0]) || !(p.eps > 0.0) ||
      !std::isfinite(p.eps) || !(p.tol >= 0.0) || p.itr_max < 0 || !p.a || !p.b)
    return FS1_EINVAL;
  if ((p.f_init == nullptr) != (p.g_init == nullptr)) return FS1_EINVAL;
  const long long spin_cap = cfg.spin_cap > 0 ? cfg.spin_cap : (1ll << 22);
  const int kind = cfg.variant == FS1_VARIANT_PLAIN ? (cfg.precision == FS1_FP64 ? KK_PLAIN_F64 : KK_PLAIN_F32)
                                                    : KK_LOG_F32;

  // team size: the fewest CTAs that hold the pair on chip, spread up to the
  // co-resident limit, as the batched path does for a single problem
  const int thr = team_threads();
  const int maxc = max_coresident_ctas(kind);
  if (maxc <= 0) return FS1_ECUDA;
  const int64_t n = p.n[0];
  const int64_t cap = elems_cap_for(kind, p.h[0] / p.eps);
  const int64_t tmin = (n + thr * cap - 1) / (thr * cap);
  const int64_t tuse = std::min<int64_t>({(n + thr - 1) / thr, (int64_t)maxc, (int64_t)kMaxTeam});
  if (tmin > maxc) return FS1_EUNSUPPORTED;
  const int64_t T = cfg.team_size > 0 ? std::max<int64_t>(tmin, cfg.team_size) : std::max<int64_t>(tmin, tuse);
  if (T > maxc) return FS1_EINVAL;
  if (T > kMaxTeam) {
    fprintf(stderr, "fs1_w1_noalloc: the problem needs a team of %lld CTAs; the static scratch serves "
            "at most %d\n", (long long)T, kMaxTeam);
    return FS1_EINVAL;
  }

  void* base = nullptr;
  fs1_status st = scratch_address(&base);
  if (st != FS1_OK) return st;
  char* sc = (char*)base;
  cudaStream_t stream = (cudaStream_t)cfg.stream;

  PairDesc d{};
  d.a = p.a;
  d.b = p.b;
  d.n = n;
  d.n_fast = n;
  d.n_mid = 1;
  d.n_slow = 1;
  d.h_fast = p.h[0];
  d.h_slow = 0.0;
  d.eps = p.eps;
  d.tol = p.tol;
  d.itr_max = p.itr_max;
  d.f_out = p.f_out;
  d.g_out = p.g_out;
  d.f_init = p.f_init;
  d.g_init = p.g_init;
  PairResult r0{NAN, NAN, 0, FS1_ETIMEOUT, 0};
  cudaError_t e;
  if ((e = cudaMemcpyAsync(sc + kOffDesc, &d, sizeof d, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(sc + kOffRes, &r0, sizeof r0, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc + kOffCtr, 0, sizeof(unsigned long long), stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc + kOffAbort, 0, sizeof(int), stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc + kOffSlots, 0, sizeof(Slot) * 2 * (size_t)T, stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc + kOffCSlots, 0, 128 * 2 * (size_t)T, stream)) != cudaSuccess) {
    fprintf(stderr, "fs1_w1_noalloc: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  const int in_f32 = p.dtype == FS1_FP32;
  const int nblk = (int)std::min<int64_t>(kCheckBlocks, (n + 255) / 256);
  noalloc_mass_check<<<nblk, 256, 0, stream>>>((const PairDesc*)(sc + kOffDesc), in_f32,
                                               (NaValOut*)(sc + kOffVal));
  note_launches(1);
  NaValOut part[kCheckBlocks];
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(part, sc + kOffVal, sizeof(NaValOut) * nblk, cudaMemcpyDeviceToHost, stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess) {
    fprintf(stderr, "fs1_w1_noalloc: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  NaValOut vo{0.0, 0.0, 0, 0};
  for (int k = 0; k < nblk; ++k) {
    vo.sa += part[k].sa;
    vo.sb += part[k].sb;
    vo.bad |= part[k].bad;
  }
  fs1_info info;
  memset(&info, 0, sizeof info);
  info.variant = cfg.variant;
  info.precision = cfg.precision;
  info.team_size = (int)T;
  if (vo.bad || !(vo.sa > 0.0) || !(vo.sb > 0.0) || std::fabs(vo.sa - vo.sb) > 1e-6 * std::max(vo.sa, vo.sb)) {
    info.status = FS1_EINVAL;
    info.w1 = NAN;
    info.marginal_err = NAN;
    if (w1_out) *w1_out = NAN;
    if (info_out) *info_out = info;
    return FS1_EINVAL;
  }

  TeamLaunch L{};
  L.pairs = (const PairDesc*)(sc + kOffDesc);
  L.results = (PairResult*)(sc + kOffRes);
  L.order = nullptr;
  L.num_pairs = 1;
  L.team_size = (int)T;
  L.num_teams = 1;
  L.in_f32 = in_f32;
  L.slots = (Slot*)(sc + kOffSlots);
  L.cslots = (unsigned long long*)(sc + kOffCSlots);
  L.counters = (unsigned long long*)(sc + kOffCtr);
  L.abort_flags = (int*)(sc + kOffAbort);
  L.spin_cap = spin_cap;
  const int ls = launch_team_1d(kind, L, stream, (int)((n + thr * T - 1) / (thr * T)));
  if (ls != FS1_OK) return (fs1_status)ls;
  note_launches(1);
  PairResult r;
  if ((e = cudaMemcpyAsync(&r, sc + kOffRes, sizeof r, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess) {
    fprintf(stderr, "fs1_w1_noalloc: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  info.status = r.status;
  info.iters = r.iters;
  info.marginal_err = r.err;
  info.w1 = r.w;
  if (w1_out) *w1_out = r.w;
  if (info_out) *info_out = info;
  return (fs1_status)r.status;
}
