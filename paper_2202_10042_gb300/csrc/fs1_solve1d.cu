// fs1_solve1d.cu -- host side of the 1D team kernel (fs1_team.cuh): the
// geometry helpers, the choice between the exact instantiation of a launch's
// point count per thread and the generic one, and the launch.
#include "fs1_team.cuh"

namespace fs1 {

int team_threads() { return kThreads; }

int team_elems_max(int kind) { return kind == KK_PLAIN_F64 ? 8 : 32; }

size_t team_smem_bytes(int kind) {
  const size_t vs = kind == KK_PLAIN_F64 ? sizeof(double) : sizeof(float);
  return 3 * vs * (size_t)team_elems_max(kind) * kThreads;
}

int elems_cap_for(int kind, double c) {
  const int emax = team_elems_max(kind);
  if (kind != KK_LOG_F32) return emax;
  // keep e^{c E} within the FP32 mantissa frame: c E <= 24 nats
  double cap = floor(24.0 / (c > 1e-30 ? c : 1e-30));
  if (cap < 1) cap = 1;
  return cap < emax ? (int)cap : emax;
}

// exact instantiations (fs1_team_exact_*.cu); each returns false when it
// holds no kernel for (kind, Eeff)
using ExactLaunch = bool (*)(int kind, int Eeff, const TeamLaunch& L, int mode, cudaStream_t st, cudaError_t& e);
bool launch_team_exact_e01_04(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e05_08(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e09_12(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e13_16(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e17_20(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e21_24(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e25_28(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_e29_32(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
bool launch_team_exact_plain(int, int, const TeamLaunch&, int, cudaStream_t, cudaError_t&);
static const ExactLaunch kExactLaunch[] = {
    launch_team_exact_e01_04, launch_team_exact_e05_08, launch_team_exact_e09_12, launch_team_exact_e13_16,
    launch_team_exact_e17_20, launch_team_exact_e21_24, launch_team_exact_e25_28, launch_team_exact_e29_32,
    launch_team_exact_plain};

bool team_exact_built(int kind, int E) {
  kind &= 0xff;
  return (kind == KK_LOG_F32 && E >= 1 && E <= 32) || (kind == KK_PLAIN_F64 && E >= 1 && E <= 8);
}

int launch_team_1d(int kind, const TeamLaunch& L, void* stream, int exact_E) {
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = (kind >> 8) & 0xff;
  kind &= 0xff;
  if (L.team_size > kMaxTeamCtas) return FS1_EINVAL;
  cudaError_t e = cudaSuccess;
  bool done = false;
  if (team_exact_built(kind, exact_E)) {
    for (ExactLaunch f : kExactLaunch)
      if (!done) done = f(kind, exact_E, L, mode, st, e);
    if (!done) {
      fprintf(stderr, "fs1: no exact team kernel for kind %d, E = %d\n", kind, exact_E);
      return FS1_ECUDA;
    }
  } else {
    switch (kind) {
      case KK_PLAIN_F64: e = launch_kind<double, double, 8, 2>(L, mode, st); break;
      case KK_PLAIN_F32: e = launch_kind<float, float, 32, 4>(L, mode, st); break;
      case KK_LOG_F32: e = launch_kind<float, XF, 32, 8>(L, mode, st); break;
      default: return FS1_EINVAL;
    }
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: team kernel launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

// CTAs of the generic instantiation that fit on the device at once: one per
// SM (its shared memory), and no instantiation fits fewer (each is bounded to
// one 512-thread CTA per SM's registers and an exact one holds E <= 32 points)
template <class V, class C, int E, int G>
static int coresident() {
  auto kfn = fs1_team_kernel<V, C, E, G>;
  const size_t smem = 3 * sizeof(V) * (size_t)E * kThreads;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

int max_coresident_ctas(int kind) {
  switch (kind & 0xff) {
    case KK_PLAIN_F64: return coresident<double, double, 8, 2>();
    case KK_PLAIN_F32: return coresident<float, float, 32, 4>();
    case KK_LOG_F32: return coresident<float, XF, 32, 8>();
  }
  return 0;
}

}  // namespace fs1
