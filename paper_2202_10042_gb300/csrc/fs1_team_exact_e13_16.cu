// Exact instantiations of the team kernel (fs1_team.cuh): stabilised FP32,
// E = G = 13, 14, 15, 16 points per thread.
#include "fs1_team.cuh"

namespace fs1 {

bool launch_team_exact_e13_16(int kind, int Eeff, const TeamLaunch& L, int mode, cudaStream_t st, cudaError_t& e) {
  return kind == KK_LOG_F32 && launch_exact_in<float, XF, 13, 14, 15, 16>(Eeff, L, mode, st, e);
}

}  // namespace fs1
