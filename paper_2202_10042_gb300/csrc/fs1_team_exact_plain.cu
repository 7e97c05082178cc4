// Exact instantiations of the team kernel (fs1_team.cuh) for the plain form:
// FP64 with E = G = 1 .. 8 points per thread.
#include "fs1_team.cuh"

namespace fs1 {

bool launch_team_exact_plain(int kind, int Eeff, const TeamLaunch& L, int mode, cudaStream_t st, cudaError_t& e) {
  return kind == KK_PLAIN_F64 && launch_exact_in<double, double, 1, 2, 3, 4, 5, 6, 7, 8>(Eeff, L, mode, st, e);
}

}  // namespace fs1
