// Instantiation of the cluster-resident 2D solver (fs1_cluster2d.cuh): rows of
// up to 512 points (16 per lane), up to 32 rows per CTA.
#include "fs1_cluster2d.cuh"

namespace fs1 {

int c2d_max_clusters_p16r32(int cs) { return c2d::max_clusters<16, 32>(cs); }

cudaError_t c2d_launch_p16r32(const c2d::Launch& L, int cs, int clusters, cudaStream_t st) {
  return c2d::launch<16, 32>(L, cs, clusters, st);
}

}  // namespace fs1
