// Instantiation of the cluster-resident 2D solver (fs1_cluster2d.cuh): rows of
// up to 128 points (4 per lane), up to 8 rows per CTA.
#include "fs1_cluster2d.cuh"

namespace fs1 {

int c2d_max_clusters_p4r8(int cs) { return c2d::max_clusters<4, 8>(cs); }

cudaError_t c2d_launch_p4r8(const c2d::Launch& L, int cs, int clusters, cudaStream_t st) {
  return c2d::launch<4, 8>(L, cs, clusters, st);
}

}  // namespace fs1
