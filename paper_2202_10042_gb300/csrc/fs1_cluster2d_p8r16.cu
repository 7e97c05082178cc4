// Instantiation of the cluster-resident 2D solver (fs1_cluster2d.cuh): rows of
// up to 256 points (8 per lane), up to 16 rows per CTA.
#include "fs1_cluster2d.cuh"

namespace fs1 {

int c2d_max_clusters_p8r16(int cs) { return c2d::max_clusters<8, 16>(cs); }

cudaError_t c2d_launch_p8r16(const c2d::Launch& L, int cs, int clusters, cudaStream_t st) {
  return c2d::launch<8, 16>(L, cs, clusters, st);
}

}  // namespace fs1
