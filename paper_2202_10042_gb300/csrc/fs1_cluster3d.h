// fs1_cluster3d.h -- host entry points of the cluster-resident 3D solver
// (fs1_cluster3d.cu).  Not part of the public C-ABI (include/fs1.h).
#pragma once
#include <cstddef>

#include "fs1_internal.h"

namespace fs1 {

// A 3D grid of at most 64 points on the fast and middle axes (and c = h / eps
// <= 8 on every axis of more than one point) in the shared memory of one
// cluster of 8 to 16 CTAs.  launch_cluster_3d solves d[0 .. count), all with
// cluster3d_ok; results[i].w is left NaN, results[i].pad holds the cluster's
// CTAs, and cost[i] (host) receives the descriptor of a grid-kernel launch of
// no iterations, warm-started from the final iterate, whose result is that
// iterate's cost.  A grid whose scalings leave the kernel's exponent range
// ends with FS1_EUNSUPPORTED (the caller solves it again with the grid kernel).
int cluster3d_ok(const PairDesc& d);
size_t cluster3d_workspace(const PairDesc* d, int count);
int launch_cluster_3d(const PairDesc* d, int count, int in_f32, PairResult* results, void* ws, size_t ws_bytes,
                      void* stream, long long* launches, PairDesc* cost);

}  // namespace fs1
