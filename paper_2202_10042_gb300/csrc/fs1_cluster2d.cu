// fs1_cluster2d.cu -- host side of the cluster-resident 2D solver
// (fs1_cluster2d.cuh): which images it takes, its workspace, its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "fs1_cluster2d.cuh"

namespace fs1 {

int c2d_max_clusters_p4r8(int cs);
int c2d_max_clusters_p8r16(int cs);
int c2d_max_clusters_p16r32(int cs);
cudaError_t c2d_launch_p4r8(const c2d::Launch& L, int cs, int clusters, cudaStream_t st);
cudaError_t c2d_launch_p8r16(const c2d::Launch& L, int cs, int clusters, cudaStream_t st);
cudaError_t c2d_launch_p16r32(const c2d::Launch& L, int cs, int clusters, cudaStream_t st);

namespace {

struct Inst {
  int PF, RS;
  int (*clusters)(int cs);
  cudaError_t (*launch)(const c2d::Launch&, int cs, int clusters, cudaStream_t);
};
// smallest first: an image takes the first instantiation that holds it
const Inst kInst[] = {{4, 8, c2d_max_clusters_p4r8, c2d_launch_p4r8},
                      {8, 16, c2d_max_clusters_p8r16, c2d_launch_p8r16},
                      {16, 32, c2d_max_clusters_p16r32, c2d_launch_p16r32}};
constexpr int kNInst = 3;

// Per instantiation and device (queried once): how many clusters of each
// size fit at once (the sizes that fit depend on how the SMs are grouped).
constexpr int kMaxDev = 64;
constexpr int kMinCS = 8;
int g_fit[kMaxDev][kNInst][c2d::kMaxCS + 1];
bool g_known[kMaxDev];

int clusters_of(int k, int cs) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
  if (!g_known[dev]) {
    for (int i = 0; i < kNInst; ++i)
      for (int c = 0; c <= c2d::kMaxCS; ++c) g_fit[dev][i][c] = c >= kMinCS ? kInst[i].clusters(c) : 0;
    g_known[dev] = true;
  }
  return g_fit[dev][k][cs];
}

// The launch shape of an image: the first instantiation whose rows hold its
// row length, and the cluster size that puts the most SMs to work (clusters
// that fit at once x CTAs per cluster) while every CTA's rows fit the
// instantiation.  (k, cs) = (-1, 0) when none does.
struct Shape {
  int k, cs;
};
Shape shape_of(const PairDesc& d) {
  for (int k = 0; k < kNInst; ++k) {
    if (32 * kInst[k].PF < d.n_fast) continue;
    Shape best{-1, 0};
    int cover = 0;
    for (int cs = c2d::kMaxCS; cs >= kMinCS; --cs) {
      if ((d.n_slow + cs - 1) / cs > kInst[k].RS) continue;
      const int n = clusters_of(k, cs);
      if (n > 0 && n * cs > cover) {
        cover = n * cs;
        best = Shape{k, cs};
      }
    }
    if (best.k >= 0) return best;
  }
  return Shape{-1, 0};
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

size_t slots(const PairDesc& d, int k) { return (size_t)d.n_slow * 32 * kInst[k].PF; }
// frames of the saved u: [cluster size][RS / kSub][SW]
size_t frames(Shape sh) { return (size_t)sh.cs * (kInst[sh.k].RS / c2d::kSub) * 32 * kInst[sh.k].PF; }

}  // namespace

int cluster2d_inst(const PairDesc& d) {
  if (d.n_mid != 1 || d.n_fast < 1 || d.n_slow < 1) return -1;
  // FP32-frame sweeps on both axes (larger c: the grid kernel); an axis of
  // one point has no recurrence, so its c does not matter
  if (d.n_fast > 1 && !(d.h_fast / d.eps <= c2d::kFrameC)) return -1;
  if (d.n_slow > 1 && !(d.h_slow / d.eps <= c2d::kFrameC)) return -1;
  return shape_of(d).k;
}

size_t cluster2d_workspace(const PairDesc* d, int count) {
  size_t b = al(sizeof(c2d::Img) * count) + al(sizeof(int) * count) + al(sizeof(int) * kNInst * (c2d::kMaxCS + 1));
  for (int i = 0; i < count; ++i) {
    const int k = cluster2d_inst(d[i]);
    if (k >= 0) b += 3 * al(sizeof(float) * slots(d[i], k)) + al(sizeof(int) * frames(shape_of(d[i])));
  }
  return b;
}

// Solve d[0 .. count) with the cluster kernel; every image must have
// cluster2d_inst >= 0.  results: device array of count entries.
int launch_cluster_2d(const PairDesc* d, int count, int in_f32, PairResult* results, const int* d_valid,
                      void* ws, size_t ws_bytes, void* stream, long long* launches) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count < 1) return FS1_OK;
  if (cluster2d_workspace(d, count) > ws_bytes) return FS1_ENOMEM;
  char* p = (char*)ws;
  c2d::Img* d_imgs = (c2d::Img*)p;
  p += al(sizeof(c2d::Img) * count);
  int* d_order = (int*)p;
  p += al(sizeof(int) * count);
  int* d_next = (int*)p;
  p += al(sizeof(int) * kNInst * (c2d::kMaxCS + 1));
  std::vector<c2d::Img> imgs(count);
  std::vector<int> group(count);   // k (kMaxCS + 1) + cs
  for (int i = 0; i < count; ++i) {
    const PairDesc& D = d[i];
    if (cluster2d_inst(D) < 0) return FS1_EINVAL;
    const Shape sh = shape_of(D);
    const int k = sh.k;
    group[i] = k * (c2d::kMaxCS + 1) + sh.cs;
    c2d::Img I{};
    I.a = D.a;
    I.b = D.b;
    I.nf = (int)D.n_fast;
    I.ns = (int)D.n_slow;
    I.R = (int)((D.n_slow + sh.cs - 1) / sh.cs);
    I.cf = D.h_fast / D.eps;
    I.cs = D.h_slow / D.eps;
    I.hf = D.h_fast;
    I.hs = D.h_slow;
    I.tol = D.tol;
    I.itr_max = D.itr_max;
    I.f_init = D.f_init;
    I.g_init = D.g_init;
    I.f_out = D.f_out;
    I.g_out = D.g_out;
    const size_t n = slots(D, k);
    I.aw = (float*)p; p += al(sizeof(float) * n);
    I.bw = (float*)p; p += al(sizeof(float) * n);
    I.us = (float*)p; p += al(sizeof(float) * n);
    I.usf = (int*)p; p += al(sizeof(int) * frames(sh));
    imgs[i] = I;
  }
  // one queue per (instantiation, cluster size), longest (points x cap) first
  const int ng = kNInst * (c2d::kMaxCS + 1);
  std::vector<int> order;
  std::vector<int> first(ng + 1, 0);
  for (int g = 0; g < ng; ++g) {
    first[g] = (int)order.size();
    std::vector<int> mine;
    for (int i = 0; i < count; ++i)
      if (group[i] == g) mine.push_back(i);
    std::stable_sort(mine.begin(), mine.end(), [&](int x, int y) {
      return (double)d[x].n * (double)d[x].itr_max > (double)d[y].n * (double)d[y].itr_max;
    });
    order.insert(order.end(), mine.begin(), mine.end());
  }
  first[ng] = (int)order.size();
  cudaError_t e = cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(c2d::Img) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, sizeof(int) * ng, st);
  for (int g = 0; g < ng && e == cudaSuccess; ++g) {
    const int n = first[g + 1] - first[g];
    if (n == 0) continue;
    const int k = g / (c2d::kMaxCS + 1), cs = g % (c2d::kMaxCS + 1);
    c2d::Launch L{d_imgs, results, d_order + first[g], n, in_f32, d_valid, d_next + g};
    e = kInst[k].launch(L, cs, std::min(n, clusters_of(k, cs)), st);
    if (launches) ++*launches;
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: cluster 2D launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

}  // namespace fs1
