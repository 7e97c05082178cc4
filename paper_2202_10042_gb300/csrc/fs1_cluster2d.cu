// fs1_cluster2d.cu -- host side of the cluster-resident 2D solver
// (fs1_cluster2d.cuh): which images it takes, its workspace, its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "fs1_cluster2d.cuh"

namespace fs1 {

int c2d_max_clusters_p4r8();
int c2d_max_clusters_p8r16();
int c2d_max_clusters_p16r32();
cudaError_t c2d_launch_p4r8(const c2d::Launch& L, int clusters, cudaStream_t st);
cudaError_t c2d_launch_p8r16(const c2d::Launch& L, int clusters, cudaStream_t st);
cudaError_t c2d_launch_p16r32(const c2d::Launch& L, int clusters, cudaStream_t st);

namespace {

struct Inst {
  int PF, RS;
  int (*clusters)();
  cudaError_t (*launch)(const c2d::Launch&, int, cudaStream_t);
};
// smallest first: an image takes the first instantiation that holds it
const Inst kInst[] = {{4, 8, c2d_max_clusters_p4r8, c2d_launch_p4r8},
                      {8, 16, c2d_max_clusters_p8r16, c2d_launch_p8r16},
                      {16, 32, c2d_max_clusters_p16r32, c2d_launch_p16r32}};
constexpr int kNInst = 3;

// co-resident clusters per instantiation on each device (queried once)
constexpr int kMaxDev = 64;
int g_clusters[kMaxDev][kNInst];
bool g_known[kMaxDev];

int clusters_of(int k) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
  if (!g_known[dev]) {
    for (int i = 0; i < kNInst; ++i) g_clusters[dev][i] = kInst[i].clusters();
    g_known[dev] = true;
  }
  return g_clusters[dev][k];
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

size_t slots(const PairDesc& d, int k) { return (size_t)d.n_slow * 32 * kInst[k].PF; }

}  // namespace

int cluster2d_inst(const PairDesc& d) {
  if (d.n_mid != 1 || d.n_fast < 1 || d.n_slow < 1) return -1;
  const int64_t R = (d.n_slow + c2d::kCS - 1) / c2d::kCS;
  for (int k = 0; k < kNInst; ++k)
    if (32 * kInst[k].PF >= d.n_fast && kInst[k].RS >= R) return clusters_of(k) > 0 ? k : -1;
  return -1;
}

size_t cluster2d_workspace(const PairDesc* d, int count) {
  size_t b = al(sizeof(c2d::Img) * count) + al(sizeof(int) * count) + al(sizeof(int) * kNInst);
  for (int i = 0; i < count; ++i) {
    const int k = cluster2d_inst(d[i]);
    if (k >= 0) b += 2 * al(sizeof(float) * slots(d[i], k)) + al(sizeof(float) * slots(d[i], k)) +
                     al(sizeof(short) * slots(d[i], k));
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
  p += al(sizeof(int) * kNInst);
  std::vector<c2d::Img> imgs(count);
  std::vector<int> inst(count);
  for (int i = 0; i < count; ++i) {
    const PairDesc& D = d[i];
    const int k = cluster2d_inst(D);
    if (k < 0) return FS1_EINVAL;
    inst[i] = k;
    c2d::Img I{};
    I.a = D.a;
    I.b = D.b;
    I.nf = (int)D.n_fast;
    I.ns = (int)D.n_slow;
    I.R = (int)((D.n_slow + c2d::kCS - 1) / c2d::kCS);
    I.cf = D.h_fast / D.eps;
    I.cs = D.h_slow / D.eps;
    I.frame_f = I.cf <= c2d::kFrameC ? 1 : 0;
    I.frame_s = I.cs <= c2d::kFrameC ? 1 : 0;
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
    I.usm = (float*)p; p += al(sizeof(float) * n);
    I.use = (short*)p; p += al(sizeof(short) * n);
    imgs[i] = I;
  }
  // one queue per instantiation, longest (points x cap) first
  std::vector<int> order;
  std::vector<int> first(kNInst + 1, 0);
  for (int k = 0; k < kNInst; ++k) {
    first[k] = (int)order.size();
    std::vector<int> mine;
    for (int i = 0; i < count; ++i)
      if (inst[i] == k) mine.push_back(i);
    std::stable_sort(mine.begin(), mine.end(), [&](int x, int y) {
      return (double)d[x].n * (double)d[x].itr_max > (double)d[y].n * (double)d[y].itr_max;
    });
    order.insert(order.end(), mine.begin(), mine.end());
  }
  first[kNInst] = (int)order.size();
  cudaError_t e = cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(c2d::Img) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, sizeof(int) * kNInst, st);
  for (int k = 0; k < kNInst && e == cudaSuccess; ++k) {
    const int n = first[k + 1] - first[k];
    if (n == 0) continue;
    c2d::Launch L{d_imgs, results, d_order + first[k], n, in_f32, d_valid, d_next + k};
    e = kInst[k].launch(L, std::min(n, clusters_of(k)), st);
    if (launches) ++*launches;
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: cluster 2D launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

}  // namespace fs1
