// fs1_cluster3d.cu -- 3D FS-1 (the separable extension in the closing remark
// of Section 4: K = K_slow (x) K_mid (x) K_fast, the 1D recurrences of eq.
// "recursion" along every line of each axis) with the grid resident in the
// distributed shared memory of one thread-block cluster, and its host side.
//
// One cluster of S CTAs owns one grid at a time and keeps u, v in shared
// memory for the whole solve.  CTA k holds the slow planes [k R, k R + R),
// R = ceil(n_slow / S) <= 8; a plane is NM rows (the middle axis, padded with
// zero rows to a multiple of 8) of SW = 64 slots (the fast axis, point j in
// slot j).  One application of K is three passes:
//   fast pass : 8 lanes per row, 8 points per lane (4 rows per warp at once):
//               the lane's (decay, value) aggregates, a 3-level Kogge-Stone
//               scan within the row's 8 lanes, the sweeps in one FP32 frame
//               per lane;
//   mid pass  : thread (plane, slot) scans the plane's middle line in blocks
//               of 8 rows (block aggregates, the carries between blocks, then
//               the sweeps), in place; no other CTA is involved;
//   slow pass : every (row, slot) line over the CTA's planes; phase A
//               publishes its aggregates in shared memory; after a cluster
//               barrier each CTA takes 1/S of the lines and, for each, reads
//               every CTA's aggregate (distributed shared memory), forms the
//               prefix (forward) and suffix (backward) over the CTAs (Horner
//               with lam^R per CTA) and writes each CTA its two carries in
//               place of its aggregates; after a second barrier phase B reads
//               its carries locally and runs the sweeps.
// State: FP32 values in power-of-two frames as in the 2D kernel (c = h / eps
// <= 8 on every axis, so a block of 8 consecutive outputs spans at most e^64):
// u and v keep one frame per slow line (row, slot) over the CTA's planes, the
// fast pass's output one per (row, lane), the mid pass's output one per
// (plane, block of 8 rows, slot).  The slow pass's aggregates are published as
// an FP32 mantissa and a 16-bit exponent (12 bytes a line instead of 16, so
// that a 64^3 grid fits 16 CTAs).  a and b are read from a padded copy that
// stays in L2.  Two state buffers alternate between u and v: the v-half's
// slow pass writes v_new = b / y over the values of u it has consumed, and
// the buffers swap when the iteration goes on (at the stop v^l is kept).
//
// One iteration of Algorithm 2 is the 2D kernel's: the v-half forms
// y = K^T u, the error terms |v y - b| and their cluster sum (FP64, one fixed
// order), then v = b / y unless the iteration stops; the u-half forms
// u = a / (K v).  At the stop u^l is rebuilt by the same u-half from v^l.
// The transport cost is not formed here: the distance-weighted passes of
// three axes need more shared memory than the state leaves.  The kernel writes
// the final log potentials, and the host has the grid kernel (fs1_solve2d.cu)
// evaluate the cost of exactly that iterate in a warm-started launch of no
// iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "fs1_cluster2d.cuh"
#include "fs1_cluster3d.h"

namespace fs1 {
namespace c3d {

using c2d::cluster_rank;
using c2d::cluster_size;
using c2d::cluster_sync;
using c2d::dsm_addr;
using c2d::dsm_ld_f2;
using c2d::dsm_ld_s32;
using c2d::fr16;
using c2d::gather_frame;
using c2d::from_log;
using c2d::kF16Zero;
using c2d::kFrameC;
using c2d::kHead;
using c2d::kSub;
using c2d::kThr;
using c2d::kWarps;
using c2d::load_in;
using c2d::Tabs;
using c2d::to16;
using c2d::to_block;
using c2d::to_log;

constexpr int kLP = 8;              // fast-axis points per lane (8 lanes per row)
constexpr int kSW = 64;             // slots of a row (fast axis at most 64 points)
constexpr int kMaxNM = 64;          // middle axis at most 64 points
constexpr int kMaxNMB = kMaxNM / kSub;
constexpr int kMaxR = kSub;         // planes per CTA: one frame block along the slow axis
                                    // (kernels for at most 4 and at most 8 planes)
constexpr int kMinCS = 8;
constexpr int kMaxCS = 16;

struct Img {
  const void* a;
  const void* b;
  int nf, nm, ns;        // fast, middle, slow lengths
  int NM;                // rows of a plane: nm rounded up to a multiple of 8
  int R;                 // planes per CTA
  double cf, cm, cs;     // h / eps per axis
  double tol;
  int64_t itr_max;
  const double* f_init;  // optional warm start (log u, log v), row major
  const double* g_init;
  double* f_out;         // final log u, log v (always written: the cost launch reads them)
  double* g_out;
  float* aw;             // [ns][NM][SW] a, b, rows padded (workspace)
  float* bw;
};

struct Launch {
  const Img* imgs;
  PairResult* results;
  const int* order;
  int nimg;
  int in_f32;
  int* next;             // work-queue head (zeroed per launch)
};

// shared memory of a CTA holding R planes of NM rows (dynamic part): two
// state buffers, the published aggregates (mantissas, exponents), the two
// buffers' line frames, the mid pass's block frames, the fast pass's lane frames
__host__ __device__ constexpr size_t plane_values(int R, int NM) { return (size_t)R * NM * kSW; }
__host__ __device__ constexpr size_t smem_bytes(int R, int NM) {
  return 4 * (2 * plane_values(R, NM) + 2 * (size_t)NM * kSW) +
         2 * (4 * (size_t)NM * kSW + (size_t)R * (NM / kSub) * kSW + (size_t)R * NM * (kSW / kLP));
}
// largest dynamic shared memory the kernel asks for (the static part is < 1 KB)
constexpr size_t kSmemCap = 227 * 1024 - 1024;

__device__ __forceinline__ float dsm_ld_f32(unsigned a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ short dsm_ld_s16(unsigned a) {
  short v;
  asm volatile("ld.shared::cluster.s16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void dsm_st_f32(unsigned a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void dsm_st_s16(unsigned a, short v) {
  asm volatile("st.shared::cluster.b16 [%0], %1;" ::"r"(a), "h"(v) : "memory");
}
// shuffles within segments of 8 lanes (one row of the fast pass)
__device__ __forceinline__ XF shfl_up8(XF a, int o) {
  return XF{__shfl_up_sync(0xffffffffu, a.m, o, 8), __shfl_up_sync(0xffffffffu, a.e, o, 8)};
}
__device__ __forceinline__ XF shfl_down8(XF a, int o) {
  return XF{__shfl_down_sync(0xffffffffu, a.m, o, 8), __shfl_down_sync(0xffffffffu, a.e, o, 8)};
}

// ---------------------------------------------------------------------------
// fast pass: lane ls (0..7) of a row holds its points 8 ls .. 8 ls + 7.  Input
// values xi (the row's, at slot 8 ls) with the line frames fi of the input
// buffer; output values xo in [0, 1] of the frame returned (one per lane).
// Every lane of the warp calls (the scan shuffles within 8-lane segments).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fast_lane(const float* xi, const short* fi, float* xo, int ls, const Tabs& T) {
  const float4 v0 = *reinterpret_cast<const float4*>(xi);
  const float4 v1 = *reinterpret_cast<const float4*>(xi + 4);
  const uint4 fw = *reinterpret_cast<const uint4*>(fi);
  float x[kLP] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  const unsigned w4[4] = {fw.x, fw.y, fw.z, fw.w};
  int f[kLP];
#pragma unroll
  for (int k = 0; k < kLP; ++k) f[k] = fr16((short)(w4[k / 2] >> (16 * (k & 1))));
  const int fe = gather_frame(x, f);
  const float lam = T.lamf;
  float rr = 0.f, qq = 0.f;
#pragma unroll
  for (int k = 0; k < kLP; ++k) rr = fmaf(lam, rr, x[k]);
#pragma unroll
  for (int k = kLP - 1; k >= 0; --k) qq = lam * (qq + x[k]);
  // Kogge-Stone over the row's 8 lanes (span 8 2^lv points)
  XF xs = xf_norm(rr, fe), zs = xf_norm(qq, fe);
#pragma unroll
  for (int lv = 0; lv < 3; ++lv) {
    const int o = 1 << lv;
    const XF y = shfl_up8(xs, o), w = shfl_down8(zs, o);
    if (ls >= o) xs = c_add(c_mul(y, T.ks[lv]), xs);
    if (ls + o < 8) zs = c_add(zs, c_mul(w, T.ks[lv]));
  }
  XF C = shfl_up8(xs, 1), D = shfl_down8(zs, 1);
  if (ls == 0) C = XF{0.f, kZeroExp};
  if (ls == 7) D = XF{0.f, kZeroExp};
  const int F = max(fe, max(C.e, D.e)) + kHead;
  const float sc = pow2f(fe - F);
  float tb[kLP];
  float sb = c_to(D, F);
#pragma unroll
  for (int k = kLP - 1; k >= 0; --k) {
    tb[k] = sb;
    sb = lam * fmaf(x[k], sc, sb);
  }
  float p = c_to(C, F);
  float o[kLP];
#pragma unroll
  for (int k = 0; k < kLP; ++k) {
    p = fmaf(lam, p, x[k] * sc);
    o[k] = p + tb[k];
  }
  *reinterpret_cast<float4*>(xo) = make_float4(o[0], o[1], o[2], o[3]);
  *reinterpret_cast<float4*>(xo + 4) = make_float4(o[4], o[5], o[6], o[7]);
  return F;
}

// ---------------------------------------------------------------------------
// mid pass: the line of one plane at one slot, NMB blocks of kSub rows.  Input
// values ym[m kSW] (ym points at the plane's slot) with frames fr(m); output
// in place, in [0, 1] of the frames ofr[s kSW] of its blocks.  Block s's
// aggregates: forward, its value at the block's last row; backward, its value
// at the row before its first.  Every sweep runs in one FP32 frame per block.
// ---------------------------------------------------------------------------
template <class FR>
__device__ __forceinline__ int mid_block(const float* ym, FR fr, int s, float (&x)[kSub]) {
  int f[kSub];
#pragma unroll
  for (int k = 0; k < kSub; ++k) {
    x[k] = ym[(s * kSub + k) * kSW];
    f[k] = fr(s * kSub + k);
  }
  return gather_frame(x, f);
}

template <class FR>
__device__ __forceinline__ void mid_line(float* ym, FR fr, short* ofr, int NMB, const Tabs& Tm, bool& bad) {
  const float lam = Tm.lams;
  const XF zero = XF{0.f, kZeroExp};
  XF af[kMaxNMB], ab[kMaxNMB];
#pragma unroll
  for (int s = 0; s < kMaxNMB; ++s) {
    af[s] = ab[s] = zero;
    if (s < NMB) {
      float x[kSub];
      const int fe = mid_block(ym, fr, s, x);
      float rr = 0.f, qq = 0.f;
#pragma unroll
      for (int k = 0; k < kSub; ++k) rr = fmaf(lam, rr, x[k]);
#pragma unroll
      for (int k = kSub - 1; k >= 0; --k) qq = lam * (qq + x[k]);
      af[s] = xf_norm(rr, fe);
      ab[s] = xf_norm(qq, fe);
    }
  }
  // backward carries at the last row of every block, from the blocks after it
  XF Ds[kMaxNMB];
  XF D = zero;
#pragma unroll
  for (int s = kMaxNMB - 1; s >= 0; --s) {
    Ds[s] = D;
    if (s < NMB) D = c_add(c_mul(D, Tm.subs[kSub]), ab[s]);
  }
  XF C = zero;   // forward carry at the row before the block
#pragma unroll
  for (int s = 0; s < kMaxNMB; ++s) {
    if (s < NMB) {
      float x[kSub];
      const int fe = mid_block(ym, fr, s, x);
      const int F = max(fe, max(C.e, Ds[s].e)) + kHead;
      const float sc = pow2f(fe - F);
      float tb[kSub];
      float sb = c_to(Ds[s], F);
#pragma unroll
      for (int k = kSub - 1; k >= 0; --k) {
        tb[k] = sb;
        sb = lam * fmaf(x[k], sc, sb);
      }
      float p = c_to(C, F);
#pragma unroll
      for (int k = 0; k < kSub; ++k) {
        p = fmaf(lam, p, x[k] * sc);
        ym[(s * kSub + k) * kSW] = p + tb[k];
      }
      ofr[s * kSW] = to16(F, bad);
      C = c_add(c_mul(C, Tm.subs[kSub]), af[s]);
    }
  }
}

// ---------------------------------------------------------------------------
// slow pass: the line (row, slot) over this CTA's nr planes, values
// ym[p stride] with frames fr(p), planes past nr as identity steps (decay 1):
// they lie after the grid's last plane, or pad a CTA's R planes to MAXR.
// load() forms the line in one frame and its aggregates (forward: at the
// CTA's last plane; backward: at the plane before its first); sweep() runs
// the sweeps with the carries C (at the plane before the first) and D (at the
// last plane, from the CTAs after), leaving y in [0, 1] of frame fe.
// ---------------------------------------------------------------------------
template <int MAXR>
struct SlowLine {
  float y[MAXR];
  int fe;
  XF af, ab;

  template <class FR>
  __device__ __forceinline__ void load(const float* ym, size_t stride, FR fr, int nr, float lam) {
    int f[MAXR];
#pragma unroll
    for (int k = 0; k < MAXR; ++k) {
      y[k] = k < nr ? ym[k * stride] : 0.f;
      f[k] = k < nr ? fr(k) : kZeroExp;
    }
    fe = gather_frame(y, f);
    float rr = 0.f, qq = 0.f;
#pragma unroll
    for (int k = 0; k < MAXR; ++k) rr = fmaf(k < nr ? lam : 1.f, rr, y[k]);
#pragma unroll
    for (int k = MAXR - 1; k >= 0; --k) qq = (k < nr ? lam : 1.f) * (qq + y[k]);
    af = xf_norm(rr, fe);
    ab = xf_norm(qq, fe);
  }

  __device__ __forceinline__ void sweep(XF C, XF D, int nr, float lam) {
    const int F = max(fe, max(C.e, D.e)) + kHead;
    const float sc = pow2f(fe - F);
    float tb[MAXR];
    float sb = c_to(D, F);
#pragma unroll
    for (int k = MAXR - 1; k >= 0; --k) {
      tb[k] = sb;
      sb = (k < nr ? lam : 1.f) * fmaf(y[k], sc, sb);
    }
    float p = c_to(C, F);
#pragma unroll
    for (int k = 0; k < MAXR; ++k) {
      p = fmaf(k < nr ? lam : 1.f, p, y[k] * sc);
      y[k] = p + tb[k];
    }
    fe = F;
  }
};

// published aggregates: [2][NML] mantissas (forward, backward) and exponents
__device__ __forceinline__ void publish(float* pm, short* pe, int NML, int i, XF f, XF b, bool& bad) {
  pm[i] = f.m;
  pe[i] = to16(f.m != 0.f ? f.e : kZeroExp, bad);
  pm[NML + i] = b.m;
  pe[NML + i] = to16(b.m != 0.f ? b.e : kZeroExp, bad);
}

// Carries of the slow lines [i0, i1) for every CTA of the cluster: for each
// line and direction one thread reads the CTAs' aggregates (forward: at each
// CTA's last plane; backward: at the plane before its first), and writes CTA
// k the forward carry sum_{j<k} af_j lam^{R (k-1-j)} in place of its forward
// aggregate and the backward carry sum_{j>k} ab_j lam^{R (j-k-1)} in place of
// its backward one.  Only this thread reads or writes those slots between the
// two cluster barriers around this step.
__device__ __forceinline__ void line_carries(float* pm, short* pe, int NML, int i0, int i1, unsigned ncta, XF lamR,
                                             bool& bad) {
  const int n = i1 - i0;
  for (int idx = threadIdx.x; idx < 2 * n; idx += kThr) {
    const int dir = idx >= n, off = (dir ? NML : 0) + i0 + idx - (dir ? n : 0);
    // the j-th CTA in the direction of the scan: j (forward), ncta - 1 - j (backward)
    float m[kMaxCS];
    short e[kMaxCS];
#pragma unroll
    for (int j = 0; j < kMaxCS; ++j) {
      m[j] = 0.f;
      e[j] = (short)kF16Zero;
      if (j < (int)ncta) {
        const unsigned k = (unsigned)(dir ? (int)ncta - 1 - j : j);
        m[j] = dsm_ld_f32(dsm_addr(pm + off, k));
        e[j] = dsm_ld_s16(dsm_addr(pe + off, k));
      }
    }
    XF c = XF{0.f, kZeroExp};
#pragma unroll
    for (int j = 0; j < kMaxCS; ++j) {
      if (j < (int)ncta) {
        const unsigned k = (unsigned)(dir ? (int)ncta - 1 - j : j);
        dsm_st_f32(dsm_addr(pm + off, k), c.m);
        dsm_st_s16(dsm_addr(pe + off, k), to16(c.m != 0.f ? c.e : kZeroExp, bad));
        c = c_add(c_mul(c, lamR), XF{m[j], fr16(e[j])});
      }
    }
  }
}
// ---------------------------------------------------------------------------
// the kernel: persistent clusters taking grids from a queue (MAXR: planes per
// CTA at most, 4 or 8)
// ---------------------------------------------------------------------------
template <int MAXR>
__global__ void __launch_bounds__(kThr, 1) fs1_cluster3d_kernel(Launch L) {
  extern __shared__ __align__(16) unsigned char c3d_smem[];
  __shared__ Tabs Ta;   // fast axis (lamf, ks) and slow axis (lams, lamR)
  __shared__ Tabs Tm;   // middle axis (lams, subs)
  __shared__ int s_flags;   // bit 1: a frame out of range
  __shared__ __align__(16) float s_err[4];
  __shared__ float s_red[2 * kWarps];
  __shared__ double s_dec;
  __shared__ int s_img;
  const unsigned rank = cluster_rank(), ncta = cluster_size();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const XF zero = XF{0.f, kZeroExp};
  if (tid == 0) s_flags = 0;
  __syncthreads();

  for (;;) {
    if (rank == 0 && tid == 0) s_img = atomicAdd(L.next, 1);
    cluster_sync();
    const int q = dsm_ld_s32(dsm_addr(&s_img, 0));
    cluster_sync();   // rank 0 overwrites s_img only after every CTA has read it
    if (q >= L.nimg) break;
    const int pid = L.order ? L.order[q] : q;
    const Img& I = L.imgs[pid];
    const int nf = I.nf, nm = I.nm, ns = I.ns, NM = I.NM, R = I.R;
    const int NMB = NM / kSub, NML = NM * kSW;
    const int plane0 = (int)rank * R;
    const int nr = max(0, min(R, ns - plane0));   // planes of this CTA
    const size_t PS = (size_t)NM * kSW;             // values of a plane
    float* const bufa = reinterpret_cast<float*>(c3d_smem);   // [R][NM][SW] state buffers
    float* const bufb = bufa + R * PS;
    float* const pm = bufb + R * PS;                         // [2][NML] aggregates, then carries
    short* const pe = reinterpret_cast<short*>(pm + 2 * NML);   //   (mantissas, exponents)
    short* const cfa = pe + 2 * NML;                         // [NM][SW] line frames of bufa, bufb
    short* const cfb = cfa + NML;
    short* const cfm = cfb + NML;                            // [R][NMB][SW] mid-pass block frames
    short* const rfy = cfm + R * NMB * kSW;                  // [R NM][SW / kLP] fast-pass lane frames
    float* U = bufa;   // u (and the passes' outputs); v in V.  An accepted
    float* V = bufb;   // v-half swaps the two (v_new is written over u)
    short* cfU = cfa;
    short* cfV = cfb;
    const float* const aw = I.aw + (size_t)plane0 * PS;
    const float* const bw = I.bw + (size_t)plane0 * PS;
    const double tol = I.tol;
    const int64_t itr_max = I.itr_max;
    bool bad = false;
    if (tid == 0) {
      s_flags = 0;
      Ta.lamf = (float)exp(-I.cf);
      Ta.lams = (float)exp(-I.cs);
      Tm.lams = (float)exp(-I.cm);
      for (int k = 0; k <= kSub; ++k) Tm.subs[k] = c_decay((double)k, I.cm, XF{});
      for (int lv = 0; lv < 3; ++lv) Ta.ks[lv] = c_decay((double)(kLP << lv), I.cf, XF{});
      Ta.lamR = c_decay((double)R, I.cs, XF{});
    }
    // ---- a, b into the padded layout; u = v = 1 / N (Algorithm 2) or the
    // warm start, one frame per slow line
    const XF init = xf_norm((float)(1.0 / ((double)nf * (double)nm * (double)ns)), 0);
    auto init_state = [&](bool all) {
      for (int i = tid; i < NML; i += kThr) {
        const int m = i / kSW, j = i % kSW;
        XF uv[MAXR], vv[MAXR];
#pragma unroll
        for (int p = 0; p < MAXR; ++p) {
          const bool real = p < nr && m < nm && j < nf;
          const int64_t gp = ((int64_t)(plane0 + p) * nm + m) * nf + j;
          uv[p] = vv[p] = zero;
          if (real) {
            uv[p] = I.f_init ? from_log(I.f_init[gp]) : init;
            if (all) vv[p] = I.g_init ? from_log(I.g_init[gp]) : init;
          }
          if (all && p < nr) {
            const size_t o = (size_t)(plane0 + p) * PS + i;
            I.aw[o] = real ? load_in(I.a, gp, L.in_f32) : 0.f;
            I.bw[o] = real ? load_in(I.b, gp, L.in_f32) : 0.f;
          }
        }
        float x[MAXR];
        cfU[i] = to16(to_block(uv, x), bad);
#pragma unroll
        for (int p = 0; p < MAXR; ++p)
          if (p < nr) U[p * PS + i] = x[p];
        if (all) {
          cfV[i] = to16(to_block(vv, x), bad);
#pragma unroll
          for (int p = 0; p < MAXR; ++p)
            if (p < nr) V[p * PS + i] = x[p];
        }
      }
    };
    init_state(true);
    __syncthreads();

    // fast pass then mid pass: (im, its line frames icf) -> U, block frames cfm
    auto fast_mid = [&](const float* im, const short* icf) {
      const int ls = lane & 7;
      for (int g = warp; g < nr * NM / 4; g += kWarps) {   // 4 rows per warp
        const int r = 4 * g + (lane >> 3), m = r % NM;
        const int F = fast_lane(im + r * kSW + kLP * ls, icf + m * kSW + kLP * ls, U + r * kSW + kLP * ls, ls, Ta);
        rfy[r * (kSW / kLP) + ls] = to16(F, bad);
      }
      __syncthreads();
      if (tid < nr * kSW) {
        const int p = tid / kSW, slot = tid % kSW;
        const short* const fy = rfy + (size_t)p * NM * (kSW / kLP) + slot / kLP;
        mid_line(U + p * PS + slot, [&](int m) { return fr16(fy[m * (kSW / kLP)]); }, cfm + p * NMB * kSW + slot,
                 NMB, Tm, bad);
      }
      __syncthreads();
    };
    // slow pass over U: phase A, the carries, phase B; epi(i, line) takes each
    // line's result
    auto slow = [&](auto&& epi) {
      for (int i = tid; i < NML; i += kThr) {
        const short* const fm = cfm + (i / kSW / kSub) * kSW + i % kSW;
        SlowLine<MAXR> l;
        l.load(U + i, PS, [&](int p) { return fr16(fm[p * NMB * kSW]); }, nr, Ta.lams);
        publish(pm, pe, NML, i, l.af, l.ab, bad);
      }
      cluster_sync();
      const int per = (NML + (int)ncta - 1) / (int)ncta;
      const int i0 = min(NML, (int)rank * per), i1 = min(NML, i0 + per);
      line_carries(pm, pe, NML, i0, i1, ncta, Ta.lamR, bad);
      cluster_sync();
      for (int i = tid; i < NML; i += kThr) {
        const short* const fm = cfm + (i / kSW / kSub) * kSW + i % kSW;
        SlowLine<MAXR> l;
        l.load(U + i, PS, [&](int p) { return fr16(fm[p * NMB * kSW]); }, nr, Ta.lams);
        l.sweep(XF{pm[i], fr16(pe[i])}, XF{pm[NML + i], fr16(pe[NML + i])}, nr, Ta.lams);
        epi(i, l);
      }
    };
    // m / y along line i into (xm, frame cf[i]); zero masses give zero
    auto divide = [&](int i, const float (&y)[MAXR], int fe, const float* mw, float* xm, short* cf) {
      XF z[MAXR];
#pragma unroll
      for (int p = 0; p < MAXR; ++p) {
        z[p] = zero;
        if (p < nr) {
          const float mv = mw[p * PS + i];
          const XF yy = xf_norm(y[p], fe);
          if (mv > 0.f) z[p] = XF{__fdividef(mv, yy.m), -yy.e};
        }
      }
      float x[MAXR];
      cf[i] = to16(to_block(z, x), bad);
#pragma unroll
      for (int p = 0; p < MAXR; ++p)
        if (p < nr) xm[p * PS + i] = x[p];
    };

    int64_t ell = 0;
    double err = 0.0;
    for (;; ++ell) {
      // ---- v-half: y = K^T u (fast, mid, slow), the error terms with v,
      // v_new = b / y over the consumed u
      fast_mid(U, cfU);
      float eh = 0.f, el = 0.f;
      slow([&](int i, SlowLine<MAXR>& l) {
        const int fv = fr16(cfV[i]);
#pragma unroll
        for (int p = 0; p < MAXR; ++p) {
          if (p < nr) {
            const XF vo = XF{V[p * PS + i], fv};
            const float pv = c_to(c_mul(vo, XF{l.y[p], l.fe}), 0);   // v (K^T u) at the point
            df_add(eh, el, fabsf(pv - bw[p * PS + i]), 0.f);
          }
        }
        divide(i, l.y, l.fe, bw, U, cfU);
      });
      warp_sum_df(eh, el);
      if (lane == 0) {
        s_red[2 * warp] = eh;
        s_red[2 * warp + 1] = el;
      }
      __syncthreads();
      if (tid == 0) {
        float h = 0.f, l = 0.f;
        for (int w = 0; w < kWarps; ++w) df_add(h, l, s_red[2 * w], s_red[2 * w + 1]);
        s_err[0] = h;
        s_err[1] = l;
      }
      cluster_sync();
      // the cluster's sum in FP64, in one fixed order in every CTA
      if (warp == 0) {
        double e = 0.0;
        if (lane < (int)ncta) {
          const float2 hl = dsm_ld_f2(dsm_addr(s_err, (unsigned)lane));
          e = (double)hl.x + (double)hl.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0) s_dec = e;
      }
      __syncthreads();
      err = s_dec;
      const bool stop = !isfinite(err) || err <= tol || ell >= itr_max;   // cluster-uniform
      if (!stop) {   // accept v_new
        float* const t = U;
        U = V;
        V = t;
        short* const tf = cfU;
        cfU = cfV;
        cfV = tf;
      }
      // At the stop, u^l is rebuilt (v^l is kept): the initial u when no
      // iteration ran, else by this same u-half from v^l, which is how
      // iteration l - 1 made it (one code path, so the result is
      // bit-identical and a resumed solve continues exactly).  s_err is
      // rewritten only after the u-half's two cluster barriers.
      if (stop && ell == 0) {
        init_state(false);
        __syncthreads();
        break;
      }
      // ---- u-half: u = a / (K v)
      fast_mid(V, cfV);
      slow([&](int i, SlowLine<MAXR>& l) { divide(i, l.y, l.fe, aw, U, cfU); });
      __syncthreads();
      if (stop) break;
    }
    const int status = !isfinite(err) ? FS1_ENUMERIC : (err <= tol ? FS1_OK : FS1_ENOTCONV);   // cluster-uniform
    // ---- the final potentials (the cost launch reads them)
    for (int i = tid; i < NML; i += kThr) {
      const int m = i / kSW, j = i % kSW;
      if (m >= nm || j >= nf) continue;
      const int fu = fr16(cfU[i]), fv = fr16(cfV[i]);
      for (int p = 0; p < nr; ++p) {
        const int64_t gp = ((int64_t)(plane0 + p) * nm + m) * nf + j;
        I.f_out[gp] = to_log(U[p * PS + i], fu);
        I.g_out[gp] = to_log(V[p * PS + i], fv);
      }
    }
    if (bad) atomicOr(&s_flags, 2);
    __syncthreads();
    cluster_sync();
    if (rank == 0 && tid == 0) {
      int fl = 0;   // flags of every CTA
      for (unsigned k = 0; k < ncta; ++k) fl |= dsm_ld_s32(dsm_addr(&s_flags, k));
      PairResult res;
      res.w = NAN;   // the cost launch fills it in
      res.err = err;
      res.iters = ell;
      res.status = (fl & 2) ? FS1_EUNSUPPORTED : status;   // a frame out of range: the grid kernel solves it
      res.pad = (int)ncta;
      L.results[pid] = res;
    }
    cluster_sync();   // s_flags and the exchange buffers are reused by the next grid
  }
  cluster_sync();     // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the kernel for at most 4 (v = 0) or 8 (v = 1) planes per CTA
using KernelFn = void (*)(Launch);
KernelFn kernel_of(int v) { return v ? fs1_cluster3d_kernel<8> : fs1_cluster3d_kernel<4>; }
int variant_of(int R) { return R > 4 ? 1 : 0; }

cudaError_t prepare(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int v, int cs, size_t smem,
                    cudaStream_t st) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (st) cudaStreamIsCapturing(st, &cst);
  if (cst == cudaStreamCaptureStatusNone) {
    cudaError_t e = cudaFuncSetAttribute(kernel_of(v), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel_of(v), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kThr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaSuccess;
}

// clusters of cs CTAs of kernel variant v with smem bytes of dynamic shared
// memory that fit on the current device at once (0: none); queried once per
// device and shape (handles used from several host threads share the table)
int clusters_of(int v, int cs, size_t smem) {
  struct Key {
    int dev, v, cs;
    size_t smem;
    int n;
  };
  static std::vector<Key> known;
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  for (const Key& k : known)
    if (k.dev == dev && k.v == v && k.cs == cs && k.smem == smem) return k.n;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  int n = 0;
  if (prepare(cfg, attr, v, cs, smem, nullptr) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, (const void*)kernel_of(v), &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  known.push_back(Key{dev, v, cs, smem, n});
  return n;
}

int rows_of(const PairDesc& d) { return (int)((d.n_mid + kSub - 1) / kSub * kSub); }

// the cluster size that puts the most SMs to work while every CTA's planes
// fit (0: none)
int cs_of(const PairDesc& d) {
  const int NM = rows_of(d);
  int best = 0, cover = 0;
  for (int cs = kMaxCS; cs >= kMinCS; --cs) {
    const int R = (int)((d.n_slow + cs - 1) / cs);
    if (R > kMaxR || smem_bytes(R, NM) > kSmemCap) continue;
    const int n = clusters_of(variant_of(R), cs, smem_bytes(R, NM));
    if (n > 0 && n * cs > cover) {
      cover = n * cs;
      best = cs;
    }
  }
  return best;
}

bool shape_ok(const PairDesc& d) {
  if (d.n_mid < 2 || d.n_fast < 1 || d.n_slow < 1 || d.n_fast > kSW || d.n_mid > kMaxNM) return false;
  // FP32-frame sweeps on every axis (an axis of one point has no recurrence)
  if (d.n_fast > 1 && !(d.h_fast / d.eps <= kFrameC)) return false;
  if (!(d.h_mid / d.eps <= kFrameC)) return false;
  if (d.n_slow > 1 && !(d.h_slow / d.eps <= kFrameC)) return false;
  return true;
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }
size_t slot_values(const PairDesc& d) { return (size_t)d.n_slow * rows_of(d) * kSW; }

}  // namespace c3d

int cluster3d_ok(const PairDesc& d) { return c3d::shape_ok(d) && c3d::cs_of(d) > 0; }

size_t cluster3d_workspace(const PairDesc* d, int count) {
  using namespace c3d;
  size_t b = al(sizeof(Img) * count) + al(sizeof(int) * count) + al(sizeof(int) * 2 * (kMaxCS + 1));
  for (int i = 0; i < count; ++i) {
    b += 2 * al(sizeof(float) * slot_values(d[i]));
    if (!d[i].f_out) b += al(sizeof(double) * d[i].n);
    if (!d[i].g_out) b += al(sizeof(double) * d[i].n);
  }
  return b;
}

int launch_cluster_3d(const PairDesc* d, int count, int in_f32, PairResult* results, void* ws, size_t ws_bytes,
                      void* stream, long long* launches, PairDesc* cost) {
  using namespace c3d;
  cudaStream_t st = (cudaStream_t)stream;
  if (count < 1) return FS1_OK;
  if (cluster3d_workspace(d, count) > ws_bytes) return FS1_ENOMEM;
  char* p = (char*)ws;
  Img* d_imgs = (Img*)p;
  p += al(sizeof(Img) * count);
  int* d_order = (int*)p;
  p += al(sizeof(int) * count);
  int* d_next = (int*)p;
  p += al(sizeof(int) * 2 * (kMaxCS + 1));
  std::vector<Img> imgs(count);
  std::vector<int> csz(count);   // queue: 2 cs + kernel variant
  std::vector<size_t> smem(count);
  for (int i = 0; i < count; ++i) {
    const PairDesc& D = d[i];
    if (!cluster3d_ok(D)) return FS1_EINVAL;
    const int cs = cs_of(D);
    Img I{};
    I.a = D.a;
    I.b = D.b;
    I.nf = (int)D.n_fast;
    I.nm = (int)D.n_mid;
    I.ns = (int)D.n_slow;
    I.NM = rows_of(D);
    I.R = (int)((D.n_slow + cs - 1) / cs);
    smem[i] = smem_bytes(I.R, I.NM);
    csz[i] = 2 * cs + variant_of(I.R);
    I.cf = D.h_fast / D.eps;
    I.cm = D.h_mid / D.eps;
    I.cs = D.h_slow / D.eps;
    I.tol = D.tol;
    I.itr_max = D.itr_max;
    I.f_init = D.f_init;
    I.g_init = D.g_init;
    const size_t n = slot_values(D);
    I.aw = (float*)p; p += al(sizeof(float) * n);
    I.bw = (float*)p; p += al(sizeof(float) * n);
    if (D.f_out) {
      I.f_out = D.f_out;
    } else {
      I.f_out = (double*)p; p += al(sizeof(double) * D.n);
    }
    if (D.g_out) {
      I.g_out = D.g_out;
    } else {
      I.g_out = (double*)p; p += al(sizeof(double) * D.n);
    }
    imgs[i] = I;
    // the cost of the final iterate: the grid kernel warm-started from it, no iterations
    cost[i] = D;
    cost[i].f_init = I.f_out;
    cost[i].g_init = I.g_out;
    cost[i].f_out = nullptr;
    cost[i].g_out = nullptr;
    cost[i].itr_max = 0;
    cost[i].tol = 0.0;
  }
  // one queue per cluster size and kernel variant, costliest (points x cap) first
  const int nq = 2 * (kMaxCS + 1);
  std::vector<int> order;
  std::vector<int> first(nq + 1, 0);
  for (int g = 0; g < nq; ++g) {
    first[g] = (int)order.size();
    std::vector<int> mine;
    for (int i = 0; i < count; ++i)
      if (csz[i] == g) mine.push_back(i);
    std::stable_sort(mine.begin(), mine.end(), [&](int x, int y) {
      return (double)d[x].n * (double)d[x].itr_max > (double)d[y].n * (double)d[y].itr_max;
    });
    order.insert(order.end(), mine.begin(), mine.end());
  }
  first[nq] = (int)order.size();
  cudaError_t e = cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(Img) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, sizeof(int) * nq, st);
  for (int g = 0; g < nq && e == cudaSuccess; ++g) {
    const int n = first[g + 1] - first[g];
    if (n == 0) continue;
    const int cs = g / 2, v = g % 2;
    size_t sm = 0;
    for (int k = first[g]; k < first[g + 1]; ++k) sm = std::max(sm, smem[order[k]]);
    const int fit = clusters_of(v, cs, sm);
    if (fit < 1) {
      e = cudaErrorInvalidConfiguration;
      break;
    }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    e = prepare(cfg, attr, v, cs, sm, st);
    if (e != cudaSuccess) break;
    cfg.gridDim = dim3(std::min(n, fit) * cs);
    Launch L{d_imgs, results, d_order + first[g], n, in_f32, d_next + g};
    e = cudaLaunchKernelEx(&cfg, kernel_of(v), L);
    if (launches) ++*launches;
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: cluster 3D launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

}  // namespace fs1
