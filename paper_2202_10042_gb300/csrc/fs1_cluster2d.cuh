// fs1_cluster2d.cuh -- 2D FS-1 (Algorithm 2) with the image resident in the
// distributed shared memory of one thread-block cluster (sm_103a).
//
// K = K_slow (x) K_fast (Section 4, block form) is applied as a pass of the 1D
// recurrences of eq. "recursion" along every row and a pass along every
// column ("2d recursion").  One cluster of S CTAs (the launch's cluster size)
// owns one image at a time and keeps its scalings u, v in shared memory for
// the whole solve: CTA k of the cluster holds the rows [k R, k R + R),
// R = ceil(n_slow / S).
//   row pass    : rows are local to a CTA; a warp scans a row, each lane a
//                 chunk of PF points, lanes joined by a Kogge-Stone scan of the
//                 (decay, value) chunk aggregates;
//   column pass : thread t scans slot t of the CTA's R rows serially; the CTA
//                 aggregates of every column are published in shared memory,
//                 one cluster barrier, and each CTA forms its forward and
//                 backward carries from the other CTAs' aggregates read
//                 through distributed shared memory (Horner over CTAs with
//                 lam^R).  HBM is read only for a and b (their working set
//                 stays in L2) and written once per solve.
// State.  A value is an FP32 number times a power-of-two frame shared by a
// block of kSub points (the log-domain stabilisation of the Remarks in
// Sections 2 and 3, the frames holding the absorbed potentials exactly):
// u and v (outputs of a column pass) keep one frame per column slot and kSub
// consecutive rows; the row-pass output Y keeps one frame per row, lane and
// kSub consecutive points of the lane's chunk.  Values lie in [0, 1] of
// their frame.  The sweeps run in FP32 inside such a frame: with
// c = h / eps <= kFrameC on both axes every output of a block is at least
// lam^kSub = e^-64 of the block's largest term, so what a frame flushes stays
// below FP32 rounding.  Images with a larger c on an axis, or beyond the
// shared-memory capacity, go to the grid kernel (fs1_solve2d.cu).
//
// Row slots.  A row of n_fast points occupies SW = 32 PF slots; point j of the
// row sits in slot (j % PF) 32 + j / PF, so lane l's k-th point is slot
// 32 k + l (bank-conflict free) and thread t of the column pass takes slot t.
// Slots past n_fast hold zeros (they lie after the row's last point, so the
// decays across them never reach a real point).
//
// One iteration of Algorithm 2 (v-half, then u-half):
//   v-half: Y = (I (x) K_f) u written over u (u is recomputed from v at the
//           stop), column pass on Y -> y = K^T u in registers, error terms
//           |v (K^T u) - b|, cluster sum of the error (FP64, fixed order,
//           every CTA decides alike), then v = b / y unless the iteration
//           stops;
//   u-half: Y = (I (x) K_f) v into the u arrays, column pass -> u = a / y.
// The stop test of iteration l is on (u^l, v^l); at the stop v^l is still in
// place and u^l = a / (K v^l) is recomputed bit-identically by the same
// u-half code once more (l = 0: the initial u).  The transport cost
//   h_f sum u (K_s (x) K_f^(c)) v + h_s sum u (K_s^(c) (x) K_f) v,
// K^(c)_ij = lam^{|i-j|} |i-j|, is formed with the distance-weighted
// operator in two more row and two more column passes.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "fs1.h"
#include "fs1_device.cuh"
#include "fs1_internal.h"

namespace fs1 {
namespace c2d {

constexpr int kMaxCS = 16;          // largest cluster (a non-portable size)
constexpr int kThr = 512;           // threads per CTA
constexpr int kWarps = kThr / 32;
constexpr int kSub = 8;             // points per frame block
constexpr double kFrameC = 8.0;     // FP32-frame sweeps need c = h / eps <= kFrameC (lam^kSub >= e^-64)
constexpr int kHead = 6;            // headroom bits above a block's largest term

// per-image descriptor (device memory)
struct Img {
  const void* a;
  const void* b;
  int nf, ns;            // fast (contiguous) and slow lengths
  int R;                 // rows per CTA: ceil(ns / cluster size)
  double cf, cs;         // h / eps per axis
  double hf, hs;
  double tol;
  int64_t itr_max;
  const double* f_init;  // optional warm start (log u, log v), row major
  const double* g_init;
  double* f_out;         // optional potentials out
  double* g_out;
  float* aw;             // [ns][SW] a, b in slot order (workspace; L2-resident while
  float* bw;             //   the image is solved)
  float* us;             // [ns][SW] u saved for the cost phase, and its column frames
  int* usf;              //   [cluster size][RS / kSub][SW]
};

struct Launch {
  const Img* imgs;
  PairResult* results;
  const int* order;      // image order (decreasing cost)
  int nimg;
  int in_f32;
  const int* valid;      // input-check flags (0: FS1_EINVAL without solving); may be null
  int* next;             // work-queue head (zeroed per launch)
};

// decay tables of the image being solved (shared memory)
struct Tabs {
  float lamf, lams;      // lam as FP32 (frame sweeps)
  XF xlamf, xlams;       // lam as extended range (cost phase)
  XF subf[kSub + 1];     // lam_f^k, k <= kSub
  XF subs[kSub + 1];     // lam_s^k
  XF ks[5];              // lam_f^{PF 2^lv}: the warp scan of the row pass
  XF lamR;               // lam_s^R: one CTA's rows
  int exact;             // 1: blocks take a common frame by their largest value (gather_frame);
                         // 0: by their largest frame (frame_max), exact enough while c <= 3
};

// ---------------------------------------------------------------------------
// cluster primitives (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ unsigned dsm_addr(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ XF dsm_ld_xf(unsigned addr) {
  float m;
  int e;
  asm volatile("ld.shared::cluster.v2.b32 {%0, %1}, [%2];" : "=f"(m), "=r"(e) : "r"(addr) : "memory");
  return XF{m, e};
}
__device__ __forceinline__ float2 dsm_ld_f2(unsigned addr) {
  float x, y;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(addr) : "memory");
  return make_float2(x, y);
}
__device__ __forceinline__ int dsm_ld_s32(unsigned addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double dsm_ld_f64(unsigned addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ float load_in(const void* p, int64_t i, int f32) {
  return f32 ? reinterpret_cast<const float*>(p)[i] : (float)reinterpret_cast<const double*>(p)[i];
}
// e^x in extended range (x = -inf gives zero)
__device__ __forceinline__ XF from_log(double x) {
  if (!(x > -INFINITY)) return XF{0.f, kZeroExp};
  const double t = x * 1.4426950408889634;
  const double e = floor(t);
  return xf_norm((float)exp2(t - e), (int)e);
}
__device__ __forceinline__ double to_log(float x, int F) {
  return x > 0.f ? log((double)x) + (double)F * 0.6931471805599453 : -INFINITY;
}
// u d as FP64
__device__ __forceinline__ double prod64(XF u, XF d) {
  if (u.m == 0.f || d.m == 0.f) return 0.0;
  return ldexp((double)u.m * (double)d.m, u.e + d.e);
}

// N extended-range values as FP32 numbers in one frame (returned), the
// largest in [0.5, 1); zeros stay zero
// frames are stored as 16-bit integers (-32768: an all-zero block); a frame
// beyond +-32767 sets `bad` (the image is then solved by the grid kernel)
constexpr int kF16Zero = -32768;
__device__ __forceinline__ int fr16(short f) { return f == (short)kF16Zero ? kZeroExp : (int)f; }
__device__ __forceinline__ short to16(int f, bool& bad) {
  if (f <= kZeroExp / 2) return (short)kF16Zero;
  bad |= f > 32767 || f < -32767;
  return (short)max(-32767, min(32767, f));
}

// N values x[k] (>= 0) given relative to frames f[k], brought into one frame
// set by the largest value (each value's own exponent counts, not only its
// frame: a frame shared by many points can lie far above a given point, and a
// common frame taken from the largest frame alone would push such points into
// FP32's subnormal range, dropping real contributions where the scalings span
// hundreds of binary orders within a few points).  The largest lands in
// [0.5, 1); values more than 2^126 below it become zero (with c = h / eps <= 8
// they are negligible in every output of the next sweep).  Returns the frame
// (kZeroExp: all zero).
template <int N>
__device__ __forceinline__ int gather_frame(float (&x)[N], const int (&f)[N]) {
  int e[N];
  int emax = kZeroExp;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int d = fexp(x[k]);   // kZeroExp for zero or subnormal
    e[k] = d == kZeroExp ? kZeroExp : f[k] + d;
    emax = max(emax, e[k]);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = e[k] == kZeroExp ? 0.f : x[k] * pow2f(f[k] - emax);
  return emax;
}

// the same by the largest frame alone (cheaper; with c <= 3 on both axes a
// point lies at most about 70 binary orders below the largest frame of the
// blocks it is combined with, far from FP32's subnormal range)
template <int N>
__device__ __forceinline__ int frame_max(float (&x)[N], const int (&f)[N]) {
  int emax = kZeroExp;
#pragma unroll
  for (int k = 0; k < N; ++k) emax = max(emax, f[k]);
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] *= pow2f(f[k] - emax);
  return emax;
}

template <int N>
__device__ __forceinline__ int to_block(const XF (&v)[N], float (&x)[N]) {
  int em = kZeroExp;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (v[k].m != 0.f) em = max(em, v[k].e + fexp(v[k].m));
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = v[k].m * pow2f(v[k].e - em);
  return em;
}


// ---------------------------------------------------------------------------
// row pass: one warp, one row; lane l holds points l PF .. l PF + PF - 1 in
// slots 32 k + l.  Input: values im with the frames icf of their column
// blocks (same slots).  Output: values om in [0, 1] and the frames
// orf[l NSB + s] of the lane's sub-blocks of SUB = min(PF, kSub) points.
// om may alias im.
// ---------------------------------------------------------------------------
template <int PF>
__device__ __forceinline__ void row_pass_f(const float* im, const short* icf, float* om, short* orf, int lane,
                                           const Tabs& T, bool& bad) {
  constexpr int SUB = PF < kSub ? PF : kSub;
  constexpr int NSB = PF / SUB;
  float x[PF];
  int fe[NSB];
#pragma unroll
  for (int s = 0; s < NSB; ++s) {
    float xs[SUB];
    int f[SUB];
#pragma unroll
    for (int k = 0; k < SUB; ++k) {
      const int slot = (s * SUB + k) * 32 + lane;
      xs[k] = im[slot];
      f[k] = fr16(icf[slot]);
    }
    fe[s] = T.exact ? gather_frame(xs, f) : frame_max(xs, f);
#pragma unroll
    for (int k = 0; k < SUB; ++k) x[s * SUB + k] = xs[k];
  }
  const float lam = T.lamf;
  // sub-block aggregates: forward to the block's last point, backward from
  // one before its first; lane aggregates over PF points
  XF af[NSB], ab[NSB];
  XF A = XF{0.f, kZeroExp}, B = XF{0.f, kZeroExp};
#pragma unroll
  for (int s = 0; s < NSB; ++s) {
    float r = 0.f, q = 0.f;
#pragma unroll
    for (int k = 0; k < SUB; ++k) r = fmaf(lam, r, x[s * SUB + k]);
#pragma unroll
    for (int k = SUB - 1; k >= 0; --k) q = lam * (q + x[s * SUB + k]);
    af[s] = xf_norm(r, fe[s]);
    ab[s] = xf_norm(q, fe[s]);
    A = c_add(c_mul(A, T.subf[SUB]), af[s]);
  }
#pragma unroll
  for (int s = NSB - 1; s >= 0; --s) B = c_add(ab[s], c_mul(B, T.subf[SUB]));
  // Kogge-Stone over the 32 lanes (span PF 2^lv)
  XF xs = A, zs = B;
#pragma unroll
  for (int lv = 0; lv < 5; ++lv) {
    const int o = 1 << lv;
    const XF y = shfl_up(xs, o), w = shfl_down(zs, o);
    if (lane >= o) xs = c_add(c_mul(y, T.ks[lv]), xs);
    if (lane + o < 32) zs = c_add(zs, c_mul(w, T.ks[lv]));
  }
  XF C = shfl_up(xs, 1), D = shfl_down(zs, 1);
  if (lane == 0) C = XF{0.f, kZeroExp};
  if (lane == 31) D = XF{0.f, kZeroExp};
  // backward carries at the last point of every sub-block
  XF Ds[NSB];
  Ds[NSB - 1] = D;
#pragma unroll
  for (int s = NSB - 2; s >= 0; --s) Ds[s] = c_add(c_mul(Ds[s + 1], T.subf[SUB]), ab[s + 1]);
#pragma unroll
  for (int s = 0; s < NSB; ++s) {
    const int F = max(fe[s], max(C.e, Ds[s].e)) + kHead;
    const float sc = pow2f(fe[s] - F);
    float t[SUB];
    float sb = c_to(Ds[s], F);
#pragma unroll
    for (int k = SUB - 1; k >= 0; --k) {
      t[k] = sb;
      sb = lam * fmaf(x[s * SUB + k], sc, sb);
    }
    float p = c_to(C, F);
#pragma unroll
    for (int k = 0; k < SUB; ++k) {
      p = fmaf(lam, p, x[s * SUB + k] * sc);
      om[(s * SUB + k) * 32 + lane] = p + t[k];
    }
    orf[lane * NSB + s] = to16(F, bad);
    C = c_add(c_mul(C, T.subf[SUB]), af[s]);   // forward carry into the next sub-block
  }
}

// distance-weighted row pass (transport cost), extended range: for every
// point k of the row, sum_j lam^{|k-j|} |k-j| x_j, handed to acc(slot,
// value).  Input with column frames as row_pass_f.
template <int PF, class Acc>
__device__ __forceinline__ void row_dist(const float* im, const short* icf, int lane, const Tabs& T, Acc acc) {
  using Op = OpDist<XF>;
  using P = PairC<XF>;
  XF x[PF];
#pragma unroll
  for (int k = 0; k < PF; ++k) x[k] = XF{im[k * 32 + lane], fr16(icf[k * 32 + lane])};
  const XF lam = T.xlamf;
  const XF z = XF{0.f, kZeroExp};
  XF p = z, A = z, s = z, B = z;
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    A = c_mul(c_add(A, p), lam);
    p = c_add(c_mul(p, lam), x[k]);
  }
#pragma unroll
  for (int k = PF - 1; k >= 0; --k) {
    B = c_mul(c_add(c_add(B, s), x[k]), lam);
    s = c_mul(c_add(s, x[k]), lam);
  }
  P xs{p, A}, zs{s, B};
#pragma unroll
  for (int lv = 0; lv < 5; ++lv) {
    const int o = 1 << lv;
    const P y = Op::up(xs, o), w = Op::down(zs, o);
    if (lane >= o) xs = Op::fwd(y, xs, T.ks[lv], (float)(PF << lv));
    if (lane + o < 32) zs = Op::bwd(zs, w, T.ks[lv], (float)(PF << lv));
  }
  P cf = Op::up(xs, 1), cb = Op::down(zs, 1);
  if (lane == 0) cf = Op::zero();
  if (lane == 31) cb = Op::zero();
  XF tb[PF];
  s = cb.p;
  B = cb.a;
#pragma unroll
  for (int k = PF - 1; k >= 0; --k) {
    tb[k] = B;
    B = c_mul(c_add(c_add(B, s), x[k]), lam);
    s = c_mul(c_add(s, x[k]), lam);
  }
  p = cf.p;
  A = cf.a;
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    A = c_mul(c_add(A, p), lam);
    p = c_add(c_mul(p, lam), x[k]);
    acc(k * 32 + lane, c_add(A, tb[k]));
  }
}

// ---------------------------------------------------------------------------
// column pass: thread t scans slot t over the CTA's rows r < nr (nr <= R <=
// RS); the CTAs of the cluster are joined through distributed shared memory.
// Phase A forms the chunk aggregates and publishes them (forward: measured at
// the chunk's last row; backward: from one row before its first); after a
// cluster barrier, phase B reads the other CTAs' aggregates, forms the
// carries and runs the final sweeps.  The input's values are ym[r SW + t]
// with frames fr(r); the result y_r = (K_s Y)_r is left as y[r] in [0, 1]
// of the frame fe[r / kSub].
// ---------------------------------------------------------------------------
template <int RS>
struct ColF {
  static constexpr int NSB = RS / kSub;
  float y[RS];
  int fe[NSB];   // input frames; after phase B the output frames
  XF af[NSB], ab[NSB];
  __device__ __forceinline__ XF get(int r) const { return XF{y[r], fe[r / kSub]}; }
};

// MASK: rows past nr are identity steps (decay 1).  Without it they decay as
// real rows; that is exact when every CTA with a later CTA holding rows has
// all RS rows (R = RS): the rows past nr then lie after the image's last row.
template <int RS, bool MASK, class FR>
__device__ __forceinline__ void colf_a(ColF<RS>& c, const float* ym, FR fr, int SW, int t, int nr, const Tabs& T,
                                       XF* pubf, XF* pubb) {
  constexpr int NSB = ColF<RS>::NSB;
  const float lam = T.lams;
  XF A = XF{0.f, kZeroExp}, B = XF{0.f, kZeroExp};
#pragma unroll
  for (int s = 0; s < NSB; ++s) {
    float yv[kSub];
    int f[kSub];
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      const int r = s * kSub + k;
      yv[k] = r < nr ? ym[r * SW + t] : 0.f;
      f[k] = r < nr ? fr(r) : kZeroExp;
    }
    const int emax = T.exact ? gather_frame(yv, f) : frame_max(yv, f);
    c.fe[s] = emax;
    float rr = 0.f, qq = 0.f;
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      c.y[s * kSub + k] = yv[k];
      rr = fmaf(!MASK || s * kSub + k < nr ? lam : 1.f, rr, c.y[s * kSub + k]);
    }
#pragma unroll
    for (int k = kSub - 1; k >= 0; --k) qq = (!MASK || s * kSub + k < nr ? lam : 1.f) * (qq + c.y[s * kSub + k]);
    c.af[s] = xf_norm(rr, emax);
    c.ab[s] = xf_norm(qq, emax);
    const int len = MASK ? max(0, min(kSub, nr - s * kSub)) : kSub;
    A = c_add(c_mul(A, T.subs[len]), c.af[s]);
  }
#pragma unroll
  for (int s = NSB - 1; s >= 0; --s) {
    const int len = MASK ? max(0, min(kSub, nr - s * kSub)) : kSub;
    B = c_add(c.ab[s], c_mul(B, T.subs[len]));
  }
  pubf[t] = A;
  pubb[t] = B;
}

// Forward and backward carries of this CTA's chunk from the other CTAs'
// aggregates (Horner over the ncta CTAs, lam^R per CTA); the remote loads
// are issued four at a time, so their latencies overlap.
__device__ __forceinline__ void col_carries(const XF* pubf, const XF* pubb, int t, unsigned rank, unsigned ncta,
                                            const Tabs& T, XF& C, XF& D) {
  constexpr int kB = 4;
  const XF z = XF{0.f, kZeroExp};
  C = z;
  D = z;
  for (unsigned k0 = 0; k0 < rank; k0 += kB) {
    XF x[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) x[i] = k0 + i < rank ? dsm_ld_xf(dsm_addr(pubf + t, k0 + i)) : z;
#pragma unroll
    for (int i = 0; i < kB; ++i)
      if (k0 + i < rank) C = c_add(c_mul(C, T.lamR), x[i]);
  }
  for (int k1 = (int)ncta - 1; k1 > (int)rank; k1 -= kB) {   // CTAs k1, k1 - 1, ... (> rank)
    XF x[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) x[i] = k1 - i > (int)rank ? dsm_ld_xf(dsm_addr(pubb + t, (unsigned)(k1 - i))) : z;
#pragma unroll
    for (int i = 0; i < kB; ++i)
      if (k1 - i > (int)rank) D = c_add(x[i], c_mul(D, T.lamR));
  }
}

template <int RS, bool MASK>
__device__ __forceinline__ void colf_b(ColF<RS>& c, int t, int nr, unsigned rank, unsigned ncta, const Tabs& T,
                                       const XF* pubf, const XF* pubb) {
  constexpr int NSB = ColF<RS>::NSB;
  const float lam = T.lams;
  XF C, D;
  col_carries(pubf, pubb, t, rank, ncta, T, C, D);
  XF Ds[NSB];
  Ds[NSB - 1] = D;
#pragma unroll
  for (int s = NSB - 2; s >= 0; --s) {
    const int len = MASK ? max(0, min(kSub, nr - (s + 1) * kSub)) : kSub;
    Ds[s] = c_add(c_mul(Ds[s + 1], T.subs[len]), c.ab[s + 1]);
  }
#pragma unroll
  for (int s = 0; s < NSB; ++s) {
    const int F = max(c.fe[s], max(C.e, Ds[s].e)) + kHead;
    const float sc = pow2f(c.fe[s] - F);
    float tb[kSub];
    float sb = c_to(Ds[s], F);
#pragma unroll
    for (int k = kSub - 1; k >= 0; --k) {
      tb[k] = sb;
      sb = (!MASK || s * kSub + k < nr ? lam : 1.f) * fmaf(c.y[s * kSub + k], sc, sb);
    }
    float p = c_to(C, F);
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      p = fmaf(!MASK || s * kSub + k < nr ? lam : 1.f, p, c.y[s * kSub + k] * sc);
      c.y[s * kSub + k] = p + tb[k];
    }
    c.fe[s] = F;
    const int len = MASK ? max(0, min(kSub, nr - s * kSub)) : kSub;
    C = c_add(c_mul(C, T.subs[len]), c.af[s]);
  }
}

// extended-range column pass with the operator Op (OpPlain<XF> or
// OpDist<XF>) for the transport cost (once per solve); input values ym with
// frames fr(r).  Output: the plain sum (OpPlain) or the distance-weighted
// sum (OpDist) of every row, left in x.
template <int RS, class Op>
struct ColX {
  XF x[RS];
};

template <class T>
__device__ __forceinline__ T dsm_ld_op(const T* p, unsigned rank);
template <>
__device__ __forceinline__ XF dsm_ld_op<XF>(const XF* p, unsigned rank) {
  return dsm_ld_xf(dsm_addr(p, rank));
}
template <>
__device__ __forceinline__ PairC<XF> dsm_ld_op<PairC<XF>>(const PairC<XF>* p, unsigned rank) {
  const unsigned a = dsm_addr(p, rank);
  return PairC<XF>{dsm_ld_xf(a), dsm_ld_xf(a + 8)};
}

template <int RS, class Op, class FR>
__device__ __forceinline__ void colx_a(ColX<RS, Op>& c, const float* ym, FR fr, int SW, int t, int nr,
                                       const Tabs& T, typename Op::T* pubf, typename Op::T* pubb) {
  constexpr bool W = !std::is_same<Op, OpPlain<XF>>::value;
  const XF lam = T.xlams;
  const XF z = XF{0.f, kZeroExp};
  XF p = z, A = z, s = z, B = z;
#pragma unroll
  for (int r = 0; r < RS; ++r) {
    c.x[r] = r < nr ? XF{ym[r * SW + t], fr(r)} : z;
    if (r < nr) {
      if (W) A = c_mul(c_add(A, p), lam);
      p = c_add(c_mul(p, lam), c.x[r]);
    }
  }
#pragma unroll
  for (int r = RS - 1; r >= 0; --r) {
    if (r < nr) {
      if (W) B = c_mul(c_add(c_add(B, s), c.x[r]), lam);
      s = c_mul(c_add(s, c.x[r]), lam);
    }
  }
  if constexpr (W) {
    pubf[t] = PairC<XF>{p, A};
    pubb[t] = PairC<XF>{s, B};
  } else {
    pubf[t] = p;
    pubb[t] = s;
  }
}

template <int RS, class Op>
__device__ __forceinline__ void colx_b(ColX<RS, Op>& c, int t, int nr, int R, unsigned rank, unsigned ncta,
                                       const Tabs& T, const typename Op::T* pubf, const typename Op::T* pubb) {
  constexpr bool W = !std::is_same<Op, OpPlain<XF>>::value;
  const XF lam = T.xlams;
  typename Op::T C = Op::zero(), D = Op::zero();
  for (unsigned k = 0; k < rank; ++k) C = Op::fwd(C, dsm_ld_op(pubf + t, k), T.lamR, (float)R);
  for (int k = (int)ncta - 1; k > (int)rank; --k) D = Op::bwd(dsm_ld_op(pubb + t, (unsigned)k), D, T.lamR, (float)R);
  XF s, B, p, A;
  if constexpr (W) {
    s = D.p; B = D.a; p = C.p; A = C.a;
  } else {
    s = D; B = XF{0.f, kZeroExp}; p = C; A = XF{0.f, kZeroExp};
  }
  XF tb[RS];
#pragma unroll
  for (int r = RS - 1; r >= 0; --r) {
    tb[r] = W ? B : s;
    if (r < nr) {
      if (W) B = c_mul(c_add(c_add(B, s), c.x[r]), lam);
      s = c_mul(c_add(s, c.x[r]), lam);
    }
  }
#pragma unroll
  for (int r = 0; r < RS; ++r) {
    if (r < nr) {
      if (W) A = c_mul(c_add(A, p), lam);
      p = c_add(c_mul(p, lam), c.x[r]);
      c.x[r] = c_add(W ? A : p, tb[r]);   // the result, in place
    }
  }
}


// bytes of dynamic shared memory of an instantiation
__host__ __device__ constexpr size_t smem_bytes(int PF, int RS) {
  return (size_t)RS * 32 * PF * 8 + (size_t)4 * 32 * PF * 8 + (size_t)RS * 32 * PF * 4 +
         (size_t)2 * (RS / kSub) * 32 * PF * 2 + (size_t)RS * 32 * (PF < kSub ? 1 : PF / kSub) * 2;
}

// ---------------------------------------------------------------------------
// the kernel: persistent clusters taking images from a queue
// ---------------------------------------------------------------------------
template <int PF, int RS>
__global__ void __launch_bounds__(kThr, 1) fs1_cluster2d_kernel(Launch L) {
  constexpr int SW = 32 * PF;
  constexpr int SUBF = PF < kSub ? PF : kSub;
  constexpr int NSF = PF / SUBF;      // row-frame blocks of a lane's chunk
  constexpr int NSB = RS / kSub;      // column-frame blocks of a slot
  static_assert(RS % kSub == 0, "RS");
  extern __shared__ __align__(16) unsigned char c2d_smem[];
  float* const um = reinterpret_cast<float*>(c2d_smem);   // [RS][SW] u (and the row-pass output Y)
  float* const vm = um + RS * SW;                          // [RS][SW] v
  XF* const xbf = reinterpret_cast<XF*>(vm + RS * SW);    // [2][SW] forward aggregates by half-step
  XF* const xbb = xbf + 2 * SW;                            // [2][SW] backward aggregates
  float* const sm_mass = reinterpret_cast<float*>(xbb + 2 * SW);   // [RS][SW] a or b of the half-step
  short* const cfu = reinterpret_cast<short*>(sm_mass + RS * SW);  // [NSB][SW] column frames of u
  short* const cfv = cfu + NSB * SW;                               // [NSB][SW] column frames of v
  short* const rfy = cfv + NSB * SW;                               // [RS][32][NSF] row frames of Y
  __shared__ Tabs T;
  __shared__ __align__(8) unsigned long long s_mbar;   // completion of the mass copy
  __shared__ int s_flags;   // bit 0: a mass copy did not complete in time; bit 1: a frame out of range
  __shared__ __align__(16) float s_err[4];   // this CTA's error partial (hi, lo) and range flag
  __shared__ float s_red[2 * kWarps];
  __shared__ double s_wred[kWarps];
  __shared__ __align__(8) double s_w;        // this CTA's transport-cost partial
  __shared__ double s_dec;                   // the cluster's error sum
  __shared__ int s_img;
  const unsigned rank = cluster_rank(), ncta = cluster_size();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool act = tid < SW;                 // a column-pass thread
  const XF zero = XF{0.f, kZeroExp};
  // frames of (row r, slot tid): Y by rows, u and v by column blocks
  auto yfr = [&](int r) { return fr16(rfy[(r * 32 + (tid & 31)) * NSF + (tid >> 5) / SUBF]); };
  auto ufr = [&](int r) { return fr16(cfu[(r / kSub) * SW + tid]); };
  auto vfr = [&](int r) { return fr16(cfv[(r / kSub) * SW + tid]); };
  if (tid == 0) {
    mbar_init(&s_mbar);
    s_flags = 0;
  }
  __syncthreads();
  unsigned mphase = 0;   // phase of s_mbar the next copy completes

  for (;;) {
    if (rank == 0 && tid == 0) s_img = atomicAdd(L.next, 1);
    cluster_sync();
    const int q = dsm_ld_s32(dsm_addr(&s_img, 0));
    cluster_sync();   // rank 0 overwrites s_img only after every CTA has read it
    if (q >= L.nimg) break;
    const int pid = L.order ? L.order[q] : q;
    if (L.valid && !L.valid[pid]) {
      if (rank == 0 && tid == 0) L.results[pid] = PairResult{NAN, NAN, 0, FS1_EINVAL, 0};
      continue;
    }
    const Img& I = L.imgs[pid];
    const int nf = I.nf, ns = I.ns, R = I.R;
    const int row0 = (int)rank * R;
    const int nr = max(0, min(R, ns - row0));   // rows of this CTA
    const float* const aw = I.aw + (size_t)row0 * SW;
    const float* const bw = I.bw + (size_t)row0 * SW;
    const double tol = I.tol;
    const int64_t itr_max = I.itr_max;
    bool bad = false;   // a frame of this thread's blocks left the 16-bit range
    const bool full = R == RS;   // column scans without identity steps (see colf_a)
    if (tid == 0) {
      s_flags = 0;
      T.lamf = (float)exp(-I.cf);
      T.lams = (float)exp(-I.cs);
      T.xlamf = c_decay(1.0, I.cf, XF{});
      T.xlams = c_decay(1.0, I.cs, XF{});
      for (int k = 0; k <= kSub; ++k) {
        T.subf[k] = c_decay((double)k, I.cf, XF{});
        T.subs[k] = c_decay((double)k, I.cs, XF{});
      }
      for (int lv = 0; lv < 5; ++lv) T.ks[lv] = c_decay((double)(PF << lv), I.cf, XF{});
      T.lamR = c_decay((double)R, I.cs, XF{});
      T.exact = (nf > 1 && I.cf > 3.0) || (ns > 1 && I.cs > 3.0);
    }
    // ---- a, b into slot order; u = v = 1 / N (Algorithm 2) or the warm start
    const XF init = xf_norm((float)(1.0 / ((double)nf * (double)ns)), 0);
    auto init_state = [&](bool all) {
      if (!act) return;
      const int j = (tid & 31) * PF + (tid >> 5);
#pragma unroll
      for (int s = 0; s < NSB; ++s) {
        XF uv[kSub], vv[kSub];
#pragma unroll
        for (int k = 0; k < kSub; ++k) {
          const int r = s * kSub + k;
          const bool real = r < nr && j < nf;
          const int64_t gp = (int64_t)(row0 + r) * nf + j;
          uv[k] = vv[k] = zero;
          if (real) {
            uv[k] = I.f_init ? from_log(I.f_init[gp]) : init;
            if (all) vv[k] = I.g_init ? from_log(I.g_init[gp]) : init;
          }
          if (all && r < nr) {
            I.aw[(int64_t)(row0 + r) * SW + tid] = real ? load_in(I.a, gp, L.in_f32) : 0.f;
            I.bw[(int64_t)(row0 + r) * SW + tid] = real ? load_in(I.b, gp, L.in_f32) : 0.f;
          }
        }
        float x[kSub];
        cfu[s * SW + tid] = to16(to_block(uv, x), bad);
#pragma unroll
        for (int k = 0; k < kSub; ++k) um[(s * kSub + k) * SW + tid] = x[k];
        if (all) {
          cfv[s * SW + tid] = to16(to_block(vv, x), bad);
#pragma unroll
          for (int k = 0; k < kSub; ++k) vm[(s * kSub + k) * SW + tid] = x[k];
        }
      }
    };
    init_state(true);
    __syncthreads();
    if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");   // aw, bw reach the bulk copies
    // this CTA's rows of a (u-half) or b (v-half) into sm_mass with one bulk
    // copy, issued before the row pass and waited for before the epilogue
    const unsigned mass_bytes = (unsigned)(nr * SW * sizeof(float));
    auto stage_mass = [&](const float* src) {
      if (tid == 0 && mass_bytes > 0) bulk_load(sm_mass, src, mass_bytes, &s_mbar);
    };
    auto wait_mass = [&]() {
      if (mass_bytes > 0) {
        if (!mbar_wait(&s_mbar, mphase, 1ll << 26)) atomicOr(&s_flags, 1);
        mphase ^= 1u;
      }
    };

    // row pass over this CTA's rows: (im, column frames icf) -> (um, rfy)
    auto row_pass = [&](const float* im, const short* icf) {
      for (int r = warp; r < nr; r += kWarps)
        row_pass_f<PF>(im + r * SW, icf + (r / kSub) * SW, um + r * SW, rfy + r * 32 * NSF, lane, T, bad);
      __syncthreads();
    };
    // m_r / y_r of the rows of this slot, block by block, into (xm, cf)
    auto divide_into = [&](const ColF<RS>& c, const float* mw, float* xm, short* cf) {
#pragma unroll
      for (int s = 0; s < NSB; ++s) {
        XF z[kSub];
#pragma unroll
        for (int k = 0; k < kSub; ++k) {
          const int r = s * kSub + k;
          z[k] = zero;
          if (r < nr) {
            const float m = mw[r * SW + tid];
            const XF y = xf_norm(c.y[r], c.fe[s]);
            if (m > 0.f) z[k] = XF{__fdividef(m, y.m), -y.e};
          }
        }
        float x[kSub];
        cf[s * SW + tid] = to16(to_block(z, x), bad);
#pragma unroll
        for (int k = 0; k < kSub; ++k) xm[(s * kSub + k) * SW + tid] = x[k];
      }
    };
    // u-half: Y = (I (x) K_f) v, u = a / ((K_s (x) I) Y)
    auto u_half = [&]() {
      stage_mass(aw);
      row_pass(vm, cfv);
      ColF<RS> c;
      if (act) {
        if (full) colf_a<RS, false>(c, um, yfr, SW, tid, nr, T, xbf + SW, xbb + SW);
        else colf_a<RS, true>(c, um, yfr, SW, tid, nr, T, xbf + SW, xbb + SW);
      }
      cluster_sync();
      wait_mass();
      if (act) {
        if (full) colf_b<RS, false>(c, tid, nr, rank, ncta, T, xbf + SW, xbb + SW);
        else colf_b<RS, true>(c, tid, nr, rank, ncta, T, xbf + SW, xbb + SW);
        divide_into(c, sm_mass, um, cfu);
      }
      __syncthreads();
    };

    int64_t ell = 0;
    double err = 0.0;
    for (;; ++ell) {
      // ---- v-half: Y = (I (x) K_f) u over u, y = (K_s (x) I) Y, error, v = b / y
      stage_mass(bw);
      row_pass(um, cfu);
      bool stop;
      {
        ColF<RS> c;
        if (act) {
          if (full) colf_a<RS, false>(c, um, yfr, SW, tid, nr, T, xbf, xbb);
          else colf_a<RS, true>(c, um, yfr, SW, tid, nr, T, xbf, xbb);
        }
        cluster_sync();
        wait_mass();
        float eh = 0.f, el = 0.f;
        if (act) {
          if (full) colf_b<RS, false>(c, tid, nr, rank, ncta, T, xbf, xbb);
          else colf_b<RS, true>(c, tid, nr, rank, ncta, T, xbf, xbb);
#pragma unroll
          for (int r = 0; r < RS; ++r) {
            if (r < nr) {
              const XF vo = XF{vm[r * SW + tid], vfr(r)};
              const float pv = c_to(c_mul(vo, c.get(r)), 0);   // v (K^T u) at the point
              df_add(eh, el, fabsf(pv - sm_mass[r * SW + tid]), 0.f);
            }
          }
        }
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
        stop = !isfinite(err) || err <= tol || ell >= itr_max;
        if (!stop && act) divide_into(c, sm_mass, vm, cfv);
      }
      __syncthreads();
      // At the stop, u^l is rebuilt: the initial u when no iteration ran,
      // else by this same u-half from v^l, which is how iteration l - 1 made
      // it (one code path, so the result is bit-identical and a resumed
      // solve continues exactly)
      if (stop && ell == 0) {
        init_state(false);
        __syncthreads();
        break;
      }
      // ---- u-half
      u_half();
      if (stop) break;
    }
    cluster_sync();   // every CTA is done with the exchange buffers
    const int status = !isfinite(err) ? FS1_ENUMERIC : (err <= tol ? FS1_OK : FS1_ENOTCONV);   // cluster-uniform
    // ---- optional potentials out
    if ((I.f_out || I.g_out) && act) {
      const int j = (tid & 31) * PF + (tid >> 5);
      for (int r = 0; r < nr && j < nf; ++r) {
        const int64_t gp = (int64_t)(row0 + r) * nf + j;
        if (I.f_out) I.f_out[gp] = to_log(um[r * SW + tid], ufr(r));
        if (I.g_out) I.g_out[gp] = to_log(vm[r * SW + tid], vfr(r));
      }
    }
    // ---- transport cost (a9): h_s u . ((K_s^(c) (x) K_f) v) + h_f u . ((K_s (x) K_f^(c)) v)
    double acc = 0.0;
    if (status != FS1_ENUMERIC) {
      float* const us = I.us + (size_t)row0 * SW;
      int* const usf = I.usf + (size_t)rank * NSB * SW;
      for (int idx = tid; idx < nr * SW; idx += kThr) us[idx] = um[idx];
      for (int idx = tid; idx < NSB * SW; idx += kThr) usf[idx] = fr16(cfu[idx]);
      __syncthreads();
      auto ug = [&](int r, int slot) { return XF{us[r * SW + slot], usf[(r / kSub) * SW + slot]}; };
      // slow axis: Z = (I (x) K_f) v by rows, then (K_s^(c) (x) I) Z by columns
      row_pass(vm, cfv);
      {
        using OpD = OpDist<XF>;
        PairC<XF>* pf = reinterpret_cast<PairC<XF>*>(xbf);
        PairC<XF>* pb = reinterpret_cast<PairC<XF>*>(xbb);
        ColX<RS, OpD> c;
        if (act) colx_a<RS, OpD>(c, um, yfr, SW, tid, nr, T, pf, pb);
        cluster_sync();
        if (act) {
          colx_b<RS, OpD>(c, tid, nr, R, rank, ncta, T, pf, pb);
#pragma unroll
          for (int r = 0; r < RS; ++r)
            if (r < nr) acc += I.hs * prod64(ug(r, tid), c.x[r]);
        }
      }
      cluster_sync();   // the exchange buffers are reused below
      // fast axis: Z = (K_s (x) I) v by columns (into the u arrays), then
      // (I (x) K_f^(c)) Z by rows
      {
        ColX<RS, OpPlain<XF>> c;
        if (act) colx_a<RS, OpPlain<XF>>(c, vm, vfr, SW, tid, nr, T, xbf, xbb);
        cluster_sync();
        if (act) {
          colx_b<RS, OpPlain<XF>>(c, tid, nr, R, rank, ncta, T, xbf, xbb);
#pragma unroll
          for (int s = 0; s < NSB; ++s) {
            XF z[kSub];
#pragma unroll
            for (int k = 0; k < kSub; ++k) z[k] = s * kSub + k < nr ? c.x[s * kSub + k] : zero;
            float x[kSub];
            cfu[s * SW + tid] = to16(to_block(z, x), bad);
#pragma unroll
            for (int k = 0; k < kSub; ++k) um[(s * kSub + k) * SW + tid] = x[k];
          }
        }
        __syncthreads();
        for (int r = warp; r < nr; r += kWarps)
          row_dist<PF>(um + r * SW, cfu + (r / kSub) * SW, lane, T,
                       [&](int slot, XF d) { acc += I.hf * prod64(ug(r, slot), d); });
      }
    }
    // cluster sum of the cost (FP64)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s_wred[warp] = acc;
    if (bad) atomicOr(&s_flags, 2);
    __syncthreads();
    if (tid == 0) {
      double w = 0.0;
      for (int k = 0; k < kWarps; ++k) w += s_wred[k];
      s_w = w;
    }
    cluster_sync();
    if (rank == 0 && tid == 0) {
      double w = 0.0;
      int fl = 0;   // flags of every CTA
      for (unsigned k = 0; k < ncta; ++k) {
        w += dsm_ld_f64(dsm_addr(&s_w, k));
        fl |= dsm_ld_s32(dsm_addr(&s_flags, k));
      }
      PairResult res;
      res.w = status == FS1_ENUMERIC || fl ? NAN : w;
      res.err = err;
      res.iters = ell;
      // a late copy fails the image; a frame out of range sends it to the grid kernel
      res.status = (fl & 1) ? FS1_ETIMEOUT : ((fl & 2) ? FS1_EUNSUPPORTED : status);
      res.pad = (int)ncta;   // CTAs that shared the image
      L.results[pid] = res;
    }
    cluster_sync();   // s_w and the exchange buffers are reused by the next image
  }
  cluster_sync();     // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// launch of one instantiation: persistent clusters of cs CTAs, as many as fit
// at once (at most one per image)
// ---------------------------------------------------------------------------
template <int PF, int RS>
cudaError_t prepare(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int cs, cudaStream_t st) {
  auto kfn = fs1_cluster2d_kernel<PF, RS>;
  const size_t smem = smem_bytes(PF, RS);
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cst);
  if (cst == cudaStreamCaptureStatusNone) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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

// clusters of cs CTAs of this instantiation that fit on the current device at
// once (0: none)
template <int PF, int RS>
int max_clusters(int cs) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  if (prepare<PF, RS>(cfg, attr, cs, nullptr) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)fs1_cluster2d_kernel<PF, RS>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int PF, int RS>
cudaError_t launch(const Launch& L, int cs, int clusters, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = prepare<PF, RS>(cfg, attr, cs, st);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3(clusters * cs);
  return cudaLaunchKernelEx(&cfg, fs1_cluster2d_kernel<PF, RS>, L);
}

}  // namespace c2d
}  // namespace fs1
