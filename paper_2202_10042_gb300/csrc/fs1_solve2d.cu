// fs1_solve2d.cu -- 2D FS-1 (Algorithm 2) and its extension to three axes
// (the closing remark of Section 4) for sm_103a.
//
// The 2D kernel K = K_slow (x) K_fast (Section 4, block form of K) is applied
// as two passes of the 1D recurrences of eq. "recursion": along every row (the
// fast, contiguous axis, lam_1 = e^{-h_fast/eps}) and then along every column
// (lam_2 = e^{-h_slow/eps}); this is the "2d recursion" of Section 4 with the
// K_0 products done row by row.  One half-step of Algorithm 2 is
//   fast pass : Y = (I (x) K_fast) X                  one warp per row
//   slow pass : y = (K_slow (x) I) Y, z = mass / y,    one CTA per tile of 8
//               and (v-half) the marginal error        columns, one warp per
//                                                      column of the tile
// executed by one persistent cooperative kernel over a batch of images, with a
// bounded grid barrier after every pass.  The state is stored per point in
// extended range (FP32 mantissa and int exponent, struct XF), so any eps and
// grid spacing are covered with FP32 relative precision.  A line of L <= 1024
// points is staged in shared memory (rows: one coalesced read of the row;
// columns: the CTA reads the tile's rows, 64 contiguous bytes each) and split
// over the 32 lanes of a warp: each lane runs the recurrences serially over
// its P = ceil(L / 32) points, the lanes are joined by a Kogge-Stone scan of
// the lane aggregates with the same associative (decay, value) operators as
// the 1D kernel, and the result leaves shared memory with coalesced stores
// (columns: fused with the pointwise division and the error).  In shared
// memory lane l's chunk starts at l P' with P' = P | 1 (odd), so the lanes'
// 8-byte accesses to their k-th points fall in distinct banks.
//
// Stop rule per image (the while condition of Algorithm 2): the error partials
// of the image's column warps are summed in a fixed order by every CTA, so all
// CTAs decide identically.  v is double-buffered by iteration parity and the
// returned iterate keeps the accepted v.  The transport cost
//   sum u (x) [h_fast (K_s (x) K_f^(c)) v + h_slow (K_s^(c) (x) K_f) v],
// K^(c)_ij = lam^{|i-j|} |i-j|, is formed with the distance-weighted operator
// in three more passes, O(N M).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "fs1.h"
#include "fs1_device.cuh"
#include "fs1_internal.h"

namespace fs1 {

namespace {

constexpr int kThreads2 = 256;
constexpr int kWarps2 = kThreads2 / 32;
constexpr int kTileCols = kWarps2;   // columns of a tile per 32 lanes a line takes
constexpr int kBatch = 4;            // epilogue loads a thread keeps in flight
// decay table of an axis: lam^j for j <= 32, then lam^{P 2^i} (i < 5) for the
// segment scans (P = ceil(L / G) points per lane of a G-lane segment), then
// lam^{P32 2^i} for the whole-warp scans of the cost phase (P32 = ceil(L / 32))
constexpr int kTab = 43;
constexpr int kTabSeg = 33;
constexpr int kTabWarp = 38;

struct Img2D {
  const void* a;
  const void* b;
  int nf, nm, ns;      // fast (contiguous), middle (1 in 2D) and slow lengths
  int g[3];            // lanes that share one line, per axis (0 fast, 1 slow, 2 middle)
  int frame[3];        // 1: the axis takes the FP32-frame line scan
  int tw_s, tw_m;      // columns of a slow / middle tile (8 x 32 / g)
  double cf, cm, cs;   // h / eps per axis
  double hf, hm, hs;
  double tol;
  int64_t itr_max;
  XF* U;               // u
  XF* V[2];            // v by iteration parity
  XF* Y;               // fast-pass output
  XF* R;               // slow-pass output and parking area
  const double* f_init;   // optional warm start (log u, log v), row major
  const double* g_init;
  double* f_out;          // optional potentials out
  double* g_out;
  float* errp;         // [2 ceil(nf nm / 8)] error partials of the slow-pass
                       // tiles (compensated pairs)
  double* wp;          // [nf nm] cost partials of the slow lines
  int* stop;           // 0 while active; 1 + k once stopped with the final v in V[k]
  // FP32 block-frame state (launches of the FP32 path; see f32_geom)
  int lp;              // padded row length (nf rounded up to 8)
  int pf[3];           // points per lane of a line, per axis
  float* U32;          // [ns][lp] u, frames U32F [ceil(ns / 8)][lp]
  float* V32[2];       // v by iteration parity, frames V32F
  float* Y32;          // [ns][lp] fast-pass output, frames Y32F [ns][lp / 8]
  int* U32F;
  int* V32F[2];
  int* Y32F;
};

struct Launch2D {
  Img2D* imgs;
  PairResult* results;
  int nimg;
  int in_f32;
  const int* row_off;  // [nimg + 1] prefix sums of the row groups (32 / g_fast rows each)
  const int* col_off;  // [nimg + 1] prefix sums of nf nm (slow lines)
  const int* tile_off; // [nimg + 1] prefix sums of ceil(nf nm / tw_s) (slow-pass tiles)
  const int* mid_off;  // [nimg + 1] prefix sums of ns ceil(nf / tw_m) (middle-pass tiles; 0 in 2D)
  const int* midl_off; // [nimg + 1] prefix sums of nf ns (middle lines; 0 in 2D)
  int any3d;           // some image has a middle axis
  int line_stride;     // per-warp shared-memory region (XF): a staged line, its
                       // backward partials, + 2 (== 2 mod 16)
  int line_ch;         // XF of the longest staged line (32 P' of the longest line)
  XF* tab;             // [nimg][3][kTab] decay tables (axis 0 fast, 1 slow, 2 middle),
                       // written by CTA 0 at start
  unsigned long long* bar;   // zeroed per launch
  int* abort_flag;
  long long spin_cap;
};

__device__ __forceinline__ float load_m(const void* p, int64_t i, int f32) {
  return f32 ? reinterpret_cast<const float*>(p)[i] : (float)reinterpret_cast<const double*>(p)[i];
}

// asynchronous 8-byte global -> shared copy (both addresses 8-byte aligned)
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ bool grid_barrier(const Launch2D& L, unsigned long long& gen, int* sm_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    gen += gridDim.x;
    __threadfence();
    red_release_add(L.bar, 1ull);
    int good = 1;
    long long spins = 0;
    while (ld_acquire(L.bar) < gen) {
      if (++spins > L.spin_cap || ((spins & 255) == 0 && ld_relaxed(L.abort_flag))) {
        good = 0;
        atomicExch(L.abort_flag, 1);
        break;
      }
    }
    *sm_ok = good;
  }
  __syncthreads();
  return *sm_ok != 0;
}

// extended-range value of e^x (x = -inf gives zero)
__device__ __forceinline__ XF xf_from_log(double x) {
  if (!(x > -INFINITY)) return XF{0.f, kZeroExp};
  const double t = x * 1.4426950408889634;
  const double e = floor(t);
  return xf_norm((float)exp2(t - e), (int)e);
}
__device__ __forceinline__ double xf_log(XF v) {
  return v.m > 0.f ? log((double)v.m) + (double)v.e * 0.6931471805599453 : -INFINITY;
}

// image owning flat item t of a prefix-offset table (nimg <= kMaxImg2D)
__device__ __forceinline__ int owner(const int* off, int nimg, int t) {
  int i = 0;
  while (i + 1 < nimg && off[i + 1] <= t) ++i;
  return i;
}

// shuffles within segments of w lanes
__device__ __forceinline__ XF shw_up(XF a, int o, int w) {
  return XF{__shfl_up_sync(0xffffffffu, a.m, o, w), __shfl_up_sync(0xffffffffu, a.e, o, w)};
}
__device__ __forceinline__ XF shw_down(XF a, int o, int w) {
  return XF{__shfl_down_sync(0xffffffffu, a.m, o, w), __shfl_down_sync(0xffffffffu, a.e, o, w)};
}
__device__ __forceinline__ PairC<XF> shw_up(PairC<XF> a, int o, int w) {
  return PairC<XF>{shw_up(a.p, o, w), shw_up(a.a, o, w)};
}
__device__ __forceinline__ PairC<XF> shw_down(PairC<XF> a, int o, int w) {
  return PairC<XF>{shw_down(a.p, o, w), shw_down(a.a, o, w)};
}

// ---------------------------------------------------------------------------
// warp line scan of L points: out = K x (plain) or the distance-weighted sum
// (WEIGHTED), by a segment of G lanes (G = 8, 16 or 32; the warp's 32 / G
// segments scan their own lines at once).  Lane l of a segment owns points
// [l P, l P + P), P = ceil(L / G); its k-th point is at index base + k step of
// in / out / tmp (base chosen by the caller for this lane).  Lv <= L points
// are valid (0: the segment has no line).  The lane's backward sums are
// parked in `tmp` (written and read back by the same lane; tmp may alias out,
// and out may alias in).  tab: lam^j (j <= 32) and lam^{P 2^i} at ks + i.
// ---------------------------------------------------------------------------
template <bool WEIGHTED>
__device__ void line_scan(const XF* in, XF* out, XF* tmp, int64_t base, int64_t step, int L, int Lv, int G,
                          const XF* tab, int ks) {
  using Op = typename std::conditional<WEIGHTED, OpDist<XF>, OpPlain<XF>>::type;
  using T = typename Op::T;
  const int lane = threadIdx.x & (G - 1);
  const int P = (L + G - 1) / G;
  const int i0 = lane * P;
  const int n = max(0, min(P, Lv - i0));
  const XF lam = tab[1];
  const XF zero = c_zero(XF{});
  T af, ab;
  {
    XF p = zero, A = zero, s = zero, B = zero;
    for (int k = 0; k < P; ++k) {
      const XF x = k < n ? in[base + k * step] : zero;
      if (WEIGHTED) A = c_mul(c_add(A, p), lam);
      p = c_add(c_mul(p, lam), x);
    }
    for (int k = P - 1; k >= 0; --k) {
      const XF x = k < n ? in[base + k * step] : zero;
      if (WEIGHTED) B = c_mul(c_add(c_add(B, s), x), lam);
      s = c_mul(c_add(s, x), lam);
    }
    if constexpr (WEIGHTED) {
      af = T{p, A};
      ab = T{s, B};
    } else {
      af = p;
      ab = s;
    }
  }
  T x = af, z = ab;
#pragma unroll
  for (int lv = 0; lv < 5; ++lv) {
    const int o = 1 << lv;
    if (o >= G) break;
    const T y = shw_up(x, o, G);
    const T w = shw_down(z, o, G);
    if (lane >= o) x = Op::fwd(y, x, tab[ks + lv], (float)(P * o));
    if (lane + o < G) z = Op::bwd(z, w, tab[ks + lv], (float)(P * o));
  }
  T cfw = shw_up(x, 1, G), cbw = shw_down(z, 1, G);
  if (lane == 0) cfw = Op::zero();
  if (lane == G - 1) cbw = Op::zero();
  if (n <= 0) return;
  {
    XF s, B;
    if constexpr (WEIGHTED) {
      s = cbw.p;
      B = cbw.a;
    } else {
      s = cbw;
      B = zero;
    }
    for (int k = P - 1; k >= n; --k) {   // carry across the lane's empty tail
      if (WEIGHTED) B = c_mul(c_add(B, s), lam);
      s = c_mul(s, lam);
    }
    for (int k = n - 1; k >= 0; --k) {
      const XF xk = in[base + k * step];
      tmp[base + k * step] = WEIGHTED ? B : s;
      if (WEIGHTED) B = c_mul(c_add(c_add(B, s), xk), lam);
      s = c_mul(c_add(s, xk), lam);
    }
  }
  {
    XF p, A;
    if constexpr (WEIGHTED) {
      p = cfw.p;
      A = cfw.a;
    } else {
      p = cfw;
      A = zero;
    }
    for (int k = 0; k < n; ++k) {
      const XF xk = in[base + k * step];
      if (WEIGHTED) A = c_mul(c_add(A, p), lam);
      p = c_add(c_mul(p, lam), xk);
      const XF bk = tmp[base + k * step];
      out[base + k * step] = c_add(WEIGHTED ? A : p, bk);
    }
  }
}

// Fast plain line scan for a line staged in shared memory, by a segment of G
// lanes (lane chunk at in[base + k], k < P): the lane's values are taken into one power-of-two
// frame (the largest exponent of the chunk) and all four sweeps run in FP32,
// as in the 1D kernel's per-thread frames; only the lane aggregates and the
// 5-level Kogge-Stone use extended range.  A value below 2^-126 of the frame
// is dropped; every output k is at least lam^P times the largest term it
// sums, so with c P <= 40 (c = h / eps of the axis) the dropped part stays
// below FP32 rounding.  Backward partials go to the float array tf at the
// same indices.  out may alias in.
__device__ void line_scan_frame(const XF* in, XF* out, float* tf, int64_t base, int L, int Lv, int G,
                                const XF* tab) {
  const int lane = threadIdx.x & (G - 1);
  const int P = (L + G - 1) / G;
  const int n = max(0, min(P, Lv - lane * P));
  const float lam = tab[1].m * pow2f(tab[1].e);   // lam as FP32 (lam >= e^-40)
  int emax = kZeroExp;
#pragma unroll 4
  for (int k = 0; k < n; ++k) emax = max(emax, in[base + k].e);
  // lane aggregates in frame emax: forward sum lam^{P-1-k} x_k (Horner, then
  // the empty tail), backward sum lam^{k+1} x_k
  float r = 0.f, q = 0.f;
#pragma unroll 4
  for (int k = 0; k < n; ++k) {
    const XF x = in[base + k];
    r = fmaf(lam, r, x.m * pow2f(x.e - emax));
  }
#pragma unroll 4
  for (int k = n - 1; k >= 0; --k) {
    const XF x = in[base + k];
    q = lam * (q + x.m * pow2f(x.e - emax));
  }
  XF x = xf_norm(r, emax), z = xf_norm(q, emax);
  if (n < P) x = c_mul(x, tab[P - n]);
#pragma unroll
  for (int lv = 0; lv < 5; ++lv) {
    const int o = 1 << lv;
    if (o >= G) break;
    const XF y = shw_up(x, o, G);
    const XF w = shw_down(z, o, G);
    if (lane >= o) x = c_add(c_mul(y, tab[kTabSeg + lv]), x);
    if (lane + o < G) z = c_add(z, c_mul(w, tab[kTabSeg + lv]));
  }
  XF cfw = shw_up(x, 1, G), cbw = shw_down(z, 1, G);
  if (lane == 0) cfw = XF{0.f, kZeroExp};
  if (lane == G - 1) cbw = XF{0.f, kZeroExp};
  if (n <= 0) return;
  // final sweeps in frame F: room for P terms of the chunk plus the carries
  const int F = max(emax, max(cfw.e, cbw.e)) + 6;
  const float sc_tail = n < P ? tab[P - n].m * pow2f(tab[P - n].e) : 1.f;
  float sb = c_to(cbw, F) * sc_tail;
#pragma unroll 4
  for (int k = n - 1; k >= 0; --k) {
    const XF xk = in[base + k];
    tf[base + k] = sb;
    sb = lam * (sb + xk.m * pow2f(xk.e - F));
  }
  float p = c_to(cfw, F);
#pragma unroll 4
  for (int k = 0; k < n; ++k) {
    const XF xk = in[base + k];
    p = fmaf(lam, p, xk.m * pow2f(xk.e - F));
    out[base + k] = xf_norm(p + tf[base + k], F);
  }
}

// line scan over global memory with the line's points at `stride`
template <bool WEIGHTED>
__device__ void line_scan_global(const XF* in, XF* out, XF* tmp, int64_t stride, int L, const XF* tab) {
  const int P = (L + 31) >> 5;
  line_scan<WEIGHTED>(in, out, tmp, (int64_t)(threadIdx.x & 31) * P * stride, stride, L, L, 32, tab, kTabWarp);
}

// Walks j = j0, j0 + step, j0 + 2 step, ... of a line of P-point lane chunks
// and yields j's shared-memory index (j / P) P' + j % P without a division
// per step.
struct ChunkPos {
  int d, m, dq, mq, P, Pp;
  __device__ ChunkPos(int j0, int P_, int step) : P(P_), Pp(P_ | 1) {
    d = j0 / P;
    m = j0 - d * P;
    dq = step / P;
    mq = step - dq * P;
  }
  __device__ int pos() const { return d * Pp + m; }
  __device__ void next() {
    d += dq;
    m += mq;
    if (m >= P) {
      m -= P;
      ++d;
    }
  }
};

// fast pass of a group of 32 / G rows (one warp, one G-lane segment per row):
// stage, scan in shared memory, store.  Rows r0 .. of an image with `nrows`
// rows of L points; segment q takes row r0 + q.
__device__ void row_pass(const XF* in, XF* out, int nrows, int r0, int L, int G, const XF* tab, bool frame, XF* s,
                         XF* t) {
  const int lane = threadIdx.x & 31;
  const int seg = lane / G, ls = lane & (G - 1);
  const int P = (L + G - 1) / G, Pp = P | 1;
  const int r = r0 + seg;
  const bool valid = r < nrows;
  const int64_t o = (int64_t)r * L;
  XF* const sseg = s + seg * G * Pp;
  if (valid) {
    // every point of the row in flight at once (asynchronous copies)
    ChunkPos q(ls, P, G);
    for (int j = ls; j < L; j += G, q.next()) cp_async8(sseg + q.pos(), in + o + j);
    cp_async_wait_all();
  }
  __syncwarp();
  if (frame)
    line_scan_frame(s, s, reinterpret_cast<float*>(t), (int64_t)lane * Pp, L, valid ? L : 0, G, tab);
  else
    line_scan<false>(s, s, t, (int64_t)lane * Pp, 1, L, valid ? L : 0, G, tab, kTabSeg);
  __syncwarp();
  if (valid) {
    ChunkPos q(ls, P, G);
    for (int j = ls; j < L; j += G, q.next()) out[o + j] = sseg[q.pos()];
  }
  __syncwarp();
}

// Column tiles (slow and middle passes, the whole CTA).  A tile holds TW =
// 8 x 32 / G columns col0 .. col0 + TW - 1 of a plane `width` points wide;
// column c is scanned by segment c % (32 / G) of warp c / (32 / G), in that
// warp's shared-memory region.  Thread t stages and (in the caller's
// epilogue) reads column t % TW at rows t / TW + k (256 / TW), so a warp
// load covers whole row segments of the tile.
struct TileMap {
  int G, spw, TW, dr, P, Pp;
  __device__ TileMap(int G_, int L) : G(G_), spw(32 / G_), TW(kTileCols * (32 / G_)), dr(kThreads2 / TW),
                                      P((L + G_ - 1) / G_), Pp(((L + G_ - 1) / G_) | 1) {}
  __device__ int col() const { return threadIdx.x % TW; }
  __device__ int row0() const { return threadIdx.x / TW; }
  // the staged line of tile column c
  __device__ XF* line(XF* sbuf, int stride, int c) const { return sbuf + (c / spw) * stride + (c % spw) * G * Pp; }
};

__device__ void col_tile_scan(const XF* Y, int width, int ns, int col0, const TileMap& M, const XF* tab, bool frame,
                              XF* sbuf, int stride) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = M.col();
  if (col0 + c < width) {
    XF* sl = M.line(sbuf, stride, c);
    ChunkPos q(M.row0(), M.P, M.dr);
    for (int r = M.row0(); r < ns; r += M.dr, q.next()) cp_async8(sl + q.pos(), Y + (int64_t)r * width + col0 + c);
    cp_async_wait_all();
  }
  __syncthreads();
  {
    const int cs = warp * M.spw + lane / M.G;   // the column this lane's segment scans
    const int Lv = col0 + cs < width ? ns : 0;
    XF* s = sbuf + warp * stride;
    const int CH = 32 * M.Pp;
    if (frame)
      line_scan_frame(s, s, reinterpret_cast<float*>(s + CH), (int64_t)lane * M.Pp, ns, Lv, M.G, tab);
    else
      line_scan<false>(s, s, s + CH, (int64_t)lane * M.Pp, 1, ns, Lv, M.G, tab, kTabSeg);
  }
  __syncthreads();
}

// CTA sum of a compensated pair in a fixed order (every thread returns it)
__device__ void cta_sum_df(float& h, float& l, float* red) {
  warp_sum_df(h, l);
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = h;
    red[2 * (threadIdx.x >> 5) + 1] = l;
  }
  __syncthreads();
  h = 0.f;
  l = 0.f;
  for (int w = 0; w < kWarps2; ++w) df_add(h, l, red[2 * w], red[2 * w + 1]);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// FP32 block-frame path: 2D images whose lane chunks span at most 64 nats on
// every axis of more than one point (c P <= 64 with c = h / eps and P the
// points per lane: c <= 8 for lines of up to 256 points, about 4 up to 512,
// 2 up to 1024), taken where the general path below would scan an axis point
// by point (solve2d_f32_ok).  Values are FP32 relative to a power-of-two frame shared by a
// block of 8 points: u and v in blocks of 8 rows of one column (frames
// [ceil(ns / 8)][Lp]), the fast pass's output Y in blocks of 8 columns of one
// row (frames [ns][Lp / 8]); rows are padded to Lp = nf rounded up to 8, so
// that lane chunks start 32-byte aligned.  Within a block values span at
// most e^{8 c} <= e^64, and a value dropped below 2^-126 of its block's
// largest contributes less than 2^-68 of that value's share to any output
// (lam^{|i-j|} differs by at most e^{8 c} across the block): below FP32
// rounding.  A pass converts its input blocks into one frame per lane chunk
// (the chunk's largest value), runs the recurrences in FP32 as
// line_scan_frame does, and writes its output normalised per block of its own
// axis.  Per point this is FP32 arithmetic and a few exponent operations
// instead of the per-point extended-range state of the general path.
// ---------------------------------------------------------------------------
constexpr int kBlk = 8;

// lanes per line and points per lane (a multiple of 8: whole blocks per lane)
__host__ __device__ inline void f32_geom(int L, int& G, int& P) {
  G = L <= 128 ? 8 : (L <= 256 ? 16 : 32);
  P = ((L + G - 1) / G + kBlk - 1) / kBlk * kBlk;
}
// floats per column of a slow-pass tile: G chunks of P + 1, rounded up to 4
// mod 32
__host__ __device__ inline int f32_cs(int G, int P) {
  const int c = G * (P + 1);
  return c + ((4 - c % 32) + 32) % 32;
}
// A lane chunk of P points of an axis with c = h / eps spans at most e^{c P};
// one FP32 frame per chunk holds that when c P <= 64 nats (2^92, leaving 2^34
// below FP32 rounding for the smallest value kept)
constexpr double kF32MaxNats = 64.0;

// Scan of the lane chunks of a segment of G lanes: x[0 .. n) holds the lane's
// values in frame em (n = 0: no points); on return x[k] = (K x)_k of the line
// in frame F (the return value).  The lane aggregates are joined by a
// Kogge-Stone scan in extended range (tab: lam^j at j <= 32, lam^{P 2^i} at
// kTabSeg + i); the lane's backward partials go to tb[k * ts] (shared memory).
// Every lane of the warp calls.
template <int P>
__device__ __forceinline__ int chunk_scan(float (&x)[P], int n, int em, int G, const XF* tab, float lam, float* tb,
                                          int ts) {
  const int lane = threadIdx.x & (G - 1);
  float r = 0.f, q = 0.f;
#pragma unroll
  for (int k = 0; k < P; ++k)
    if (k < n) r = fmaf(lam, r, x[k]);
#pragma unroll
  for (int k = P - 1; k >= 0; --k)
    if (k < n) q = lam * (q + x[k]);
  XF xa = xf_norm(r, em), za = xf_norm(q, em);
  if (n < P) xa = c_mul(xa, tab[P - n]);
#pragma unroll
  for (int lv = 0; lv < 5; ++lv) {
    const int o = 1 << lv;
    if (o >= G) break;
    const XF y = shw_up(xa, o, G);
    const XF w = shw_down(za, o, G);
    if (lane >= o) xa = c_add(c_mul(y, tab[kTabSeg + lv]), xa);
    if (lane + o < G) za = c_add(za, c_mul(w, tab[kTabSeg + lv]));
  }
  XF cfw = shw_up(xa, 1, G), cbw = shw_down(za, 1, G);
  if (lane == 0) cfw = XF{0.f, kZeroExp};
  if (lane == G - 1) cbw = XF{0.f, kZeroExp};
  if (n <= 0) return kZeroExp;
  const int F = max(em, max(cfw.e, cbw.e)) + 6;
  const float s = pow2f(em - F);
  const float sc_tail = n < P ? tab[P - n].m * pow2f(tab[P - n].e) : 1.f;
  float sb = c_to(cbw, F) * sc_tail;
#pragma unroll
  for (int k = P - 1; k >= 0; --k)
    if (k < n) {
      tb[k * ts] = sb;
      sb = lam * (sb + x[k] * s);
    }
  float p = c_to(cfw, F);
#pragma unroll
  for (int k = 0; k < P; ++k)
    if (k < n) {
      p = fmaf(lam, p, x[k] * s);
      x[k] = p + tb[k * ts];
    }
  return F;
}

// Fast pass of a group of 32 / G rows (one warp, one G-lane segment per row)
// on the FP32 state: row r of X (u or v, frames per 8-row block of a column)
// to row r of Y (frames per 8-column block).  tb: the warp's P x 32 floats of
// shared memory.
template <int P>
__device__ void row_pass_f32(const float* X, const int* XFr, float* Y, int* YFr, int nrows, int r0, int L, int Lp,
                             int G, const XF* tab, float lam, float* tb) {
  const int lane = threadIdx.x & 31, seg = lane / G, ls = lane & (G - 1);
  const int r = r0 + seg;
  const int j0 = ls * P;
  const int n = r < nrows ? max(0, min(P, L - j0)) : 0;
  float x[P];
  int em = kZeroExp;
  const float* xr = X + (int64_t)r * Lp + j0;
  const int* fr = XFr + (int64_t)(r / kBlk) * Lp + j0;
#pragma unroll
  for (int k4 = 0; k4 < P / 4; ++k4) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 f = make_int4(0, 0, 0, 0);
    if (4 * k4 < n) {
      v = *reinterpret_cast<const float4*>(xr + 4 * k4);
      f = *reinterpret_cast<const int4*>(fr + 4 * k4);
    }
    const float vv[4] = {v.x, v.y, v.z, v.w};
    const int ff[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 4 * k4 + i;
      x[k] = k < n ? vv[i] : 0.f;
      if (x[k] != 0.f) em = max(em, ff[i] + fexp(x[k]));
    }
  }
#pragma unroll
  for (int k4 = 0; k4 < P / 4; ++k4)
    if (4 * k4 < n) {
      const int4 f = *reinterpret_cast<const int4*>(fr + 4 * k4);
      const int ff[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) x[4 * k4 + i] *= pow2f(ff[i] - em);
    }
  const int F = chunk_scan<P>(x, n, em, G, tab, lam, tb + lane, 32);
  if (n <= 0) return;
  float* yr = Y + (int64_t)r * Lp + j0;
  int* yf = YFr + (int64_t)r * (Lp / kBlk) + j0 / kBlk;
#pragma unroll
  for (int b = 0; b < P / kBlk; ++b)
    if (kBlk * b < n) {
      int fb = kZeroExp;
#pragma unroll
      for (int i = 0; i < kBlk; ++i)
        if (kBlk * b + i < n) fb = max(fb, fexp(x[kBlk * b + i]));
      const float sc = fb == kZeroExp ? 0.f : pow2f(-fb);
      float o[kBlk];
#pragma unroll
      for (int i = 0; i < kBlk; ++i) o[i] = kBlk * b + i < n ? x[kBlk * b + i] * sc : 0.f;
      reinterpret_cast<float4*>(yr + kBlk * b)[0] = make_float4(o[0], o[1], o[2], o[3]);
      reinterpret_cast<float4*>(yr + kBlk * b)[1] = make_float4(o[4], o[5], o[6], o[7]);
      yf[b] = fb == kZeroExp ? kZeroExp : F + fb;
    }
}

// Slow pass of one tile of TW = 8 x 32 / G columns (the whole CTA) on the
// FP32 state: stage the tile of Y and its block frames, scan every column in
// G-lane segments, then the update z = mass / y of the half-step, normalised
// per block of 8 rows of a column, with (v-half) the marginal-error terms of
// the accepted v.  Shared memory: values [TW][CS] with chunks of P + 1 (an
// odd stride: the lanes of a column read distinct banks) and CS = 4 mod 32
// (a warp's staging writes, 8 columns x 4 rows, hit distinct banks); frames
// [ns + ns / P][TW / 8], row r at r + r / P (the lanes of a column read
// distinct banks); lane frames [TW][G].
template <int P>
__device__ void col_pass_f32(const Img2D& I, int tile, const float* Yv, const int* YFr, const void* mass, int in_f32,
                             const float* Vold, const int* VFold, float* Z, int* ZF, bool vhalf, const XF* tab,
                             float* sbuf, float& eh, float& el) {
  const int G = I.g[1];
  const int spw = 32 / G, TW = kTileCols * spw, nbt = TW / kBlk;
  const int W = I.nf, Lp = I.lp, ns = I.ns;
  const int col0 = tile * TW;
  const int CS = f32_cs(G, P);
  float* vals = sbuf;                                   // [TW][CS]
  int* frs = reinterpret_cast<int*>(sbuf + TW * CS);    // [ns + ns / P][nbt]
  int* lfs = frs + (ns + ns / P) * nbt;                 // [TW][G]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < ns * TW; idx += kThreads2) {
    const int r = idx / TW, c = idx - r * TW;
    const int col = col0 + c;
    const float v = col < W ? __ldcg(Yv + (int64_t)r * Lp + col) : 0.f;
    vals[c * CS + (r / P) * (P + 1) + r % P] = v;
  }
  for (int idx = tid; idx < ns * nbt; idx += kThreads2) {
    const int r = idx / nbt, b = idx - r * nbt;
    const int blk = col0 / kBlk + b;
    frs[(r + r / P) * nbt + b] = blk < Lp / kBlk ? __ldcg(YFr + (int64_t)r * (Lp / kBlk) + blk) : kZeroExp;
  }
  __syncthreads();
  {
    const int warp = tid >> 5, lane = tid & 31;
    const int seg = lane / G, ls = lane & (G - 1);
    const int c = warp * spw + seg;
    const int n = col0 + c < W ? max(0, min(P, ns - ls * P)) : 0;
    float* chunk = vals + c * CS + ls * (P + 1);
    const int* fc = frs + (ls * (P + 1)) * nbt + c / kBlk;   // row ls P + k at (ls P + k + ls) nbt
    float x[P];
    int em = kZeroExp;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      x[k] = k < n ? chunk[k] : 0.f;
      if (x[k] != 0.f) em = max(em, fc[k * nbt] + fexp(x[k]));
    }
#pragma unroll
    for (int k = 0; k < P; ++k)
      if (k < n) x[k] *= pow2f(fc[k * nbt] - em);
    const float lam = tab[1].m * pow2f(tab[1].e);
    // backward partials in the chunk's own slots (x holds the chunk)
    const int F = chunk_scan<P>(x, n, em, G, tab, lam, chunk, 1);
#pragma unroll
    for (int k = 0; k < P; ++k)
      if (k < n) chunk[k] = x[k];
    lfs[c * G + ls] = F;
  }
  __syncthreads();
  // update: thread t takes column t % TW and blocks t / TW, t / TW + 256 / TW, ...
  const int c = tid % TW;
  const int col = col0 + c;
  if (col < W) {
    const int nb = (ns + kBlk - 1) / kBlk;
    for (int blk = tid / TW; blk < nb; blk += kThreads2 / TW) {
      const int r0 = blk * kBlk;
      const int ls = r0 / P;
      const int F = lfs[c * G + ls];
      const float* yc = vals + c * CS + ls * (P + 1) + (r0 - ls * P);
      float q[kBlk], m[kBlk];
#pragma unroll
      for (int i = 0; i < kBlk; ++i) m[i] = r0 + i < ns ? load_m(mass, (int64_t)(r0 + i) * W + col, in_f32) : 0.f;
      int fb = kZeroExp;
#pragma unroll
      for (int i = 0; i < kBlk; ++i) {
        q[i] = m[i] > 0.f ? __fdividef(m[i], yc[i]) : 0.f;
        fb = max(fb, fexp(q[i]));
      }
      if (vhalf) {
        // marginal-error terms |v_old y - m| of the accepted v
        const int vf = __ldcg(VFold + (int64_t)blk * Lp + col);
        const int fe = vf + F;
        const bool fast = fe >= -60 && fe <= 60;
        const float s2 = fast ? pow2f(fe) : 0.f;
#pragma unroll
        for (int i = 0; i < kBlk; ++i)
          if (r0 + i < ns) {
            const float vv = __ldcg(Vold + (int64_t)(r0 + i) * Lp + col);
            const float pv = fast ? vv * yc[i] * s2 : c_to(c_mul(xf_norm(vv, vf), xf_norm(yc[i], F)), 0);
            df_add(eh, el, fabsf(pv - m[i]), 0.f);
          }
      }
      const float sc = fb == kZeroExp ? 0.f : pow2f(-fb);
#pragma unroll
      for (int i = 0; i < kBlk; ++i)
        if (r0 + i < ns) Z[(int64_t)(r0 + i) * Lp + col] = q[i] * sc;
      ZF[(int64_t)blk * Lp + col] = fb == kZeroExp ? kZeroExp : fb - F;
    }
  }
  __syncthreads();   // the tile's shared memory is reused by the next tile
}

// the FP32 fast pass of row group grp of image I (dispatch on P)
__device__ void row_f32(const Img2D& I, const float* X, const int* XFr, int grp, const XF* tab, float* tb) {
  const int r0 = grp * (32 / I.g[0]);
  const float lam = tab[1].m * pow2f(tab[1].e);
  switch (I.pf[0]) {
    case 8: row_pass_f32<8>(X, XFr, I.Y32, I.Y32F, I.ns, r0, I.nf, I.lp, I.g[0], tab, lam, tb); break;
    case 16: row_pass_f32<16>(X, XFr, I.Y32, I.Y32F, I.ns, r0, I.nf, I.lp, I.g[0], tab, lam, tb); break;
    case 24: row_pass_f32<24>(X, XFr, I.Y32, I.Y32F, I.ns, r0, I.nf, I.lp, I.g[0], tab, lam, tb); break;
    default: row_pass_f32<32>(X, XFr, I.Y32, I.Y32F, I.ns, r0, I.nf, I.lp, I.g[0], tab, lam, tb); break;
  }
}

// the FP32 slow pass of one tile (dispatch on P)
__device__ void col_f32(const Img2D& I, int tile, const void* mass, int in_f32, const float* Vold, const int* VFold,
                        float* Z, int* ZF, bool vhalf, const XF* tab, float* sbuf, float& eh, float& el) {
  switch (I.pf[1]) {
    case 8:
      col_pass_f32<8>(I, tile, I.Y32, I.Y32F, mass, in_f32, Vold, VFold, Z, ZF, vhalf, tab, sbuf, eh, el);
      break;
    case 16:
      col_pass_f32<16>(I, tile, I.Y32, I.Y32F, mass, in_f32, Vold, VFold, Z, ZF, vhalf, tab, sbuf, eh, el);
      break;
    case 24:
      col_pass_f32<24>(I, tile, I.Y32, I.Y32F, mass, in_f32, Vold, VFold, Z, ZF, vhalf, tab, sbuf, eh, el);
      break;
    default:
      col_pass_f32<32>(I, tile, I.Y32, I.Y32F, mass, in_f32, Vold, VFold, Z, ZF, vhalf, tab, sbuf, eh, el);
      break;
  }
}

// u (or v) of the FP32 state from log values (warm start) or 1 / N: one
// thread per block of 8 rows of a column
__device__ void init_f32(const Img2D& I, const double* logs, float* X, int* XFr) {
  const int64_t N = (int64_t)I.nf * I.ns;
  const XF init = xf_norm((float)(1.0 / (double)N), 0);
  const int nb = (I.ns + kBlk - 1) / kBlk;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nb * I.lp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int blk = (int)(t / I.lp), col = (int)(t - (int64_t)blk * I.lp);
    XF v[kBlk];
    int fb = kZeroExp;
#pragma unroll
    for (int i = 0; i < kBlk; ++i) {
      const int r = blk * kBlk + i;
      v[i] = XF{0.f, kZeroExp};
      if (r < I.ns && col < I.nf) v[i] = logs ? xf_from_log(logs[(int64_t)r * I.nf + col]) : init;
      if (v[i].m != 0.f) fb = max(fb, v[i].e);
    }
#pragma unroll
    for (int i = 0; i < kBlk; ++i) {
      const int r = blk * kBlk + i;
      if (r < I.ns) X[(int64_t)r * I.lp + col] = v[i].m != 0.f ? v[i].m * pow2f(v[i].e - fb) : 0.f;
    }
    XFr[(int64_t)blk * I.lp + col] = fb;
  }
}

// u and the returned v of the FP32 state into the extended-range arrays the
// cost phase and the potentials read
__device__ void to_xf(const Img2D& I, int k) {
  const int64_t N = (int64_t)I.nf * I.ns;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(p / I.nf), col = (int)(p - (int64_t)r * I.nf);
    const int64_t q = (int64_t)r * I.lp + col, qf = (int64_t)(r / kBlk) * I.lp + col;
    I.U[p] = xf_norm(I.U32[q], I.U32F[qf]);
    I.V[k][p] = xf_norm(I.V32[k][q], I.V32F[k][qf]);
  }
}

// F32: the launch's images all take the FP32 block-frame path (2D, lane
// chunks of at most 64 nats on every axis); otherwise the per-point
// extended-range state.  The FP32 path keeps a lane's chunk (up to 32
// points) in registers; it is latency-bound, and three CTAs per SM (80
// registers, a few spilled) ran 25 % faster on 800^2 and 1024^2 images than
// two (121 registers, none spilled) and than four (64, spilling in the loops).
template <bool F32>
__global__ void __launch_bounds__(kThreads2, F32 ? 3 : 4) fs1_solve2d_kernel(Launch2D L) {
  extern __shared__ XF sline[];   // kWarps2 regions of L.line_stride XF
  __shared__ float sred[2 * kWarps2];
  __shared__ int srow[kMaxImg2D + 1], scol[kMaxImg2D + 1], stile[kMaxImg2D + 1];
  __shared__ int smid[kMaxImg2D + 1], smidl[kMaxImg2D + 1];
  __shared__ int srowa[kMaxImg2D + 1];      // prefix sums of the rows (nm ns), one per warp in the cost phase
  __shared__ signed char sstate[kMaxImg2D];  // 0 active, 1 stops this iteration, 2 stopped earlier
  __shared__ bool sframe[kMaxImg2D][3];      // the axis takes the FP32-frame line scan (c P <= 40)
  __shared__ int sok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarps2 + warp;
  const int nw = gridDim.x * kWarps2;
  const int nimg = L.nimg;
  unsigned long long gen = 0;

  for (int i = threadIdx.x; i <= nimg; i += blockDim.x) {
    srow[i] = L.row_off[i];
    scol[i] = L.col_off[i];
    stile[i] = L.tile_off[i];
    smid[i] = L.mid_off[i];
    smidl[i] = L.midl_off[i];
  }
  // descriptor check (every CTA decides alike): lanes per line must be 8, 16
  // or 32 and the tile widths must match them, or the loops below would not
  // advance; a bad descriptor ends the launch (its results stay
  // FS1_ETIMEOUT) instead of running
  {
    bool okd = true;
    for (int i = 0; i < nimg; ++i) {
      const Img2D& I = L.imgs[i];
      for (int ax = 0; ax < 3; ++ax) okd = okd && (I.g[ax] == 8 || I.g[ax] == 16 || I.g[ax] == 32);
      okd = okd && I.tw_s == kTileCols * (32 / max(1, I.g[1])) && I.tw_m == kTileCols * (32 / max(1, I.g[2]));
      if (F32)
        for (int ax = 0; ax < 2; ++ax)
          okd = okd && I.nm == 1 && (I.pf[ax] == 8 || I.pf[ax] == 16 || I.pf[ax] == 24 || I.pf[ax] == 32) &&
                I.g[ax] * I.pf[ax] >= (ax == 0 ? I.nf : I.ns) && I.lp % kBlk == 0 && I.lp >= I.nf;
    }
    if (!okd) {
      if (threadIdx.x == 0) atomicExch(L.abort_flag, 1);
      return;
    }
  }
  XF* const s_own = sline + warp * L.line_stride;            // this warp's region
  XF* const t_own = s_own + L.line_ch;
  for (int t = threadIdx.x; t < nimg * 3; t += blockDim.x) sframe[t / 3][t % 3] = L.imgs[t / 3].frame[t % 3] != 0;
  if (threadIdx.x == 0) {
    srowa[0] = 0;
    for (int i = 0; i < nimg; ++i) srowa[i + 1] = srowa[i] + L.imgs[i].nm * L.imgs[i].ns;
  }
  // decay tables [image][axis][j] in global memory (CTA 0; the grid barrier
  // below publishes them)
  for (int t = threadIdx.x; blockIdx.x == 0 && t < nimg * 3 * kTab; t += blockDim.x) {
    const int i = t / (3 * kTab), ax = (t / kTab) % 3, j = t % kTab;
    const Img2D& I = L.imgs[i];
    const double c = ax == 0 ? I.cf : (ax == 1 ? I.cs : I.cm);
    const int len = ax == 0 ? I.nf : (ax == 1 ? I.ns : I.nm);
    const int Pseg = F32 && ax < 2 ? I.pf[ax] : (len + I.g[ax] - 1) / I.g[ax], Pw = (len + 31) >> 5;
    const double k = j < kTabSeg ? (double)j
                   : (j < kTabWarp ? (double)Pseg * (double)(1 << (j - kTabSeg))
                                   : (double)Pw * (double)(1 << (j - kTabWarp)));
    L.tab[t] = c_decay(k, c, XF{});
  }
  auto tab = [&](int i, int ax) -> const XF* { return L.tab + (i * 3 + ax) * kTab; };
  // u = v = 1 / N  (the initialisation of Algorithm 2), or a warm start
  for (int i = 0; i < nimg && F32; ++i) {
    const Img2D& I = L.imgs[i];
    init_f32(I, I.f_init, I.U32, I.U32F);
    init_f32(I, I.g_init, I.V32[0], I.V32F[0]);
  }
  for (int i = 0; i < nimg && !F32; ++i) {
    const Img2D& I = L.imgs[i];
    const int64_t N = (int64_t)I.nf * I.nm * I.ns;
    const XF init = xf_norm((float)(1.0 / (double)N), 0);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
      I.U[p] = I.f_init ? xf_from_log(I.f_init[p]) : init;
      I.V[0][p] = I.g_init ? xf_from_log(I.g_init[p]) : init;
    }
  }
  if (!grid_barrier(L, gen, &sok)) return;

  const int rows = srow[nimg], tiles = stile[nimg], mids = smid[nimg];
  // middle pass of a half-step (3D images): Z = (I (x) K_m (x) I) Y, one CTA
  // per tile of 8 columns of one slab; Z is the image's R buffer
  auto mid_pass = [&]() -> bool {
    for (int t = blockIdx.x; t < mids; t += gridDim.x) {
      const int i = owner(smid, nimg, t);
      if (sstate[i]) continue;   // CTA-uniform
      const Img2D& I = L.imgs[i];
      const TileMap M(I.g[2], I.nm);
      const int ntf = (I.nf + M.TW - 1) / M.TW;
      const int tt = t - smid[i];
      const int64_t base = (int64_t)(tt / ntf) * I.nf * I.nm;   // the slab
      const int col0 = (tt % ntf) * M.TW;
      col_tile_scan(I.Y + base, I.nf, I.nm, col0, M, tab(i, 2), sframe[i][2], sline, L.line_stride);
      const int c = M.col();
      if (col0 + c < I.nf) {
        const XF* sc = M.line(sline, L.line_stride, c);
        ChunkPos q(M.row0(), M.P, M.dr);
        for (int r = M.row0(); r < I.nm; r += M.dr, q.next())
          I.R[base + (int64_t)r * I.nf + col0 + c] = sc[q.pos()];
      }
      __syncthreads();   // the tile's shared memory is reused by the next tile
    }
    return grid_barrier(L, gen, &sok);
  };

  for (int64_t ell = 0;; ++ell) {
    const int par = (int)(ell & 1);
    __syncthreads();
    bool any = false;
    for (int i = 0; i < nimg; ++i) any |= ld_relaxed(L.imgs[i].stop) == 0;
    if (!any) break;
    for (int i = threadIdx.x; i < nimg; i += blockDim.x) sstate[i] = ld_relaxed(L.imgs[i].stop) == 0 ? 0 : 2;
    __syncthreads();
    // ---- v-half, fast pass: Y = (I (x) K_f) U
    for (int t = gw; t < rows; t += nw) {
      const int i = owner(srow, nimg, t);
      if (sstate[i]) continue;
      const Img2D& I = L.imgs[i];
      if (F32)
        row_f32(I, I.U32, I.U32F, t - srow[i], tab(i, 0), reinterpret_cast<float*>(sline) + warp * 32 * 32);
      else
        row_pass(I.U, I.Y, I.nm * I.ns, (t - srow[i]) * (32 / I.g[0]), I.nf, I.g[0], tab(i, 0), sframe[i][0],
                 s_own, t_own);
    }
    if (!grid_barrier(L, gen, &sok)) return;
    if (L.any3d && !mid_pass()) return;
    // ---- v-half, slow pass: y = (K_s (x) I) Z, v_new = b / y, error partials
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int i = owner(stile, nimg, t);
      if (sstate[i]) continue;   // CTA-uniform
      const Img2D& I = L.imgs[i];
      const int W = I.nf * I.nm;   // points of a slab: the slow lines' stride
      const TileMap M(I.g[1], I.ns);
      const int tile = t - stile[i];
      const int col0 = tile * M.TW;
      float eh = 0.f, el = 0.f;
      if (F32)
        col_f32(I, tile, I.b, L.in_f32, I.V32[par], I.V32F[par], I.V32[par ^ 1], I.V32F[par ^ 1], true, tab(i, 1),
                reinterpret_cast<float*>(sline), eh, el);
      else
        col_tile_scan(I.nm > 1 ? I.R : I.Y, W, I.ns, col0, M, tab(i, 1), sframe[i][1], sline, L.line_stride);
      XF* Vn = I.V[par ^ 1];
      const int c = M.col();
      if (!F32 && col0 + c < W) {
        const XF* sc = M.line(sline, L.line_stride, c);
        const int r0 = M.row0();
        const int dr = M.dr;
        ChunkPos q(r0, M.P, dr);
        for (int rb = r0; rb < I.ns; rb += dr * kBatch) {
          float mb[kBatch];
          XF vb[kBatch];
#pragma unroll
          for (int b = 0; b < kBatch; ++b)
            if (rb + dr * b < I.ns) {
              const int64_t p = (int64_t)(rb + dr * b) * W + col0 + c;
              mb[b] = load_m(I.b, p, L.in_f32);
              vb[b] = I.V[par][p];
            }
#pragma unroll
          for (int b = 0; b < kBatch; ++b, q.next())
            if (rb + dr * b < I.ns) {
              const int64_t p = (int64_t)(rb + dr * b) * W + col0 + c;
              const XF y = sc[q.pos()];
              const float m = mb[b];
              Vn[p] = m > 0.f ? xf_norm(__fdividef(m, y.m), -y.e) : XF{0.f, kZeroExp};
              const float pv = c_to(c_mul(vb[b], y), 0);   // v_old (K^T u) at p
              df_add(eh, el, fabsf(pv - m), 0.f);
            }
        }
      }
      cta_sum_df(eh, el, sred);
      if (threadIdx.x == 0) {
        I.errp[2 * tile] = eh;
        I.errp[2 * tile + 1] = el;
      }
    }
    if (!grid_barrier(L, gen, &sok)) return;
    // ---- decisions (every CTA, identical fixed-order sums)
    for (int i = warp; i < nimg; i += kWarps2) {
      if (sstate[i]) continue;
      const Img2D& I = L.imgs[i];
      float h = 0.f, l = 0.f;
      const int nt = (I.nf * I.nm + I.tw_s - 1) / I.tw_s;
      // lane sums tiles lane, lane + 32, ... in that order; four loads in
      // flight per lane (a zero pair past the end adds nothing)
      for (int c0 = lane; c0 < nt; c0 += 128) {
        float eh[4], el[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c0 + 32 * u;
          eh[u] = c < nt ? __ldcg(I.errp + 2 * c) : 0.f;
          el[u] = c < nt ? __ldcg(I.errp + 2 * c + 1) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) df_add(h, l, eh[u], el[u]);
      }
      warp_sum_df(h, l);
      if (lane == 0) {
        const double err = (double)h + (double)l;
        const bool numeric = !isfinite(err);
        const bool stop = numeric || err <= I.tol || ell >= I.itr_max;
        if (stop) {
          sstate[i] = 1;
          if (blockIdx.x == 0) {
            L.results[i].err = err;
            L.results[i].iters = ell;
            L.results[i].status = numeric ? FS1_ENUMERIC : (err <= I.tol ? FS1_OK : FS1_ENOTCONV);
          }
        }
      }
    }
    __syncthreads();
    // ---- u-half, fast pass: Y = (I (x) K_f) v_new
    for (int t = gw; t < rows; t += nw) {
      const int i = owner(srow, nimg, t);
      if (sstate[i]) continue;
      const Img2D& I = L.imgs[i];
      if (F32)
        row_f32(I, I.V32[par ^ 1], I.V32F[par ^ 1], t - srow[i], tab(i, 0),
                reinterpret_cast<float*>(sline) + warp * 32 * 32);
      else
        row_pass(I.V[par ^ 1], I.Y, I.nm * I.ns, (t - srow[i]) * (32 / I.g[0]), I.nf, I.g[0], tab(i, 0),
                 sframe[i][0], s_own, t_own);
    }
    if (!grid_barrier(L, gen, &sok)) return;
    if (L.any3d && !mid_pass()) return;
    // ---- u-half, slow pass: u = a / ((K_s (x) I) Z)
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int i = owner(stile, nimg, t);
      if (sstate[i]) continue;   // CTA-uniform
      const Img2D& I = L.imgs[i];
      const int W = I.nf * I.nm;
      const TileMap M(I.g[1], I.ns);
      const int col0 = (t - stile[i]) * M.TW;
      if (F32) {
        float eh = 0.f, el = 0.f;
        col_f32(I, t - stile[i], I.a, L.in_f32, nullptr, nullptr, I.U32, I.U32F, false, tab(i, 1),
                reinterpret_cast<float*>(sline), eh, el);
        continue;   // col_f32 ends with a block barrier
      }
      col_tile_scan(I.nm > 1 ? I.R : I.Y, W, I.ns, col0, M, tab(i, 1), sframe[i][1], sline, L.line_stride);
      const int c = M.col();
      if (col0 + c < W) {
        const XF* sc = M.line(sline, L.line_stride, c);
        const int r0 = M.row0();
        const int dr = M.dr;
        ChunkPos q(r0, M.P, dr);
        for (int rb = r0; rb < I.ns; rb += dr * kBatch) {
          float mb[kBatch];
#pragma unroll
          for (int b = 0; b < kBatch; ++b)
            if (rb + dr * b < I.ns) mb[b] = load_m(I.a, (int64_t)(rb + dr * b) * W + col0 + c, L.in_f32);
#pragma unroll
          for (int b = 0; b < kBatch; ++b, q.next())
            if (rb + dr * b < I.ns) {
              const int64_t p = (int64_t)(rb + dr * b) * W + col0 + c;
              const XF y = sc[q.pos()];
              I.U[p] = mb[b] > 0.f ? xf_norm(__fdividef(mb[b], y.m), -y.e) : XF{0.f, kZeroExp};
            }
        }
      }
      __syncthreads();   // the tile's shared memory is reused by the next tile
    }
    // images that stop here keep v_old = V[par]
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < nimg; i += blockDim.x)
        if (sstate[i] == 1) L.imgs[i].stop[0] = 1 + par;
    if (!grid_barrier(L, gen, &sok)) return;
  }

  // FP32 path: u and the returned v into the extended-range arrays
  if (F32) {
    for (int i = 0; i < nimg; ++i) to_xf(L.imgs[i], (ld_relaxed(L.imgs[i].stop) - 1) & 1);
    if (!grid_barrier(L, gen, &sok)) return;
  }
  // optional potentials out: log u and log v of the returned iterate (before
  // the cost passes, which reuse the v buffer in 3D)
  for (int i = 0; i < nimg; ++i) {
    const Img2D& I = L.imgs[i];
    if (!I.f_out && !I.g_out) continue;
    const int k = (ld_relaxed(I.stop) - 1) & 1;
    const int64_t N = (int64_t)I.nf * I.nm * I.ns;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
      if (I.f_out) I.f_out[p] = xf_log(I.U[p]);
      if (I.g_out) I.g_out[p] = xf_log(I.V[k][p]);
    }
  }

  // ---- transport cost: sum over axes a of h_a u . (K with the distance-
  // weighted K_a^(c) on axis a) v
  // rows: Y = (I (x) K_f^(c)) v (weighted); V1 = (I (x) K_f) v in the free v buffer
  const int wrows = srowa[nimg];
  for (int t = gw; t < wrows; t += nw) {
    const int i = owner(srowa, nimg, t);
    const Img2D& I = L.imgs[i];
    const int k = (ld_relaxed(I.stop) - 1) & 1;
    const int64_t o = (int64_t)(t - srowa[i]) * I.nf;
    line_scan_global<true>(I.V[k] + o, I.Y + o, I.R + o, 1, I.nf, tab(i, 0));
    __syncwarp();
    line_scan_global<false>(I.V[k] + o, I.V[k ^ 1] + o, I.R + o, 1, I.nf, tab(i, 0));
  }
  if (!grid_barrier(L, gen, &sok)) return;
  // middle lines (3D): R = K_m Y, V[k] = K_m^(c) V1, Y = K_m V1
  if (L.any3d) {
    const int mlines = smidl[nimg];
    for (int t = gw; t < mlines; t += nw) {
      const int i = owner(smidl, nimg, t);
      const Img2D& I = L.imgs[i];
      const int k = (ld_relaxed(I.stop) - 1) & 1;
      const int tl = t - smidl[i];
      const int64_t o = (int64_t)(tl / I.nf) * I.nf * I.nm + tl % I.nf;
      line_scan_global<false>(I.Y + o, I.R + o, I.R + o, I.nf, I.nm, tab(i, 2));
      __syncwarp();
      line_scan_global<true>(I.V[k ^ 1] + o, I.V[k] + o, I.V[k] + o, I.nf, I.nm, tab(i, 2));
      __syncwarp();
      line_scan_global<false>(I.V[k ^ 1] + o, I.Y + o, I.Y + o, I.nf, I.nm, tab(i, 2));
    }
    if (!grid_barrier(L, gen, &sok)) return;
  }
  // slow lines: 2D:  h_f u.(K_s Y) + h_s u.(K_s^(c) V1)
  //             3D:  h_f u.(K_s R) + h_m u.(K_s V[k]) + h_s u.(K_s^(c) Y)
  const int slines = scol[nimg];
  for (int t = gw; t < slines; t += nw) {
    const int i = owner(scol, nimg, t);
    const Img2D& I = L.imgs[i];
    const int k = (ld_relaxed(I.stop) - 1) & 1;
    const int W = I.nf * I.nm;
    const int col = t - scol[i];
    XF* const out = I.nm > 1 ? I.V[k ^ 1] : I.R;
    double acc = 0.0;
    auto accumulate = [&](double hax) {
      __syncwarp();
      for (int r = lane; r < I.ns; r += 32) {
        const int64_t p = (int64_t)r * W + col;
        const XF w = out[p], u = I.U[p];
        acc += hax * ldexp((double)u.m * (double)w.m, u.e + w.e);
      }
      __syncwarp();
    };
    if (I.nm > 1) {
      line_scan_global<false>(I.R + col, out + col, out + col, W, I.ns, tab(i, 1));
      accumulate(I.hf);
      line_scan_global<false>(I.V[k] + col, out + col, out + col, W, I.ns, tab(i, 1));
      accumulate(I.hm);
      line_scan_global<true>(I.Y + col, out + col, out + col, W, I.ns, tab(i, 1));
      accumulate(I.hs);
    } else {
      line_scan_global<false>(I.Y + col, out + col, out + col, W, I.ns, tab(i, 1));
      accumulate(I.hf);
      line_scan_global<true>(I.V[k ^ 1] + col, out + col, out + col, W, I.ns, tab(i, 1));
      accumulate(I.hs);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) I.wp[col] = acc;
  }
  if (!grid_barrier(L, gen, &sok)) return;
  if (blockIdx.x == 0) {
    for (int i = warp; i < nimg; i += kWarps2) {
      const Img2D& I = L.imgs[i];
      double s = 0.0;
      for (int c = lane; c < I.nf * I.nm; c += 32) s += __ldcg(I.wp + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) L.results[i].w = L.results[i].status == FS1_ENUMERIC ? NAN : s;
    }
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Lanes that share a line of L points with c = h / eps: the fewest of 8, 16,
// 32 that keep P = ceil(L / G) <= 16 points per lane and keep the FP32-frame
// scan (c P <= 40) when 32 lanes would allow it.  Fewer lanes per line mean a
// shorter lane scan and more points per lane for short lines.
int line_lanes(int L, double c) {
  const bool frame32 = c * ((L + 31) / 32) <= 40.0;
  for (int G = 8; G < 32; G *= 2) {
    const int P = (L + G - 1) / G;
    if (P <= 16 && (!frame32 || c * P <= 40.0)) return G;
  }
  return 32;
}

// bytes of the FP32 state of an image (values, frames)
size_t f32_bytes(const PairDesc& d) {
  const size_t lp = ((size_t)d.n_fast + kBlk - 1) / kBlk * kBlk, ns = (size_t)d.n_slow;
  const size_t nb = (ns + kBlk - 1) / kBlk;
  return 4 * align256(sizeof(float) * ns * lp) + 3 * align256(sizeof(int) * nb * lp) +
         align256(sizeof(int) * ns * (lp / kBlk));
}

}  // namespace

// Launch class of a grid image.  The general path sizes every CTA's staging
// for the widest layout of its launch: one image that scans an axis point by
// point in extended range doubles the per-warp region of all of them and
// halves the CTAs per SM, so such images get a launch of their own (27 images
// of sides 513-1024 from the serving mix: 2.95 s in one launch, 2.11 s in
// two).  The FP32 path takes images its lane chunks hold (c P <= 64 on both
// axes) that the general path would scan point by point (c P > 40 there):
// same-box A/B on batches of 600^2 to 1024^2 images, it ran 1.3-1.7x faster
// than the per-point scans but 0.8-0.9x the general path's FP32-frame scans.
int solve2d_class(const PairDesc& d) {
  const int len[3] = {(int)d.n_fast, (int)d.n_slow, (int)d.n_mid};
  const double c[3] = {d.h_fast / d.eps, d.h_slow / d.eps, d.n_mid > 1 ? d.h_mid / d.eps : 0.0};
  bool per_point = false, f32 = d.n_mid == 1 && d.n_fast <= kMaxLine2D && d.n_slow <= kMaxLine2D;
  for (int ax = 0; ax < 3; ++ax) {
    if (len[ax] < 2) continue;
    const int Go = line_lanes(len[ax], c[ax]);
    per_point = per_point || c[ax] * ((len[ax] + Go - 1) / Go) > 40.0;
    int G, P;
    f32_geom(len[ax], G, P);
    f32 = f32 && c[ax] * P <= kF32MaxNats;
  }
  return !per_point ? 0 : (f32 ? 2 : 1);
}

int solve2d_f32_ok(const PairDesc& d) { return solve2d_class(d) == 2 ? 1 : 0; }

size_t solve2d_workspace(const PairDesc* d, int count) {
  size_t b = align256(sizeof(Img2D) * count) + 5 * align256(sizeof(int) * (count + 1)) + 256 + 256 +
             align256(sizeof(XF) * 3 * kTab * count);
  for (int i = 0; i < count; ++i) {
    const size_t W = (size_t)d[i].n_fast * d[i].n_mid;
    const size_t n = W * d[i].n_slow;
    b += 5 * align256(sizeof(XF) * n) + align256(sizeof(float) * 2 * W) + align256(sizeof(double) * W) + 256;
    if (solve2d_f32_ok(d[i])) b += f32_bytes(d[i]);
  }
  return b;
}

int launch_solve_2d(const PairDesc* d, int count, int in_f32, PairResult* results, void* ws, size_t ws_bytes,
                    long long spin_cap, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count < 1 || count > kMaxImg2D) return FS1_EINVAL;
  for (int i = 0; i < count; ++i)
    if (d[i].n_fast > kMaxLine2D || d[i].n_mid > kMaxLine2D || d[i].n_slow > kMaxLine2D) return FS1_EUNSUPPORTED;
  if (solve2d_workspace(d, count) > ws_bytes) return FS1_ENOMEM;
  char* p = (char*)ws;
  Img2D* d_imgs = (Img2D*)p;
  p += align256(sizeof(Img2D) * count);
  int* d_row = (int*)p;
  p += align256(sizeof(int) * (count + 1));
  int* d_col = (int*)p;
  p += align256(sizeof(int) * (count + 1));
  int* d_tile = (int*)p;
  p += align256(sizeof(int) * (count + 1));
  int* d_mid = (int*)p;
  p += align256(sizeof(int) * (count + 1));
  int* d_midl = (int*)p;
  p += align256(sizeof(int) * (count + 1));
  unsigned long long* d_bar = (unsigned long long*)p;
  p += 256;
  int* d_abort = (int*)p;
  p += 256;
  XF* d_tab = (XF*)p;
  p += align256(sizeof(XF) * 3 * kTab * count);
  std::vector<Img2D> imgs(count);
  std::vector<int> row(count + 1, 0), col(count + 1, 0), tile(count + 1, 0), mid(count + 1, 0), midl(count + 1, 0);
  int any3d = 0;
  int pp_max = 1;
  bool any_ext = false;   // some axis takes the per-point extended-range scan (XF partials)
  char* stops = nullptr;
  // the FP32 block-frame path when every image of the call takes it
  bool f32 = true;
  for (int i = 0; i < count; ++i) f32 = f32 && solve2d_f32_ok(d[i]);
  size_t smem_f32 = (size_t)kWarps2 * 32 * 32 * sizeof(float);   // the fast pass's backward partials
  for (int i = 0; i < count; ++i) {
    const PairDesc& D = d[i];
    Img2D I{};
    I.a = D.a;
    I.b = D.b;
    I.nf = (int)D.n_fast;
    I.nm = (int)D.n_mid;
    I.ns = (int)D.n_slow;
    I.cf = D.h_fast / D.eps;
    I.cm = D.n_mid > 1 ? D.h_mid / D.eps : 0.0;
    I.cs = D.h_slow / D.eps;
    I.hf = D.h_fast;
    I.hm = D.h_mid;
    I.hs = D.h_slow;
    I.tol = D.tol;
    I.itr_max = D.itr_max;
    I.f_init = D.f_init;
    I.g_init = D.g_init;
    I.f_out = D.f_out;
    I.g_out = D.g_out;
    const size_t W = (size_t)I.nf * I.nm;
    const size_t n = W * I.ns;
    I.U = (XF*)p; p += align256(sizeof(XF) * n);
    I.V[0] = (XF*)p; p += align256(sizeof(XF) * n);
    I.V[1] = (XF*)p; p += align256(sizeof(XF) * n);
    I.Y = (XF*)p; p += align256(sizeof(XF) * n);
    I.R = (XF*)p; p += align256(sizeof(XF) * n);
    I.errp = (float*)p; p += align256(sizeof(float) * 2 * W);
    I.wp = (double*)p; p += align256(sizeof(double) * W);
    I.stop = (int*)p;
    if (!stops) stops = p;
    p += 256;
    const int len[3] = {I.nf, I.ns, I.nm};
    const double cax[3] = {I.cf, I.cs, I.cm};
    for (int ax = 0; ax < 3; ++ax) {
      I.g[ax] = line_lanes(len[ax], cax[ax]);
      const int P = (len[ax] + I.g[ax] - 1) / I.g[ax];
      I.frame[ax] = cax[ax] * P <= 40.0 ? 1 : 0;
      if (ax < 2 || I.nm > 1) {
        pp_max = std::max(pp_max, P | 1);
        any_ext = any_ext || !I.frame[ax];
      }
    }
    if (f32) {
      I.lp = (I.nf + kBlk - 1) / kBlk * kBlk;
      for (int ax = 0; ax < 3; ++ax) f32_geom(len[ax], I.g[ax], I.pf[ax]);
      const size_t nb = ((size_t)I.ns + kBlk - 1) / kBlk, np = (size_t)I.ns * I.lp;
      I.U32 = (float*)p; p += align256(sizeof(float) * np);
      I.V32[0] = (float*)p; p += align256(sizeof(float) * np);
      I.V32[1] = (float*)p; p += align256(sizeof(float) * np);
      I.Y32 = (float*)p; p += align256(sizeof(float) * np);
      I.U32F = (int*)p; p += align256(sizeof(int) * nb * I.lp);
      I.V32F[0] = (int*)p; p += align256(sizeof(int) * nb * I.lp);
      I.V32F[1] = (int*)p; p += align256(sizeof(int) * nb * I.lp);
      I.Y32F = (int*)p; p += align256(sizeof(int) * I.ns * (I.lp / kBlk));
      // slow pass tile: values [TW][G][P + 1], frames [ns][TW / 8], lane frames [TW][G]
      const int TW = kTileCols * (32 / I.g[1]);
      smem_f32 = std::max(smem_f32, sizeof(float) * ((size_t)TW * f32_cs(I.g[1], I.pf[1]) +
                                                     (size_t)(I.ns + I.ns / I.pf[1]) * (TW / kBlk) +
                                                     (size_t)TW * I.g[1]));
    } else if (solve2d_f32_ok(D)) {
      p += f32_bytes(D);   // the workspace counts it; this call takes the general path
    }
    I.tw_s = kTileCols * (32 / I.g[1]);
    I.tw_m = kTileCols * (32 / I.g[2]);
    const int rpw = 32 / I.g[0];   // rows a warp takes at once
    row[i + 1] = row[i] + (I.nm * I.ns + rpw - 1) / rpw;
    col[i + 1] = col[i] + (int)W;
    tile[i + 1] = tile[i] + ((int)W + I.tw_s - 1) / I.tw_s;
    mid[i + 1] = mid[i] + (I.nm > 1 ? I.ns * ((I.nf + I.tw_m - 1) / I.tw_m) : 0);
    midl[i + 1] = midl[i] + (I.nm > 1 ? I.nf * I.ns : 0);
    any3d |= I.nm > 1;
    imgs[i] = I;   // after every field is set
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < count && e == cudaSuccess; ++i) e = cudaMemsetAsync(imgs[i].stop, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(Img2D) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_row, row.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_col, col.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tile, tile.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mid, mid.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_midl, midl.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bar, 0, 512, st);
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: 2D setup failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  // per-warp region: the staged line (CH XF) and its backward partials (CH XF
  // for the extended-range scan, CH floats for the frame scan), + 2 so that
  // the stride is 2 mod 16 and the tile's warps start in different banks
  const int line_ch = 32 * pp_max;
  const int line_stride = line_ch + (any_ext ? line_ch : line_ch / 2) + 2;
  const size_t smem = f32 ? smem_f32 : sizeof(XF) * (size_t)kWarps2 * line_stride;
  Launch2D L{d_imgs, results, count, in_f32, d_row, d_col, d_tile, d_mid, d_midl, any3d, line_stride, line_ch,
             d_tab, d_bar, d_abort, spin_cap};
  const void* kfn = f32 ? (const void*)fs1_solve2d_kernel<true> : (const void*)fs1_solve2d_kernel<false>;
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads2, smem);
  if (e != cudaSuccess || per_sm < 1) {
    fprintf(stderr, "fs1: 2D kernel does not fit (%zu B shared memory): %s\n", smem, cudaGetErrorString(e));
    return FS1_EUNSUPPORTED;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = per_sm * sms;
  void* args[] = {&L};
  e = cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kThreads2), args, smem, st);
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: 2D launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

}  // namespace fs1
