// fs1_stream.cu -- stabilised 1D FS-1 for a pair too large to keep on chip.
//
// The team kernel (fs1_team.cuh) holds a pair's state in the registers and
// shared memory of co-resident CTAs; a pair beyond that capacity runs here
// with its state in device memory.  The grid is cut into chunks of 8192
// points (one 512-thread CTA, 16 points per thread).  One half-step of
// Algorithm 1 is ONE launch over the chunks:
//   carries : every chunk reads its forward carry (the value at the point
//             before it) and backward carry (at its last point) of the
//             input, which the previous launch's last chunk formed by one
//             scan over all chunks' (decay, value) aggregates; they are
//             complete when the launch starts, so no chunk waits for another;
//   half    : the chunk loads its input (128-bit, coalesced), forms the thread
//             carries with the team kernel's in-CTA scan plus its chunk
//             carries, runs the recurrences of Section 3, eq. "recursion",
//             divides the masses by them (the psi or phi update of
//             Algorithm 1), stores the output with its chunk aggregates and
//             (v-half) the chunk's marginal-error partial;
//   last    : the last chunk to finish (a ticket counter, no waiting) takes
//             the while condition of Algorithm 1 after a v-half (the error
//             partials summed in FP64 in chunk order), advances the
//             iteration count after a u-half, and scans the chunk aggregates
//             of the launch's output into the carries the next launch reads.
// Every launch first reads the stop flag and returns once the loop has
// ended, so the host issues iterations in captured blocks and reads the flag
// between blocks.  Up to kMaxStreamPairs pairs share the launches: the grid
// covers the chunks of all of them (each chunk finds its pair from the
// chunk offsets), every pair keeps its own loop state and last-chunk ticket,
// and a pair that stops lowers a count of active pairs that the host polls.
//
// State: per point an FP32 value relative to a power-of-two frame shared by
// the 16 points of a thread (4 + 0.25 bytes per point), as the team kernel
// holds its registers.  Within a chunk, thread t's points 4q .. 4q + 3 sit at
// float4 index q * 512 + t, so every 128-bit access of a warp is contiguous.
// The masses are copied once into the same order (FP32).  The transport cost
// is formed as in the team kernel with the distance-weighted operator
// (OpDist): chunk aggregates, a sequential scan over the chunks, and the
// per-chunk sums of u (A + B) in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fs1_team.cuh"

namespace fs1 {

namespace {

constexpr int kST = 512;                 // threads of a chunk's CTA
constexpr int kSW = kST / 32;            // its warps
constexpr int kSE = 16;                  // points per thread per chunk
constexpr int kChunk = kST * kSE;        // points per chunk (one CTA)

struct StreamState {
  long long ell;   // completed iterations
  int stop;        // 1 once the loop has ended
  int status;      // FS1_OK, FS1_ENOTCONV, FS1_ENUMERIC or FS1_ETIMEOUT
  int par;         // v buffer holding the accepted v
  unsigned done;   // chunks of the running launch that have finished
  double err;      // marginal error of the last v-half
  int fail;        // 1: a chunk's staging copy did not complete in its bounded wait
};

struct StreamArgs {
  int nch;               // chunks
  int64_t n;             // points
  double c;              // h / eps
  float lamf;            // lam = e^{-c} in FP32
  double h, tol;
  long long itr_max;
  const void* a;         // the caller's masses (natural order)
  const void* b;
  int in_f32;
  float* AW;             // [nch * kChunk] masses in run order, zeros past n
  float* BW;
  float* U;              // [nch * kChunk] values relative to their run's frame
  float* V[2];
  int* FU;               // [nch * kST] frames of the runs
  int* FV[2];
  XF* agg_f[3];          // chunk aggregates of U, V[0], V[1]: forward (value at the chunk's
  XF* agg_b[3];          // last point) and backward (value at the point before its first)
  XF* car_f[3];          // chunk carries of U, V[0], V[1]: forward (value at the point before
  XF* car_b[3];          // the chunk, from the chunks before it) and backward (at its last point,
                         // from the chunks after it)
  XF* dec;               // [nch] lam^{kChunk d}
  DecayTables<XF>* tabs; // the in-CTA decay tables (written once by the init kernel)
  float* errp;           // [2 nch] compensated error partials
  PairC<XF>* dagg_f;     // cost phase: distance-weighted chunk aggregates and carries
  PairC<XF>* dagg_b;
  PairC<XF>* dcar_f;
  PairC<XF>* dcar_b;
  double* costp;         // [nch]
  StreamState* st;
  PairResult* result;
  const double* f_init;
  const double* g_init;
  double* f_out;
  double* g_out;
};

// pairs of one batch of launches (the kernel parameter holds their arguments)
constexpr int kMaxStreamPairs = 8;
struct StreamBatch {
  int npairs;
  int* nactive;                     // pairs whose loop has not ended
  int choff[kMaxStreamPairs + 1];   // first chunk (CTA) of each pair in the grid
  StreamArgs A[kMaxStreamPairs];
};
static_assert(sizeof(StreamBatch) <= 4000, "kernel parameter size");

// decay tables of a CTA whose threads hold Eeff "points" of decay exp(-c) each
__device__ void fill_tables(DecayTables<XF>& tb, double c, int Eeff) {
  for (int i = threadIdx.x; i < 66; i += blockDim.x) {
    if (i < 33) {
      tb.dt[i] = c_decay((double)Eeff * i, c, XF{});
      tb.dtf[i] = (float)exp(-(double)Eeff * i * c);
    } else {
      tb.dw[i - 33] = c_decay(32.0 * Eeff * (i - 33), c, XF{});
    }
  }
  if (threadIdx.x == 0) tb.narrow = (c * 32.0 * Eeff <= 40.0) ? 1 : 0;
}

// the 16 values of thread t's run in chunk ch (float4 index q 512 + t)
__device__ __forceinline__ void ld_run(const float* X, int ch, int t, float (&x)[kSE]) {
  const float4* p = reinterpret_cast<const float4*>(X + (size_t)ch * kChunk) + t;
#pragma unroll
  for (int q = 0; q < kSE / 4; ++q) {
    const float4 v = p[q * kST];
    x[4 * q] = v.x;
    x[4 * q + 1] = v.y;
    x[4 * q + 2] = v.z;
    x[4 * q + 3] = v.w;
  }
}
__device__ __forceinline__ void st_run(float* X, int ch, int t, const float (&x)[kSE]) {
  float4* p = reinterpret_cast<float4*>(X + (size_t)ch * kChunk) + t;
#pragma unroll
  for (int q = 0; q < kSE / 4; ++q) p[q * kST] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}
// values given relative to frame F, renormalised so that the largest lies in
// [0.5, 1); returns the run's frame (kZeroExp for an all-zero run)
__device__ __forceinline__ int normalise_run(float (&x)[kSE], int F) {
  int em = kZeroExp;
#pragma unroll
  for (int k = 0; k < kSE; ++k) em = max(em, fexp(x[k]));
  if (em == kZeroExp) return kZeroExp;
  const float s = pow2f(-em);
#pragma unroll
  for (int k = 0; k < kSE; ++k) x[k] *= s;
  return F + em;
}

// Totals of the CTA from its threads' aggregates: forward to the CTA's last
// point, backward to the point before its first point (every thread calls;
// the totals are valid in warp 0).  sw: 32 entries of shared memory.
template <class Op>
__device__ void cta_totals(typename Op::T af, typename Op::T ab, const DecayTables<XF>& tb,
                           typename Op::T* sw, typename Op::T& tf, typename Op::T& tbk) {
  using T = typename Op::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T wf = warp_sum_c(Op::prop(af, tb.dt[31 - lane], (float)(kSE * (31 - lane))));
  const T wb = warp_sum_c(Op::prop(ab, tb.dt[lane], (float)(kSE * lane)));
  if (lane == 0) {
    sw[warp] = wf;
    sw[kSW + warp] = wb;
  }
  __syncthreads();
  if (warp == 0) {
    T xf = Op::zero(), xb = Op::zero();
    if (lane < kSW) {
      xf = Op::prop(sw[lane], tb.dw[kSW - 1 - lane], (float)(32 * kSE * (kSW - 1 - lane)));
      xb = Op::prop(sw[kSW + lane], tb.dw[lane], (float)(32 * kSE * lane));
    }
    tf = warp_sum_c(xf);
    tbk = warp_sum_c(xb);
  }
}

// compensated CTA sum of an FP32 pair in a fixed order (valid in every thread)
__device__ void cta_sum_pair(float& h, float& l, float* red) {
  warp_sum_df(h, l);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[2 * warp] = h;
    red[2 * warp + 1] = l;
  }
  __syncthreads();
  h = 0.f;
  l = 0.f;
  for (int w = 0; w < kSW; ++w) df_add(h, l, red[2 * w], red[2 * w + 1]);
}

__device__ __forceinline__ XF xf_of_log(double x) {
  if (!(x > -INFINITY)) return XF{0.f, kZeroExp};
  const double t = x * 1.4426950408889634;
  const double e = floor(t);
  return xf_norm((float)exp2(t - e), (int)e);
}
__device__ __forceinline__ double log_of(float m, int F) {
  return m > 0.f ? log((double)m) + (double)F * 0.6931471805599453 : -INFINITY;
}

// forward (to the run's last point) and backward (from the point before its
// first) totals of a run's values with decay lam between points
__device__ __forceinline__ void run_aggregates(const float (&x)[kSE], float lam, float& af, float& ab) {
  float pw = 1.f;
  af = 0.f;
  ab = 0.f;
#pragma unroll
  for (int k = kSE - 1; k >= 0; --k) {
    af = af + pw * x[k];
    pw = pw * lam;
    ab = lam * (ab + x[k]);
  }
}

// The carries of every chunk of array src from its chunk aggregates, by one
// CTA: thread t takes the m consecutive chunks t m ..., the threads' block
// aggregates are joined by the team kernel's in-CTA scan with decay
// lam^{kChunk} per chunk (the tables tb are refilled for it), and each thread
// sweeps its block:
//   car_f[j] = lam^{kChunk} car_f[j - 1] + agg_f[j - 1],  car_f[0] = 0
//   car_b[j] = lam^{kChunk} car_b[j + 1] + agg_b[j + 1],  car_b[nch - 1] = 0
// (agg_f: the chunk's value at its last point; agg_b: at the point before
// its first).  Every thread of the CTA calls; the aggregates were written by
// other CTAs (read through L2).
__device__ __forceinline__ XF ldcg_xf(const XF* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return XF{v.x, __float_as_int(v.y)};
}

__device__ void chunk_carry_scan(const StreamArgs& A, int src, DecayTables<XF>& tb, XchgSmem<XF>& X) {
  const int tid = threadIdx.x;
  const int m = (A.nch + kST - 1) / kST;
  const int j0 = tid * m;
  const double cc = A.c * (double)kChunk;
  const XF d1 = c_decay(1.0, cc, XF{});
  const XF* AF = A.agg_f[src];
  const XF* AB = A.agg_b[src];
  __syncthreads();   // tb may still be read by the half-step's scans
  fill_tables(tb, cc, m);
  __syncthreads();
  XF af = XF{0.f, kZeroExp}, ab = XF{0.f, kZeroExp};
  for (int k = 0; k < m; ++k) af = c_add(c_mul(af, d1), j0 + k < A.nch ? ldcg_xf(AF + j0 + k) : XF{0.f, kZeroExp});
  for (int k = m - 1; k >= 0; --k) ab = c_add(c_mul(ab, d1), j0 + k < A.nch ? ldcg_xf(AB + j0 + k) : XF{0.f, kZeroExp});
  XF cf, cb;
  {
    TeamLaunch L{};
    TeamCtx tc{0, 0, 1, 0, nullptr};
    unsigned epoch = 0, xc = 0;
    int dec;
    exchange<OpPlain<XF>, XF, kSW>(L, tc, epoch, xc, af, ab, 0.f, m, tb, X, cf, cb, 0.f, 0.f, dec, nullptr, nullptr);
  }
  XF r = cf;
  for (int k = 0; k < m && j0 + k < A.nch; ++k) {
    A.car_f[src][j0 + k] = r;
    r = c_add(c_mul(r, d1), ldcg_xf(AF + j0 + k));
  }
  XF t = cb;
  for (int k = m - 1; k >= 0; --k) {
    if (j0 + k < A.nch) A.car_b[src][j0 + k] = t;
    if (j0 + k < A.nch) t = c_add(c_mul(t, d1), ldcg_xf(AB + j0 + k));
  }
}

// the carries of u after the init kernel (one CTA per pair)
__global__ void __launch_bounds__(kST, 1) stream_carry_kernel(StreamArgs A, int src) {
  __shared__ DecayTables<XF> tb;
  __shared__ XchgSmem<XF> X;
  if (threadIdx.x == 0) X.ok = 1;
  chunk_carry_scan(A, src, tb, X);
}

// masses in run order, u = v = 1/N (or the warm start), the chunk aggregates
// of u, the chunk decay table and the loop state
__global__ void __launch_bounds__(kST, 1) stream_init_kernel(StreamArgs A) {
  __shared__ DecayTables<XF> tb;
  __shared__ XF sw[2 * kSW];
  fill_tables(tb, A.c, kSE);
  __syncthreads();
  const int tid = threadIdx.x, ch = blockIdx.x;
  const int64_t g0 = (int64_t)ch * kChunk + (int64_t)tid * kSE;
  const int ne = (int)max((int64_t)0, min((int64_t)kSE, A.n - g0));
  float am[kSE], bm[kSE];
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    am[k] = k < ne ? (A.in_f32 ? ((const float*)A.a)[g0 + k] : (float)((const double*)A.a)[g0 + k]) : 0.f;
    bm[k] = k < ne ? (A.in_f32 ? ((const float*)A.b)[g0 + k] : (float)((const double*)A.b)[g0 + k]) : 0.f;
  }
  st_run(A.AW, ch, tid, am);
  st_run(A.BW, ch, tid, bm);
  // u and v of the run, each in one frame
  float u[kSE], v[kSE];
  int fu = kZeroExp, fv = kZeroExp;
  {
    XF xu[kSE], xv[kSE];
    const XF init = xf_norm((float)(1.0 / (double)A.n), 0);
#pragma unroll
    for (int k = 0; k < kSE; ++k) {
      xu[k] = xv[k] = XF{0.f, kZeroExp};
      if (k < ne) {
        xu[k] = A.f_init ? xf_of_log(A.f_init[g0 + k]) : init;
        xv[k] = A.g_init ? xf_of_log(A.g_init[g0 + k]) : init;
      }
      if (xu[k].m != 0.f) fu = max(fu, xu[k].e);
      if (xv[k].m != 0.f) fv = max(fv, xv[k].e);
    }
#pragma unroll
    for (int k = 0; k < kSE; ++k) {
      u[k] = xu[k].m != 0.f ? xu[k].m * pow2f(xu[k].e - fu) : 0.f;
      v[k] = xv[k].m != 0.f ? xv[k].m * pow2f(xv[k].e - fv) : 0.f;
    }
  }
  st_run(A.U, ch, tid, u);
  st_run(A.V[0], ch, tid, v);
  A.FU[(size_t)ch * kST + tid] = fu;
  A.FV[0][(size_t)ch * kST + tid] = fv;
  float af, ab;
  run_aggregates(u, A.lamf, af, ab);
  XF tf, tbk;
  cta_totals<OpPlain<XF>>(c_from(af, fu, XF{}), c_from(ab, fu, XF{}), tb, sw, tf, tbk);
  if (ch == 0 && tid == 0) *A.tabs = tb;
  if (tid == 0) {
    A.agg_f[0][ch] = tf;
    A.agg_b[0][ch] = tbk;
    A.dec[ch] = c_decay((double)kChunk * (double)ch, A.c, XF{});
  }
  if (ch == 0 && tid == 0) *A.st = StreamState{0, 0, FS1_OK, 0, 0u, NAN, 0};
}


// the decay tables of the launch, copied from global memory
__device__ __forceinline__ void copy_tables(DecayTables<XF>& tb, const DecayTables<XF>* g) {
  constexpr int nw = (int)(sizeof(DecayTables<XF>) / sizeof(int));
  static_assert(sizeof(DecayTables<XF>) % sizeof(int) == 0, "table size");
  const int* src = reinterpret_cast<const int*>(g);
  int* dst = reinterpret_cast<int*>(&tb);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
}

// One half-step over the chunks of the batch's pairs (vhalf 1: y = K^T u,
// v_new = b / y and the error of the accepted v; vhalf 0: y = K v, u = a / y).
// The chunk's masses (and, in a v-half, its accepted v) are staged in shared
// memory by bulk copies issued at the start, so that they arrive while the
// carries are formed; dynamic shared memory: kChunk floats per staged array.
constexpr unsigned kStageBytes = kChunk * sizeof(float);
__global__ void __launch_bounds__(kST, 2) stream_step_kernel(const __grid_constant__ StreamBatch B, int vhalf) {
  extern __shared__ __align__(16) float4 s_stage[];   // [masses | accepted v], kChunk / 4 each
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ DecayTables<XF> tb;
  __shared__ XchgSmem<XF> X;
  __shared__ XF sw[2 * kSW];
  __shared__ float sred[2 * kSW];
  __shared__ double sdred[kSW];
  __shared__ int sstop, spar, slast;
  int pr = 0;
  while (pr + 1 < B.npairs && B.choff[pr + 1] <= (int)blockIdx.x) ++pr;
  const StreamArgs& A = B.A[pr];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ch = (int)blockIdx.x - B.choff[pr];
  if (tid == 0) {
    sstop = A.st->stop;
    spar = A.st->par;
    X.ok = 1;
    mbar_init(&s_mbar);
  }
  copy_tables(tb, A.tabs);
  __syncthreads();
  if (sstop) return;
  const int par = spar;
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(&s_mbar, vhalf ? 2 * kStageBytes : kStageBytes);
    bulk_copy(s_stage, (vhalf ? A.BW : A.AW) + (size_t)ch * kChunk, kStageBytes, &s_mbar);
    if (vhalf) bulk_copy(s_stage + kChunk / 4, A.V[par] + (size_t)ch * kChunk, kStageBytes, &s_mbar);
  }
  // v-half: input u, output v[par ^ 1]; u-half: input the accepted v[par], output u
  const float* Xin = vhalf ? A.U : A.V[par];
  const int* Fin = vhalf ? A.FU : A.FV[par];
  const int src = vhalf ? 0 : 1 + par;
  float* Z = vhalf ? A.V[par ^ 1] : A.U;
  int* FZ = vhalf ? A.FV[par ^ 1] : A.FU;
  const int zsrc = vhalf ? 1 + (par ^ 1) : 0;
  const float lam = A.lamf;
  const size_t run = (size_t)ch * kST + tid;
  const XF zero = XF{0.f, kZeroExp};

  float x[kSE];
  ld_run(Xin, ch, tid, x);
  const int e = Fin[run];
  // chunk carries of the input (formed by the previous launch's last chunk)
  const XF CF = A.car_f[src][ch], CB = A.car_b[src][ch];
  // thread carries: the in-CTA scan, plus the chunk carries placed at the thread
  XF cf, cb;
  {
    float af, ab;
    run_aggregates(x, lam, af, ab);
    TeamLaunch L{};
    TeamCtx tc{0, 0, 1, 0, nullptr};
    unsigned epoch = 0, xc = 0;
    int dec;
    exchange<OpPlain<XF>, XF, kSW>(L, tc, epoch, xc, c_from(af, e, XF{}), c_from(ab, e, XF{}), 0.f, kSE, tb, X, cf,
                              cb, 0.f, 0.f, dec, nullptr, nullptr);
    cf = c_add(cf, c_mul(CF, c_mul(tb.dt[lane], tb.dw[warp])));
    cb = c_add(cb, c_mul(CB, c_mul(tb.dt[31 - lane], tb.dw[kSW - 1 - warp])));
  }
  // the recurrences with the carries folded in, in frame F (as the team kernel)
  const int F = max(e + 5, max(c_exp(cf), c_exp(cb)) + 2);
  const float sc = pow2f(e - F);
  float xn[kSE];
  float r = c_to(cf, F);
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    r = lam * r + x[k] * sc;
    xn[k] = r;
  }
  // the staged masses and accepted v (bounded wait; a copy that does not
  // complete marks the pair failed and is waited for again before the CTA ends)
  const bool staged = mbar_wait(&s_mbar, 0, 1ll << 24);
  if (!staged && tid == 0) atomicExch(&A.st->fail, 1);
  const float4* mq = s_stage + tid;
  const float4* vq = s_stage + kChunk / 4 + tid;
  const int fo = vhalf ? A.FV[par][run] : 0;
  // error terms v_old y - m: v_old y scaled by 2^(fo + F) in FP32 when that
  // scale keeps the product in range (|fo + F| <= 60: v_old y is within
  // 2^-60 .. 2^60 of the mass it is compared with), in extended range otherwise
  const int fe = fo + F;
  const bool fast = fe >= -60 && fe <= 60;
  const float s2 = fast ? pow2f(fe) : 0.f;
  float s = c_to(cb, F), ep = 0.f;
#pragma unroll
  for (int q = kSE / 4 - 1; q >= 0; --q) {
    const float4 m4 = mq[q * kST];
    float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vhalf) v4 = vq[q * kST];
    const float mm[4] = {m4.x, m4.y, m4.z, m4.w};
    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      const int k = 4 * q + i;
      const float y = xn[k] + s;
      // masses past the end are zero, so are their outputs and error terms
      if (vhalf) {
        if (fast)
          ep += fabsf(vv[i] * y * s2 - mm[i]);
        else
          ep += fabsf(c_to(c_mul(XF{vv[i], fo}, XF{y, F}), 0) - mm[i]);
      }
      xn[k] = vdiv(mm[i], y);
      s = lam * (s + x[k] * sc);
    }
  }
  const int fz = normalise_run(xn, -F);
  st_run(Z, ch, tid, xn);
  FZ[run] = fz;
  float zf, zb;
  run_aggregates(xn, lam, zf, zb);
  XF tf, tbk;
  cta_totals<OpPlain<XF>>(c_from(zf, fz, XF{}), c_from(zb, fz, XF{}), tb, sw, tf, tbk);
  if (tid == 0) {
    A.agg_f[zsrc][ch] = tf;
    A.agg_b[zsrc][ch] = tbk;
  }
  if (vhalf) {
    float h = ep, l = 0.f;
    cta_sum_pair(h, l, sred);
    if (tid == 0) {
      A.errp[2 * ch] = h;
      A.errp[2 * ch + 1] = l;
    }
  }
  if (!staged) mbar_wait(&s_mbar, 0, 1ll << 24);   // no copy may land after the CTA ends
  // the last chunk to finish takes the loop's bookkeeping
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    slast = atomicAdd(&A.st->done, 1u) == (unsigned)A.nch - 1u;
  }
  __syncthreads();
  if (!slast) return;
  __threadfence();
  if (vhalf) {
    // the while condition of Algorithm 1: the chunks' error pairs summed in
    // FP64 (each thread over chunks tid, tid + 512, ..., then a fixed tree)
    double ev = 0.0;
    for (int j = tid; j < A.nch; j += kST) ev += (double)__ldcg(A.errp + 2 * j) + (double)__ldcg(A.errp + 2 * j + 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (lane == 0) sdred[warp] = ev;
    __syncthreads();
    if (tid == 0) {
      double err = 0.0;
      for (int w = 0; w < kSW; ++w) err += sdred[w];
      StreamState* st = A.st;
      st->err = err;
      const int status = st->fail ? FS1_ETIMEOUT
                         : !isfinite(err)
                             ? FS1_ENUMERIC
                             : (err <= A.tol ? FS1_OK : (st->ell >= A.itr_max ? FS1_ENOTCONV : -1));
      if (status >= 0) {
        st->stop = 1;
        st->status = status;
        atomicSub(B.nactive, 1);
      } else {
        st->par = par ^ 1;   // accept v_new
      }
      st->done = 0u;
      sstop = status >= 0;
    }
  } else if (tid == 0) {
    StreamState* st = A.st;
    st->ell += 1;   // a full iteration done
    if (st->fail) {
      st->stop = 1;
      st->status = FS1_ETIMEOUT;
      atomicSub(B.nactive, 1);
    }
    st->done = 0u;
    sstop = st->fail;
  }
  // the carries of this launch's output for the next launch
  __syncthreads();
  if (!sstop) chunk_carry_scan(A, zsrc, tb, X);
}


// Cost phase 1: distance-weighted chunk aggregates of the accepted v.
__global__ void __launch_bounds__(kST, 1) stream_cost_agg_kernel(StreamArgs A) {
  using DT = PairC<XF>;
  __shared__ DecayTables<XF> tb;
  __shared__ DT sw[2 * kSW];
  copy_tables(tb, A.tabs);
  __syncthreads();
  const int tid = threadIdx.x, ch = blockIdx.x;
  const int par = A.st->par;
  const float lam = A.lamf;
  float x[kSE];
  ld_run(A.V[par], ch, tid, x);
  const int e = A.FV[par][(size_t)ch * kST + tid];
  float p = 0.f, Aa = 0.f;
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    Aa = lam * (Aa + p);
    p = lam * p + x[k];
  }
  float s = 0.f, Bb = 0.f;
#pragma unroll
  for (int k = kSE - 1; k >= 0; --k) {
    Bb = lam * (Bb + s + x[k]);
    s = lam * (s + x[k]);
  }
  DT af{c_from(p, e, XF{}), c_from(Aa, e, XF{})};
  DT ab{c_from(s, e, XF{}), c_from(Bb, e, XF{})};
  DT tf, tbk;
  cta_totals<OpDist<XF>>(af, ab, tb, sw, tf, tbk);
  if (tid == 0) {
    A.dagg_f[ch] = tf;
    A.dagg_b[ch] = tbk;
  }
}

// Cost phase 2: the chunk carries of the distance-weighted scan (one thread;
// runs once per solve).
__global__ void stream_cost_carry_kernel(StreamArgs A) {
  if (threadIdx.x != 0) return;
  using Op = OpDist<XF>;
  const XF lamR = c_decay((double)kChunk, A.c, XF{});
  const float R = (float)kChunk;
  PairC<XF> fc = Op::zero();
  for (int q = 0; q < A.nch; ++q) {
    A.dcar_f[q] = fc;
    fc = Op::fwd(fc, A.dagg_f[q], lamR, R);
  }
  PairC<XF> bc = Op::zero();
  for (int q = A.nch - 1; q >= 0; --q) {
    A.dcar_b[q] = bc;
    bc = Op::bwd(A.dagg_b[q], bc, lamR, R);
  }
}

// Cost phase 3: per chunk, sum_k u_k (A_k + B_k) h in FP64, A / B the
// distance-weighted forward / backward sums of v (as the team kernel).
__global__ void __launch_bounds__(kST, 1) stream_cost_kernel(StreamArgs A) {
  using DT = PairC<XF>;
  using OpD = OpDist<XF>;
  __shared__ DecayTables<XF> tb;
  __shared__ XchgSmem<DT> XD;
  __shared__ double sred[kSW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ch = blockIdx.x;
  if (tid == 0) XD.ok = 1;
  copy_tables(tb, A.tabs);
  __syncthreads();
  const int par = A.st->par;
  const size_t run = (size_t)ch * kST + tid;
  const float lam = A.lamf;
  float v[kSE], u[kSE];
  ld_run(A.V[par], ch, tid, v);
  ld_run(A.U, ch, tid, u);
  const int fv = A.FV[par][run];
  const int fu = A.FU[run];
  float p = 0.f, Aa = 0.f;
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    Aa = lam * (Aa + p);
    p = lam * p + v[k];
  }
  float s = 0.f, Bb = 0.f;
#pragma unroll
  for (int k = kSE - 1; k >= 0; --k) {
    Bb = lam * (Bb + s + v[k]);
    s = lam * (s + v[k]);
  }
  DT dcf, dcb;
  {
    TeamLaunch L{};
    TeamCtx tc{0, 0, 1, 0, nullptr};
    unsigned epoch = 0, xc = 0;
    int dec;
    exchange<OpD, XF, kSW>(L, tc, epoch, xc, DT{c_from(p, fv, XF{}), c_from(Aa, fv, XF{})},
                      DT{c_from(s, fv, XF{}), c_from(Bb, fv, XF{})}, 0.f, kSE, tb, XD, dcf, dcb, 0.f, 0.f, dec,
                      nullptr, nullptr);
    dcf = OpD::add(dcf, OpD::prop(A.dcar_f[ch], c_mul(tb.dt[lane], tb.dw[warp]), (float)(kSE * tid)));
    dcb = OpD::add(dcb, OpD::prop(A.dcar_b[ch], c_mul(tb.dt[31 - lane], tb.dw[kSW - 1 - warp]),
                                  (float)(kSE * (kST - 1 - tid))));
  }
  int F = max(max(c_exp(dcf.p), c_exp(dcf.a)), max(c_exp(dcb.p), c_exp(dcb.a))) + 2;
  F = max(F, fv + 12);
  const float sc = pow2f(fv - F);
  float BBk[kSE];
  float ss = c_to(dcb.p, F), BB = c_to(dcb.a, F);
#pragma unroll
  for (int k = kSE - 1; k >= 0; --k) {
    BBk[k] = BB;
    BB = lam * (BB + ss + v[k] * sc);
    ss = lam * (ss + v[k] * sc);
  }
  float pp = c_to(dcf.p, F), AA = c_to(dcf.a, F);
  double wpart = 0.0;
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    AA = lam * (AA + pp);
    pp = lam * pp + v[k] * sc;
    if (u[k] != 0.f) wpart += ldexp((double)u[k] * (double)(AA + BBk[k]), fu + F);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wpart += __shfl_xor_sync(0xffffffffu, wpart, o);
  if (lane == 0) sred[warp] = wpart;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kSW; ++w) t += sred[w];
    A.costp[ch] = t;
  }
}

// The result and (optionally) the log potentials of the returned iterate.
__global__ void stream_final_kernel(StreamArgs A) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const StreamState st = *A.st;
    double w = 0.0;
    for (int q = 0; q < A.nch; ++q) w += A.costp[q];
    PairResult R;
    R.w = st.status == FS1_ENUMERIC ? NAN : w * A.h;
    R.err = st.err;
    R.iters = st.ell;
    R.status = st.status;
    R.pad = 0;
    *A.result = R;
  }
  if (A.f_out || A.g_out) {
    const int par = A.st->par;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
      // point i = chunk ch, thread t, point k of the thread's run
      const int64_t ch = i / kChunk;
      const int r = (int)(i - ch * kChunk), t = r / kSE, k = r % kSE;
      const size_t at = (size_t)ch * kChunk + (size_t)(k >> 2) * (4 * kST) + (size_t)t * 4 + (k & 3);
      const size_t run = (size_t)ch * kST + t;
      if (A.f_out) A.f_out[i] = log_of(A.U[at], A.FU[run]);
      if (A.g_out) A.g_out[i] = log_of(A.V[par][at], A.FV[par][run]);
    }
  }
}

size_t align256s(size_t x) { return (x + 255) / 256 * 256; }

// Lays out one pair's arrays from p (advanced past them) and fills its
// arguments.
StreamArgs stream_args(const PairDesc& P, int in_f32, PairResult* d_result, char*& p) {
  const int nch = (int)((P.n + kChunk - 1) / kChunk);
  const size_t pts = (size_t)nch * kChunk;
  const size_t runs = (size_t)nch * kST;
  StreamArgs A{};
  A.a = P.a;
  A.b = P.b;
  A.in_f32 = in_f32;
  A.nch = nch;
  A.n = P.n;
  A.c = P.h_fast / P.eps;
  A.lamf = (float)std::exp(-A.c);
  A.h = P.h_fast;
  A.tol = P.tol;
  A.itr_max = P.itr_max;
  A.AW = (float*)p; p += align256s(sizeof(float) * pts);
  A.BW = (float*)p; p += align256s(sizeof(float) * pts);
  A.U = (float*)p; p += align256s(sizeof(float) * pts);
  A.V[0] = (float*)p; p += align256s(sizeof(float) * pts);
  A.V[1] = (float*)p; p += align256s(sizeof(float) * pts);
  A.FU = (int*)p; p += align256s(sizeof(int) * runs);
  A.FV[0] = (int*)p; p += align256s(sizeof(int) * runs);
  A.FV[1] = (int*)p; p += align256s(sizeof(int) * runs);
  for (int i = 0; i < 3; ++i) {
    A.agg_f[i] = (XF*)p; p += align256s(sizeof(XF) * nch);
    A.agg_b[i] = (XF*)p; p += align256s(sizeof(XF) * nch);
    A.car_f[i] = (XF*)p; p += align256s(sizeof(XF) * nch);
    A.car_b[i] = (XF*)p; p += align256s(sizeof(XF) * nch);
  }
  A.dec = (XF*)p; p += align256s(sizeof(XF) * nch);
  A.tabs = (DecayTables<XF>*)p; p += align256s(sizeof(DecayTables<XF>));
  A.errp = (float*)p; p += align256s(sizeof(float) * 2 * nch);
  A.dagg_f = (PairC<XF>*)p; p += align256s(sizeof(PairC<XF>) * nch);
  A.dagg_b = (PairC<XF>*)p; p += align256s(sizeof(PairC<XF>) * nch);
  A.dcar_f = (PairC<XF>*)p; p += align256s(sizeof(PairC<XF>) * nch);
  A.dcar_b = (PairC<XF>*)p; p += align256s(sizeof(PairC<XF>) * nch);
  A.costp = (double*)p; p += align256s(sizeof(double) * nch);
  A.st = (StreamState*)p; p += 256;
  A.result = d_result;
  A.f_init = P.f_init;
  A.g_init = P.g_init;
  A.f_out = P.f_out;
  A.g_out = P.g_out;
  if (A.f_init == nullptr || A.g_init == nullptr) A.f_init = A.g_init = nullptr;
  return A;
}

// Pairs P[0 .. count) (at most kMaxStreamPairs) through the shared launches.
int solve_stream_group(const PairDesc* P, const int* in_f32, int count, PairResult* d_results, char* p,
                       cudaStream_t st, long long& nl) {
  StreamBatch B{};
  B.npairs = count;
  B.nactive = (int*)p;
  p += 256;
  int grid = 0;
  long long itr_max = 0;
  for (int i = 0; i < count; ++i) {
    B.A[i] = stream_args(P[i], in_f32[i], d_results + i, p);
    B.choff[i] = grid;
    grid += B.A[i].nch;
    itr_max = std::max<long long>(itr_max, (long long)P[i].itr_max);
  }
  B.choff[count] = grid;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(B.nactive, &B.npairs, sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    fprintf(stderr, "fs1: streaming solve failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  for (int i = 0; i < count; ++i) {
    stream_init_kernel<<<B.A[i].nch, kST, 0, st>>>(B.A[i]);
    stream_carry_kernel<<<1, kST, 0, st>>>(B.A[i], 0);
    nl += 2;
  }
  // Iterations in blocks of 16 (two launches each), captured once as a CUDA
  // graph (direct launches if capture is unavailable).  One block stays in
  // flight ahead of the host: the active count copied after block k is read
  // after block k + 1 has been issued (launches after the stop return at once).
  const int block = 16;
  auto issue_block = [&]() {
    for (int i = 0; i < block; ++i) {
      stream_step_kernel<<<grid, kST, 2 * kStageBytes, st>>>(B, 1);
      stream_step_kernel<<<grid, kST, kStageBytes, st>>>(B, 0);
    }
  };
  if ((e = cudaFuncSetAttribute(stream_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * kStageBytes))) != cudaSuccess) {
    fprintf(stderr, "fs1: streaming solve failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    issue_block();
    if (cudaStreamEndCapture(st, &graph) != cudaSuccess || graph == nullptr ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
      exec = nullptr;
  }
  cudaGetLastError();
  int* h_active = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if ((e = cudaMallocHost(&h_active, 2 * sizeof(int))) != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return FS1_ENOMEM;
  }
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  auto run_block = [&](int slot) {
    if (exec)
      cudaGraphLaunch(exec, st);
    else
      issue_block();
    nl += 2 * block;
    cudaMemcpyAsync(h_active + slot, B.nactive, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(ev[slot], st);
  };
  const long long max_blocks = itr_max / block + 3;   // every loop ends by then in any case
  run_block(0);
  for (long long k = 0;; ++k) {
    if (k + 1 < max_blocks) run_block((int)((k + 1) & 1));
    if ((e = cudaEventSynchronize(ev[k & 1])) != cudaSuccess) break;
    if (h_active[k & 1] <= 0 || k + 1 >= max_blocks) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaFreeHost(h_active);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: streaming solve failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  for (int i = 0; i < count; ++i) {
    const StreamArgs& A = B.A[i];
    stream_cost_agg_kernel<<<A.nch, kST, 0, st>>>(A);
    stream_cost_carry_kernel<<<1, 32, 0, st>>>(A);
    stream_cost_kernel<<<A.nch, kST, 0, st>>>(A);
    stream_final_kernel<<<(A.f_out || A.g_out) ? 1024 : 1, 256, 0, st>>>(A);
    nl += 4;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) {
    fprintf(stderr, "fs1: streaming solve failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

}  // namespace

size_t stream_workspace(const int64_t* n, int count) {
  size_t b = 0;
  for (int i = 0; i < count; ++i) {
    if (i % kMaxStreamPairs == 0) b += 256;   // a group's active count
    const size_t nch = (size_t)((n[i] + kChunk - 1) / kChunk);
    const size_t pts = nch * kChunk;
    b += 5 * align256s(sizeof(float) * pts) + 3 * align256s(sizeof(int) * nch * kST) +
         13 * align256s(sizeof(XF) * nch) + align256s(sizeof(DecayTables<XF>)) + align256s(sizeof(float) * 2 * nch) +
         4 * align256s(sizeof(PairC<XF>) * nch) + align256s(sizeof(double) * nch) + 256;
  }
  return b;
}

int solve_stream_batch(const PairDesc* P, const int* in_f32, int count, PairResult* d_results, void* ws,
                       size_t ws_bytes, void* stream, long long* launches) {
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> n(count);
  for (int i = 0; i < count; ++i) {
    if (P[i].n < 1) return FS1_EINVAL;
    if ((P[i].n + kChunk - 1) / kChunk > (1 << 30)) return FS1_EUNSUPPORTED;
    n[i] = P[i].n;
  }
  if (stream_workspace(n.data(), count) > ws_bytes) return FS1_ENOMEM;
  char* p = (char*)ws;
  long long nl = 0;
  for (int g = 0; g < count; g += kMaxStreamPairs) {
    const int m = std::min(kMaxStreamPairs, count - g);
    const int r = solve_stream_group(P + g, in_f32 + g, m, d_results + g, p, st, nl);
    if (r != FS1_OK) return r;
    p += stream_workspace(n.data() + g, m);
  }
  if (launches) *launches = nl;
  return FS1_OK;
}

}  // namespace fs1
