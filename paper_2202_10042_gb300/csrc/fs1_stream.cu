// fs1_stream.cu -- stabilised 1D FS-1 for a pair too large to keep on chip.
//
// The team kernel (fs1_team.cuh) holds a pair's state in the registers and
// shared memory of co-resident CTAs; a pair beyond that capacity runs here
// with its state in device memory.  The grid is cut into chunks of 8192
// points (one 512-thread CTA, 16 points per thread).  One half-step of
// Algorithm 1 is three launches, with no waits between CTAs:
//   carry : an exclusive scan over the chunks' stored (decay, value)
//           aggregates of the half-step's input gives every chunk the forward
//           value at the point before it and the backward value at its last
//           point (one CTA, the team kernel's in-CTA scan over per-thread
//           runs of chunks);
//   half  : every chunk loads its input, forms the thread carries with the
//           in-CTA scan of the team kernel plus its chunk carries, runs the
//           recurrences of Section 3, eq. "recursion", divides the masses by
//           them (the psi or phi update of Algorithm 1), stores the output
//           with its chunk aggregates for the next half-step and (v-half) the
//           chunk's marginal-error partial;
//   decide: (v-half) the error partials are summed in a fixed order and the
//           while condition of Algorithm 1 is taken on the device.
// Every launch first reads the stop flag and returns once the loop has
// ended, so the host issues iterations in blocks and reads the flag between
// blocks.  Values are extended range (XF) per point; a thread's 16 points are
// taken into one power-of-two frame when loaded, as the team kernel keeps its
// registers.  The transport cost is formed as in the team kernel with the
// distance-weighted operator (OpDist): chunk aggregates, a sequential scan
// over the chunks, and the per-chunk sums of u (A + B) in FP64.
#include "fs1_team.cuh"

namespace fs1 {

namespace {

constexpr int kSE = 16;                  // points per thread per chunk
constexpr int kChunk = kThreads * kSE;   // points per chunk (one CTA)

struct StreamState {
  long long ell;   // completed iterations
  int stop;        // 1 once the loop has ended
  int status;      // FS1_OK, FS1_ENOTCONV or FS1_ENUMERIC
  int par;         // v buffer holding the accepted v
  int pad;
  double err;      // marginal error of the last v-half
};

struct StreamArgs {
  const void* a;
  const void* b;
  int in_f32;
  int nch;               // chunks
  int64_t n;             // points
  double c;              // h / eps
  double h, tol;
  long long itr_max;
  XF* U;                 // [nch * kChunk] each
  XF* V[2];
  XF* agg_f[3];          // chunk aggregates of U, V[0], V[1]: forward (value at the chunk's
  XF* agg_b[3];          // last point) and backward (value at the point before its first)
  XF* car_f;             // chunk carries of the current half-step's input
  XF* car_b;
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

// a thread's kSE points of X (zeros past ne) in one power-of-two frame:
// X[g0 + k] = x[k] * 2^frame, x[k] in [0, 1); returns the frame
__device__ __forceinline__ int load_run(const XF* X, int64_t g0, int ne, float (&x)[kSE]) {
  XF v[kSE];
  int e = kZeroExp;
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    v[k] = k < ne ? X[g0 + k] : XF{0.f, kZeroExp};
    e = (v[k].m != 0.f && v[k].e > e) ? v[k].e : e;
  }
#pragma unroll
  for (int k = 0; k < kSE; ++k) x[k] = v[k].m != 0.f ? v[k].m * pow2f(v[k].e - e) : 0.f;
  return e;
}

// Totals of the CTA from its threads' aggregates: forward to the CTA's last
// point, backward to the point before its first point (every thread calls;
// the totals are valid in warp 0).  sw: 32 XF of shared memory.
template <class Op>
__device__ void cta_totals(typename Op::T af, typename Op::T ab, const DecayTables<XF>& tb,
                           typename Op::T* sw, typename Op::T& tf, typename Op::T& tbk) {
  using T = typename Op::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T wf = warp_sum_c(Op::prop(af, tb.dt[31 - lane], (float)(kSE * (31 - lane))));
  const T wb = warp_sum_c(Op::prop(ab, tb.dt[lane], (float)(kSE * lane)));
  if (lane == 0) {
    sw[warp] = wf;
    sw[kWarps + warp] = wb;
  }
  __syncthreads();
  if (warp == 0) {
    T xf = Op::zero(), xb = Op::zero();
    if (lane < kWarps) {
      xf = Op::prop(sw[lane], tb.dw[kWarps - 1 - lane], (float)(32 * kSE * (kWarps - 1 - lane)));
      xb = Op::prop(sw[kWarps + lane], tb.dw[lane], (float)(32 * kSE * lane));
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
  for (int w = 0; w < kWarps; ++w) df_add(h, l, red[2 * w], red[2 * w + 1]);
}

__device__ __forceinline__ XF xf_of_log(double x) {
  if (!(x > -INFINITY)) return XF{0.f, kZeroExp};
  const double t = x * 1.4426950408889634;
  const double e = floor(t);
  return xf_norm((float)exp2(t - e), (int)e);
}
__device__ __forceinline__ double log_of_xf(XF v) {
  return v.m > 0.f ? log((double)v.m) + (double)v.e * 0.6931471805599453 : -INFINITY;
}

// u = v = 1/N (or the warm start) and the chunk aggregates of u
__global__ void __launch_bounds__(kThreads, 1) stream_init_kernel(StreamArgs A) {
  __shared__ DecayTables<XF> tb;
  __shared__ XF sw[2 * kWarps];
  fill_tables(tb, A.c, kSE);
  const int tid = threadIdx.x, ch = blockIdx.x;
  const int64_t g0 = (int64_t)ch * kChunk + (int64_t)tid * kSE;
  const int ne = (int)max((int64_t)0, min((int64_t)kSE, A.n - g0));
  const XF init = xf_norm((float)(1.0 / (double)A.n), 0);
#pragma unroll
  for (int k = 0; k < kSE; ++k) {
    XF u = XF{0.f, kZeroExp}, v = XF{0.f, kZeroExp};
    if (k < ne) {
      u = A.f_init ? xf_of_log(A.f_init[g0 + k]) : init;
      v = A.g_init ? xf_of_log(A.g_init[g0 + k]) : init;
    }
    A.U[g0 + k] = u;
    A.V[0][g0 + k] = v;
  }
  __syncthreads();
  float x[kSE];
  const int e = load_run(A.U, g0, ne, x);
  const float lam = (float)exp(-A.c);
  float af = 0.f, ab = 0.f, pw = 1.f;
#pragma unroll
  for (int k = kSE - 1; k >= 0; --k) {
    af = af + pw * x[k];
    pw = pw * lam;
    ab = lam * (ab + x[k]);
  }
  XF tf, tbk;
  cta_totals<OpPlain<XF>>(c_from(af, e, XF{}), c_from(ab, e, XF{}), tb, sw, tf, tbk);
  if (tid == 0) {
    A.agg_f[0][ch] = tf;
    A.agg_b[0][ch] = tbk;
  }
  if (ch == 0 && tid == 0) *A.st = StreamState{0, 0, FS1_OK, 0, 0, NAN};
}

// Chunk carries of the half-step's input (which: 0 u, 1 the accepted v).
// One CTA; thread t takes chunks [t P, t P + P).
__global__ void __launch_bounds__(kThreads, 1) stream_carry_kernel(StreamArgs A, int which) {
  __shared__ DecayTables<XF> tb;
  __shared__ XchgSmem<XF> X;
  __shared__ int sstop, spar;
  const int tid = threadIdx.x;
  if (tid == 0) {
    sstop = A.st->stop;
    spar = A.st->par;
    X.ok = 1;
  }
  const int P = (A.nch + kThreads - 1) / kThreads;
  const double cR = A.c * (double)kChunk;   // decay exponent of one chunk
  fill_tables(tb, cR, P);
  __syncthreads();
  if (sstop) return;
  const int src = which == 0 ? 0 : 1 + spar;
  const XF* F = A.agg_f[src];
  const XF* B = A.agg_b[src];
  const XF lamR = c_decay(1.0, cR, XF{});
  const XF zero = c_zero(XF{});
  const int q0 = tid * P;
  XF af = zero, ab = zero;
  for (int j = 0; j < P; ++j) {
    const int q = q0 + j;
    af = c_add(c_mul(af, lamR), q < A.nch ? F[q] : zero);
  }
  for (int j = P - 1; j >= 0; --j) {
    const int q = q0 + j;
    ab = c_add(q < A.nch ? B[q] : zero, c_mul(ab, lamR));
  }
  TeamLaunch L{};
  TeamCtx tc{0, 0, 1, 0, nullptr};
  unsigned epoch = 0, xc = 0;
  XF cf, cb;
  int dec;
  exchange<OpPlain<XF>, XF>(L, tc, epoch, xc, af, ab, 0.f, P, tb, X, cf, cb, 0.f, 0.f, dec, nullptr, nullptr);
  XF fc = cf;
  for (int j = 0; j < P; ++j) {
    const int q = q0 + j;
    if (q >= A.nch) break;
    A.car_f[q] = fc;
    fc = c_add(c_mul(fc, lamR), F[q]);
  }
  XF bc = cb;
  for (int j = P - 1; j >= 0; --j) {
    const int q = q0 + j;
    if (q < A.nch) {
      A.car_b[q] = bc;
      bc = c_add(B[q], c_mul(bc, lamR));
    } else {
      bc = c_mul(bc, lamR);   // (never read: chunks past the end hold nothing)
    }
  }
}

// One half-step over the chunks (vhalf 1: y = K^T u, v_new = b / y and the
// error of the accepted v; vhalf 0: y = K v, u = a / y).
__global__ void __launch_bounds__(kThreads, 2) stream_half_kernel(StreamArgs A, int vhalf) {
  __shared__ DecayTables<XF> tb;
  __shared__ XchgSmem<XF> X;
  __shared__ XF sw[2 * kWarps];
  __shared__ float sred[2 * kWarps];
  __shared__ int sstop, spar;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ch = blockIdx.x;
  if (tid == 0) {
    sstop = A.st->stop;
    spar = A.st->par;
    X.ok = 1;
  }
  fill_tables(tb, A.c, kSE);
  __syncthreads();
  if (sstop) return;
  const int par = spar;
  const XF* Xin = vhalf ? A.U : A.V[par];
  XF* Z = vhalf ? A.V[par ^ 1] : A.U;
  const int zsrc = vhalf ? 1 + (par ^ 1) : 0;
  const void* M = vhalf ? A.b : A.a;
  const XF* Vold = A.V[par];
  const int64_t g0 = (int64_t)ch * kChunk + (int64_t)tid * kSE;
  const int ne = (int)max((int64_t)0, min((int64_t)kSE, A.n - g0));
  const float lam = (float)exp(-A.c);

  float x[kSE];
  const int e = load_run(Xin, g0, ne, x);
  // carries of the input: in-CTA scan, then the chunk carries placed at the thread
  XF cf, cb;
  {
    float af = 0.f, ab = 0.f, pw = 1.f;
#pragma unroll
    for (int k = kSE - 1; k >= 0; --k) {
      af = af + pw * x[k];
      pw = pw * lam;
      ab = lam * (ab + x[k]);
    }
    TeamLaunch L{};
    TeamCtx tc{0, 0, 1, 0, nullptr};
    unsigned epoch = 0, xc = 0;
    int dec;
    exchange<OpPlain<XF>, XF>(L, tc, epoch, xc, c_from(af, e, XF{}), c_from(ab, e, XF{}), 0.f, kSE, tb, X, cf,
                              cb, 0.f, 0.f, dec, nullptr, nullptr);
    const XF CF = A.car_f[ch], CB = A.car_b[ch];
    cf = c_add(cf, c_mul(CF, c_mul(tb.dt[lane], tb.dw[warp])));
    cb = c_add(cb, c_mul(CB, c_mul(tb.dt[31 - lane], tb.dw[kWarps - 1 - warp])));
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
  float s = c_to(cb, F), af = 0.f, ab = 0.f, pw = 1.f, ep = 0.f;
#pragma unroll
  for (int k = kSE - 1; k >= 0; --k) {
    const float y = xn[k] + s;
    const float m = k < ne ? load_mass<float>(M, g0 + k, A.in_f32) : 0.f;
    const float z = k < ne ? vdiv(m, y) : 0.f;
    if (vhalf && k < ne) {
      const XF vo = Vold[g0 + k];
      ep += fabsf(vo.m * y * pow2f(vo.e + F) - m);
    }
    xn[k] = z;
    af = af + pw * z;
    pw = pw * lam;
    ab = lam * (ab + z);
    s = lam * (s + x[k] * sc);
  }
  const int fz = -F;
#pragma unroll
  for (int k = 0; k < kSE; ++k)
    if (k < ne) Z[g0 + k] = xf_norm(xn[k], fz);
  XF tf, tbk;
  cta_totals<OpPlain<XF>>(c_from(af, fz, XF{}), c_from(ab, fz, XF{}), tb, sw, tf, tbk);
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
  } else if (ch == 0 && tid == 0) {
    A.st->ell += 1;   // a full iteration done (read by the next decide)
  }
}

// The while condition of Algorithm 1 after a v-half (one warp).
__global__ void stream_decide_kernel(StreamArgs A) {
  StreamState* st = A.st;
  if (st->stop) return;
  const int lane = threadIdx.x & 31;
  float h = 0.f, l = 0.f;
  for (int q = lane; q < A.nch; q += 32) df_add(h, l, A.errp[2 * q], A.errp[2 * q + 1]);
  warp_sum_df(h, l);
  if (lane == 0) {
    const double err = (double)h + (double)l;
    st->err = err;
    if (!(isfinite(h) && isfinite(l))) {
      st->stop = 1;
      st->status = FS1_ENUMERIC;
    } else if (((h - (float)A.tol) + (l - (float)(A.tol - (double)(float)A.tol))) <= 0.f) {
      st->stop = 1;
      st->status = FS1_OK;
    } else if (st->ell >= A.itr_max) {
      st->stop = 1;
      st->status = FS1_ENOTCONV;
    } else {
      st->par ^= 1;   // accept v_new
    }
  }
}

// Cost phase 1: distance-weighted chunk aggregates of the accepted v.
__global__ void __launch_bounds__(kThreads, 1) stream_cost_agg_kernel(StreamArgs A) {
  using DT = PairC<XF>;
  __shared__ DecayTables<XF> tb;
  __shared__ DT sw[2 * kWarps];
  fill_tables(tb, A.c, kSE);
  __syncthreads();
  const int tid = threadIdx.x, ch = blockIdx.x;
  const int64_t g0 = (int64_t)ch * kChunk + (int64_t)tid * kSE;
  const int ne = (int)max((int64_t)0, min((int64_t)kSE, A.n - g0));
  const float lam = (float)exp(-A.c);
  float x[kSE];
  const int e = load_run(A.V[A.st->par], g0, ne, x);
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
__global__ void __launch_bounds__(kThreads, 1) stream_cost_kernel(StreamArgs A) {
  using DT = PairC<XF>;
  using OpD = OpDist<XF>;
  __shared__ DecayTables<XF> tb;
  __shared__ XchgSmem<DT> XD;
  __shared__ double sred[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ch = blockIdx.x;
  if (tid == 0) XD.ok = 1;
  fill_tables(tb, A.c, kSE);
  __syncthreads();
  const int64_t g0 = (int64_t)ch * kChunk + (int64_t)tid * kSE;
  const int ne = (int)max((int64_t)0, min((int64_t)kSE, A.n - g0));
  const float lam = (float)exp(-A.c);
  float v[kSE], u[kSE];
  const int fv = load_run(A.V[A.st->par], g0, ne, v);
  const int fu = load_run(A.U, g0, ne, u);
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
    exchange<OpD, XF>(L, tc, epoch, xc, DT{c_from(p, fv, XF{}), c_from(Aa, fv, XF{})},
                      DT{c_from(s, fv, XF{}), c_from(Bb, fv, XF{})}, 0.f, kSE, tb, XD, dcf, dcb, 0.f, 0.f, dec,
                      nullptr, nullptr);
    const int t = tid;
    dcf = OpD::add(dcf, OpD::prop(A.dcar_f[ch], c_mul(tb.dt[lane], tb.dw[warp]), (float)(kSE * t)));
    dcb = OpD::add(dcb, OpD::prop(A.dcar_b[ch], c_mul(tb.dt[31 - lane], tb.dw[kWarps - 1 - warp]),
                                  (float)(kSE * (kThreads - 1 - t))));
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
    if (k < ne) wpart += ldexp((double)u[k] * (double)(AA + BBk[k]), fu + F);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wpart += __shfl_xor_sync(0xffffffffu, wpart, o);
  if (lane == 0) sred[warp] = wpart;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += sred[w];
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
      if (A.f_out) A.f_out[i] = log_of_xf(A.U[i]);
      if (A.g_out) A.g_out[i] = log_of_xf(A.V[par][i]);
    }
  }
}

size_t align256s(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t stream_workspace(int64_t n) {
  const size_t nch = (size_t)((n + kChunk - 1) / kChunk);
  const size_t pts = nch * kChunk;
  return 3 * align256s(sizeof(XF) * pts) + 8 * align256s(sizeof(XF) * nch) + align256s(sizeof(float) * 2 * nch) +
         4 * align256s(sizeof(PairC<XF>) * nch) + align256s(sizeof(double) * nch) + 256 + 256;
}

int stream_launches_per_iteration() { return 5; }

int solve_stream_1d(const PairDesc& P, int in_f32, PairResult* d_result, void* ws, size_t ws_bytes, void* stream,
                    long long* launches) {
  cudaStream_t st = (cudaStream_t)stream;
  if (P.n < 1) return FS1_EINVAL;
  if (stream_workspace(P.n) > ws_bytes) return FS1_ENOMEM;
  const int64_t nch64 = (P.n + kChunk - 1) / kChunk;
  if (nch64 > (1 << 30)) return FS1_EUNSUPPORTED;
  const int nch = (int)nch64;
  const size_t pts = (size_t)nch * kChunk;
  char* p = (char*)ws;
  StreamArgs A{};
  A.a = P.a;
  A.b = P.b;
  A.in_f32 = in_f32;
  A.nch = nch;
  A.n = P.n;
  A.c = P.h_fast / P.eps;
  A.h = P.h_fast;
  A.tol = P.tol;
  A.itr_max = P.itr_max;
  A.U = (XF*)p; p += align256s(sizeof(XF) * pts);
  A.V[0] = (XF*)p; p += align256s(sizeof(XF) * pts);
  A.V[1] = (XF*)p; p += align256s(sizeof(XF) * pts);
  for (int i = 0; i < 3; ++i) {
    A.agg_f[i] = (XF*)p; p += align256s(sizeof(XF) * nch);
    A.agg_b[i] = (XF*)p; p += align256s(sizeof(XF) * nch);
  }
  A.car_f = (XF*)p; p += align256s(sizeof(XF) * nch);
  A.car_b = (XF*)p; p += align256s(sizeof(XF) * nch);
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
  long long nl = 0;
  cudaError_t e;
  stream_init_kernel<<<nch, kThreads, 0, st>>>(A);
  ++nl;
  // Iterations in blocks of 16, captured once as a CUDA graph (direct
  // launches if capture is unavailable).  One block stays in flight ahead of
  // the host: the stop flag copied after block k is read after block k + 1
  // has been issued (launches after the stop return at once).
  const int block = 16;
  auto issue_block = [&]() {
    for (int i = 0; i < block; ++i) {
      stream_carry_kernel<<<1, kThreads, 0, st>>>(A, 0);
      stream_half_kernel<<<nch, kThreads, 0, st>>>(A, 1);
      stream_decide_kernel<<<1, 32, 0, st>>>(A);
      stream_carry_kernel<<<1, kThreads, 0, st>>>(A, 1);
      stream_half_kernel<<<nch, kThreads, 0, st>>>(A, 0);
    }
  };
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    issue_block();
    if (cudaStreamEndCapture(st, &graph) != cudaSuccess || graph == nullptr ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
      exec = nullptr;
  }
  cudaGetLastError();
  int* h_stop = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if ((e = cudaMallocHost(&h_stop, 2 * sizeof(int))) != cudaSuccess) {
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
    nl += 5 * block;
    cudaMemcpyAsync(h_stop + slot, &A.st->stop, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(ev[slot], st);
  };
  const long long max_blocks = P.itr_max / block + 3;   // the loop ends by then in any case
  run_block(0);
  for (long long k = 0;; ++k) {
    if (k + 1 < max_blocks) run_block((int)((k + 1) & 1));
    if ((e = cudaEventSynchronize(ev[k & 1])) != cudaSuccess) break;
    if (h_stop[k & 1] || k + 1 >= max_blocks) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaFreeHost(h_stop);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: streaming solve failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  stream_cost_agg_kernel<<<nch, kThreads, 0, st>>>(A);
  stream_cost_carry_kernel<<<1, 32, 0, st>>>(A);
  stream_cost_kernel<<<nch, kThreads, 0, st>>>(A);
  stream_final_kernel<<<(P.f_out || P.g_out) ? 1024 : 1, 256, 0, st>>>(A);
  nl += 4;
  if ((e = cudaGetLastError()) != cudaSuccess) {
    fprintf(stderr, "fs1: streaming solve failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  if (launches) *launches = nl;
  return FS1_OK;
}

}  // namespace fs1
