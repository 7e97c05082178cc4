// fs1_solve1d.cu -- the 1D FS-1 solver kernel for sm_103a.
//
// One "team" of T CTAs owns one (a, b) pair at a time and runs the whole
// Sinkhorn loop of Algorithm 1 with the pair's state on chip: every thread
// holds E consecutive grid points of u and v in registers (the masses a, b sit
// in shared memory), so HBM is read once per pair and written once per pair.
//
// Each half-step of Algorithm 1 (the r/s sweeps on phi with the psi update,
// then the p/q sweeps on psi with the phi update) is a bidirectional chunked
// parallel scan of the recurrences of Section 3, eq. "recursion":
//   thread   : the recurrences run serially over the thread's E points;
//   warp     : Kogge-Stone over the 32 thread aggregates (shuffles);
//   CTA      : the same over the warp aggregates (shared memory);
//   team     : every CTA publishes its aggregates to a global slot, passes one
//              bounded team barrier, and scans the T published aggregates.
// The aggregates of the half-step's output are formed while the output is
// produced, so one team barrier per half-step is the only global sync.  The
// marginal error of the while condition of Algorithm 1 (FP64 reduction of FP32
// terms) rides on the same barrier, and every CTA takes the stop decision from
// the same FP64 sum.
//
// Variants (template parameters):
//   V = double, C = double : plain FS-1 (Algorithm 1 as written), FP64.
//   V = float,  C = float  : plain FS-1, FP32 (no stabilisation).
//   V = float,  C = XF     : stabilised FS-1.  Values are FP32 mantissas in a
//                            per-thread power-of-two frame chosen every half-step
//                            from the largest term (the excess magnitude is
//                            absorbed into the frame, as the Remark in Section 2
//                            absorbs it into alpha, beta), and carries are
//                            extended-range values combined by exponent
//                            alignment (a max-shifted log-sum-exp in base 2).
// At the end the transport cost sum_ij u_i K_ij |i-j| h v_j is formed in O(N)
// with the distance-weighted recurrences (OpDist) and reduced in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "fs1.h"
#include "fs1_device.cuh"
#include "fs1_internal.h"

namespace fs1 {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

template <class C>
struct DecayTables {
  C dt[33];   // lam^{Eeff j}: thread offsets inside a warp
  C dw[33];   // lam^{32 Eeff j}: warp offsets inside a CTA
  C dS;       // lam^{S}: one CTA slice
  C dq[5];    // lam^{S q 2^i}: lane groups of the team scan
};

template <class OpT>
struct HierState {
  OpT excl_f, excl_b;     // within the warp
  OpT wexcl_f, wexcl_b;   // warp within the CTA
  OpT cta_f, cta_b;       // CTA totals
};

// word-wise L1-bypassing load / store of a trivially copyable value
template <class T>
__device__ __forceinline__ T load_cg(const void* p) {
  static_assert(sizeof(T) % 4 == 0, "");
  T v;
  unsigned* w = reinterpret_cast<unsigned*>(&v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); ++i) w[i] = __ldcg(reinterpret_cast<const unsigned*>(p) + i);
  return v;
}
template <class T>
__device__ __forceinline__ void store_cg(void* p, const T& v) {
  const unsigned* w = reinterpret_cast<const unsigned*>(&v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); ++i) __stcg(reinterpret_cast<unsigned*>(p) + i, w[i]);
}

// ---------------------------------------------------------------------------
// team barrier: bounded, abortable.  Returns false when it gave up.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool team_barrier(unsigned long long* ctr, unsigned long long target,
                                             int* abort_flag, long long cap, int* sm_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(ctr, 1ull);
    int ok = 1;
    long long spins = 0;
    while (ld_acquire(ctr) < target) {
      if (++spins > cap || ld_relaxed(abort_flag)) {
        ok = 0;
        atomicExch(abort_flag, 1);
        break;
      }
      if (spins > 64) __nanosleep(64);
    }
    *sm_ok = ok;
  }
  __syncthreads();
  return *sm_ok != 0;
}

// ---------------------------------------------------------------------------
// hierarchical scan, phase A: warp and CTA levels (before the team barrier)
// ---------------------------------------------------------------------------
template <class Op, class C>
__device__ __forceinline__ void scan_local(typename Op::T af, typename Op::T ab, int Eeff,
                                           const DecayTables<C>& tb, typename Op::T* sm_wf,
                                           typename Op::T* sm_wb, HierState<typename Op::T>& st) {
  using T = typename Op::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = af;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = Op::up(x, o);
    if (lane >= o) x = Op::fwd(y, x, tb.dt[o], (float)(Eeff * o));
  }
  T ex = Op::up(x, 1);
  st.excl_f = lane == 0 ? Op::zero() : ex;
  if (lane == 31) sm_wf[warp] = x;
  T z = ab;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = Op::down(z, o);
    if (lane + o < 32) z = Op::bwd(z, y, tb.dt[o], (float)(Eeff * o));
  }
  T eb = Op::down(z, 1);
  st.excl_b = lane == 31 ? Op::zero() : eb;
  if (lane == 0) sm_wb[warp] = z;
  __syncthreads();
  // CTA level, redundantly in every warp (no second block barrier needed)
  T wx = lane < kWarps ? sm_wf[lane] : Op::zero();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = Op::up(wx, o);
    if (lane >= o) wx = Op::fwd(y, wx, tb.dw[o], (float)(32 * Eeff * o));
  }
  T pf = Op::idx(wx, warp > 0 ? warp - 1 : 0);
  st.wexcl_f = warp == 0 ? Op::zero() : pf;
  st.cta_f = Op::idx(wx, kWarps - 1);
  T wz = lane < kWarps ? sm_wb[lane] : Op::zero();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = Op::down(wz, o);
    if (lane + o < 32) wz = Op::bwd(wz, y, tb.dw[o], (float)(32 * Eeff * o));
  }
  T pb = Op::idx(wz, warp + 1 < kWarps ? warp + 1 : 0);
  st.wexcl_b = warp == kWarps - 1 ? Op::zero() : pb;
  st.cta_b = Op::idx(wz, 0);
}

// phase C: the thread's carries from the team carries of its CTA
template <class Op, class C>
__device__ __forceinline__ void scan_carries(const HierState<typename Op::T>& st, typename Op::T tcf,
                                             typename Op::T tcb, int Eeff, const DecayTables<C>& tb,
                                             typename Op::T& cf, typename Op::T& cb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto wcf = Op::fwd(tcf, st.wexcl_f, tb.dw[warp], (float)(32 * Eeff * warp));
  cf = Op::fwd(wcf, st.excl_f, tb.dt[lane], (float)(Eeff * lane));
  const int wr = kWarps - 1 - warp;
  auto wcb = Op::bwd(st.wexcl_b, tcb, tb.dw[wr], (float)(32 * Eeff * wr));
  cb = Op::bwd(st.excl_b, wcb, tb.dt[31 - lane], (float)(Eeff * (31 - lane)));
}

// slot byte offsets
constexpr int kSlotF = 0, kSlotB = 16, kSlotErr = 32;

// team level (warp 0): scan the T published CTA aggregates, return this CTA's
// exclusive carries and the FP64 sum of the published error partials.
template <class Op, class C>
__device__ __forceinline__ void scan_team(const Slot* slots, int T, int rank, const DecayTables<C>& tb,
                                          int S, typename Op::T& tcf, typename Op::T& tcb,
                                          double& err_sum) {
  using OT = typename Op::T;
  const int lane = threadIdx.x & 31;
  const int q = (T + 31) >> 5;
  const int j0 = lane * q, j1 = min(T, j0 + q);
  OT af = Op::zero(), ab = Op::zero();
  double es = 0.0;
  for (int j = j0; j < j1; ++j) {
    af = Op::fwd(af, load_cg<OT>(slots[j].raw + kSlotF), tb.dS, (float)S);
    es += load_cg<double>(slots[j].raw + kSlotErr);
  }
  for (int j = j1 - 1; j >= j0; --j) ab = Op::bwd(load_cg<OT>(slots[j].raw + kSlotB), ab, tb.dS, (float)S);
  // lane-level scans
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int o = 1 << i;
    OT y = Op::up(af, o);
    if (lane >= o) af = Op::fwd(y, af, tb.dq[i], (float)S * (float)(q * o));
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int o = 1 << i;
    OT y = Op::down(ab, o);
    if (lane + o < 32) ab = Op::bwd(ab, y, tb.dq[i], (float)S * (float)(q * o));
  }
  OT exf = Op::up(af, 1);
  if (lane == 0) exf = Op::zero();
  OT exb = Op::down(ab, 1);
  if (lane == 31) exb = Op::zero();
  const int owner = rank / q;
  OT rf = exf, rb = exb;
  if (lane == owner) {
    for (int j = owner * q; j < rank; ++j) rf = Op::fwd(rf, load_cg<OT>(slots[j].raw + kSlotF), tb.dS, (float)S);
    for (int j = min(T, owner * q + q) - 1; j > rank; --j)
      rb = Op::bwd(load_cg<OT>(slots[j].raw + kSlotB), rb, tb.dS, (float)S);
  }
  tcf = Op::idx(rf, owner);
  tcb = Op::idx(rb, owner);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) es += __shfl_xor_sync(0xffffffffu, es, o);
  err_sum = es;
}

// ---------------------------------------------------------------------------
// one exchange round: local scan, publish, team barrier, team scan, carries
// ---------------------------------------------------------------------------
template <class Op, class C>
struct Exchange {
  typename Op::T* sm_wf;
  typename Op::T* sm_wb;
  double* sm_err;      // [kWarps]
  typename Op::T* sm_tc;  // [2]: team carries
  double* sm_errsum;
  int* sm_ok;
};

template <class Op, class C>
__device__ __forceinline__ bool exchange(const TeamLaunch& L, int team, int rank, unsigned long long& nbar,
                                         typename Op::T af, typename Op::T ab, double err_part, int Eeff,
                                         const DecayTables<C>& tb, const Exchange<Op, C>& X,
                                         typename Op::T& cf, typename Op::T& cb, double& err_total) {
  using OT = typename Op::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // CTA error partial: fixed-order FP64 reduction
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) err_part += __shfl_xor_sync(0xffffffffu, err_part, o);
  if (lane == 0) X.sm_err[warp] = err_part;
  HierState<OT> st;
  scan_local<Op, C>(af, ab, Eeff, tb, X.sm_wf, X.sm_wb, st);   // contains __syncthreads
  const int T = L.team_size;
  const int S = kThreads * Eeff;
  bool ok = true;
  if (T == 1) {
    if (threadIdx.x == 0) {
      double e = 0.0;
      for (int w = 0; w < kWarps; ++w) e += X.sm_err[w];
      *X.sm_errsum = e;
    }
    __syncthreads();
    err_total = *X.sm_errsum;
    scan_carries<Op, C>(st, Op::zero(), Op::zero(), Eeff, tb, cf, cb);
    return true;
  }
  ++nbar;
  Slot* slots = L.slots + ((size_t)team * 2 + (nbar & 1)) * T;
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int w = 0; w < kWarps; ++w) e += X.sm_err[w];
    Slot* s = slots + rank;
    store_cg<OT>(s->raw + kSlotF, st.cta_f);
    store_cg<OT>(s->raw + kSlotB, st.cta_b);
    store_cg<double>(s->raw + kSlotErr, e);
  }
  ok = team_barrier(L.counters + team, nbar * (unsigned long long)T, L.abort_flags + team, L.spin_cap,
                    X.sm_ok);
  if (!ok) return false;
  if (warp == 0) {
    OT tcf, tcb;
    double es;
    scan_team<Op, C>(slots, T, rank, tb, S, tcf, tcb, es);
    if (lane == 0) {
      X.sm_tc[0] = tcf;
      X.sm_tc[1] = tcb;
      *X.sm_errsum = es;
    }
  }
  __syncthreads();
  err_total = *X.sm_errsum;
  scan_carries<Op, C>(st, X.sm_tc[0], X.sm_tc[1], Eeff, tb, cf, cb);
  return true;
}

// ---------------------------------------------------------------------------
// the solver kernel
// ---------------------------------------------------------------------------
template <class V> __device__ __forceinline__ V vdiv(V a, V b) { return a / b; }
template <> __device__ __forceinline__ float vdiv<float>(float a, float b) { return __fdividef(a, b); }

template <class V>
__device__ __forceinline__ V load_mass(const void* p, int64_t i, int in_f32) {
  return in_f32 ? (V)(reinterpret_cast<const float*>(p)[i]) : (V)(reinterpret_cast<const double*>(p)[i]);
}

template <class V, class C, int E>
__global__ void __launch_bounds__(kThreads, 1) fs1_team_kernel(TeamLaunch L, int mode) {
  constexpr bool EXT = sizeof(C) != sizeof(V) || !std::is_same<C, V>::value;
  using OpP = OpPlain<C>;
  using OpD = OpDist<C>;
  using PT = typename OpP::T;
  using DT = typename OpD::T;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm_a = reinterpret_cast<V*>(smem_raw);
  V* sm_b = sm_a + E * kThreads;

  __shared__ DecayTables<C> tb;
  __shared__ DT sm_wf[kWarps], sm_wb[kWarps], sm_tc[2];
  __shared__ double sm_err[kWarps], sm_errsum;
  __shared__ int sm_ok;

  Exchange<OpP, C> XP{reinterpret_cast<PT*>(sm_wf), reinterpret_cast<PT*>(sm_wb), sm_err,
                      reinterpret_cast<PT*>(sm_tc), &sm_errsum, &sm_ok};
  Exchange<OpD, C> XD{sm_wf, sm_wb, sm_err, sm_tc, &sm_errsum, &sm_ok};

  const int T = L.team_size;
  const int team = blockIdx.x / T;
  const int rank = blockIdx.x % T;
  const int tid = threadIdx.x;
  if (team >= L.num_teams) return;
  unsigned long long nbar = 0;

  for (int pi = team; pi < L.num_pairs; pi += L.num_teams) {
    const int pid = L.order ? L.order[pi] : pi;
    const PairDesc P = L.pairs[pid];
    const int64_t N = P.n;
    const double c = P.h_fast / P.eps;
    const V lam = (V)exp(-c);
    const int Eeff = (int)((N + (int64_t)T * kThreads - 1) / ((int64_t)T * kThreads));
    const int S = kThreads * Eeff;
    const int64_t s0 = (int64_t)rank * S;
    const int64_t g0 = s0 + (int64_t)tid * Eeff;   // first grid point of this thread
    int ne = (int)max((int64_t)0, min((int64_t)Eeff, N - g0));

    // decay tables (FP64 exponent arithmetic, once per pair)
    if (tid < 33) tb.dt[tid] = c_decay((double)Eeff * tid, c, C{});
    else if (tid < 66) tb.dw[tid - 33] = c_decay(32.0 * Eeff * (tid - 33), c, C{});
    else if (tid == 66) tb.dS = c_decay((double)S, c, C{});
    else if (tid >= 67 && tid < 72) {
      const int q = (T + 31) >> 5;
      tb.dq[tid - 67] = c_decay((double)S * q * (double)(1 << (tid - 67)), c, C{});
    }
    // masses into shared memory, [k][thread] layout
    for (int i = tid; i < S; i += kThreads) {
      const int64_t gi = s0 + i;
      V va = 0, vb = 0;
      if (gi < N && mode == 0) {
        va = load_mass<V>(P.a, gi, L.in_f32);
        vb = load_mass<V>(P.b, gi, L.in_f32);
      }
      const int tt = i / Eeff, kk = i - tt * Eeff;
      sm_a[kk * kThreads + tt] = va;
      sm_b[kk * kThreads + tt] = vb;
    }

    // state: u (xu, frame fu), v (xv, frame fv); hx = frame + exponent of max
    V xu[E], xv[E], xn[E], t[E];
    int fu = 0, fv = 0, hu = kZeroExp, hv = kZeroExp;
    {
      const V init = (V)(1.0 / (double)N);
      const double* fi = mode == 1 ? P.f_init : P.f_init;
      if (fi != nullptr) {
        // warm start (or the kernel-apply mode): log values -> frame + mantissas
        double fmax = -INFINITY;
        for (int k = 0; k < E; ++k)
          if (k < ne) fmax = fmax > fi[g0 + k] ? fmax : fi[g0 + k];
        if (EXT) fu = isfinite(fmax) ? (int)floor(fmax * 1.4426950408889634) : 0;
        for (int k = 0; k < E; ++k)
          xu[k] = (k < ne) ? (V)exp2(fi[g0 + k] * 1.4426950408889634 - (double)fu) : (V)0;
      } else {
        for (int k = 0; k < E; ++k) xu[k] = (k < ne) ? init : (V)0;
      }
      if (P.g_init != nullptr && mode == 0) {
        double gmax = -INFINITY;
        for (int k = 0; k < E; ++k)
          if (k < ne) gmax = gmax > P.g_init[g0 + k] ? gmax : P.g_init[g0 + k];
        if (EXT) fv = isfinite(gmax) ? (int)floor(gmax * 1.4426950408889634) : 0;
        for (int k = 0; k < E; ++k)
          xv[k] = (k < ne) ? (V)exp2(P.g_init[g0 + k] * 1.4426950408889634 - (double)fv) : (V)0;
      } else {
        for (int k = 0; k < E; ++k) xv[k] = (k < ne) ? init : (V)0;
      }
      V mu = 0, mv = 0;
      for (int k = 0; k < E; ++k) { mu = xu[k] > mu ? xu[k] : mu; mv = xv[k] > mv ? xv[k] : mv; }
      if (EXT) {
        hu = mu > 0 ? fu + fexp((float)mu) : kZeroExp;
        hv = mv > 0 ? fv + fexp((float)mv) : kZeroExp;
      }
    }
    __syncthreads();

    // aggregates of the initial u
    PT cf, cb;
    double err = 0.0;
    {
      V r = 0, s = 0;
      for (int k = 0; k < E; ++k)
        if (k < Eeff) r = lam * r + xu[k];
      for (int k = E - 1; k >= 0; --k)
        if (k < Eeff) s = lam * (s + xu[k]);
      if (!exchange<OpP, C>(L, team, rank, nbar, c_from(r, fu, C{}), c_from(s, fu, C{}), 0.0, Eeff, tb,
                            XP, cf, cb, err))
        goto timed_out;
    }

    {
      int64_t ell = 0;
      int status = FS1_OK;
      double err_last = 0.0;
      for (;;) {
        // ---------------- v-half: y = K^T u, v_new = b / y, marginal error
        {
          int F = 0;
          if (EXT) {
            F = max(hu + 5, max(c_exp(cf), c_exp(cb)) + 2);
          }
          const V sc = EXT ? (V)pow2f(fu - F) : (V)1;
          V s = (V)c_to(cb, F);
#pragma unroll
          for (int k = E - 1; k >= 0; --k)
            if (k < Eeff) {
              t[k] = s;
              s = lam * (s + xu[k] * sc);
            }
          const V sc2 = EXT ? (V)pow2f(fv + F) : (V)1;
          V r = (V)c_to(cf, F), r2 = 0, ab = 0, pw = lam, zmax = 0;
          float ep = 0.f;
#pragma unroll
          for (int k = 0; k < E; ++k)
            if (k < Eeff) {
              r = lam * r + xu[k] * sc;
              const V y = r + t[k];
              const V m = sm_b[k * kThreads + tid];
              V z = (k < ne) ? vdiv(m, y) : (V)0;
              if (mode == 1) z = y;   // kernel-apply mode: keep K^T u itself
              if (k < ne) ep += (float)fabs(xv[k] * y * sc2 - m);
              xn[k] = z;
              zmax = z > zmax ? z : zmax;
              r2 = lam * r2 + z;
              ab = ab + pw * z;
              pw = pw * lam;
            }
          const int fz = EXT ? -F : 0;
          const int fzo = (mode == 1) ? F : fz;  // frame of y itself in apply mode
          if (mode == 1) {
            // write log(K^T u) and finish this pair
            if (P.g_out != nullptr)
              for (int k = 0; k < E; ++k)
                if (k < ne) P.g_out[g0 + k] = log((double)xn[k]) + (double)fzo * 0.6931471805599453;
            break;
          }
          double et;
          if (!exchange<OpP, C>(L, team, rank, nbar, c_from(r2, fz, C{}), c_from(ab, fz, C{}), (double)ep,
                                Eeff, tb, XP, cf, cb, et))
            goto timed_out;
          err_last = et;
          if (!isfinite(et)) { status = FS1_ENUMERIC; break; }
          if (ell >= P.itr_max || et <= P.tol) break;
          // accept v_new
#pragma unroll
          for (int k = 0; k < E; ++k) xv[k] = xn[k];
          fv = fz;
          hv = (EXT && zmax > 0) ? fz + fexp((float)zmax) : kZeroExp;
        }
        // ---------------- u-half: y = K v, u = a / y
        {
          int F = 0;
          if (EXT) F = max(hv + 5, max(c_exp(cf), c_exp(cb)) + 2);
          const V sc = EXT ? (V)pow2f(fv - F) : (V)1;
          V s = (V)c_to(cb, F);
#pragma unroll
          for (int k = E - 1; k >= 0; --k)
            if (k < Eeff) {
              t[k] = s;
              s = lam * (s + xv[k] * sc);
            }
          V r = (V)c_to(cf, F), r2 = 0, ab = 0, pw = lam, zmax = 0;
#pragma unroll
          for (int k = 0; k < E; ++k)
            if (k < Eeff) {
              r = lam * r + xv[k] * sc;
              const V y = r + t[k];
              const V m = sm_a[k * kThreads + tid];
              const V z = (k < ne) ? vdiv(m, y) : (V)0;
              xu[k] = z;
              zmax = z > zmax ? z : zmax;
              r2 = lam * r2 + z;
              ab = ab + pw * z;
              pw = pw * lam;
            }
          const int fz = EXT ? -F : 0;
          fu = fz;
          hu = (EXT && zmax > 0) ? fz + fexp((float)zmax) : kZeroExp;
          double dummy;
          if (!exchange<OpP, C>(L, team, rank, nbar, c_from(r2, fz, C{}), c_from(ab, fz, C{}), 0.0, Eeff, tb,
                                XP, cf, cb, dummy))
            goto timed_out;
        }
        ++ell;
      }
      if (mode == 1) continue;

      // ---------------- transport cost: sum_k u_k (A_k + B_k) h, A/B the
      // distance-weighted forward / backward sums of v (O(N) recurrences)
      double wpart = 0.0;
      if (status == FS1_OK) {
        V p = 0, A = 0;
        for (int k = 0; k < E; ++k)
          if (k < Eeff) {
            A = lam * (A + p);
            p = lam * p + xv[k];
          }
        V s = 0, B = 0;
        for (int k = E - 1; k >= 0; --k)
          if (k < Eeff) {
            B = lam * (B + s + xv[k]);
            s = lam * (s + xv[k]);
          }
        DT af{c_from(p, fv, C{}), c_from(A, fv, C{})};
        DT ab{c_from(s, fv, C{}), c_from(B, fv, C{})};
        DT dcf, dcb;
        double dummy;
        if (!exchange<OpD, C>(L, team, rank, nbar, af, ab, 0.0, Eeff, tb, XD, dcf, dcb, dummy)) goto timed_out;
        int F = 0;
        if (EXT) {
          F = max(max(c_exp(dcf.p), c_exp(dcf.a)), max(c_exp(dcb.p), c_exp(dcb.a))) + 2;
          F = max(F, hv + 12);
        }
        const V sc = EXT ? (V)pow2f(fv - F) : (V)1;
        V ss = (V)c_to(dcb.p, F), BB = (V)c_to(dcb.a, F);
        for (int k = E - 1; k >= 0; --k)
          if (k < Eeff) {
            t[k] = BB;
            BB = lam * (BB + ss + xv[k] * sc);
            ss = lam * (ss + xv[k] * sc);
          }
        V pp = (V)c_to(dcf.p, F), AA = (V)c_to(dcf.a, F);
        for (int k = 0; k < E; ++k)
          if (k < Eeff) {
            AA = lam * (AA + pp);
            pp = lam * pp + xv[k] * sc;
            if (k < ne) wpart += ldexp((double)xu[k] * (double)(AA + t[k]), fu + F);
          }
        wpart *= P.h_fast;
        double wtot;
        PT z0 = OpP::zero(), c0, c1;
        if (!exchange<OpP, C>(L, team, rank, nbar, z0, z0, wpart, Eeff, tb, XP, c0, c1, wtot)) goto timed_out;
        wpart = wtot;
      }
      // optional potentials out
      if (P.f_out != nullptr)
        for (int k = 0; k < E; ++k)
          if (k < ne) P.f_out[g0 + k] = log((double)xu[k]) + (double)fu * 0.6931471805599453;
      if (P.g_out != nullptr)
        for (int k = 0; k < E; ++k)
          if (k < ne) P.g_out[g0 + k] = log((double)xv[k]) + (double)fv * 0.6931471805599453;
      if (rank == 0 && tid == 0) {
        PairResult R;
        R.w = status == FS1_OK ? wpart : NAN;
        R.err = err_last;
        R.iters = ell;
        R.status = status;
        if (status == FS1_OK && err_last > P.tol) R.status = FS1_ENOTCONV;
        R.pad = 0;
        L.results[pid] = R;
      }
    }
    __syncthreads();
    continue;
  timed_out:
    if (rank == 0 && tid == 0) {
      PairResult R{NAN, NAN, 0, FS1_ETIMEOUT, 0};
      L.results[pid] = R;
    }
    return;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int team_threads() { return kThreads; }

int team_elems_max(int kind) { return kind == KK_PLAIN_F64 ? 4 : 16; }

size_t team_smem_bytes(int kind) {
  const size_t vs = kind == KK_PLAIN_F64 ? sizeof(double) : sizeof(float);
  return 2 * vs * (size_t)team_elems_max(kind) * kThreads;
}

int elems_cap_for(int kind, double c) {
  const int emax = team_elems_max(kind);
  if (kind != KK_LOG_F32) return emax;
  // keep e^{c E} within the FP32 mantissa frame: c E <= 24 nats
  double cap = floor(24.0 / (c > 1e-30 ? c : 1e-30));
  if (cap < 1) cap = 1;
  return cap < emax ? (int)cap : emax;
}

template <class V, class C, int E>
static cudaError_t launch_kind(const TeamLaunch& L, int mode, cudaStream_t st) {
  auto kfn = fs1_team_kernel<V, C, E>;
  const size_t smem = 2 * sizeof(V) * (size_t)E * kThreads;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.num_teams * L.team_size;
  if (L.team_size > 1) {
    TeamLaunch Lc = L;
    void* args[] = {&Lc, &mode};
    return cudaLaunchCooperativeKernel((const void*)kfn, dim3(grid), dim3(kThreads), args, smem, st);
  }
  kfn<<<grid, kThreads, smem, st>>>(L, mode);
  return cudaGetLastError();
}

int launch_team_1d(int kind, const TeamLaunch& L, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = (kind >> 8) & 0xff;
  kind &= 0xff;
  cudaError_t e;
  switch (kind) {
    case KK_PLAIN_F64: e = launch_kind<double, double, 4>(L, mode, st); break;
    case KK_PLAIN_F32: e = launch_kind<float, float, 16>(L, mode, st); break;
    case KK_LOG_F32: e = launch_kind<float, XF, 16>(L, mode, st); break;
    default: return FS1_EINVAL;
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: team kernel launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

template <class V, class C, int E>
static int coresident() {
  auto kfn = fs1_team_kernel<V, C, E>;
  const size_t smem = 2 * sizeof(V) * (size_t)E * kThreads;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

int max_coresident_ctas(int kind) {
  switch (kind & 0xff) {
    case KK_PLAIN_F64: return coresident<double, double, 4>();
    case KK_PLAIN_F32: return coresident<float, float, 16>();
    case KK_LOG_F32: return coresident<float, XF, 16>();
  }
  return 0;
}

}  // namespace fs1
