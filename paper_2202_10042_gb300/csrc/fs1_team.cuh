// fs1_team.cuh -- the 1D FS-1 solver kernel for sm_103a (the team kernel).
//
// Included by fs1_solve1d.cu (host side and the generic instantiations) and by
// the fs1_team_exact_*.cu units, which instantiate the kernel at fixed point
// counts per thread so that the instantiations compile in parallel.
//
// One "team" of T CTAs owns one (a, b) pair at a time and runs the whole
// Sinkhorn loop of Algorithm 1 with the pair's state on chip: every thread
// holds E consecutive grid points of u and v in registers (the masses a, b sit
// in shared memory), so HBM is read once per pair and written once per pair.
//
// Each half-step of Algorithm 1 (the r/s sweeps on phi with the psi update,
// then the p/q sweeps on psi with the phi update) is a bidirectional chunked
// parallel scan of the recurrences of Section 3, eq. "recursion":
//   thread : the recurrences run serially over the thread's E points;
//   warp   : Kogge-Stone over the 32 thread aggregates (shuffles), in plain
//            FP32 inside one per-warp frame when the warp's values span a
//            narrow exponent range, in extended range otherwise;
//   CTA    : every warp forms its CTA-local carry as one decay-weighted sum
//            of the other warps' totals (no serial scan over warps);
//   team   : warp 0 publishes the CTA totals and the error partial as
//            epoch-tagged 64-bit words; thread j < T polls slot j (every
//            word validates itself, so one L2 round trip suffices) and the
//            CTA's warps reduce the slots into its team carries.  This is the
//            only global synchronisation of a half-step.
// The aggregates of a half-step's output are formed while the output is
// produced.  The marginal error of the while condition of Algorithm 1 (FP32
// terms, summed as compensated FP32 pairs within warps, across warps and
// across CTAs in a fixed order) rides on the same exchange, and every warp of
// every CTA takes the stop decision from the same compensated sum.
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
// with distance-weighted recurrences (OpDist) and reduced in FP64.
//
// Points per thread.  A pair of N points on a team of T CTAs gives every
// thread Eeff = ceil(N / (512 T)) consecutive points.  The kernel is a
// template on E (registers for up to E points) and G (the guard grain): the
// serial loops run in chunks of G points, a chunk entirely below Eeff without
// per-point guards and the chunk that straddles Eeff with its points past
// Eeff turned into identity steps (decay 1, input 0).  Per-point guards would
// split the unrolled loop into one basic block per point and keep the
// compiler from overlapping the shared-memory loads, reciprocals and
// recurrence chains of neighbouring points.  G = E gives the exact kernel of
// one point count (one guard, taken); the generic kernel (E = 32, G = 8 for
// the stabilised variant: 4 % faster than G = 4 on batches of uneven pairs,
// the identity steps notwithstanding; G = 4 for plain FP32, G = 2 for FP64)
// serves batches whose pairs have different point counts.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <type_traits>

#include "fs1.h"
#include "fs1_device.cuh"
#include "fs1_internal.h"

namespace fs1 {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kSlotWords = 16;      // 64-bit words per exchange slot (payload <= 10)

template <class C, int ND = 257>
struct DecayTables {
  C dt[33];        // lam^{Eeff j}: thread offsets inside a warp
  C dw[33];        // lam^{32 Eeff j}: warp offsets inside a CTA
  C dT[ND];        // lam^{S j}: CTA offsets inside a team (S = points per CTA)
  float dtf[33];   // lam^{Eeff j} in FP32 for the narrow warp scan
  int narrow;      // 1 if c * 32 * Eeff <= 40 (a warp's decay fits one FP32 frame)
};

// Units.  A CTA of the team kernel is one unit of 16 warps (the team member),
// or, for pairs small enough to fit a few warps, 16 / GW independent units of
// GW warps, each solving its own pair (a team of one unit).  A unit
// synchronises its own warps only: __syncthreads for the whole CTA, the warp
// barrier for one warp, a named barrier otherwise: ids 1-4 for units of 4
// warps, 5-6 for units of 8 (both widths can run at once in one CTA).
template <int GW>
__device__ __forceinline__ void unit_sync() {
  if constexpr (GW == kWarps) {
    __syncthreads();
  } else if constexpr (GW == 1) {
    __syncwarp();
  } else {
    constexpr int base = GW == 8 ? 5 : 1;
    asm volatile("bar.sync %0, %1;" ::"r"(base + (int)(threadIdx.x / (32 * GW))), "n"(32 * GW) : "memory");
  }
}


// where a CTA sits: its team, rank, team size and the team's slots
struct TeamCtx {
  int team, rank, T;
  size_t slot_base;                // first slot of the team's [2][T] slot block
  int* abort;
  int ticket;                      // index of the team's pair broadcast word (queues)
};

// Team of this CTA at level k of a level schedule: CTA c is rank c % T_k of
// team c / T_k, the level's teams have their own slots and ticket words, and
// the level serves the queue of the class of team size T_k (classes sorted by
// increasing team size, levels by decreasing).  Every team of level k + 1 is
// made of CTAs of one team of level k (T_{k+1} divides T_k), so those CTAs
// leave level k together, when their team finds its queue empty.
__device__ __forceinline__ void level_ctx(const TeamLaunch& L, int k, TeamCtx& tc, int& cls) {
  const int T = L.level_T[k];
  tc.T = T;
  tc.rank = (int)blockIdx.x % T;
  tc.team = (int)blockIdx.x / T;
  const size_t first = (size_t)blockIdx.x - (size_t)tc.rank;
  tc.slot_base = (size_t)k * 2 * (size_t)L.grid + 2 * first;
  tc.ticket = k * L.grid + (int)first;
  tc.abort = L.abort_flags + blockIdx.x / L.level_T[0];
  cls = L.nlevel - 1 - k;
}

template <class T>
struct SlotPayload {
  T f, b;
  float eh, el;    // error partial as a compensated FP32 pair
};

// per-CTA shared state of an exchange; warp aggregates are double-buffered by
// exchange parity so that a fast warp can publish the next exchange while a
// slow one still reads the current one
template <class T, int NW = kWarps, int NST = kMaxTeamCtas>
struct XchgSmem {
  T wf[2][NW], wb[2][NW];
  float eh[2][NW], el[2][NW];
  T pf[NW], pb[NW];                     // partial team carries (one per warp)
  float ph[NW], pl[NW];
  int ok;
  SlotPayload<T> stage[NST];            // validated team slots
};

// split an error partial into a compensated FP32 pair
__device__ __forceinline__ void to_df(float x, float& hi, float& lo) { hi = x; lo = 0.f; }
__device__ __forceinline__ void to_df(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// ---------------------------------------------------------------------------
// exchange slots: payload words tagged with the exchange epoch
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void slot_publish(Slot* s, const T& f, const T& b, float eh, float el, unsigned tag) {
  SlotPayload<T> pl{f, b, eh, el};
  constexpr int nw = (int)(sizeof(SlotPayload<T>) / 4);
  static_assert(nw <= kSlotWords, "slot too small");
  const unsigned* w = reinterpret_cast<const unsigned*>(&pl);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(s->raw);
  const unsigned long long t = (unsigned long long)tag << 32;
#pragma unroll
  for (int i = 0; i < nw; i += 2) {
    const unsigned long long w0 = t | w[i];
    const unsigned long long w1 = t | (i + 1 < nw ? w[i + 1] : 0u);
    st_relaxed_v2(dst + i, w0, w1);
  }
}

// returns true when every word carries `tag`
template <class T>
__device__ __forceinline__ bool slot_try_read(const Slot* s, unsigned tag, SlotPayload<T>& out) {
  constexpr int nw = (int)(sizeof(SlotPayload<T>) / 4);
  unsigned* w = reinterpret_cast<unsigned*>(&out);
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(s->raw);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < nw; i += 2) {
    unsigned long long w0, w1;
    ld_relaxed_v2(src + i, w0, w1);
    ok &= (unsigned)(w0 >> 32) == tag;
    ok &= (unsigned)(w1 >> 32) == tag;
    w[i] = (unsigned)w0;
    if (i + 1 < nw) w[i + 1] = (unsigned)w1;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// warp-level scans of the thread aggregates (phase A)
// ---------------------------------------------------------------------------
// generic: inclusive forward / backward Kogge-Stone with the operator
template <class Op, class C, class TB>
__device__ __forceinline__ void warp_scan_generic(typename Op::T af, typename Op::T ab, int Eeff,
                                                  const TB& tb, typename Op::T& excl_f,
                                                  typename Op::T& excl_b, typename Op::T& wtot_f,
                                                  typename Op::T& wtot_b) {
  using T = typename Op::T;
  const int lane = threadIdx.x & 31;
  T x = af, z = ab;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = Op::up(x, o);
    const T w = Op::down(z, o);
    if (lane >= o) x = Op::fwd(y, x, tb.dt[o], (float)(Eeff * o));
    if (lane + o < 32) z = Op::bwd(z, w, tb.dt[o], (float)(Eeff * o));
  }
  const T ex = Op::up(x, 1);
  const T eb = Op::down(z, 1);
  excl_f = lane == 0 ? Op::zero() : ex;
  excl_b = lane == 31 ? Op::zero() : eb;
  wtot_f = Op::idx(x, 31);
  wtot_b = Op::idx(z, 0);
}

// narrow stabilised path: one FP32 frame per warp (exact power-of-two shifts)
template <class TB>
__device__ __forceinline__ bool warp_scan_narrow(XF af, XF ab, const TB& tb, XF& excl_f,
                                                 XF& excl_b, XF& wtot_f, XF& wtot_b) {
  const int lane = threadIdx.x & 31;
  const int emax = __reduce_max_sync(0xffffffffu, max(af.e, ab.e));
  const int lo_f = af.m != 0.f ? af.e : INT_MAX;
  const int lo_b = ab.m != 0.f ? ab.e : INT_MAX;
  const int emin = __reduce_min_sync(0xffffffffu, min(lo_f, lo_b));
  if (!tb.narrow || (emin != INT_MAX && emax - emin > 50)) return false;
  float x = af.m * pow2f(af.e - emax);
  float z = ab.m * pow2f(ab.e - emax);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, x, o);
    const float w = __shfl_down_sync(0xffffffffu, z, o);
    if (lane >= o) x = fmaf(tb.dtf[o], y, x);
    if (lane + o < 32) z = fmaf(tb.dtf[o], w, z);
  }
  const float ex = __shfl_up_sync(0xffffffffu, x, 1);
  const float eb = __shfl_down_sync(0xffffffffu, z, 1);
  excl_f = xf_norm(lane == 0 ? 0.f : ex, emax);
  excl_b = xf_norm(lane == 31 ? 0.f : eb, emax);
  wtot_f = xf_norm(__shfl_sync(0xffffffffu, x, 31), emax);
  wtot_b = xf_norm(__shfl_sync(0xffffffffu, z, 0), emax);
  return true;
}

// ---------------------------------------------------------------------------
// compact exchange slots of the stabilised path: two 64-bit words, read with
// one 16-byte load.  Every slot sits alone in its own 128-byte line, so
// each line is polled once per CTA per round (dense slots would put several
// pollers of one CTA on the same line, and that line's L2 slice is the
// bottleneck of the exchange).  Bits of a word: payload [0, 56), epoch tag
// [56, 64); a word left from an earlier exchange of the same parity is at
// least two epochs old, so its tag differs.
//   w0: frac(f) 23 | exp(f) 16 | exp(b) 16
//   w1: frac(b) 23 | error partial (FP32 without its sign) 31
// Exponents must fit 16 bits; pairs whose potentials could exceed that use
// the generic slots (decided per pair from c N).
// ---------------------------------------------------------------------------
constexpr int kCompactWords = 16;   // one 128-byte line per compact slot
constexpr int kExpNone = -32768;

__device__ __forceinline__ void xf_bits(XF x, unsigned& frac, unsigned& e16) {
  const XF n = xf_norm(x.m, x.e);   // mantissa in [0.5, 1): 23 fraction bits
  frac = __float_as_uint(n.m) & 0x7FFFFFu;
  e16 = n.m != 0.f ? ((unsigned)n.e & 0xFFFFu) : ((unsigned)kExpNone & 0xFFFFu);
}
__device__ __forceinline__ XF xf_unbits(unsigned frac, unsigned e16) {
  const int e = (int)(short)(e16 & 0xFFFFu);
  if (e == kExpNone) return XF{0.f, kZeroExp};
  return XF{__uint_as_float(frac | (126u << 23)), e};
}

// publish / poll a CTA's slot: compact words for XF carries when `compact`,
// tagged 32-bit chunks (generic slots) otherwise
template <class T>
__device__ __forceinline__ void publish(const TeamLaunch& L, const TeamCtx& tc, unsigned epoch, bool compact,
                                        const T& f, const T& b, float eh, float el) {
  const size_t slot = tc.slot_base + (size_t)(epoch & 1) * tc.T + tc.rank;
  if constexpr (std::is_same<T, XF>::value) {
    if (compact) {
      unsigned long long* w = L.cslots + slot * kCompactWords;
      unsigned ff, fe, bf, be;
      xf_bits(f, ff, fe);
      xf_bits(b, bf, be);
      const unsigned long long tag = (unsigned long long)(epoch & 0xFFu) << 56;
      const float ev = eh + el;
      const unsigned long long w0 = tag | ff | ((unsigned long long)fe << 23) | ((unsigned long long)be << 39);
      const unsigned long long w1 =
          tag | bf | ((unsigned long long)(__float_as_uint(ev) & 0x7FFFFFFFu) << 23);
      st_relaxed_v2(w, w0, w1);
      return;
    }
  }
  slot_publish<T>(L.slots + slot, f, b, eh, el, epoch);
}
template <class T>
__device__ __forceinline__ bool try_read(const TeamLaunch& L, const TeamCtx& tc, int j, unsigned epoch, bool compact,
                                         SlotPayload<T>& out) {
  const size_t slot = tc.slot_base + (size_t)(epoch & 1) * tc.T + j;
  if constexpr (std::is_same<T, XF>::value) {
    if (compact) {
      const unsigned long long* w = L.cslots + slot * kCompactWords;
      unsigned long long w0, w1;
      ld_relaxed_v2(w, w0, w1);
      const unsigned tg = epoch & 0xFFu;
      if ((unsigned)(w0 >> 56) != tg || (unsigned)(w1 >> 56) != tg) return false;
      out.f = xf_unbits((unsigned)(w0 & 0x7FFFFFu), (unsigned)(w0 >> 23));
      out.b = xf_unbits((unsigned)(w1 & 0x7FFFFFu), (unsigned)(w0 >> 39));
      out.eh = __uint_as_float((unsigned)(w1 >> 23) & 0x7FFFFFFFu);
      out.el = 0.f;
      return true;
    }
  }
  return slot_try_read<T>(L.slots + slot, epoch, out);
}

// sums over the 16 lanes of each half-warp
__device__ __forceinline__ XF hw_sum(XF t) {
  int e = t.m != 0.f ? t.e : kZeroExp;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  float v = t.m * pow2f(t.e - e);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return xf_norm(v, e);
}
__device__ __forceinline__ float hw_sum(float t) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}
__device__ __forceinline__ double hw_sum(double t) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}
template <class C>
__device__ __forceinline__ PairC<C> hw_sum(PairC<C> t) {
  return PairC<C>{hw_sum(t.p), hw_sum(t.a)};
}
__device__ __forceinline__ void hw_sum_df(float& hi, float& lo) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, h2, l2);
  }
}

// ---------------------------------------------------------------------------
// one exchange.  Every thread ends with its carries: the forward value at the
// point before its first point and the backward value at its last point.
//   A  warp: Kogge-Stone of the thread aggregates; warp totals to shared
//      memory (double-buffered); the error partial as a compensated pair.
//   B  every warp forms its own CTA-local carry as one decay-weighted sum of
//      the other warps' totals (lam^{32 Eeff k} table), with no serial
//      CTA-level scan; warp 0 also forms the CTA totals and publishes them.
//   C  (teams) every thread tid < T polls slot tid; after a block barrier the
//      16 warps each reduce 16 staged slots into partial team carries of this
//      CTA (decay-weighted by the lam^{S k} table), and after a second block
//      barrier every warp sums the 16 partials.
// The stop decision is taken by every warp from the same compensated FP32 sum,
// so all warps and all CTAs agree.  Returns false when a bounded wait gave
// up.  decision: 0 continue, 1 error <= tol, 2 error not finite.
// ---------------------------------------------------------------------------
template <class Op, class C, int GW = kWarps, class EV, class TB, class XS>
__device__ __forceinline__ bool exchange(const TeamLaunch& L, const TeamCtx& tc, unsigned& epoch,
                                         unsigned& xc, typename Op::T af, typename Op::T ab, EV err_part,
                                         int Eeff, const TB& tb, XS& X,
                                         typename Op::T& cf, typename Op::T& cb, float tol_h, float tol_l,
                                         int& decision, float* err_h, float* err_l, bool compact = false) {
  using T = typename Op::T;
  constexpr int NW = GW;   // warps of the unit
  const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) & (GW - 1);
  const int T_ = tc.T, rank = tc.rank;
  const int par = (int)(xc++ & 1u);
  // ---- A
  float eh, el;
  to_df(err_part, eh, el);
  warp_sum_df(eh, el);
  T excl_f, excl_b, wt_f, wt_b;
  bool done = false;
  if constexpr (std::is_same<T, XF>::value) done = warp_scan_narrow(af, ab, tb, excl_f, excl_b, wt_f, wt_b);
  if (!done) warp_scan_generic<Op, C>(af, ab, Eeff, tb, excl_f, excl_b, wt_f, wt_b);
  if (lane == 0) {
    X.wf[par][warp] = wt_f;
    X.wb[par][warp] = wt_b;
    X.eh[par][warp] = eh;
    X.el[par][warp] = el;
  }
  unit_sync<GW>();
  // ---- B: CTA-local carries of this warp, CTA error sum (every warp)
  const float Wf = (float)(32 * Eeff);
  T tf = Op::zero(), tbk = Op::zero();
  if (lane < warp) tf = Op::prop(X.wf[par][lane], tb.dw[warp - 1 - lane], Wf * (float)(warp - 1 - lane));
  if (lane > warp && lane < NW)
    tbk = Op::prop(X.wb[par][lane], tb.dw[lane - warp - 1], Wf * (float)(lane - warp - 1));
  const T pf = warp_sum_c(tf);
  const T pb = warp_sum_c(tbk);
  float th = lane < NW ? X.eh[par][lane] : 0.f;
  float tl = lane < NW ? X.el[par][lane] : 0.f;
  warp_sum_df(th, tl);
  T tcf = Op::zero(), tcb = Op::zero();
  if (GW == kWarps && T_ > 1) {
    ++epoch;
    if (warp == 0) {
      // CTA totals, published by lane 0
      T xf = Op::zero(), xb = Op::zero();
      if (lane < NW) {
        xf = Op::prop(X.wf[par][lane], tb.dw[NW - 1 - lane], Wf * (float)(NW - 1 - lane));
        xb = Op::prop(X.wb[par][lane], tb.dw[lane], Wf * (float)lane);
      }
      const T ctf = warp_sum_c(xf);
      const T ctb = warp_sum_c(xb);
      if (lane == 0) publish<T>(L, tc, epoch, compact, ctf, ctb, th, tl);
    }
    // ---- C: every thread with tid < T polls slot tid (independent loads)
    if ((int)threadIdx.x < T_) {
      SlotPayload<T> p;
      long long spins = 0;
      bool good = true;
      while (!try_read<T>(L, tc, threadIdx.x, epoch, compact, p)) {
        if (++spins > L.spin_cap || ((spins & 63) == 0 && ld_relaxed(tc.abort))) {
          good = false;
          break;
        }
        // the pollers have no other work: spin, and sleep only when a
        // wait runs long (a sleep's wake-up is much coarser than an L2 trip)
        if (spins > 8192) __nanosleep(256);
      }
      if (good) {
        X.stage[threadIdx.x] = p;
      } else {
        atomicExch(tc.abort, 1);
        atomicExch(&X.ok, 0);
      }
    }
    unit_sync<GW>();
    if (!X.ok) return false;
    // partial team carries: warp w reduces slots 16 w .. 16 w + 15; lanes
    // 0-15 the forward terms, lanes 16-31 the backward terms
    const float Sf = (float)(32 * GW * Eeff);
    const int j = 16 * warp + (lane & 15);
    T term = Op::zero();
    float ph = 0.f, pl = 0.f;
    if (j < T_) {
      const int k = lane < 16 ? rank - 1 - j : j - rank - 1;
      if (k >= 0) term = Op::prop(lane < 16 ? X.stage[j].f : X.stage[j].b, tb.dT[k], Sf * (float)k);
      if (lane < 16) {
        ph = X.stage[j].eh;
        pl = X.stage[j].el;
      }
    }
    const T part = hw_sum(term);
    hw_sum_df(ph, pl);
    if (lane == 0) {
      X.pf[warp] = part;
      X.ph[warp] = ph;
      X.pl[warp] = pl;
    }
    if (lane == 16) X.pb[warp] = part;
    unit_sync<GW>();
    const T q = lane < 16 ? X.pf[lane] : X.pb[lane - 16];
    const T tot = hw_sum(q);
    tcf = Op::idx(tot, 0);
    tcb = Op::idx(tot, 16);
    th = lane < 16 ? X.ph[lane] : 0.f;
    tl = lane < 16 ? X.pl[lane] : 0.f;
    warp_sum_df(th, tl);
  }
  // ---- decision (compensated FP32, identical in every warp) and carries
  decision = !(isfinite(th) && isfinite(tl)) ? 2 : (((th - tol_h) + (tl - tol_l)) <= 0.f ? 1 : 0);
  if (err_h) {
    *err_h = th;
    *err_l = tl;
  }
  const T wcf = Op::fwd(tcf, pf, tb.dw[warp], Wf * (float)warp);
  cf = Op::fwd(wcf, excl_f, tb.dt[lane], (float)(Eeff * lane));
  const int wr = NW - 1 - warp;
  const T wcb = Op::bwd(pb, tcb, tb.dw[wr], Wf * (float)wr);
  cb = Op::bwd(excl_b, wcb, tb.dt[31 - lane], (float)(Eeff * (31 - lane)));
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

// The serial loops of a half-step over the thread's points, in chunks of G
// (see the header): f(k, on) with k a compile-time index after unrolling and
// on = false for the identity steps of the chunk that straddles Eeff.
template <int E, int G, class F>
__device__ __forceinline__ void steps_up(int Eeff, F&& f) {
#pragma unroll
  for (int j = 0; j < E; j += G) {
    if (j + G <= Eeff) {
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (j + i < E) f(j + i, true);
    } else if (j < Eeff) {
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (j + i < E) f(j + i, j + i < Eeff);
    }
  }
}
template <int E, int G, class F>
__device__ __forceinline__ void steps_down(int Eeff, F&& f) {
#pragma unroll
  for (int j = ((E - 1) / G) * G; j >= 0; j -= G) {
    if (j + G <= Eeff) {
#pragma unroll
      for (int i = G - 1; i >= 0; --i)
        if (j + i < E) f(j + i, true);
    } else if (j < Eeff) {
#pragma unroll
      for (int i = G - 1; i >= 0; --i)
        if (j + i < E) f(j + i, j + i < Eeff);
    }
  }
}

// Shared state of the units of one width: decay tables, exchange state (one
// per element type, no aliasing between them) and queue tickets, per unit.
template <class C, int GW>
struct UnitSmem {
  static constexpr int NU = kWarps / GW;
  static constexpr int ND = GW == kWarps ? 257 : 1;
  static constexpr int NST = GW == kWarps ? kMaxTeamCtas : 1;
  DecayTables<C, ND> tb[NU];
  XchgSmem<typename OpDist<C>::T, GW, NST> XD[NU];
  XchgSmem<typename OpPlain<C>::T, GW, NST> XP[NU];
  int item[NU];
};

// The pair loop of units of GW warps: the whole CTA as a member of a team
// (static teams, uniform teams or a level schedule), or 16 / GW units each
// solving pairs of its own queue.  tid is the thread's index in its unit.
// Returns false when a bounded wait gave up.
template <class V, class C, int E, int G, int GW>
__device__ __forceinline__ bool team_body(const TeamLaunch& L, int mode, unsigned char* smem_raw,
                                          UnitSmem<C, GW>* us) {
  constexpr bool EXT = std::is_same<C, XF>::value;
  using OpP = OpPlain<C>;
  using OpD = OpDist<C>;
  using PT = typename OpP::T;
  using DT = typename OpD::T;

  constexpr int NT = 32 * GW, NU = kWarps / GW;
  const int unit = GW == kWarps ? 0 : (int)threadIdx.x / NT;
  const int tid = GW == kWarps ? (int)threadIdx.x : (int)threadIdx.x % NT;

  V* sm_a = reinterpret_cast<V*>(smem_raw) + (size_t)unit * 3 * E * NT;
  V* sm_b = sm_a + E * NT;
  V* sm_v = sm_b + E * NT;   // the accepted v (for the marginal error; temp in the cost phase)

  auto& tb = us->tb[unit];
  auto& XD = us->XD[unit];
  auto& XP = us->XP[unit];
  int& sm_item = us->item[unit];
  TeamCtx tc;
  // level schedules run on the generic instantiations only (the host picks
  // an exact one for batches of one point count per thread, which have one
  // class), so that the exact kernels carry none of their state
  constexpr bool kLevels = G < E && GW == kWarps;
  int cls = -1, lvl = 0;
  if constexpr (GW < kWarps) {
    // every unit is a team of one on the units' queue of its width (a team
    // of one never waits on another CTA: no ticket word, no abort flag)
    tc.T = 1;
    tc.rank = 0;
    tc.team = (int)blockIdx.x * NU + unit;
    tc.slot_base = 0;
    tc.abort = L.abort_flags;
    tc.ticket = 0;
    cls = L.unit_class + (GW == 8 ? 0 : (GW == 4 ? 1 : 2));
  } else if (kLevels && L.nlevel > 0) {
    level_ctx(L, 0, tc, cls);
  } else if (L.cta_team) {
    tc.team = L.cta_team[blockIdx.x];
    tc.rank = L.cta_rank[blockIdx.x];
    tc.T = L.team_T[tc.team];
    tc.slot_base = (size_t)L.team_slot[tc.team];
    tc.abort = L.abort_flags + tc.team;
    tc.ticket = tc.team;
    cls = L.team_class[tc.team];
  } else {
    tc.T = L.team_size;
    tc.team = blockIdx.x / tc.T;
    tc.rank = blockIdx.x % tc.T;
    tc.slot_base = (size_t)tc.team * 2 * tc.T;
    tc.abort = L.abort_flags + tc.team;
    tc.ticket = 0;
  }
  int T = tc.T, team = tc.team, rank = tc.rank;
  if (GW == kWarps && team >= L.num_teams) return true;
  unsigned epoch = 0, xc = 0, seq = 0;
  if (tid == 0) {
    XD.ok = 1;
    XP.ok = 1;
  }
  unit_sync<GW>();

  for (;;) {   // the levels of a level schedule (one pass otherwise)
  for (int pi = team;; pi += L.num_teams) {
    int pid;
    if (cls < 0) {
      if (pi >= L.num_pairs) break;
      pid = L.order ? L.order[pi] : pi;
    } else {
      // next pair of the class queue; the team's rank 0 takes the ticket and
      // broadcasts it to the other CTAs of the team through a tagged word
      ++seq;
      if (tid == 0) {
        unsigned long long* const tk = L.tickets + (kLevels ? tc.ticket : team);
        int item;
        if (rank == 0) {
          item = atomicAdd(L.class_next + cls, 1);
          if (T > 1) {
            const unsigned long long w = ((unsigned long long)seq << 32) | (unsigned)item;
            asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(tk), "l"(w) : "memory");
          }
        } else {
          long long spins = 0;
          unsigned long long w = 0;
          for (;;) {
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(tk) : "memory");
            if ((unsigned)(w >> 32) == seq) break;
            if (++spins > L.spin_cap || ((spins & 63) == 0 && ld_relaxed(tc.abort))) {
              atomicExch(tc.abort, 1);
              w = 0xFFFFFFFFull;   // -1: give up
              break;
            }
          }
          item = (int)(unsigned)w;
        }
        sm_item = item;
      }
      unit_sync<GW>();
      const int item = sm_item;
      if (item < 0) return false;   // the ticket wait gave up (the other CTAs time out too)
      if (item >= L.class_off[cls + 1] - L.class_off[cls]) break;
      pid = L.order[L.class_off[cls] + item];
    }
    if (L.valid != nullptr && !L.valid[pid]) {
      if (rank == 0 && tid == 0) L.results[pid] = PairResult{NAN, NAN, 0, FS1_EINVAL, 0};
      unit_sync<GW>();   // sm_item is rewritten by the next ticket
      continue;
    }
    const PairDesc P = L.pairs[pid];
    const int64_t N = P.n;
    const double c = P.h_fast / P.eps;
    const V lam = (V)exp(-c);
    const int Eeff = (int)((N + (int64_t)T * NT - 1) / ((int64_t)T * NT));
    if (Eeff > E) {
      // the host picks the kernel from the point counts; a pair that does
      // not fit this instantiation's registers and shared memory is refused
      if (rank == 0 && tid == 0) L.results[pid] = PairResult{NAN, NAN, 0, FS1_EINVAL, 0};
      unit_sync<GW>();
      continue;
    }
    const int S = NT * Eeff;
    const int64_t s0 = (int64_t)rank * S;
    const int64_t g0 = s0 + (int64_t)tid * Eeff;   // first grid point of this thread
    const int ne = (int)max((int64_t)0, min((int64_t)Eeff, N - g0));
    // compact exchange slots need every exponent within 16 bits: the
    // potentials span at most about c N nats plus the mass range
    const bool compact = EXT && (c * (double)N + 200.0) * 1.4426950408889634 < 30000.0;

    // decay tables (FP64 exponent arithmetic, once per pair)
    for (int i = tid; i < 33 + 33 + UnitSmem<C, GW>::ND; i += NT) {
      if (i < 33) {
        tb.dt[i] = c_decay((double)Eeff * i, c, C{});
        tb.dtf[i] = (float)exp(-(double)Eeff * i * c);
      } else if (i < 66) {
        tb.dw[i - 33] = c_decay(32.0 * Eeff * (i - 33), c, C{});
      } else {
        tb.dT[i - 66] = c_decay((double)S * (i - 66), c, C{});
      }
    }
    if (tid == 0) tb.narrow = (c * 32.0 * Eeff <= 40.0) ? 1 : 0;
    // masses into shared memory, [k][thread] layout
    for (int i = tid; i < S; i += NT) {
      const int64_t gi = s0 + i;
      V va = 0, vb = 0;
      if (gi < N && mode == 0) {
        va = load_mass<V>(P.a, gi, L.in_f32);
        vb = load_mass<V>(P.b, gi, L.in_f32);
      }
      const int tt = i / Eeff, kk = i - tt * Eeff;
      sm_a[kk * NT + tt] = va;
      sm_b[kk * NT + tt] = vb;
    }

    // state: u in registers (xu, frame fu); v in registers (xn, frame fv)
    // with a copy of the accepted v in shared memory (sm_v) for the marginal
    // error; h* = frame + exponent of the largest value
    V xu[E], xn[E];
    int fu = 0, fv = 0, hu = kZeroExp, hv = kZeroExp;
    {
      const V init = (V)(1.0 / (double)N);
      if (P.f_init != nullptr) {
        // warm start (or the kernel-apply mode): log values -> frame + mantissas
        double fmax = -INFINITY;
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (k < ne) fmax = fmax > P.f_init[g0 + k] ? fmax : P.f_init[g0 + k];
        if (EXT) fu = isfinite(fmax) ? (int)floor(fmax * 1.4426950408889634) : 0;
#pragma unroll
        for (int k = 0; k < E; ++k)
          xu[k] = (k < ne) ? (V)exp2(P.f_init[g0 + k] * 1.4426950408889634 - (double)fu) : (V)0;
      } else {
#pragma unroll
        for (int k = 0; k < E; ++k) xu[k] = (k < ne) ? init : (V)0;
      }
      if (P.g_init != nullptr && mode == 0) {
        double gmax = -INFINITY;
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (k < ne) gmax = gmax > P.g_init[g0 + k] ? gmax : P.g_init[g0 + k];
        if (EXT) fv = isfinite(gmax) ? (int)floor(gmax * 1.4426950408889634) : 0;
#pragma unroll
        for (int k = 0; k < E; ++k)
          xn[k] = (k < ne) ? (V)exp2(P.g_init[g0 + k] * 1.4426950408889634 - (double)fv) : (V)0;
      } else {
#pragma unroll
        for (int k = 0; k < E; ++k) xn[k] = (k < ne) ? init : (V)0;
      }
      V mu = 0, mv = 0;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        mu = xu[k] > mu ? xu[k] : mu;
        mv = xn[k] > mv ? xn[k] : mv;
        sm_v[k * NT + tid] = xn[k];
      }
      if (EXT) {
        hu = mu > 0 ? fu + fexp((float)mu) : kZeroExp;
        hv = mv > 0 ? fv + fexp((float)mv) : kZeroExp;
      }
    }
    unit_sync<GW>();

    // aggregates of the initial u, in the same operation order as the
    // u-half's aggregates: a warm start from the potentials of a run stopped
    // after l iterations then reproduces that run's carries exactly (the
    // frames differ by a power of two, which scales every rounding exactly)
    PT cf, cb;
    {
      V af = 0, ab = 0, pw = 1;
      steps_down<E, G>(Eeff, [&](const int k, const bool on) {
        const V lk = on ? lam : (V)1, xk = on ? xu[k] : (V)0;
        af = af + pw * xk;
        pw = pw * lk;
        ab = lk * (ab + xk);
      });
      int dec;
      if (!exchange<OpP, C, GW>(L, tc, epoch, xc, c_from(af, fu, C{}), c_from(ab, fu, C{}), (V)0, Eeff, tb, XP,
                            cf, cb, 0.f, 0.f, dec, nullptr, nullptr, compact))
        goto timed_out;
    }

    {
      int64_t ell = 0;
      int status = FS1_OK;
      float eh_last = 0.f, el_last = 0.f;
      const float tol_h = (float)P.tol;
      const float tol_l = (float)(P.tol - (double)tol_h);
      for (;;) {
        // ---------------- v-half: y = K^T u, v_new = b / y, marginal error
        {
          const int F = EXT ? max(hu + 5, max(c_exp(cf), c_exp(cb)) + 2) : 0;
          const V sc = EXT ? (V)pow2f(fu - F) : (V)1;
          const V sc2 = EXT ? (V)pow2f(fv + F) : (V)1;
          // forward recurrence with the carry folded in: xn[k] = r_k
          V r = (V)c_to(cf, F);
          steps_up<E, G>(Eeff, [&](const int k, const bool on) {
            const V lk = on ? lam : (V)1, xk = on ? xu[k] : (V)0;
            r = lk * r + xk * sc;
            xn[k] = r;
          });
          // backward recurrence; output, error term and output aggregates
          // (an identity step has k >= Eeff >= ne, so z = 0 and its error
          // term is skipped: af, ab, pw, s and zmax pass through unchanged)
          V s = (V)c_to(cb, F), af = 0, ab = 0, pw = 1, zmax = 0, ep = 0;
          steps_down<E, G>(Eeff, [&](const int k, const bool on) {
            const V lk = on ? lam : (V)1, xk = on ? xu[k] : (V)0;
            const V y = xn[k] + s;
            const V m = sm_b[k * NT + tid];
            V z = (k < ne) ? vdiv(m, y) : (V)0;
            if (mode == 1) z = (k < ne) ? y : (V)0;   // kernel-apply mode: keep K^T u
            if (k < ne) ep += fabs(sm_v[k * NT + tid] * y * sc2 - m);
            xn[k] = z;
            zmax = z > zmax ? z : zmax;
            af = af + pw * z;
            pw = pw * lk;
            ab = lk * (ab + z);
            s = lk * (s + xk * sc);
          });
          const int fz = EXT ? -F : 0;
          if (mode == 1) {
            if (P.g_out != nullptr)
#pragma unroll
              for (int k = 0; k < E; ++k)
                if (k < ne) P.g_out[g0 + k] = log((double)xn[k]) + (double)F * 0.6931471805599453;
            break;
          }
          int dec;
          if (!exchange<OpP, C, GW>(L, tc, epoch, xc, c_from(af, fz, C{}), c_from(ab, fz, C{}), ep, Eeff, tb, XP,
                                cf, cb, tol_h, tol_l, dec, &eh_last, &el_last, compact))
            goto timed_out;
          if (dec != 0 || ell >= P.itr_max) {
            if (dec == 2) status = FS1_ENUMERIC;
            // the returned iterate keeps the accepted v
#pragma unroll
            for (int k = 0; k < E; ++k) xn[k] = sm_v[k * NT + tid];
            break;
          }
          // accept v_new
#pragma unroll
          for (int k = 0; k < E; ++k) sm_v[k * NT + tid] = xn[k];
          fv = fz;
          hv = (EXT && zmax > 0) ? fz + fexp((float)zmax) : kZeroExp;
        }
        // ---------------- u-half: y = K v, u = a / y
        {
          const int F = EXT ? max(hv + 5, max(c_exp(cf), c_exp(cb)) + 2) : 0;
          const V sc = EXT ? (V)pow2f(fv - F) : (V)1;
          V r = (V)c_to(cf, F);
          steps_up<E, G>(Eeff, [&](const int k, const bool on) {
            const V lk = on ? lam : (V)1, xk = on ? xn[k] : (V)0;
            r = lk * r + xk * sc;
            xu[k] = r;
          });
          V s = (V)c_to(cb, F), af = 0, ab = 0, pw = 1, zmax = 0;
          steps_down<E, G>(Eeff, [&](const int k, const bool on) {
            const V lk = on ? lam : (V)1, xk = on ? xn[k] : (V)0;
            const V y = xu[k] + s;
            const V m = sm_a[k * NT + tid];
            const V z = (k < ne) ? vdiv(m, y) : (V)0;
            xu[k] = z;
            zmax = z > zmax ? z : zmax;
            af = af + pw * z;
            pw = pw * lk;
            ab = lk * (ab + z);
            s = lk * (s + xk * sc);
          });
          const int fz = EXT ? -F : 0;
          fu = fz;
          hu = (EXT && zmax > 0) ? fz + fexp((float)zmax) : kZeroExp;
          int dec;
          if (!exchange<OpP, C, GW>(L, tc, epoch, xc, c_from(af, fz, C{}), c_from(ab, fz, C{}), (V)0, Eeff, tb,
                                XP, cf, cb, 0.f, 0.f, dec, nullptr, nullptr, compact))
            goto timed_out;
        }
        ++ell;
      }
      if (mode == 1) {
        unit_sync<GW>();
        continue;
      }

      // ---------------- transport cost: sum_k u_k (A_k + B_k) h, A/B the
      // distance-weighted forward / backward sums of v (O(N) recurrences)
      double wpart = 0.0;
      if (status == FS1_OK) {
        V p = 0, A = 0;
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (k < Eeff) {
            A = lam * (A + p);
            p = lam * p + xn[k];
          }
        V s = 0, B = 0;
#pragma unroll
        for (int k = E - 1; k >= 0; --k)
          if (k < Eeff) {
            B = lam * (B + s + xn[k]);
            s = lam * (s + xn[k]);
          }
        DT af{c_from(p, fv, C{}), c_from(A, fv, C{})};
        DT ab{c_from(s, fv, C{}), c_from(B, fv, C{})};
        DT dcf, dcb;
        int dec;
        if (!exchange<OpD, C, GW>(L, tc, epoch, xc, af, ab, (V)0, Eeff, tb, XD, dcf, dcb, 0.f, 0.f, dec, nullptr,
                              nullptr))
          goto timed_out;
        int F = 0;
        if (EXT) {
          F = max(max(c_exp(dcf.p), c_exp(dcf.a)), max(c_exp(dcb.p), c_exp(dcb.a))) + 2;
          F = max(F, hv + 12);
        }
        const V sc = EXT ? (V)pow2f(fv - F) : (V)1;
        V ss = (V)c_to(dcb.p, F), BB = (V)c_to(dcb.a, F);
#pragma unroll
        for (int k = E - 1; k >= 0; --k)
          if (k < Eeff) {
            sm_v[k * NT + tid] = BB;   // temp: backward distance sums
            BB = lam * (BB + ss + xn[k] * sc);
            ss = lam * (ss + xn[k] * sc);
          }
        V pp = (V)c_to(dcf.p, F), AA = (V)c_to(dcf.a, F);
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (k < Eeff) {
            AA = lam * (AA + pp);
            pp = lam * pp + xn[k] * sc;
            if (k < ne) wpart += ldexp((double)xu[k] * (double)(AA + sm_v[k * NT + tid]), fu + F);
          }
        wpart *= P.h_fast;
        float wh = 0.f, wl = 0.f;
        PT z0 = OpP::zero(), c0, c1;
        if (!exchange<OpP, C, GW>(L, tc, epoch, xc, z0, z0, wpart, Eeff, tb, XP, c0, c1, 0.f, 0.f, dec, &wh,
                              &wl))
          goto timed_out;
        wpart = (double)wh + (double)wl;
      }
      // optional potentials out
      if (P.f_out != nullptr)
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (k < ne) P.f_out[g0 + k] = log((double)xu[k]) + (double)fu * 0.6931471805599453;
      if (P.g_out != nullptr)
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (k < ne) P.g_out[g0 + k] = log((double)xn[k]) + (double)fv * 0.6931471805599453;
      if (rank == 0 && tid == 0) {
        const double err_last = (double)eh_last + (double)el_last;
        PairResult R;
        R.w = status == FS1_OK ? wpart : NAN;
        R.err = err_last;
        R.iters = ell;
        R.status = status;
        if (status == FS1_OK && !(err_last <= P.tol)) R.status = FS1_ENOTCONV;
        R.pad = T;
        L.results[pid] = R;
      }
    }
    unit_sync<GW>();
    continue;
  timed_out:
    if (rank == 0 && tid == 0) {
      PairResult R{NAN, NAN, 0, FS1_ETIMEOUT, 0};
      L.results[pid] = R;
    }
    return false;
  }
  // the team's queue is empty: its CTAs go on as the teams of the next level
  if (!kLevels || ++lvl >= L.nlevel) break;
  level_ctx(L, lvl, tc, cls);
  T = tc.T;
  team = tc.team;
  rank = tc.rank;
  // the level's slots start zeroed (tag 0): keep the compact slots' 8-bit
  // tags of its first two exchanges away from 0
  if (((epoch + 1u) & 0xFFu) == 0u || ((epoch + 2u) & 0xFFu) == 0u) epoch += 2u;
  unit_sync<GW>();   // sm_item is rewritten by the next ticket
  }
  return true;
}

template <class V, class C, int E, int G, int GW>
__device__ __noinline__ bool unit_phase(const TeamLaunch& L, unsigned char* smem_raw, UnitSmem<C, GW>* us) {
  return team_body<V, C, E, G, GW>(L, 0, smem_raw, us);
}

// The kernel: the pair loop of 16-warp units (team members); then, in the
// generic stabilised instantiation and when the launch has units' queues,
// units of 8 warps, each of which goes on as 2 units of 4 once its queue is
// empty, each of those as 4 units of one warp.  The 16-warp units' shared
// state is reused by the narrower units after a block barrier; the units of
// 8, 4 and 1 warps have separate shared state (a unit may still run while
// its neighbour has gone on as narrower units).
template <class V, class C, int E, int G>
__global__ void __launch_bounds__(kThreads, 1) fs1_team_kernel(TeamLaunch L, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kUnits = G < E && std::is_same<C, XF>::value;
  using S16 = UnitSmem<C, kWarps>;
  using S8 = UnitSmem<C, 8>;
  using S4 = UnitSmem<C, 4>;
  using S1 = UnitSmem<C, 1>;
  constexpr size_t kOff4 = (sizeof(S8) + 15) / 16 * 16;
  constexpr size_t kOff1 = kOff4 + (sizeof(S4) + 15) / 16 * 16;
  constexpr size_t kNarrow = kOff1 + sizeof(S1);
  constexpr size_t kStat = kUnits && kNarrow > sizeof(S16) ? kNarrow : sizeof(S16);
  __shared__ __align__(16) unsigned char stat[kStat];
  if (!team_body<V, C, E, G, kWarps>(L, mode, smem_raw, reinterpret_cast<S16*>(stat))) return;
  if constexpr (kUnits) {
    if (!L.unit_queues || mode != 0) return;
    __syncthreads();
    if (!unit_phase<V, C, E, G, 8>(L, smem_raw, reinterpret_cast<S8*>(stat))) return;
    if (!unit_phase<V, C, E, G, 4>(L, smem_raw, reinterpret_cast<S4*>(stat + kOff4))) return;
    unit_phase<V, C, E, G, 1>(L, smem_raw, reinterpret_cast<S1*>(stat + kOff1));
  }
}

// ---------------------------------------------------------------------------
// launch of one instantiation
// ---------------------------------------------------------------------------
template <class V, class C, int E, int G>
cudaError_t launch_kind(const TeamLaunch& L, int mode, cudaStream_t st) {
  auto kfn = fs1_team_kernel<V, C, E, G>;
  const size_t smem = 3 * sizeof(V) * (size_t)E * kThreads;
  // under stream capture the attribute was already set by an eager launch of
  // the same signature (graphs are captured on a signature's second call)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusNone) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // heterogeneous launches carry their grid; team_size is then the largest team
  const int grid = L.grid > 0 ? L.grid : L.num_teams * L.team_size;
  if (L.team_size > 1) {
    TeamLaunch Lc = L;
    void* args[] = {&Lc, &mode};
    return cudaLaunchCooperativeKernel((const void*)kfn, dim3(grid), dim3(kThreads), args, smem, st);
  }
  kfn<<<grid, kThreads, smem, st>>>(L, mode);
  return cudaGetLastError();
}

// Exact instantiations E = G = Es...: launches the one with E == Eeff and
// returns true, or returns false when none of Es is Eeff.
template <class V, class C, int... Es>
bool launch_exact_in(int Eeff, const TeamLaunch& L, int mode, cudaStream_t st, cudaError_t& e) {
  return ((Eeff == Es ? (e = launch_kind<V, C, Es, Es>(L, mode, st), true) : false) || ...);
}

}  // namespace fs1
