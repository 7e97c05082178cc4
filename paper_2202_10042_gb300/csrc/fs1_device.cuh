// fs1_device.cuh -- device-side building blocks of the FS-1 kernels (sm_103a).
//
// Scan elements.  The forward / backward Horner recurrences of FS-1
// (Section 3, eq. "recursion") are first-order linear recurrences with a
// constant ratio lam = e^{-h/eps}; over a span of L cells they compose as
//     (x1 over L1) then (x2 over L2)  ->  lam^{L2} x1 + x2        (forward)
//     (x1 over L1) then (x2 over L2)  ->  x1 + lam^{L1} x2        (backward)
// which is the associative (decay, value) operator the chunked parallel scans
// use.  In the stabilised variant the values live in "extended range": an
// FP32 mantissa times an integer power of two (struct XF), so that values of
// any magnitude e^{+-10^4} keep FP32 relative precision and a max-shifted
// combine (align to the larger exponent, add mantissas) is exact in its shift.
// This is the log-sum-exp combine in base 2 with the shift taken as an
// integer; the per-thread frames of the state play the role of the absorbed
// potentials alpha/eps, beta/eps of the Remark in Section 2.
#pragma once
#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace fs1 {

constexpr int kZeroExp = -(1 << 28);   // exponent of the extended-range zero

// 8-byte aligned: one 64-bit load or store per value in shared and global memory
struct __align__(8) XF {
  float m;  // 0 or in [0.5, 1)
  int e;
};

// 2^k as a float for k in [-126, 127]; 0 below.
__device__ __forceinline__ float pow2f(int k) {
  k = k > 127 ? 127 : k;
  return (k < -126) ? 0.f : __int_as_float((k + 127) << 23);
}

// exponent of |m| such that |m| in [2^(e-1), 2^e); kZeroExp for 0 / subnormal
__device__ __forceinline__ int fexp(float m) {
  int eb = (__float_as_int(m) >> 23) & 0xff;
  return eb == 0 ? kZeroExp : eb - 126;
}

__device__ __forceinline__ XF xf_norm(float m, int e) {
  int b = __float_as_int(m);
  int eb = (b >> 23) & 0xff;
  if (eb == 0) return XF{0.f, kZeroExp};
  if (eb == 0xff) return XF{m, e};   // inf / nan propagate (the caller detects them)
  XF r;
  r.m = __int_as_float((b & 0x807fffff) | (126 << 23));
  r.e = e + eb - 126;
  return r;
}

// ---------------------------------------------------------------------------
// carry arithmetic: overloads for extended range (XF) and plain float/double
// ---------------------------------------------------------------------------
__device__ __forceinline__ XF c_zero(XF) { return XF{0.f, kZeroExp}; }
__device__ __forceinline__ float c_zero(float) { return 0.f; }
__device__ __forceinline__ double c_zero(double) { return 0.0; }

__device__ __forceinline__ XF c_add(XF a, XF b) {
  const bool sw = a.e < b.e;
  const float am = sw ? b.m : a.m, bm = sw ? a.m : b.m;
  const int ae = sw ? b.e : a.e, be = sw ? a.e : b.e;
  return xf_norm(fmaf(bm, pow2f(be - ae), am), ae);
}
__device__ __forceinline__ float c_add(float a, float b) { return a + b; }
__device__ __forceinline__ double c_add(double a, double b) { return a + b; }

// Products of normalised mantissas stay in [0.25, 1): no renormalisation is
// needed before the next c_add (which normalises), and exponents remain a
// bound within two bits.
__device__ __forceinline__ XF c_mul(XF a, XF b) {
  int e = a.e + b.e;
  e = e < kZeroExp ? kZeroExp : e;
  return XF{a.m * b.m, e};
}
__device__ __forceinline__ float c_mul(float a, float b) { return a * b; }
__device__ __forceinline__ double c_mul(double a, double b) { return a * b; }

// multiply by a plain non-negative scalar (span lengths of the weighted scan)
__device__ __forceinline__ XF c_scale(XF a, float s) { return xf_norm(a.m * s, a.e); }
__device__ __forceinline__ float c_scale(float a, float s) { return a * s; }
__device__ __forceinline__ double c_scale(double a, float s) { return a * (double)s; }

// exponent bound used to pick a common frame (plain values have frame 0)
__device__ __forceinline__ int c_exp(XF a) { return a.e; }
__device__ __forceinline__ int c_exp(float) { return kZeroExp; }
__device__ __forceinline__ int c_exp(double) { return kZeroExp; }

// value of a carry expressed in frame F (i.e. divided by 2^F)
__device__ __forceinline__ float c_to(XF a, int F) {
  int d = a.e - F;
  return a.m * pow2f(d < -200 ? -200 : d);
}
__device__ __forceinline__ float c_to(float a, int) { return a; }
__device__ __forceinline__ double c_to(double a, int) { return a; }

// a value v given relative to frame F, as a carry
__device__ __forceinline__ XF c_from(float v, int F, XF) { return xf_norm(v, F); }
__device__ __forceinline__ float c_from(float v, int, float) { return v; }
__device__ __forceinline__ double c_from(double v, int, double) { return v; }

// lam^L = exp(-L c) as a carry; c = h / eps in FP64
__device__ __forceinline__ XF c_decay(double L, double c, XF) {
  double t = L * c * 1.4426950408889634;  // log2(e)
  if (t == 0.0) return XF{0.5f, 1};
  double fl = floor(t);
  // lam^L = 2^-t = 2^-(fl) * 2^-(t-fl), with 2^-(t-fl) in (0.5, 1]
  float m = (float)exp2(-(t - fl));
  return xf_norm(m, -(int)fl);
}
__device__ __forceinline__ float c_decay(double L, double c, float) { return (float)exp(-L * c); }
__device__ __forceinline__ double c_decay(double L, double c, double) { return exp(-L * c); }

// warp shuffles of carries
__device__ __forceinline__ XF shfl_up(XF a, int o) {
  return XF{__shfl_up_sync(0xffffffffu, a.m, o), __shfl_up_sync(0xffffffffu, a.e, o)};
}
__device__ __forceinline__ XF shfl_down(XF a, int o) {
  return XF{__shfl_down_sync(0xffffffffu, a.m, o), __shfl_down_sync(0xffffffffu, a.e, o)};
}
__device__ __forceinline__ XF shfl_idx(XF a, int l) {
  return XF{__shfl_sync(0xffffffffu, a.m, l), __shfl_sync(0xffffffffu, a.e, l)};
}
__device__ __forceinline__ float shfl_up(float a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
__device__ __forceinline__ float shfl_down(float a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
__device__ __forceinline__ float shfl_idx(float a, int l) { return __shfl_sync(0xffffffffu, a, l); }
__device__ __forceinline__ double shfl_up(double a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
__device__ __forceinline__ double shfl_down(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
__device__ __forceinline__ double shfl_idx(double a, int l) { return __shfl_sync(0xffffffffu, a, l); }

// ---------------------------------------------------------------------------
// scan operators on (value) and on (value, distance-weighted value)
// ---------------------------------------------------------------------------
// Plain operator: element = aggregate of a span.
//   fwd(left, right, d, L) = d * left + right     (d = lam^L, L = right span)
//   bwd(left, right, d, L) = left + d * right     (d = lam^L, L = left span)
template <class C>
struct OpPlain {
  using T = C;
  static __device__ __forceinline__ T zero() { return c_zero(C{}); }
  static __device__ __forceinline__ T fwd(T l, T r, C d, float) { return c_add(c_mul(l, d), r); }
  static __device__ __forceinline__ T bwd(T l, T r, C d, float) { return c_add(l, c_mul(r, d)); }
  // an aggregate carried across L empty points (d = lam^L): its contribution
  // to a point L beyond its end
  static __device__ __forceinline__ T prop(T x, C d, float) { return c_mul(x, d); }
  static __device__ __forceinline__ T add(T x, T y) { return c_add(x, y); }
  static __device__ __forceinline__ T up(T a, int o) { return shfl_up(a, o); }
  static __device__ __forceinline__ T down(T a, int o) { return shfl_down(a, o); }
  static __device__ __forceinline__ T idx(T a, int l) { return shfl_idx(a, l); }
};

// Distance-weighted operator for the O(N) transport cost: element = (P, A)
// with P = sum lam^{dist} x and A = sum lam^{dist} dist x, both measured from
// the span's far end; composing spans adds L * P to A (see the derivation in
// oracle-independent form in the kernel that uses it).
template <class C>
struct PairC {
  C p, a;
};
template <class C>
struct OpDist {
  using T = PairC<C>;
  static __device__ __forceinline__ T zero() { return T{c_zero(C{}), c_zero(C{})}; }
  static __device__ __forceinline__ T fwd(T l, T r, C d, float L) {
    // P = d Pl + Pr ; A = d (Al + L Pl) + Ar
    return T{c_add(c_mul(l.p, d), r.p), c_add(c_mul(c_add(l.a, c_scale(l.p, L)), d), r.a)};
  }
  static __device__ __forceinline__ T prop(T x, C d, float L) {
    return T{c_mul(x.p, d), c_mul(c_add(x.a, c_scale(x.p, L)), d)};
  }
  static __device__ __forceinline__ T add(T x, T y) { return T{c_add(x.p, y.p), c_add(x.a, y.a)}; }
  static __device__ __forceinline__ T bwd(T l, T r, C d, float L) {
    // Q = Ql + d Qr ; B = Bl + d (Br + L Qr)
    return T{c_add(l.p, c_mul(r.p, d)), c_add(l.a, c_mul(c_add(r.a, c_scale(r.p, L)), d))};
  }
  static __device__ __forceinline__ T up(T a, int o) { return T{shfl_up(a.p, o), shfl_up(a.a, o)}; }
  static __device__ __forceinline__ T down(T a, int o) { return T{shfl_down(a.p, o), shfl_down(a.a, o)}; }
  static __device__ __forceinline__ T idx(T a, int l) { return T{shfl_idx(a.p, l), shfl_idx(a.a, l)}; }
};

// ---------------------------------------------------------------------------
// warp-wide sums of carries (one term per lane; zero terms allowed)
// ---------------------------------------------------------------------------
// Extended range: align every term to the warp's largest exponent (exact
// power-of-two shifts; terms 2^-126 below the largest vanish) and add in FP32.
__device__ __forceinline__ XF warp_sum_c(XF t) {
  const int e = __reduce_max_sync(0xffffffffu, t.m != 0.f ? t.e : kZeroExp);
  float v = t.m * pow2f(t.e - e);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return xf_norm(v, e);
}
__device__ __forceinline__ float warp_sum_c(float t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}
__device__ __forceinline__ double warp_sum_c(double t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}
template <class C>
__device__ __forceinline__ PairC<C> warp_sum_c(PairC<C> t) {
  return PairC<C>{warp_sum_c(t.p), warp_sum_c(t.a)};
}

// compensated FP32 (double-float) sum across the warp; identical in every lane
__device__ __forceinline__ void warp_sum_df(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = hi + h2;   // TwoSum(hi, h2)
    const float bp = s - hi;
    const float er = (hi - (s - bp)) + (h2 - bp);
    hi = s;
    lo = lo + l2 + er;
  }
}
// local compensated accumulation: (hi, lo) += (h2, l2)
__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
  const float s = hi + h2;
  const float bp = s - hi;
  const float er = (hi - (s - bp)) + (h2 - bp);
  hi = s;
  lo = lo + l2 + er;
}

// ---------------------------------------------------------------------------
// memory-model helpers for the team exchange
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 64-bit words of the team exchange: each carries a 32-bit payload and the
// 32-bit epoch tag of the exchange that wrote it, so a reader validates every
// word on its own and needs no separate flag or barrier round trip.
__device__ __forceinline__ void st_relaxed_v2(unsigned long long* p, unsigned long long a,
                                              unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long* p, unsigned long long& a,
                                              unsigned long long& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long a) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// one-dimensional bulk copy global -> shared (TMA), completion counted on an
// mbarrier of this CTA; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void mbar_init(unsigned long long* mbar) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* mbar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(src), "r"(bytes), "r"(m)
               : "memory");
}
// wait for phase `parity` of the mbarrier to complete; gives up (false)
// after `cap` polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, unsigned parity, long long cap) {
  const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
  for (long long i = 0; i < cap; ++i) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(m), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// expect `bytes` more of transaction on the mbarrier's current phase (one
// arrival: call once per phase, then issue the copies with bulk_copy)
__device__ __forceinline__ void mbar_expect(unsigned long long* mbar, unsigned bytes) {
  const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes) : "memory");
}
// a bulk copy counted against the bytes announced by mbar_expect
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* mbar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(src), "r"(bytes), "r"(m)
               : "memory");
}

}  // namespace fs1
