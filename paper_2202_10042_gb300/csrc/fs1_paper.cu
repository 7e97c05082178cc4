// fs1_paper.cu -- the stabilised FS-1 of the Remarks in Sections 2 and 3 as
// the paper writes it, in FP64, for sm_103a.
//
// State per grid point: the scalings phi~ (u), psi~ (v) and the absorbed
// potentials A = alpha/eps, B = beta/eps.  At the top of every iteration,
// when max|phi~| or max|psi~| exceeds tau, the Remark in Section 2 absorbs
// them: A += ln phi~, B += ln psi~, phi~ = psi~ = 1.  The kernel products are
// those of the rescaled K~ = diag(e^A) K diag(e^B): the Remark in Section 3
// replaces lines 5, 6, 10 and 11 of Algorithm 1 by recurrences whose factor
// between points k and k+1 is lam e^{S_{k+1}-S_k} (forward) or
// lam e^{S_k-S_{k+1}} (backward) for the scale field S of the output (B for
// the v-update, A for the u-update), on the input e^{A+B} phi~ (or psi~).
//
// One CTA of 512 threads owns a pair (N <= 16384).  Thread t owns the
// contiguous chunk [t E, t E + E), E = ceil(N / 512).  With per-point factors
// a chunk acts on the value entering it as an affine map r -> D r + X (D the
// product of its factors); the maps are composed by a warp Kogge-Stone scan
// and a scan over the 16 warp totals, so every thread gets the value that
// enters its chunk (forward: r at the point before its first point; backward:
// s at its last point) and finishes the sweep serially.  The transport cost of
// the final iterate uses the distance-weighted recurrences with the same
// factors, whose chunk maps act on the pair (r, G).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "fs1.h"
#include "fs1_internal.h"

namespace fs1 {

namespace {

constexpr int kT = 512;
constexpr int kW = kT / 32;
constexpr unsigned kFull = 0xffffffffu;

// an affine map s -> d s + x (the effect of a span of points on the value
// entering it)
struct Map {
  double d, x;
};
__device__ __forceinline__ Map after(Map first, Map second) {   // second o first
  return Map{second.d * first.d, second.d * first.x + second.x};
}

// the distance-weighted sweep's map on (r, G): r -> p r + x, G -> q r + p G + g
struct Map2 {
  double p, q, x, g;
};
__device__ __forceinline__ Map2 after(Map2 a, Map2 b) {   // b o a
  return Map2{b.p * a.p, b.q * a.p + b.p * a.q, b.p * a.x + b.x, b.q * a.x + b.p * a.g + b.g};
}

__device__ __forceinline__ Map shfl(Map m, int o, bool up) {
  return up ? Map{__shfl_up_sync(kFull, m.d, o), __shfl_up_sync(kFull, m.x, o)}
            : Map{__shfl_down_sync(kFull, m.d, o), __shfl_down_sync(kFull, m.x, o)};
}
__device__ __forceinline__ Map2 shfl(Map2 m, int o, bool up) {
  if (up)
    return Map2{__shfl_up_sync(kFull, m.p, o), __shfl_up_sync(kFull, m.q, o), __shfl_up_sync(kFull, m.x, o),
                __shfl_up_sync(kFull, m.g, o)};
  return Map2{__shfl_down_sync(kFull, m.p, o), __shfl_down_sync(kFull, m.q, o), __shfl_down_sync(kFull, m.x, o),
              __shfl_down_sync(kFull, m.g, o)};
}
__device__ __forceinline__ Map identity(Map) { return Map{1.0, 0.0}; }
__device__ __forceinline__ Map2 identity(Map2) { return Map2{1.0, 0.0, 0.0, 0.0}; }

// The composition of the maps of all threads before this one in scan order
// (FWD: ascending thread index; else descending), as a map.  sw: kW entries
// of shared memory.
template <bool FWD, class M>
__device__ M exclusive_map(M m, M* sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  M inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const M y = shfl(inc, o, FWD);
    if (FWD ? lane >= o : lane + o < 32) inc = after(y, inc);
  }
  M ex = shfl(inc, 1, FWD);
  if (FWD ? lane == 0 : lane == 31) ex = identity(m);
  if (FWD ? lane == 31 : lane == 0) sw[warp] = inc;
  __syncthreads();
  M cw = identity(m);   // the warps before this one, composed in scan order
  if (FWD)
    for (int w = 0; w < warp; ++w) cw = after(cw, sw[w]);
  else
    for (int w = kW - 1; w > warp; --w) cw = after(cw, sw[w]);
  __syncthreads();   // sw is reused by the next scan
  return after(cw, ex);
}

__device__ double block_sum(double v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kW; ++w) t += sred[w];   // fixed order: every thread gets the same sum
  __syncthreads();
  return t;
}

// maximum over the CTA; NaNs are ignored (fmax), as a comparison with tau
// ignores them
__device__ double block_max(double v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = -INFINITY;
  for (int w = 0; w < kW; ++w) t = fmax(t, sred[w]);
  __syncthreads();
  return t;
}

struct Arrays {
  double *ph, *ps, *A, *B, *eab, *ffb, *fbb, *ffa, *fba, *y;
};

// factors of the scale field S between k and k+1 (0 at the last point)
__device__ void set_factors(const double* S, double* ff, double* fb, int64_t N, double lam, int64_t k0, int64_t k1) {
  for (int64_t k = k0; k < k1; ++k) {
    if (k + 1 < N) {
      const double d = S[k + 1] - S[k];
      ff[k] = lam * exp(d);
      fb[k] = lam * exp(-d);
    } else {
      ff[k] = fb[k] = 0.0;
    }
  }
}

// y = e^S K e^-S x over the pair: forward r_k = ff_{k-1} r_{k-1} + x_k, backward
// s_k = fb_k (s_{k+1} + x_{k+1}), y = r + s (eq. "recursion" with the factors
// of the Remark in Section 3).  x_k = eab_k w_k.
__device__ void sweep(const double* eab, const double* w, const double* ff, const double* fb, double* y, int64_t N,
                      int64_t k0, int64_t k1, Map* sw) {
  // forward: chunk map on r_{k0-1}
  Map m{1.0, 0.0};
  for (int64_t k = k0; k < k1; ++k) {
    const double f = k > 0 ? ff[k - 1] : 0.0;
    m = Map{f * m.d, f * m.x + eab[k] * w[k]};
  }
  const Map pre = exclusive_map<true>(m, sw);
  double r = pre.x;   // r at k0 - 1 (the composition applied to r_{-1} = 0)
  for (int64_t k = k0; k < k1; ++k) {
    r = (k > 0 ? ff[k - 1] : 0.0) * r + eab[k] * w[k];
    y[k] = r;
  }
  // backward: chunk map from s_{k1-1} to s_{k0-1}
  Map b{1.0, 0.0};
  for (int64_t k = k1 - 2; k >= k0 - 1 && k >= 0; --k) b = Map{fb[k] * b.d, fb[k] * (b.x + eab[k + 1] * w[k + 1])};
  if (k0 == 0 && k1 > k0) b = Map{0.0, 0.0};   // nothing lies left of point 0
  const Map post = exclusive_map<false>(b, sw);
  double s = post.x;   // s at k1 - 1 (s_{N-1} = 0)
  if (k1 > k0) y[k1 - 1] += s;
  for (int64_t k = k1 - 2; k >= k0; --k) {
    s = fb[k] * (s + eab[k + 1] * w[k + 1]);
    y[k] += s;
  }
}

// distance-weighted sweep: forward G_k = ff_{k-1} (G_{k-1} + r_{k-1}),
// backward H_k = fb_k (H_{k+1} + s_{k+1} + x_{k+1}); returns
// sum_k phi~_k h (G_k + H_k) over this thread's chunk
__device__ double wsweep_dot(const double* eab, const double* w, const double* ff, const double* fb,
                             const double* ph, double h, int64_t N, int64_t k0, int64_t k1, Map2* sw2, double* y) {
  Map2 m{1.0, 0.0, 0.0, 0.0};
  for (int64_t k = k0; k < k1; ++k) {
    const double f = k > 0 ? ff[k - 1] : 0.0;
    // (r, G) -> (f r + x, f r + f G)
    m = after(m, Map2{f, f, eab[k] * w[k], 0.0});
  }
  const Map2 pre = exclusive_map<true>(m, sw2);
  double r = pre.x, G = pre.g;
  for (int64_t k = k0; k < k1; ++k) {
    const double f = k > 0 ? ff[k - 1] : 0.0;
    G = f * (G + r);
    r = f * r + eab[k] * w[k];
    y[k] = G;
  }
  // backward on (s, H): (s, H) -> (f (s + x), f (H + s + x)) with x = x_{k+1}
  Map2 b{1.0, 0.0, 0.0, 0.0};
  for (int64_t k = k1 - 2; k >= k0 - 1 && k >= 0; --k) {
    const double f = fb[k], x = eab[k + 1] * w[k + 1];
    b = after(b, Map2{f, f, f * x, f * x});
  }
  if (k0 == 0 && k1 > k0) b = Map2{0.0, 0.0, 0.0, 0.0};
  const Map2 post = exclusive_map<false>(b, sw2);
  double s = post.x, H = post.g;
  double acc = 0.0;
  if (k1 > k0) acc += ph[k1 - 1] * h * (y[k1 - 1] + H);
  for (int64_t k = k1 - 2; k >= k0; --k) {
    const double f = fb[k], x = eab[k + 1] * w[k + 1];
    H = f * (H + s + x);
    s = f * (s + x);
    acc += ph[k] * h * (y[k] + H);
  }
  return acc;
}

__device__ __forceinline__ double mass(const void* p, int64_t i, int f32) {
  return f32 ? (double)reinterpret_cast<const float*>(p)[i] : reinterpret_cast<const double*>(p)[i];
}

__global__ void __launch_bounds__(kT) fs1_paper_kernel(const PairDesc* pairs, PairResult* results, double* ws,
                                                       const int64_t* off, int in_f32, double tau,
                                                       const int* valid) {
  __shared__ Map sw[kW];
  __shared__ Map2 sw2[kW];
  __shared__ double sred[kW];
  const int pid = blockIdx.x;
  const PairDesc P = pairs[pid];
  const int64_t N = P.n;
  if ((valid && !valid[pid]) || N > kMaxPaperN) {
    if (threadIdx.x == 0) results[pid] = PairResult{NAN, NAN, 0, N > kMaxPaperN ? FS1_EUNSUPPORTED : FS1_EINVAL, 0};
    return;
  }
  double* base = ws + off[pid];
  Arrays S{base, base + N, base + 2 * N, base + 3 * N, base + 4 * N, base + 5 * N,
           base + 6 * N, base + 7 * N, base + 8 * N, base + 9 * N};
  const int64_t E = (N + kT - 1) / kT;
  const int64_t k0 = min(N, (int64_t)threadIdx.x * E), k1 = min(N, k0 + E);
  const double h = P.h_fast, lam = exp(-h / P.eps);

  // the stabilised form needs a, b > 0 (the logarithms of absorption)
  double amin = INFINITY;
  for (int64_t k = k0; k < k1; ++k) amin = fmin(amin, fmin(mass(P.a, k, in_f32), mass(P.b, k, in_f32)));
  amin = -block_max(-amin, sred);
  if (!(amin > 0.0)) {
    if (threadIdx.x == 0) results[pid] = PairResult{NAN, NAN, 0, FS1_EINVAL, 0};
    return;
  }

  // the initialisation of Algorithm 1 (phi = psi = 1/N), or a warm start: the given log
  // potentials become the absorbed A, B with phi~ = psi~ = 1
  const bool warm = P.f_init != nullptr;
  for (int64_t k = k0; k < k1; ++k) {
    S.A[k] = warm ? P.f_init[k] : 0.0;
    S.B[k] = warm ? P.g_init[k] : 0.0;
    S.ph[k] = S.ps[k] = warm ? 1.0 : 1.0 / (double)N;
    S.eab[k] = exp(S.A[k] + S.B[k]);
  }
  __syncthreads();
  set_factors(S.B, S.ffb, S.fbb, N, lam, k0, k1);
  set_factors(S.A, S.ffa, S.fba, N, lam, k0, k1);
  __syncthreads();

  int64_t ell = 0;
  double err = 0.0;
  int status = FS1_OK;
  for (;;) {
    // absorption test (Remark, Section 2): infinity norms against tau
    double mx = 0.0;
    for (int64_t k = k0; k < k1; ++k) mx = fmax(mx, fmax(fabs(S.ph[k]), fabs(S.ps[k])));
    mx = block_max(mx, sred);
    if (mx > tau) {
      for (int64_t k = k0; k < k1; ++k) {
        S.A[k] += log(S.ph[k]);
        S.B[k] += log(S.ps[k]);
        S.ph[k] = S.ps[k] = 1.0;
        S.eab[k] = exp(S.A[k] + S.B[k]);
      }
      __syncthreads();
      set_factors(S.B, S.ffb, S.fbb, N, lam, k0, k1);
      set_factors(S.A, S.ffa, S.fba, N, lam, k0, k1);
      __syncthreads();
    }
    // r, s sweeps on phi~: y = e^B K^T (e^A phi~)
    sweep(S.eab, S.ph, S.ffb, S.fbb, S.y, N, k0, k1, sw);
    // the while condition: sum_j |psi_j (K^T phi)_j - v_j|
    double e = 0.0;
    for (int64_t k = k0; k < k1; ++k) e += fabs(S.ps[k] * S.y[k] - mass(P.b, k, in_f32));
    err = block_sum(e, sred);
    if (!isfinite(err)) {
      status = FS1_ENUMERIC;
      break;
    }
    if (ell >= P.itr_max || err <= P.tol) break;
    // psi~ = v / (r + s)
    for (int64_t k = k0; k < k1; ++k) S.ps[k] = mass(P.b, k, in_f32) / S.y[k];
    __syncthreads();
    // p, q sweeps on psi~: y = e^A K (e^B psi~); phi~ = u / (p + q)
    sweep(S.eab, S.ps, S.ffa, S.fba, S.y, N, k0, k1, sw);
    for (int64_t k = k0; k < k1; ++k) S.ph[k] = mass(P.a, k, in_f32) / S.y[k];
    __syncthreads();
    ++ell;
  }
  // transport cost of the final iterate: sum phi~_k h (G_k + H_k), the
  // e^A-scaled distance-weighted sweeps of e^{A+B} psi~
  double w = NAN;
  if (status == FS1_OK) {
    __syncthreads();
    w = block_sum(wsweep_dot(S.eab, S.ps, S.ffa, S.fba, S.ph, h, N, k0, k1, sw2, S.y), sred);
    if (!isfinite(w)) status = FS1_ENUMERIC;
  }
  if (P.f_out)
    for (int64_t k = k0; k < k1; ++k) P.f_out[k] = S.A[k] + log(S.ph[k]);
  if (P.g_out)
    for (int64_t k = k0; k < k1; ++k) P.g_out[k] = S.B[k] + log(S.ps[k]);
  if (threadIdx.x == 0) {
    PairResult R;
    R.w = status == FS1_OK ? w : NAN;
    R.err = err;
    R.iters = ell;
    R.status = status;
    if (status == FS1_OK && !(err <= P.tol)) R.status = FS1_ENOTCONV;
    R.pad = 0;
    results[pid] = R;
  }
}

}  // namespace

int launch_paper_1d(const PairDesc* d_pairs, int count, PairResult* d_results, double* ws, const int64_t* d_off,
                    int in_f32, double tau, const int* d_valid, void* stream) {
  fs1_paper_kernel<<<count, kT, 0, (cudaStream_t)stream>>>(d_pairs, d_results, ws, d_off, in_f32, tau, d_valid);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "fs1: paper-form launch failed: %s\n", cudaGetErrorString(e));
    return FS1_ECUDA;
  }
  return FS1_OK;
}

}  // namespace fs1
