/*
 * fs1.h -- C ABI of the GB300 (sm_103a) FS-1 solver.
 *
 * FS-1 (Liao, Chen, Wang, Bai, Jin, Wu, "Fast Sinkhorn I: an O(N) algorithm for
 * the Wasserstein-1 metric") runs the Sinkhorn iteration of Section 2,
 * eq. "update_sinkhorn", for the entropic Wasserstein-1 problem on a uniform
 * grid (eq. "disc entropy problem"; 2D: eq. "2d disc entropy problem"), with
 * every kernel product K x replaced by the forward and backward first-order
 * recurrences of Section 3, eq. "recursion" (Section 4, eq. "2d recursion" in
 * 2D).  The problem statement follows Algorithm 1 / Algorithm 2: inputs are
 * two histograms a, b (the paper's u, v), the grid spacing h, eps, tol and
 * itr_max; the output is W_eps, the transport cost sum_ij u_i K_ij C_ij v_j of
 * the final iterate (the value Algorithm 1 returns).
 *
 * Conventions
 *   - All functions return an fs1_status; none aborts or throws.
 *   - Pointers in fs1_problem are DEVICE pointers unless the problem's
 *     `location` is FS1_MEM_HOST, in which case the library copies them into
 *     a grow-only device staging buffer of the handle (and the optional
 *     outputs back) on the handle's stream.
 *   - Calls are ordered on the handle's CUDA stream (fs1_config.stream; NULL =
 *     the legacy default stream).  fs1_w1 and fs1_solve_batch synchronise that
 *     stream before returning, so their host outputs are valid on return.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - W1 values and marginal errors are always FP64.
 */
#ifndef FS1_H
#define FS1_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fs1_status {
  FS1_OK = 0,
  FS1_EINVAL = 1,       /* bad size, spacing, eps, tol, pointer, dtype; negative or
                           non-finite mass; total masses differing by more than
                           1e-6 relative; a configuration the kernels do not cover */
  FS1_ENOMEM = 2,       /* device allocation failed or the HBM budget is exceeded */
  FS1_ENUMERIC = 3,     /* a non-finite marginal error: the iteration overflowed (the
                           paper's "terminates abnormally", Section 5.2); info.iters
                           holds the iteration at which it was detected */
  FS1_ETIMEOUT = 4,     /* a bounded device-side wait (team barrier) gave up; the
                           kernel returned without hanging the GPU */
  FS1_ENOTCONV = 5,     /* itr_max reached with err > tol.  A warning: w1 is valid */
  FS1_ECUDA = 6,        /* a CUDA runtime call failed */
  FS1_EUNSUPPORTED = 7  /* a valid request this build does not implement */
} fs1_status;

enum fs1_variant {
  FS1_VARIANT_PLAIN = 0, /* Algorithm 1 / 2 as written: linear u, v, no stabilisation */
  FS1_VARIANT_LOG = 1,   /* log-domain stabilised (Remarks in Sections 2 and 3):
                            the scalings are kept as FP32 mantissas times per-thread
                            power-of-two frames that absorb their magnitude every
                            half-step, and the chunk carries are combined with a
                            max-shifted (exponent-aligned) sum */
  FS1_VARIANT_PAPER = 2  /* the stabilised form of the Remarks as written, FP64: scalings
                            phi~, psi~ and absorbed potentials A = alpha/eps, B = beta/eps
                            per point; when max|phi~| or max|psi~| exceeds tau they are
                            absorbed (A += ln phi~, B += ln psi~, phi~ = psi~ = 1), and the
                            sweeps use the per-point factors lam e^{+-(S_{k+1} - S_k)} of
                            the replaced lines 5, 6, 10, 11.  1D, one CTA per pair,
                            N <= 16384, a and b > 0 */
};

enum fs1_precision { FS1_FP64 = 0, FS1_FP32 = 1 };
enum fs1_location { FS1_MEM_DEVICE = 0, FS1_MEM_HOST = 1 };

typedef struct fs1_config {
  int variant;          /* enum fs1_variant (default FS1_VARIANT_LOG) */
  int precision;        /* enum fs1_precision of the iteration arithmetic
                           (default FS1_FP32; FS1_VARIANT_PLAIN also takes FS1_FP64;
                           FS1_VARIANT_PAPER takes FS1_FP64 only) */
  int check_every;      /* marginal-error test every k iterations; 1 = the paper's
                           rule (default 1; only 1 is implemented) */
  int team_size;        /* CTAs that share one pair; 0 = pick from the size */
  long long spin_cap;   /* polls of a team barrier before FS1_ETIMEOUT (default 1<<22) */
  size_t hbm_budget;    /* bytes of device workspace the handle may hold; 0 = no limit */
  void* stream;         /* cudaStream_t the handle works on (NULL = default stream) */
  int autotune;         /* 1 (default): the first batch of each size class times short
                           trial solves for the candidate team sizes and keeps the best
                           (cached in the handle, and in the file named by the environment
                           variable FS1_AUTOTUNE_CACHE when set); 0: fixed heuristic.
                           Ignored when team_size > 0 */
  int trial_iters;      /* iterations of an autotune trial (default 48) */
  int use_graph;        /* 1 (default): from the second 1D call with the same launch
                           signature on, the call's device work (header copy, slot reset,
                           input check, team kernel, result copy) is one replayed CUDA
                           graph; 0: direct launches */
  double tau;           /* absorption threshold of FS1_VARIANT_PAPER (default 1e10) */
  int grid2d;           /* 2D and 3D solver: 0 (default) keeps an image resident in the
                           shared memory of one thread-block cluster of 8 to 16 CTAs
                           when it fits (2D grids of at most 512 x 512 points, 3D grids
                           of at most 64 points on the fast and middle axes and 128 on
                           the slow one, every axis with h / eps <= 8); 1 always uses
                           the grid kernel that keeps the state in device memory */
  int units;            /* stabilised 1D batches: 1 (default) solves each small pair
                           (at most 32 points per thread on 8 warps, within the frame
                           cap of h / eps) on a unit of 8, 4 or one warp, 2, 4 or 16
                           pairs side by side per CTA, after the pairs that need whole
                           CTAs, when a batch has more such pairs than co-resident CTAs
                           (fewer get a whole CTA each); 0 gives every pair whole CTAs.
                           Ignored when team_size > 0 */
} fs1_config;

typedef struct fs1_problem {
  int ndim;             /* 1 (Algorithm 1), 2 (Algorithm 2) or 3 (Algorithm 2 with a
                           third axis: the extension the closing remark of Section 4
                           states, K = K_slow (x) K_mid (x) K_fast) */
  int dtype;            /* enum fs1_precision of a and b */
  int location;         /* enum fs1_location of a, b and the optional arrays */
  int reserved;
  int64_t n[3];         /* n[0]: points along the fast (contiguous) axis.  2D: n[1]
                           along the slow axis; arrays are n[1] rows of n[0] contiguous
                           values, the paper's column-major flattening with its first
                           index (spacing h[0]) running fastest.  3D: n[1] along the
                           middle axis, n[2] along the slow one; arrays are n[2] slabs
                           of n[1] rows of n[0].  Unused entries are ignored.  2D / 3D
                           axes longer than 1024 give FS1_EUNSUPPORTED.  A 1D pair is
                           solved with its state on chip when it fits: at most
                           (co-resident CTAs, 152 on a GB300) x 512 threads x 32
                           points (8 for plain FP64), and in the stabilised variant
                           at most max(1, floor(24 eps / h[0])) points per thread.
                           A larger stabilised pair with h[0] / eps <= 5 is solved
                           with its state in device memory (fs1_info.team_size 0),
                           after the call's other problems, up to 8 such pairs
                           sharing each launch; a larger pair of the plain variants
                           or with h[0] / eps > 5 gives FS1_EUNSUPPORTED */
  double h[3];          /* grid spacings of the axes in the order of n */
  double eps;           /* entropic regularisation, > 0 */
  double tol;           /* stop when the column-marginal L1 error <= tol (>= 0) */
  int64_t itr_max;      /* iteration cap (>= 0) */
  const void* a;        /* histogram a (the paper's u): n[0]*n[1] values >= 0, sum > 0 */
  const void* b;        /* histogram b (the paper's v); same total mass as a */
  double* f_out;        /* optional: log u of the final iterate (FP64, n[0]*n[1] values,
                           same layout as a) */
  double* g_out;        /* optional: log v of the final iterate */
  const double* f_init; /* optional warm start: log u, log v of an earlier run's final */
  const double* g_init; /*   iterate (both or neither).  With the FP32 variants and the
                           same team size, a run of l1 iterations resumed for l2 more
                           ends bit-identical to one run of l1 + l2 iterations */
} fs1_problem;

typedef struct fs1_info {
  int status;           /* fs1_status of this problem */
  int variant;
  int precision;
  int team_size;        /* CTAs that shared the pair: 1D on chip, the team; 1D in device
                           memory, 0; 2D resident in a cluster's shared memory, the
                           cluster's CTAs (8 to 16); 2D / 3D on the grid kernel, 0 */
  int64_t iters;        /* completed Sinkhorn iterations l */
  double marginal_err;  /* || diag(v) K^T u - b ||_1 of the returned iterate (FP64) */
  double w1;            /* transport cost <P, C> of the returned iterate (FP64) */
  float ms;             /* device time of the solve (ms) */
  float reserved;
} fs1_info;

typedef struct fs1_handle fs1_handle;

/* Fill *cfg with the defaults listed above. */
fs1_status fs1_config_default(fs1_config* cfg);

/* Create a handle on the current CUDA device.  cfg may be NULL (defaults).
 * The handle owns its device workspace (team exchange slots, barrier counters,
 * result and descriptor arrays), which grows on demand within hbm_budget, a
 * pinned host mirror of the launch header and results, a private stream on
 * which graphs are captured (they are launched on cfg.stream), up to four
 * captured graphs, and the autotuner's table (read from FS1_AUTOTUNE_CACHE
 * when that environment variable names a readable file). */
fs1_status fs1_create(const fs1_config* cfg, fs1_handle** out);

/* Solve one problem (Algorithm 1 in 1D, Algorithm 2 in 2D and 3D).
 * w1_out: host double, may be NULL.  info_out: host, may be NULL.
 * Returns the problem's status (FS1_ENOTCONV is a warning; w1 is valid). */
fs1_status fs1_w1(fs1_handle* h, const fs1_problem* prob, double* w1_out, fs1_info* info_out);

/* Solve `count` independent problems.  1D problems of one input dtype run in
 * ONE persistent launch whatever their sizes: they are put in classes by the
 * fewest CTAs that hold a pair on chip, the GPU's CTAs are split over the
 * classes in proportion to their work (N * itr_max), and each class's teams
 * take its pairs from a queue in decreasing cost.  2D and 3D problems run
 * in launches of up to 64 grids.  Each problem's inputs are checked on the
 * device first; a failing problem gets FS1_EINVAL and is not solved.
 * w1_out (count doubles) and infos (count entries) are host arrays and may be
 * NULL.  Returns the worst status over the batch. */
fs1_status fs1_solve_batch(fs1_handle* h, const fs1_problem* probs, int64_t count,
                           double* w1_out, fs1_info* infos);

/* Apply the Gibbs kernel once with the GPU recurrences, in the log domain:
 * out_k = log sum_j exp(-|k-j| h / eps + in_j) over a 1D grid of n points
 * (the sweeps of eq. "recursion" with the stabilised arithmetic of the handle's
 * variant).  in/out: device FP64 arrays of n values (-inf allowed in `in`).
 * n must fit on chip as a 1D pair (see fs1_problem.n); larger n gives
 * FS1_EUNSUPPORTED.  Exposed for testing the scan primitive on its own. */
fs1_status fs1_kernel_apply_log(fs1_handle* h, const double* in, double* out, int64_t n,
                                double hx, double eps);

/* Test hook for the bounded device-side waits (the paper has no
 * counterpart): one stabilised pair (a, b: device FP64 arrays of n points,
 * 1024 <= n <= 32768) launched as a team of two CTAs of which only rank 0
 * runs.  Its waits for the partner's exchange slot poll at most spin_cap
 * times and give up, and the pair's result is FS1_ETIMEOUT (in *pair_status)
 * with no fault and the handle still usable.  Returns FS1_OK when the launch
 * ran, FS1_EINVAL for bad arguments or a handle of another variant. */
fs1_status fs1_test_missing_partner(fs1_handle* h, const double* a, const double* b, int64_t n, double hx,
                                    double eps, long long spin_cap, fs1_status* pair_status);

/* Release the handle and its device memory. */
void fs1_destroy(fs1_handle* h);

/* fs1_w1_noalloc -- fs1_w1 for callers that may not allocate.
 * The paper has no counterpart: this is a deployment variant of fs1_w1.
 * Some callers cannot call cudaMalloc (a memory manager already owns the
 * device's memory, an embedding forbids the library from holding device
 * memory, or a latency-critical path cannot afford an allocation that may
 * synchronise the device).  This entry point solves ONE 1D, device-located
 * problem with the same kernel as fs1_w1 and allocates nothing, on the device
 * or the host: its device scratch (descriptor, result, exchange slots, barrier
 * counter, input-check partials) is a fixed file-scope __device__ array of
 * about 84 KiB that every GPU loading the library holds until exit.  No
 * handle is needed: cfg (may be NULL for the defaults) supplies the variant,
 * precision, team size, spin cap and stream.  Every call, with the problem's
 * device current, looks up the array's device address (cudaGetSymbolAddress,
 * which allocates nothing).  The call is synchronous (it synchronises
 * cfg->stream before returning) and may not be issued on a stream that is
 * being captured.  Every call reuses the array (it is cleared where it must
 * start from zero); calls that overlap on the GPU race on it, so serialise
 * them.  With the same configuration and team size the result is
 * bit-identical to fs1_w1's.  Errors: problems that would need a team of more
 * than 160 CTAs give FS1_EINVAL (and a message on stderr); a pair beyond the
 * on-chip capacity (see fs1_problem.n) gives FS1_EUNSUPPORTED; host-located
 * problems, negative or non-finite entries and unequal masses give FS1_EINVAL.
 * w1_out, info_out: host, may be NULL; info_out->ms is not measured (0). */
fs1_status fs1_w1_noalloc(const fs1_config* cfg, const fs1_problem* prob, double* w1_out,
                          fs1_info* info_out);

/* Human-readable name of a status code (static string). */
const char* fs1_status_string(fs1_status s);

/* Counters of a handle, written to out[0..3]: graph replays, graphs
 * captured, size classes in the autotuner's table, autotune trial launches. */
fs1_status fs1_handle_stats(const fs1_handle* h, int64_t* out);

/* Which 1D solver kernel the handle's team launches took, written to
 * out[0..1]: the number of launches (autotune trials included) that used an
 * exact instantiation, and the points per thread of the most recent team
 * launch when it used one (0 when it used the generic kernel).  A team of T
 * CTAs gives each of its 512-thread CTAs' threads ceil(N / (512 T)) points of
 * an N-point pair; when every pair of a launch has the same count E and an
 * exact kernel is built for it (stabilised FP32: E = 1 .. 32; plain FP64:
 * E = 1 .. 8), that kernel runs its per-thread loops without per-point
 * guards.  out: host, 2 elements.  FS1_EINVAL for a NULL argument. */
fs1_status fs1_handle_launch_stats(const fs1_handle* h, int64_t* out);

/* Library version string. */
const char* fs1_version(void);

/* Number of CUDA kernels this library has launched in the calling process
 * (all handles, all devices).  Used to report launch counts of a timed region. */
int64_t fs1_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* FS1_H */
