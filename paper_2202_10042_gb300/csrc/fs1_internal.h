// fs1_internal.h -- structures shared by the host runtime and the kernels.
// Not part of the public C-ABI (include/fs1.h).
#pragma once
#include <cstddef>
#include <cstdint>

namespace fs1 {

// Per-pair input of a solve launch (device memory).
struct PairDesc {
  const void* a;          // histogram a (dtype of the launch), n[0]*n[1] values
  const void* b;          // histogram b
  int64_t n;              // number of grid points (1D: N; 2D / 3D: the product of the axes)
  int64_t n_fast;         // fast-axis (contiguous) length; 1D: n
  int64_t n_mid;          // middle-axis length (3D); 1 otherwise
  int64_t n_slow;         // slow-axis length (2D, 3D); 1D: 1
  double h_fast, h_mid, h_slow;  // grid spacings
  double eps, tol;
  int64_t itr_max;
  double* f_out;          // optional log potentials out (FP64), may be null
  double* g_out;
  const double* f_init;   // optional warm start (FP64 log potentials), may be null
  const double* g_init;
};

// Per-pair result (device memory).
struct PairResult {
  double w;       // transport cost <P, C> of the final iterate
  double err;     // marginal L1 error of the final iterate
  int64_t iters;  // completed iterations
  int status;     // fs1_status value
  int pad;        // CTAs that solved the problem: a 1D team, or the cluster of a 2D image resident on
                  // chip (0: the 2D grid kernel, the streamed path, the paper form)
};

// Exchange slot of one CTA of a team (one per CTA and buffer parity): up to
// 16 64-bit words, each a 32-bit payload tagged with the exchange epoch.  Slots
// must be zeroed before every launch.
struct alignas(16) Slot {
  unsigned char raw[128];
};

struct TeamLaunch {
  const PairDesc* pairs;
  PairResult* results;
  const int* order;                // pair order (cost-sorted); may be null
  int num_pairs;
  int team_size;                   // T: CTAs per team
  int num_teams;
  int in_f32;                      // 1: a, b are float; 0: double
  Slot* slots;                     // [num_teams][2][team_size] generic slots
  unsigned long long* cslots;      // [num_teams][2][team_size][16] compact slots
                                   // (stabilised path); zeroed per launch
  unsigned long long* counters;    // [num_teams] reserved (zeroed per launch)
  int* abort_flags;                // [num_teams] (zeroed per launch)
  long long spin_cap;              // bounded-wait polls before giving up
  // Heterogeneous teams with dynamic work queues (all null / 0: uniform teams
  // of team_size CTAs taking pairs team, team + num_teams, ...).
  int grid;                        // CTAs of the launch (0: num_teams * team_size)
  const int* cta_team;             // [grid] team of each CTA
  const int* cta_rank;             // [grid] rank of each CTA in its team
  const int* team_T;               // [num_teams] CTAs of each team
  const int* team_slot;            // [num_teams] first slot of the team's [2][T] slots
  const int* team_class;           // [num_teams] work class served by the team
  const int* class_off;            // [nclass + 1] offsets of each class's pairs in `order`
  int* class_next;                 // [nclass] queue heads (zeroed per launch)
  unsigned long long* tickets;     // [num_teams] pair broadcast words (zeroed per launch);
                                   // [nlevel][grid] under a level schedule
  // Level schedule (nlevel > 0): every CTA starts in a team of level_T[0]
  // CTAs serving the queue of the largest class; a team whose queue is empty
  // splits into the teams of the next level (level_T decreasing, each
  // dividing the one before), which serve the next class down.  Slots are
  // [nlevel][2 grid]; cta_team .. team_class describe level 0.
  int nlevel;
  const int* level_T;              // [nlevel]
  // Units (generic stabilised kernel, unit_queues = 1): after the teams'
  // queues, every CTA solves small pairs as 2 units of 8 warps on the queue
  // of class unit_class, each unit then as 2 units of 4 warps on the queue of
  // class unit_class + 1 and each of those as 4 single warps on the queue of
  // class unit_class + 2 (a pair per unit, its points in the unit's threads).
  int unit_queues;
  int unit_class;
  const int* valid;                // [num_pairs] 0: the pair failed the input check and is
                                   // reported FS1_EINVAL without solving; null: all valid
};

// Largest team: the team reduction stages one slot per CTA in shared memory.
constexpr int kMaxTeamCtas = 256;

enum KernelKind {
  KK_PLAIN_F64 = 0,   // plain FS-1 (Algorithm 1 as written), FP64
  KK_PLAIN_F32 = 1,   // plain FS-1, FP32 (no stabilisation)
  KK_LOG_F32 = 2,     // stabilised FS-1: FP32 mantissas in extended range
  KK_PAPER_F64 = 3,   // the Remarks' tau-triggered absorption as written, FP64
};

// 2D / 3D solver (fs1_solve2d.cu): up to kMaxImg2D grids per launch.
constexpr int kMaxImg2D = 64;
constexpr int kMaxLine2D = 1024;   // longest line along any axis (staged in shared memory)
size_t solve2d_workspace(const PairDesc* host_descs, int count);
// Launch class of a grid image: 0 the general path with FP32-frame scans on
// every axis, 1 the general path scanning some axis point by point in
// extended range, 2 the FP32 block-frame path (2D, axes of at most 1024
// points whose lane chunks of P points have P h / eps <= 64, where the
// general path would scan point by point).  A launch_solve_2d call whose
// images are all of class 2 runs the FP32 path; callers launch the classes
// separately.
int solve2d_class(const PairDesc& d);
int solve2d_f32_ok(const PairDesc& d);
int launch_solve_2d(const PairDesc* host_descs, int count, int in_f32, PairResult* d_results, void* ws,
                    size_t ws_bytes, long long spin_cap, void* stream);

// Cluster-resident 2D solver (fs1_cluster2d.cu): an image in the shared
// memory of one 16-CTA cluster.  cluster2d_inst: the instantiation that holds
// the image (-1: none; the grid kernel solves it).  launch_cluster_2d solves
// d[0 .. count), all with cluster2d_inst >= 0; an image whose scalings leave
// the kernel's exponent range ends with FS1_EUNSUPPORTED (the caller solves it
// again with the grid kernel).  *launches is incremented per kernel launch.
int cluster2d_inst(const PairDesc& d);
size_t cluster2d_workspace(const PairDesc* d, int count);
int launch_cluster_2d(const PairDesc* d, int count, int in_f32, PairResult* results, const int* d_valid, void* ws,
                      size_t ws_bytes, void* stream, long long* launches);

// Stabilised 1D solver with the state in device memory (fs1_stream.cu), for
// pairs beyond the team kernel's on-chip capacity: workspace bytes for pairs
// of n[0 .. count) points, and the solve of count pairs (host descriptors;
// d_results: device array of count; *launches: kernels issued), up to 8
// pairs sharing each half-step launch.
size_t stream_workspace(const int64_t* n, int count);
// largest h / eps of a streamed pair: the 16 values of a thread's run share
// one FP32 frame, so they may span at most 16 h / eps = 80 nats (e^-80 is
// still a normal FP32 number relative to the run's largest value)
constexpr double kStreamMaxC = 5.0;
int solve_stream_batch(const PairDesc* host_desc, const int* in_f32, int count, PairResult* d_results, void* ws,
                       size_t ws_bytes, void* stream, long long* launches);

// Paper-form solver (fs1_paper.cu): one CTA per pair, N <= kMaxPaperN.
constexpr int kMaxPaperN = 16384;
// FP64 doubles of per-pair workspace per grid point
constexpr int kPaperArrays = 10;
// d_off[i]: offset (in doubles) of pair i's kPaperArrays x N workspace in ws;
// d_valid: input-check flags (may be null).
int launch_paper_1d(const PairDesc* d_pairs, int count, PairResult* d_results, double* ws, const int64_t* d_off,
                    int in_f32, double tau, const int* d_valid, void* stream);

// Host-side launch helpers (fs1_solve1d.cu).
int team_threads();
int team_elems_max(int kind);
size_t team_smem_bytes(int kind);
// Largest elements-per-thread the stabilised variant allows for c = h/eps.
int elems_cap_for(int kind, double c);
// Launch the 1D team kernel; cooperative when team_size > 1.
// exact_E > 0: every pair of the launch has that many points per thread, and
// the exact instantiation is used when one is built for it
int launch_team_1d(int kind, const TeamLaunch& L, void* stream, int exact_E = 0);
// whether an exact instantiation of E points per thread is built for kind
bool team_exact_built(int kind, int E);
int max_coresident_ctas(int kind);
// Add k to the process-wide count of kernels this library launched.
void note_launches(long long k);

}  // namespace fs1
