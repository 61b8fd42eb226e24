// Internal declarations shared by the CUDA translation units of libpds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pds.h"

namespace pds {

constexpr int kMaxLinks = PDS_MAX_LINKS;
constexpr int kMaxState = 2 * PDS_MAX_LINKS;
constexpr int kMaxTheta = PDS_MAX_THETA;
constexpr int kMaxTraj = PDS_MAX_TRAJECTORIES;

// Everything a rollout thread needs about the problem; passed by value as a
// kernel parameter (constant bank, broadcast to all threads).
struct ChainParams {
  int n, M, T, W, D, S, P;
  int K;            // adjoint checkpoint stride
  int fast_math;    // 1: hardware sin/cos and reciprocal approximations
  int units_per_thread;  // rollout units per thread: 0 automatic, 1, or 2 (where the two-unit kernel applies)
  int max_seg;      // checkpoint slots per unit = ceil(max window length / K)
  float dt, g;
  float inv_so2;    // 1 / sigma_obs^2
  float obs_const;  // -(D/2) log(2 pi sigma_obs^2), once per observed step
  float inv_sd2;    // 1 / sigma_def^2
  float def_const;  // -(S/2) log(2 pi sigma_def^2), once per defect
  float c_lim;
  float lim_const;  // -sum_k log(hi_k - lo_k)
  int csvgd;        // 1: constrained SVGD (observation likelihood, MDMM constraints)
  float c_mdmm;     // MDMM damping c
  float mass[kMaxLinks], length[kMaxLinks], damping[kMaxLinks];
  int mass_theta[kMaxLinks], length_theta[kMaxLinks], damp_theta[kMaxLinks];  // theta row or -1
  int obs_col[kMaxState];  // observation column of each state component or -1
  float s0[kMaxTraj * kMaxState];  // start state of trajectory r at s0[r * kMaxState]
  float lo[kMaxTheta], hi[kMaxTheta];
  const float* obs;        // device [R][T][D]
  const float* obs_s;      // device [R][T][S]: the same observations in state order, unobserved components 0
  const float* obs_b;      // device [R][T][S] float2: obs_s with each value twice, (x, x)
  unsigned int obs_mask;   // bit j: state component j is observed
  int R;                   // trajectories (each with its own shooting states)
  int combine;             // R > 1: 0 equally weighted mixture (sum), 1 product
};

// Arm-and-box system parameters (added to ChainParams-based problems with
// kind == PDS_SYSTEM_ARM_BOX; ChainParams then has n = 2, M = 4, S = 4).
struct ArmBoxParams {
  float box_mass, box_side, box_com_depth, w_mass0, w_mass1, w_depth, damping;
  const float* base;  // device [T][9]: pivot omega, alpha, (a - g), pivot coordinates
};

// Rigid double pendulum (kind == PDS_SYSTEM_RIGID_DOUBLE_PENDULUM; ChainParams
// then has n = 2, S = 4 and M = the number of estimated parameters).
constexpr int kRigid2Params = 11;
struct Rigid2Params {
  float p[kRigid2Params];          // nominal values [m1, I1, c1x, c1y, b1, l, m2, I2, c2x, c2y, b2]
  int theta_row[kRigid2Params];    // particle row of each parameter, or -1 (fixed)
  int theta_param[kRigid2Params];  // parameter of each theta row (first M entries)
};

// Per-window partial results written by the rollout kernel, reduced over
// windows by the window-reduction kernel.  All [row][N] slabs.
struct Partials {
  float* lp;      // [W][N] window log-likelihood (observation + defect terms)
  float* th;      // [W][M][N] d/dtheta
  float* start;   // [W][S][N] d/d(window start state)
  float* next;    // [W][S][N] d/d(next shooting state) from the defect term
  float* tape;    // checkpoints [max_seg][S][U] then segment states [K][S][U]
  // constrained SVGD only (else NULL)
  float* th2;     // [W][M][N] -dPsi_def/dtheta of the window's defect constraint
  float* gdef;    // [W][N] defect constraint value g_def,w+1 (w < W-1)
};

// One problem of a batched launch (device-side job table entry).
struct BatchJob {
  ChainParams c;
  const float* X;    // particles [P][N]
  int N;
  int pad_;
  Partials parts;
  int32_t* status;   // [N] or NULL
};

// 128 consecutive units of one problem.
struct WorkItem {
  int job;
  int unit0;
};

// Launchers (return cudaGetLastError()).
// nu = 0: all units; otherwise the gradient kernel on units [u0, u0 + nu).
cudaError_t launch_rollout(const ChainParams& c, const float* X, int N, const Partials& parts, int grad,
                           int32_t* status, cudaStream_t st, size_t u0 = 0, size_t nu = 0);
cudaError_t launch_window_reduce(const ChainParams& c, const float* X, int N, const Partials& parts, float* logp,
                                 float* grad, int32_t* status, cudaStream_t st);
cudaError_t launch_simulate(const ChainParams& c, const float* theta, int N, float* states, cudaStream_t st);
cudaError_t launch_armbox_rollout(const ChainParams& c, const ArmBoxParams& ab, const float* X, int N,
                                  const Partials& parts, int grad, int32_t* status, cudaStream_t st);
cudaError_t launch_rigid2_rollout(const ChainParams& c, const Rigid2Params& r, const float* X, int N,
                                  const Partials& parts, int grad, int32_t* status, cudaStream_t st);
cudaError_t launch_rigid2_simulate(const ChainParams& c, const Rigid2Params& r, const float* theta, int N,
                                   float* states, cudaStream_t st);
cudaError_t launch_armbox_simulate(const ChainParams& c, const ArmBoxParams& ab, const float* theta, int N,
                                   float* states, cudaStream_t st);

struct SvgdParams {
  int N, M, P;
  float lo[kMaxTheta], hi[kMaxTheta];
  float lr, b1, b2, eps;
  int clamp;
  int fast_math;   // 1: __expf for the kernel values
  int csvgd;       // 1: constrained SVGD; the gradient then has P + M rows
  int lam0;        // constrained SVGD: first multiplier row (rows lam0..P-1 move by lr * g)
};

// Device-resident SVGD control block (no host round trip inside a step).
struct SvgdCtl {
  unsigned int hist[2048];   // radix-select histogram
  unsigned int prefix;       // resolved high bits of the median's bit pattern
  unsigned int rank;         // rank of the median within the current bucket
  int step;                  // Adam step count
  float bc1, bc2;            // Adam bias corrections 1 - beta^t
  float bw;                  // bandwidth of the current step
  float med;                 // median squared distance
  // sampled bracket [lo, hi] around the median (large N)
  float lo, hi;
  unsigned long long below;  // pairs with d < lo
  unsigned long long inside; // pairs with lo <= d <= hi (= candidates)
  int mode;                  // 0: select among candidates; 1: full radix passes over all pairs
  int tc_error;              // set if a tensor-core pass gave up waiting for its products
  unsigned int gmax[16];     // max |g_u| per component (float bits); reset at the end of each step
  unsigned int n_live;       // particles with finite coordinates and gradient (the others sit out the step)
  unsigned int live_blocks;  // blocks of the liveness pass that have finished
  // a step split in two phases (median on the coordinates, then the
  // gradient): particles whose coordinates are finite but whose gradient is
  // not, and the blocks of that check that have finished
  unsigned int gdead, gblocks;
  // candidate selection: keys are bit patterns relative to the bracket's
  // lower end, lob; bins are key >> cshift; cbin the median's bin, ccount
  // the candidates in it
  unsigned int lob, cshift, cbin, ccount;
};

struct SvgdWork {
  float* tc;       // tensor-core operand rows (a, b, v split in tf32 parts), or NULL
  float* mimg;     // tensor-core distance tiles for the median passes, or NULL
  int* mwork;      // their tiles (row tile, column tile), upper triangle
  int n_mwork;
  float* samp;     // sampled pair distances (bracket estimate)
  float* cand;     // candidate distances inside the sampled bracket
  unsigned long long cand_cap;
  float* cbuf;     // candidates of the median's bin (svgd_cbin_capacity floats)
  float* u;        // [M][N] unit-box coordinates
  float* gu;       // [M][N] gradient in unit-box coordinates
  float* phi_part; // [chunks][M][N] partial phi sums
  float* adam_m;   // [P][N]
  float* adam_v;   // [P][N]
  SvgdCtl* ctl;
  int chunks;
  int small_median;   // 1: for N <= kSmallMedianN the median in one block (all pairs in shared memory)
  int wait_limit;     // mbarrier polls before a tensor-core pass gives up (0: test once, never wait)
  int* status_flags;  // device alias of a mapped host word: kStatus* bits of the steps since the host last read it
};

// Bits of SvgdWork::status_flags, set by the last kernel of a step.
constexpr int kStatusTimeout = 1;    // a tensor-core pass gave up waiting (the step's results are not valid)
constexpr int kStatusNoneLive = 2;   // no particle had finite coordinates and gradient
// (not an error) the second phase of a split step found particles with finite
// coordinates but a gradient that is not finite, and had the median computed
// again by the full passes; the state then stops splitting its steps
constexpr int kStatusGradDead = 4;
constexpr int kWaitLimitDefault = 1 << 24;
constexpr int kSmallMedianN = 256;  // N(N-1)/2 <= 32640 pair distances (128 KB) in shared memory
constexpr int kDrainLimit = 1 << 24;  // polls of the waits that let copies and products in flight finish

// phase: kSvgdAll, or (where svgd_step_splits holds) kSvgdTheta -- the
// median bandwidth, which reads only the coordinates -- then kSvgdGrad, the
// rest, which also reads G.  The two phases in that order give the same
// results as kSvgdAll.
constexpr int kSvgdAll = 0, kSvgdTheta = 1, kSvgdGrad = 2;
cudaError_t launch_svgd_step(const SvgdParams& sp, const SvgdWork& w, float* X, const float* G, float* bw_out,
                             float* phi_out, cudaStream_t st, int* launches, int phase = kSvgdAll);
bool svgd_step_splits(const SvgdParams& sp, const SvgdWork& w);
int svgd_phi_chunks(int N);
unsigned long long svgd_cand_capacity(int N);  // 0 when the bracket path is not used
int svgd_cbin_capacity();
int svgd_sample_size();
size_t phi_tc_floats(int N, int M);
size_t median_tc_floats(int N, int M);
int median_tc_work_items(int N, int* out);
cudaError_t launch_median_tc(int N, int M, const float* u, float* img, const int* work, int n_work, SvgdCtl* ctl,
                             float* cand, unsigned long long cap, int mode, int only_in_fallback, bool prep,
                             int wait_limit, cudaStream_t st);
cudaError_t launch_phi_tc(int N, int M, const SvgdWork& w, int* slots_used, cudaStream_t st);
int phi_tc_slots(int N);
int svgd_phi_partials(int N);
cudaError_t svgd_setup_device();
cudaError_t mmd2_sums_async(const float* x, int n, const float* y, int m, int d, float inv_h, double* acc3,
                            cudaStream_t st);
cudaError_t knn_log_ratio_async(const float* p, int n, const float* q, int m, int d, int k, float* scratch2n,
                                double* acc1, cudaStream_t st);

// Record an error message for pds_last_error() and return `code`.
int set_error(int code, const char* msg);
void set_launch_count(int n);

}  // namespace pds

// Objects behind the opaque handles of pds.h.
struct pds_problem {
  int kind = PDS_SYSTEM_PLANAR_CHAIN;
  pds::ChainParams c;
  pds::ArmBoxParams ab{};
  pds::Rigid2Params r2{};
  float* d_base = nullptr;  // arm-and-box pivot motion table
  cudaStream_t stream;
  float* d_obs = nullptr;
  float* d_obs_s = nullptr;  // the observations in state order (chain rollouts)
  int cap_N = 0;          // workspace capacity in particles
  int cap_K = 0;          // checkpoint stride the tape was sized for
  int cap_cs = 0;         // workspace has the constrained-SVGD partials
  int cap_R = 0;          // trajectories the workspace was sized for
  pds::Partials parts{};
  // buffers used by pds_iterate / pds_iterate_host / batches
  int it_N = 0;
  float* d_grad = nullptr;
  float* d_logp = nullptr;
  float* d_x = nullptr;
  // pds_iterate_host: the particles' rows are copied in groups of windows,
  // each group's rollout starting on a stream of its own as its rows land
  static constexpr int kCopyGroups = 8;
  cudaStream_t ov_copy = nullptr;
  cudaStream_t ov_roll[kCopyGroups] = {};
  cudaEvent_t ov_start = nullptr;
  cudaEvent_t ov_copied[kCopyGroups] = {};
  cudaEvent_t ov_rolled[kCopyGroups] = {};
};

// What a captured SVGD step depends on besides the state's own buffers.
struct SvgdGraphKey {
  float* X;
  const float* G;
  float* bw_out;
  float* phi_out;
  int full_passes, phi_cuda_cores, median_cuda_cores, wait_limit;
  pds::SvgdParams sp;
};

struct pds_svgd {
  pds::SvgdParams sp;
  pds::SvgdWork w{};
  int* h_status = nullptr;  // mapped host word behind w.status_flags
  // the step replayed from a CUDA graph (PDS_OPT_GRAPH): captured on the
  // second call with the same key and replayed on later ones; the graphs of
  // the two most recent keys are kept (a caller that alternates two sets of
  // buffers, such as its own loop and pds_iterate_host, keeps both)
  int use_graph = 1;
  static constexpr int kGraphs = 2;
  struct Graph {
    SvgdGraphKey key{};
    int calls = 0;                  // calls made with key (0: slot unused)
    cudaGraphExec_t exec = nullptr;
    int launches = 0;               // kernels inside the graph
    long long used = 0;             // last use, for replacing the older slot
  } graphs[kGraphs];
  long long graph_clock = 0;
  // where the graph runs when the caller's stream cannot be captured (the
  // legacy or per-thread default stream): an own stream, ordered after and
  // before the caller's stream by two events
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  cudaStream_t stream;
  int full_passes = 0;
  int phi_cuda_cores = 0;
  int median_cuda_cores = 0;
  // pds_iterate's whole iteration as one graph (planar chains on a stream
  // that can be captured): the step's median phase on a high-priority side
  // stream beside the likelihood, both reading only the particles, then the
  // step's gradient phase.  Captured on the second iteration with the same
  // key, replayed afterwards.
  struct IterKey {
    const void* prob;
    float* X;
    float* logp;
    float* grad;
    int N;
    pds::ChainParams c;
    pds::Partials parts;
    SvgdGraphKey step;
  };
  IterKey iter_key{};
  int iter_calls = 0;
  int grad_dead_seen = 0;  // kStatusGradDead seen: steps are no longer split (until pds_svgd_reset)
  cudaGraphExec_t iter_exec = nullptr;
  int iter_launches = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace pds {
// Programmatic dependent launch (sm_90 and later).  A kernel that
// launch_pdl starts may be scheduled while the kernel before it on the
// stream is still finishing; its first statement is PDS_PDL_ENTRY, which
// waits until that kernel has completed and its writes are visible
// (griddepcontrol.wait; a no-op when the kernel was launched plainly) and
// then lets the next kernel be scheduled in turn.  Nothing is read or
// written before the wait, so the order of all memory effects is that of
// plain launches; only launch latency and block start-up overlap.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#define PDS_PDL_ENTRY()          \
  do {                           \
    ::pds::pdl_wait();           \
    ::pds::pdl_launch_dependents(); \
  } while (0)
#endif
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

int ensure_workspace(pds_problem* p, int N);
int ensure_iter_buffers(pds_problem* p, int N);
template <int NL>
cudaError_t launch_batch_rollout_nl(const BatchJob*, const WorkItem*, int, unsigned int*, int, int, int, int, int,
                                    cudaStream_t);
template <int NL>
int batch_rollout_blocks_per_sm_nl(int fast, int upt);
}  // namespace pds
