/*
 * pds.h -- C ABI of the GB300 (sm_103a) library for probabilistic inference
 * of simulation parameters by multiple-shooting SVGD over a differentiable
 * planar articulated-body simulator.
 *
 * The operations follow the paper's problem statement (Sec. III, Algorithm 1
 * inputs): a differentiable simulator f_sim, an observation function f_obs,
 * the start state of the measured trajectory, the measured trajectory, a
 * step-size rule (Adam) and a kernel (RBF).  The library evaluates, for every
 * particle, the multiple-shooting log-likelihood (Sec. IV-C, Eqs. 2, 4, 5)
 * plus the parameter-limit prior (Sec. IV-D) and its gradient, and applies the
 * SVGD update of Eq. (1).
 *
 * Conventions shared by every entry point:
 *  - Return PDS_OK (0) on success, a negative PDS_ERR_* code otherwise;
 *    pds_last_error() gives a message for the calling thread.  No C++
 *    exception crosses the ABI.
 *  - Pointers documented "device" must be CUDA device (or managed) memory
 *    owned by the caller; "host" pointers are read during the call only.
 *  - Particle arrays are structure-of-arrays: element (row r, particle i)
 *    lives at [r * N + i] (particle index fastest).
 *  - Calls are asynchronous on the CUDA stream given at creation unless
 *    stated otherwise; the caller synchronises before reading results.
 *  - Objects are not thread-safe: one host thread drives one object at a time.
 */
#ifndef PDS_H_
#define PDS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDS_OK 0
#define PDS_ERR_ARG (-1)         /* invalid argument (NULL, size out of range) */
#define PDS_ERR_CUDA (-2)        /* a CUDA runtime call or launch failed       */
#define PDS_ERR_OOM (-3)         /* device allocation failed                   */
#define PDS_ERR_NONFINITE (-4)   /* an SVGD step found no finite particle      */
#define PDS_ERR_TIMEOUT (-5)     /* a bounded device wait ran out              */
#define PDS_ERR_BUDGET (-6)      /* job larger than the server's memory budget */
#define PDS_ERR_UNSUPPORTED (-7) /* configuration outside the compiled range   */

#define PDS_SYSTEM_PLANAR_CHAIN 1
#define PDS_SYSTEM_ARM_BOX 2
#define PDS_SYSTEM_RIGID_DOUBLE_PENDULUM 3

#define PDS_PARAM_MASS 0    /* point mass at the tip of a link [kg]          */
#define PDS_PARAM_LENGTH 1  /* link length [m]                               */
#define PDS_PARAM_DAMPING 2 /* viscous joint damping [N m s / rad]           */

#define PDS_MAX_LINKS 8
#define PDS_MAX_THETA 16
#define PDS_MAX_WINDOW_STEPS 4096
#define PDS_MAX_TRAJECTORIES 8

/* Articulated system (Appendix B-A: the simulator computes joint
 * accelerations with the articulated-body algorithm and integrates them with
 * semi-implicit Euler).  PDS_SYSTEM_PLANAR_CHAIN: a planar serial chain of
 * revolute joints with relative joint angles, q = 0 hanging straight down
 * along -y, a point mass at the tip of each link and joint torque
 * tau_i = -damping_i * qd_i.  State s = [q_0..q_{n-1}, qd_0..qd_{n-1}]. */
typedef struct pds_system_desc {
  int kind;               /* PDS_SYSTEM_PLANAR_CHAIN                        */
  int n_links;            /* 1..PDS_MAX_LINKS                                */
  const double* mass;     /* host [n_links]; used where theta does not override */
  const double* length;   /* host [n_links]                                  */
  const double* damping;  /* host [n_links]                                  */
  double gravity;         /* magnitude of gravity along -y [m/s^2]           */
  int n_theta;            /* M = dim theta, 1..PDS_MAX_THETA                 */
  const int* theta_kind;  /* host [M], PDS_PARAM_*                           */
  const int* theta_link;  /* host [M], 0-based link index; each (kind, link) at most once */
} pds_system_desc;

/* Arm shaking a box (the paper's Panda-arm experiment, Sec. V-C, as a
 * synthetic system).  A serial arm of n_arm revolute joints (axes alternate
 * z, y, z, ... of the link frames; joint j+1 sits arm_len[j] along the local
 * z axis of link j; joint 1 at the world origin; gravity along -z) follows
 * prescribed trajectories q_j(t) = sum_k amp[j][k] sin(2 pi freq[j][k] t +
 * phase[j][k]).  At the tip of the last link a box hangs on two passive
 * revolute joints at the same point (axis x, then axis y: a U-joint) with
 * viscous damping.  The box is a solid cube (box_mass, box_side, its centre
 * box_com_depth below the joint) plus two point weights (weight_mass[k]) at
 * (x_k, y_k, -weight_depth) in the box frame.  theta = (x1, y1, x2, y2);
 * state s = [q1, q2, qd1, qd2] of the box joints. */
typedef struct pds_armbox_desc {
  int n_arm;             /* 1..8 */
  const double* arm_len; /* host [n_arm] */
  const double* amp;     /* host [n_arm][3] rad */
  const double* freq;    /* host [n_arm][3] Hz */
  const double* phase;   /* host [n_arm][3] rad */
  double box_mass, box_side, box_com_depth;
  double weight_mass[2];
  double weight_depth;
  double gravity;
  double damping;        /* box joint damping [N m s / rad] */
} pds_armbox_desc;

typedef struct pds_problem* pds_problem_t;
typedef struct pds_svgd* pds_svgd_t;
typedef struct pds_sgld* pds_sgld_t;

/* Create a multiple-shooting inference problem (Sec. IV-C).
 *  dt, T      : time step and number of steps of the measured trajectory.
 *  windows    : number of shooting windows W, 1 <= W <= T.  Window w covers
 *               steps t_w+1..t_{w+1} with t_w = floor(w*T/W); window 0 starts
 *               at s0, window w > 0 at the particle's shooting state s^s_w.
 *               At most PDS_MAX_WINDOW_STEPS steps per window.
 *  obs        : host [T][D] float; row t-1 is the observation x_t (Eq. 2).
 *  obs_index  : host [D]; observation column d is state component obs_index[d]
 *               (f_obs selects state components; each at most once).
 *  sigma_obs  : observation noise std (Eq. 2); sigma_def: defect std (Eq. 4).
 *  s0         : host [2n] known start state s_0 (Sec. III).
 *  theta_lo/hi: host [M] parameter box of the uniform prior (Sec. IV-D).
 *  c_lim      : stiffness of the smooth limit penalty added to log p_lim,
 *               -(c_lim/2) * ||clamp(u,0,1) - u||^2 with u the unit-box
 *               coordinates of theta (0 disables it).
 *  cuda_stream: cudaStream_t the problem's work is queued on (NULL = legacy
 *               default stream).
 * The problem copies everything it needs to the device; it owns that memory
 * and its workspace.  Particle layout: P = M + (W-1)*2n rows: theta first,
 * then s^s_1 .. s^s_{W-1}, each 2n rows. */
int pds_problem_create(const pds_system_desc* sys, double dt, int T, int windows,
                       const float* obs, int D, const int* obs_index,
                       double sigma_obs, double sigma_def, const float* s0,
                       const float* theta_lo, const float* theta_hi, double c_lim,
                       void* cuda_stream, pds_problem_t* out);

/* Multiple-shooting problem of the arm-and-box system; arguments as
 * pds_problem_create (obs_index indexes the box state [q1, q2, qd1, qd2];
 * theta box and particles have M = 4, S = 4).  The arm's pivot motion is
 * tabulated on the host for every time step and kept on the device.  The
 * gradient comes from tangents propagated forward through each window
 * (theta and the window's start state: 8 directions). */
int pds_problem_create_armbox(const pds_armbox_desc* sys, double dt, int T, int windows,
                              const float* obs, int D, const int* obs_index, double sigma_obs,
                              double sigma_def, const float* s0, const float* theta_lo,
                              const float* theta_hi, double c_lim, void* cuda_stream,
                              pds_problem_t* out);

/* Rigid double pendulum with general inertia and centre of mass: the
 * 11-parameter model of the physical double pendulum of Sec. V's real-world
 * experiment (App. Table params-ibm-pendulum).  Two rigid links on parallel
 * revolute joints (axis z); joint 1 at the origin, joint 2 at (0, -l) in link
 * 1's frame; gravity along -y.  Link k has mass m_k, centre of mass
 * (ckx, cky) in its frame, rotational inertia I_k about its COM (the inertia
 * tensor I_k times the identity; only the z component acts) and viscous joint
 * friction -b_k qd_k.  State s = [q1, q2, qd1, qd2] (q = 0: link frames
 * aligned with the world; a COM along -y then hangs at rest).  Parameters,
 * in the table's order:
 *   0 m1, 1 I1, 2 c1x, 3 c1y, 4 b1, 5 l, 6 m2, 7 I2, 8 c2x, 9 c2y, 10 b2. */
typedef struct pds_rigid2_desc {
  double param[11];       /* nominal values; estimated entries are overridden */
  double gravity;
  int n_theta;            /* 1..11 estimated parameters                      */
  const int* theta_param; /* host [n_theta]: distinct indices into param      */
} pds_rigid2_desc;

/* Create a multiple-shooting problem of the rigid double pendulum; the other
 * arguments are as for pds_problem_create (S = 4, P = M + (W-1)*4).  The
 * gradient comes from a hand-written reverse sweep with checkpoints every K
 * steps, as for the chains.  Constrained SVGD and trajectory sets are not
 * supported for this system (PDS_ERR_UNSUPPORTED); batched execution and the
 * server run it on its own branch, like the arm-and-box system. */
int pds_problem_create_rigid2(const pds_rigid2_desc* sys, double dt, int T, int windows,
                              const float* obs, int D, const int* obs_index, double sigma_obs,
                              double sigma_def, const float* s0, const float* theta_lo,
                              const float* theta_hi, double c_lim, void* cuda_stream,
                              pds_problem_t* out);

/* Release the problem and all device memory it owns (synchronises its stream). */
int pds_problem_destroy(pds_problem_t p);

/* Report M (= dim theta), S (= 2n, state size) and P (= M + (W-1)*S, or as
 * pds_problem_set_csvgd / pds_problem_set_trajectories change it). */
int pds_problem_layout(pds_problem_t p, int* M, int* S, int* P);

/* Adjoint checkpoint stride K (default 1): the reverse sweep keeps one
 * state every K steps and recomputes the states in between (the gradient is
 * the same for every K up to rounding).  K = 1 keeps every state
 * (T x 2n x N floats of device memory per problem) and recomputes nothing;
 * larger K trades recomputation for memory.  1 <= K <= PDS_MAX_WINDOW_STEPS. */
int pds_problem_set_checkpoint_stride(pds_problem_t p, int K);

/* Tuning options of a problem (pds_problem_set_option / _get_option):
 *  PDS_OPT_CHECKPOINT_STRIDE: K as in pds_problem_set_checkpoint_stride.
 *  PDS_OPT_FAST_MATH: 0 (default) = CUDA's sinf/cosf and IEEE division in the
 *    rollout; 1 = the hardware approximations __sincosf / __fdividef (results
 *    stay within the same parity tolerances against the FP64 oracle:
 *    relative 1e-4 on log p, 1e-3 on the gradient). */
#define PDS_OPT_CHECKPOINT_STRIDE 1
#define PDS_OPT_FAST_MATH 2
/*  PDS_OPT_UNITS_PER_THREAD: rollout units (particle-windows) per GPU thread
 *    in pds_loglik_grad.  1 = one; 2 = two particles of a window per thread,
 *    each quantity held as a pair so that the step's FP32 arithmetic issues
 *    as paired (f32x2) instructions; 0 (default) = two for the chain lengths
 *    where that measured faster (2, 4 and 5 links), else one.  Two apply only
 *    to planar chains with K = 1, every state component observed, an even
 *    particle count and no constrained SVGD; elsewhere one is used.  Both
 *    give the same results bit for bit. */
#define PDS_OPT_UNITS_PER_THREAD 8
int pds_problem_set_option(pds_problem_t p, int option, int value);
int pds_problem_get_option(pds_problem_t p, int option, int* value);

/* Autotuner of the likelihood launch (the paper picks no launch shapes;
 * this is the library's own): times pds_loglik_grad on `particles` (device,
 * [P][N], the caller's; read only) for the candidates K = 1 with one and
 * two units per thread (PDS_OPT_UNITS_PER_THREAD) and K = 5, 10, 25, 50
 * with one, three calls each after a warm-up call, in the problem's math
 * mode, and keeps the fastest: the problem's K and units per thread are set
 * to it.  choice (host, 3 ints, may be NULL) receives units per thread, K
 * and the chosen configuration's time per call in microseconds.  Blocks the
 * calling thread until the timings are done.  Every candidate gives the
 * same log p and gradient up to the rounding that K changes (K = 1 with one
 * or two units per thread: the same bits).  Planar chains only
 * (PDS_ERR_UNSUPPORTED otherwise); the options are left unchanged on error. */
int pds_problem_autotune(pds_problem_t p, const float* particles, int N, int* choice);

/* Constrained SVGD (Sec. IV-E, Eq. mdmm-loss, Algorithm 1).  With enable = 1
 * the likelihood is the observation term only, and the defect terms and the
 * parameter limits become equality constraints.  Each particle carries
 * MDMM multipliers, which the modified differential multiplier method
 * updates:
 *   g_def,w = ||s^s_w - s_end(w-1)||^2 / sigma_def^2        (w = 1..W-1)
 *   g_lim,k = clamp(u_k, 0, 1) - u_k,  u = (theta - lo) / (hi - lo)
 *   Psi     = sum_w (lam_def,w g_def,w + c/2 g_def,w^2)
 *           + sum_k (lam_lim,k g_lim,k + c/2 g_lim,k^2)
 * The particle layout becomes P = M + (W-1)*S + (W-1) + M: theta, the
 * shooting states, lam_def, lam_lim.  pds_loglik_grad then returns
 * log p_obs and needs a grad buffer of P + M rows:
 *   rows [0, M)        d log p_obs / d theta   (phi's input);
 *   shooting rows      d (log p_obs - Psi) / d s^s;
 *   lam_def rows       g_def;  lam_lim rows g_lim;
 *   rows [P, P + M)    -dPsi/dtheta, with the multipliers held fixed.
 * c >= 0 is the MDMM damping.  enable = 0 restores the multiple-shooting
 * likelihood and layout.  Returns PDS_ERR_UNSUPPORTED for the arm-and-box
 * system.  The iteration buffers are released (pds_iterate reallocates
 * them). */
int pds_problem_set_csvgd(pds_problem_t p, int enable, double c);

/* A set of R trajectories (Sec. IV-C, Eqs. traj_likelihood_sum / _prod):
 * replaces the problem's observations and start state.  Every trajectory
 * has its own shooting states; the particle layout becomes
 * P = M + R (W-1) S (theta, then trajectory 0's shooting states, ...).
 *  obs     : host [R][T][D] float, copied to the device.
 *  s0      : host [R][S] float.
 *  combine : PDS_COMBINE_SUM, the equally weighted Gaussian mixture
 *            log p = logsumexp_r(log p_ms,r) - log R (plus log p_lim once);
 *            PDS_COMBINE_PRODUCT, log p = sum_r log p_ms,r (plus log p_lim
 *            once).
 * The gradient of the sum weights trajectory r by its responsibility
 * softmax_r(log p_ms,r).  1 <= R <= PDS_MAX_TRAJECTORIES.
 * PDS_ERR_UNSUPPORTED for the arm-and-box system, for constrained SVGD,
 * and in batches. */
#define PDS_COMBINE_SUM 0
#define PDS_COMBINE_PRODUCT 1
int pds_problem_set_trajectories(pds_problem_t p, int R, const float* obs, const float* s0, int combine);

/* Allocate the workspace for up to N_max particles now, so that later calls
 * with N <= N_max allocate nothing (e.g. before capturing a CUDA graph).
 * Calls with a larger N grow the workspace (synchronising the stream). */
int pds_problem_reserve(pds_problem_t p, int N_max);

/* log p(theta_bar) and its gradient for N particles (Sec. IV-C, Eq. 5 in log
 * space, plus log p_lim of Sec. IV-D):
 *   log p = sum_t log N(x_t | f_obs(s_t), sigma_obs^2 I)
 *         + sum_{w=1}^{W-1} log N(s^s_w | s_end(w-1), sigma_def^2 I)
 *         - sum_k log(hi_k - lo_k) - (c_lim/2) ||clamp(u,0,1) - u||^2
 *  particles: device [P][N] float (read only).
 *  logp     : device [N] float (written).
 *  grad     : device [P][N] float, d log p / d particles (ascent direction),
 *             or NULL to evaluate log p only.
 *  status   : device [N] int32 or NULL; 0 = finite, 1 = log p or a gradient
 *             entry was not finite (the particle's values are then
 *             meaningless).
 * 1 <= N <= 1<<20. */
int pds_loglik_grad(pds_problem_t p, const float* particles, int N, float* logp,
                    float* grad, int32_t* status);

/* f_sim (Sec. III): roll out T steps from s0 for N parameter vectors.
 *  theta : device [M][N]; states: device [T+1][2n][N] (row 0 = s0). */
int pds_simulate(pds_problem_t p, const float* theta, int N, float* states);

/* SVGD state for N particles of P rows whose first M rows are theta
 * (Eq. 1 / Algorithm 1).  The kernel is the RBF kernel
 * k(a, b) = exp(-||u_a - u_b||^2 / bw) on unit-box coordinates
 * u = (theta - lo) / (hi - lo); bw is the lower median of the N(N-1)/2
 * pairwise squared distances divided by log N (1 if N < 2 or the median is
 * 0), the median heuristic of Sec. IV-A.  theta moves by Adam ascent
 * (lr, beta1, beta2, eps) on phi in u coordinates, then (if clamp) is clipped
 * to the box; rows M..P-1 (shooting states) move by Adam ascent on their own
 * gradient.  theta_lo/hi: host [M].  1 <= N <= 65536, 1 <= M <= 16. */
int pds_svgd_create(int N, int M, int P, const float* theta_lo, const float* theta_hi,
                    double lr, double beta1, double beta2, double eps, int clamp,
                    void* cuda_stream, pds_svgd_t* out);
int pds_svgd_destroy(pds_svgd_t s);

/* SVGD options: PDS_OPT_FAST_MATH 0 (default) = expf for the kernel values,
 * 1 = the hardware approximation __expf.  PDS_OPT_MEDIAN_FULL_PASSES 0
 * (default) = for N >= 2048 bracket the median from a sample of pairs and
 * select among the pairs inside the bracket (falling back to the full passes
 * if the bracket misses), and for N <= 256 select it in one block with every
 * pair distance in shared memory; 1 = always three radix passes over all
 * pairs, recomputing the distances in each.  All give the same exact median.  PDS_OPT_PHI_CUDA_CORES 0 (default) = for
 * N >= 256 the kernel-matrix products of phi run on the tensor cores
 * (tcgen05: the exponent product in tf32 with split operands, the product of
 * the kernel values with the gradients and coordinates in fp16 with split
 * operands; fp32 accumulation); 1 = CUDA cores. */
#define PDS_OPT_MEDIAN_FULL_PASSES 3
#define PDS_OPT_PHI_CUDA_CORES 4
/* PDS_OPT_MEDIAN_CUDA_CORES 0 (default) = for N >= 2048 the pair distances of
 * the median passes come from tensor-core products (split tf32, fp32
 * accumulation, clamped at 0); 1 = CUDA cores. */
#define PDS_OPT_MEDIAN_CUDA_CORES 5
/* PDS_OPT_WAIT_LIMIT (value >= 0, default 2^24): how many times a warp of a
 * tensor-core pass polls an mbarrier for the copy or product it needs before
 * it gives up; 0 tests the barrier once and never waits.  A pass that gives
 * up lets the copies and products it has in flight finish (with the default
 * limit), frees its tensor memory and returns; the step then completes with
 * results that are not valid, and PDS_ERR_TIMEOUT is reported as below.  The
 * default is far above any wait a healthy pass makes (a few microseconds);
 * small values exist to exercise that path. */
#define PDS_OPT_WAIT_LIMIT 6
/* PDS_OPT_GRAPH 1 (default): a step's kernels (about 25) are captured into a
 * CUDA graph on the second pds_svgd_step call with the same particles, grad,
 * bandwidth_out and phi_out pointers and the same options, and every later
 * call with them replays the graph, which saves the gaps between the
 * launches.  Calls with other pointers or options launch directly and
 * re-capture on their second use.  On the legacy or per-thread default
 * stream, which cannot be captured, the graph runs on a stream of the
 * state's own, ordered after the caller's stream and the caller's stream
 * after it by two events.  If the caller is capturing the state's stream
 * already, the kernels go into the caller's graph instead.  The first call
 * with new pointers also does the kernels' one-time set-up.  0: launch
 * every kernel every time. */
#define PDS_OPT_GRAPH 7
int pds_svgd_set_option(pds_svgd_t s, int option, int value);

/* Constrained SVGD update (Algorithm 1) for particles laid out as
 * pds_problem_set_csvgd describes; n_def = W - 1 defect multipliers, and the
 * last M rows are the limit multipliers.  Each step then
 *  - moves theta by Adam ascent in u on phi (Eq. 1, from grad rows [0, M))
 *    plus the constraint direction (grad rows [P, P + M) times hi - lo),
 *    without clipping to the box;
 *  - moves the shooting states by Adam ascent on their rows;
 *  - moves every multiplier by lam += lr * g (its grad row).
 * grad must then have P + M rows.  enable = 0 restores the plain update.
 * PDS_ERR_ARG if n_def does not fit the layout. */
int pds_svgd_set_csvgd(pds_svgd_t s, int enable, int n_def);

/* One SVGD + Adam update in place.
 *  particles    : device [P][N] float (read and written).
 *  grad         : device [P][N] float, d log p / d particles.
 *  bandwidth_out: device float scalar or NULL (the bandwidth bw used).
 *  phi_out      : device [M][N] float or NULL (phi in u coordinates).
 * Two conditions are found by the device while a step runs, after the call
 * that queued it has returned: a tensor-core pass that gave up waiting
 * (PDS_ERR_TIMEOUT; that step's particles are not valid) and a step in which
 * no particle had finite coordinates and gradient (PDS_ERR_NONFINITE; every
 * particle then sits out and keeps NaN).  The kernel writes them to a word of
 * mapped host memory; the next pds_svgd_step or pds_iterate on the state
 * returns the code (TIMEOUT first) instead of queuing work, and clears it.
 * pds_svgd_status synchronises the state's stream and returns it at once;
 * pds_iterate_host returns it after its final synchronisation. */
int pds_svgd_step(pds_svgd_t s, float* particles, const float* grad,
                  float* bandwidth_out, float* phi_out);

/* Synchronise the state's stream, then return and clear the status the
 * device reported for the steps run so far: PDS_OK, PDS_ERR_TIMEOUT or
 * PDS_ERR_NONFINITE (see pds_svgd_step). */
int pds_svgd_status(pds_svgd_t s);

/* Reset Adam moments and the step count to zero. */
int pds_svgd_reset(pds_svgd_t s);

/* Algorithm 1 loop on the device: `iters` times { log p and gradient of all
 * particles; SVGD + Adam update }.  particles: device [P][N] in/out;
 * logp: device [N] or NULL, receives log p evaluated in the last iteration
 * (before its update).  N must equal the SVGD state's N.  For a planar chain
 * whose problem and SVGD state share one stream that can be captured (not a
 * default stream), and whose step takes the sampled median bracket, each
 * iteration runs as one CUDA graph (captured on the second call with the
 * same buffers and settings): the step's median bandwidth, which reads only
 * the coordinates, on a high-priority side stream beside the likelihood,
 * then the rest of the step.  The results are those of pds_loglik_grad
 * followed by pds_svgd_step, bit for bit. */
int pds_iterate(pds_problem_t p, pds_svgd_t s, float* particles, int iters, float* logp);

/* Same as pds_iterate for host-resident data: copies particles (host [P][N])
 * to the device, runs `iters` iterations, copies the updated particles and
 * the last log p (host [N] or NULL) back, and synchronises the stream.
 * For a single planar-chain trajectory the copy in is made in groups of
 * windows (theta and the shooting states that the group's windows read),
 * and each group's rollout starts, on a stream of the problem's own, as
 * soon as its rows have landed, so that the copy overlaps the first
 * rollout.  The results are those of pds_iterate bit for bit.  Pinned
 * host memory gives the fastest copies and the overlap. */
int pds_iterate_host(pds_problem_t p, pds_svgd_t s, float* particles_host, int iters,
                     float* logp_host);

/* ---- Batched execution of many problems (uneven chain length, trajectory
 * length, window count and particle count).  Every iteration runs one
 * persistent rollout launch per chain length over all problems' (particle,
 * window) units -- work items ordered longest window first and taken through
 * an atomic counter -- each on a CUDA-graph branch of its own, and each
 * problem's window reduction and SVGD update on a branch of its own (up to
 * 64) that waits only for its chain length's rollout.  The iteration is
 * captured once into a CUDA graph (on the first pds_batch_iterate after
 * creation or autotuning)
 * and replayed (the first iteration after creation or autotuning runs with
 * plain launches).  Results equal those of running each problem alone with the
 * same settings, up to rounding.  No counterpart in the paper, which runs one
 * problem at a time; this is Algorithm 1 applied to many problems at once. */
typedef struct pds_batch* pds_batch_t;

/* problems/svgds/particles: arrays of n_jobs handles and device particle
 * buffers ([P_j][N_j], owned by the caller, updated in place every
 * iteration).  logp: NULL or n_jobs device pointers ([N_j] each), written
 * with log p of the particles before each update.  The batch takes over the
 * problems' checkpoint-stride and fast-math settings (per chain length) and
 * queues its work on cuda_stream; do not use the problems or SVGD states
 * elsewhere while the batch exists. */
int pds_batch_create(int n_jobs, pds_problem_t const* problems, pds_svgd_t const* svgds,
                     float* const* particles, float* const* logp, void* cuda_stream,
                     pds_batch_t* out);
int pds_batch_destroy(pds_batch_t b);

/* Autotuner: for every chain length present, time the batched rollout for
 * checkpoint strides K in {1, 5, 10, 25, 50}, exact or (allow_fast_math) fast
 * math, one or (K = 1, where every problem of that chain length observes
 * every state component and has an even particle count) two particles per
 * thread as PDS_OPT_UNITS_PER_THREAD describes, and the two largest
 * persistent grid sizes, and keep the fastest.  choices: NULL or
 * [5 * number of chain lengths] ints receiving (links, K, fast_math, grid
 * blocks, units per thread) per chain length.  Synchronises.  Before any
 * autotuning a chain length runs with the first problem's K, fast math and
 * units per thread. */
int pds_batch_autotune(pds_batch_t b, int allow_fast_math, int* choices);

/* Run `iters` iterations of every problem (graph replays; asynchronous). */
int pds_batch_iterate(pds_batch_t b, int iters);

/* Number of chain-length groups and kernel launches per iteration (inside
 * the graph). */
int pds_batch_info(pds_batch_t b, int* n_groups, int* launches_per_iter);

/* ---- Serving with continuous batching.  Jobs (one problem, its initial
 * particles, an iteration count) enter a FIFO queue.  Each pds_server_tick
 * admits queued jobs while their estimated device memory (problem workspace,
 * adjoint tape, SVGD state, particles) fits the budget and the active-job
 * limit, runs one SVGD iteration of every active job in one batched launch
 * (pds_batch over the active set, rebuilt when it changes), copies the
 * particles and last log p of jobs that reached their iteration count to the
 * host and releases their device memory.  Every job's state stays on the
 * device between ticks.  Jobs use SVGD with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) and clamping to the box, as pds_svgd_create.  The server queues
 * its work on cuda_stream and synchronises it at the end of every tick.  No
 * counterpart in the paper (Algorithm 1 for a stream of requests). */
#define PDS_JOB_QUEUED 0
#define PDS_JOB_ACTIVE 1
#define PDS_JOB_DONE 2
typedef struct pds_server* pds_server_t;
int pds_server_create(size_t mem_budget_bytes, int max_active, void* cuda_stream, pds_server_t* out);
int pds_server_destroy(pds_server_t s);
/* Checkpoint stride and math variant of the rollouts of jobs admitted from
 * now on (defaults 1 and fast math). */
int pds_server_set_rollout_options(pds_server_t s, int checkpoint_stride, int fast_math);
/* Arguments as pds_problem_create plus N particles (host [P][N], copied),
 * the Adam learning rate and the number of SVGD iterations.  Fails with
 * PDS_ERR_BUDGET if the job alone exceeds the memory budget. */
int pds_server_submit(pds_server_t s, const pds_system_desc* sys, double dt, int T, int windows,
                      const float* obs, int D, const int* obs_index, double sigma_obs,
                      double sigma_def, const float* s0, const float* theta_lo,
                      const float* theta_hi, double c_lim, int N, const float* particles,
                      double lr, int iterations, long long* job_id);
/* Same for a rigid double pendulum job (arguments as pds_problem_create_rigid2). */
int pds_server_submit_rigid2(pds_server_t s, const pds_rigid2_desc* sys, double dt, int T, int windows,
                             const float* obs, int D, const int* obs_index, double sigma_obs,
                             double sigma_def, const float* s0, const float* theta_lo,
                             const float* theta_hi, double c_lim, int N, const float* particles,
                             double lr, int iterations, long long* job_id);
/* Same for an arm-and-box job (arguments as pds_problem_create_armbox). */
int pds_server_submit_armbox(pds_server_t s, const pds_armbox_desc* sys, double dt, int T,
                             int windows, const float* obs, int D, const int* obs_index,
                             double sigma_obs, double sigma_def, const float* s0,
                             const float* theta_lo, const float* theta_hi, double c_lim, int N,
                             const float* particles, double lr, int iterations, long long* job_id);
/* One scheduling step (admit, iterate, retire); synchronises the stream. */
int pds_server_tick(pds_server_t s, int* n_active, int* n_retired);
/* PDS_JOB_* state and iterations done so far. */
int pds_server_status(pds_server_t s, long long job_id, int* state, int* iterations_done);
/* Copy a finished job's particles (host [P][N]) and last log p (host [N] or
 * NULL) and forget the job. */
int pds_server_result(pds_server_t s, long long job_id, float* particles, float* logp);
/* Remove a queued or active job (its device memory is released). */
int pds_server_cancel(pds_server_t s, long long job_id);
int pds_server_stats(pds_server_t s, int* queued, int* active, size_t* bytes_in_use);

/* Convergence gate of the server: the posterior metrics of Sec. IV used to
 * decide when a job has reached its posterior.  With metric != PDS_GATE_NONE,
 * every `every` iterations of a job the server snapshots its theta particles
 * in unit-box coordinates u = (theta - lo) / (hi - lo) and, from the second
 * snapshot on, evaluates between the new snapshot (n live particles) and the
 * previous one (m live particles):
 *   PDS_GATE_MMD2:   the unbiased MMD^2 with kernel exp(-||u - u'||^2 / (h M))
 *                    (as pds_mmd2 with bandwidth h M: h per coordinate);
 *   PDS_GATE_KNN_KL: the KNN estimate of KL(new || previous) with k = 3 (as
 *                    pds_knn_kl); terms of coincident points are left out.
 * Particles that sit out (last log p or a theta coordinate not finite) take
 * no part.  When the
 * value is <= threshold the job retires at once (its iterations_done is then
 * below its cap); otherwise it runs on to its iteration count.  Set the gate
 * before submitting jobs (PDS_ERR_ARG otherwise); h is used by MMD^2 only
 * (> 0).  pds_server_job_gate reports the number of metric evaluations and
 * the last value (NaN before the first) of a job that is queued, active or
 * done and not yet collected. */
#define PDS_GATE_NONE 0
#define PDS_GATE_MMD2 1
#define PDS_GATE_KNN_KL 2
int pds_server_set_gate(pds_server_t s, int metric, int every, double threshold, double h);
int pds_server_job_gate(pds_server_t s, long long job_id, int* checks, double* last_value);

/* Median-heuristic bandwidth of N particles without allocating any device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc -- for example code running inside another
 * framework's allocator or memory-pool callback, or a process whose device
 * memory is fully reserved up front -- and so cannot create the workspace
 * that pds_svgd_create allocates.  It computes the same bandwidth as
 * pds_svgd_step with a zero gradient (lower median of the pairwise squared
 * distances of the unit-box coordinates over the live particles, divided by
 * log of their number; 1 if fewer than 2 are live or the median is 0).  A
 * particle with a coordinate that is not finite sits out, as in
 * pds_svgd_step.
 *  theta        : device [M][N] float (e.g. the first M rows of a particle array).
 *  theta_lo/hi  : host [M] box.
 *  bandwidth_out: device float scalar (written).
 *  cuda_stream  : cudaStream_t the work is queued on (NULL = legacy default).
 * Its scratch is one file-scope device array of 16 KiB + 4 MiB that every GPU
 * loading the library holds until the process exits; 1 <= N <= 65536 (pair
 * counts are 32-bit, as in pds_svgd_create), N * M <= 1048576 and
 * 1 <= M <= 16 (PDS_ERR_ARG otherwise, with a message).  The first call on
 * each device looks up that array's device address (with that device
 * current); make that first call before any stream capture.  With lazy
 * module loading (CUDA's default) that first call, or the first launch of
 * any SVGD kernel of the library on the device, also loads the library's
 * device code and reserves the array, which allocates device memory: make
 * the first call at start-up, outside the context that cannot allocate.
 * Every call shares the one array and clears what must start at zero, so
 * calls whose work overlaps on the GPU (different streams, or several host
 * threads) race and must be serialised by the caller.  After that first call
 * the entry point allocates nothing and returns after queuing its kernels. */
int pds_bandwidth_noalloc(const float* theta, int N, int M, const float* theta_lo,
                          const float* theta_hi, float* bandwidth_out, void* cuda_stream);

/* ---- Sobol initialisation (App. A-A: particles start from the
 * deterministic Sobol sequence over the parameter limits).
 * Writes theta device [M][N] float (e.g. the first M rows of a particle
 * array): theta[k][i] = lo_k + x_k(skip + i) (hi_k - lo_k), x(n) the n-th
 * point of the unscrambled Sobol sequence in Gray-code order (point 0 is the
 * origin), with the direction numbers of Joe and Kuo (2008) for dimensions
 * 1..16.  x has at most 24 significant bits for indices below 2^24, so it is
 * exact in fp32.  1 <= N <= 2^24, 1 <= M <= 16, 0 <= skip and
 * skip + N <= 2^32; theta_lo/hi host [M] with hi > lo.  One kernel launch
 * queued on cuda_stream. */
int pds_sobol_box(float* theta, int N, int M, const float* theta_lo, const float* theta_hi, long long skip,
                  void* cuda_stream);

/* ---- Stochastic gradient Langevin dynamics (Welling and Teh 2011), the
 * other estimator run with the multiple-shooting likelihood in Sec. V-B.
 * Each particle is an independent chain; one step moves, in place,
 *   theta rows r < M:  u = (theta - lo) / (hi - lo),
 *                      u += (eps_t / 2) (hi - lo) g + sqrt(eps_t) xi,
 *                      clipped to [0, 1] if clamp, theta = lo + u (hi - lo);
 *   rows r >= M:       x += (eps_t / 2) g + sqrt(eps_t) xi;
 * with g = d log p / d particles, eps_t = a (b + t)^(-gamma) for the step
 * count t = 1, 2, ... (incremented by every step, zeroed by reset), and
 * xi ~ N(0, 1) from a counter-based generator: SplitMix64 from `seed`,
 * outputs 2k + 1 and 2k + 2 with k = (t - 1) P N + r N + i, combined by the
 * Box-Muller transform with u1 = (z1 >> 11 + 1) 2^-53, u2 = (z2 >> 11) 2^-53
 * (computed in fp32).  The draws depend on (seed, t, r, i) only.
 *  pds_sgld_create: 1 <= N <= 65536, 0 <= M <= 16, M <= P <= 65535,
 *    theta_lo/hi host [M] (may be NULL when M = 0), a > 0, gamma >= 0,
 *    b > -1; allocates nothing on the device.
 *  pds_sgld_step: particles device [P][N] float (read and written), grad
 *    device [P][N] float; eps_out host float or NULL (receives eps_t).
 *    One kernel launch queued on the state's stream. */
int pds_sgld_create(int N, int M, int P, const float* theta_lo, const float* theta_hi, double a, double b,
                    double gamma, unsigned long long seed, int clamp, void* cuda_stream, pds_sgld_t* out);
int pds_sgld_destroy(pds_sgld_t s);
int pds_sgld_reset(pds_sgld_t s);
int pds_sgld_step(pds_sgld_t s, float* particles, const float* grad, float* eps_out);

/* ---- Posterior metrics (Sec. IV: Eq. knn-kl and the maximum mean
 * discrepancy).  Sample sets are device arrays [d][n] float (coordinate-
 * major, like particles), 1 <= d <= 64.  Both synchronise the stream and
 * return the value on the host.
 *
 * pds_knn_kl: the k-nearest-neighbour estimate of KL(P || Q) with
 * k_i = l_i = k (1 <= k <= 8; the paper uses 3):
 *   (d / n) sum_i log( nu_k(i) / rho_k(i) ) + log( m / (n - 1) ),
 * nu_k(i) the Euclidean distance from p_i to its k-th nearest neighbour in
 * Q, rho_k(i) the same in P without p_i.  p [d][n], q [d][m], n >= k + 1,
 * m >= k.  Coincident points make a ratio 0 or infinite.
 *
 * pds_mmd2: the unbiased estimate of the squared maximum mean discrepancy
 * with the kernel exp(-||x - y||^2 / h), h > 0:
 *   1/(n(n-1)) sum_{i!=j} k(x_i,x_j) + 1/(m(m-1)) sum_{i!=j} k(y_i,y_j)
 *   - 2/(nm) sum_{i,j} k(x_i,y_j).   x [d][n], y [d][m], n, m >= 2. */
int pds_knn_kl(const float* p, int n, const float* q, int m, int d, int k, double* kl, void* cuda_stream);
int pds_mmd2(const float* x, int n, const float* y, int m, int d, double h, double* mmd2, void* cuda_stream);

/* Number of kernel launches the last pds_loglik_grad / pds_svgd_step /
 * pds_iterate call made (for launch accounting). */
int pds_last_launch_count(void);

/* Human-readable name of a status code; message of the last error on the
 * calling thread. */
const char* pds_strerror(int code);
const char* pds_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PDS_H_ */
