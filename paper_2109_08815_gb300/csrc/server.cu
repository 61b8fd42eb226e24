// Serving loop with continuous batching.
//
// Jobs (a problem, its initial particles and an iteration count) are
// submitted to a FIFO queue.  Every tick admits queued jobs while their
// estimated device memory fits the budget (and the active-job limit), runs
// one SVGD iteration of every active job in one batched launch (pds_batch,
// rebuilt when the active set changes), and retires the jobs that reached
// their iteration count: their particles and last log p are copied to the
// host and their device memory is released, so waiting jobs can enter on the
// next tick.  Every job's state stays resident on the device between ticks.
//
// Convergence gate (optional, pds_server_set_gate): every `every` iterations
// the server takes a snapshot of each active job's theta particles in
// unit-box coordinates and evaluates a posterior metric (Sec. IV: the
// unbiased RBF MMD^2, or the KNN-KL estimate with k = 3) between this
// snapshot and the previous one, over the live particles (finite theta and
// last log p; the MMD kernel's bandwidth is h per coordinate, h M in all).  A job
// whose metric is at or below the threshold has reached its posterior and
// retires before its iteration cap.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <deque>
#include <map>
#include <vector>

#include "pds_internal.cuh"

using namespace pds;

namespace {

struct Job {
  long long id = 0;
  int state = 0;  // PDS_JOB_*
  int kind = PDS_SYSTEM_PLANAR_CHAIN;
  // creation arguments (host copies)
  pds_system_desc sys{};
  pds_armbox_desc arm{};
  pds_rigid2_desc r2{};
  std::vector<int> theta_param;
  std::vector<double> arm_len, amp, freq, phase;
  std::vector<double> mass, length, damping;
  std::vector<int> theta_kind, theta_link, obs_index;
  std::vector<float> obs, s0, lo, hi, x0;
  double dt = 0, sigma_obs = 0, sigma_def = 0, c_lim = 0, lr = 0;
  int T = 0, W = 0, D = 0, N = 0, P = 0, iterations = 0, done_iters = 0;
  size_t bytes = 0;
  // device state while active
  pds_problem_t prob = nullptr;
  pds_svgd_t svgd = nullptr;
  float* d_x = nullptr;
  float* d_logp = nullptr;
  // convergence gate: unit-box snapshots [M][N] (now, previous), KNN
  // scratch [2N], sums and live counts
  float* d_u[2] = {nullptr, nullptr};
  float* d_gscr = nullptr;
  double* d_acc = nullptr;  // [0..2] metric sums, [3..4] live counts
  double h_acc[5] = {0, 0, 0, 0, 0};
  int u_cur = 0, snapshots = 0, gate_checks = 0;
  bool gate_pending = false;
  double gate_value = NAN;
  // results
  std::vector<float> x_out, logp_out;
};

struct GateUnit {
  float lo[PDS_MAX_THETA], inv_w[PDS_MAX_THETA];
};

// u[k][i] = (theta[k][i] - lo_k) / (hi_k - lo_k); a particle that sits out
// (its last log p or a theta coordinate not finite) gets NaN in every row and
// is not counted.
__global__ void __launch_bounds__(256) gate_unit_kernel(const float* __restrict__ x, const float* __restrict__ logp,
                                                        int N, int M, GateUnit g, float* __restrict__ u,
                                                        double* __restrict__ live) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = false;
  if (i < N) {
    ok = isfinite(logp[i]);
    for (int k = 0; k < M; ++k) ok &= isfinite(x[(size_t)k * N + i]);
    for (int k = 0; k < M; ++k) u[(size_t)k * N + i] = ok ? (x[(size_t)k * N + i] - g.lo[k]) * g.inv_w[k] : NAN;
  }
  const unsigned b = __ballot_sync(0xffffffffu, ok);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(live, (double)__popc(b));
}

}  // namespace

struct pds_server {
  size_t budget = 0, in_use = 0;
  int max_active = 0;
  int K = 1, fast = 1;
  cudaStream_t stream = nullptr;
  long long next_id = 1;
  std::deque<long long> queue;
  std::vector<long long> active;
  std::map<long long, Job> jobs;
  pds_batch_t batch = nullptr;
  bool batch_dirty = true;
  int gate_metric = PDS_GATE_NONE, gate_every = 0;
  double gate_threshold = 0.0, gate_h = 0.1;
};

// Device bytes a job holds while active (problem workspace and buffers,
// SVGD state, particles).
static size_t job_bytes(int n, int M, int T, int W, int D, int N, int K) {
  const size_t S = 2 * (size_t)n, P = (size_t)M + (size_t)(W - 1) * S, U = (size_t)N * W;
  int hmax = 0;
  for (int w = 0; w < W; ++w) {
    const int h = (int)(((long long)(w + 1) * T) / W - ((long long)w * T) / W);
    if (h > hmax) hmax = h;
  }
  const size_t segs = (size_t)((hmax + K - 1) / K);
  size_t b = 0;
  b += (size_t)T * (D + S) * 4;                             // observations, and their state-ordered copy
  b += (size_t)W * (1 + M + 2 * S) * N * 4;                 // per-window partials
  b += (segs + (size_t)K) * S * U * 4;                      // adjoint tape
  b += (2 * P * N + N) * 4;                                 // iteration buffers (grad, x, logp)
  b += (size_t)svgd_phi_partials(N) * M * N * 4 + 2 * (size_t)M * N * 4 + 2 * P * N * 4;  // SVGD state
  b += svgd_cand_capacity(N) * 4 + (svgd_cand_capacity(N) ? (size_t)svgd_sample_size() * 4 : 0);
  if (N >= 256) b += phi_tc_floats(N, M) * 4;
  if (N >= 2048) b += median_tc_floats(N, M) * 4 + (size_t)median_tc_work_items(N, nullptr) * 2 * sizeof(int);
  b += P * N * 4 + (size_t)N * 4;                           // particles, log p
  b += (2 * (size_t)M * N + 2 * (size_t)N) * 4 + 5 * 8;     // convergence-gate snapshots and scratch
  return b + (64u << 10);
}

static void release(Job& j) {
  if (j.prob) pds_problem_destroy(j.prob);
  if (j.svgd) pds_svgd_destroy(j.svgd);
  cudaFree(j.d_x);
  cudaFree(j.d_logp);
  cudaFree(j.d_u[0]);
  cudaFree(j.d_u[1]);
  cudaFree(j.d_gscr);
  cudaFree(j.d_acc);
  j.prob = nullptr;
  j.svgd = nullptr;
  j.d_x = nullptr;
  j.d_logp = nullptr;
  j.d_u[0] = j.d_u[1] = nullptr;
  j.d_gscr = nullptr;
  j.d_acc = nullptr;
}

static int job_theta_count(const Job& j) {
  return j.kind == PDS_SYSTEM_ARM_BOX ? 4 : j.kind == PDS_SYSTEM_RIGID_DOUBLE_PENDULUM ? j.r2.n_theta : j.sys.n_theta;
}

// Queue the gate's snapshot and, from the second snapshot on, its metric.
static cudaError_t gate_enqueue(pds_server* s, Job& j) {
  const int M = job_theta_count(j), N = j.N;
  GateUnit g;
  for (int k = 0; k < M; ++k) {
    g.lo[k] = j.lo[k];
    g.inv_w[k] = 1.0f / (j.hi[k] - j.lo[k]);
  }
  float* now = j.d_u[j.u_cur];
  float* prev = j.d_u[j.u_cur ^ 1];
  double* live_now = j.d_acc + 3 + j.u_cur;
  cudaError_t e = cudaMemsetAsync(live_now, 0, sizeof(double), s->stream);
  if (e != cudaSuccess) return e;
  gate_unit_kernel<<<(N + 255) / 256, 256, 0, s->stream>>>(j.d_x, j.d_logp, N, M, g, now, live_now);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (j.snapshots > 0) {
    if (s->gate_metric == PDS_GATE_MMD2)
      e = mmd2_sums_async(now, N, prev, N, M, (float)(1.0 / (s->gate_h * M)), j.d_acc, s->stream);
    else
      e = knn_log_ratio_async(now, N, prev, N, M, 3, j.d_gscr, j.d_acc, s->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(j.h_acc, j.d_acc, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return e;
    j.gate_pending = true;
  }
  ++j.snapshots;
  j.u_cur ^= 1;
  return cudaSuccess;
}

// Metric of the last queued check, after the stream has synchronised.
static double gate_value(const pds_server* s, const Job& j) {
  const double n_now = j.h_acc[3 + (j.u_cur ^ 1)], n_prev = j.h_acc[3 + j.u_cur];
  if (s->gate_metric == PDS_GATE_MMD2) {
    if (n_now < 2 || n_prev < 2) return NAN;
    return j.h_acc[0] / (n_now * (n_now - 1)) + j.h_acc[1] / (n_prev * (n_prev - 1)) -
           2.0 * j.h_acc[2] / (n_now * n_prev);
  }
  if (n_now < 4 || n_prev < 3) return NAN;
  return (double)job_theta_count(j) / n_now * j.h_acc[0] + log(n_prev / (n_now - 1));
}

static int activate(pds_server* s, Job& j) {
  int rc;
  int M = 4;
  if (j.kind == PDS_SYSTEM_RIGID_DOUBLE_PENDULUM) {
    pds_rigid2_desc r = j.r2;
    r.theta_param = j.theta_param.data();
    M = r.n_theta;
    rc = pds_problem_create_rigid2(&r, j.dt, j.T, j.W, j.obs.data(), j.D, j.obs_index.data(), j.sigma_obs,
                                   j.sigma_def, j.s0.data(), j.lo.data(), j.hi.data(), j.c_lim, s->stream, &j.prob);
  } else if (j.kind == PDS_SYSTEM_ARM_BOX) {
    pds_armbox_desc a = j.arm;
    a.arm_len = j.arm_len.data();
    a.amp = j.amp.data();
    a.freq = j.freq.data();
    a.phase = j.phase.data();
    rc = pds_problem_create_armbox(&a, j.dt, j.T, j.W, j.obs.data(), j.D, j.obs_index.data(), j.sigma_obs,
                                   j.sigma_def, j.s0.data(), j.lo.data(), j.hi.data(), j.c_lim, s->stream, &j.prob);
  } else {
    pds_system_desc sys = j.sys;
    sys.mass = j.mass.data();
    sys.length = j.length.data();
    sys.damping = j.damping.data();
    sys.theta_kind = j.theta_kind.data();
    sys.theta_link = j.theta_link.data();
    M = sys.n_theta;
    rc = pds_problem_create(&sys, j.dt, j.T, j.W, j.obs.data(), j.D, j.obs_index.data(), j.sigma_obs, j.sigma_def,
                            j.s0.data(), j.lo.data(), j.hi.data(), j.c_lim, s->stream, &j.prob);
  }
  if (rc != PDS_OK) return rc;
  pds_problem_set_option(j.prob, PDS_OPT_CHECKPOINT_STRIDE, s->K);
  pds_problem_set_option(j.prob, PDS_OPT_FAST_MATH, s->fast);
  rc = pds_svgd_create(j.N, M, j.P, j.lo.data(), j.hi.data(), j.lr, 0.9, 0.999, 1e-8, 1, s->stream, &j.svgd);
  if (rc != PDS_OK) { release(j); return rc; }
  cudaError_t e;
  if ((e = cudaMalloc(&j.d_x, (size_t)j.P * j.N * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&j.d_logp, (size_t)j.N * sizeof(float))) != cudaSuccess) {
    release(j);
    return set_error(PDS_ERR_OOM, "server: particle allocation failed");
  }
  e = cudaMemcpyAsync(j.d_x, j.x0.data(), (size_t)j.P * j.N * sizeof(float), cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) { release(j); return set_error(PDS_ERR_CUDA, "server: particle upload failed"); }
  const int M_gate = job_theta_count(j);
  if ((e = cudaMalloc(&j.d_u[0], (size_t)M_gate * j.N * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&j.d_u[1], (size_t)M_gate * j.N * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&j.d_gscr, 2 * (size_t)j.N * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&j.d_acc, 5 * sizeof(double))) != cudaSuccess) {
    release(j);
    return set_error(PDS_ERR_OOM, "server: gate allocation failed");
  }
  rc = pds_problem_reserve(j.prob, j.N);
  if (rc != PDS_OK) { release(j); return rc; }
  j.x0.clear();
  j.x0.shrink_to_fit();
  return PDS_OK;
}

extern "C" {

int pds_server_create(size_t mem_budget_bytes, int max_active, void* cuda_stream, pds_server_t* out) {
  if (!out) return set_error(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (mem_budget_bytes == 0 || max_active < 1) return set_error(PDS_ERR_ARG, "bad server budget or limit");
  pds_server* s = new pds_server();
  s->budget = mem_budget_bytes;
  s->max_active = max_active;
  s->stream = (cudaStream_t)cuda_stream;
  *out = s;
  return PDS_OK;
}

int pds_server_set_rollout_options(pds_server_t s, int checkpoint_stride, int fast_math) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  if (checkpoint_stride < 1 || checkpoint_stride > PDS_MAX_WINDOW_STEPS || (fast_math != 0 && fast_math != 1))
    return set_error(PDS_ERR_ARG, "bad rollout options");
  s->K = checkpoint_stride;
  s->fast = fast_math;
  return PDS_OK;
}

int pds_server_destroy(pds_server_t s) {
  if (!s) return PDS_OK;
  cudaStreamSynchronize(s->stream);
  if (s->batch) pds_batch_destroy(s->batch);
  for (auto& kv : s->jobs) release(kv.second);
  delete s;
  return PDS_OK;
}

int pds_server_submit(pds_server_t s, const pds_system_desc* sys, double dt, int T, int windows, const float* obs,
                      int D, const int* obs_index, double sigma_obs, double sigma_def, const float* s0,
                      const float* theta_lo, const float* theta_hi, double c_lim, int N, const float* particles,
                      double lr, int iterations, long long* job_id) {
  if (!s || !sys || !obs || !obs_index || !s0 || !theta_lo || !theta_hi || !particles || !job_id)
    return set_error(PDS_ERR_ARG, "NULL argument");
  *job_id = 0;
  const int n = sys->n_links, M = sys->n_theta;
  if (n < 1 || n > PDS_MAX_LINKS || M < 1 || M > PDS_MAX_THETA || T < 1 || windows < 1 || windows > T || D < 1 ||
      D > 2 * n || N < 1 || N > 65536 || iterations < 1 || !(lr > 0.0))
    return set_error(PDS_ERR_ARG, "job outside the supported sizes");
  const size_t bytes = job_bytes(n, M, T, windows, D, N, s->K);
  if (bytes > s->budget) return set_error(PDS_ERR_BUDGET, "job needs more device memory than the server budget");
  Job j;
  j.id = s->next_id++;
  j.sys = *sys;
  j.mass.assign(sys->mass, sys->mass + n);
  j.length.assign(sys->length, sys->length + n);
  j.damping.assign(sys->damping, sys->damping + n);
  j.theta_kind.assign(sys->theta_kind, sys->theta_kind + M);
  j.theta_link.assign(sys->theta_link, sys->theta_link + M);
  j.obs_index.assign(obs_index, obs_index + D);
  j.obs.assign(obs, obs + (size_t)T * D);
  j.s0.assign(s0, s0 + 2 * n);
  j.lo.assign(theta_lo, theta_lo + M);
  j.hi.assign(theta_hi, theta_hi + M);
  j.dt = dt; j.T = T; j.W = windows; j.D = D; j.N = N; j.P = M + (windows - 1) * 2 * n;
  j.sigma_obs = sigma_obs; j.sigma_def = sigma_def; j.c_lim = c_lim; j.lr = lr; j.iterations = iterations;
  j.x0.assign(particles, particles + (size_t)j.P * N);
  j.bytes = bytes;
  j.state = PDS_JOB_QUEUED;
  *job_id = j.id;
  s->queue.push_back(j.id);
  s->jobs.emplace(j.id, std::move(j));
  return PDS_OK;
}

int pds_server_submit_rigid2(pds_server_t s, const pds_rigid2_desc* sys, double dt, int T, int windows,
                             const float* obs, int D, const int* obs_index, double sigma_obs, double sigma_def,
                             const float* s0, const float* theta_lo, const float* theta_hi, double c_lim, int N,
                             const float* particles, double lr, int iterations, long long* job_id) {
  if (!s || !sys || !sys->theta_param || !obs || !obs_index || !s0 || !theta_lo || !theta_hi || !particles ||
      !job_id)
    return set_error(PDS_ERR_ARG, "NULL argument");
  *job_id = 0;
  const int M = sys->n_theta;
  if (M < 1 || M > 11 || T < 1 || windows < 1 || windows > T || D < 1 || D > 4 || N < 1 || N > 65536 ||
      iterations < 1 || !(lr > 0.0))
    return set_error(PDS_ERR_ARG, "job outside the supported sizes");
  const size_t bytes = job_bytes(2, M, T, windows, D, N, s->K);
  if (bytes > s->budget) return set_error(PDS_ERR_BUDGET, "job needs more device memory than the server budget");
  Job j;
  j.id = s->next_id++;
  j.kind = PDS_SYSTEM_RIGID_DOUBLE_PENDULUM;
  j.r2 = *sys;
  j.theta_param.assign(sys->theta_param, sys->theta_param + M);
  j.obs_index.assign(obs_index, obs_index + D);
  j.obs.assign(obs, obs + (size_t)T * D);
  j.s0.assign(s0, s0 + 4);
  j.lo.assign(theta_lo, theta_lo + M);
  j.hi.assign(theta_hi, theta_hi + M);
  j.dt = dt; j.T = T; j.W = windows; j.D = D; j.N = N; j.P = M + (windows - 1) * 4;
  j.sigma_obs = sigma_obs; j.sigma_def = sigma_def; j.c_lim = c_lim; j.lr = lr; j.iterations = iterations;
  j.x0.assign(particles, particles + (size_t)j.P * N);
  j.bytes = bytes;
  j.state = PDS_JOB_QUEUED;
  *job_id = j.id;
  s->queue.push_back(j.id);
  s->jobs.emplace(j.id, std::move(j));
  return PDS_OK;
}

int pds_server_submit_armbox(pds_server_t s, const pds_armbox_desc* sys, double dt, int T, int windows,
                             const float* obs, int D, const int* obs_index, double sigma_obs, double sigma_def,
                             const float* s0, const float* theta_lo, const float* theta_hi, double c_lim, int N,
                             const float* particles, double lr, int iterations, long long* job_id) {
  if (!s || !sys || !sys->arm_len || !sys->amp || !sys->freq || !sys->phase || !obs || !obs_index || !s0 ||
      !theta_lo || !theta_hi || !particles || !job_id)
    return set_error(PDS_ERR_ARG, "NULL argument");
  *job_id = 0;
  const int na = sys->n_arm;
  if (na < 1 || na > PDS_MAX_LINKS || T < 1 || windows < 1 || windows > T || D < 1 || D > 4 || N < 1 ||
      N > 65536 || iterations < 1 || !(lr > 0.0))
    return set_error(PDS_ERR_ARG, "job outside the supported sizes");
  const size_t bytes = job_bytes(2, 4, T, windows, D, N, s->K) + (size_t)T * 9 * 4;
  if (bytes > s->budget) return set_error(PDS_ERR_BUDGET, "job needs more device memory than the server budget");
  Job j;
  j.id = s->next_id++;
  j.kind = PDS_SYSTEM_ARM_BOX;
  j.arm = *sys;
  j.arm_len.assign(sys->arm_len, sys->arm_len + na);
  j.amp.assign(sys->amp, sys->amp + 3 * na);
  j.freq.assign(sys->freq, sys->freq + 3 * na);
  j.phase.assign(sys->phase, sys->phase + 3 * na);
  j.obs_index.assign(obs_index, obs_index + D);
  j.obs.assign(obs, obs + (size_t)T * D);
  j.s0.assign(s0, s0 + 4);
  j.lo.assign(theta_lo, theta_lo + 4);
  j.hi.assign(theta_hi, theta_hi + 4);
  j.dt = dt; j.T = T; j.W = windows; j.D = D; j.N = N; j.P = 4 + (windows - 1) * 4;
  j.sigma_obs = sigma_obs; j.sigma_def = sigma_def; j.c_lim = c_lim; j.lr = lr; j.iterations = iterations;
  j.x0.assign(particles, particles + (size_t)j.P * N);
  j.bytes = bytes;
  j.state = PDS_JOB_QUEUED;
  *job_id = j.id;
  s->queue.push_back(j.id);
  s->jobs.emplace(j.id, std::move(j));
  return PDS_OK;
}

int pds_server_tick(pds_server_t s, int* n_active, int* n_retired) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  int retired = 0;
  // admission, first in first out
  while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
    Job& j = s->jobs[s->queue.front()];
    if (s->in_use + j.bytes > s->budget) break;
    int rc = activate(s, j);
    if (rc != PDS_OK) return rc;
    s->in_use += j.bytes;
    j.state = PDS_JOB_ACTIVE;
    s->active.push_back(j.id);
    s->queue.pop_front();
    s->batch_dirty = true;
  }
  if (!s->active.empty()) {
    if (s->batch_dirty) {
      if (s->batch) pds_batch_destroy(s->batch);
      s->batch = nullptr;
      std::vector<pds_problem_t> probs;
      std::vector<pds_svgd_t> svgds;
      std::vector<float*> xs, lps;
      for (long long id : s->active) {
        Job& j = s->jobs[id];
        probs.push_back(j.prob);
        svgds.push_back(j.svgd);
        xs.push_back(j.d_x);
        lps.push_back(j.d_logp);
      }
      int rc = pds_batch_create((int)probs.size(), probs.data(), svgds.data(), xs.data(), lps.data(), s->stream,
                                &s->batch);
      if (rc != PDS_OK) return rc;
      s->batch_dirty = false;
    }
    int rc = pds_batch_iterate(s->batch, 1);
    if (rc != PDS_OK) return rc;
    std::vector<long long> still;
    std::vector<long long> finishing;
    const bool gate = s->gate_metric != PDS_GATE_NONE;
    for (long long id : s->active) {
      Job& j = s->jobs[id];
      ++j.done_iters;
      if (gate && j.done_iters % s->gate_every == 0) {
        cudaError_t ge = gate_enqueue(s, j);
        if (ge != cudaSuccess) return set_error(PDS_ERR_CUDA, "server: gate launch failed");
      }
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, "server: tick failed");
    for (long long id : s->active) {
      Job& j = s->jobs[id];
      bool converged = false;
      if (j.gate_pending) {
        j.gate_pending = false;
        j.gate_value = gate_value(s, j);
        ++j.gate_checks;
        converged = j.gate_value <= s->gate_threshold;
      }
      if (converged || j.done_iters >= j.iterations) finishing.push_back(id);
      else still.push_back(id);
    }
    for (long long id : finishing) {
      Job& j = s->jobs[id];
      j.x_out.resize((size_t)j.P * j.N);
      j.logp_out.resize(j.N);
      cudaMemcpyAsync(j.x_out.data(), j.d_x, j.x_out.size() * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
      cudaMemcpyAsync(j.logp_out.data(), j.d_logp, j.logp_out.size() * sizeof(float), cudaMemcpyDeviceToHost,
                      s->stream);
    }
    if (!finishing.empty()) {
      e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, "server: result copy failed");
      for (long long id : finishing) {
        Job& j = s->jobs[id];
        release(j);
        s->in_use -= j.bytes;
        j.state = PDS_JOB_DONE;
        ++retired;
      }
      s->active = still;
      s->batch_dirty = true;
      if (s->batch) pds_batch_destroy(s->batch);
      s->batch = nullptr;
    }
  }
  if (n_active) *n_active = (int)s->active.size();
  if (n_retired) *n_retired = retired;
  return PDS_OK;
}

int pds_server_status(pds_server_t s, long long job_id, int* state, int* iterations_done) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return set_error(PDS_ERR_ARG, "unknown job");
  if (state) *state = it->second.state;
  if (iterations_done) *iterations_done = it->second.done_iters;
  return PDS_OK;
}

int pds_server_result(pds_server_t s, long long job_id, float* particles, float* logp) {
  if (!s || !particles) return set_error(PDS_ERR_ARG, "NULL argument");
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return set_error(PDS_ERR_ARG, "unknown job");
  Job& j = it->second;
  if (j.state != PDS_JOB_DONE) return set_error(PDS_ERR_ARG, "job not finished");
  memcpy(particles, j.x_out.data(), j.x_out.size() * sizeof(float));
  if (logp) memcpy(logp, j.logp_out.data(), j.logp_out.size() * sizeof(float));
  s->jobs.erase(it);
  return PDS_OK;
}

int pds_server_cancel(pds_server_t s, long long job_id) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return set_error(PDS_ERR_ARG, "unknown job");
  Job& j = it->second;
  if (j.state == PDS_JOB_QUEUED) {
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
      if (*q == job_id) { s->queue.erase(q); break; }
  } else if (j.state == PDS_JOB_ACTIVE) {
    cudaStreamSynchronize(s->stream);
    if (s->batch) pds_batch_destroy(s->batch);
    s->batch = nullptr;
    s->batch_dirty = true;
    std::vector<long long> still;
    for (long long id : s->active)
      if (id != job_id) still.push_back(id);
    s->active = still;
    release(j);
    s->in_use -= j.bytes;
  } else {
    return set_error(PDS_ERR_ARG, "job already finished");
  }
  s->jobs.erase(it);
  return PDS_OK;
}

int pds_server_set_gate(pds_server_t s, int metric, int every, double threshold, double h) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  if (metric != PDS_GATE_NONE && metric != PDS_GATE_MMD2 && metric != PDS_GATE_KNN_KL)
    return set_error(PDS_ERR_ARG, "unknown gate metric");
  if (metric != PDS_GATE_NONE && (every < 1 || !isfinite(threshold) || (metric == PDS_GATE_MMD2 && !(h > 0.0))))
    return set_error(PDS_ERR_ARG, "gate needs every >= 1, a finite threshold and h > 0 for MMD^2");
  if (!s->active.empty() || !s->queue.empty()) return set_error(PDS_ERR_ARG, "set the gate before submitting jobs");
  s->gate_metric = metric;
  s->gate_every = every;
  s->gate_threshold = threshold;
  s->gate_h = h > 0.0 ? h : 0.1;
  return PDS_OK;
}

int pds_server_job_gate(pds_server_t s, long long job_id, int* checks, double* last_value) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return set_error(PDS_ERR_ARG, "unknown job");
  if (checks) *checks = it->second.gate_checks;
  if (last_value) *last_value = it->second.gate_value;
  return PDS_OK;
}

int pds_server_stats(pds_server_t s, int* queued, int* active, size_t* bytes_in_use) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL server");
  if (queued) *queued = (int)s->queue.size();
  if (active) *active = (int)s->active.size();
  if (bytes_in_use) *bytes_in_use = s->in_use;
  return PDS_OK;
}

}  // extern "C"
