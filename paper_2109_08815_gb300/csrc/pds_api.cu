// C ABI of libpds (declared in include/pds.h): argument checking, device
// memory ownership and kernel dispatch.  No torch types cross this boundary.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "pds_internal.cuh"

namespace pds {
template <int NL>
cudaError_t launch_rollout_nl(const ChainParams&, const float*, int, const Partials&, int, int32_t*, cudaStream_t, size_t,
                              size_t);
template <int NL>
cudaError_t launch_simulate_nl(const ChainParams&, const float*, int, float*, cudaStream_t);

static thread_local std::string g_err;
static thread_local int g_launches = 0;

static int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int set_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

void set_launch_count(int n) { g_launches = n; }

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? PDS_ERR_OOM : PDS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t launch_rollout(const ChainParams& c, const float* X, int N, const Partials& parts, int grad,
                           int32_t* status, cudaStream_t st, size_t u0, size_t nu) {
  switch (c.n) {
    case 1: return launch_rollout_nl<1>(c, X, N, parts, grad, status, st, u0, nu);
    case 2: return launch_rollout_nl<2>(c, X, N, parts, grad, status, st, u0, nu);
    case 3: return launch_rollout_nl<3>(c, X, N, parts, grad, status, st, u0, nu);
    case 4: return launch_rollout_nl<4>(c, X, N, parts, grad, status, st, u0, nu);
    case 5: return launch_rollout_nl<5>(c, X, N, parts, grad, status, st, u0, nu);
    case 6: return launch_rollout_nl<6>(c, X, N, parts, grad, status, st, u0, nu);
    case 7: return launch_rollout_nl<7>(c, X, N, parts, grad, status, st, u0, nu);
    case 8: return launch_rollout_nl<8>(c, X, N, parts, grad, status, st, u0, nu);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_simulate(const ChainParams& c, const float* theta, int N, float* states, cudaStream_t st) {
  switch (c.n) {
    case 1: return launch_simulate_nl<1>(c, theta, N, states, st);
    case 2: return launch_simulate_nl<2>(c, theta, N, states, st);
    case 3: return launch_simulate_nl<3>(c, theta, N, states, st);
    case 4: return launch_simulate_nl<4>(c, theta, N, states, st);
    case 5: return launch_simulate_nl<5>(c, theta, N, states, st);
    case 6: return launch_simulate_nl<6>(c, theta, N, states, st);
    case 7: return launch_simulate_nl<7>(c, theta, N, states, st);
    case 8: return launch_simulate_nl<8>(c, theta, N, states, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pds

using namespace pds;

static void free_parts(Partials& p) {
  cudaFree(p.lp);
  cudaFree(p.th);
  cudaFree(p.start);
  cudaFree(p.next);
  cudaFree(p.tape);
  cudaFree(p.th2);
  cudaFree(p.gdef);
  p = Partials{};
}

int pds::ensure_workspace(pds_problem* p, int N) {
  if (N <= p->cap_N && p->cap_K == p->c.K && p->cap_cs == p->c.csvgd && p->cap_R == p->c.R) return PDS_OK;
  const int newN = N > p->cap_N ? N : p->cap_N;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  free_parts(p->parts);
  p->cap_N = 0;
  const ChainParams& c = p->c;
  // windows of all trajectories: the partials and the tape are per (trajectory, window)
  const size_t Nn = (size_t)newN, W = (size_t)c.W * (size_t)c.R, S = (size_t)c.S, M = (size_t)c.M;
  const size_t U = Nn * W;
  const size_t tape = ((size_t)c.max_seg + (size_t)c.K) * S * U;
  if ((e = cudaMalloc(&p->parts.lp, W * Nn * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->parts.th, W * (M ? M : 1) * Nn * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->parts.start, W * S * Nn * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->parts.next, W * S * Nn * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->parts.tape, tape * sizeof(float))) != cudaSuccess ||
      (c.csvgd && (e = cudaMalloc(&p->parts.th2, W * (M ? M : 1) * Nn * sizeof(float))) != cudaSuccess) ||
      (c.csvgd && (e = cudaMalloc(&p->parts.gdef, W * Nn * sizeof(float))) != cudaSuccess)) {
    free_parts(p->parts);
    return cuda_fail(e, "workspace allocation");
  }
  p->cap_cs = c.csvgd;
  p->cap_R = c.R;
  p->cap_N = newN;
  p->cap_K = c.K;
  return PDS_OK;
}

static void update_segments(ChainParams& c) {
  int hmax = 0;
  for (int w = 0; w < c.W; ++w) {
    const int h = (int)(((long long)(w + 1) * c.T) / c.W - ((long long)w * c.T) / c.W);
    if (h > hmax) hmax = h;
  }
  c.max_seg = (hmax + c.K - 1) / c.K;
}

int pds::ensure_iter_buffers(pds_problem* p, int N) {
  if (p->it_N >= N) return PDS_OK;
  cudaStreamSynchronize(p->stream);
  cudaFree(p->d_grad);
  cudaFree(p->d_logp);
  cudaFree(p->d_x);
  p->d_grad = p->d_logp = p->d_x = nullptr;
  p->it_N = 0;
  cudaError_t e;
  // the constrained method's gradient has M more rows (-dPsi/dtheta)
  const size_t grows = (size_t)p->c.P + (p->c.csvgd ? (size_t)p->c.M : 0);
  if ((e = cudaMalloc(&p->d_grad, grows * N * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_logp, (size_t)N * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_x, (size_t)p->c.P * N * sizeof(float))) != cudaSuccess)
    return cuda_fail(e, "iteration buffers");
  p->it_N = N;
  return PDS_OK;
}

// The chain rollout reads each step's observations in state order, with
// compile-time offsets and 8-byte loads: a [R][T][S] copy of the [R][T][D]
// observations, unobserved components 0 (their residuals are skipped).
// The observations in state order, [R][T][S] (unobserved components 0),
// followed at *out_b (16-byte aligned) by the same values each written twice,
// [R][T][S] float2, for the kernel that steps two particles per thread.
static cudaError_t upload_state_ordered_obs(const ChainParams& c, int R, const float* obs, cudaStream_t st,
                                            float** out, float** out_b) {
  const size_t n = (size_t)R * c.T * c.S;
  const size_t off = (n + 3) / 4 * 4;
  std::vector<float> h(off + 2 * n, 0.f);
  for (size_t rt = 0; rt < (size_t)R * c.T; ++rt)
    for (int j = 0; j < c.S; ++j)
      if (c.obs_col[j] >= 0) h[rt * c.S + j] = obs[rt * c.D + c.obs_col[j]];
  for (size_t k = 0; k < n; ++k) h[off + 2 * k] = h[off + 2 * k + 1] = h[k];
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, h.size() * sizeof(float));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  *out = d;
  *out_b = d + off;
  return cudaSuccess;
}

extern "C" {

const char* pds_strerror(int code) {
  switch (code) {
    case PDS_OK: return "ok";
    case PDS_ERR_ARG: return "invalid argument";
    case PDS_ERR_CUDA: return "CUDA error";
    case PDS_ERR_OOM: return "out of device memory";
    case PDS_ERR_NONFINITE: return "non-finite value";
    case PDS_ERR_TIMEOUT: return "device wait timed out";
    case PDS_ERR_BUDGET: return "over the memory budget";
    case PDS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* pds_last_error(void) { return g_err.c_str(); }

int pds_last_launch_count(void) { return g_launches; }

int pds_problem_create(const pds_system_desc* sys, double dt, int T, int windows, const float* obs, int D,
                       const int* obs_index, double sigma_obs, double sigma_def, const float* s0,
                       const float* theta_lo, const float* theta_hi, double c_lim, void* cuda_stream,
                       pds_problem_t* out) {
  if (!out) return fail(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!sys || !obs || !obs_index || !s0 || !theta_lo || !theta_hi)
    return fail(PDS_ERR_ARG, "NULL argument");
  if (sys->kind != PDS_SYSTEM_PLANAR_CHAIN) return fail(PDS_ERR_UNSUPPORTED, "unknown system kind %d", sys->kind);
  const int n = sys->n_links;
  if (n < 1 || n > PDS_MAX_LINKS) return fail(PDS_ERR_UNSUPPORTED, "n_links %d outside 1..%d", n, PDS_MAX_LINKS);
  if (!sys->mass || !sys->length || !sys->damping) return fail(PDS_ERR_ARG, "NULL link parameter array");
  const int M = sys->n_theta;
  if (M < 1 || M > PDS_MAX_THETA) return fail(PDS_ERR_UNSUPPORTED, "n_theta %d outside 1..%d", M, PDS_MAX_THETA);
  if (M > 0 && (!sys->theta_kind || !sys->theta_link)) return fail(PDS_ERR_ARG, "NULL theta map");
  if (!(dt > 0.0) || T < 1 || windows < 1 || windows > T) return fail(PDS_ERR_ARG, "bad dt/T/windows");
  if (D < 1 || D > 2 * n) return fail(PDS_ERR_ARG, "D %d outside 1..%d", D, 2 * n);
  if (!(sigma_obs > 0.0) || !(sigma_def > 0.0) || !(c_lim >= 0.0)) return fail(PDS_ERR_ARG, "bad sigma or c_lim");

  ChainParams c;
  memset(&c, 0, sizeof(c));
  c.n = n; c.M = M; c.T = T; c.W = windows; c.D = D; c.S = 2 * n; c.P = M + (windows - 1) * 2 * n;
  c.K = 1;
  c.dt = (float)dt;
  c.g = (float)sys->gravity;
  c.inv_so2 = (float)(1.0 / (sigma_obs * sigma_obs));
  c.obs_const = (float)(-0.5 * D * log(2.0 * M_PI * sigma_obs * sigma_obs));
  c.inv_sd2 = (float)(1.0 / (sigma_def * sigma_def));
  c.def_const = (float)(-0.5 * (2 * n) * log(2.0 * M_PI * sigma_def * sigma_def));
  c.c_lim = (float)c_lim;
  for (int j = 0; j < PDS_MAX_LINKS; ++j) { c.mass_theta[j] = c.length_theta[j] = c.damp_theta[j] = -1; }
  for (int j = 0; j < 2 * PDS_MAX_LINKS; ++j) c.obs_col[j] = -1;
  for (int j = 0; j < n; ++j) {
    c.mass[j] = (float)sys->mass[j];
    c.length[j] = (float)sys->length[j];
    c.damping[j] = (float)sys->damping[j];
  }
  double lim = 0.0;
  for (int k = 0; k < M; ++k) {
    const int kind = sys->theta_kind[k], link = sys->theta_link[k];
    if (link < 0 || link >= n) return fail(PDS_ERR_ARG, "theta_link[%d] = %d out of range", k, link);
    int* slot = kind == PDS_PARAM_MASS ? c.mass_theta : kind == PDS_PARAM_LENGTH ? c.length_theta
              : kind == PDS_PARAM_DAMPING ? c.damp_theta : nullptr;
    if (!slot) return fail(PDS_ERR_ARG, "theta_kind[%d] = %d unknown", k, kind);
    if (slot[link] >= 0) return fail(PDS_ERR_ARG, "theta entry %d duplicates a parameter", k);
    slot[link] = k;
    if (!(theta_hi[k] > theta_lo[k])) return fail(PDS_ERR_ARG, "theta box %d empty", k);
    c.lo[k] = theta_lo[k];
    c.hi[k] = theta_hi[k];
    lim -= log((double)theta_hi[k] - (double)theta_lo[k]);
  }
  c.lim_const = (float)lim;
  for (int d = 0; d < D; ++d) {
    const int idx = obs_index[d];
    if (idx < 0 || idx >= 2 * n) return fail(PDS_ERR_ARG, "obs_index[%d] = %d out of range", d, idx);
    if (c.obs_col[idx] >= 0) return fail(PDS_ERR_ARG, "obs_index repeats state %d", idx);
    c.obs_col[idx] = d;
    c.obs_mask |= 1u << idx;
  }
  for (int j = 0; j < 2 * n; ++j) c.s0[j] = s0[j];
  c.R = 1;
  c.combine = 0;
  int hmax = 0;
  for (int w = 0; w < windows; ++w) {
    const int h = (int)(((long long)(w + 1) * T) / windows - ((long long)w * T) / windows);
    if (h > hmax) hmax = h;
  }
  if (hmax > PDS_MAX_WINDOW_STEPS) return fail(PDS_ERR_UNSUPPORTED, "window of %d steps > %d", hmax,
                                                PDS_MAX_WINDOW_STEPS);
  update_segments(c);

  pds_problem* p = new pds_problem();
  p->c = c;
  p->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMalloc(&p->d_obs, (size_t)T * D * sizeof(float));
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaMalloc obs"); }
  e = cudaMemcpyAsync(p->d_obs, obs, (size_t)T * D * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) { cudaFree(p->d_obs); delete p; return cuda_fail(e, "copy obs"); }
  p->c.obs = p->d_obs;
  float* obs_b = nullptr;
  e = upload_state_ordered_obs(p->c, 1, obs, p->stream, &p->d_obs_s, &obs_b);
  if (e != cudaSuccess) { cudaFree(p->d_obs); delete p; return cuda_fail(e, "copy obs (state order)"); }
  p->c.obs_s = p->d_obs_s;
  p->c.obs_b = obs_b;
  *out = p;
  return PDS_OK;
}

int pds_problem_destroy(pds_problem_t p) {
  if (!p) return PDS_OK;
  cudaStreamSynchronize(p->stream);
  if (p->ov_copy) {
    cudaStreamSynchronize(p->ov_copy);
    cudaStreamDestroy(p->ov_copy);
  }
  for (int g = 0; g < pds_problem::kCopyGroups; ++g) {
    if (p->ov_roll[g]) {
      cudaStreamSynchronize(p->ov_roll[g]);
      cudaStreamDestroy(p->ov_roll[g]);
    }
    if (p->ov_copied[g]) cudaEventDestroy(p->ov_copied[g]);
    if (p->ov_rolled[g]) cudaEventDestroy(p->ov_rolled[g]);
  }
  if (p->ov_start) cudaEventDestroy(p->ov_start);
  free_parts(p->parts);
  cudaFree(p->d_obs);
  cudaFree(p->d_obs_s);
  cudaFree(p->d_base);
  cudaFree(p->d_grad);
  cudaFree(p->d_logp);
  cudaFree(p->d_x);
  delete p;
  return PDS_OK;
}

int pds_problem_layout(pds_problem_t p, int* M, int* S, int* P) {
  if (!p) return fail(PDS_ERR_ARG, "NULL problem");
  if (M) *M = p->c.M;
  if (S) *S = p->c.S;
  if (P) *P = p->c.P;
  return PDS_OK;
}

int pds_problem_set_checkpoint_stride(pds_problem_t p, int K) {
  if (!p) return fail(PDS_ERR_ARG, "NULL problem");
  if (K < 1 || K > PDS_MAX_WINDOW_STEPS) return fail(PDS_ERR_ARG, "K %d outside 1..%d", K, PDS_MAX_WINDOW_STEPS);
  p->c.K = K;
  update_segments(p->c);
  return PDS_OK;
}

int pds_problem_set_option(pds_problem_t p, int option, int value) {
  if (!p) return fail(PDS_ERR_ARG, "NULL problem");
  switch (option) {
    case PDS_OPT_CHECKPOINT_STRIDE: return pds_problem_set_checkpoint_stride(p, value);
    case PDS_OPT_FAST_MATH:
      if (value != 0 && value != 1) return fail(PDS_ERR_ARG, "fast math must be 0 or 1");
      p->c.fast_math = value;
      return PDS_OK;
    case PDS_OPT_UNITS_PER_THREAD:
      if (value < 0 || value > 2) return fail(PDS_ERR_ARG, "units per thread must be 0, 1 or 2");
      p->c.units_per_thread = value;
      return PDS_OK;
    default: return fail(PDS_ERR_ARG, "unknown option %d", option);
  }
}

int pds_problem_get_option(pds_problem_t p, int option, int* value) {
  if (!p || !value) return fail(PDS_ERR_ARG, "NULL argument");
  switch (option) {
    case PDS_OPT_CHECKPOINT_STRIDE: *value = p->c.K; return PDS_OK;
    case PDS_OPT_FAST_MATH: *value = p->c.fast_math; return PDS_OK;
    case PDS_OPT_UNITS_PER_THREAD: *value = p->c.units_per_thread; return PDS_OK;
    default: return fail(PDS_ERR_ARG, "unknown option %d", option);
  }
}

int pds_problem_autotune(pds_problem_t p, const float* particles, int N, int* choice) {
  g_launches = 0;
  if (!p || !particles) return fail(PDS_ERR_ARG, "NULL argument");
  if (N < 1 || N > (1 << 20)) return fail(PDS_ERR_ARG, "N %d outside 1..2^20", N);
  if (p->kind != PDS_SYSTEM_PLANAR_CHAIN) return fail(PDS_ERR_UNSUPPORTED, "the autotuner is built for planar chains");
  int rc = ensure_iter_buffers(p, N);
  if (rc != PDS_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
    if (t0) cudaEventDestroy(t0);
    return cuda_fail(e, "cudaEventCreate");
  }
  const int K0 = p->c.K, U0 = p->c.units_per_thread;
  // candidates: K = 1 with one or two units per thread, then larger strides
  // (one unit); each timed over 3 calls after one that warms up
  const int cand[][2] = {{1, 1}, {1, 2}, {5, 1}, {10, 1}, {25, 1}, {50, 1}};
  int best_K = K0, best_U = U0;
  float best = 1e30f;
  for (const auto& kc : cand) {
    if (kc[0] > PDS_MAX_WINDOW_STEPS) continue;
    p->c.K = kc[0];
    p->c.units_per_thread = kc[1];
    update_segments(p->c);
    float tot = 0.f;
    for (int r = 0; r < 4 && rc == PDS_OK; ++r) {
      if ((e = cudaEventRecord(t0, p->stream)) != cudaSuccess) break;
      rc = pds_loglik_grad(p, particles, N, p->d_logp, p->d_grad, nullptr);
      if (rc != PDS_OK) break;
      if ((e = cudaEventRecord(t1, p->stream)) != cudaSuccess || (e = cudaEventSynchronize(t1)) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (r > 0) tot += ms;
    }
    if (rc != PDS_OK || e != cudaSuccess) break;
    if (tot < best) {
      best = tot;
      best_K = kc[0];
      best_U = kc[1];
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc == PDS_OK && e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
  if (rc != PDS_OK) {
    p->c.K = K0;
    p->c.units_per_thread = U0;
    update_segments(p->c);
    return rc;
  }
  p->c.K = best_K;
  p->c.units_per_thread = best_U;
  update_segments(p->c);
  if (choice) {
    choice[0] = best_U;
    choice[1] = best_K;
    choice[2] = (int)(best / 3.f * 1000.f);  // microseconds per call
  }
  return PDS_OK;
}

int pds_problem_set_csvgd(pds_problem_t p, int enable, double c) {
  if (!p) return fail(PDS_ERR_ARG, "NULL problem");
  if (enable != 0 && enable != 1) return fail(PDS_ERR_ARG, "enable must be 0 or 1");
  if (enable && p->kind != PDS_SYSTEM_PLANAR_CHAIN)
    return fail(PDS_ERR_UNSUPPORTED, "constrained SVGD is built for planar chains");
  if (enable && p->c.R > 1) return fail(PDS_ERR_UNSUPPORTED, "constrained SVGD is built for one trajectory");
  if (enable && !(c >= 0.0 && c < 1e30)) return fail(PDS_ERR_ARG, "MDMM damping c must be finite and >= 0");
  cudaStreamSynchronize(p->stream);
  ChainParams& cp = p->c;
  cp.csvgd = enable;
  cp.c_mdmm = enable ? (float)c : 0.f;
  cp.P = cp.M + (cp.W - 1) * cp.S + (enable ? (cp.W - 1) + cp.M : 0);
  // the iteration buffers depend on P
  cudaFree(p->d_grad);
  cudaFree(p->d_logp);
  cudaFree(p->d_x);
  p->d_grad = p->d_logp = p->d_x = nullptr;
  p->it_N = 0;
  return PDS_OK;
}

int pds_problem_set_trajectories(pds_problem_t p, int R, const float* obs, const float* s0, int combine) {
  if (!p || !obs || !s0) return fail(PDS_ERR_ARG, "NULL argument");
  if (R < 1 || R > PDS_MAX_TRAJECTORIES) return fail(PDS_ERR_ARG, "R %d outside 1..%d", R, PDS_MAX_TRAJECTORIES);
  if (combine != PDS_COMBINE_SUM && combine != PDS_COMBINE_PRODUCT) return fail(PDS_ERR_ARG, "unknown combine %d", combine);
  if (p->kind != PDS_SYSTEM_PLANAR_CHAIN) return fail(PDS_ERR_UNSUPPORTED, "trajectory sets are built for planar chains");
  if (p->c.csvgd) return fail(PDS_ERR_UNSUPPORTED, "constrained SVGD is built for one trajectory");
  ChainParams& c = p->c;
  const size_t bytes = (size_t)R * c.T * c.D * sizeof(float);
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  float* d = nullptr;
  if ((e = cudaMalloc(&d, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc observations");
  if ((e = cudaMemcpyAsync(d, obs, bytes, cudaMemcpyHostToDevice, p->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(p->stream)) != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "copy observations");
  }
  float* ds = nullptr;
  float* dsb = nullptr;
  if ((e = upload_state_ordered_obs(c, R, obs, p->stream, &ds, &dsb)) != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "copy observations (state order)");
  }
  cudaFree(p->d_obs);
  cudaFree(p->d_obs_s);
  p->d_obs = d;
  p->d_obs_s = ds;
  c.obs = d;
  c.obs_s = ds;
  c.obs_b = dsb;
  for (int r = 0; r < R; ++r)
    for (int j = 0; j < c.S; ++j) c.s0[r * kMaxState + j] = s0[(size_t)r * c.S + j];
  c.R = R;
  c.combine = combine;
  c.P = c.M + R * (c.W - 1) * c.S;
  // the iteration buffers depend on P
  cudaFree(p->d_grad);
  cudaFree(p->d_logp);
  cudaFree(p->d_x);
  p->d_grad = p->d_logp = p->d_x = nullptr;
  p->it_N = 0;
  return PDS_OK;
}

int pds_svgd_set_csvgd(pds_svgd_t s, int enable, int n_def) {
  if (!s) return fail(PDS_ERR_ARG, "NULL svgd");
  if (enable != 0 && enable != 1) return fail(PDS_ERR_ARG, "enable must be 0 or 1");
  if (enable) {
    const int lam0 = s->sp.P - n_def - s->sp.M;
    if (n_def < 0 || lam0 < s->sp.M) return fail(PDS_ERR_ARG, "n_def %d does not fit P %d, M %d", n_def, s->sp.P, s->sp.M);
    s->sp.lam0 = lam0;
  } else {
    s->sp.lam0 = 0;
  }
  s->sp.csvgd = enable;
  return PDS_OK;
}

int pds_problem_reserve(pds_problem_t p, int N_max) {
  if (!p) return fail(PDS_ERR_ARG, "NULL problem");
  if (N_max < 1 || N_max > (1 << 20)) return fail(PDS_ERR_ARG, "N_max %d outside 1..2^20", N_max);
  return ensure_workspace(p, N_max);
}

int pds_loglik_grad(pds_problem_t p, const float* particles, int N, float* logp, float* grad, int32_t* status) {
  g_launches = 0;
  if (!p || !particles || !logp) return fail(PDS_ERR_ARG, "NULL argument");
  if (N < 1 || N > (1 << 20)) return fail(PDS_ERR_ARG, "N %d outside 1..2^20", N);
  int rc = ensure_workspace(p, N);
  if (rc != PDS_OK) return rc;
  cudaError_t e =
      (p->kind == PDS_SYSTEM_ARM_BOX)
          ? launch_armbox_rollout(p->c, p->ab, particles, N, p->parts, grad != nullptr, status, p->stream)
      : (p->kind == PDS_SYSTEM_RIGID_DOUBLE_PENDULUM)
          ? launch_rigid2_rollout(p->c, p->r2, particles, N, p->parts, grad != nullptr, status, p->stream)
          : launch_rollout(p->c, particles, N, p->parts, grad != nullptr, status, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rollout launch");
  e = launch_window_reduce(p->c, particles, N, p->parts, logp, grad, status, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "window reduce launch");
  g_launches = 2;
  return PDS_OK;
}

int pds_simulate(pds_problem_t p, const float* theta, int N, float* states) {
  g_launches = 0;
  if (!p || !theta || !states) return fail(PDS_ERR_ARG, "NULL argument");
  if (N < 1 || N > (1 << 20)) return fail(PDS_ERR_ARG, "N %d outside 1..2^20", N);
  cudaError_t e = (p->kind == PDS_SYSTEM_ARM_BOX) ? launch_armbox_simulate(p->c, p->ab, theta, N, states, p->stream)
                   : (p->kind == PDS_SYSTEM_RIGID_DOUBLE_PENDULUM)
                       ? launch_rigid2_simulate(p->c, p->r2, theta, N, states, p->stream)
                       : launch_simulate(p->c, theta, N, states, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "simulate launch");
  g_launches = 1;
  return PDS_OK;
}

int pds_svgd_create(int N, int M, int P, const float* theta_lo, const float* theta_hi, double lr, double beta1,
                    double beta2, double eps, int clamp, void* cuda_stream, pds_svgd_t* out) {
  if (!out) return fail(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (N < 1 || N > 65536) return fail(PDS_ERR_ARG, "N %d outside 1..65536", N);
  if (M < 1 || M > PDS_MAX_THETA || P < M) return fail(PDS_ERR_ARG, "bad M %d / P %d", M, P);
  if (!theta_lo || !theta_hi) return fail(PDS_ERR_ARG, "NULL box");
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0))
    return fail(PDS_ERR_ARG, "bad Adam constants");
  pds_svgd* s = new pds_svgd();
  memset(&s->sp, 0, sizeof(s->sp));
  s->sp.N = N; s->sp.M = M; s->sp.P = P;
  for (int k = 0; k < M; ++k) {
    if (!(theta_hi[k] > theta_lo[k])) { delete s; return fail(PDS_ERR_ARG, "theta box %d empty", k); }
    s->sp.lo[k] = theta_lo[k];
    s->sp.hi[k] = theta_hi[k];
  }
  s->sp.lr = (float)lr; s->sp.b1 = (float)beta1; s->sp.b2 = (float)beta2; s->sp.eps = (float)eps;
  s->sp.clamp = clamp ? 1 : 0;
  s->stream = (cudaStream_t)cuda_stream;
  s->w.chunks = svgd_phi_partials(N);
  s->w.cand_cap = svgd_cand_capacity(N);
  const size_t MN = (size_t)M * N, PN = (size_t)P * N;
  cudaError_t e = cudaSuccess;
  if ((s->w.cand_cap && (e = cudaMalloc(&s->w.cand, s->w.cand_cap * sizeof(float))) != cudaSuccess) ||
      (s->w.cand_cap && (e = cudaMalloc(&s->w.samp, svgd_sample_size() * sizeof(float))) != cudaSuccess) ||
      (s->w.cand_cap && (e = cudaMalloc(&s->w.cbuf, svgd_cbin_capacity() * sizeof(float))) != cudaSuccess) ||
      (N >= 256 && (e = cudaMalloc(&s->w.tc, phi_tc_floats(N, M) * sizeof(float))) != cudaSuccess) ||
      (N >= 2048 && (e = cudaMalloc(&s->w.mimg, median_tc_floats(N, M) * sizeof(float))) != cudaSuccess) ||
      (e = cudaMalloc(&s->w.u, MN * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->w.gu, MN * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->w.phi_part, (size_t)s->w.chunks * MN * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->w.adam_m, PN * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->w.adam_v, PN * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->w.ctl, sizeof(SvgdCtl))) != cudaSuccess ||
      (e = cudaHostAlloc(&s->h_status, sizeof(int), cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&s->w.status_flags, s->h_status, 0)) != cudaSuccess) {
    pds_svgd_destroy(s);
    return cuda_fail(e, "svgd allocation");
  }
  *(volatile int*)s->h_status = 0;
  s->w.wait_limit = kWaitLimitDefault;
  s->w.small_median = 1;
  if (N >= 2048) {
    const int n_items = median_tc_work_items(N, nullptr);
    std::vector<int> items(2 * (size_t)n_items);
    median_tc_work_items(N, items.data());
    if ((e = cudaMalloc(&s->w.mwork, items.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(s->w.mwork, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
      pds_svgd_destroy(s);
      return cuda_fail(e, "svgd allocation");
    }
    s->w.n_mwork = n_items;
  }
  *out = s;
  return pds_svgd_reset(s);
}

// Forget the captured SVGD steps (their graphs and the calls counted towards a capture).
static void drop_graph_slot(pds_svgd::Graph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.calls = 0;
}
static void drop_graph(pds_svgd* s) {
  for (auto& g : s->graphs) drop_graph_slot(g);
  if (s->iter_exec) cudaGraphExecDestroy(s->iter_exec);
  s->iter_exec = nullptr;
  s->iter_calls = 0;
}

int pds_svgd_set_option(pds_svgd_t s, int option, int value) {
  if (!s) return fail(PDS_ERR_ARG, "NULL svgd");
  if (option == PDS_OPT_WAIT_LIMIT) {
    if (value < 0) return fail(PDS_ERR_ARG, "wait limit %d < 0", value);
    s->w.wait_limit = value;
    return PDS_OK;
  }
  if (option == PDS_OPT_GRAPH) {
    if (value != 0 && value != 1) return fail(PDS_ERR_ARG, "option value must be 0 or 1");
    if (!value) drop_graph(s);
    s->use_graph = value;
    return PDS_OK;
  }
  if (value != 0 && value != 1) return fail(PDS_ERR_ARG, "option value must be 0 or 1");
  switch (option) {
    case PDS_OPT_FAST_MATH: s->sp.fast_math = value; return PDS_OK;
    case PDS_OPT_MEDIAN_FULL_PASSES: s->full_passes = value; return PDS_OK;
    case PDS_OPT_PHI_CUDA_CORES: s->phi_cuda_cores = value; return PDS_OK;
    case PDS_OPT_MEDIAN_CUDA_CORES: s->median_cuda_cores = value; return PDS_OK;
    default: return fail(PDS_ERR_ARG, "unknown option %d", option);
  }
}

int pds_svgd_reset(pds_svgd_t s) {
  if (!s) return fail(PDS_ERR_ARG, "NULL svgd");
  const size_t PN = (size_t)s->sp.P * s->sp.N;
  cudaError_t e;
  if ((e = cudaMemsetAsync(s->w.adam_m, 0, PN * sizeof(float), s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->w.adam_v, 0, PN * sizeof(float), s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->w.ctl, 0, sizeof(SvgdCtl), s->stream)) != cudaSuccess)
    return cuda_fail(e, "svgd reset");
  s->grad_dead_seen = 0;
  return PDS_OK;
}

int pds_svgd_destroy(pds_svgd_t s) {
  if (!s) return PDS_OK;
  cudaStreamSynchronize(s->stream);
  if (s->gstream) cudaStreamSynchronize(s->gstream);
  if (s->side) cudaStreamSynchronize(s->side);
  cudaFree(s->w.cand);
  cudaFree(s->w.samp);
  cudaFree(s->w.cbuf);
  cudaFree(s->w.tc);
  cudaFree(s->w.mimg);
  cudaFree(s->w.mwork);
  cudaFree(s->w.u);
  cudaFree(s->w.gu);
  cudaFree(s->w.phi_part);
  cudaFree(s->w.adam_m);
  cudaFree(s->w.adam_v);
  cudaFree(s->w.ctl);
  if (s->h_status) cudaFreeHost(s->h_status);
  drop_graph(s);
  if (s->gstream) cudaStreamDestroy(s->gstream);
  if (s->gev_in) cudaEventDestroy(s->gev_in);
  if (s->gev_out) cudaEventDestroy(s->gev_out);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  delete s;
  return PDS_OK;
}

// Status that the device reported for steps already run (the mapped host
// word, cleared by reading): PDS_ERR_TIMEOUT before PDS_ERR_NONFINITE.
static int take_status(pds_svgd* s) {
  if (!s->h_status) return PDS_OK;
  volatile int* h = s->h_status;
  const int f = *h;
  if (!f) return PDS_OK;
  *h = 0;
  if (f & kStatusGradDead) s->grad_dead_seen = 1;
  if (!(f & (kStatusTimeout | kStatusNoneLive))) return PDS_OK;
  if (f & kStatusTimeout)
    return fail(PDS_ERR_TIMEOUT, "a tensor-core pass of an SVGD step gave up waiting for its copies or products; "
                                 "that step's particles are not valid");
  return fail(PDS_ERR_NONFINITE, "an SVGD step found no particle with finite coordinates and gradient");
}

int pds_svgd_status(pds_svgd_t s) {
  if (!s) return fail(PDS_ERR_ARG, "NULL svgd");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess && s->gstream) e = cudaStreamSynchronize(s->gstream);
  if (e != cudaSuccess) return cuda_fail(e, "svgd status");
  return take_status(s);
}

// The workspace view of a step under the state's options.
static SvgdWork svgd_work(const pds_svgd* s) {
  SvgdWork w = s->w;
  if (s->full_passes) {
    w.cand_cap = 0;
    w.small_median = 0;
  }
  if (s->phi_cuda_cores) w.tc = nullptr;
  if (s->median_cuda_cores) w.mimg = nullptr;
  return w;
}

// The ~25 kernels of one step (or of one of its phases), launched one by one on st.
static cudaError_t svgd_launch_all(pds_svgd* s, float* X, const float* G, float* bw_out, float* phi_out,
                                   cudaStream_t st, int* n, int phase = kSvgdAll) {
  return launch_svgd_step(s->sp, svgd_work(s), X, G, bw_out, phi_out, st, n, phase);
}

static bool default_stream(cudaStream_t st) {
  return st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
}

// The caller is capturing st (its own graph then takes the kernels).
static bool being_captured(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown: launch directly
  }
  return cs != cudaStreamCaptureStatusNone;
}

// The stream the step's graph is captured on and replayed on: the caller's,
// or (for a default stream, which cannot be captured) the state's own.
static cudaError_t graph_stream(pds_svgd* s, cudaStream_t* out) {
  if (!default_stream(s->stream)) {
    *out = s->stream;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (!s->gstream && (e = cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if (!s->gev_in && (e = cudaEventCreateWithFlags(&s->gev_in, cudaEventDisableTiming)) != cudaSuccess) return e;
  if (!s->gev_out && (e = cudaEventCreateWithFlags(&s->gev_out, cudaEventDisableTiming)) != cudaSuccess) return e;
  *out = s->gstream;
  return cudaSuccess;
}

// Order gs after the caller's stream (before = true) or the caller's stream
// after gs; nothing when gs is the caller's stream.
static cudaError_t join(pds_svgd* s, cudaStream_t gs, bool before) {
  if (gs == s->stream) return cudaSuccess;
  cudaError_t e;
  if (before) {
    if ((e = cudaEventRecord(s->gev_in, s->stream)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(gs, s->gev_in, 0);
  }
  if ((e = cudaEventRecord(s->gev_out, gs)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s->stream, s->gev_out, 0);
}

int pds_svgd_step(pds_svgd_t s, float* particles, const float* grad, float* bandwidth_out, float* phi_out) {
  g_launches = 0;
  if (!s || !particles || !grad) return fail(PDS_ERR_ARG, "NULL argument");
  const int st = take_status(s);  // reported by a step already run: this one is not queued
  if (st != PDS_OK) return st;
  int n = 0;
  cudaError_t e = cudaSuccess;
  auto direct = [&]() {
    e = svgd_launch_all(s, particles, grad, bandwidth_out, phi_out, s->stream, &n);
    g_launches = n;
    return e == cudaSuccess ? PDS_OK : cuda_fail(e, "svgd launch");
  };
  if (!s->use_graph || being_captured(s->stream)) return direct();
  SvgdGraphKey k;
  memset(&k, 0, sizeof(k));
  k.X = particles;
  k.G = grad;
  k.bw_out = bandwidth_out;
  k.phi_out = phi_out;
  k.full_passes = s->full_passes;
  k.phi_cuda_cores = s->phi_cuda_cores;
  k.median_cuda_cores = s->median_cuda_cores;
  k.wait_limit = s->w.wait_limit;
  k.sp = s->sp;
  pds_svgd::Graph* gr = nullptr;
  for (auto& g : s->graphs)
    if (g.calls > 0 && memcmp(&k, &g.key, sizeof(k)) == 0) gr = &g;
  if (!gr) {
    // a new key takes the slot used longest ago
    gr = &s->graphs[0];
    for (auto& g : s->graphs)
      if (g.used < gr->used) gr = &g;
    drop_graph_slot(*gr);
    gr->key = k;
  }
  gr->used = ++s->graph_clock;
  // first call with these buffers: launch directly (it also does each
  // kernel's one-time set-up, which is not captured)
  if (!gr->exec && gr->calls++ == 0) return direct();
  cudaStream_t gs = nullptr;
  if ((e = graph_stream(s, &gs)) != cudaSuccess || (e = join(s, gs, true)) != cudaSuccess)
    return cuda_fail(e, "svgd graph stream");
  if (!gr->exec) {
    // second call: capture the step once, then replay it
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t el = svgd_launch_all(s, particles, grad, bandwidth_out, phi_out, gs, &n);
      e = cudaStreamEndCapture(gs, &g);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gr->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      // capture refused: launch directly from now on
      cudaGetLastError();
      gr->exec = nullptr;
      s->use_graph = 0;
      if ((e = join(s, gs, false)) != cudaSuccess) return cuda_fail(e, "svgd graph stream");
      return direct();
    }
    gr->launches = n;
  }
  e = cudaGraphLaunch(gr->exec, gs);
  g_launches = gr->launches;
  if (e != cudaSuccess) return cuda_fail(e, "svgd graph launch");
  if ((e = join(s, gs, false)) != cudaSuccess) return cuda_fail(e, "svgd graph stream");
  return PDS_OK;
}

// One SVGD iteration with the step's median phase beside the likelihood.
// The median needs only the coordinates, which the likelihood does not
// change, so it runs on a high-priority side stream while the rollout runs
// (its blocks fill the SMs that the rollout's last wave leaves idle); the
// step's gradient phase waits for both.  The results are those of
// pds_loglik_grad followed by pds_svgd_step.
static bool iterate_overlaps(const pds_problem* p, pds_svgd* s) {
  // a divergent particle (finite coordinates, gradient not finite) makes the
  // split step compute the median twice: such a state runs its steps whole
  if (s->h_status && (*(volatile int*)s->h_status & kStatusGradDead)) s->grad_dead_seen = 1;
  return p->kind == PDS_SYSTEM_PLANAR_CHAIN && s->use_graph && p->stream == s->stream && !default_stream(s->stream) &&
         svgd_step_splits(s->sp, svgd_work(s)) && !s->grad_dead_seen;
}

static cudaError_t iterate_enqueue(pds_problem* p, pds_svgd* s, float* X, float* lp, cudaStream_t st, int* n) {
  const int N = s->sp.N;
  cudaError_t e;
  // the rollout goes first, so that its first wave takes every SM; the
  // median phase's blocks (highest priority) then take the slots that the
  // rollout's blocks free, and fill its last, part-empty wave
  if ((e = cudaEventRecord(s->ev_fork, st)) != cudaSuccess) return e;
  if ((e = launch_rollout(p->c, X, N, p->parts, 1, nullptr, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s->side, s->ev_fork, 0)) != cudaSuccess) return e;
  if ((e = svgd_launch_all(s, X, p->d_grad, nullptr, nullptr, s->side, n, kSvgdTheta)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(s->ev_join, s->side)) != cudaSuccess) return e;
  if ((e = launch_window_reduce(p->c, X, N, p->parts, lp, p->d_grad, nullptr, st)) != cudaSuccess) return e;
  *n += 2;
  if ((e = cudaStreamWaitEvent(st, s->ev_join, 0)) != cudaSuccess) return e;
  return svgd_launch_all(s, X, p->d_grad, nullptr, nullptr, st, n, kSvgdGrad);
}

// The side stream (highest priority) and its two events, created on first use.
static int ensure_side(pds_svgd* s) {
  if (s->side) return PDS_OK;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaError_t e;
  if ((e = cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, hi)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "iteration streams");
  return PDS_OK;
}

static int iterate_overlapped(pds_problem* p, pds_svgd* s, float* X, float* lp) {
  const int st_rc = take_status(s);  // reported by a step already run: this one is not queued
  if (st_rc != PDS_OK) return st_rc;
  cudaError_t e = cudaSuccess;
  if (int rc = ensure_side(s)) return rc;
  pds_svgd::IterKey k;
  memset(&k, 0, sizeof(k));
  k.prob = p;
  k.X = X;
  k.logp = lp;
  k.grad = p->d_grad;
  k.N = s->sp.N;
  k.c = p->c;
  k.parts = p->parts;
  k.step.X = X;
  k.step.G = p->d_grad;
  k.step.full_passes = s->full_passes;
  k.step.phi_cuda_cores = s->phi_cuda_cores;
  k.step.median_cuda_cores = s->median_cuda_cores;
  k.step.wait_limit = s->w.wait_limit;
  k.step.sp = s->sp;
  if (memcmp(&k, &s->iter_key, sizeof(k)) != 0) {
    if (s->iter_exec) cudaGraphExecDestroy(s->iter_exec);
    s->iter_exec = nullptr;
    s->iter_calls = 0;
    s->iter_key = k;
  }
  int n = 0;
  if (!s->iter_exec && s->iter_calls++ == 0) {
    // first iteration with this key: direct launches (they also do each
    // kernel's one-time set-up, which is not captured)
    e = iterate_enqueue(p, s, X, lp, s->stream, &n);
    g_launches = n;
    return e == cudaSuccess ? PDS_OK : cuda_fail(e, "iteration launch");
  }
  if (!s->iter_exec) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t el = iterate_enqueue(p, s, X, lp, s->stream, &n);
      e = cudaStreamEndCapture(s->stream, &g);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->iter_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->iter_exec = nullptr;
      return cuda_fail(e, "iteration graph capture");
    }
    s->iter_launches = n;
  }
  e = cudaGraphLaunch(s->iter_exec, s->stream);
  g_launches = s->iter_launches;
  return e == cudaSuccess ? PDS_OK : cuda_fail(e, "iteration graph launch");
}

int pds_iterate(pds_problem_t p, pds_svgd_t s, float* particles, int iters, float* logp) {
  if (!p || !s || !particles) return fail(PDS_ERR_ARG, "NULL argument");
  if (iters < 0) return fail(PDS_ERR_ARG, "iters < 0");
  if (s->sp.M != p->c.M || s->sp.P != p->c.P) return fail(PDS_ERR_ARG, "SVGD state does not match the problem");
  if (s->sp.csvgd != p->c.csvgd ||
      (p->c.csvgd && s->sp.lam0 != p->c.M + (p->c.W - 1) * p->c.S))
    return fail(PDS_ERR_ARG, "constrained SVGD set on one of problem and SVGD state only");
  const int N = s->sp.N;
  int rc = ensure_iter_buffers(p, N);
  if (rc != PDS_OK) return rc;
  rc = ensure_workspace(p, N);
  if (rc != PDS_OK) return rc;
  int total = 0;
  const bool capturable = !being_captured(s->stream);
  for (int it = 0; it < iters; ++it) {
    float* lp = (logp && it == iters - 1) ? logp : p->d_logp;
    if (capturable && iterate_overlaps(p, s)) {
      // log p always into the problem's buffer (the graph's key stays the
      // same for every iteration), copied out after the last one
      rc = iterate_overlapped(p, s, particles, p->d_logp);
      if (rc != PDS_OK) return rc;
      total += g_launches;
      if (lp != p->d_logp) {
        const cudaError_t e =
            cudaMemcpyAsync(lp, p->d_logp, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy log p");
      }
      continue;
    }
    rc = pds_loglik_grad(p, particles, N, lp, p->d_grad, nullptr);
    if (rc != PDS_OK) return rc;
    total += g_launches;
    rc = pds_svgd_step(s, particles, p->d_grad, nullptr, nullptr);
    if (rc != PDS_OK) return rc;
    total += g_launches;
  }
  g_launches = total;
  return PDS_OK;
}

// The copy streams and events of a problem (created on first use).
static int ensure_copy_streams(pds_problem* p) {
  if (p->ov_copy) return PDS_OK;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&p->ov_copy, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&p->ov_start, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "copy streams");
  for (int g = 0; g < pds_problem::kCopyGroups; ++g)
    if ((e = cudaStreamCreateWithFlags(&p->ov_roll[g], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->ov_copied[g], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->ov_rolled[g], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "copy streams");
  return PDS_OK;
}

// The first log p + gradient of pds_iterate_host with its copy in: the
// particle rows [P][N] go over in groups of windows (theta and the shooting
// states up to the group's last defect target), and each group's rollout
// units (contiguous, u = w N + i) start on a stream of their own as soon as
// their rows have landed, so that the copy hides behind the rollout.  The
// kernels and their arithmetic are those of pds_loglik_grad.
// s (may be NULL): the SVGD state whose step's median phase starts on its
// side stream as soon as the first group of rows, which holds theta, has
// landed; the caller then runs the step's gradient phase after ev_join.
static int loglik_grad_copy_in(pds_problem* p, const float* host, int N, int* launches, pds_svgd* s) {
  const ChainParams& c = p->c;
  const int G = c.W < pds_problem::kCopyGroups ? c.W : pds_problem::kCopyGroups;
  cudaError_t e = cudaSuccess;
  if (int rc = ensure_copy_streams(p)) return rc;
  // the copies wait for earlier work on the problem's stream (it may still read d_x)
  if ((e = cudaEventRecord(p->ov_start, p->stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(p->ov_copy, p->ov_start, 0)) != cudaSuccess)
    return cuda_fail(e, "copy order");
  size_t row0 = 0;
  for (int g = 0; g < G; ++g) {
    const int w0 = (int)(((long long)g * c.W) / G), w1 = (int)(((long long)(g + 1) * c.W) / G);
    // rows of theta and of the shooting states s^s_1 .. s^s_min(w1, W-1)
    const size_t row1 = (size_t)c.M + (size_t)c.S * (size_t)(w1 < c.W - 1 ? w1 : c.W - 1);
    if (row1 > row0) {
      e = cudaMemcpyAsync(p->d_x + row0 * N, host + row0 * N, (row1 - row0) * N * sizeof(float),
                          cudaMemcpyHostToDevice, p->ov_copy);
      if (e != cudaSuccess) return cuda_fail(e, "copy particles to device");
      row0 = row1;
    }
    if ((e = cudaEventRecord(p->ov_copied[g], p->ov_copy)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->ov_roll[g], p->ov_copied[g], 0)) != cudaSuccess)
      return cuda_fail(e, "copy order");
    if (g == 0 && s) {
      int n = 0;
      if ((e = cudaStreamWaitEvent(s->side, p->ov_copied[0], 0)) != cudaSuccess ||
          (e = svgd_launch_all(s, p->d_x, p->d_grad, nullptr, nullptr, s->side, &n, kSvgdTheta)) != cudaSuccess ||
          (e = cudaEventRecord(s->ev_join, s->side)) != cudaSuccess)
        return cuda_fail(e, "svgd median phase");
      *launches += n;
    }
    e = launch_rollout(c, p->d_x, N, p->parts, 1, nullptr, p->ov_roll[g], (size_t)w0 * N, (size_t)(w1 - w0) * N);
    if (e != cudaSuccess) return cuda_fail(e, "rollout launch");
    if ((e = cudaEventRecord(p->ov_rolled[g], p->ov_roll[g])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->stream, p->ov_rolled[g], 0)) != cudaSuccess)
      return cuda_fail(e, "copy order");
  }
  e = launch_window_reduce(c, p->d_x, N, p->parts, p->d_logp, p->d_grad, nullptr, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "window reduce launch");
  *launches += G + 1;
  return PDS_OK;
}

int pds_iterate_host(pds_problem_t p, pds_svgd_t s, float* particles_host, int iters, float* logp_host) {
  if (!p || !s || !particles_host) return fail(PDS_ERR_ARG, "NULL argument");
  if (iters < 0) return fail(PDS_ERR_ARG, "iters < 0");
  const int N = s->sp.N;
  int rc = ensure_iter_buffers(p, N);
  if (rc != PDS_OK) return rc;
  const size_t bytes = (size_t)p->c.P * N * sizeof(float);
  cudaError_t e = cudaSuccess;
  // the copy in overlaps the first rollout for a single planar-chain
  // trajectory (the units of a group of windows are contiguous)
  const bool copy_in = iters >= 1 && s->sp.M == p->c.M && s->sp.P == p->c.P && !s->sp.csvgd && !p->c.csvgd &&
                       p->kind == PDS_SYSTEM_PLANAR_CHAIN && p->c.R == 1;
  int launches = 0;
  if (copy_in) {
    if ((rc = take_status(s)) != PDS_OK) return rc;
    if ((rc = ensure_workspace(p, N)) != PDS_OK) return rc;
    // the step's median phase beside the copies and the rollout (direct
    // launches), then its gradient phase
    const bool split = svgd_step_splits(s->sp, svgd_work(s)) && s->stream == p->stream &&
                       !being_captured(p->stream) && !s->grad_dead_seen;
    if (split && (rc = ensure_side(s)) != PDS_OK) return rc;
    if ((rc = loglik_grad_copy_in(p, particles_host, N, &launches, split ? s : nullptr)) != PDS_OK) return rc;
    if (split) {
      int n = 0;
      if ((e = cudaStreamWaitEvent(p->stream, s->ev_join, 0)) != cudaSuccess ||
          (e = svgd_launch_all(s, p->d_x, p->d_grad, nullptr, nullptr, p->stream, &n, kSvgdGrad)) != cudaSuccess)
        return cuda_fail(e, "svgd gradient phase");
      launches += n;
    } else {
      if ((rc = pds_svgd_step(s, p->d_x, p->d_grad, nullptr, nullptr)) != PDS_OK) return rc;
      launches += g_launches;
    }
    if (iters > 1) {
      if ((rc = pds_iterate(p, s, p->d_x, iters - 1, p->d_logp)) != PDS_OK) return rc;
      launches += g_launches;
    }
  } else {
    e = cudaMemcpyAsync(p->d_x, particles_host, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy particles to device");
    if ((rc = pds_iterate(p, s, p->d_x, iters, p->d_logp)) != PDS_OK) return rc;
    launches = g_launches;
  }
  e = cudaMemcpyAsync(particles_host, p->d_x, bytes, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess && logp_host)
    e = cudaMemcpyAsync(logp_host, p->d_logp, (size_t)N * sizeof(float), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy results to host");
  g_launches = launches;
  if (s->stream != p->stream && (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
    return cuda_fail(e, "svgd stream");
  return take_status(s);
}

}  // extern "C"
