// Window reduction and parameter-limit prior (Sec. IV-C Eq. 5 as a sum of
// logs over windows, Sec. IV-D prior), fixed summation order over windows
// (deterministic).
//
// Grid: x over particles, y over row groups.  y = 0: log p of the particle;
// y = w in 1..W-1: the gradient of shooting state s^s_w, the start-state
// adjoint of window w plus the defect adjoint of window w-1; y = W + k: the
// gradient of theta_k (sum over the W windows plus the prior's).  In constrained-SVGD mode y = 0 also
// writes the constraint values and the constraint gradient of theta.  Non-finite results are ORed into
// status[i], which the rollout kernel zeroed for this call.
#include <math.h>

#include "pds_internal.cuh"

namespace pds {

__global__ void __launch_bounds__(256) window_reduce_kernel(const ChainParams c, const float* __restrict__ X, int N,
                                                            Partials parts, float* __restrict__ logp,
                                                            float* __restrict__ grad, int32_t* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int y = blockIdx.y;
  bool finite = true;
  if (c.R > 1) {
    // a set of trajectories: a_r = sum_w lp of trajectory r; the mixture's
    // responsibilities w_r = softmax(a) (sum) or 1 (product) weight each
    // trajectory's gradients; the limit prior counts once
    double a[kMaxTraj];
    double amax = -INFINITY;
    for (int r = 0; r < c.R; ++r) {
      double s = 0.0;
      for (int w = 0; w < c.W; ++w) s += (double)parts.lp[((size_t)r * c.W + w) * N + i];
      a[r] = s;
      amax = fmax(amax, s);
    }
    double wt[kMaxTraj];
    double lp = 0.0;
    if (c.combine == 0) {
      double z = 0.0;
      for (int r = 0; r < c.R; ++r) z += exp(a[r] - amax);
      for (int r = 0; r < c.R; ++r) wt[r] = exp(a[r] - amax) / z;
      lp = amax + log(z) - log((double)c.R);
    } else {
      for (int r = 0; r < c.R; ++r) { wt[r] = 1.0; lp += a[r]; }
    }
    if (y == 0) {
      float pen = 0.f;
      for (int k = 0; k < c.M; ++k) {
        const float width = c.hi[k] - c.lo[k];
        const float uk = (X[(size_t)k * N + i] - c.lo[k]) / width;
        const float cu = fminf(1.f, fmaxf(0.f, uk));
        pen += (cu - uk) * (cu - uk);
        if (grad) {
          double g = 0.0;
          for (int r = 0; r < c.R; ++r) {
            float gr = 0.f;
            for (int w = 0; w < c.W; ++w) gr += parts.th[(((size_t)r * c.W + w) * c.M + k) * N + i];
            g += wt[r] * (double)gr;
          }
          const float gf = (float)g + c.c_lim * (cu - uk) / width;
          finite = finite && isfinite(gf);
          grad[(size_t)k * N + i] = gf;
        }
      }
      lp += (double)c.lim_const - 0.5 * (double)c.c_lim * (double)pen;
      const float lpf = (float)lp;
      finite = finite && isfinite(lpf);
      logp[i] = lpf;
    } else {
      const int r = y / c.W, w = y - r * c.W;
      if (w >= 1) {
        const int S = c.S;
        const float* st = parts.start + (size_t)y * S * N + i;
        const float* nx = parts.next + (size_t)(y - 1) * S * N + i;
        float* out = grad + ((size_t)c.M + (size_t)(r * (c.W - 1) + w - 1) * S) * N + i;
        const float wr = (float)wt[r];
        for (int s2 = 0; s2 < S; ++s2) {
          const float g = wr * (st[(size_t)s2 * N] + nx[(size_t)s2 * N]);
          finite = finite && isfinite(g);
          out[(size_t)s2 * N] = g;
        }
      }
    }
  } else if (c.csvgd && y == 0) {
    // constrained SVGD (Sec. IV-E): log p_obs; theta rows d log p_obs/dtheta;
    // multiplier rows g_def and g_lim; rows P..P+M-1 -dPsi/dtheta (defect and
    // limit constraints, multipliers fixed)
    const int Pms = c.M + (c.W - 1) * c.S;
    double lp = 0.0;
    for (int w = 0; w < c.W; ++w) lp += (double)parts.lp[(size_t)w * N + i];
    const float lpf = (float)lp;
    finite = isfinite(lpf);
    logp[i] = lpf;
    if (grad) {
      for (int w = 0; w + 1 < c.W; ++w) {
        const float g = parts.gdef[(size_t)w * N + i];
        finite = finite && isfinite(g);
        grad[(size_t)(Pms + w) * N + i] = g;
      }
      for (int k = 0; k < c.M; ++k) {
        float go = 0.f, gc = 0.f;
        for (int w = 0; w < c.W; ++w) {
          go += parts.th[((size_t)w * c.M + k) * N + i];
          gc += parts.th2[((size_t)w * c.M + k) * N + i];
        }
        const float width = c.hi[k] - c.lo[k];
        const float uk = (X[(size_t)k * N + i] - c.lo[k]) / width;
        const float gl = fminf(1.f, fmaxf(0.f, uk)) - uk;
        const float dg_du = (uk < 0.f || uk > 1.f) ? -1.f : 0.f;  // d clamp / du is 0 outside the box
        const float lam = X[(size_t)(Pms + c.W - 1 + k) * N + i];
        gc -= (lam + c.c_mdmm * gl) * dg_du / width;
        finite = finite && isfinite(go) && isfinite(gc);
        grad[(size_t)k * N + i] = go;
        grad[(size_t)(Pms + c.W - 1 + k) * N + i] = gl;
        grad[(size_t)(c.P + k) * N + i] = gc;
      }
    }
  } else if (y == 0) {
    // log-likelihood: windows summed in double, in window order
    double lp = 0.0;
    for (int w = 0; w < c.W; ++w) lp += (double)parts.lp[(size_t)w * N + i];
    // limit prior: -sum log(hi - lo) - (c/2) sum (clamp(u) - u)^2 in unit-box coordinates
    float pen = 0.f;
    for (int k = 0; k < c.M; ++k) {
      const float width = c.hi[k] - c.lo[k];
      const float uk = (X[(size_t)k * N + i] - c.lo[k]) / width;
      const float cu = fminf(1.f, fmaxf(0.f, uk));
      pen += (cu - uk) * (cu - uk);
    }
    lp += (double)c.lim_const - 0.5 * (double)c.c_lim * (double)pen;
    const float lpf = (float)lp;
    finite = finite && isfinite(lpf);
    logp[i] = lpf;
  } else if (y >= c.W) {
    // theta component k: sum over the windows plus the limit prior's gradient
    const int k = y - c.W;
    const float width = c.hi[k] - c.lo[k];
    const float uk = (X[(size_t)k * N + i] - c.lo[k]) / width;
    const float cu = fminf(1.f, fmaxf(0.f, uk));
    float g = 0.f;
    for (int w = 0; w < c.W; ++w) g += parts.th[((size_t)w * c.M + k) * N + i];
    g += c.c_lim * (cu - uk) / width;
    finite = isfinite(g);
    grad[(size_t)k * N + i] = g;
  } else {
    const int w = y;
    const int S = c.S;
    const float* st = parts.start + (size_t)w * S * N + i;
    const float* nx = parts.next + (size_t)(w - 1) * S * N + i;
    float* out = grad + ((size_t)c.M + (size_t)(w - 1) * S) * N + i;
    for (int s = 0; s < S; ++s) {
      const float g = st[(size_t)s * N] + nx[(size_t)s * N];
      finite = finite && isfinite(g);
      out[(size_t)s * N] = g;
    }
  }
  if (status && !finite) atomicOr(status + i, 1);
}

cudaError_t launch_window_reduce(const ChainParams& c, const float* X, int N, const Partials& parts, float* logp,
                                 float* grad, int32_t* status, cudaStream_t st) {
  // one trajectory, unconstrained: the theta rows get their own block rows
  const int rows = !grad ? 1 : (c.R > 1 ? c.W * c.R : (c.csvgd ? c.W : c.W + c.M));
  dim3 grid((N + 255) / 256, rows);
  window_reduce_kernel<<<grid, 256, 0, st>>>(c, X, N, parts, logp, grad, status);
  return cudaGetLastError();
}

}  // namespace pds
