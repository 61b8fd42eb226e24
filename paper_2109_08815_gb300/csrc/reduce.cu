// Window reduction and parameter-limit prior (Sec. IV-C Eq. 5 as a sum of
// logs over windows, Sec. IV-D prior), one thread per particle, fixed
// summation order over windows (deterministic).
#include <math.h>

#include "pds_internal.cuh"

namespace pds {

__global__ void __launch_bounds__(256) window_reduce_kernel(const ChainParams c, const float* __restrict__ X, int N,
                                                            Partials parts, float* __restrict__ logp,
                                                            float* __restrict__ grad, int32_t* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  bool finite = true;
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
    if (grad) {
      float g = 0.f;
      for (int w = 0; w < c.W; ++w) g += parts.th[((size_t)w * c.M + k) * N + i];
      g += c.c_lim * (cu - uk) / width;
      finite = finite && isfinite(g);
      grad[(size_t)k * N + i] = g;
    }
  }
  lp += (double)c.lim_const - 0.5 * (double)c.c_lim * (double)pen;
  const float lpf = (float)lp;
  finite = finite && isfinite(lpf);
  logp[i] = lpf;
  if (grad) {
    const int S = c.S;
    for (int w = 1; w < c.W; ++w) {
      for (int s = 0; s < S; ++s) {
        const float g = parts.start[((size_t)w * S + s) * N + i] + parts.next[((size_t)(w - 1) * S + s) * N + i];
        finite = finite && isfinite(g);
        grad[((size_t)c.M + (size_t)(w - 1) * S + s) * N + i] = g;
      }
    }
  }
  if (status) status[i] = finite ? 0 : 1;
}

cudaError_t launch_window_reduce(const ChainParams& c, const float* X, int N, const Partials& parts, float* logp,
                                 float* grad, int32_t* status, cudaStream_t st) {
  window_reduce_kernel<<<(N + 255) / 256, 256, 0, st>>>(c, X, N, parts, logp, grad, status);
  return cudaGetLastError();
}

}  // namespace pds
