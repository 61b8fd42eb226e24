// Stochastic gradient Langevin dynamics (Welling and Teh 2011), the second
// estimator the paper runs on the multiple-shooting likelihood (Sec. V-B):
// every particle is an independent chain on the augmented vector
//   u   <- u + (eps_t / 2) g_u + sqrt(eps_t) xi          (theta rows, u = (theta - lo) / (hi - lo))
//   s^s <- s^s + (eps_t / 2) g   + sqrt(eps_t) xi          (shooting rows)
//   eps_t = a (b + t)^(-gamma),  t = 1, 2, ...
// with g_u = (hi - lo) d log p / d theta.  xi ~ N(0, 1) is drawn per
// (step, row, particle) from a counter-based generator: SplitMix64 (Steele,
// Lea and Flood 2014) outputs 2k + 1 and 2k + 2 from the seed, with
// k = (t - 1) P N + r N + i, turned into one normal by the Box-Muller
// transform (u1 = (top 53 bits + 1) 2^-53 in (0, 1], u2 = top 53 bits 2^-53
// in [0, 1): sqrt(-2 ln u1) cos(2 pi u2)).  Any step of any chain can thus be
// redrawn without state, and the draws do not depend on the launch shape.
//
// The update is one elementwise pass over the [P][N] particle array: 8 bytes
// read and 4 written per element, plus two 64-bit hashes, a logarithm, a
// square root and a cosine.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "pds_internal.cuh"

namespace pds {

struct SgldArgs {
  float lo[kMaxTheta];
  float w[kMaxTheta];
  int N, M, P, clamp;
  float half_eps, sqrt_eps;
  unsigned long long seed, kbase;
};

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t index) {
  uint64_t z = seed + index * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Standard normal number k of the stream `seed`, in fp32.  ln u1 is taken as
// log1p(-(1 - u1)) when u1 > 1/2, where 1 - u1 is formed exactly in integers,
// so that draws near u1 = 1 keep their relative accuracy.
__device__ __forceinline__ float langevin_normal(uint64_t seed, uint64_t k) {
  const uint64_t a = splitmix64_at(seed, 2 * k + 1) >> 11;  // u1 = (a + 1) 2^-53
  const uint64_t b = splitmix64_at(seed, 2 * k + 2) >> 11;  // u2 = b 2^-53
  float ln_u1;
  if (a >= (1ull << 52))
    ln_u1 = log1pf(-(float)((1ull << 53) - 1 - a) * 0x1p-53f);
  else
    ln_u1 = logf((float)(a + 1) * 0x1p-53f);
  const float r = sqrtf(-2.f * ln_u1);
  return r * cospif((float)b * 0x1p-52f);  // cos(2 pi u2)
}

// blockIdx.y = row r, x over particles.
__global__ void __launch_bounds__(256) sgld_kernel(SgldArgs A, float* __restrict__ X, const float* __restrict__ G) {
  const int r = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const size_t idx = (size_t)r * A.N + i;
  const float xi = langevin_normal(A.seed, A.kbase + idx);
  const float g = G[idx];
  float x = X[idx];
  if (r < A.M) {
    const float lo = A.lo[r], w = A.w[r];
    float u = (x - lo) / w;
    u += A.half_eps * g * w + A.sqrt_eps * xi;
    if (A.clamp) u = fminf(1.f, fmaxf(0.f, u));
    x = lo + u * w;
  } else {
    x += A.half_eps * g + A.sqrt_eps * xi;
  }
  X[idx] = x;
}

}  // namespace pds

struct pds_sgld {
  pds::SgldArgs args;
  double a, b, gamma;
  long long t = 0;
  cudaStream_t stream;
};

using namespace pds;

extern "C" {

int pds_sgld_create(int N, int M, int P, const float* theta_lo, const float* theta_hi, double a, double b,
                    double gamma, unsigned long long seed, int clamp, void* cuda_stream, pds_sgld_t* out) {
  if (!out) return set_error(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (N < 1 || N > 65536) return set_error(PDS_ERR_ARG, "pds_sgld_create: N outside 1..65536");
  if (M < 0 || M > kMaxTheta || P < M || P < 1 || P > 65535)
    return set_error(PDS_ERR_ARG, "pds_sgld_create: need 0 <= M <= 16, M <= P, 1 <= P <= 65535");
  if (M > 0 && (!theta_lo || !theta_hi)) return set_error(PDS_ERR_ARG, "pds_sgld_create: NULL box");
  if (!(a > 0.0) || !isfinite(a) || !isfinite(b) || !(gamma >= 0.0) || !isfinite(gamma) || !(b + 1.0 > 0.0))
    return set_error(PDS_ERR_ARG, "pds_sgld_create: need a > 0, gamma >= 0, b > -1 (finite)");
  pds_sgld* s = new pds_sgld();
  memset(&s->args, 0, sizeof(s->args));
  for (int k = 0; k < M; ++k) {
    if (!(theta_hi[k] > theta_lo[k])) {
      delete s;
      return set_error(PDS_ERR_ARG, "pds_sgld_create: empty theta box");
    }
    s->args.lo[k] = theta_lo[k];
    s->args.w[k] = theta_hi[k] - theta_lo[k];
  }
  s->args.N = N;
  s->args.M = M;
  s->args.P = P;
  s->args.clamp = clamp ? 1 : 0;
  s->args.seed = seed;
  s->a = a;
  s->b = b;
  s->gamma = gamma;
  s->stream = (cudaStream_t)cuda_stream;
  *out = s;
  return PDS_OK;
}

int pds_sgld_destroy(pds_sgld_t s) {
  delete s;
  return PDS_OK;
}

int pds_sgld_reset(pds_sgld_t s) {
  if (!s) return set_error(PDS_ERR_ARG, "NULL handle");
  s->t = 0;
  return PDS_OK;
}

int pds_sgld_step(pds_sgld_t s, float* particles, const float* grad, float* eps_out) {
  if (!s || !particles || !grad) return set_error(PDS_ERR_ARG, "NULL argument");
  const long long t = s->t + 1;
  const double eps = s->a * pow(s->b + (double)t, -s->gamma);
  if (!(eps > 0.0) || !isfinite(eps)) return set_error(PDS_ERR_ARG, "pds_sgld_step: step size not finite and > 0");
  SgldArgs A = s->args;
  A.half_eps = (float)(0.5 * eps);
  A.sqrt_eps = (float)sqrt(eps);
  A.kbase = (unsigned long long)(t - 1) * (unsigned long long)A.P * (unsigned long long)A.N;
  const dim3 grid((A.N + 255) / 256, A.P);
  sgld_kernel<<<grid, 256, 0, s->stream>>>(A, particles, grad);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, cudaGetErrorString(e));
  s->t = t;
  if (eps_out) *eps_out = (float)eps;
  set_launch_count(1);
  return PDS_OK;
}

}  // extern "C"
