// Sobol initialisation of the particles (App. A-A: the estimators start from
// the deterministic Sobol sequence over the parameter limits).
//
// Dimension k of point n is x_k(n) = XOR of the direction numbers v_k[j] over
// the set bits j of the Gray code n ^ (n >> 1), as a 32-bit binary fraction
// (Antonov and Saleev's Gray-code ordering of Sobol's construction), so that
// point 0 is the origin and every point is computed on its own.  Direction
// numbers: dimension 1 has v[j] = 2^(31-j); dimension d >= 2 has a primitive
// polynomial of degree s with coefficients a and initial odd integers
// m_1..m_s, v[j] = m_{j+1} 2^(31-j) for j < s and
//   v[j] = v[j-s] ^ (v[j-s] >> s) ^ XOR_{k=1}^{s-1} a_k v[j-k]   (j >= s),
// a_k the k-th coefficient bit of a (Bratley and Fox 1988).  The (s, a, m)
// values are those of Joe and Kuo (2008), dimensions 2..16.
//
// theta_k = lo_k + x_k (hi_k - lo_k) in fp32.  For indices below 2^24 every
// x_k has at most 24 significant bits and converts to fp32 exactly.
#include <stdint.h>

#include "pds_internal.cuh"

namespace pds {

namespace {

struct SobolPoly {
  int s, a;
  int m[6];
};

// Dimensions 2..16: degree s, coefficient bits a, initial direction integers m.
constexpr SobolPoly kSobolPolys[kMaxTheta - 1] = {
    {1, 0, {1}},
    {2, 1, {1, 3}},
    {3, 1, {1, 3, 1}},
    {3, 2, {1, 1, 1}},
    {4, 1, {1, 1, 3, 3}},
    {4, 4, {1, 3, 5, 13}},
    {5, 2, {1, 1, 5, 5, 17}},
    {5, 4, {1, 1, 5, 5, 5}},
    {5, 7, {1, 1, 7, 11, 19}},
    {5, 11, {1, 1, 5, 1, 1}},
    {5, 13, {1, 1, 1, 3, 11}},
    {5, 14, {1, 3, 5, 5, 31}},
    {6, 1, {1, 3, 3, 9, 7, 49}},
    {6, 13, {1, 1, 1, 15, 21, 21}},
    {6, 16, {1, 3, 1, 13, 27, 49}},
};

struct SobolArgs {
  uint32_t v[kMaxTheta][32];
  float lo[kMaxTheta];
  float w[kMaxTheta];
  uint32_t skip;
  int N, M;
};

void direction_numbers(int dim, uint32_t v[32]) {
  if (dim == 0) {
    for (int j = 0; j < 32; ++j) v[j] = 1u << (31 - j);
    return;
  }
  const SobolPoly& p = kSobolPolys[dim - 1];
  for (int j = 0; j < 32; ++j) {
    if (j < p.s) {
      v[j] = (uint32_t)p.m[j] << (31 - j);
    } else {
      uint32_t x = v[j - p.s] ^ (v[j - p.s] >> p.s);
      for (int k = 1; k < p.s; ++k)
        if ((p.a >> (p.s - 1 - k)) & 1) x ^= v[j - k];
      v[j] = x;
    }
  }
}

}  // namespace

// blockIdx.y = dimension k, x over particles.
__global__ void __launch_bounds__(256) sobol_box_kernel(SobolArgs A, float* __restrict__ theta) {
  const int k = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const uint32_t n = A.skip + (uint32_t)i;
  const uint32_t g = n ^ (n >> 1);
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if ((g >> j) & 1u) x ^= A.v[k][j];
  const float u = (float)x * 0x1p-32f;
  theta[(size_t)k * A.N + i] = fmaf(u, A.w[k], A.lo[k]);
}

}  // namespace pds

using namespace pds;

extern "C" {

int pds_sobol_box(float* theta, int N, int M, const float* theta_lo, const float* theta_hi, long long skip,
                  void* cuda_stream) {
  if (!theta || !theta_lo || !theta_hi) return set_error(PDS_ERR_ARG, "NULL argument");
  if (N < 1 || N > (1 << 24)) return set_error(PDS_ERR_ARG, "pds_sobol_box: N outside 1..2^24");
  if (M < 1 || M > kMaxTheta) return set_error(PDS_ERR_ARG, "pds_sobol_box: M outside 1..16");
  if (skip < 0 || skip + (long long)N > (1ll << 32))
    return set_error(PDS_ERR_ARG, "pds_sobol_box: point indices must lie in 0..2^32-1");
  SobolArgs A{};
  for (int k = 0; k < M; ++k) {
    if (!(theta_hi[k] > theta_lo[k])) return set_error(PDS_ERR_ARG, "pds_sobol_box: empty theta box");
    direction_numbers(k, A.v[k]);
    A.lo[k] = theta_lo[k];
    A.w[k] = theta_hi[k] - theta_lo[k];
  }
  A.skip = (uint32_t)skip;
  A.N = N;
  A.M = M;
  const dim3 grid((N + 255) / 256, M);
  sobol_box_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(A, theta);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, cudaGetErrorString(e));
  set_launch_count(1);
  return PDS_OK;
}

}  // extern "C"
