// Posterior metrics on the device (Sec. IV, Eq. knn-kl and the MMD of the
// evaluation): sample sets are device arrays [d][n] (coordinate-major, like
// the particles), d <= 64.
//
//   KNN-KL (after Wang, Kulkarni and Verdu 2009), k_i = l_i = k:
//     D(P || Q) ~ (d / n) sum_i log( nu_k(i) / rho_k(i) ) + log( m / (n - 1) )
//   nu_k(i): Euclidean distance from p_i to its k-th nearest neighbour in Q;
//   rho_k(i): the same in P without p_i (the digamma terms cancel for k = l).
//
//   MMD^2 with k(x, y) = exp(-||x - y||^2 / h), unbiased (Gretton et al. 2012):
//     1/(n(n-1)) sum_{i!=j} k(x_i,x_j) + 1/(m(m-1)) sum_{i!=j} k(y_i,y_j)
//     - 2/(nm) sum_{i,j} k(x_i,y_j).
//
// Both are brute force: one thread per query point, reference points staged
// through shared memory in tiles of 128; the k nearest distances are kept
// sorted in registers (k <= 8); kernel sums accumulate per thread in double.
#include <math.h>

#include "pds_internal.cuh"

namespace pds {

constexpr int kMetTile = 128;
constexpr int kMetMaxK = 8;

template <int DM>
__global__ void __launch_bounds__(kMetTile) knn_kernel(const float* __restrict__ qry, int n, const float* __restrict__ ref,
                                                       int m, int d, int k, int exclude_self,
                                                       float* __restrict__ dist_k) {
  __shared__ float tile[DM][kMetTile];
  const int i = blockIdx.x * kMetTile + threadIdx.x;
  float x[DM];
#pragma unroll
  for (int c = 0; c < DM; ++c) x[c] = (c < d && i < n) ? qry[(size_t)c * n + i] : 0.f;
  float best[kMetMaxK];
#pragma unroll
  for (int b = 0; b < kMetMaxK; ++b) best[b] = INFINITY;
  for (int j0 = 0; j0 < m; j0 += kMetTile) {
    const int jl = j0 + threadIdx.x;
#pragma unroll
    for (int c = 0; c < DM; ++c) tile[c][threadIdx.x] = (c < d && jl < m) ? ref[(size_t)c * m + jl] : 0.f;
    __syncthreads();
    const int jn = min(kMetTile, m - j0);
    for (int jj = 0; jj < jn; ++jj) {
      if (exclude_self && j0 + jj == i) continue;
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < DM; ++c) {
        const float e = x[c] - tile[c][jj];
        s = fmaf(e, e, s);
      }
      if (s < best[kMetMaxK - 1]) {
        // insert into the sorted list of the kMetMaxK smallest
#pragma unroll
        for (int b = kMetMaxK - 1; b > 0; --b) {
          const bool move = s < best[b - 1];
          best[b] = move ? best[b - 1] : (s < best[b] ? s : best[b]);
        }
        best[0] = s < best[0] ? s : best[0];
      }
    }
    __syncthreads();
  }
  if (i < n) {
    float r = best[0];
#pragma unroll
    for (int b = 1; b < kMetMaxK; ++b)
      if (b == k - 1) r = best[b];
    dist_k[i] = sqrtf(r);
  }
}

// sum_i log(nu_i / rho_i) into acc[0] (double); with skip_nonfinite, terms
// that are not finite (a query point that is not finite, or a distance 0)
// are left out.
__global__ void __launch_bounds__(256) knn_log_ratio_kernel(const float* __restrict__ nu, const float* __restrict__ rho,
                                                            int n, double* __restrict__ acc, int skip_nonfinite = 0) {
  __shared__ double part[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = i < n ? log((double)nu[i]) - log((double)rho[i]) : 0.0;
  if (skip_nonfinite && !isfinite(v)) v = 0.0;
  part[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc, part[0]);
}

// sum over pairs (i in A, j in B; i != j when A and B are the same set) of
// exp(-||a_i - b_j||^2 / h) into acc[0] (double).
template <int DM, bool SKIP_NONFINITE = false>
__global__ void __launch_bounds__(kMetTile) rbf_sum_kernel(const float* __restrict__ A, int n, const float* __restrict__ B,
                                                           int m, int d, float inv_h, int same,
                                                           double* __restrict__ acc) {
  __shared__ float tile[DM][kMetTile];
  __shared__ double part[kMetTile];
  const int i = blockIdx.x * kMetTile + threadIdx.x;
  float x[DM];
#pragma unroll
  for (int c = 0; c < DM; ++c) x[c] = (c < d && i < n) ? A[(size_t)c * n + i] : 0.f;
  double s_all = 0.0;
  for (int j0 = 0; j0 < m; j0 += kMetTile) {
    const int jl = j0 + threadIdx.x;
#pragma unroll
    for (int c = 0; c < DM; ++c) tile[c][threadIdx.x] = (c < d && jl < m) ? B[(size_t)c * m + jl] : 0.f;
    __syncthreads();
    const int jn = min(kMetTile, m - j0);
    float s_tile = 0.f;
    for (int jj = 0; jj < jn; ++jj) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < DM; ++c) {
        const float e = x[c] - tile[c][jj];
        s = fmaf(e, e, s);
      }
      const bool skip = (same && (j0 + jj == i)) || (SKIP_NONFINITE && !(s <= INFINITY));
      s_tile += skip ? 0.f : expf(-s * inv_h);
    }
    s_all += (double)s_tile;
    __syncthreads();
  }
  part[threadIdx.x] = i < n ? s_all : 0.0;
  __syncthreads();
  for (int s = kMetTile / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc, part[0]);
}

template <int DM>
static cudaError_t launch_knn(const float* q, int n, const float* r, int m, int d, int k, int self, float* out,
                              cudaStream_t st) {
  knn_kernel<DM><<<(n + kMetTile - 1) / kMetTile, kMetTile, 0, st>>>(q, n, r, m, d, k, self, out);
  return cudaGetLastError();
}

static cudaError_t knn(const float* q, int n, const float* r, int m, int d, int k, int self, float* out,
                       cudaStream_t st) {
  if (d <= 4) return launch_knn<4>(q, n, r, m, d, k, self, out, st);
  if (d <= 16) return launch_knn<16>(q, n, r, m, d, k, self, out, st);
  return launch_knn<64>(q, n, r, m, d, k, self, out, st);
}

template <int DM, bool SKIP>
static cudaError_t launch_rbf(const float* a, int n, const float* b, int m, int d, float inv_h, int same, double* acc,
                              cudaStream_t st) {
  rbf_sum_kernel<DM, SKIP><<<(n + kMetTile - 1) / kMetTile, kMetTile, 0, st>>>(a, n, b, m, d, inv_h, same, acc);
  return cudaGetLastError();
}

template <bool SKIP = false>
static cudaError_t rbf(const float* a, int n, const float* b, int m, int d, float inv_h, int same, double* acc,
                       cudaStream_t st) {
  if (d <= 4) return launch_rbf<4, SKIP>(a, n, b, m, d, inv_h, same, acc, st);
  if (d <= 16) return launch_rbf<16, SKIP>(a, n, b, m, d, inv_h, same, acc, st);
  return launch_rbf<64, SKIP>(a, n, b, m, d, inv_h, same, acc, st);
}

// Asynchronous parts of the metrics for callers inside the library (the
// server's convergence gate), on sets whose points that are not finite
// take no part: acc3 receives the three kernel sums of MMD^2 (xx without
// the diagonal, yy without the diagonal, xy), acc1 the sum of the KNN log
// ratios; the caller divides by the live counts.
cudaError_t mmd2_sums_async(const float* x, int n, const float* y, int m, int d, float inv_h, double* acc3,
                            cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(acc3, 0, 3 * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = rbf<true>(x, n, x, n, d, inv_h, 1, acc3, st)) != cudaSuccess) return e;
  if ((e = rbf<true>(y, m, y, m, d, inv_h, 1, acc3 + 1, st)) != cudaSuccess) return e;
  return rbf<true>(x, n, y, m, d, inv_h, 0, acc3 + 2, st);
}

cudaError_t knn_log_ratio_async(const float* p, int n, const float* q, int m, int d, int k, float* scratch2n,
                                double* acc1, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(acc1, 0, sizeof(double), st)) != cudaSuccess) return e;
  if ((e = knn(p, n, q, m, d, k, 0, scratch2n, st)) != cudaSuccess) return e;
  if ((e = knn(p, n, p, n, d, k, 1, scratch2n + n, st)) != cudaSuccess) return e;
  knn_log_ratio_kernel<<<(n + 255) / 256, 256, 0, st>>>(scratch2n, scratch2n + n, n, acc1, 1);
  return cudaGetLastError();
}

}  // namespace pds

using namespace pds;

extern "C" {

int pds_knn_kl(const float* p, int n, const float* q, int m, int d, int k, double* kl, void* cuda_stream) {
  if (!p || !q || !kl) return set_error(PDS_ERR_ARG, "NULL argument");
  if (d < 1 || d > 64) return set_error(PDS_ERR_ARG, "dimension d outside 1..64");
  if (k < 1 || k > kMetMaxK) return set_error(PDS_ERR_ARG, "k outside 1..8");
  if (n < k + 1 || m < k || n > (1 << 20) || m > (1 << 20)) return set_error(PDS_ERR_ARG, "set sizes too small or large");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float* nu = nullptr;
  double* acc = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&nu, 2 * (size_t)n * sizeof(float), st)) != cudaSuccess)
    return set_error(PDS_ERR_OOM, "knn scratch");
  if ((e = cudaMallocAsync(&acc, sizeof(double), st)) != cudaSuccess) {
    cudaFreeAsync(nu, st);
    return set_error(PDS_ERR_OOM, "knn scratch");
  }
  float* rho = nu + n;
  double h = 0.0;
  if ((e = cudaMemsetAsync(acc, 0, sizeof(double), st)) == cudaSuccess &&
      (e = knn(p, n, q, m, d, k, 0, nu, st)) == cudaSuccess && (e = knn(p, n, p, n, d, k, 1, rho, st)) == cudaSuccess) {
    knn_log_ratio_kernel<<<(n + 255) / 256, 256, 0, st>>>(nu, rho, n, acc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  cudaFreeAsync(nu, st);
  cudaFreeAsync(acc, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, cudaGetErrorString(e));
  *kl = (double)d / n * h + log((double)m / (double)(n - 1));
  set_launch_count(4);
  return PDS_OK;
}

int pds_mmd2(const float* x, int n, const float* y, int m, int d, double h, double* mmd2, void* cuda_stream) {
  if (!x || !y || !mmd2) return set_error(PDS_ERR_ARG, "NULL argument");
  if (d < 1 || d > 64) return set_error(PDS_ERR_ARG, "dimension d outside 1..64");
  if (n < 2 || m < 2 || n > (1 << 20) || m > (1 << 20)) return set_error(PDS_ERR_ARG, "set sizes outside 2..2^20");
  if (!(h > 0.0) || !isfinite(h)) return set_error(PDS_ERR_ARG, "bandwidth h must be finite and > 0");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* acc = nullptr;
  cudaError_t e = cudaMallocAsync(&acc, 3 * sizeof(double), st);
  if (e != cudaSuccess) return set_error(PDS_ERR_OOM, "mmd scratch");
  double s[3] = {0.0, 0.0, 0.0};
  const float inv_h = (float)(1.0 / h);
  if ((e = cudaMemsetAsync(acc, 0, 3 * sizeof(double), st)) == cudaSuccess &&
      (e = rbf(x, n, x, n, d, inv_h, 1, acc, st)) == cudaSuccess &&
      (e = rbf(y, m, y, m, d, inv_h, 1, acc + 1, st)) == cudaSuccess &&
      (e = rbf(x, n, y, m, d, inv_h, 0, acc + 2, st)) == cudaSuccess)
    e = cudaMemcpyAsync(s, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(acc, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, cudaGetErrorString(e));
  *mmd2 = s[0] / ((double)n * (n - 1)) + s[1] / ((double)m * (m - 1)) - 2.0 * s[2] / ((double)n * m);
  set_launch_count(3);
  return PDS_OK;
}

}  // extern "C"
