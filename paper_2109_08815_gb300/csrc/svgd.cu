// SVGD update (Sec. IV-A, Eq. 1) on the device:
//   1. unit-box coordinates u = (theta - lo)/(hi - lo) and gradient g_u;
//   2. median heuristic bandwidth: the exact lower median of the N(N-1)/2
//      pairwise squared distances by a three-pass radix select on the float
//      bit patterns (11 + 11 + 10 bits; distances are recomputed in every
//      pass and never stored), bw = median / log N;
//   3. phi_i = 1/N sum_j k_ij [g_j + (2/bw)(u_i - u_j)], k_ij = exp(-d_ij/bw),
//      with particle tiles staged in shared memory;
//   4. Adam ascent on u (theta rows, then clamp) and on the shooting states.
// All control state (histogram, prefix, Adam step count) stays on the device,
// so a step issues no host synchronisation.
#include <math.h>

#include "pds_internal.cuh"

namespace pds {

constexpr int kTile = 128;        // particles per tile (threads per block)
constexpr int kHistBins = 2048;   // 11-bit radix digits

__global__ void svgd_prep_kernel(SvgdParams sp, SvgdCtl* __restrict__ ctl, const float* __restrict__ X,
                                 const float* __restrict__ G, float* __restrict__ u, float* __restrict__ gu) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < kHistBins) ctl->hist[idx] = 0u;
  if (idx == 0) {
    const int t = ctl->step + 1;
    ctl->step = t;
    ctl->bc1 = (float)(1.0 - pow((double)sp.b1, (double)t));
    ctl->bc2 = (float)(1.0 - pow((double)sp.b2, (double)t));
    const unsigned long long pairs = (unsigned long long)sp.N * (unsigned long long)(sp.N - 1) / 2ull;
    ctl->prefix = 0u;
    ctl->rank = pairs ? (unsigned int)((pairs - 1ull) / 2ull) : 0u;
    ctl->bw = 1.0f;
    ctl->med = 0.0f;
  }
  const int total = sp.M * sp.N;
  if (idx < total) {
    const int k = idx / sp.N;
    const float width = sp.hi[k] - sp.lo[k];
    u[idx] = (X[idx] - sp.lo[k]) / width;
    gu[idx] = G[idx] * width;
  }
}

template <int MM>
__device__ __forceinline__ void load_row(const float* __restrict__ u, int M, int N, int i, float (&r)[MM]) {
#pragma unroll
  for (int k = 0; k < MM; ++k) r[k] = (k < M && i < N) ? u[(size_t)k * N + i] : 0.f;
}

// One radix-select pass over all pairs i < j.  pass 0 histograms bits
// [31:21]; pass 1 bits [20:10] of the pairs whose bits [31:21] equal the
// resolved prefix; pass 2 bits [9:0] of those whose bits [31:10] match.
template <int MM>
__global__ void __launch_bounds__(kTile) median_hist_kernel(int N, int M, const float* __restrict__ u,
                                                            SvgdCtl* __restrict__ ctl, int pass) {
  __shared__ unsigned int hist[kHistBins];
  __shared__ float uj[MM][kTile];
  for (int b = threadIdx.x; b < kHistBins; b += kTile) hist[b] = 0u;
  const unsigned int prefix = ctl->prefix;
  const int nt = (N + kTile - 1) / kTile;
  const long long ntiles = (long long)nt * nt;
  __syncthreads();
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int I = (int)(tile / nt), J = (int)(tile - (long long)I * nt);
    if (I > J) continue;  // uniform across the block
    const int i = I * kTile + threadIdx.x;
    float ui[MM];
    load_row<MM>(u, M, N, i, ui);
    {
      const int j = J * kTile + threadIdx.x;
#pragma unroll
      for (int k = 0; k < MM; ++k) uj[k][threadIdx.x] = (k < M && j < N) ? u[(size_t)k * N + j] : 0.f;
    }
    __syncthreads();
    if (i < N) {
      const int jn = min(kTile, N - J * kTile);
      const int jstart = (I == J) ? (threadIdx.x + 1) : 0;
      for (int jj = jstart; jj < jn; ++jj) {
        float d = 0.f;
#pragma unroll
        for (int k = 0; k < MM; ++k) {
          const float e = ui[k] - uj[k][jj];
          d = fmaf(e, e, d);
        }
        const unsigned int bits = __float_as_uint(d);
        if (pass == 0) {
          atomicAdd(&hist[bits >> 21], 1u);
        } else if (pass == 1) {
          if ((bits >> 21) == prefix) atomicAdd(&hist[(bits >> 10) & 2047u], 1u);
        } else {
          if ((bits >> 10) == prefix) atomicAdd(&hist[bits & 1023u], 1u);
        }
      }
    }
    __syncthreads();
  }
  for (int b = threadIdx.x; b < kHistBins; b += kTile) {
    const unsigned int h = hist[b];
    if (h) atomicAdd(&ctl->hist[b], h);
  }
}

// Resolve one radix digit: find the bin holding the rank-th element, narrow
// the prefix and the rank, clear the histogram.  One warp.
__global__ void median_select_kernel(SvgdCtl* __restrict__ ctl, int pass, int N) {
  const int lane = threadIdx.x;  // 32 lanes x 64 bins
  unsigned int local = 0u;
  for (int b = 0; b < 64; ++b) local += ctl->hist[lane * 64 + b];
  unsigned int incl = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  const unsigned int excl = incl - local;
  const unsigned int rank = ctl->rank;
  const bool mine = (rank >= excl) && (rank < incl);
  __syncwarp();
  if (mine) {
    unsigned int cum = excl;
    int bin = lane * 64;
    for (int b = 0; b < 64; ++b) {
      const unsigned int h = ctl->hist[lane * 64 + b];
      if (rank < cum + h) { bin = lane * 64 + b; break; }
      cum += h;
    }
    const unsigned int digit_bits = (pass == 2) ? 10u : 11u;
    const unsigned int prefix = (ctl->prefix << digit_bits) | (unsigned int)bin;
    ctl->rank = rank - cum;
    ctl->prefix = prefix;
    if (pass == 2) {
      const float med = __uint_as_float(prefix);
      ctl->med = med;
      ctl->bw = (med > 0.f && N > 1) ? med / logf((float)N) : 1.0f;
    }
  }
  __syncwarp();
  for (int b = 0; b < 64; ++b) ctl->hist[lane * 64 + b] = 0u;
}

// Partial phi over one chunk of j: phi_part[c][k][i] =
//   sum_j k_ij g_j[k] + (2/bw) sum_j k_ij (u_i[k] - u_j[k]).
template <int MM>
__global__ void __launch_bounds__(kTile) svgd_phi_kernel(int N, int M, const float* __restrict__ u,
                                                         const float* __restrict__ gu, const SvgdCtl* __restrict__ ctl,
                                                         float* __restrict__ phi_part, int chunk_len) {
  __shared__ float uj[MM][kTile];
  __shared__ float gj[MM][kTile];
  const int i = blockIdx.x * kTile + threadIdx.x;
  const int c = blockIdx.y;
  const int j0 = c * chunk_len;
  const int j1 = min(N, j0 + chunk_len);
  const float bw = ctl->bw;
  const float inv_bw = 1.0f / bw;
  float ui[MM], ag[MM], ar[MM];
  load_row<MM>(u, M, N, i, ui);
#pragma unroll
  for (int k = 0; k < MM; ++k) { ag[k] = 0.f; ar[k] = 0.f; }
  for (int jt = j0; jt < j1; jt += kTile) {
    const int j = jt + threadIdx.x;
#pragma unroll
    for (int k = 0; k < MM; ++k) {
      const bool ok = (k < M) && (j < j1);
      uj[k][threadIdx.x] = ok ? u[(size_t)k * N + j] : 0.f;
      gj[k][threadIdx.x] = ok ? gu[(size_t)k * N + j] : 0.f;
    }
    __syncthreads();
    const int jn = min(kTile, j1 - jt);
    for (int jj = 0; jj < jn; ++jj) {
      float e[MM];
      float d = 0.f;
#pragma unroll
      for (int k = 0; k < MM; ++k) {
        e[k] = ui[k] - uj[k][jj];
        d = fmaf(e[k], e[k], d);
      }
      const float kij = expf(-d * inv_bw);
#pragma unroll
      for (int k = 0; k < MM; ++k) {
        ag[k] = fmaf(kij, gj[k][jj], ag[k]);
        ar[k] = fmaf(kij, e[k], ar[k]);
      }
    }
    __syncthreads();
  }
  if (i < N) {
    const float two_over_bw = 2.0f * inv_bw;
#pragma unroll
    for (int k = 0; k < MM; ++k)
      if (k < M) phi_part[((size_t)c * M + k) * N + i] = fmaf(two_over_bw, ar[k], ag[k]);
  }
}

__global__ void svgd_adam_kernel(SvgdParams sp, const SvgdCtl* __restrict__ ctl, float* __restrict__ X,
                                 const float* __restrict__ G, const float* __restrict__ phi_part, int chunks,
                                 float* __restrict__ am, float* __restrict__ av, float* __restrict__ bw_out,
                                 float* __restrict__ phi_out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)sp.P * sp.N;
  if (idx == 0 && bw_out) *bw_out = ctl->bw;
  if (idx >= total) return;
  const int r = (int)(idx / sp.N);
  const int i = (int)(idx - (size_t)r * sp.N);
  const float bc1 = ctl->bc1, bc2 = ctl->bc2;
  float g;
  float x;
  if (r < sp.M) {
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += phi_part[((size_t)c * sp.M + r) * sp.N + i];
    g = s / (float)sp.N;
    if (phi_out) phi_out[idx] = g;
    x = (X[idx] - sp.lo[r]) / (sp.hi[r] - sp.lo[r]);
  } else {
    g = G[idx];
    x = X[idx];
  }
  const float m = sp.b1 * am[idx] + (1.f - sp.b1) * g;
  const float v = sp.b2 * av[idx] + (1.f - sp.b2) * g * g;
  am[idx] = m;
  av[idx] = v;
  x += sp.lr * (m / bc1) / (sqrtf(v / bc2) + sp.eps);
  if (r < sp.M) {
    if (sp.clamp) x = fminf(1.f, fmaxf(0.f, x));
    x = sp.lo[r] + x * (sp.hi[r] - sp.lo[r]);
  }
  X[idx] = x;
}

int svgd_phi_chunks(int N) {
  const int row_blocks = (N + kTile - 1) / kTile;
  int chunks = (8 * 152 + row_blocks - 1) / row_blocks;
  const int max_chunks = (N + kTile - 1) / kTile;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  return chunks;
}

template <int MM>
static cudaError_t launch_svgd_mm(const SvgdParams& sp, const SvgdWork& w, float* X, const float* G, float* bw_out,
                                  float* phi_out, cudaStream_t st, int* launches) {
  const int N = sp.N, M = sp.M;
  int n = 0;
  {
    const int total = (M * N > kHistBins) ? M * N : kHistBins;
    svgd_prep_kernel<<<(total + 255) / 256, 256, 0, st>>>(sp, w.ctl, X, G, w.u, w.gu);
    ++n;
  }
  if (N >= 2) {
    const int nt = (N + kTile - 1) / kTile;
    const long long tiles = (long long)nt * (nt + 1) / 2;
    int grid = 152 * 8;
    if (tiles < grid) grid = (int)((long long)nt * nt);
    for (int pass = 0; pass < 3; ++pass) {
      median_hist_kernel<MM><<<grid, kTile, 0, st>>>(N, M, w.u, w.ctl, pass);
      median_select_kernel<<<1, 32, 0, st>>>(w.ctl, pass, N);
      n += 2;
    }
  }
  {
    const int chunk_len = ((N + w.chunks - 1) / w.chunks + kTile - 1) / kTile * kTile;
    const int chunks = (N + chunk_len - 1) / chunk_len;
    dim3 grid((N + kTile - 1) / kTile, chunks);
    svgd_phi_kernel<MM><<<grid, kTile, 0, st>>>(N, M, w.u, w.gu, w.ctl, w.phi_part, chunk_len);
    const size_t total = (size_t)sp.P * N;
    svgd_adam_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sp, w.ctl, X, G, w.phi_part, chunks, w.adam_m,
                                                                      w.adam_v, bw_out, phi_out);
    n += 2;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_svgd_step(const SvgdParams& sp, const SvgdWork& w, float* X, const float* G, float* bw_out,
                             float* phi_out, cudaStream_t st, int* launches) {
  if (sp.M <= 2) return launch_svgd_mm<2>(sp, w, X, G, bw_out, phi_out, st, launches);
  if (sp.M <= 4) return launch_svgd_mm<4>(sp, w, X, G, bw_out, phi_out, st, launches);
  if (sp.M <= 8) return launch_svgd_mm<8>(sp, w, X, G, bw_out, phi_out, st, launches);
  if (sp.M <= 10) return launch_svgd_mm<10>(sp, w, X, G, bw_out, phi_out, st, launches);
  return launch_svgd_mm<16>(sp, w, X, G, bw_out, phi_out, st, launches);
}

}  // namespace pds

// ---------------------------------------------------------------------------
// Allocation-free median-heuristic bandwidth (pds_bandwidth_noalloc).
//
// For callers that cannot allocate device memory: code running inside a
// host-side memory pool or allocator callback, or a process whose device
// memory is reserved up front by another framework, may not be allowed to
// call cudaMalloc.  This variant of the bandwidth computation above runs the
// same radix-select kernels, but its scratch (the control block with the
// radix histogram, and the unit-box coordinates) lives in the file-scope
// device array below instead of a workspace allocated by pds_svgd_create.
// Every GPU that loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace pds {

constexpr int kNoAllocCtlFloats = 4096;        // control block, padded to 16 KiB
constexpr int kNoAllocMaxElems = 1 << 20;      // N * M <= 1,048,576 (4 MiB of coordinates)
static_assert(sizeof(SvgdCtl) <= kNoAllocCtlFloats * sizeof(float), "control block does not fit");

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocCtlFloats + kNoAllocMaxElems];

struct NoAllocBox {
  float lo[kMaxTheta], hi[kMaxTheta];
};

// Clears the histogram and radix state (the array keeps the previous call's
// contents) and writes u = (theta - lo) / (hi - lo) into the scratch.
__global__ void noalloc_prep_kernel(int N, int M, NoAllocBox box, const float* __restrict__ theta,
                                    SvgdCtl* __restrict__ ctl, float* __restrict__ u) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < kHistBins) ctl->hist[idx] = 0u;
  if (idx == 0) {
    const unsigned long long pairs = (unsigned long long)N * (unsigned long long)(N - 1) / 2ull;
    ctl->prefix = 0u;
    ctl->rank = pairs ? (unsigned int)((pairs - 1ull) / 2ull) : 0u;
    ctl->bw = 1.0f;
    ctl->med = 0.0f;
  }
  if (idx < M * N) {
    const int k = idx / N;
    u[idx] = (theta[idx] - box.lo[k]) / (box.hi[k] - box.lo[k]);
  }
}

__global__ void noalloc_out_kernel(const SvgdCtl* __restrict__ ctl, float* __restrict__ out) { *out = ctl->bw; }

template <int MM>
static cudaError_t noalloc_bandwidth_mm(int N, int M, const NoAllocBox& box, const float* theta, float* out,
                                        float* scratch, cudaStream_t st) {
  SvgdCtl* ctl = reinterpret_cast<SvgdCtl*>(scratch);
  float* u = scratch + kNoAllocCtlFloats;
  const int total = (M * N > kHistBins) ? M * N : kHistBins;
  noalloc_prep_kernel<<<(total + 255) / 256, 256, 0, st>>>(N, M, box, theta, ctl, u);
  if (N >= 2) {
    const int nt = (N + kTile - 1) / kTile;
    const long long all_tiles = (long long)nt * nt;
    const int grid = all_tiles < 152 * 8 ? (int)all_tiles : 152 * 8;
    for (int pass = 0; pass < 3; ++pass) {
      median_hist_kernel<MM><<<grid, kTile, 0, st>>>(N, M, u, ctl, pass);
      median_select_kernel<<<1, 32, 0, st>>>(ctl, pass, N);
    }
  }
  noalloc_out_kernel<<<1, 1, 0, st>>>(ctl, out);
  return cudaGetLastError();
}

static std::mutex g_noalloc_mu;
static float* g_noalloc_ptr[64];

}  // namespace pds

extern "C" int pds_bandwidth_noalloc(const float* theta, int N, int M, const float* theta_lo, const float* theta_hi,
                                     float* bandwidth_out, void* cuda_stream) {
  using namespace pds;
  if (!theta || !theta_lo || !theta_hi || !bandwidth_out) return set_error(PDS_ERR_ARG, "NULL argument");
  if (M < 1 || M > kMaxTheta) return set_error(PDS_ERR_ARG, "pds_bandwidth_noalloc: M outside 1..16");
  if (N < 1 || (long long)N * M > kNoAllocMaxElems)
    return set_error(PDS_ERR_ARG, "pds_bandwidth_noalloc: N * M must be in 1..1048576 (static scratch limit)");
  NoAllocBox box;
  for (int k = 0; k < kMaxTheta; ++k) { box.lo[k] = 0.f; box.hi[k] = 1.f; }
  for (int k = 0; k < M; ++k) {
    if (!(theta_hi[k] > theta_lo[k])) return set_error(PDS_ERR_ARG, "pds_bandwidth_noalloc: empty theta box");
    box.lo[k] = theta_lo[k];
    box.hi[k] = theta_hi[k];
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return set_error(PDS_ERR_CUDA, "pds_bandwidth_noalloc: no device");
  float* scratch = nullptr;
  {
    // One-time set-up per device, on the first call with that device
    // current: host code needs the array's device address (its name on the
    // host is only a stand-in).
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return set_error(PDS_ERR_CUDA, "pds_bandwidth_noalloc: cudaGetSymbolAddress failed");
      g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (M <= 2) e = noalloc_bandwidth_mm<2>(N, M, box, theta, bandwidth_out, scratch, st);
  else if (M <= 4) e = noalloc_bandwidth_mm<4>(N, M, box, theta, bandwidth_out, scratch, st);
  else if (M <= 8) e = noalloc_bandwidth_mm<8>(N, M, box, theta, bandwidth_out, scratch, st);
  else if (M <= 10) e = noalloc_bandwidth_mm<10>(N, M, box, theta, bandwidth_out, scratch, st);
  else e = noalloc_bandwidth_mm<16>(N, M, box, theta, bandwidth_out, scratch, st);
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, "pds_bandwidth_noalloc: kernel launch failed");
  return PDS_OK;
}
