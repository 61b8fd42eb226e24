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

// Start of a step: the control block, u = (theta - lo) / (hi - lo), and
// (G != NULL) the gradient in u coordinates with its per-component maximum.
// A split step passes G = NULL here and computes the gradient's part in
// svgd_grad_live_kernel.
__global__ void svgd_prep_kernel(SvgdParams sp, SvgdCtl* __restrict__ ctl, const float* __restrict__ X,
                                 const float* __restrict__ G, float* __restrict__ u, float* __restrict__ gu,
                                 int mode) {
  PDS_PDL_ENTRY();
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
    ctl->below = 0ull;
    ctl->inside = 0ull;
    ctl->mode = mode;
    ctl->n_live = 0u;
    ctl->live_blocks = 0u;
    ctl->tc_error = 0;
    ctl->gdead = 0u;
    ctl->gblocks = 0u;
  }
  const int total = sp.M * sp.N;
  const int k = idx < total ? idx / sp.N : -1;
  if (idx < total) u[idx] = (X[idx] - sp.lo[k]) / (sp.hi[k] - sp.lo[k]);
  if (!G) return;
  unsigned int gbits = 0u;
  if (idx < total) {
    const float g = G[idx] * (sp.hi[k] - sp.lo[k]);
    gu[idx] = g;
    if (isfinite(g)) gbits = __float_as_uint(fabsf(g));  // particles that are not finite sit out
  }
  // per-component max |g_u| (scales of the fp16 second product of the
  // tensor-core phi); one atomic per warp when the warp holds one component
  const int k0 = __shfl_sync(0xffffffffu, k, 0);
  if (__all_sync(0xffffffffu, k == k0)) {
    const unsigned int m = __reduce_max_sync(0xffffffffu, gbits);
    if ((threadIdx.x & 31) == 0 && k0 >= 0 && m) atomicMax(&ctl->gmax[k0], m);
  } else if (k >= 0 && gbits) {
    atomicMax(&ctl->gmax[k], gbits);
  }
}

// Liveness of each particle (gu = NULL: of its coordinates only, the first
// phase of a split step): a particle whose unit-box coordinates or
// gradient are not all finite sits out this step (its coordinates in u become
// NaN, so it takes no part in the median's pairs or in the other particles'
// kernel sums, and its own direction is NaN).  Counts the live particles;
// the last block sets the median's rank over the live pairs.
__global__ void __launch_bounds__(256) svgd_live_kernel(int N, int M, SvgdCtl* __restrict__ ctl,
                                                        float* __restrict__ u, const float* __restrict__ gu) {
  PDS_PDL_ENTRY();
  __shared__ unsigned int blk;
  __shared__ bool last;
  if (threadIdx.x == 0) blk = 0u;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    // all loads issued together: accumulate without short-circuiting
    bool live = true;
    for (int k = 0; k < M; ++k) live &= isfinite(u[(size_t)k * N + i]) & (!gu || isfinite(gu[(size_t)k * N + i]));
    if (live) atomicAdd(&blk, 1u);
    else
      for (int k = 0; k < M; ++k) u[(size_t)k * N + i] = __int_as_float(0x7fc00000);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (blk) atomicAdd(&ctl->n_live, blk);
    __threadfence();
    last = atomicAdd(&ctl->live_blocks, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long nl = atomicAdd(&ctl->n_live, 0u);
    const unsigned long long pairs = nl * (nl > 0 ? nl - 1ull : 0ull) / 2ull;
    ctl->rank = pairs ? (unsigned int)((pairs - 1ull) / 2ull) : 0u;
  }
}

// Second phase of a split step: the gradient in u coordinates and its
// per-component maximum, and the particles whose coordinates are finite (so
// the first phase's median counted them) but whose gradient is not.  They
// sit out as in svgd_live_kernel; if there are any, the last block takes
// them out of the live count, sets the median's rank over the remaining
// pairs and the full radix passes (mode 1) to compute it again, exactly.
__global__ void __launch_bounds__(256) svgd_grad_live_kernel(SvgdParams sp, SvgdCtl* __restrict__ ctl,
                                                             const float* __restrict__ G, float* __restrict__ u,
                                                             float* __restrict__ gu, int* __restrict__ status) {
  PDS_PDL_ENTRY();
  __shared__ unsigned int blk;
  __shared__ bool last;
  __shared__ unsigned int wmax[8][16];  // per warp and component: max |g_u| bits
  if (threadIdx.x == 0) blk = 0u;
  __syncthreads();
  const int N = sp.N, M = sp.M;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int wid = threadIdx.x >> 5;
  const bool in = i < N;
  bool ufin = in, gfin = in;
  for (int k = 0; k < M; ++k) {
    float g = 0.f;
    if (in) {
      g = G[(size_t)k * N + i] * (sp.hi[k] - sp.lo[k]);
      gu[(size_t)k * N + i] = g;
      gfin &= isfinite(g);
      ufin &= isfinite(u[(size_t)k * N + i]);
    }
    const unsigned int bits = (in && isfinite(g)) ? __float_as_uint(fabsf(g)) : 0u;
    const unsigned int m = __reduce_max_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0) wmax[wid][k] = m;
  }
  __syncthreads();
  // one atomic per block and component
  if (threadIdx.x < M) {
    unsigned int m = 0u;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = max(m, wmax[q][threadIdx.x]);
    if (m) atomicMax(&ctl->gmax[threadIdx.x], m);
  }
  if (ufin && !gfin) {
    for (int k = 0; k < M; ++k) u[(size_t)k * N + i] = __int_as_float(0x7fc00000);
    atomicAdd(&blk, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (blk) atomicAdd(&ctl->gdead, blk);
    __threadfence();
    last = atomicAdd(&ctl->gblocks, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const unsigned int dead = atomicAdd(&ctl->gdead, 0u);
  if (!dead) return;
  for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) ctl->hist[b] = 0u;
  if (threadIdx.x == 0) {
    const unsigned long long nl = ctl->n_live - dead;
    const unsigned long long pairs = nl * (nl > 0 ? nl - 1ull : 0ull) / 2ull;
    ctl->n_live = (unsigned int)nl;
    ctl->rank = pairs ? (unsigned int)((pairs - 1ull) / 2ull) : 0u;
    ctl->prefix = 0u;
    ctl->bw = 1.0f;
    ctl->med = 0.0f;
    ctl->mode = 1;
    if (status) {
      volatile int* h = status;
      *h = *h | kStatusGradDead;
    }
  }
}

template <int MM>
struct Pad4 {
  static constexpr int Q = (MM + 3) / 4;  // float4 groups per particle
};

template <int MM>
__device__ __forceinline__ void load_row(const float* __restrict__ u, int M, int N, int i, float (&r)[MM]) {
#pragma unroll
  for (int k = 0; k < MM; ++k) r[k] = (k < M && i < N) ? u[(size_t)k * N + i] : 0.f;
}

// Unpack a shared-memory row of float4 into MM scalars (the padding lanes of
// the last float4 are loaded but never used).
template <int MM>
__device__ __forceinline__ void unpack_row(const float4* __restrict__ src, float (&v)[MM]) {
#pragma unroll
  for (int q = 0; q < Pad4<MM>::Q; ++q) {
    const float4 t = src[q];
    if (4 * q + 0 < MM) v[4 * q + 0] = t.x;
    if (4 * q + 1 < MM) v[4 * q + 1] = t.y;
    if (4 * q + 2 < MM) v[4 * q + 2] = t.z;
    if (4 * q + 3 < MM) v[4 * q + 3] = t.w;
  }
}

// Stage particle j's coordinates (zero padded to a multiple of 4) into a
// shared-memory row of float4 so the inner loops read them with 128-bit
// broadcast loads.
template <int MM>
__device__ __forceinline__ void stage_row(const float* __restrict__ u, int M, int N, int j, bool ok,
                                          float4* __restrict__ dst) {
  constexpr int Q = Pad4<MM>::Q;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = 4 * q + r;
      v[r] = (ok && k < M) ? u[(size_t)k * N + j] : 0.f;
    }
    dst[q] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

template <int MM>
__device__ __forceinline__ float sqdist(const float (&a)[MM], const float4* __restrict__ b) {
  float v[MM];
  unpack_row<MM>(b, v);
  float d = 0.f;
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    const float e = a[k] - v[k];
    d = fmaf(e, e, d);
  }
  return d;
}

constexpr int kRows = 2;                 // rows (particles i) per thread
constexpr int kSpan = kTile * kRows;     // particles per square tile

__device__ __forceinline__ void hist_add(unsigned int* hist, float d, int pass, unsigned int prefix) {
  if (!(d == d)) return;  // a pair with a particle that sits out the step
  const unsigned int bits = __float_as_uint(d);
  if (pass == 0) {
    atomicAdd(&hist[bits >> 21], 1u);
  } else if (pass == 1) {
    if ((bits >> 21) == prefix) atomicAdd(&hist[(bits >> 10) & 2047u], 1u);
  } else {
    if ((bits >> 10) == prefix) atomicAdd(&hist[bits & 1023u], 1u);
  }
}

// One radix-select pass over all pairs i < j.  pass 0 histograms bits
// [31:21]; pass 1 bits [20:10] of the pairs whose bits [31:21] equal the
// resolved prefix; pass 2 bits [9:0] of those whose bits [31:10] match.
// Square tiles of kSpan x kSpan particles; a thread owns kRows rows.
template <int MM>
__global__ void __launch_bounds__(kTile) median_hist_kernel(int N, int M, const float* __restrict__ u,
                                                            SvgdCtl* __restrict__ ctl, int pass,
                                                            int only_in_fallback) {
  PDS_PDL_ENTRY();
  constexpr int Q = Pad4<MM>::Q;
  __shared__ unsigned int hist[kHistBins];
  __shared__ float4 uj[kSpan][Q];
  if (only_in_fallback && ctl->mode != 1) return;  // the sampled bracket held the median
  for (int b = threadIdx.x; b < kHistBins; b += kTile) hist[b] = 0u;
  const unsigned int prefix = ctl->prefix;
  const int nt = (N + kSpan - 1) / kSpan;
  const long long ntiles = (long long)nt * nt;
  __syncthreads();
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int I = (int)(tile / nt), J = (int)(tile - (long long)I * nt);
    if (I > J) continue;  // uniform across the block
    const int i0 = I * kSpan + threadIdx.x, i1 = i0 + kTile;
    float a0[MM], a1[MM];
    load_row<MM>(u, M, N, i0, a0);
    load_row<MM>(u, M, N, i1, a1);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int jl = threadIdx.x + r * kTile;
      const int j = J * kSpan + jl;
      stage_row<MM>(u, M, N, j, j < N, uj[jl]);
    }
    __syncthreads();
    const int jn = min(kSpan, N - J * kSpan);
    if (I < J) {
      for (int jj = 0; jj < jn; ++jj) {
        const float d0 = sqdist<MM>(a0, uj[jj]);
        const float d1 = sqdist<MM>(a1, uj[jj]);
        if (i0 < N) hist_add(hist, d0, pass, prefix);
        if (i1 < N) hist_add(hist, d1, pass, prefix);
      }
    } else {
      // diagonal tile: only j > i
      const int l0 = threadIdx.x, l1 = threadIdx.x + kTile;
      for (int jj = l0 + 1; jj < jn; ++jj) {
        const float d0 = sqdist<MM>(a0, uj[jj]);
        if (i0 < N) hist_add(hist, d0, pass, prefix);
        if (jj > l1 && i1 < N) hist_add(hist, sqdist<MM>(a1, uj[jj]), pass, prefix);
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
__global__ void median_select_kernel(SvgdCtl* __restrict__ ctl, int pass, int N, int required_mode) {
  PDS_PDL_ENTRY();
  if (required_mode >= 0 && ctl->mode != required_mode) return;
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
      const unsigned int nl = ctl->n_live;
      ctl->bw = (med > 0.f && nl > 1) ? med / logf((float)nl) : 1.0f;
    }
  }
  __syncwarp();
  for (int b = 0; b < 64; ++b) ctl->hist[lane * 64 + b] = 0u;
}

// ---- small N: the whole median in one block --------------------------------
// For N <= kSmallMedianN every pair distance fits in shared memory (at most
// 32640 floats).  One block computes them once, with the same arithmetic as
// median_hist_kernel (sum over the padded coordinates in order, fmaf), and
// runs the same three radix digits (11, 11, 10 bits) over shared memory
// instead of over recomputed distances in three launches.  Pairs with a
// particle that sits out are NaN and skipped; the rank over the live pairs
// comes from the liveness pass.  The same exact lower median and bandwidth.
constexpr int kSmallThreads = 512;

template <int MM>
__global__ void __launch_bounds__(kSmallThreads) median_small_kernel(int N, int M, const float* __restrict__ u,
                                                                     SvgdCtl* __restrict__ ctl) {
  PDS_PDL_ENTRY();
  extern __shared__ float sm_small[];
  __shared__ unsigned int hist[kHistBins];
  __shared__ unsigned int s_prefix, s_rank;
  __shared__ int s_found;
  float* us = sm_small;               // [MM][N] coordinates (0 beyond M)
  float* dist = sm_small + MM * N;    // [N (N - 1) / 2] pair distances, i < j, row by row
  const int t = threadIdx.x;
  for (int e = t; e < MM * N; e += blockDim.x) {
    const int k = e / N;
    us[e] = k < M ? u[(size_t)k * N + (e - k * N)] : 0.f;
  }
  if (t == 0) {
    s_prefix = 0u;
    s_rank = ctl->rank;
    s_found = 1;
  }
  __syncthreads();
  const int pairs = N * (N - 1) / 2;
  for (int q = t; q < N * N; q += blockDim.x) {
    const int i = q / N, j = q - i * N;
    if (j <= i) continue;
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < MM; ++k) {
      const float e = us[k * N + i] - us[k * N + j];
      d = fmaf(e, e, d);
    }
    dist[i * N - i * (i + 1) / 2 + (j - i - 1)] = d;
  }
  __syncthreads();
  for (int pass = 0; pass < 3; ++pass) {
    for (int b = t; b < kHistBins; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const unsigned int prefix = s_prefix;
    for (int p = t; p < pairs; p += blockDim.x) {
      const float d = dist[p];
      if (!(d == d)) continue;  // a pair with a particle that sits out the step
      const unsigned int bits = __float_as_uint(d);
      if (pass == 0) atomicAdd(&hist[bits >> 21], 1u);
      else if (pass == 1) { if ((bits >> 21) == prefix) atomicAdd(&hist[(bits >> 10) & 2047u], 1u); }
      else if ((bits >> 10) == prefix) atomicAdd(&hist[bits & 1023u], 1u);
    }
    __syncthreads();
    if (t < 32) {
      // the bin holding the rank (as median_select_kernel)
      const int lane = t;
      unsigned int local = 0u;
      for (int b = 0; b < 64; ++b) local += hist[lane * 64 + b];
      unsigned int incl = local;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      const unsigned int excl = incl - local;
      const unsigned int rank = s_rank;
      const bool any = __shfl_sync(0xffffffffu, incl, 31) > rank;
      if (lane == 0 && !any) s_found = 0;
      if (rank >= excl && rank < incl) {
        unsigned int cum = excl;
        int bin = lane * 64;
        for (int b = 0; b < 64; ++b) {
          const unsigned int h = hist[lane * 64 + b];
          if (rank < cum + h) { bin = lane * 64 + b; break; }
          cum += h;
        }
        const unsigned int digit_bits = (pass == 2) ? 10u : 11u;
        s_rank = rank - cum;
        s_prefix = (prefix << digit_bits) | (unsigned int)bin;
      }
    }
    __syncthreads();
  }
  if (t == 0 && s_found) {
    const float med = __uint_as_float(s_prefix);
    ctl->med = med;
    const unsigned int nl = ctl->n_live;
    ctl->bw = (med > 0.f && nl > 1) ? med / logf((float)nl) : 1.0f;
  }
}

template <int MM>
static cudaError_t launch_median_small(int N, int M, const float* u, SvgdCtl* ctl, cudaStream_t st) {
  const size_t smem = ((size_t)MM * N + (size_t)N * (N - 1) / 2) * sizeof(float);
  static bool attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(median_small_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(((size_t)MM * kSmallMedianN +
                                                      (size_t)kSmallMedianN * (kSmallMedianN - 1) / 2) *
                                                     sizeof(float)));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  launch_pdl(median_small_kernel<MM>, dim3(1), dim3(kSmallThreads), smem, st, N, M, u, ctl);
  return cudaGetLastError();
}

// ---- sampled bracket around the median (large N) -------------------------
// A sample of kSample ordered pairs (i != j, from a counter-based hash) is
// sorted in shared memory; the order statistics at ranks kSample/2 -+ 2
// sqrt(kSample) (4 standard deviations of the sample median's rank) bracket
// the median of all pairs with high probability.  One pass over all pairs
// then counts the pairs below the bracket and collects those inside it; the
// radix select finishes on the candidates only.  If the bracket missed the
// median, or the candidates overflow their buffer, the three full passes
// over all pairs run instead, so the result is always the exact median.
constexpr int kSample = 16384;
constexpr int kSampleThreads = 1024;
constexpr int kSampleMargin = 256;     // 2 sqrt(kSample)

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  // SplitMix64 finaliser (Steele, Lea and Flood, 2014)
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Distances of kSample hashed ordered pairs (one per thread, many blocks).
template <int MM>
__global__ void __launch_bounds__(256) median_sample_dist_kernel(int N, int M, const float* __restrict__ u,
                                                                 float* __restrict__ samp) {
  PDS_PDL_ENTRY();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= kSample) return;
  const unsigned long long h = mix64((unsigned long long)s);
  const int i = (int)((h & 0xffffffffull) % (unsigned long long)N);
  int j = (int)((h >> 32) % (unsigned long long)(N - 1));
  if (j >= i) ++j;
  float d = 0.f;
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    if (k < M) {
      const float e = u[(size_t)k * N + i] - u[(size_t)k * N + j];
      d = fmaf(e, e, d);
    }
  }
  samp[s] = d;
}

// The two order statistics of the sample that bracket the median, by a
// radix select in one block (three passes of 11, 11 and 10 bits; both ranks
// resolved together with one histogram each).
__global__ void __launch_bounds__(kSampleThreads) median_sample_sort_kernel(const float* __restrict__ samp,
                                                                            SvgdCtl* __restrict__ ctl) {
  PDS_PDL_ENTRY();
  constexpr int kPer = kSample / kSampleThreads;
  __shared__ unsigned int hist[2][kHistBins];
  __shared__ unsigned int prefix[2], rank[2];
  unsigned int v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) v[k] = __float_as_uint(samp[threadIdx.x + k * kSampleThreads]);
  if (threadIdx.x < 2) {
    prefix[threadIdx.x] = 0u;
    rank[threadIdx.x] = threadIdx.x == 0 ? (unsigned)(kSample / 2 - kSampleMargin) : (unsigned)(kSample / 2 + kSampleMargin);
  }
  for (int pass = 0; pass < 3; ++pass) {
    for (int b = threadIdx.x; b < 2 * kHistBins; b += kSampleThreads) hist[b / kHistBins][b % kHistBins] = 0u;
    __syncthreads();
    const unsigned int shift = pass == 0 ? 21u : pass == 1 ? 10u : 0u;
    const unsigned int mask = pass == 2 ? 1023u : 2047u;
    const unsigned int hi_shift = pass == 0 ? 32u : pass == 1 ? 21u : 10u;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const unsigned int pf = prefix[q];
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const bool match = hi_shift == 32u || (v[k] >> hi_shift) == pf;
        if (match) atomicAdd(&hist[q][(v[k] >> shift) & mask], 1u);
      }
    }
    __syncthreads();
    // warp q resolves order statistic q
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 2) {
      const unsigned int* h = hist[warp];
      unsigned int local = 0u;
      for (int b = 0; b < 64; ++b) local += h[lane * 64 + b];
      unsigned int incl = local;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      const unsigned int excl = incl - local;
      const unsigned int r = rank[warp];
      if (r >= excl && r < incl) {
        unsigned int cum = excl;
        int bin = lane * 64;
        for (int b = 0; b < 64; ++b) {
          const unsigned int c = h[lane * 64 + b];
          if (r < cum + c) { bin = lane * 64 + b; break; }
          cum += c;
        }
        rank[warp] = r - cum;
        prefix[warp] = (prefix[warp] << (pass == 2 ? 10u : 11u)) | (unsigned int)bin;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ctl->lo = __uint_as_float(prefix[0]);
    ctl->hi = __uint_as_float(prefix[1]);
    // candidates are max(d, 0) in [max(lo, 0), hi]: keys relative to the
    // lower end span at most 2^32; 2048 bins of key >> cshift cover them
    const unsigned int lob = __float_as_uint(fmaxf(__uint_as_float(prefix[0]), 0.f));
    const unsigned int span = prefix[1] >= lob ? prefix[1] - lob : 0u;
    const int bits = 32 - __clz(span);
    ctl->lob = lob;
    ctl->cshift = bits > 11 ? (unsigned int)(bits - 11) : 0u;
  }
}

constexpr int kCandBuf = 8192;       // per-block shared candidate buffer (floats)
constexpr int kCandFlushEvery = 16;  // j steps between flush checks (adds <= 16 * kSpan)

__device__ __forceinline__ void cand_flush(float* __restrict__ buf, unsigned int* __restrict__ count,
                                           SvgdCtl* __restrict__ ctl, float* __restrict__ cand,
                                           unsigned long long cap) {
  __shared__ unsigned long long base;
  const unsigned int n = *count;
  if (threadIdx.x == 0) base = n ? atomicAdd(&ctl->inside, (unsigned long long)n) : 0ull;
  __syncthreads();
  for (unsigned int k = threadIdx.x; k < n; k += blockDim.x)
    if (base + k < cap) cand[base + k] = buf[k];
  __syncthreads();
  if (threadIdx.x == 0) *count = 0u;
  __syncthreads();
}

// One pass over all pairs i < j: count d < lo, collect lo <= d <= hi.
template <int MM>
__global__ void __launch_bounds__(kTile) median_bracket_kernel(int N, int M, const float* __restrict__ u,
                                                               SvgdCtl* __restrict__ ctl, float* __restrict__ cand,
                                                               unsigned long long cap) {
  PDS_PDL_ENTRY();
  constexpr int Q = Pad4<MM>::Q;
  __shared__ float4 uj[kSpan][Q];
  __shared__ float buf[kCandBuf];
  __shared__ unsigned int count;
  __shared__ unsigned long long below_blk;
  if (threadIdx.x == 0) { count = 0u; below_blk = 0ull; }
  const float lo = ctl->lo, hi = ctl->hi;
  const int nt = (N + kSpan - 1) / kSpan;
  const long long ntiles = (long long)nt * nt;
  unsigned int below = 0u;
  __syncthreads();
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int I = (int)(tile / nt), J = (int)(tile - (long long)I * nt);
    if (I > J) continue;  // uniform across the block
    const int i0 = I * kSpan + threadIdx.x, i1 = i0 + kTile;
    float a0[MM], a1[MM];
    load_row<MM>(u, M, N, i0, a0);
    load_row<MM>(u, M, N, i1, a1);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int jl = threadIdx.x + r * kTile;
      const int j = J * kSpan + jl;
      stage_row<MM>(u, M, N, j, j < N, uj[jl]);
    }
    __syncthreads();
    const int jn = min(kSpan, N - J * kSpan);
    const bool diag = (I == J);
    const int l0 = threadIdx.x, l1 = threadIdx.x + kTile;
    for (int jb = 0; jb < jn; jb += kCandFlushEvery) {
      const int je = min(jn, jb + kCandFlushEvery);
      for (int jj = jb; jj < je; ++jj) {
        const float d0 = sqdist<MM>(a0, uj[jj]);
        const float d1 = sqdist<MM>(a1, uj[jj]);
        const bool v0 = (i0 < N) && (!diag || jj > l0);
        const bool v1 = (i1 < N) && (!diag || jj > l1);
        below += (v0 && d0 < lo) + (v1 && d1 < lo);
        const bool c0 = v0 && d0 >= lo && d0 <= hi;
        const bool c1 = v1 && d1 >= lo && d1 <= hi;
        const unsigned int m0 = __ballot_sync(0xffffffffu, c0);
        const unsigned int m1 = __ballot_sync(0xffffffffu, c1);
        const int lane = threadIdx.x & 31;
        if (m0 | m1) {
          unsigned int wbase = 0u;
          if (lane == 0) wbase = atomicAdd(&count, (unsigned int)(__popc(m0) + __popc(m1)));
          wbase = __shfl_sync(0xffffffffu, wbase, 0);
          const unsigned int lt = (1u << lane) - 1u;
          if (c0) buf[wbase + __popc(m0 & lt)] = d0;
          if (c1) buf[wbase + __popc(m0) + __popc(m1 & lt)] = d1;
        }
      }
      __syncthreads();
      if (count > kCandBuf - kCandFlushEvery * kSpan) cand_flush(buf, &count, ctl, cand, cap);
    }
    __syncthreads();
  }
  cand_flush(buf, &count, ctl, cand, cap);
  atomicAdd(&below_blk, (unsigned long long)below);
  __syncthreads();
  if (threadIdx.x == 0 && below_blk) atomicAdd(&ctl->below, below_blk);
}

// Decide between the candidate path and the full passes.
__global__ void median_resolve_kernel(SvgdCtl* __restrict__ ctl, unsigned long long cap) {
  PDS_PDL_ENTRY();
  const unsigned long long rank = ctl->rank;
  const unsigned long long below = ctl->below, inside = ctl->inside;
  if (below <= rank && rank < below + inside && inside <= cap) {
    ctl->mode = 0;
    ctl->rank = (unsigned int)(rank - below);
  } else {
    ctl->mode = 1;
  }
}

// ---- selection among the candidates by keys relative to the bracket ------
// One histogram pass of key >> cshift (2048 bins), the bin that holds the
// rank, a compaction of that bin's candidates, and an exact radix select
// over the remaining cshift low bits in one block.  The same median as three
// radix passes over the candidates' full bit patterns.
constexpr int kCbinCap = 1 << 20;  // compacted candidates of the median's bin (floats)

int svgd_cbin_capacity() { return kCbinCap; }

__device__ __forceinline__ unsigned int cand_key(float v, unsigned int lob) { return __float_as_uint(v) - lob; }

__global__ void __launch_bounds__(256) median_cand_key_hist_kernel(const float* __restrict__ cand,
                                                                   SvgdCtl* __restrict__ ctl) {
  PDS_PDL_ENTRY();
  __shared__ unsigned int hist[kHistBins];
  if (ctl->mode != 0) return;
  for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  const unsigned long long n = ctl->inside;
  const unsigned int lob = ctl->lob, sh = ctl->cshift;
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long n4 = n / 4;
  const float4* c4 = reinterpret_cast<const float4*>(cand);
  auto add = [&](float v) { atomicAdd(&hist[min(cand_key(v, lob) >> sh, (unsigned int)kHistBins - 1u)], 1u); };
  unsigned long long k = tid;
  for (; k + stride < n4; k += 2 * stride) {
    const float4 a = __ldg(c4 + k), b = __ldg(c4 + k + stride);
    add(a.x); add(a.y); add(a.z); add(a.w);
    add(b.x); add(b.y); add(b.z); add(b.w);
  }
  if (k < n4) {
    const float4 a = __ldg(c4 + k);
    add(a.x); add(a.y); add(a.z); add(a.w);
  }
  for (unsigned long long e = 4 * n4 + tid; e < n; e += stride) add(__ldg(cand + e));
  __syncthreads();
  for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) {
    const unsigned int h = hist[b];
    if (h) atomicAdd(&ctl->hist[b], h);
  }
}

// The bin holding the rank (one warp); clears the histogram and the bin count.
__global__ void median_cand_bin_kernel(SvgdCtl* __restrict__ ctl) {
  PDS_PDL_ENTRY();
  if (ctl->mode != 0) return;
  const int lane = threadIdx.x;
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
  __syncwarp();
  if (rank >= excl && rank < incl) {
    unsigned int cum = excl;
    int bin = lane * 64;
    for (int b = 0; b < 64; ++b) {
      const unsigned int h = ctl->hist[lane * 64 + b];
      if (rank < cum + h) { bin = lane * 64 + b; break; }
      cum += h;
    }
    ctl->cbin = (unsigned int)bin;
    ctl->rank = rank - cum;
    ctl->ccount = 0u;
  }
  __syncwarp();
  for (int b = 0; b < 64; ++b) ctl->hist[lane * 64 + b] = 0u;
}

// Candidates of the median's bin into cbuf (up to its capacity; ccount
// counts them all).  Each thread takes 4 consecutive candidates (one float4)
// per iteration; a warp reserves its slots with one atomic.
__global__ void __launch_bounds__(256) median_cand_compact_kernel(const float* __restrict__ cand,
                                                                  SvgdCtl* __restrict__ ctl,
                                                                  float* __restrict__ cbuf) {
  PDS_PDL_ENTRY();
  if (ctl->mode != 0) return;
  const unsigned long long n = ctl->inside;
  const unsigned int lob = ctl->lob, sh = ctl->cshift, bin = ctl->cbin;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long groups = (n + 3) / 4;
  const unsigned long long groups_up = (groups + 31) / 32 * 32;  // whole warps in the loop
  const int lane = threadIdx.x & 31;
  const float4* c4 = reinterpret_cast<const float4*>(cand);
  const unsigned long long n4 = n / 4;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups_up; g += stride) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (g < n4) {
      const float4 a = __ldg(c4 + g);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if (g < groups) {
      for (int q = 0; q < 4; ++q)
        if (4 * g + q < n) v[q] = __ldg(cand + 4 * g + q);
    }
    unsigned int mask = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (g < groups && 4 * g + q < n && min(cand_key(v[q], lob) >> sh, (unsigned int)kHistBins - 1u) == bin)
        mask |= 1u << q;
    const unsigned int mine = __popc(mask);
    unsigned int incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
      unsigned int base = 0u;
      if (lane == 31) base = atomicAdd(&ctl->ccount, total);
      base = __shfl_sync(0xffffffffu, base, 31);
      unsigned int pos = base + incl - mine;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (mask & (1u << q)) {
          if (pos < (unsigned int)kCbinCap) cbuf[pos] = v[q];
          ++pos;
        }
    }
  }
}

// Exact rank-th smallest key of the median's bin: radix passes of up to 11
// bits over the cshift low bits, in one block; reads the compacted bin, or
// (if it overflowed cbuf) filters all candidates.  Sets the median and the
// bandwidth over the live particles.
constexpr int kFinalThreads = 1024;
__global__ void __launch_bounds__(kFinalThreads) median_cand_final_kernel(const float* __restrict__ cand,
                                                                          const float* __restrict__ cbuf,
                                                                          SvgdCtl* __restrict__ ctl) {
  PDS_PDL_ENTRY();
  __shared__ unsigned int hist[kHistBins];
  __shared__ unsigned int s_prefix, s_rank;
  if (ctl->mode != 0) return;
  const unsigned int lob = ctl->lob, sh = ctl->cshift, bin = ctl->cbin;
  const unsigned int cnt = ctl->ccount;
  const bool compact = cnt <= (unsigned int)kCbinCap;
  const float* src = compact ? cbuf : cand;
  const unsigned long long n = compact ? (unsigned long long)cnt : ctl->inside;
  if (threadIdx.x == 0) {
    s_prefix = 0u;
    s_rank = ctl->rank;
  }
  int done = 0;  // low bits resolved so far
  while (done < (int)sh) {
    const int d = min(11, (int)sh - done);  // digit width
    const int lowsh = (int)sh - done - d;   // shift of this digit within the key
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const unsigned int prefix = s_prefix;
    for (unsigned long long e = threadIdx.x; e < n; e += blockDim.x) {
      const unsigned int key = cand_key(__ldg(src + e), lob);
      if (min(key >> sh, (unsigned int)kHistBins - 1u) != bin) continue;
      const unsigned int low = key & ((sh < 32 ? (1u << sh) : 0u) - 1u);
      if ((low >> (lowsh + d)) != prefix) continue;
      atomicAdd(&hist[(low >> lowsh) & ((1u << d) - 1u)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      unsigned int local = 0u;
      for (int b = 0; b < 64; ++b) local += hist[lane * 64 + b];
      unsigned int incl = local;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      const unsigned int excl = incl - local;
      const unsigned int rank = s_rank;
      if (rank >= excl && rank < incl) {
        unsigned int cum = excl;
        int digit = lane * 64;
        for (int b = 0; b < 64; ++b) {
          if (rank < cum + hist[lane * 64 + b]) { digit = lane * 64 + b; break; }
          cum += hist[lane * 64 + b];
        }
        s_rank = rank - cum;
        s_prefix = (prefix << d) | (unsigned int)digit;
      }
    }
    __syncthreads();
    done += d;
  }
  if (threadIdx.x == 0) {
    const unsigned int key = (bin << sh) | s_prefix;
    const float med = __uint_as_float(lob + key);
    ctl->med = med;
    const unsigned int nl = ctl->n_live;
    ctl->bw = (med > 0.f && nl > 1) ? med / logf((float)nl) : 1.0f;
  }
}

int svgd_sample_size() { return kSample; }

// One-time per-device set-up of the SVGD kernels (none needed at present;
// kept as the place to do it before any stream capture).
cudaError_t svgd_setup_device() { return cudaSuccess; }

unsigned long long svgd_cand_capacity(int N) {
  if (N < 2048) return 0ull;
  const unsigned long long pairs = (unsigned long long)N * (unsigned long long)(N - 1) / 2ull;
  unsigned long long cap = pairs / 12ull;  // 8 % of the pairs; the bracket expects 3.1 %
  if (cap < (1ull << 20)) cap = 1ull << 20;
  return cap;
}

// Partial phi over one chunk of j: phi_part[c][k][i] =
//   sum_j k_ij g_j[k] + (2/bw) sum_j k_ij (u_i[k] - u_j[k]).
// A block owns kSpan rows (kRows per thread); j is staged kTile at a time.
template <int MM, bool FAST>
__global__ void __launch_bounds__(kTile) svgd_phi_kernel(int N, int M, const float* __restrict__ u,
                                                         const float* __restrict__ gu, const SvgdCtl* __restrict__ ctl,
                                                         float* __restrict__ phi_part, int chunk_len) {
  PDS_PDL_ENTRY();
  constexpr int Q = Pad4<MM>::Q;
  __shared__ float4 uj[kTile][Q];
  __shared__ float4 gj[kTile][Q];
  const int i0 = blockIdx.x * kSpan + threadIdx.x, i1 = i0 + kTile;
  const int c = blockIdx.y;
  const int j0 = c * chunk_len;
  const int j1 = min(N, j0 + chunk_len);
  const float bw = ctl->bw;
  const float inv_bw = 1.0f / bw;
  float a0[MM], a1[MM], g0[MM], g1[MM], r0[MM], r1[MM];
  load_row<MM>(u, M, N, i0, a0);
  load_row<MM>(u, M, N, i1, a1);
#pragma unroll
  for (int k = 0; k < MM; ++k) { g0[k] = 0.f; g1[k] = 0.f; r0[k] = 0.f; r1[k] = 0.f; }
  for (int jt = j0; jt < j1; jt += kTile) {
    const int j = jt + threadIdx.x;
    // a particle that sits out the step (u is NaN) is staged far away (its
    // kernel value underflows to 0) with a zero gradient
    const bool live = j < j1 && isfinite(u[(size_t)(j < N ? j : 0)]);
    if (live || j >= j1) {
      stage_row<MM>(u, M, N, j, j < j1, uj[threadIdx.x]);
      stage_row<MM>(gu, M, N, j, j < j1, gj[threadIdx.x]);
    } else {
#pragma unroll
      for (int q = 0; q < Pad4<MM>::Q; ++q) {
        uj[threadIdx.x][q] = make_float4(1e18f, 1e18f, 1e18f, 1e18f);
        gj[threadIdx.x][q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    const int jn = min(kTile, j1 - jt);
    for (int jj = 0; jj < jn; ++jj) {
      float v[MM], e0[MM], e1[MM];
      unpack_row<MM>(uj[jj], v);
      float d0 = 0.f, d1 = 0.f;
#pragma unroll
      for (int k = 0; k < MM; ++k) {
        e0[k] = a0[k] - v[k];
        e1[k] = a1[k] - v[k];
        d0 = fmaf(e0[k], e0[k], d0);
        d1 = fmaf(e1[k], e1[k], d1);
      }
      const float k0 = FAST ? __expf(-d0 * inv_bw) : expf(-d0 * inv_bw);
      const float k1 = FAST ? __expf(-d1 * inv_bw) : expf(-d1 * inv_bw);
      float gg[MM];
      unpack_row<MM>(gj[jj], gg);
#pragma unroll
      for (int k = 0; k < MM; ++k) {
        g0[k] = fmaf(k0, gg[k], g0[k]);
        g1[k] = fmaf(k1, gg[k], g1[k]);
        r0[k] = fmaf(k0, e0[k], r0[k]);
        r1[k] = fmaf(k1, e1[k], r1[k]);
      }
    }
    __syncthreads();
  }
  const float two_over_bw = 2.0f * inv_bw;
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    if (k < M) {
      if (i0 < N) phi_part[((size_t)c * M + k) * N + i0] = fmaf(two_over_bw, r0[k], g0[k]);
      if (i1 < N) phi_part[((size_t)c * M + k) * N + i1] = fmaf(two_over_bw, r1[k], g1[k]);
    }
  }
}

// The step's last kernel.  It also reports, into the mapped host word
// status (may be NULL), a tensor-core pass of this step that gave up waiting
// and a step in which no particle was live.
__global__ void svgd_adam_kernel(SvgdParams sp, SvgdCtl* __restrict__ ctl, float* __restrict__ X,
                                 const float* __restrict__ G, const float* __restrict__ phi_part, int chunks,
                                 float* __restrict__ am, float* __restrict__ av, float* __restrict__ bw_out,
                                 float* __restrict__ phi_out, int* __restrict__ status) {
  PDS_PDL_ENTRY();
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)sp.P * sp.N;
  if (idx == 0 && bw_out) *bw_out = ctl->bw;
  if (idx == 0 && status) {
    const int f = (ctl->tc_error ? kStatusTimeout : 0) | (ctl->n_live == 0u ? kStatusNoneLive : 0);
    if (f) {
      volatile int* h = status;
      *h = *h | f;
    }
  }
  if (idx < 16) ctl->gmax[idx] = 0u;  // for the next step's prep kernel
  if (idx >= total) return;
  const int r = (int)(idx / sp.N);
  const int i = (int)(idx - (size_t)r * sp.N);
  const float bc1 = ctl->bc1, bc2 = ctl->bc2;
  if (sp.csvgd && r >= sp.lam0) {
    // MDMM multipliers: lambda' = g (Algorithm 1), a gradient-ascent step
    X[idx] = X[idx] + sp.lr * G[idx];
    return;
  }
  float g;
  float x;
  if (r < sp.M) {
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += phi_part[((size_t)c * sp.M + r) * sp.N + i];
    const unsigned int nl = ctl->n_live;  // the 1/N of Eq. 1 over the live particles
    g = s / (float)(nl ? nl : 1u);
    if (phi_out) phi_out[idx] = g;
    const float width = sp.hi[r] - sp.lo[r];
    // constrained SVGD: plus the constraint direction -dPsi/dtheta, in u
    if (sp.csvgd) g += G[(size_t)(sp.P + r) * sp.N + i] * width;
    x = (X[idx] - sp.lo[r]) / width;
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
    if (sp.clamp && !sp.csvgd) x = fminf(1.f, fmaxf(0.f, x));
    x = sp.lo[r] + x * (sp.hi[r] - sp.lo[r]);
  }
  X[idx] = x;
}

int svgd_phi_chunks(int N) {
  const int row_blocks = (N + kSpan - 1) / kSpan;
  int chunks = (8 * 152 + row_blocks - 1) / row_blocks;
  const int max_chunks = (N + kTile - 1) / kTile;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  return chunks;
}

// Partial-phi buffers to allocate: enough for the CUDA-core chunks and the
// tensor-core path's per-row slots.
int svgd_phi_partials(int N) {
  const int c = svgd_phi_chunks(N);
  const int s = N >= 256 ? phi_tc_slots(N) : 0;
  return c > s ? c : s;
}

template <int MM>
static cudaError_t launch_svgd_mm(const SvgdParams& sp, const SvgdWork& w, float* X, const float* G, float* bw_out,
                                  float* phi_out, cudaStream_t st, int* launches, int phase) {
  const int N = sp.N, M = sp.M;
  int n = 0;
  const bool bracket = (N >= 2) && w.cand && w.cbuf && w.cand_cap > 0;
  // with the sampled bracket the step can run as two phases (kSvgdTheta
  // then kSvgdGrad, the second after the first on another stream): the
  // median over the particles with finite coordinates, then the gradient,
  // which takes out the particles with a gradient that is not finite and
  // then has the full passes redo the median exactly.  kSvgdAll takes the
  // gradient's liveness first and the bracket once.
  const bool split = bracket && phase != kSvgdAll;
  if (phase != kSvgdAll && !bracket) return cudaErrorInvalidValue;
  const bool doA = phase != kSvgdGrad, doB = phase != kSvgdTheta;
  // pair distances on the tensor cores (N >= 2048): every pass over the
  // pairs then sees the same distances
  const bool tcm = w.mimg && w.mwork && N >= 2048;
  const int nt = (N + kSpan - 1) / kSpan;
  const long long all_tiles = (long long)nt * nt;
  const int grid = all_tiles < 152 * 8 ? (int)all_tiles : 152 * 8;
  bool prepped = false;  // the tensor-core images of u are current
  if (doA) {
    const int total = (M * N > kHistBins) ? M * N : kHistBins;
    launch_pdl(svgd_prep_kernel, dim3((total + 255) / 256), dim3(256), 0, st, sp, w.ctl, X, split ? nullptr : G, w.u,
               w.gu, bracket ? 0 : 1);
    launch_pdl(svgd_live_kernel, dim3((N + 255) / 256), dim3(256), 0, st, N, M, w.ctl, w.u,
               split ? (const float*)nullptr : (const float*)w.gu);
    n += 2;
    if (bracket) {
      cudaError_t e = svgd_setup_device();
      if (e != cudaSuccess) return e;
      launch_pdl(median_sample_dist_kernel<MM>, dim3(kSample / 256), dim3(256), 0, st, N, M, w.u, w.samp);
      launch_pdl(median_sample_sort_kernel, dim3(1), dim3(kSampleThreads), 0, st, w.samp, w.ctl);
      n += 2;
      if (tcm) {
        e = launch_median_tc(N, M, w.u, w.mimg, w.mwork, w.n_mwork, w.ctl, w.cand, w.cand_cap, 0, 0, true,
                             w.wait_limit, st);
        if (e != cudaSuccess) return e;
        prepped = true;
        n += 2;
      } else {
        launch_pdl(median_bracket_kernel<MM>, dim3(grid), dim3(kTile), 0, st, N, M, w.u, w.ctl, w.cand, w.cand_cap);
        n += 1;
      }
      launch_pdl(median_resolve_kernel, dim3(1), dim3(1), 0, st, w.ctl, w.cand_cap);
      // one pass of keys relative to the bracket, then the median's bin
      launch_pdl(median_cand_key_hist_kernel, dim3(152 * 4), dim3(256), 0, st, w.cand, w.ctl);
      launch_pdl(median_cand_bin_kernel, dim3(1), dim3(32), 0, st, w.ctl);
      launch_pdl(median_cand_compact_kernel, dim3(152 * 4), dim3(256), 0, st, w.cand, w.ctl, w.cbuf);
      launch_pdl(median_cand_final_kernel, dim3(1), dim3(kFinalThreads), 0, st, w.cand, w.cbuf, w.ctl);
      n += 5;
    }
  }
  if (!doB) {
    if (launches) *launches += n;
    return cudaGetLastError();
  }
  if (split) {
    launch_pdl(svgd_grad_live_kernel, dim3((N + 255) / 256), dim3(256), 0, st, sp, w.ctl, G, w.u, w.gu,
               w.status_flags);
    n += 1;
    prepped = false;  // the gradient may have taken particles out of u: the full passes rebuild the images
  }
  if (N >= 2) {
    // full passes over all pairs: always for small N or when asked, otherwise
    // only if the bracket missed or the gradient took particles out (the
    // kernels return at once otherwise); the smallest N in one block
    const bool small = !bracket && !tcm && w.small_median && N <= kSmallMedianN;
    if (small) {
      cudaError_t e = launch_median_small<MM>(N, M, w.u, w.ctl, st);
      if (e != cudaSuccess) return e;
      n += 1;
    }
    for (int pass = 0; pass < 3 && !small; ++pass) {
      if (tcm) {
        cudaError_t e = launch_median_tc(N, M, w.u, w.mimg, w.mwork, w.n_mwork, w.ctl, nullptr, 0ull, pass + 1,
                                         bracket ? 1 : 0, !prepped, w.wait_limit, st);
        if (e != cudaSuccess) return e;
        n += prepped ? 1 : 2;
        prepped = true;
      } else {
        launch_pdl(median_hist_kernel<MM>, dim3(grid), dim3(kTile), 0, st, N, M, w.u, w.ctl, pass, bracket ? 1 : 0);
        n += 1;
      }
      launch_pdl(median_select_kernel, dim3(1), dim3(32), 0, st, w.ctl, pass, N, 1);
      n += 1;
    }
  }
  {
    const int chunks0 = svgd_phi_chunks(N);
    const int chunk_len = ((N + chunks0 - 1) / chunks0 + kTile - 1) / kTile * kTile;
    const int chunks = (N + chunk_len - 1) / chunk_len;
    int chunks_used = chunks;
    if (w.tc && N >= 256) {
      // tensor-core path: the kernel-matrix products on tcgen05 (chunks0 chunks of 128-column tiles)
      int slots = 0;
      cudaError_t e = launch_phi_tc(N, M, w, &slots, st);
      if (e != cudaSuccess) return e;
      chunks_used = slots;
      n += 1;
    } else {
      dim3 grid((N + kSpan - 1) / kSpan, chunks);
      if (sp.fast_math)
        launch_pdl(svgd_phi_kernel<MM, true>, dim3(grid), dim3(kTile), 0, st, N, M, w.u, w.gu, w.ctl, w.phi_part, chunk_len);
      else
        launch_pdl(svgd_phi_kernel<MM, false>, dim3(grid), dim3(kTile), 0, st, N, M, w.u, w.gu, w.ctl, w.phi_part, chunk_len);
    }
    const size_t total = (size_t)sp.P * N;
    launch_pdl(svgd_adam_kernel, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, st, sp, w.ctl, X, G, w.phi_part, chunks_used,
                                                                      w.adam_m, w.adam_v, bw_out, phi_out,
                                                                      w.status_flags);
    n += 2;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_svgd_step(const SvgdParams& sp, const SvgdWork& w, float* X, const float* G, float* bw_out,
                             float* phi_out, cudaStream_t st, int* launches, int phase) {
  if (sp.M <= 2) return launch_svgd_mm<2>(sp, w, X, G, bw_out, phi_out, st, launches, phase);
  if (sp.M <= 4) return launch_svgd_mm<4>(sp, w, X, G, bw_out, phi_out, st, launches, phase);
  if (sp.M <= 8) return launch_svgd_mm<8>(sp, w, X, G, bw_out, phi_out, st, launches, phase);
  if (sp.M <= 10) return launch_svgd_mm<10>(sp, w, X, G, bw_out, phi_out, st, launches, phase);
  if (sp.M <= 12) return launch_svgd_mm<12>(sp, w, X, G, bw_out, phi_out, st, launches, phase);
  return launch_svgd_mm<16>(sp, w, X, G, bw_out, phi_out, st, launches, phase);
}

bool svgd_step_splits(const SvgdParams& sp, const SvgdWork& w) {
  return sp.N >= 2 && w.cand && w.cbuf && w.cand_cap > 0;
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
constexpr int kNoAllocMaxN = 65536;
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
    ctl->prefix = 0u;
    ctl->rank = 0u;
    ctl->bw = 1.0f;
    ctl->med = 0.0f;
    ctl->mode = 1;
    ctl->n_live = 0u;
    ctl->live_blocks = 0u;
  }
  if (idx < M * N) {
    const int k = idx / N;
    u[idx] = (theta[idx] - box.lo[k]) / (box.hi[k] - box.lo[k]);
  }
}

// As pds_svgd_step's liveness pass, on the coordinates alone: a particle
// with a coordinate that is not finite sits out (its u becomes NaN, so its
// pairs are skipped), the live particles are counted, and the last block
// sets the median's rank over the live pairs.
__global__ void __launch_bounds__(256) noalloc_live_kernel(int N, int M, SvgdCtl* __restrict__ ctl,
                                                           float* __restrict__ u) {
  __shared__ unsigned int blk;
  __shared__ bool last;
  if (threadIdx.x == 0) blk = 0u;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    bool live = true;
    for (int k = 0; k < M; ++k) live &= isfinite(u[(size_t)k * N + i]);
    if (live) atomicAdd(&blk, 1u);
    else
      for (int k = 0; k < M; ++k) u[(size_t)k * N + i] = __int_as_float(0x7fc00000);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (blk) atomicAdd(&ctl->n_live, blk);
    __threadfence();
    last = atomicAdd(&ctl->live_blocks, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long nl = atomicAdd(&ctl->n_live, 0u);
    const unsigned long long pairs = nl * (nl > 0 ? nl - 1ull : 0ull) / 2ull;
    ctl->rank = pairs ? (unsigned int)((pairs - 1ull) / 2ull) : 0u;
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
  noalloc_live_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, M, ctl, u);
  if (N >= 2) {
    const int nt = (N + kSpan - 1) / kSpan;
    const long long all_tiles = (long long)nt * nt;
    const int grid = all_tiles < 152 * 8 ? (int)all_tiles : 152 * 8;
    for (int pass = 0; pass < 3; ++pass) {
      median_hist_kernel<MM><<<grid, kTile, 0, st>>>(N, M, u, ctl, pass, 0);
      median_select_kernel<<<1, 32, 0, st>>>(ctl, pass, N, -1);
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
  // the radix histogram and the median's rank count pairs in 32 bits
  // (N (N - 1) / 2 < 2^31 for N <= 65536), as in pds_svgd_create
  if (N > kNoAllocMaxN)
    return set_error(PDS_ERR_ARG, "pds_bandwidth_noalloc: N must be at most 65536 (32-bit pair counts)");
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
