// Pairwise squared distances on the tensor cores for the median heuristic.
//
//   d_ij = |u_i|^2 + |u_j|^2 - 2 u_i . u_j = a_i . b_j,
//   a_i = (-2 u_i, n_i, 1),  b_j = (u_j, 1, n_j),  n = |u|^2,
// one tcgen05.mma (kind::tf32, split operands for fp32-level accuracy) per
// 128 x 128 tile of pairs into tensor memory; the CUDA cores then read the
// tile and either count and collect it against the sampled bracket, or add it
// to a radix-digit histogram.  Only tiles with I <= J are visited and only
// pairs i < j counted.  Every pass over the pairs (bracket, or the full radix
// passes when the bracket misses) uses this kernel, so all see bit-identical
// distances; a distance is clamped at zero by its bit pattern (negative
// rounding residue, and -0, become +0).
//
// The grid is persistent: CTA b takes the contiguous run
// [b T / G, (b+1) T / G) of the T upper-triangle tiles in row-major order,
// so every CTA gets the same number of tiles to within one.  Two shared-memory
// stages hold (row tile A, column tile B); A is copied only when the row
// changes.  Two TMEM accumulators let the products of tiles k+1 and k+2 run
// while tile k is read.  Eight warps read a tile: warp w owns TMEM lanes
// 32 (w mod 4) .. + 31 (its rows) and column half w / 4, and releases the
// accumulator through an mbarrier as soon as its loads are done.  No warp
// is set apart to feed the pipeline: the first warp past product k copies
// tile k+2 into the stage product k has left, and the last warp to release
// accumulator k mod 2 issues the product of tile k+2 into it (a shared
// counter elects each; the mbarriers order them), so every product is
// issued as early as its operands and accumulator allow.  In the
// bracket pass each warp appends its candidates to its own shared buffer
// and flushes it to global memory with one atomic when full.
#include <math.h>

#include "pds_internal.cuh"
#include "tc.cuh"

namespace pds {

constexpr int kMtRows = 128;
constexpr int kMtBins = 2048;
constexpr int kMtWarps = 8;  // 4 lane quarters x 2 column halves
constexpr int kMtThreads = 32 * kMtWarps;
constexpr int kMtCandW = 1024;  // candidate buffer per warp (floats)

template <int MM>
struct MtDims {
  static constexpr int KA = ((MM + 2 + 7) / 8) * 8;
  static constexpr int kA = kMtRows * KA * 4;  // one tile image (hi or lo), bytes
  static constexpr int kTile = 2 * kA;          // hi + lo
  static constexpr int kStage = 2 * kTile;      // row tile A + column tile B
  static constexpr int kCand = kMtWarps * kMtCandW * 4;
  static constexpr int kBytes = 2 * kStage + kCand + 128;
};

__device__ __forceinline__ void mt_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(tc::to_tf32(x));
  lo = __uint_as_float(tc::to_tf32(x - hi));
}

// Tile images (hi, lo) of a_i and b_j for every particle; rows N..Npad-1
// are zero (never counted).
template <int MM>
// only_in_fallback: the images are rebuilt only when the full passes run
// (the second phase of a split step may have taken particles out of u).
__global__ void median_tc_prep_kernel(int N, int Npad, int M, const float* __restrict__ u, float* __restrict__ imgA,
                                      float* __restrict__ imgB, const SvgdCtl* __restrict__ ctl,
                                      int only_in_fallback) {
  PDS_PDL_ENTRY();
  if (only_in_fallback && ctl->mode != 1) return;
  using D = MtDims<MM>;
  constexpr int KA = D::KA;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Npad) return;
  float x[MM];
  float n = 0.f;
  const bool live = j < N;
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    x[k] = (live && k < M) ? u[(size_t)k * N + j] : 0.f;
    n = fmaf(x[k], x[k], n);
  }
  const int tile = j / kMtRows, r = j % kMtRows;
  float* A = imgA + (size_t)tile * (D::kTile / 4);
  float* B = imgB + (size_t)tile * (D::kTile / 4);
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    const float a = k < MM ? -2.f * x[k] : (k == MM ? n : (k == MM + 1 ? (live ? 1.f : 0.f) : 0.f));
    const float b = k < MM ? x[k] : (k == MM ? (live ? 1.f : 0.f) : (k == MM + 1 ? n : 0.f));
    const uint32_t o = tc::kmajor_offset(r, k, KA) >> 2;
    float h, l;
    mt_split(a, h, l);
    A[o] = h;
    A[D::kA / 4 + o] = l;
    mt_split(b, h, l);
    B[o] = h;
    B[D::kA / 4 + o] = l;
  }
}

// mode 0: bracket (count d < lo, collect lo <= d <= hi); mode 1..3: radix
// pass 0..2 histogram.  tiles[f] = (row tile I, column tile J), J >= I.
template <int MM>
__global__ void __launch_bounds__(kMtThreads, 2) median_tc_kernel(int N, const float* __restrict__ imgA,
                                                                  const float* __restrict__ imgB,
                                                                  const int2* __restrict__ tiles, int n_tiles,
                                                                  SvgdCtl* __restrict__ ctl, float* __restrict__ cand,
                                                                  unsigned long long cap, int mode,
                                                                  int only_in_fallback, int wait_limit) {
  PDS_PDL_ENTRY();
  using D = MtDims<MM>;
  constexpr int KA = D::KA;
  // wait_limit: mbarrier polls before a wait gives up (the kernel then
  // flags ctl->tc_error); the waits that let copies and products in flight
  // finish before shared memory and TMEM are released take kDrainLimit
  extern __shared__ __align__(1024) unsigned char smem[];
  float* cbuf = (float*)(smem + 2 * D::kStage);  // per-warp candidates, or the histogram in radix modes
  uint64_t* bars = (uint64_t*)(smem + 2 * D::kStage + D::kCand);  // full[2], mma[2], free[2]
  uint32_t* tslot = (uint32_t*)(bars + 6);
  uint32_t* passed = tslot + 1;    // [2] warps past product k, per stage (elects the copy's issuer)
  uint32_t* released = tslot + 3;  // [2] warps done reading accumulator s (elects the product's issuer)
  uint32_t* failed = tslot + 5;    // a warp gave up

  if (only_in_fallback && ctl->mode != 1) return;  // uniform: the bracket held the median
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int f0 = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int f1 = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  const int nk = f1 - f0;
  unsigned int* hist = (unsigned int*)cbuf;
  float* wbuf = cbuf + warp * kMtCandW;
  // bracket on the clamped distance max(d, 0): with lo > 0, max(d, 0) < lo
  // iff d < lo; with lo = 0 nothing is below and inside means d <= hi
  const float lo = ctl->lo > 0.f ? ctl->lo : -INFINITY;
  const float hi = ctl->hi;
  const unsigned int prefix = ctl->prefix;
  const int pass = mode - 1;

  if (mode != 0)
    for (int b = t; b < kMtBins; b += kMtThreads) hist[b] = 0u;
  if (t == 0) {
    for (int b = 0; b < 4; ++b) tc::mbar_init(bars + b, 1);
    tc::mbar_init(bars + 4, kMtWarps);
    tc::mbar_init(bars + 5, kMtWarps);
    for (int b = 0; b < 5; ++b) passed[b] = 0u;
  }
  if (warp == 0) tc::tmem_alloc(tslot, 256);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;

  // Copies and products are issued by whichever warp can first do so (one
  // elected lane; operands warp-uniform).  In flight there is at most one
  // copy per stage and one product per accumulator (stage s is refilled only
  // once the product that read it is done, accumulator s only once every
  // warp has read it), so each thread remembers, per stage and accumulator,
  // the latest copy and product it issued there.
  int my_load[2] = {-1, -1}, my_mma[2] = {-1, -1};
  auto load = [&](int k, int2 tj, bool needA) {  // tile f0 + k, coordinates tj, into stage k & 1
    const int s = k & 1;
    unsigned char* stg = smem + s * D::kStage;
    tc::mbar_expect_tx(bars + s, needA ? 2 * D::kTile : D::kTile);
    if (needA) tc::bulk_g2s(stg, imgA + (size_t)tj.x * (D::kTile / 4), D::kTile, bars + s);
    tc::bulk_g2s(stg + D::kTile, imgB + (size_t)tj.y * (D::kTile / 4), D::kTile, bars + s);
    my_load[s] = k;
  };
  // product of tile k into accumulator k & 1, issued by a whole warp
  auto issue = [&](int k) {
    const int s = k & 1;
    tc::fence_after();
    constexpr uint32_t id = tc::idesc_tf32(128, 128);
    const uint32_t sbo = 32 * KA;
    const uint32_t a_h = tc::smem_u32(smem + s * D::kStage), a_l = a_h + D::kA;
    const uint32_t b_h = a_h + D::kTile, b_l = b_h + D::kA;
    const uint32_t Aop[3] = {a_h, a_h, a_l};
    const uint32_t Bop[3] = {b_h, b_l, b_h};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int ks = 0; ks < KA / 8; ++ks)
        tc::mma_ss_el(tbase + 128 * s, tc::smem_desc(Aop[p] + ks * 256, 128, sbo),
                      tc::smem_desc(Bop[p] + ks * 256, 128, sbo), id, (p > 0 || ks > 0) ? 1u : 0u);
    tc::mma_commit_el(bars + 2 + s);
    my_mma[s] = k;
  };

  bool ok = true;
  if (t == 0 && nk > 0) {
    load(0, tiles[f0], true);
    if (nk > 1) load(1, tiles[f0 + 1], true);
  }
  if (warp == 0 && nk > 0) {
    // the first two products (both accumulators start free)
    ok = __all_sync(0xffffffffu, tc::mbar_test(bars + 0, 0) || tc::mbar_wait(bars + 0, 0, wait_limit)) != 0;
    if (ok) issue(0);
    if (ok && nk > 1) {
      ok = __all_sync(0xffffffffu, tc::mbar_test(bars + 1, 0) || tc::mbar_wait(bars + 1, 0, wait_limit)) != 0;
      if (ok) issue(1);
    }
  }
  // tile coordinates ahead of their use: this tile's, and the next copy's
  int2 tj = nk > 0 ? tiles[f0] : make_int2(0, 0);

  unsigned int below = 0u;  // pairs below the bracket (this thread)
  unsigned int cnt = 0u;    // candidates in this warp's buffer (warp-uniform)
  auto flush = [&]() {      // warp: move its buffer to the global candidates
    unsigned long long base = 0ull;
    if (lane == 0) base = atomicAdd(&ctl->inside, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (unsigned int e = lane; e < cnt; e += 32)
      if (base + e < cap) cand[base + e] = wbuf[e];
    __syncwarp();
    cnt = 0u;
  };
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  const int c0 = half * 64;

  for (int k = 0; k < nk; ++k) {
    const int s = k & 1;
    const int2 tl = (lane == 0 && k + 2 < nk) ? tiles[f0 + k + 2] : make_int2(0, 0);
    bool w = ok && (tc::mbar_test(bars + 2 + s, (uint32_t)(k >> 1) & 1u) ||
                    tc::mbar_wait(bars + 2 + s, (uint32_t)(k >> 1) & 1u, wait_limit));
    ok = __all_sync(0xffffffffu, w) != 0;
    if (!ok) break;
    tc::fence_after();
    // product k is done, so stage s is free: the first warp past it copies
    // tile k + 2 there (the row tile only when the row changes)
    if (lane == 0 && k + 2 < nk && atomicAdd(passed + s, 1u) % kMtWarps == 0u) load(k + 2, tl, tl.x != tj.x);

    uint32_t r0[32], r1[32];
    tc::tmem_ld32(tbase + lane_off + 128 * s + c0, r0);
    tc::tmem_ld32(tbase + lane_off + 128 * s + c0 + 32, r1);
    tc::tmem_wait_ld();
    tc::fence_before();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(bars + 4 + s);
    const int2 tj_next = k + 1 < nk ? tiles[f0 + k + 1] : tj;
    // the last warp to release accumulator s issues the product of tile
    // k + 2 into it, once the release barrier (every warp's loads) and the
    // copy have completed
    uint32_t rel = 0u;
    if (lane == 0 && k + 2 < nk) rel = atomicAdd(released + s, 1u);
    rel = __shfl_sync(0xffffffffu, rel, 0);
    if (k + 2 < nk && rel % kMtWarps == kMtWarps - 1) {
      bool w2 = tc::mbar_test(bars + 4 + s, (uint32_t)(k >> 1) & 1u) ||
                tc::mbar_wait(bars + 4 + s, (uint32_t)(k >> 1) & 1u, wait_limit);
      if (w2)
        w2 = tc::mbar_test(bars + s, (uint32_t)((k + 2) >> 1) & 1u) ||
             tc::mbar_wait(bars + s, (uint32_t)((k + 2) >> 1) & 1u, wait_limit);
      ok = __all_sync(0xffffffffu, w2) != 0;
      if (!ok) break;
      issue(k + 2);
    }
    const int i = tj.x * kMtRows + quarter * 32 + lane;
    const bool diag = tj.x == tj.y;
    const bool full = !diag && (tj.y + 1) * kMtRows <= N && (tj.x + 1) * kMtRows <= N;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t(&r)[32] = h ? r1 : r0;
      const int jb = tj.y * kMtRows + c0 + 32 * h;
      // valid columns q of this chunk: [jmin, jmax)
      const int jmax = full ? 32 : (i < N ? min(32, N - jb) : 0);
      const int jmin = diag ? (i - jb + 1) : 0;
      if (mode == 0) {
        unsigned int inmask = 0u;
        if (full) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float d = __uint_as_float(r[q]);
            const bool b = d < lo;
            below += b ? 1u : 0u;
            inmask |= (!b && d <= hi) ? (1u << q) : 0u;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float d = __uint_as_float(r[q]);
            const bool valid = q < jmax && q >= jmin;
            const bool b = d < lo;
            below += (valid && b) ? 1u : 0u;
            inmask |= (valid && !b && d <= hi) ? (1u << q) : 0u;
          }
        }
        // warp-aggregated append to this warp's buffer
        const unsigned int mine = __popc(inmask);
        unsigned int incl = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += o;
        }
        const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
          if (cnt + total > (unsigned)kMtCandW) flush();
          unsigned int pos = cnt + incl - mine;
          if (inmask) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (inmask & (1u << q)) wbuf[pos++] = __uint_as_float((unsigned int)max((int)r[q], 0));
          }
          __syncwarp();
          cnt += total;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const unsigned int bits = (unsigned int)max((int)r[q], 0);
          // pairs with a particle that sits out the step are NaN
          if (q < jmax && q >= jmin && (r[q] & 0x7fffffffu) <= 0x7f800000u) {
            if (pass == 0) atomicAdd(&hist[bits >> 21], 1u);
            else if (pass == 1) { if ((bits >> 21) == prefix) atomicAdd(&hist[(bits >> 10) & 2047u], 1u); }
            else if ((bits >> 10) == prefix) atomicAdd(&hist[bits & 1023u], 1u);
          }
        }
      }
    }
    tj = tj_next;
  }
  if (!ok && lane == 0) {
    ctl->tc_error = 1;
    *failed = 1u;
  }

  if (mode == 0) {
    if (cnt) flush();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) below += __shfl_xor_sync(0xffffffffu, below, off);
    if (lane == 0 && below) atomicAdd(&ctl->below, (unsigned long long)below);
  }
  __syncthreads();
  if (*failed) {
    // a warp gave up: let the copies and products in flight finish (bounded)
    // before the shared memory and TMEM are released
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (my_load[s] >= 0) tc::mbar_wait(bars + s, (uint32_t)(my_load[s] >> 1) & 1u, kDrainLimit);
      if (my_mma[s] >= 0) tc::mbar_wait(bars + 2 + s, (uint32_t)(my_mma[s] >> 1) & 1u, kDrainLimit);
    }
  }
  __syncthreads();
  if (mode != 0) {
    for (int b = t; b < kMtBins; b += kMtThreads) {
      const unsigned int h = hist[b];
      if (h) atomicAdd(&ctl->hist[b], h);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// Upper-triangle tiles (I, J), J >= I, in row-major order; returns their
// number and writes them to out (2 ints each) when out is not NULL.
int median_tc_work_items(int N, int* out) {
  const int nt = (N + kMtRows - 1) / kMtRows;
  int n = 0;
  for (int I = 0; I < nt; ++I)
    for (int J = I; J < nt; ++J) {
      if (out) { out[2 * n] = I; out[2 * n + 1] = J; }
      ++n;
    }
  return n;
}

size_t median_tc_floats(int N, int M) {
  const size_t nt = (size_t)(N + kMtRows - 1) / kMtRows;
  const int MM = M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 10 ? 10 : M <= 12 ? 12 : 16;
  const int KA = ((MM + 2 + 7) / 8) * 8;  // as MtDims<MM>
  return 2 * nt * (size_t)(2 * kMtRows * KA);
}

template <int MM>
static cudaError_t median_tc_mm(int N, int M, const float* u, float* img, const int* work, int n_work, SvgdCtl* ctl,
                                float* cand, unsigned long long cap, int mode, int only_in_fallback, bool prep,
                                int wait_limit, cudaStream_t st) {
  using D = MtDims<MM>;
  const int Npad = (N + kMtRows - 1) / kMtRows * kMtRows;
  const int nt = Npad / kMtRows;
  float* imgA = img;
  float* imgB = img + (size_t)nt * (D::kTile / 4);
  if (prep)
    launch_pdl(median_tc_prep_kernel<MM>, dim3((Npad + 127) / 128), dim3(128), 0, st, N, Npad, M, u, imgA, imgB,
               (const SvgdCtl*)ctl, only_in_fallback);
  // per device: shared-memory opt-in and the persistent grid (resident CTAs
  // per SM, at most 2: each holds 256 of the SM's 512 TMEM columns)
  static int grid_of[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (grid_of[dev] == 0) {
    cudaError_t e =
        cudaFuncSetAttribute(median_tc_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, D::kBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(median_tc_kernel<MM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the kernel's registers and shared memory
    // (the maximum shared-memory carveout is requested above)
    int sms = 0, smem_sm = 0, smem_rsv = 0;
    cudaFuncAttributes fa;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, median_tc_kernel<MM>)) != cudaSuccess)
      return e;
    const int regs = (fa.numRegs + 7) / 8 * 8;
    const int by_regs = 65536 / (regs * kMtThreads);
    const int by_smem = smem_sm / (D::kBytes + smem_rsv);
    int per_sm = by_regs < by_smem ? by_regs : by_smem;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid_of[dev] = sms * (per_sm < 2 ? per_sm : 2);
  }
  const int grid = n_work < grid_of[dev] ? n_work : grid_of[dev];
  if (grid < 1) return cudaSuccess;
  launch_pdl(median_tc_kernel<MM>, dim3(grid), dim3(kMtThreads), D::kBytes, st, N, imgA, imgB, reinterpret_cast<const int2*>(work),
                                                           n_work, ctl, cand, cap, mode, only_in_fallback,
                                                           wait_limit);
  return cudaGetLastError();
}

cudaError_t launch_median_tc(int N, int M, const float* u, float* img, const int* work, int n_work, SvgdCtl* ctl,
                             float* cand, unsigned long long cap, int mode, int only_in_fallback, bool prep,
                             int wait_limit, cudaStream_t st) {
  if (M <= 2) return median_tc_mm<2>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, wait_limit, st);
  if (M <= 4) return median_tc_mm<4>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, wait_limit, st);
  if (M <= 8) return median_tc_mm<8>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, wait_limit, st);
  if (M <= 10) return median_tc_mm<10>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, wait_limit, st);
  if (M <= 12) return median_tc_mm<12>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, wait_limit, st);
  return median_tc_mm<16>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, wait_limit, st);
}

}  // namespace pds
