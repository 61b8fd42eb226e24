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
// distances.  Tiles: A (row tile) loaded once per CTA, B (column tiles)
// double-buffered by bulk async copies; two TMEM accumulators, so the
// product of the next tile runs while the current one is read.
#include <math.h>

#include "pds_internal.cuh"
#include "tc.cuh"

namespace pds {

constexpr int kMtRows = 128;
constexpr int kMtBins = 2048;
constexpr int kMtCand = 8192;  // shared candidate buffer (floats)

template <int MM>
struct MtDims {
  static constexpr int KA = ((MM + 2 + 7) / 8) * 8;
  static constexpr int kA = kMtRows * KA * 4;          // one tile image (hi or lo), bytes
  static constexpr int kTile = 2 * kA;                  // hi + lo
  static constexpr int kBytes = kTile + 2 * kTile + kMtCand * 4 + 256;
};

__device__ __forceinline__ void mt_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(tc::to_tf32(x));
  lo = __uint_as_float(tc::to_tf32(x - hi));
}

// Tile images (hi, lo) of a_i and b_j for every particle; rows N..Npad-1
// are zero (never counted).
template <int MM>
__global__ void median_tc_prep_kernel(int N, int Npad, int M, const float* __restrict__ u, float* __restrict__ imgA,
                                      float* __restrict__ imgB) {
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
// pass 0..2 histogram.  Work item w: row tile I = work[3w], column tiles
// [work[3w+1], work[3w+2]).
template <int MM>
__global__ void __launch_bounds__(128, 2) median_tc_kernel(int N, const float* __restrict__ imgA,
                                                           const float* __restrict__ imgB,
                                                           const int* __restrict__ work, SvgdCtl* __restrict__ ctl,
                                                           float* __restrict__ cand, unsigned long long cap, int mode,
                                                           int only_in_fallback) {
  using D = MtDims<MM>;
  constexpr int KA = D::KA;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB[2] = {smem + D::kTile, smem + 2 * D::kTile};
  float* buf = (float*)(smem + 3 * D::kTile);              // candidates, or the histogram in radix modes
  uint64_t* bars = (uint64_t*)(smem + 3 * D::kTile + kMtCand * 4);  // full[0], full[1], a, mma[0], mma[1]
  uint32_t* tslot = (uint32_t*)(bars + 5);
  unsigned int* count = tslot + 1;
  unsigned long long* below_blk = (unsigned long long*)(bars + 6);
  unsigned long long* base_sh = below_blk + 1;

  if (only_in_fallback && ctl->mode != 1) return;  // uniform: the bracket held the median
  const int t = threadIdx.x, warp = t >> 5;
  const int I = work[3 * blockIdx.x], J0 = work[3 * blockIdx.x + 1], J1 = work[3 * blockIdx.x + 2];
  const int nJ = J1 - J0;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  unsigned int* hist = (unsigned int*)buf;
  const float lo = ctl->lo, hi = ctl->hi;
  const unsigned int prefix = ctl->prefix;
  const int pass = mode - 1;

  if (mode == 0) {
    if (t == 0) { *count = 0u; *below_blk = 0ull; }
  } else {
    for (int b = t; b < kMtBins; b += 128) hist[b] = 0u;
  }
  if (t == 0)
    for (int b = 0; b < 5; ++b) tc::mbar_init(bars + b, 1);
  if (warp == 0) tc::tmem_alloc(tslot, 256);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;

  if (t == 0 && nJ > 0) {
    tc::mbar_expect_tx(bars + 2, D::kTile);
    tc::bulk_g2s(sA, imgA + (size_t)I * (D::kTile / 4), D::kTile, bars + 2);
    for (int s = 0; s < 2 && s < nJ; ++s) {
      tc::mbar_expect_tx(bars + s, D::kTile);
      tc::bulk_g2s(sB[s], imgB + (size_t)(J0 + s) * (D::kTile / 4), D::kTile, bars + s);
    }
  }
  uint32_t ph_full[2] = {0u, 0u}, ph_mma[2] = {0u, 0u};
  bool ok = true;

  auto issue_gram = [&](int k) {  // thread 0: product of column tile J0 + k into accumulator k % 2
    const int s = k & 1;
    tc::fence_after();
    constexpr uint32_t id = tc::idesc_tf32(128, 128);
    const uint32_t sbo = 32 * KA;
    const uint32_t a_h = tc::smem_u32(sA), a_l = a_h + D::kA;
    const uint32_t b_h = tc::smem_u32(sB[s]), b_l = b_h + D::kA;
    const uint32_t Aop[3] = {a_h, a_h, a_l};
    const uint32_t Bop[3] = {b_h, b_l, b_h};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int ks = 0; ks < KA / 8; ++ks)
        tc::mma_ss(tbase + 128 * s, tc::smem_desc(Aop[p] + ks * 256, 128, sbo),
                   tc::smem_desc(Bop[p] + ks * 256, 128, sbo), id, (p > 0 || ks > 0) ? 1u : 0u);
    tc::mma_commit(bars + 3 + s);
  };

  if (nJ > 0) {
    bool w = true;
    if (t == 0) {
      w = tc::mbar_wait(bars + 2, 0, 1 << 24) && tc::mbar_wait(bars + 0, 0, 1 << 24);
      if (w) issue_gram(0);
    }
    ok = __syncthreads_and(w) != 0;
    ph_full[0] = 1u;
  }
  const int i = I * kMtRows + t;
  unsigned int below = 0u;

  for (int k = 0; k < nJ && ok; ++k) {
    const int s = k & 1;
    // next tile's product while this one is read
    bool w = true;
    if (t == 0 && k + 1 < nJ) {
      const int s1 = (k + 1) & 1;
      w = tc::mbar_wait(bars + s1, ph_full[s1], 1 << 24);
      if (w) issue_gram(k + 1);
    }
    if (k + 1 < nJ) ph_full[(k + 1) & 1] ^= 1u;
    // this tile's product done: its B buffer may be refilled
    w = w && tc::mbar_wait(bars + 3 + s, ph_mma[s], 1 << 24);
    ph_mma[s] ^= 1u;
    ok = __syncthreads_and(w) != 0;
    tc::fence_after();
    if (!ok) break;
    if (t == 0 && k + 2 < nJ) {
      tc::mbar_expect_tx(bars + s, D::kTile);
      tc::bulk_g2s(sB[s], imgB + (size_t)(J0 + k + 2) * (D::kTile / 4), D::kTile, bars + s);
    }
    const int J = J0 + k;
    const bool diag = (J == I);
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tbase + 128 * s + lane_off + c0, r);
      tc::tmem_wait_ld();
      const int jb = J * kMtRows + c0;
      if (mode == 0) {
        // valid pairs of this chunk: j < N and (off the diagonal tile, or j > i)
        const int jmax = min(32, N - jb);
        const int jmin = diag ? (i - jb + 1) : 0;
        unsigned int inmask = 0u;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const float d = fmaxf(__uint_as_float(r[q]), 0.f);
          const bool valid = (q < jmax) && (q >= jmin) && (i < N);
          below += (valid && d < lo) ? 1u : 0u;
          inmask |= (valid && d >= lo && d <= hi) ? (1u << q) : 0u;
        }
        // warp-aggregated append: one shared atomic per warp
        const unsigned int mine = __popc(inmask);
        unsigned int incl = mine;
        const int lane = t & 31;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += o;
        }
        const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned int base = 0u;
        if (lane == 31 && total) base = atomicAdd(count, total);
        base = __shfl_sync(0xffffffffu, base, 31) + (incl - mine);
        if (inmask) {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (inmask & (1u << q)) buf[base++] = fmaxf(__uint_as_float(r[q]), 0.f);
        }
        __syncthreads();
        if (*count > (unsigned)(kMtCand - 128 * 32)) {
          // flush the shared candidates to the global buffer
          const unsigned int nb = *count;
          if (t == 0) *base_sh = atomicAdd(&ctl->inside, (unsigned long long)nb);
          __syncthreads();
          const unsigned long long base = *base_sh;
          for (unsigned int e = t; e < nb; e += 128)
            if (base + e < cap) cand[base + e] = buf[e];
          __syncthreads();
          if (t == 0) *count = 0u;
          __syncthreads();
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const float d = fmaxf(__uint_as_float(r[q]), 0.f);
          const int j = jb + q;
          const bool valid = (i < N) && (j < N) && (!diag || j > i);
          if (valid) {
            const unsigned int bits = __float_as_uint(d);
            if (pass == 0) atomicAdd(&hist[bits >> 21], 1u);
            else if (pass == 1) { if ((bits >> 21) == prefix) atomicAdd(&hist[(bits >> 10) & 2047u], 1u); }
            else if ((bits >> 10) == prefix) atomicAdd(&hist[bits & 1023u], 1u);
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();  // accumulator s free for the product of tile k + 2
  }
  if (!ok && t == 0) ctl->tc_error = 1;

  if (mode == 0) {
    // final flush and the below count
    __syncthreads();
    const unsigned int nb = *count;
    if (t == 0 && nb) *base_sh = atomicAdd(&ctl->inside, (unsigned long long)nb);
    __syncthreads();
    if (nb) {
      const unsigned long long base = *base_sh;
      for (unsigned int e = t; e < nb; e += 128)
        if (base + e < cap) cand[base + e] = buf[e];
    }
    atomicAdd(below_blk, (unsigned long long)below);
    __syncthreads();
    if (t == 0 && *below_blk) atomicAdd(&ctl->below, *below_blk);
  } else {
    __syncthreads();
    for (int b = t; b < kMtBins; b += 128) {
      const unsigned int h = hist[b];
      if (h) atomicAdd(&ctl->hist[b], h);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// Work items over the upper triangle of tiles: (I, J0, J1) with J0 >= I,
// at most `chunk` column tiles each.
int median_tc_work_items(int N, int chunk, int* out) {
  const int nt = (N + kMtRows - 1) / kMtRows;
  int n = 0;
  for (int I = 0; I < nt; ++I)
    for (int J = I; J < nt; J += chunk) {
      if (out) { out[3 * n] = I; out[3 * n + 1] = J; out[3 * n + 2] = J + chunk < nt ? J + chunk : nt; }
      ++n;
    }
  return n;
}

size_t median_tc_floats(int N, int M) {
  const size_t nt = (size_t)(N + kMtRows - 1) / kMtRows;
  const int MM = M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 10 ? 10 : 16;
  const int KA = ((MM + 2 + 7) / 8) * 8;  // as MtDims<MM>
  return 2 * nt * (size_t)(2 * kMtRows * KA);
}

template <int MM>
static cudaError_t median_tc_mm(int N, int M, const float* u, float* img, const int* work, int n_work, SvgdCtl* ctl,
                                float* cand, unsigned long long cap, int mode, int only_in_fallback, bool prep,
                                cudaStream_t st) {
  using D = MtDims<MM>;
  const int Npad = (N + kMtRows - 1) / kMtRows * kMtRows;
  const int nt = Npad / kMtRows;
  float* imgA = img;
  float* imgB = img + (size_t)nt * (D::kTile / 4);
  if (prep) median_tc_prep_kernel<MM><<<(Npad + 127) / 128, 128, 0, st>>>(N, Npad, M, u, imgA, imgB);
  static bool attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e =
        cudaFuncSetAttribute(median_tc_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, D::kBytes);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  median_tc_kernel<MM><<<n_work, 128, D::kBytes, st>>>(N, imgA, imgB, work, ctl, cand, cap, mode, only_in_fallback);
  return cudaGetLastError();
}

cudaError_t launch_median_tc(int N, int M, const float* u, float* img, const int* work, int n_work, SvgdCtl* ctl,
                             float* cand, unsigned long long cap, int mode, int only_in_fallback, bool prep,
                             cudaStream_t st) {
  if (M <= 2) return median_tc_mm<2>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, st);
  if (M <= 4) return median_tc_mm<4>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, st);
  if (M <= 8) return median_tc_mm<8>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, st);
  if (M <= 10) return median_tc_mm<10>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, st);
  return median_tc_mm<16>(N, M, u, img, work, n_work, ctl, cand, cap, mode, only_in_fallback, prep, st);
}

}  // namespace pds
