// SVGD direction phi (Eq. 1) on the tensor cores.
//
// With n_j = |u_j|^2 and L = log2(e) / bw, the kernel value is
//   k_ij = exp(-|u_i - u_j|^2 / bw) = 2^(a_i . b_j),
//   a_i = (2L u_i, -L n_i, -L),  b_j = (u_j, 1, n_j),
// so the exponents of a 128 x 128 tile are one small matrix product
// (K = M + 2, padded to a multiple of 8) computed by tcgen05.mma into tensor
// memory.  The sums phi needs are a second product with the kernel tile:
//   O_i = sum_j k_ij v_j,  v_j = (g_j, u_j, 1),
//   phi_i = O_g + (2/bw) (u_i O_1 - O_u)            (times 1/N later).
// Both products run in kind::tf32 with fp32 accumulation; every operand is
// split into a tf32 high part and a tf32 remainder so the products keep
// fp32-level accuracy (a.b = ah.bh + ah.bl + al.bh, v = vh + vl).  The
// exponentials are taken on the CUDA cores between the two products, read
// from and written back to tensor memory in place.
//
// The kernel is persistent and warp-specialised: one CTA per SM takes the
// contiguous run [b T / G, (b+1) T / G) of the T = (N/128)^2 tiles (row tile
// I, column tile J) in row-major order.  A producer warp streams the column
// tiles' operands through up to six shared-memory stages (bulk async copies).
// One issuer warp issues the exponent products into the TMEM exponent
// buffers, running ahead of the sixteen exponent warps that turn them into
// kernel values in place; a second issuer warp issues each tile's second
// product into one of two TMEM output accumulators once its kernel values
// are written.  The products are tiny (tens of cycles of tensor work each),
// so the issue latency sets the pace: the two issuers work side by side, each
// runs as a whole converged warp (operands in uniform registers, one lane
// elected per instruction), and they neither divide nor rebuild descriptors
// (a tile's row and column are counted on; descriptors are offsets from one
// base).  When a CTA's run leaves a row
// tile, four of the exponent warps read that row's accumulator and write its
// partial phi to the slot (CTA index - first CTA of the row); the last CTA of
// a row zeroes the slots no CTA used, and the Adam kernel adds the slots in a
// fixed order, so the result is deterministic.
#include <cuda_fp16.h>
#include <math.h>

#include "pds_internal.cuh"
#include "tc.cuh"

namespace pds {

constexpr int kTcRows = 128;

// Column layout (compile-time, MM >= M; unused slots are zero):
//   a, b: [0, MM) coordinates, MM and MM + 1 the norm terms;
//   v:    fp16 high parts [0, MM) scaled gradient, [MM, 2 MM) coordinates,
//         2 MM the constant 1; low parts [2 MM + 1, 3 MM + 1) gradient and
//         [3 MM + 1, 4 MM + 1) coordinates.
template <int MM>
struct TcDims {
  static constexpr int KA = ((MM + 2 + 7) / 8) * 8;         // exponent product depth
  static constexpr int NV = ((4 * MM + 1 + 15) / 16) * 16;  // columns of v (high and low parts)
};

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(tc::to_tf32(x));
  lo = __uint_as_float(tc::to_tf32(x - hi));
}

// Tensor-memory plan (512 columns): NE exponent buffers of 128 columns, then
// two output sets (one per row segment in flight) of NV columns each: the
// second product takes v's fp16 high and low parts as one operand of NV
// columns, so each 16-deep slice of K is a single instruction, and the
// epilogue adds the two parts.  Three exponent buffers let the exponent
// product of tile k+1 queue behind the second product of tile k-1 without
// waiting for it; M = 16 (NV = 80) leaves room for two.
template <int MM>
struct TcAcc {
  static constexpr int NV = TcDims<MM>::NV;
  static constexpr int NE = (3 * 128 + 2 * NV <= 512) ? 3 : 2;
  static constexpr int kOcol = 128 * NE;  // first output column
};

template <int MM>
struct TcSmem {
  static constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  static constexpr int kA = kTcRows * KA * 4;     // one operand tile (128 rows x KA), bytes
  static constexpr int kV = NV * kTcRows * 2;  // one v^T tile in fp16 (high and low parts), bytes
  static constexpr int kStage = 2 * kA + kV;  // b (hi, lo) + v^T of one column tile
  // as many stages as fit (at most 6): the copy of tile k + S - 1 starts when
  // the second product of tile k - 1 frees its stage, so S >= 4 hides its
  // latency behind at least two tiles of work
  static constexpr int kFit = (220 * 1024 - 2 * 2 * kA - 256) / kStage;
  static constexpr int kStages = kFit > 6 ? 6 : (kFit < 2 ? 2 : kFit);
  static constexpr int kBytes = 2 * 2 * kA + kStages * kStage + 256;  // two a slots, the stages, barriers
};

// Byte offset of element (row, k) in a K-major fp16 tile of K_total
// columns: core matrices of 8 rows x 8 elements (128 B), consecutive along K
// (leading byte offset 128), then along rows (stride byte offset 16 K_total).
__host__ __device__ __forceinline__ uint32_t kmajor_offset16(int row, int k, int K_total) {
  return (uint32_t)((row >> 3) * (K_total >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Power-of-two scale of a gradient component for fp16: the exponent s with
// max |g| 2^-s < 2^14 (0 for zero, subnormal or non-finite maxima).
__device__ __forceinline__ int phi_g_shift(unsigned int gmax_bits) {
  const int E = (int)((gmax_bits >> 23) & 0xFFu);
  if (E == 0 || E == 255) return 0;
  return E - 126 - 14;
}

// Operand tiles for every particle, written directly in the shared-memory
// image the products read (K-major core-matrix layout), one image per tile
// of 128 particles: imgA[tile] = (a hi, a lo), imgBV[tile] = (b hi, b lo,
// v^T hi, v^T lo).  Rows N .. Npad-1 are zero (their v is 0, so they add
// nothing).
template <int MM>
__global__ void phi_tc_prep_kernel(int N, int Npad, int M, const float* __restrict__ u, const float* __restrict__ gu,
                                   const SvgdCtl* __restrict__ ctl, float* __restrict__ imgA,
                                   float* __restrict__ imgBV) {
  PDS_PDL_ENTRY();
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  using SM = TcSmem<MM>;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Npad) return;
  float x[MM], g[MM];
  float n = 0.f, L = 0.f;
  // a particle that sits out the step (u is NaN) is treated as padding
  bool live = j < N && isfinite(u[(size_t)(j < N ? j : 0)]);
  if (live) L = 1.4426950408889634f / ctl->bw;
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    const bool on = live && k < M;
    x[k] = on ? u[(size_t)k * N + j] : 0.f;
    g[k] = on ? gu[(size_t)k * N + j] : 0.f;
    n = fmaf(x[k], x[k], n);
  }
  const int tile = j / kTcRows, r = j % kTcRows;
  float* A = imgA + (size_t)tile * (2 * SM::kA / 4);
  float* BV = imgBV + (size_t)tile * (SM::kStage / 4);
  float* Bh = BV;
  float* Bl = BV + SM::kA / 4;
  __half* V = reinterpret_cast<__half*>(BV + 2 * SM::kA / 4);
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    const float a = k < MM ? 2.f * L * x[k] : (k == MM ? -L * n : (k == MM + 1 ? -L : 0.f));
    const float b = k < MM ? x[k] : (k == MM ? (live ? 1.f : 0.f) : (k == MM + 1 ? n : 0.f));
    const uint32_t o = tc::kmajor_offset(r, k, KA) >> 2;
    float h, l;
    split_tf32(a, h, l);
    A[o] = h;
    A[SM::kA / 4 + o] = l;
    split_tf32(b, h, l);
    Bh[o] = h;
    Bl[o] = l;
  }
  // v = (g 2^-s, u, 1) in fp16 high parts, then the low parts of g 2^-s and u
#pragma unroll
  for (int c = 0; c < 2 * MM; ++c) {
    const float v = c < MM ? ldexpf(g[c], -phi_g_shift(ctl->gmax[c])) : x[c - MM];
    const __half h = __float2half_rn(v);
    V[kmajor_offset16(c, r, kTcRows) >> 1] = h;
    V[kmajor_offset16(2 * MM + 1 + c, r, kTcRows) >> 1] = __float2half_rn(v - __half2float(h));
  }
  V[kmajor_offset16(2 * MM, r, kTcRows) >> 1] = __float2half_rn(live ? 1.f : 0.f);
#pragma unroll
  for (int c = 4 * MM + 1; c < NV; ++c) V[kmajor_offset16(c, r, kTcRows) >> 1] = __float2half_rn(0.f);
}

constexpr int kPhiExpWarps = 16;                      // 4 lane quarters x 4 column quarters
constexpr int kPhiGramWarp = kPhiExpWarps;            // warp issuing the exponent products
constexpr int kPhiPvWarp = kPhiExpWarps + 1;          // warp issuing the second products
constexpr int kPhiProducer = kPhiExpWarps + 2;        // warp streaming the operands
constexpr int kPhiThreads = 32 * (kPhiExpWarps + 3);
constexpr int kPhiEpiWarp0 = 12;                      // warps 12..15 (column quarter 3) read the outputs

// First CTA whose run [b T / G, (b+1) T / G) contains tile x.
__host__ __device__ inline int phi_tc_first_cta(long long x, long long T, int G) {
  return (int)(((x + 1) * G + T - 1) / T) - 1;
}

template <int MM>
__global__ void __launch_bounds__(kPhiThreads, 1) phi_tc_kernel(int N, int Npad, int M, const float* __restrict__ imgA,
                                                                const float* __restrict__ imgBV,
                                                                const float* __restrict__ u,
                                                                SvgdCtl* __restrict__ ctl, float* __restrict__ phi_part,
                                                                int slots, int wait_limit) {
  PDS_PDL_ENTRY();
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  using SM = TcSmem<MM>;
  constexpr int S = SM::kStages;
  constexpr int NE = TcAcc<MM>::NE;
  // wait_limit: mbarrier polls before a wait gives up (the kernel then
  // flags ctl->tc_error); the waits that let copies and products in flight
  // finish before shared memory and TMEM are released take kDrainLimit
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                       // two a slots (hi | lo), by row parity
  unsigned char* sStage = smem + 2 * 2 * SM::kA;  // S stages of (b hi | b lo | v hi | v lo)
  uint64_t* bars = (uint64_t*)(sStage + S * SM::kStage);
  uint64_t* full = bars;             // [S]   operands of a tile landed
  uint64_t* s_free = full + S;       // [S]   a stage's second product done (the stage may be refilled)
  uint64_t* g_done = s_free + S;     // [NE]  exponent product done
  uint64_t* p_ready = g_done + NE;   // [NE]  kernel values written (16 warps)
  uint64_t* pv_done = p_ready + NE;  // [NE]  second product done
  uint64_t* o_ready = pv_done + NE;  // [2]   a row segment's outputs complete
  uint64_t* o_free = o_ready + 2;    // [2]   a row segment's outputs read (4 warps)
  uint32_t* tslot = (uint32_t*)(o_free + 2);
  static_assert((2 * 6 + 3 * 3 + 4) * 8 + 4 <= 256, "barriers exceed their 256 bytes");

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nt = Npad / kTcRows;
  const long long T = (long long)nt * nt;
  const int G = gridDim.x;
  const int f0 = (int)(((long long)blockIdx.x * T) / G);
  const int f1 = (int)(((long long)(blockIdx.x + 1) * T) / G);
  const int nk = f1 - f0;
  const int I0 = f0 / nt, J0 = f0 % nt;  // first tile's row and column; later tiles are counted on
  // Stages in use.  The copy of a row's first tile j rewrites the a slot of
  // the row two back.  The ring orders that copy after the second product of
  // tile j - Se, which was issued only once the exponent products of tiles
  // <= j - Se had completed; the row two back ends at tile j - nt - 1 or
  // earlier, so Se <= nt + 1 keeps the slot until its last reader is done.
  const int Se = S < nt + 1 ? S : nt + 1;

  if (t == 0) {
    for (int b = 0; b < S; ++b) {
      tc::mbar_init(full + b, 1);
      tc::mbar_init(s_free + b, 1);
    }
    for (int b = 0; b < NE; ++b) {
      tc::mbar_init(g_done + b, 1);
      tc::mbar_init(p_ready + b, kPhiExpWarps);
      tc::mbar_init(pv_done + b, 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(o_ready + b, 1);
      tc::mbar_init(o_free + b, 4);
    }
  }
  if (warp == 0) tc::tmem_alloc(tslot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  bool ok = true;
  // waits that are usually already complete test the barrier first
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    return tc::mbar_test(bar, parity) || tc::mbar_wait(bar, parity, wait_limit);
  };

  if (warp == kPhiProducer) {
    // ------------------------------------------------------------ producer
    // operands of tile k into stage k mod Se once the second product of tile
    // k - Se left it (a with the row's first tile)
    if (lane == 0 && nk > 0) {
      int I = I0, J = J0, st = 0, last = -1;
      uint32_t ph = 0;  // parity of this use of stage st: (k / Se) & 1
      for (int k = 0; k < nk; ++k) {
        if (k >= Se && !wait(s_free + st, ph ^ 1u)) {
          ok = false;
          break;
        }
        const bool needA = (k == 0) || (J == 0);
        tc::mbar_expect_tx(full + st, SM::kStage + (needA ? 2 * SM::kA : 0));
        if (needA)
          tc::bulk_g2s(sA + ((I - I0) & 1) * 2 * SM::kA, imgA + (size_t)I * (2 * SM::kA / 4), 2 * SM::kA, full + st);
        tc::bulk_g2s(sStage + st * SM::kStage, imgBV + (size_t)J * (SM::kStage / 4), SM::kStage, full + st);
        last = k;
        if (++J == nt) {
          J = 0;
          ++I;
        }
        if (++st == Se) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (!ok) {
        ctl->tc_error = 1;
        // let the copies in flight land (bounded) before shared memory is released
        for (int k = last - Se + 1 > 0 ? last - Se + 1 : 0; k <= last; ++k)
          tc::mbar_wait(full + k % Se, (uint32_t)(k / Se) & 1u, kDrainLimit);
      }
    }
  } else if (warp == kPhiGramWarp || warp == kPhiPvWarp) {
    // ------------------------------------------------------------ issuers
    if (nk > 0) {
      auto wait = [&](uint64_t* bar, uint32_t parity) {
        const bool w = tc::mbar_test(bar, parity) || tc::mbar_wait(bar, parity, wait_limit);
        return __all_sync(0xffffffffu, w) != 0;
      };
      const uint32_t s0 = tc::smem_u32(smem);
      constexpr uint32_t oA = 0, oS = 2 * 2 * SM::kA;  // offsets of the a slots and the stages
      int last = -1;
      if (warp == kPhiGramWarp) {
        // exponent product of tile k into buffer k % NE once the second
        // product of tile k - NE left it and the operands landed
        const uint64_t dG = tc::smem_desc(s0, 128, 32 * KA);
        int st = 0, slot = 0, J = J0;
        uint32_t ph = 0;
        for (int k = 0; k < nk; ++k) {
          if (k >= NE) ok = wait(pv_done + (k - NE) % NE, (uint32_t)((k - NE) / NE) & 1u);
          if (ok) ok = wait(full + st, ph);
          if (!ok) break;
          tc::fence_after();
          constexpr uint32_t id = tc::idesc_tf32(128, 128);
          const uint64_t a_h = dG + ((oA + slot * 2 * SM::kA) >> 4), a_l = a_h + (SM::kA >> 4);
          const uint64_t b_h = dG + ((oS + st * SM::kStage) >> 4), b_l = b_h + (SM::kA >> 4);
          const uint64_t Aop[3] = {a_h, a_h, a_l};
          const uint64_t Bop[3] = {b_h, b_l, b_h};
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int ks = 0; ks < KA / 8; ++ks)
              tc::mma_ss_el(tbase + 128 * (k % NE), Aop[p] + ks * 16, Bop[p] + ks * 16, id,
                            (p > 0 || ks > 0) ? 1u : 0u);
          tc::mma_commit_el(g_done + k % NE);
          last = k;
          if (++J == nt) {
            J = 0;
            slot ^= 1;
          }
          if (++st == Se) {
            st = 0;
            ph ^= 1u;
          }
        }
        if (!ok) {
          if (lane == 0) ctl->tc_error = 1;
          if (last >= 0) tc::mbar_wait(g_done + last % NE, (uint32_t)(last / NE) & 1u, kDrainLimit);
        }
      } else {
        // second product of tile k once every exponent warp wrote its kernel
        // values (and the output set was read for segment seg - 2)
        const uint64_t dV = tc::smem_desc(s0, 128, 16 * kTcRows);
        int st = 0, J = J0, seg = 0;
        for (int k = 0; k < nk; ++k) {
          if (k > 0 && J == 0) ++seg;
          const bool first = (k == 0) || (J == 0);
          const bool lst = (k == nk - 1) || (J == nt - 1);
          ok = wait(p_ready + k % NE, (uint32_t)(k / NE) & 1u);
          if (ok && first && seg >= 2) ok = wait(o_free + (seg & 1), (uint32_t)((seg - 2) >> 1) & 1u);
          if (!ok) break;
          tc::fence_after();
          constexpr uint32_t id = tc::idesc_f16(128, NV);
          const uint64_t v_h = dV + ((oS + st * SM::kStage + 2 * SM::kA) >> 4);
          const uint32_t tE = tbase + 128 * (k % NE), tO = tbase + TcAcc<MM>::kOcol + NV * (seg & 1);
#pragma unroll
          for (int ks = 0; ks < kTcRows / 16; ++ks)
            tc::mma_ts_f16_el(tO, tE + 32 * (ks >> 1) + 8 * (ks & 1), v_h + ks * 16, id,
                              (!first || ks > 0) ? 1u : 0u);
          tc::mma_commit_el(pv_done + k % NE);
          tc::mma_commit_el(s_free + st);
          if (lst) tc::mma_commit_el(o_ready + (seg & 1));
          last = k;
          if (++J == nt) J = 0;
          if (++st == Se) st = 0;
        }
        if (!ok) {
          if (lane == 0) ctl->tc_error = 1;
          if (last >= 0) tc::mbar_wait(pv_done + last % NE, (uint32_t)(last / NE) & 1u, kDrainLimit);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ exponent warps
    const int quarter = warp & 3, cq = warp >> 2;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const bool epi = warp >= kPhiEpiWarp0;
    int seg = 0, I = I0, J = J0;  // tile k's row segment, row and column
    for (int k = 0; k < nk; ++k) {
      if (k > 0 && J == 0) ++seg;
      const bool w = tc::mbar_test(g_done + k % NE, (uint32_t)(k / NE) & 1u) ||
                     tc::mbar_wait(g_done + k % NE, (uint32_t)(k / NE) & 1u, wait_limit);
      ok = __all_sync(0xffffffffu, w) != 0;
      if (!ok) break;
      tc::fence_after();
      const uint32_t tE = tbase + 128 * (k % NE) + lane_off + 32 * cq;
      uint32_t r[32];
      tc::tmem_ld32(tE, r);
      tc::tmem_wait_ld();
      uint32_t pk[16];  // kernel values in fp16, two per column (even j in the low half)
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float e0, e1;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(__uint_as_float(r[2 * q])));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(__uint_as_float(r[2 * q + 1])));
        const __half2 h2 = __floats2half2_rn(e0, e1);
        pk[q] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      tc::tmem_st16(tE, pk);
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(p_ready + k % NE);
      const bool row_end = J == nt - 1;
      const bool last = (k == nk - 1) || row_end;
      if (epi && last) {
        // this row segment's outputs: wait for its last second product, then read them
        const bool w2 = tc::mbar_test(o_ready + (seg & 1), (uint32_t)(seg >> 1) & 1u) ||
                        tc::mbar_wait(o_ready + (seg & 1), (uint32_t)(seg >> 1) & 1u, wait_limit);
        ok = __all_sync(0xffffffffu, w2) != 0;
        if (!ok) break;
        tc::fence_after();
        const uint32_t tO = tbase + TcAcc<MM>::kOcol + NV * (seg & 1) + lane_off;
        float o[NV];
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += 32) {
          uint32_t rr[32];
          tc::tmem_ld32(tO + c0, rr);
          tc::tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (c0 + c < NV) o[c0 + c] = __uint_as_float(rr[c]);
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(o_free + (seg & 1));
        const int i = I * kTcRows + quarter * 32 + lane;
        // slot of this CTA in row I; the row's last CTA zeroes the unused ones
        const int b0 = phi_tc_first_cta((long long)I * nt, T, G);
        const int slot = blockIdx.x - b0;
        if (i < N) {
          const float two_over_bw = 2.0f / ctl->bw;
          const float o1s = o[2 * MM];
#pragma unroll
          for (int c = 0; c < MM; ++c) {
            if (c < M) {
              const float ui = u[(size_t)c * N + i];
              const float og = ldexpf(o[c] + o[2 * MM + 1 + c], phi_g_shift(ctl->gmax[c]));
              const float ou = o[MM + c] + o[3 * MM + 1 + c];
              phi_part[((size_t)slot * M + c) * N + i] = og + two_over_bw * (ui * o1s - ou);
            }
          }
          if (row_end)
            for (int sl = slot + 1; sl < slots; ++sl)
              for (int c = 0; c < M; ++c) phi_part[((size_t)sl * M + c) * N + i] = 0.f;
        }
      }
      if (++J == nt) {
        J = 0;
        ++I;
      }
    }
    if (!ok && lane == 0) ctl->tc_error = 1;
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// Persistent grid of the tensor-core phi: one CTA per SM (each holds all
// 512 TMEM columns), at most one per tile.
static int phi_tc_grid(int N) {
  static int sms_of[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (sms_of[dev] == 0 && cudaDeviceGetAttribute(&sms_of[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  const long long nt = (N + kTcRows - 1) / kTcRows;
  return (int)(nt * nt < sms_of[dev] ? nt * nt : sms_of[dev]);
}

// Number of partial-phi slots: the most CTAs whose runs meet one row tile.
int phi_tc_slots(int N) {
  const int G = phi_tc_grid(N);
  if (G <= 0) return 0;
  const long long nt = (N + kTcRows - 1) / kTcRows, T = nt * nt;
  int most = 1;
  for (long long I = 0; I < nt; ++I) {
    const int n = phi_tc_first_cta((I + 1) * nt - 1, T, G) - phi_tc_first_cta(I * nt, T, G) + 1;
    if (n > most) most = n;
  }
  return most;
}

template <int MM>
static cudaError_t launch_phi_tc_mm(int N, int M, const SvgdWork& w, int* slots_used, cudaStream_t st) {
  using SM = TcSmem<MM>;
  const int Npad = (N + kTcRows - 1) / kTcRows * kTcRows;
  const int ntiles = Npad / kTcRows;
  float* imgA = w.tc;
  float* imgBV = imgA + (size_t)ntiles * (2 * SM::kA / 4);
  const int G = phi_tc_grid(N);
  const int slots = phi_tc_slots(N);
  if (G <= 0 || slots <= 0 || slots > w.chunks) return cudaErrorInvalidConfiguration;
  launch_pdl(phi_tc_prep_kernel<MM>, dim3((Npad + 127) / 128), dim3(128), 0, st, N, Npad, M, w.u, w.gu, w.ctl, imgA, imgBV);
  // at least 116 KB so that two CTAs never share an SM (each allocates all
  // 512 TMEM columns)
  const int smem = SM::kBytes > 116 * 1024 ? SM::kBytes : 116 * 1024;
  static bool attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(phi_tc_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(phi_tc_kernel<MM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  launch_pdl(phi_tc_kernel<MM>, dim3(G), dim3(kPhiThreads), smem, st, N, Npad, M, imgA, imgBV, w.u, w.ctl, w.phi_part, slots,
                                                  w.wait_limit);
  *slots_used = slots;
  return cudaGetLastError();
}

size_t phi_tc_floats(int N, int M) {
  const size_t Npad = (size_t)(N + kTcRows - 1) / kTcRows * kTcRows;
  const int MM = M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 10 ? 10 : M <= 12 ? 12 : 16;
  const int KA = ((MM + 2 + 7) / 8) * 8, NV = ((4 * MM + 1 + 15) / 16) * 16;  // as TcDims<MM>
  return Npad * (4 * (size_t)KA + (size_t)NV / 2);  // a, b (tf32 hi, lo) and v (fp16) per particle
}

cudaError_t launch_phi_tc(int N, int M, const SvgdWork& w, int* slots_used, cudaStream_t st) {
  if (M <= 2) return launch_phi_tc_mm<2>(N, M, w, slots_used, st);
  if (M <= 4) return launch_phi_tc_mm<4>(N, M, w, slots_used, st);
  if (M <= 8) return launch_phi_tc_mm<8>(N, M, w, slots_used, st);
  if (M <= 10) return launch_phi_tc_mm<10>(N, M, w, slots_used, st);
  if (M <= 12) return launch_phi_tc_mm<12>(N, M, w, slots_used, st);
  return launch_phi_tc_mm<16>(N, M, w, slots_used, st);
}

}  // namespace pds
