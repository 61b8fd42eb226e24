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
// from and written back to tensor memory in place.  One CTA owns 128 rows i
// and loops over a chunk of 128-column tiles j; partial sums per chunk are
// added by the Adam kernel.
#include <math.h>

#include "pds_internal.cuh"
#include "tc.cuh"

namespace pds {

constexpr int kTcRows = 128;

// Column layout (compile-time, MM >= M; unused slots are zero):
//   a, b: [0, MM) coordinates, MM and MM + 1 the norm terms;
//   v:    [0, MM) gradient, [MM, 2 MM) coordinates, 2 MM the constant 1.
template <int MM>
struct TcDims {
  static constexpr int KA = ((MM + 2 + 7) / 8) * 8;        // exponent product depth
  static constexpr int NV = ((2 * MM + 1 + 15) / 16) * 16;  // columns of v
};

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(tc::to_tf32(x));
  lo = __uint_as_float(tc::to_tf32(x - hi));
}

template <int MM>
struct TcSmem {
  static constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  static constexpr int kA = kTcRows * KA * 4;   // one operand tile (128 rows x KA), bytes
  static constexpr int kV = NV * kTcRows * 4;   // one v^T tile, bytes
  static constexpr int kStage = 2 * kA + 2 * kV;  // b (hi, lo) + v^T (hi, lo) of one column tile
  static constexpr int kBytes = 2 * kA + 2 * kStage + 128;
};

// Operand tiles for every particle, written directly in the shared-memory
// image the products read (K-major core-matrix layout), one image per tile
// of 128 particles: imgA[tile] = (a hi, a lo), imgBV[tile] = (b hi, b lo,
// v^T hi, v^T lo).  Rows N .. Npad-1 are zero (their v is 0, so they add
// nothing).
template <int MM>
__global__ void phi_tc_prep_kernel(int N, int Npad, int M, const float* __restrict__ u, const float* __restrict__ gu,
                                   const SvgdCtl* __restrict__ ctl, float* __restrict__ imgA,
                                   float* __restrict__ imgBV) {
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  using SM = TcSmem<MM>;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Npad) return;
  float x[MM], g[MM];
  float n = 0.f, L = 0.f;
  const bool live = j < N;
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
  float* Vh = BV + 2 * SM::kA / 4;
  float* Vl = BV + 2 * SM::kA / 4 + SM::kV / 4;
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
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const float v = c < MM ? g[c] : (c < 2 * MM ? x[c - MM] : (c == 2 * MM && live ? 1.f : 0.f));
    const uint32_t o = tc::kmajor_offset(c, r, kTcRows) >> 2;
    float h, l;
    split_tf32(v, h, l);
    Vh[o] = h;
    Vl[o] = l;
  }
}

template <int MM>
__global__ void __launch_bounds__(128, 2) phi_tc_kernel(int N, int Npad, int M, const float* __restrict__ imgA,
                                                        const float* __restrict__ imgBV, const float* __restrict__ u,
                                                        SvgdCtl* __restrict__ ctl, float* __restrict__ phi_part,
                                                        int tiles_per_chunk) {
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  using SM = TcSmem<MM>;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                              // a hi | a lo
  unsigned char* sStage[2] = {smem + 2 * SM::kA, smem + 2 * SM::kA + SM::kStage};
  uint64_t* bars = (uint64_t*)(smem + 2 * SM::kA + 2 * SM::kStage);  // full[0], full[1], a, mma
  uint32_t* tslot = (uint32_t*)(bars + 4);

  const int t = threadIdx.x, warp = t >> 5;
  const int i0 = blockIdx.x * kTcRows;
  const int ntiles = Npad / kTcRows;
  const int jt0 = blockIdx.y * tiles_per_chunk;
  const int jt1 = min(ntiles, jt0 + tiles_per_chunk);
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

  if (t == 0) {
    for (int b = 0; b < 4; ++b) tc::mbar_init(bars + b, 1);
  }
  if (warp == 0) tc::tmem_alloc(tslot, 256);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tE = tbase, tO = tbase + 128;

  // prologue: this CTA's a tile and the first two column tiles
  if (t == 0 && jt1 > jt0) {
    tc::mbar_expect_tx(bars + 2, 2 * SM::kA);
    tc::bulk_g2s(sA, imgA + (size_t)blockIdx.x * (2 * SM::kA / 4), 2 * SM::kA, bars + 2);
    for (int s = 0; s < 2 && jt0 + s < jt1; ++s) {
      tc::mbar_expect_tx(bars + s, SM::kStage);
      tc::bulk_g2s(sStage[s], imgBV + (size_t)(jt0 + s) * (SM::kStage / 4), SM::kStage, bars + s);
    }
  }
  bool ok = true;
  if (jt1 > jt0) ok = __syncthreads_and(tc::mbar_wait(bars + 2, 0, 1 << 24)) != 0;
  uint32_t ph_full[2] = {0u, 0u}, ph_mma = 0u;

  for (int jt = jt0; jt < jt1 && ok; ++jt) {
    const int s = (jt - jt0) & 1;
    ok = __syncthreads_and(tc::mbar_wait(bars + s, ph_full[s], 1 << 24)) != 0;
    ph_full[s] ^= 1;
    if (!ok) break;
    const unsigned char* sB = sStage[s];
    const unsigned char* sV = sStage[s] + 2 * SM::kA;
    // exponents E = a b^T (three split products)
    if (t == 0) {
      tc::fence_after();
      constexpr uint32_t id = tc::idesc_tf32(128, 128);
      const uint32_t sbo = 32 * KA;
      const uint32_t a_h = tc::smem_u32(sA), a_l = a_h + SM::kA;
      const uint32_t b_h = tc::smem_u32(sB), b_l = b_h + SM::kA;
      const uint32_t Aop[3] = {a_h, a_h, a_l};
      const uint32_t Bop[3] = {b_h, b_l, b_h};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int ks = 0; ks < KA / 8; ++ks)
          tc::mma_ss(tE, tc::smem_desc(Aop[p] + ks * 256, 128, sbo), tc::smem_desc(Bop[p] + ks * 256, 128, sbo), id,
                     (p > 0 || ks > 0) ? 1u : 0u);
      tc::mma_commit(bars + 3);
    }
    ok = __syncthreads_and(tc::mbar_wait(bars + 3, ph_mma, 1 << 24)) != 0;
    ph_mma ^= 1;
    tc::fence_after();
    if (!ok) break;
    // kernel values k = 2^E, rounded to tf32, written back in place
#pragma unroll
    for (int c0 = 0; c0 < 128; c0 += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tE + lane_off + c0, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 32; ++k) r[k] = tc::to_tf32(exp2f(__uint_as_float(r[k])));
      tc::tmem_st32(tE + lane_off + c0, r);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    __syncthreads();
    // O += K v (v split in two); then refill this stage with tile jt + 2
    if (t == 0) {
      tc::fence_after();
      constexpr uint32_t id = tc::idesc_tf32(128, NV);
      const uint32_t sbo = 32 * kTcRows;
      const uint32_t v_h = tc::smem_u32(sV), v_l = v_h + SM::kV;
#pragma unroll
      for (int ks = 0; ks < kTcRows / 8; ++ks)
        tc::mma_ts(tO, tE + ks * 8, tc::smem_desc(v_h + ks * 256, 128, sbo), id, (jt > jt0 || ks > 0) ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < kTcRows / 8; ++ks)
        tc::mma_ts(tO, tE + ks * 8, tc::smem_desc(v_l + ks * 256, 128, sbo), id, 1u);
      tc::mma_commit(bars + 3);
    }
    ok = __syncthreads_and(tc::mbar_wait(bars + 3, ph_mma, 1 << 24)) != 0;
    ph_mma ^= 1;
    tc::fence_after();
    if (t == 0 && ok && jt + 2 < jt1) {
      tc::mbar_expect_tx(bars + s, SM::kStage);
      tc::bulk_g2s(sStage[s], imgBV + (size_t)(jt + 2) * (SM::kStage / 4), SM::kStage, bars + s);
    }
  }

  const int i = i0 + t;
  if (jt1 > jt0 && ok) {
    float o[64];
#pragma unroll
    for (int c0 = 0; c0 < NV; c0 += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tO + lane_off + c0, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 32; ++k) o[c0 + k] = __uint_as_float(r[k]);
    }
    if (i < N) {
      const float two_over_bw = 2.0f / ctl->bw;
      const float o1 = o[2 * MM];
#pragma unroll
      for (int k = 0; k < MM; ++k) {
        if (k < M) {
          const float ui = u[(size_t)k * N + i];
          phi_part[((size_t)blockIdx.y * M + k) * N + i] = o[k] + two_over_bw * (ui * o1 - o[MM + k]);
        }
      }
    }
  } else if (jt1 > jt0) {
    if (t == 0) ctl->tc_error = 1;
  } else if (i < N) {
    // empty chunk: contributes zeros
    for (int k = 0; k < M; ++k) phi_part[((size_t)blockIdx.y * M + k) * N + i] = 0.f;
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

template <int MM>
static cudaError_t launch_phi_tc_mm(int N, int M, const SvgdWork& w, int chunks, cudaStream_t st) {
  using SM = TcSmem<MM>;
  const int Npad = (N + kTcRows - 1) / kTcRows * kTcRows;
  const int ntiles = Npad / kTcRows;
  const int tiles_per_chunk = (ntiles + chunks - 1) / chunks;
  float* imgA = w.tc;
  float* imgBV = imgA + (size_t)ntiles * (2 * SM::kA / 4);
  phi_tc_prep_kernel<MM><<<(Npad + 127) / 128, 128, 0, st>>>(N, Npad, M, w.u, w.gu, w.ctl, imgA, imgBV);
  const int smem = SM::kBytes;
  static bool attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(phi_tc_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  dim3 grid(ntiles, chunks);
  phi_tc_kernel<MM><<<grid, 128, smem, st>>>(N, Npad, M, imgA, imgBV, w.u, w.ctl, w.phi_part, tiles_per_chunk);
  return cudaGetLastError();
}

size_t phi_tc_floats(int N, int M) {
  const size_t Npad = (size_t)(N + kTcRows - 1) / kTcRows * kTcRows;
  const int MM = M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 10 ? 10 : 16;
  const int KA = ((MM + 2 + 7) / 8) * 8, NV = ((2 * MM + 1 + 15) / 16) * 16;  // as TcDims<MM>
  return Npad * (4 * (size_t)KA + 2 * (size_t)NV);
}

cudaError_t launch_phi_tc(int N, int M, const SvgdWork& w, int chunks, cudaStream_t st) {
  if (M <= 2) return launch_phi_tc_mm<2>(N, M, w, chunks, st);
  if (M <= 4) return launch_phi_tc_mm<4>(N, M, w, chunks, st);
  if (M <= 8) return launch_phi_tc_mm<8>(N, M, w, chunks, st);
  if (M <= 10) return launch_phi_tc_mm<10>(N, M, w, chunks, st);
  return launch_phi_tc_mm<16>(N, M, w, chunks, st);
}

}  // namespace pds
