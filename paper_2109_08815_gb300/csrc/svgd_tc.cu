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

// Operand rows for every particle (rows N .. Npad-1 are zero: their v is 0,
// so they add nothing).
template <int MM>
__global__ void phi_tc_prep_kernel(int N, int Npad, int M, const float* __restrict__ u, const float* __restrict__ gu,
                                   const SvgdCtl* __restrict__ ctl, float* __restrict__ ah, float* __restrict__ al,
                                   float* __restrict__ bh, float* __restrict__ bl, float* __restrict__ vh,
                                   float* __restrict__ vl) {
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
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
  float a[KA], b[KA], v[NV];
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    a[k] = k < MM ? 2.f * L * x[k] : (k == MM ? -L * n : (k == MM + 1 ? -L : 0.f));
    b[k] = k < MM ? x[k] : (k == MM ? (live ? 1.f : 0.f) : (k == MM + 1 ? n : 0.f));
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = k < MM ? g[k] : (k < 2 * MM ? x[k - MM] : (k == 2 * MM && live ? 1.f : 0.f));
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    float h, l;
    split_tf32(a[k], h, l);
    ah[(size_t)j * KA + k] = h;
    al[(size_t)j * KA + k] = l;
    split_tf32(b[k], h, l);
    bh[(size_t)j * KA + k] = h;
    bl[(size_t)j * KA + k] = l;
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float h, l;
    split_tf32(v[k], h, l);
    vh[(size_t)j * NV + k] = h;
    vl[(size_t)j * NV + k] = l;
  }
}

template <int MM>
struct TcSmem {
  static constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  static constexpr int kA = kTcRows * KA * 4;   // one operand tile of rows x KA
  static constexpr int kV = NV * kTcRows * 4;   // v^T tile
  static constexpr int kBytes = 4 * kA + 2 * kV + 64;
};

template <int MM>
__global__ void __launch_bounds__(128, 2) phi_tc_kernel(int N, int Npad, int M, const float* __restrict__ ah,
                                                        const float* __restrict__ al, const float* __restrict__ bh,
                                                        const float* __restrict__ bl, const float* __restrict__ vh,
                                                        const float* __restrict__ vl, const float* __restrict__ u,
                                                        SvgdCtl* __restrict__ ctl, float* __restrict__ phi_part,
                                                        int tiles_per_chunk) {
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  using SM = TcSmem<MM>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* sAh = (float*)(smem);
  float* sAl = (float*)(smem + SM::kA);
  float* sBh = (float*)(smem + 2 * SM::kA);
  float* sBl = (float*)(smem + 3 * SM::kA);
  float* sVh = (float*)(smem + 4 * SM::kA);
  float* sVl = (float*)(smem + 4 * SM::kA + SM::kV);
  uint64_t* mbar = (uint64_t*)(smem + 4 * SM::kA + 2 * SM::kV);
  uint32_t* tslot = (uint32_t*)(smem + 4 * SM::kA + 2 * SM::kV + 16);

  const int t = threadIdx.x, warp = t >> 5;
  const int i0 = blockIdx.x * kTcRows;
  const int ntiles = Npad / kTcRows;
  const int jt0 = blockIdx.y * tiles_per_chunk;
  const int jt1 = min(ntiles, jt0 + tiles_per_chunk);
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

  // this CTA's rows of a (the exponent product's A operand)
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    const uint32_t o = tc::kmajor_offset(t, k, KA) >> 2;
    sAh[o] = ah[(size_t)(i0 + t) * KA + k];
    sAl[o] = al[(size_t)(i0 + t) * KA + k];
  }
  if (t == 0) tc::mbar_init(mbar, 1);
  if (warp == 0) tc::tmem_alloc(tslot, 256);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tE = tbase, tO = tbase + 128;
  uint32_t phase = 0;
  bool ok = true;

  for (int jt = jt0; jt < jt1 && ok; ++jt) {
    const int j0 = jt * kTcRows;
    // stage b (rows j) and v^T of this tile
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      const uint32_t o = tc::kmajor_offset(t, k, KA) >> 2;
      sBh[o] = bh[(size_t)(j0 + t) * KA + k];
      sBl[o] = bl[(size_t)(j0 + t) * KA + k];
    }
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const uint32_t o = tc::kmajor_offset(c, t, kTcRows) >> 2;
      sVh[o] = vh[(size_t)(j0 + t) * NV + c];
      sVl[o] = vl[(size_t)(j0 + t) * NV + c];
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    // exponents E = a b^T (three split products)
    if (t == 0) {
      tc::fence_after();
      constexpr uint32_t id = tc::idesc_tf32(128, 128);
      const uint32_t sbo = 32 * KA;
      const float* Aop[3] = {sAh, sAh, sAl};
      const float* Bop[3] = {sBh, sBl, sBh};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int ks = 0; ks < KA / 8; ++ks)
          tc::mma_ss(tE, tc::smem_desc(tc::smem_u32(Aop[p]) + ks * 256, 128, sbo),
                     tc::smem_desc(tc::smem_u32(Bop[p]) + ks * 256, 128, sbo), id, (p > 0 || ks > 0) ? 1u : 0u);
      tc::mma_commit(mbar);
    }
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase, 1 << 24)) != 0;
    phase ^= 1;
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
    // O += K v (v split in two)
    if (t == 0) {
      tc::fence_after();
      constexpr uint32_t id = tc::idesc_tf32(128, NV);
      const uint32_t sbo = 32 * kTcRows;
#pragma unroll
      for (int ks = 0; ks < kTcRows / 8; ++ks)
        tc::mma_ts(tO, tE + ks * 8, tc::smem_desc(tc::smem_u32(sVh) + ks * 256, 128, sbo), id,
                   (jt > jt0 || ks > 0) ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < kTcRows / 8; ++ks)
        tc::mma_ts(tO, tE + ks * 8, tc::smem_desc(tc::smem_u32(sVl) + ks * 256, 128, sbo), id, 1u);
      tc::mma_commit(mbar);
    }
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase, 1 << 24)) != 0;  // tiles and E free again
    phase ^= 1;
    tc::fence_after();
  }

  if (ok && jt1 > jt0) {
    // O row of this thread: columns [0, NV)
    float o[64];
#pragma unroll
    for (int c0 = 0; c0 < NV; c0 += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tO + lane_off + c0, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 32; ++k) o[c0 + k] = __uint_as_float(r[k]);
    }
    const int i = i0 + t;
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
  } else if (jt1 > jt0 && t == 0) {
    ctl->tc_error = 1;
  }
  if (jt1 <= jt0) {
    // empty chunk: contribute zeros
    const int i = i0 + t;
    if (i < N)
      for (int k = 0; k < M; ++k) phi_part[((size_t)blockIdx.y * M + k) * N + i] = 0.f;
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

template <int MM>
static cudaError_t launch_phi_tc_mm(int N, int M, const SvgdWork& w, int chunks, cudaStream_t st) {
  const int Npad = (N + kTcRows - 1) / kTcRows * kTcRows;
  const int ntiles = Npad / kTcRows;
  const int tiles_per_chunk = (ntiles + chunks - 1) / chunks;
  constexpr int KA = TcDims<MM>::KA, NV = TcDims<MM>::NV;
  float* ah = w.tc;
  float* al = ah + (size_t)Npad * KA;
  float* bh = al + (size_t)Npad * KA;
  float* bl = bh + (size_t)Npad * KA;
  float* vh = bl + (size_t)Npad * KA;
  float* vl = vh + (size_t)Npad * NV;
  phi_tc_prep_kernel<MM><<<(Npad + 127) / 128, 128, 0, st>>>(N, Npad, M, w.u, w.gu, w.ctl, ah, al, bh, bl, vh, vl);
  // at most two CTAs per SM: their tensor-memory allocations (256 columns each) always fit
  const int smem = TcSmem<MM>::kBytes < 100 * 1024 ? 100 * 1024 : TcSmem<MM>::kBytes;
  static bool attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(phi_tc_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  dim3 grid(ntiles, chunks);
  phi_tc_kernel<MM><<<grid, 128, smem, st>>>(N, Npad, M, ah, al, bh, bl, vh, vl, w.u, w.ctl, w.phi_part,
                                             tiles_per_chunk);
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
