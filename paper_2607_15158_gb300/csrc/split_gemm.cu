// Split-precision GEMM on the sm_103a tensor cores (tcgen05 + TMA + TMEM).
//
// C = op(A) op(B) for fp64 (or complex fp64) operands, computed as sums of
// low-precision slice products with fp32 accumulation, in one of two
// formats. bf16 x3 (CTM_PREC_SPLIT_BF16):
//   * every fp64 value x is split into three bf16 slices x = s0 + s1 + s2 + e
//     (the slices of x rounded to fp32, each the bf16 rounding of the
//     remainder; |e| <= 2^-24 |x|);
//   * a product keeps the six slice products of order >= 2^-16
//     (s0 t0, s0 t1, s1 t0, s0 t2, s1 t1, s2 t0); the leading s0 t0 is
//     accumulated in its own fp32 accumulator in tensor memory and the five
//     smaller ones in a second, so that their additions cost ulps of a
//     2^-8 smaller running sum, and the two are added once per partial;
// 3xTF32 (CTM_PREC_SPLIT_TF32): x = t0 + t1 + e with tf32 slices of the fp32
// rounding (|e| <= 2^-22 |x|), three products t0 u0 (own accumulator),
// t0 u1 + t1 u0 (second accumulator), tcgen05 kind::tf32 at half the bf16
// rate. Both formats stage 128-byte K rows (64 bf16 or 32 tf32 values), so
// tiles, swizzle and descriptors are shared.
//   * complex data uses the real embedding A_emb = [A_r | A_i] (M x 2K),
//     B_emb = [[B_r, B_i], [-B_i, B_r]] (2K x 2N), C_emb = [C_r | C_i];
//   * K is split over CTAs, at most KB_SPLIT_MAX K blocks of 64 each (the
//     error of an fp32 accumulator grows with the number of MMA steps it
//     takes); fp32 partials are reduced in fp64.
//
// Kernel: one CTA = 128 output rows x BNc (<= 160) output columns; A and B
// slices are K-major, staged by TMA in 64-element (128-byte, 128B-swizzled)
// K blocks through a two-stage mbarrier pipeline; one thread issues the
// tcgen05.mma instructions, four warps drain the accumulator with
// tcgen05.ld. Every mbarrier wait is bounded (2 s of %globaltimer), after
// which the CTA records DEV_MBAR_TIMEOUT, skips its work, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "split_gemm.h"

namespace ctm {

namespace {

constexpr int BM = 128;          // rows per CTA (tcgen05 M)
constexpr int BK = 64;           // bf16 K elements per stage (128 bytes)
constexpr int KROW = 128;        // bytes of one staged K row (either format)
constexpr int STAGES = 2;
constexpr int MAX_BNC = 160;     // columns per CTA
constexpr int A_SLICE_BYTES = BM * KROW;     // 16 KB
constexpr uint64_t WAIT_NS = 2000000000ull;  // bound of every mbarrier wait
#ifndef CTM_KB_SPLIT_MAX
#define CTM_KB_SPLIT_MAX 8
#endif
constexpr int KB_SPLIT_MAX = CTM_KB_SPLIT_MAX;   // K blocks per fp32 partial

// ---------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (globaltimer() - t0 > WAIT_NS) {
      atomicOr(err, DEV_MBAR_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (sm_100 descriptor version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;               // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // SWIZZLE_128B
  return d;
}
// instruction descriptor of kind::f16: bf16 x bf16 -> f32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// instruction descriptor of kind::tf32: tf32 x tf32 -> f32 (format code 2),
// both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// slice formats: NS slices per operand, NP slice products (the first in its
// own accumulator), element bytes EB, K elements per 128-byte row KE
struct FmtBF16 {
  static constexpr int NS = 3, NP = 6, EB = 2, KE = 64;
};
struct FmtTF32 {
  static constexpr int NS = 2, NP = 3, EB = 4, KE = 32;
};

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct MmaParams {
  int M;          // output rows
  int Np;         // padded output columns (row length of the partials)
  int BNc;        // columns per CTA, multiple of 16, <= MAX_BNC
  int kb_total;   // K blocks of 64
  int kb_split;   // K blocks per split
  float* part;    // [nks][M][Np] fp32 partial sums
  int* err;
};

template <typename F>
__global__ void __launch_bounds__(128, 1)
    split_mma_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, MmaParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int BNc = p.BNc;
  const uint32_t b_slice_bytes = (uint32_t)BNc * KROW;
  const uint32_t stage_bytes = F::NS * A_SLICE_BYTES + F::NS * b_slice_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 done = smem_u32(bars + 2 * STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tile = blockIdx.x, chunk = blockIdx.y, ks = blockIdx.z;
  const int kb0 = ks * p.kb_split;
  const int nkb = min(p.kb_split, p.kb_total - kb0);
  // two accumulators of BNc columns each: [0, acc1) for s0 t0, [acc1, ..)
  // for the five smaller slice products
  uint32_t acc1 = 32;
  while ((int)acc1 < BNc) acc1 <<= 1;
  const uint32_t ncols = 2 * acc1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  __shared__ int failed;
  if (threadIdx.x == 0) failed = 0;
  __syncthreads();

  if (nkb > 0 && warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, ((kb / STAGES) - 1) & 1, p.err)) {
        failed = 1;
        break;
      }
      const uint32_t full = full0 + 8 * s;
      mbar_expect_tx(full, stage_bytes);
      uint8_t* st = smem + s * stage_bytes;
      const int kx = (kb0 + kb) * F::KE;
      for (int sl = 0; sl < F::NS; ++sl)
        tma_load_3d(smem_u32(st + sl * A_SLICE_BYTES), &tmA, kx, m_tile * BM, sl, full);
      for (int sl = 0; sl < F::NS; ++sl)
        tma_load_3d(smem_u32(st + F::NS * A_SLICE_BYTES + sl * b_slice_bytes), &tmB, kx,
                    chunk * BNc, sl, full);
    }
  } else if (nkb > 0 && warp == 1 && lane == 0) {
    // MMA issuer: NP slice products per K block, four 32-byte K steps each
    const uint32_t idesc = F::EB == 2 ? idesc_bf16(BM, BNc) : idesc_tf32(BM, BNc);
    const int pa[6] = {0, 0, 1, 0, 1, 2};
    const int pb[6] = {0, 1, 0, 2, 1, 0};
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(full0 + 8 * s, (kb / STAGES) & 1, p.err)) {
        ok = false;
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = smem_u32(smem + s * stage_bytes);
      for (int pr = 0; pr < F::NP; ++pr) {
        const uint32_t a0 = st + pa[pr] * A_SLICE_BYTES;
        const uint32_t b0 = st + F::NS * A_SLICE_BYTES + pb[pr] * b_slice_bytes;
        const uint32_t d = pr == 0 ? tmem : tmem + acc1;
        const bool first = kb == 0 && (pr == 0 || pr == 1);
        for (int kk = 0; kk < KROW / 32; ++kk) {
          if (F::EB == 2)
            mma_bf16(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
                     (first && kk == 0) ? 0u : 1u);
          else
            mma_tf32(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
                     (first && kk == 0) ? 0u : 1u);
        }
      }
      mma_commit(empty0 + 8 * s);
    }
    if (ok) mma_commit(done);
  }
  // epilogue: all four warps, TMEM lanes 32w .. 32w+31 = rows of this warp
  __syncwarp();
  bool have = nkb > 0;
  if (have && !mbar_wait(done, 0, p.err)) have = false;
  __syncthreads();
  if (failed) have = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have) {
    const int row = m_tile * BM + warp * 32 + lane;
    float* out = p.part + ((size_t)ks * p.M + row) * p.Np + (size_t)chunk * BNc;
    for (int c0 = 0; c0 < BNc; c0 += 16) {
      uint32_t r[16], q[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + acc1 + (uint32_t)c0, q);
      if (row < p.M) {
        // 64 contiguous bytes of this thread's row (Np, BNc and c0 are
        // multiples of 16 floats, so the row segment is 64-byte aligned);
        // one rounded addition joins the two accumulators
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __fadd_rn(__uint_as_float(r[i]), __uint_as_float(q[i]));
        float4* o4 = reinterpret_cast<float4*>(out + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          o4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

// ------------------------------------------------------------ slicing
// x -> three bf16 slices of its fp32 rounding xf: s0 + s1 + s2 = xf exactly
// (each remainder has at most 16, then 8 significant bits, so the fp32
// subtractions are exact); |x - xf| <= 2^-24 |x|. One fp64 operation per
// value: GB300's fp64 pipe is ~60x narrower than its fp32 pipe.
__device__ __forceinline__ void split3(double x, __nv_bfloat16& s0, __nv_bfloat16& s1,
                                       __nv_bfloat16& s2) {
  const float xf = f32_of(x);   // integer pipes, not the narrow fp64 pipe
  s0 = __float2bfloat16_rn(xf);
  const float r1 = xf - __bfloat162float(s0);
  s1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(s1);
  s2 = __float2bfloat16_rn(r2);
}

// tf32 rounding of an fp32 value (nearest, ties away from zero): the 13 low
// mantissa bits are dropped after adding half of the last kept bit
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// the NS slices of x in format F (bf16: split3; tf32: t0 = tf32(xf),
// t1 = tf32(xf - t0), the subtraction exact in fp32)
template <typename F> struct SliceT;
template <> struct SliceT<FmtBF16> { using T = __nv_bfloat16; };
template <> struct SliceT<FmtTF32> { using T = float; };

__device__ __forceinline__ void slices_of(FmtBF16, double x, __nv_bfloat16* v) {
  split3(x, v[0], v[1], v[2]);
}
__device__ __forceinline__ void slices_of(FmtTF32, double x, float* v) {
  const float xf = f32_of(x);
  v[0] = tf32_rn(xf);
  v[1] = tf32_rn(xf - v[0]);
}
__device__ __forceinline__ __nv_bfloat16 negv(__nv_bfloat16 a) { return __hneg(a); }
__device__ __forceinline__ float negv(float a) { return -a; }
template <typename T> __device__ __forceinline__ T zero_slice();
template <> __device__ __forceinline__ __nv_bfloat16 zero_slice<__nv_bfloat16>() {
  return __float2bfloat16(0.0f);
}
template <> __device__ __forceinline__ float zero_slice<float>() { return 0.0f; }

template <typename F, typename T>
__device__ __forceinline__ void put_slices(T* out, long slice, long o, const T* v, bool neg) {
#pragma unroll
  for (int i = 0; i < F::NS; ++i) out[i * slice + o] = neg ? negv(v[i]) : v[i];
}


__device__ __forceinline__ void put_digits(__nv_bfloat16* out, long slice, long o,
                                           const __nv_bfloat16* d, bool neg) {
#pragma unroll
  for (int i = 0; i < 8; ++i) out[i * slice + o] = neg ? __hneg(d[i]) : d[i];
}

// A slices: out[s][m][kr], kr < K: Re op(A)(m, kr); K <= kr < 2K: Im
// (complex); zero up to Kp. A 32 x 32 shared tile of op(A) is read along A's
// contiguous axis (rows for op N / R, columns for op T / C) and each element
// is read once and written to both halves.
template <typename T, typename F>
__global__ void prep_a_kernel(const T* A, long lda, int op, int M, int K, int Kp,
                              typename SliceT<F>::T* out) {
  using S = typename SliceT<F>::T;
  __shared__ T tile[32][33];
  constexpr bool cx = sizeof(T) == 16;
  const int Kr = cx ? 2 * K : K;
  const long slice = (long)M * Kp;
  const int tiles_k = (K + 31) / 32, tiles_m = (M + 31) / 32;
  const bool trans = (op == OP_T || op == OP_C);
  const bool cj = (op == OP_C || op == OP_R);
  for (int t = blockIdx.x; t < tiles_k * tiles_m; t += gridDim.x) {
    const int k0 = (t % tiles_k) * 32, m0 = (t / tiles_k) * 32;
    // tile[m - m0][kk - k0] = op(A)(m, kk) before conjugation
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      if (!trans) {
        const int m = m0 + yy, kk = k0 + threadIdx.x;
        tile[yy][threadIdx.x] = (m < M && kk < K) ? A[(long)m * lda + kk] : zero_of(T());
      } else {
        const int kk = k0 + yy, m = m0 + threadIdx.x;
        tile[threadIdx.x][yy] = (m < M && kk < K) ? A[(long)kk * lda + m] : zero_of(T());
      }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      const int m = m0 + yy, kk = k0 + threadIdx.x;
      if (m < M && kk < K) {
        const T v = tile[yy][threadIdx.x];
        S sv[3];
        if constexpr (cx) {
          slices_of(F(), v.x, sv);
          put_slices<F>(out, slice, (long)m * Kp + kk, sv, false);
          slices_of(F(), v.y, sv);
          put_slices<F>(out, slice, (long)m * Kp + K + kk, sv, cj);
        } else {
          slices_of(F(), v, sv);
          put_slices<F>(out, slice, (long)m * Kp + kk, sv, false);
        }
      }
    }
    __syncthreads();
  }
  // padding columns kr >= Kr
  const S z = zero_slice<S>();
  const S zz[3] = {z, z, z};
  const int pc = Kp - Kr;
  const long tid = (long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x * blockDim.y;
  for (long idx = tid; idx < (long)M * pc; idx += nth)
    put_slices<F>(out, slice, (idx / pc) * Kp + Kr + idx % pc, zz, false);
}

// B slices (K-major rows = output real columns): out[s][j][kr] = B_emb[kr][j]
// with B_emb = [[B_r, B_i], [-B_i, B_r]] for complex, B for real. A 32 x 32
// shared tile of op(B) is read along B's contiguous axis and written along
// kr; the padding rows and columns are zeroed.
template <typename T, typename F>
__global__ void prep_b_kernel(const T* B, long ldb, int op, int K, int N, int Kp, int Np,
                              typename SliceT<F>::T* out) {
  using S = typename SliceT<F>::T;
  __shared__ T tile[32][33];
  constexpr bool cx = sizeof(T) == 16;
  const int Kr = cx ? 2 * K : K;
  const int Nr = cx ? 2 * N : N;
  const long slice = (long)Np * Kp;
  const int tk = (K + 31) / 32, tn = (N + 31) / 32;
  const bool trans = (op == OP_T || op == OP_C);
  const bool cj = (op == OP_C || op == OP_R);
  for (int t = blockIdx.x; t < tk * tn; t += gridDim.x) {
    const int k0 = (t % tk) * 32, n0 = (t / tk) * 32;
    // tile[kk - k0][jj - n0] = op(B)(kk, jj) before conjugation
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      if (!trans) {
        const int kk = k0 + yy, jj = n0 + threadIdx.x;
        tile[yy][threadIdx.x] = (kk < K && jj < N) ? B[(long)kk * ldb + jj] : zero_of(T());
      } else {
        const int jj = n0 + yy, kk = k0 + threadIdx.x;
        tile[threadIdx.x][yy] = (kk < K && jj < N) ? B[(long)jj * ldb + kk] : zero_of(T());
      }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      const int jj = n0 + yy, kk = k0 + threadIdx.x;
      if (jj < N && kk < K) {
        const T v = tile[threadIdx.x][yy];
        S re[3], im[3];
        if constexpr (cx) {
          // the slices of -x are the negated slices of x: each part is
          // sliced once
          slices_of(F(), v.x, re);
          slices_of(F(), v.y, im);
          put_slices<F>(out, slice, (long)jj * Kp + kk, re, false);
          put_slices<F>(out, slice, (long)jj * Kp + K + kk, im, !cj);
          put_slices<F>(out, slice, (long)(N + jj) * Kp + kk, im, cj);
          put_slices<F>(out, slice, (long)(N + jj) * Kp + K + kk, re, false);
        } else {
          slices_of(F(), v, re);
          put_slices<F>(out, slice, (long)jj * Kp + kk, re, false);
        }
      }
    }
    __syncthreads();
  }
  const S z = zero_slice<S>();
  const S zz[3] = {z, z, z};
  const long tid = (long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x * blockDim.y;
  // padding rows j >= Nr
  for (long idx = tid; idx < (long)(Np - Nr) * Kp; idx += nth)
    put_slices<F>(out, slice, (long)Nr * Kp + idx, zz, false);
  // padding columns kr >= Kr of the rows j < Nr
  const int pc = Kp - Kr;
  for (long idx = tid; idx < (long)Nr * pc; idx += nth)
    put_slices<F>(out, slice, (idx / pc) * Kp + Kr + idx % pc, zz, false);
}

// error-free sum of two fp32 values (Knuth's TwoSum): hi + lo == a + b
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

// C[m][j] = sum over splits of the partials, complex from [C_r | C_i]. The
// sum is carried as an unevaluated fp32 pair (TwoSum on the fp32 pipe) and
// converted to fp64 once, because this GPU's fp64 pipe (conversions and
// additions alike) would bound the kernel; the pair is exact up to the
// rounding of its low part, ~2^-48 relative.
template <typename T>
__global__ void reduce_kernel(const float* part, int nks, int M, int N, int Np, T* C, long ldc) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)M * N;
       idx += (long)gridDim.x * blockDim.x) {
    const int m = (int)(idx / N), j = (int)(idx % N);
    const float* row = part + (size_t)m * Np + j;
    const size_t sstep = (size_t)M * Np;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    int s = 0;
    // eight splits' loads in flight at a time (the sum keeps the split order)
    for (; s + 8 <= nks; s += 8) {
      float a[8], b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a[u] = __ldcs(row + (s + u) * sstep);
        if constexpr (sizeof(T) == 16) b[u] = __ldcs(row + (s + u) * sstep + N);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        two_sum_acc(rh, rl, a[u]);
        if constexpr (sizeof(T) == 16) two_sum_acc(ih, il, b[u]);
      }
    }
    for (; s < nks; ++s) {
      two_sum_acc(rh, rl, __ldcs(row + s * sstep));
      if constexpr (sizeof(T) == 16) two_sum_acc(ih, il, __ldcs(row + s * sstep + N));
    }
    const double re = f64_of(rh) + f64_of(rl);
    if constexpr (sizeof(T) == 16) C[(long)m * ldc + j] = make_double2(re, f64_of(ih) + f64_of(il));
    else C[(long)m * ldc + j] = re;
  }
}

// ------------------------------------------- fp64-accurate products (Ozaki)
// C = op(A) op(B) to fp64 accuracy on the bf16 tensor cores, for the
// products whose result must be fp64-accurate in split contexts (the Gram
// matrices of the CholeskyQR passes, rho = Z_L^H Z_R and the projectors
// Z_R v s^-1/2): an error-free splitting of the operands in the manner of
// Ozaki et al. (2012), "Error-free transformations of matrix multiplication
// by using fast routines of matrix multiplication and its applications".
//   * every row m of op(A) (every column n of op(B)) gets the exponent E of
//     its largest entry, |x| < 2^E; each entry is written as the 56-bit
//     fixed-point integer F = trunc(|x| 2^(56 - E)) and cut into eight 7-bit
//     digits d_0 .. d_7 (most significant first), stored with the sign of x
//     as bf16 (integers below 128 are exact in bf16);
//   * a digit product d_s e_t is an integer below 2^14, exact in fp32; the
//     products of equal weight w = s + t (w <= 7; the dropped ones are below
//     2^-53 of the row / column maxima) are accumulated in tensor memory,
//     one fp32 accumulator per weight, over at most OZ_KB_DRAIN K blocks of
//     64: at most 8 * 128 * 127^2 < 2^24, so every partial sum is an exact
//     integer;
//   * each accumulator is drained after OZ_KB_DRAIN K blocks and added,
//     scaled by 2^-7w, into an unevaluated fp32 pair (TwoSum) per output;
//     the pairs of the K splits are summed the same way and the result is
//     hi + lo scaled by 2^(E_m + E_n - 14), to about 2^-48 relative.
// The operand digits stage through shared memory in three quarter stages
// per K block (digits 0-3 of A with 0-3 of B, 0-3 with 4-7, 4-7 with 0-3),
// which cover every product of weight <= 7.
constexpr int OZ_NS = 8;          // digits per operand
constexpr int OZ_BITS = 7;        // bits per digit
constexpr int OZ_BN = 64;         // output columns per CTA (one accumulator width)
constexpr int OZ_KB_DRAIN = 2;    // K blocks per exact accumulation
constexpr int OZ_Q_BYTES = 4 * A_SLICE_BYTES + 4 * OZ_BN * KROW;   // 96 KB per quarter stage

struct OzParams {
  int M;          // output rows (real-embedded)
  int Np;         // padded output columns
  int kb_total;   // K blocks of 64
  int kb_split;   // K blocks per CTA
  float2* part;   // [nks][M][Np] (hi, lo)
  int* err;
};

__global__ void __launch_bounds__(192, 1)
    oz_mma_kernel(const __grid_constant__ CUtensorMap tmA,
                  const __grid_constant__ CUtensorMap tmB, OzParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * OZ_Q_BYTES);
  // full[2], empty[2], chunk done, drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 cdone = smem_u32(bars + 2 * STAGES), drained = smem_u32(bars + 2 * STAGES + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tile = blockIdx.x, chunk = blockIdx.y, ks = blockIdx.z;
  const int kb0 = ks * p.kb_split;
  const int nkb = min(p.kb_split, p.kb_total - kb0);
  const int nchunks = (nkb + OZ_KB_DRAIN - 1) / OZ_KB_DRAIN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(cdone, 1);
    mbar_init(drained, 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  __shared__ int failed;
  if (threadIdx.x == 0) failed = 0;
  __syncthreads();
  // quarter q: A digits from a_off, B digits from b_off
  const int q_a[3] = {0, 0, 4}, q_b[3] = {0, 4, 0};

  if (nkb > 0 && warp == 0 && lane == 0) {
    // TMA producer: three quarter stages per K block
    for (int kb = 0; kb < nkb; ++kb) {
      for (int q = 0; q < 3; ++q) {
        const int it = 3 * kb + q, s = it % STAGES;
        if (it >= STAGES && !mbar_wait(empty0 + 8 * s, ((it / STAGES) - 1) & 1, p.err)) {
          failed = 1;
          break;
        }
        const uint32_t full = full0 + 8 * s;
        mbar_expect_tx(full, OZ_Q_BYTES);
        uint8_t* st = smem + s * OZ_Q_BYTES;
        const int kx = (kb0 + kb) * BK;
        for (int i = 0; i < 4; ++i)
          tma_load_3d(smem_u32(st + i * A_SLICE_BYTES), &tmA, kx, m_tile * BM, q_a[q] + i, full);
        for (int i = 0; i < 4; ++i)
          tma_load_3d(smem_u32(st + 4 * A_SLICE_BYTES + i * OZ_BN * KROW), &tmB, kx,
                      chunk * OZ_BN, q_b[q] + i, full);
      }
      if (failed) break;
    }
  } else if (nkb > 0 && warp == 1 && lane == 0) {
    // MMA issuer: the products of weight <= 7 of each quarter, into the
    // accumulator of their weight; a chunk of OZ_KB_DRAIN K blocks starts
    // each accumulator afresh once the epilogue has drained the last one
    const uint32_t idesc = idesc_bf16(BM, OZ_BN);
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      if (c > 0) {
        if (!mbar_wait(drained, (c - 1) & 1, p.err)) {
          ok = false;
          failed = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      unsigned used = 0;   // accumulators written in this chunk
      const int kbe = min(nkb, (c + 1) * OZ_KB_DRAIN);
      for (int kb = c * OZ_KB_DRAIN; kb < kbe && ok; ++kb) {
        for (int q = 0; q < 3; ++q) {
          const int it = 3 * kb + q, s = it % STAGES;
          if (!mbar_wait(full0 + 8 * s, (it / STAGES) & 1, p.err)) {
            ok = false;
            failed = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + s * OZ_Q_BYTES);
          for (int i = 0; i < 4; ++i) {
            for (int j = 0; j < 4; ++j) {
              const int w = q_a[q] + i + q_b[q] + j;
              if (w >= OZ_NS) continue;
              const uint32_t a0 = st + i * A_SLICE_BYTES;
              const uint32_t b0 = st + 4 * A_SLICE_BYTES + j * OZ_BN * KROW;
              const uint32_t d = tmem + (uint32_t)(w * OZ_BN);
              const bool fresh = !(used >> w & 1u);
              used |= 1u << w;
              for (int kk = 0; kk < KROW / 32; ++kk)
                mma_bf16(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
                         (fresh && kk == 0) ? 0u : 1u);
            }
          }
          mma_commit(empty0 + 8 * s);
        }
      }
      if (ok) mma_commit(cdone);
    }
  } else if (warp >= 2 && nkb > 0) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its quarter)
    const int quarter = warp & 3;
    float hi[OZ_BN], lo[OZ_BN];
#pragma unroll
    for (int i = 0; i < OZ_BN; ++i) hi[i] = lo[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(cdone, c & 1, p.err)) {
        ok = false;
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < OZ_BN; c0 += 16) {
        float scale = 1.f;
#pragma unroll 1
        for (int w = 0; w < OZ_NS; ++w) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(w * OZ_BN + c0), r);
#pragma unroll
          for (int i = 0; i < 16; ++i) two_sum_acc(hi[c0 + i], lo[c0 + i], __uint_as_float(r[i]) * scale);
          scale *= 0.0078125f;   // 2^-7
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(drained) : "memory");
    }
    const int row = m_tile * BM + quarter * 32 + lane;
    if (ok && row < p.M) {
      float2* out = p.part + ((size_t)ks * p.M + row) * p.Np + (size_t)chunk * OZ_BN;
#pragma unroll
      for (int i = 0; i < OZ_BN; ++i) out[i] = make_float2(hi[i], lo[i]);
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
}

// biased exponent field of |x| (0 for zero and subnormals)
__device__ __forceinline__ int bexp(double x) {
  return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu);
}

// the eight signed 7-bit digits of x against the exponent field eb of its
// row / column maximum: F = trunc(|x| 2^(56 - E)), E = eb - 1022
__device__ __forceinline__ void oz_digits(double x, int eb, __nv_bfloat16* d) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  unsigned long long m = ((unsigned long long)(hi & 0xfffffu) << 32) | lo;
  unsigned long long F = 0;
  if (ex > 0) {
    m |= 1ull << 52;
    const int sh = ex - eb + 3;   // <= 3 since ex <= eb
    F = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
  }
  const bool neg = (hi >> 31) != 0;
#pragma unroll
  for (int s = 0; s < OZ_NS; ++s) {
    const int v = (int)((F >> (OZ_BITS * (OZ_NS - 1 - s))) & 127ull);
    d[s] = __float2bfloat16_rn((float)(neg ? -v : v));
  }
}

// exponent fields of the rows of op(A) (M x K): ea[m] = max over k; 32 x 32
// tiles, one atomicMax per row and tile
template <typename T>
__global__ void oz_rowexp_kernel(const T* A, long lda, int op, int M, int K, int* ea) {
  __shared__ int tile[32][33];
  const int tiles_k = (K + 31) / 32, tiles_m = (M + 31) / 32;
  const bool trans = (op == OP_T || op == OP_C);
  for (int t = blockIdx.x; t < tiles_k * tiles_m; t += gridDim.x) {
    const int k0 = (t % tiles_k) * 32, m0 = (t / tiles_k) * 32;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      int e = 0;
      if (!trans) {
        const int m = m0 + yy, kk = k0 + threadIdx.x;
        if (m < M && kk < K) {
          const T v = A[(long)m * lda + kk];
          if constexpr (sizeof(T) == 16) e = max(bexp(v.x), bexp(v.y));
          else e = bexp(v);
        }
        tile[yy][threadIdx.x] = e;
      } else {
        const int kk = k0 + yy, m = m0 + threadIdx.x;
        if (m < M && kk < K) {
          const T v = A[(long)kk * lda + m];
          if constexpr (sizeof(T) == 16) e = max(bexp(v.x), bexp(v.y));
          else e = bexp(v);
        }
        tile[threadIdx.x][yy] = e;
      }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      int e = tile[yy][threadIdx.x];
      for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
      if (threadIdx.x == 0 && m0 + yy < M && e > 0) atomicMax(ea + m0 + yy, e);
    }
    __syncthreads();
  }
}

// A digits: out[s][m][kr] as prep_a_kernel (real embedding [Re | Im]), with
// the fixed-point digits of each row against ea[m]
template <typename T>
__global__ void oz_prep_a_kernel(const T* A, long lda, int op, int M, int K, int Kp,
                                 const int* ea, __nv_bfloat16* out) {
  __shared__ T tile[32][33];
  constexpr bool cx = sizeof(T) == 16;
  const int Kr = cx ? 2 * K : K;
  const long slice = (long)M * Kp;
  const int tiles_k = (K + 31) / 32, tiles_m = (M + 31) / 32;
  const bool trans = (op == OP_T || op == OP_C);
  const bool cj = (op == OP_C || op == OP_R);
  for (int t = blockIdx.x; t < tiles_k * tiles_m; t += gridDim.x) {
    const int k0 = (t % tiles_k) * 32, m0 = (t / tiles_k) * 32;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      if (!trans) {
        const int m = m0 + yy, kk = k0 + threadIdx.x;
        tile[yy][threadIdx.x] = (m < M && kk < K) ? A[(long)m * lda + kk] : zero_of(T());
      } else {
        const int kk = k0 + yy, m = m0 + threadIdx.x;
        tile[threadIdx.x][yy] = (m < M && kk < K) ? A[(long)kk * lda + m] : zero_of(T());
      }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      const int m = m0 + yy, kk = k0 + threadIdx.x;
      if (m < M && kk < K) {
        const T v = tile[yy][threadIdx.x];
        const int eb = ea[m];
        __nv_bfloat16 d[OZ_NS];
        if constexpr (cx) {
          oz_digits(v.x, eb, d);
          put_digits(out, slice, (long)m * Kp + kk, d, false);
          oz_digits(v.y, eb, d);
          put_digits(out, slice, (long)m * Kp + K + kk, d, cj);
        } else {
          oz_digits(v, eb, d);
          put_digits(out, slice, (long)m * Kp + kk, d, false);
        }
      }
    }
    __syncthreads();
  }
  const int pc = Kp - Kr;
  const long tid = (long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x * blockDim.y;
  const __nv_bfloat16 z = __float2bfloat16(0.0f);
  for (long idx = tid; idx < (long)M * pc; idx += nth)
    for (int s = 0; s < OZ_NS; ++s) out[s * slice + (idx / pc) * Kp + Kr + idx % pc] = z;
}

// exponent fields of the columns of op(B) (K x N): eb[n] = max over k
template <typename T>
__global__ void oz_colexp_kernel(const T* B, long ldb, int op, int K, int N, int* eb) {
  __shared__ int tile[32][33];
  const int tk = (K + 31) / 32, tn = (N + 31) / 32;
  const bool trans = (op == OP_T || op == OP_C);
  for (int t = blockIdx.x; t < tk * tn; t += gridDim.x) {
    const int k0 = (t % tk) * 32, n0 = (t / tk) * 32;
    // tile[jj - n0][kk - k0]
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      int e = 0;
      if (!trans) {
        const int kk = k0 + yy, jj = n0 + threadIdx.x;
        if (kk < K && jj < N) {
          const T v = B[(long)kk * ldb + jj];
          if constexpr (sizeof(T) == 16) e = max(bexp(v.x), bexp(v.y));
          else e = bexp(v);
        }
        tile[threadIdx.x][yy] = e;
      } else {
        const int jj = n0 + yy, kk = k0 + threadIdx.x;
        if (kk < K && jj < N) {
          const T v = B[(long)jj * ldb + kk];
          if constexpr (sizeof(T) == 16) e = max(bexp(v.x), bexp(v.y));
          else e = bexp(v);
        }
        tile[yy][threadIdx.x] = e;
      }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      int e = tile[yy][threadIdx.x];
      for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
      if (threadIdx.x == 0 && n0 + yy < N && e > 0) atomicMax(eb + n0 + yy, e);
    }
    __syncthreads();
  }
}

// B digits: out[s][j][kr] as prep_b_kernel (B_emb = [[B_r, B_i], [-B_i, B_r]])
template <typename T>
__global__ void oz_prep_b_kernel(const T* B, long ldb, int op, int K, int N, int Kp, int Np,
                                 const int* ebx, __nv_bfloat16* out) {
  __shared__ T tile[32][33];
  constexpr bool cx = sizeof(T) == 16;
  const int Kr = cx ? 2 * K : K;
  const int Nr = cx ? 2 * N : N;
  const long slice = (long)Np * Kp;
  const int tk = (K + 31) / 32, tn = (N + 31) / 32;
  const bool trans = (op == OP_T || op == OP_C);
  const bool cj = (op == OP_C || op == OP_R);
  for (int t = blockIdx.x; t < tk * tn; t += gridDim.x) {
    const int k0 = (t % tk) * 32, n0 = (t / tk) * 32;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      if (!trans) {
        const int kk = k0 + yy, jj = n0 + threadIdx.x;
        tile[yy][threadIdx.x] = (kk < K && jj < N) ? B[(long)kk * ldb + jj] : zero_of(T());
      } else {
        const int jj = n0 + yy, kk = k0 + threadIdx.x;
        tile[threadIdx.x][yy] = (kk < K && jj < N) ? B[(long)jj * ldb + kk] : zero_of(T());
      }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      const int jj = n0 + yy, kk = k0 + threadIdx.x;
      if (jj < N && kk < K) {
        const T v = tile[threadIdx.x][yy];
        const int e = ebx[jj];
        __nv_bfloat16 re[OZ_NS], im[OZ_NS];
        if constexpr (cx) {
          oz_digits(v.x, e, re);
          oz_digits(v.y, e, im);
          put_digits(out, slice, (long)jj * Kp + kk, re, false);
          put_digits(out, slice, (long)jj * Kp + K + kk, im, !cj);
          put_digits(out, slice, (long)(N + jj) * Kp + kk, im, cj);
          put_digits(out, slice, (long)(N + jj) * Kp + K + kk, re, false);
        } else {
          oz_digits(v, e, re);
          put_digits(out, slice, (long)jj * Kp + kk, re, false);
        }
      }
    }
    __syncthreads();
  }
  const __nv_bfloat16 z = __float2bfloat16(0.0f);
  const long tid = (long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x * blockDim.y;
  for (long idx = tid; idx < (long)(Np - Nr) * Kp; idx += nth)
    for (int s = 0; s < OZ_NS; ++s) out[s * slice + (long)Nr * Kp + idx] = z;
  const int pc = Kp - Kr;
  for (long idx = tid; idx < (long)Nr * pc; idx += nth)
    for (int s = 0; s < OZ_NS; ++s) out[s * slice + (idx / pc) * Kp + Kr + idx % pc] = z;
}

// C[m][j] = (sum over K splits of the pairs) 2^(E_m + E_j - 14), complex
// from [C_r | C_i]; the pairs are summed with TwoSum and converted to fp64
// once, and the power of two is applied to the exponent field
template <typename T>
__global__ void oz_reduce_kernel(const float2* part, int nks, int M, int N, int Np,
                                 const int* ea, const int* ebx, T* C, long ldc) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)M * N;
       idx += (long)gridDim.x * blockDim.x) {
    const int m = (int)(idx / N), j = (int)(idx % N);
    const size_t sstep = (size_t)M * Np;
    const float2* row = part + (size_t)m * Np + j;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int s = 0; s < nks; ++s) {
      const float2 a = row[s * sstep];
      two_sum_acc(rh, rl, a.x);
      two_sum_acc(rh, rl, a.y);
      if constexpr (sizeof(T) == 16) {
        const float2 b = row[s * sstep + N];
        two_sum_acc(ih, il, b.x);
        two_sum_acc(ih, il, b.y);
      }
    }
    const int e1 = ea[m], e2 = ebx[j];
    // 2^(E_m + E_j - 14) with E = field - 1022
    const int sc = (e1 > 0 && e2 > 0) ? e1 + e2 - 2044 - 14 : -2000;
    const double f = sc > -1022 && sc < 1023 ? __hiloint2double((sc + 1023) << 20, 0) : 0.0;
    const double re = (f64_of(rh) + f64_of(rl)) * f;
    if constexpr (sizeof(T) == 16)
      C[(long)m * ldc + j] = make_double2(re, (f64_of(ih) + f64_of(il)) * f);
    else
      C[(long)m * ldc + j] = re;
  }
}

unsigned grid_cap(long n, long cap = 152L * 8) {
  long g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encoder() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

// 3-D map over [ns][rows][Kp] slices (bf16 or tf32-in-fp32) with a
// (128 bytes, box_rows, 1) box, 128B swizzle; ns = 0: the format's count
bool make_map(CUtensorMap* map, const void* base, int rows, int Kp, int box_rows, bool tf32,
              int ns = 0) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) return false;
  const int eb = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows,
                        (cuuint64_t)(ns > 0 ? ns : (tf32 ? 2 : 3))};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * eb, (cuuint64_t)Kp * eb * rows};
  cuuint32_t box[3] = {(cuuint32_t)(KROW / eb), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
             const_cast<void*>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

// ------------------------------------------------------------ context
struct SplitCtx {
  bool cx = false;
  bool tf32 = false;        // 3xTF32 slices instead of bf16 x3
  int N = 0, k = 0;
  std::string msg;
  // cached corner operands: [corner][op N / op H] slices, and their sources
  void* corner_src[4] = {nullptr};
  void* cslices[4][2] = {{nullptr}};
  int corner_Kp = 0;
  // generic operand buffers (grown on demand)
  void* abuf = nullptr;
  size_t abuf_bytes = 0;
  void* bbuf = nullptr;
  size_t bbuf_bytes = 0;
  float* part = nullptr;
  size_t part_bytes = 0;
  // fp64-accurate products: digits of both operands, exponent fields, partials
  void* oz_a = nullptr;
  size_t oz_a_bytes = 0;
  void* oz_b = nullptr;
  size_t oz_b_bytes = 0;
  int* oz_e = nullptr;
  size_t oz_e_bytes = 0;
  void* oz_part = nullptr;
  size_t oz_part_bytes = 0;
  long oz_launches = 0;
  int* err = nullptr;       // device error flag of the owning context
  // per-launch CUDA events around the tensor-core kernel (profiling)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  long prof_launches = 0;
  double prof_flops = 0.0, prof_bytes = 0.0, prof_ms = 0.0;
};

namespace {

ctm_status sfail(SplitCtx* sc, ctm_status st, const char* m) {
  sc->msg = m;
  return st;
}

ctm_status grow(SplitCtx* sc, void** p, size_t* have, size_t need) {
  if (*have >= need) return CTM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    return sfail(sc, CTM_ENOMEM, "split-precision buffer allocation failed");
  }
  *have = need;
  return CTM_OK;
}

int pad_to(int x, int m) { return (x + m - 1) / m * m; }

// column chunking of Nr real output columns into CTAs of <= MAX_BNC columns
void chunking(int Nr, int* nchunks, int* BNc) {
  int nc = (Nr + MAX_BNC - 1) / MAX_BNC;
  if (nc < 1) nc = 1;
  int b = pad_to((Nr + nc - 1) / nc, 16);
  if (b < 16) b = 16;
  *nchunks = nc;
  *BNc = b;
}

int choose_splits(int tiles, int kb_total, int kb_max) {
  int best = 1;
  double best_t = 1e30;
  const int smin = (kb_total + kb_max - 1) / kb_max;
  const int smax = std::max(smin, std::min(std::max(32, smin), kb_total / 4));
  for (int s = smin; s <= smax; ++s) {
    const int per = (kb_total + s - 1) / s;
    const int used = (kb_total + per - 1) / per;
    const long ctas = (long)tiles * used;
    const long waves = (ctas + 151) / 152;
    const double t = (double)waves * (per + 2);
    if (t < best_t - 1e-9) { best_t = t; best = used; }
  }
  return best;
}

// real K of the current problem (set by the caller before run_mma)
thread_local int g_kr_real = 0;
inline double Kr_used(int Kp, const SplitCtx*) { return g_kr_real > 0 ? g_kr_real : Kp; }

// slices per operand, K elements per 128-byte row, bytes per slice element
inline int ns_of(const SplitCtx* sc) { return sc->tf32 ? 2 : 3; }
inline int ke_of(const SplitCtx* sc) { return sc->tf32 ? 32 : 64; }
inline int eb_of(const SplitCtx* sc) { return sc->tf32 ? 4 : 2; }

// run the tensor-core kernel on prepared slices: A [ns][M][Kp], B [ns][Np][Kp]
ctm_status run_mma(SplitCtx* sc, const void* As, const void* Bs, int M, int Kp,
                   int Nr, int nchunks, int BNc, void* C, long ldc, int Nout, cudaStream_t s,
                   long* launches) {
  const int Np = nchunks * BNc;
  const int kb_total = Kp / ke_of(sc);
  const int mt = (M + BM - 1) / BM;
  // the same K elements per fp32 partial in both formats
  const int nks = choose_splits(mt * nchunks, kb_total, KB_SPLIT_MAX * BK / ke_of(sc));
  const int kb_split = (kb_total + nks - 1) / nks;
  {
    ctm_status st = grow(sc, (void**)&sc->part, &sc->part_bytes, (size_t)nks * M * Np * 4);
    if (st != CTM_OK) return st;
  }
  CUtensorMap ta, tb;
  if (!make_map(&ta, As, M, Kp, BM, sc->tf32) || !make_map(&tb, Bs, Np, Kp, BNc, sc->tf32))
    return sfail(sc, CTM_ECUDA, "cuTensorMapEncodeTiled failed");
  MmaParams p;
  p.M = M;
  p.Np = Np;
  p.BNc = BNc;
  p.kb_total = kb_total;
  p.kb_split = kb_split;
  p.part = sc->part;
  p.err = sc->err;
  const int ns = ns_of(sc);
  const size_t smem = 1024 + (size_t)STAGES * (ns * A_SLICE_BYTES + ns * (size_t)BNc * KROW) +
                      (2 * STAGES + 1) * 8 + 16;
  static size_t configured_bf16 = 0, configured_tf32 = 0;
  const void* kfn = sc->tf32 ? (const void*)split_mma_kernel<FmtTF32>
                             : (const void*)split_mma_kernel<FmtBF16>;
  if (raise_smem(kfn, sc->tf32 ? configured_tf32 : configured_bf16, smem) != cudaSuccess)
    return sfail(sc, CTM_ECUDA, "cannot reserve shared memory for the tensor-core kernel");
  dim3 grid(mt, nchunks, nks);
  if (sc->prof && sc->ev_used + 2 > sc->ev.size()) {
    // every launch of the profiled region is timed: the event pool grows
    const size_t old = sc->ev.size();
    sc->ev.resize(old + 8192);
    for (size_t i = old; i < sc->ev.size(); ++i)
      if (cudaEventCreate(&sc->ev[i]) != cudaSuccess) {
        sc->ev.resize(i);
        break;
      }
  }
  const bool timed = sc->prof && sc->ev_used + 2 <= sc->ev.size();
  if (timed) cudaEventRecord(sc->ev[sc->ev_used], s);
  if (sc->tf32) split_mma_kernel<FmtTF32><<<grid, 128, smem, s>>>(ta, tb, p);
  else split_mma_kernel<FmtBF16><<<grid, 128, smem, s>>>(ta, tb, p);
  if (timed) {
    cudaEventRecord(sc->ev[sc->ev_used + 1], s);
    sc->ev_used += 2;
    // tensor-pipe work: the slice products (six bf16 or three tf32) of the
    // real-embedded (unpadded) problem; bytes: all slices of both operands
    // once, plus the fp32 partials
    sc->prof_launches += 1;
    const double np = sc->tf32 ? 3.0 : 6.0;
    sc->prof_flops += np * 2.0 * (double)M * (double)Nr * (double)Kr_used(Kp, sc);
    sc->prof_bytes += (double)ns * eb_of(sc) * ((double)M * Kp + (double)nchunks * BNc * Kp) +
                      4.0 * (double)nks * M * Np;
  }
  if (launches) ++*launches;
  if (sc->cx)
    reduce_kernel<cplx><<<grid_cap((long)M * Nout), 256, 0, s>>>(sc->part, nks, M, Nout, Np,
                                                                 (cplx*)C, ldc);
  else
    reduce_kernel<double><<<grid_cap((long)M * Nout), 256, 0, s>>>(sc->part, nks, M, Nout, Np,
                                                                   (double*)C, ldc);
  if (launches) ++*launches;
  if (cudaGetLastError() != cudaSuccess) return sfail(sc, CTM_ECUDA, "split GEMM launch failed");
  (void)Nr;
  return CTM_OK;
}

ctm_status prep_a(SplitCtx* sc, const void* A, long lda, int op, int M, int K, int Kp,
                  void* out, cudaStream_t s, long* launches) {
  const long tiles = (long)((K + 31) / 32) * ((M + 31) / 32);
  const unsigned g = (unsigned)std::max<long>(1, std::min<long>(tiles, 152L * 16));
  const dim3 b(32, 8);
  if (sc->tf32) {
    if (sc->cx) prep_a_kernel<cplx, FmtTF32><<<g, b, 0, s>>>((const cplx*)A, lda, op, M, K, Kp, (float*)out);
    else prep_a_kernel<double, FmtTF32><<<g, b, 0, s>>>((const double*)A, lda, op, M, K, Kp, (float*)out);
  } else {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
    if (sc->cx) prep_a_kernel<cplx, FmtBF16><<<g, b, 0, s>>>((const cplx*)A, lda, op, M, K, Kp, o);
    else prep_a_kernel<double, FmtBF16><<<g, b, 0, s>>>((const double*)A, lda, op, M, K, Kp, o);
  }
  if (launches) ++*launches;
  return cudaGetLastError() == cudaSuccess ? CTM_OK : sfail(sc, CTM_ECUDA, "slice launch failed");
}

ctm_status prep_b(SplitCtx* sc, const void* B, long ldb, int op, int K, int N, int Kp, int Np,
                  void* out, cudaStream_t s, long* launches) {
  long tiles = (long)((K + 31) / 32) * ((N + 31) / 32);
  if (tiles > 152L * 8) tiles = 152L * 8;
  if (tiles < 1) tiles = 1;
  const dim3 blk(32, 8);
  const unsigned g = (unsigned)tiles;
  if (sc->tf32) {
    float* o = static_cast<float*>(out);
    if (sc->cx) prep_b_kernel<cplx, FmtTF32><<<g, blk, 0, s>>>((const cplx*)B, ldb, op, K, N, Kp, Np, o);
    else prep_b_kernel<double, FmtTF32><<<g, blk, 0, s>>>((const double*)B, ldb, op, K, N, Kp, Np, o);
  } else {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
    if (sc->cx) prep_b_kernel<cplx, FmtBF16><<<g, blk, 0, s>>>((const cplx*)B, ldb, op, K, N, Kp, Np, o);
    else prep_b_kernel<double, FmtBF16><<<g, blk, 0, s>>>((const double*)B, ldb, op, K, N, Kp, Np, o);
  }
  if (launches) ++*launches;
  return cudaGetLastError() == cudaSuccess ? CTM_OK : sfail(sc, CTM_ECUDA, "slice launch failed");
}

}  // namespace

ctm_status split_create(SplitCtx** out, bool cx, bool tf32, int N, int k, int* err,
                        cudaStream_t s) {
  (void)s;
  *out = nullptr;
  if (!get_encoder()) return CTM_EUNSUPPORTED;
  SplitCtx* sc = new SplitCtx();
  sc->cx = cx;
  sc->tf32 = tf32;
  sc->N = N;
  sc->k = k;
  sc->err = err;
  *out = sc;
  return CTM_OK;
}

ctm_status split_profile(SplitCtx* sc, int on, double* ms, long* launches, double* flops,
                         double* bytes) {
  if (on >= 0) {
    if (on && sc->ev.empty()) {
      sc->ev.resize(8192);
      for (auto& e : sc->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return sfail(sc, CTM_ECUDA, "event creation failed");
    }
    sc->prof = on != 0;
    sc->ev_used = 0;
    sc->prof_launches = 0;
    sc->prof_flops = sc->prof_bytes = sc->prof_ms = 0.0;
    return CTM_OK;
  }
  // read: fold the recorded pairs into the totals
  for (size_t i = 0; i + 1 < sc->ev_used; i += 2) {
    if (cudaEventSynchronize(sc->ev[i + 1]) != cudaSuccess)
      return sfail(sc, CTM_ECUDA, "event synchronisation failed");
    float t = 0.f;
    cudaEventElapsedTime(&t, sc->ev[i], sc->ev[i + 1]);
    sc->prof_ms += t;
  }
  sc->ev_used = 0;
  if (ms) *ms = sc->prof_ms;
  if (launches) *launches = sc->prof_launches;
  if (flops) *flops = sc->prof_flops;
  if (bytes) *bytes = sc->prof_bytes;
  return CTM_OK;
}

void split_destroy(SplitCtx* sc) {
  if (!sc) return;
  for (auto& e : sc->ev) cudaEventDestroy(e);
  for (int i = 0; i < 4; ++i)
    for (int o = 0; o < 2; ++o)
      if (sc->cslices[i][o]) cudaFree(sc->cslices[i][o]);
  if (sc->abuf) cudaFree(sc->abuf);
  if (sc->bbuf) cudaFree(sc->bbuf);
  if (sc->part) cudaFree(sc->part);
  if (sc->oz_a) cudaFree(sc->oz_a);
  if (sc->oz_b) cudaFree(sc->oz_b);
  if (sc->oz_e) cudaFree(sc->oz_e);
  if (sc->oz_part) cudaFree(sc->oz_part);
  delete sc;
}

ctm_status split_prepare_corners(SplitCtx* sc, void* const* Q, int N, unsigned mask,
                                 cudaStream_t s, long* launches) {
  const int Kr = sc->cx ? 2 * N : N;
  const int Kp = pad_to(Kr, ke_of(sc));
  sc->corner_Kp = Kp;
  for (int i = 0; i < 4; ++i) {
    if (!(mask >> i & 1u)) continue;
    sc->corner_src[i] = Q[i];
    for (int o = 0; o < 2; ++o) {
      if (!sc->cslices[i][o]) {
        if (cudaMalloc(&sc->cslices[i][o], (size_t)ns_of(sc) * N * Kp * eb_of(sc)) != cudaSuccess) {
          cudaGetLastError();
          return sfail(sc, CTM_ENOMEM, "corner slice allocation failed");
        }
      }
      const int op = o == 0 ? OP_N : (sc->cx ? OP_C : OP_T);
      ctm_status st = prep_a(sc, Q[i], N, op, N, N, Kp, sc->cslices[i][o], s, launches);
      if (st != CTM_OK) return st;
    }
  }
  return CTM_OK;
}

ctm_status split_apply(SplitCtx* sc, const void* Q, bool herm, const void* Zin, void* Zout, int N,
                       int k, cudaStream_t s, long* launches) {
  int ci = -1;
  for (int i = 0; i < 4; ++i)
    if (sc->corner_src[i] == Q) ci = i;
  if (ci < 0) return sfail(sc, CTM_EINVAL, "corner was not prepared");
  const int Kp = sc->corner_Kp;
  const int Nr = sc->cx ? 2 * k : k;
  g_kr_real = sc->cx ? 2 * N : N;
  int nchunks, BNc;
  chunking(Nr, &nchunks, &BNc);
  const int Np = nchunks * BNc;
  ctm_status st = grow(sc, (void**)&sc->bbuf, &sc->bbuf_bytes,
                       (size_t)ns_of(sc) * Np * Kp * eb_of(sc));
  if (st != CTM_OK) return st;
  st = prep_b(sc, Zin, k, OP_N, N, k, Kp, Np, sc->bbuf, s, launches);
  if (st != CTM_OK) return st;
  return run_mma(sc, sc->cslices[ci][herm ? 1 : 0], sc->bbuf, N, Kp, Nr, nchunks, BNc, Zout, k, k,
                 s, launches);
}

ctm_status split_gemm(SplitCtx* sc, int opA, const void* A, long lda, int opB, const void* B,
                      long ldb, int M, int N, int K, void* C, long ldc, cudaStream_t s,
                      long* launches) {
  const int Kr = sc->cx ? 2 * K : K;
  const int Kp = pad_to(Kr, ke_of(sc));
  const int Nr = sc->cx ? 2 * N : N;
  g_kr_real = Kr;
  int nchunks, BNc;
  chunking(Nr, &nchunks, &BNc);
  const int Np = nchunks * BNc;
  const size_t per = (size_t)ns_of(sc) * eb_of(sc);
  ctm_status st = grow(sc, (void**)&sc->abuf, &sc->abuf_bytes, per * M * Kp);
  if (st != CTM_OK) return st;
  st = grow(sc, (void**)&sc->bbuf, &sc->bbuf_bytes, per * Np * Kp);
  if (st != CTM_OK) return st;
  st = prep_a(sc, A, lda, opA, M, K, Kp, sc->abuf, s, launches);
  if (st != CTM_OK) return st;
  st = prep_b(sc, B, ldb, opB, K, N, Kp, Np, sc->bbuf, s, launches);
  if (st != CTM_OK) return st;
  return run_mma(sc, sc->abuf, sc->bbuf, M, Kp, Nr, nchunks, BNc, C, ldc, N, s, launches);
}

ctm_status oz_gemm(SplitCtx* sc, int opA, const void* A, long lda, int opB, const void* B,
                   long ldb, int M, int N, int K, void* C, long ldc, cudaStream_t s,
                   long* launches) {
  if (M <= 0 || N <= 0 || K <= 0) return sfail(sc, CTM_EINVAL, "empty fp64-accurate product");
  const bool cx = sc->cx;
  const int Kr = cx ? 2 * K : K;
  const int Kp = pad_to(Kr, BK);
  const int Nr = cx ? 2 * N : N;
  const int Np = pad_to(Nr, OZ_BN);
  const int nchunks = Np / OZ_BN;
  const int mt = (M + BM - 1) / BM;
  const int kb_total = Kp / BK;
  // about two waves of CTAs, at least OZ_KB_DRAIN K blocks each
  const long tiles = (long)mt * nchunks;
  int nks = (int)std::max<long>(1, std::min<long>((2 * 152 + tiles - 1) / tiles,
                                                  (kb_total + OZ_KB_DRAIN - 1) / OZ_KB_DRAIN));
  const int kb_split = (kb_total + nks - 1) / nks;
  nks = (kb_total + kb_split - 1) / kb_split;
  ctm_status st = grow(sc, &sc->oz_a, &sc->oz_a_bytes, (size_t)OZ_NS * M * Kp * 2);
  if (st == CTM_OK) st = grow(sc, &sc->oz_b, &sc->oz_b_bytes, (size_t)OZ_NS * Np * Kp * 2);
  if (st == CTM_OK) st = grow(sc, (void**)&sc->oz_e, &sc->oz_e_bytes, (size_t)(M + N) * sizeof(int));
  if (st == CTM_OK) st = grow(sc, &sc->oz_part, &sc->oz_part_bytes, (size_t)nks * M * Np * 8);
  if (st != CTM_OK) return st;
  int* ea = sc->oz_e;
  int* ebx = sc->oz_e + M;
  if (cudaMemsetAsync(sc->oz_e, 0, (size_t)(M + N) * sizeof(int), s) != cudaSuccess)
    return sfail(sc, CTM_ECUDA, "exponent reset failed");
  const dim3 blk(32, 8);
  const unsigned ga = (unsigned)std::max<long>(1, std::min<long>((long)((K + 31) / 32) * ((M + 31) / 32), 152L * 16));
  const unsigned gb = (unsigned)std::max<long>(1, std::min<long>((long)((K + 31) / 32) * ((N + 31) / 32), 152L * 16));
  __nv_bfloat16* da = static_cast<__nv_bfloat16*>(sc->oz_a);
  __nv_bfloat16* db = static_cast<__nv_bfloat16*>(sc->oz_b);
  if (cx) {
    oz_rowexp_kernel<cplx><<<ga, blk, 0, s>>>((const cplx*)A, lda, opA, M, K, ea);
    oz_colexp_kernel<cplx><<<gb, blk, 0, s>>>((const cplx*)B, ldb, opB, K, N, ebx);
    oz_prep_a_kernel<cplx><<<ga, blk, 0, s>>>((const cplx*)A, lda, opA, M, K, Kp, ea, da);
    oz_prep_b_kernel<cplx><<<gb, blk, 0, s>>>((const cplx*)B, ldb, opB, K, N, Kp, Np, ebx, db);
  } else {
    oz_rowexp_kernel<double><<<ga, blk, 0, s>>>((const double*)A, lda, opA, M, K, ea);
    oz_colexp_kernel<double><<<gb, blk, 0, s>>>((const double*)B, ldb, opB, K, N, ebx);
    oz_prep_a_kernel<double><<<ga, blk, 0, s>>>((const double*)A, lda, opA, M, K, Kp, ea, da);
    oz_prep_b_kernel<double><<<gb, blk, 0, s>>>((const double*)B, ldb, opB, K, N, Kp, Np, ebx, db);
  }
  if (launches) *launches += 4;
  CUtensorMap ta, tb;
  if (!make_map(&ta, sc->oz_a, M, Kp, BM, false, OZ_NS) ||
      !make_map(&tb, sc->oz_b, Np, Kp, OZ_BN, false, OZ_NS))
    return sfail(sc, CTM_ECUDA, "cuTensorMapEncodeTiled failed");
  OzParams p;
  p.M = M;
  p.Np = Np;
  p.kb_total = kb_total;
  p.kb_split = kb_split;
  p.part = static_cast<float2*>(sc->oz_part);
  p.err = sc->err;
  const size_t smem = 1024 + (size_t)STAGES * OZ_Q_BYTES + (2 * STAGES + 2) * 8 + 16;
  static size_t configured = 0;
  if (raise_smem((const void*)oz_mma_kernel, configured, smem) != cudaSuccess)
    return sfail(sc, CTM_ECUDA, "cannot reserve shared memory for the fp64-accurate product");
  oz_mma_kernel<<<dim3(mt, nchunks, nks), 192, smem, s>>>(ta, tb, p);
  ++sc->oz_launches;
  if (cx)
    oz_reduce_kernel<cplx><<<grid_cap((long)M * N), 256, 0, s>>>(
        p.part, nks, M, N, Np, ea, ebx, (cplx*)C, ldc);
  else
    oz_reduce_kernel<double><<<grid_cap((long)M * N), 256, 0, s>>>(
        p.part, nks, M, N, Np, ea, ebx, (double*)C, ldc);
  if (launches) *launches += 2;
  if (cudaGetLastError() != cudaSuccess) return sfail(sc, CTM_ECUDA, "fp64-accurate product launch failed");
  return CTM_OK;
}

size_t split_partial_splits(size_t N, bool cx) {
  const size_t kb = ((cx ? 2 : 1) * N + BK - 1) / BK;
  return std::max<size_t>(32, (kb + KB_SPLIT_MAX - 1) / KB_SPLIT_MAX);
}

const char* split_last_error(const SplitCtx* sc) {
  return sc ? sc->msg.c_str() : "split precision not initialised";
}

}  // namespace ctm
