// Tensor-core GEMMs of the wall-model MLP (no counterpart in the paper):
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in tensor memory)
// issued by one thread per CTA on operand tiles staged in shared memory.
//
//   forward      z[b][n]  = sum_k a(b, k) W[n][k] + bias[n],  a = x_n or GELU(z_prev)
//   data grad    da[b][k] = (sum_n dz[b][n] W[n][k]) GELU'(z_prev[b][k])
//   weight grad  dW[n][k] = sum_b dz[b][n] a(b, k),  dbias[n] = sum_b dz[b][n]
//
// Every GEMM is D[M = 128][N] += A[128][K] B[N][K]^T with both operands
// K-major: a CTA owns 128 rows of D and stages A and B as BF16 in the canonical
// no-swizzle layout (8-row x 16-byte core matrices, the K groups outermost):
// A from the FP32 activations with coalesced vector loads, B as a straight copy
// of a weight image kept in that layout (rebuilt whenever the weights change).
// One thread issues K/16 MMAs whose completion it commits to an mbarrier; the
// eight warps then read the accumulators with tcgen05.ld (warp w its TMEM lanes
// 32 (w % 4) .. + 31, half of the columns each), stage them in shared memory
// and write the rows out coalesced.
// The weight gradient reduces over the batch: its M is the layer's outputs,
// its N the layer's inputs plus a column of ones (the bias gradient), and its K
// runs over the CTA's batch rows in 64-row chunks accumulated in TMEM.  Waits
// are bounded: on a timeout a kernel records PNP_ERR_TIMEOUT, waits once more
// (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "pnp_common.cuh"
#include "pnp_wall.cuh"

namespace pnp {

namespace {

constexpr int kTcRows = 128;      // rows of D per CTA (M of every MMA)
constexpr int kTcThreads = 256;   // eight warps: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31
constexpr int kWgK = 64;          // batch rows per weight-gradient chunk (four MMAs of K = 16)
constexpr unsigned long long kTcWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float gelu_tc(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d_tc(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Byte offset of element (r, k) of an R-row K-major tile: core matrix (r / 8,
// k / 8) of 8 rows x 16 bytes, K groups outermost, so the core matrices
// adjacent in K are R/8 * 128 bytes apart (the leading-dimension offset) and
// those adjacent in M/N 128 bytes (the stride-dimension offset).
__device__ __forceinline__ uint32_t canon(int r, int k, int R) {
  return (uint32_t)((((k >> 3) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: start address, leading- and stride-
// dimension byte offsets (each >> 4), the fixed version bits 0b001 at 46-48,
// no base offset, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t start, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((start >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits
// 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// the generic-proxy writes of the staged tiles become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one full warp; the address lands in *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init1(unsigned long long* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(b)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase with this parity to complete
__device__ __forceinline__ bool mbar_wait_tc(unsigned long long* b, unsigned parity) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_test(b, parity)) return true;
    if ((it & 255) == 0 && now_ns() - t0 > kTcWaitNs) break;
  }
  return false;
}

__device__ __forceinline__ uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// The shared tail of every kernel: K / 16 MMAs on the staged tiles (thread 0),
// the bounded wait for their completion (phase `parity`), true when it came.
__device__ __forceinline__ bool mma_tiles(uint32_t tmem, const __nv_bfloat16* sA, const __nv_bfloat16* sB, int N,
                                          int Kdim, bool accumulate, unsigned long long* bar, unsigned parity) {
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x == 0) {
    const uint32_t lboA = (kTcRows / 8) * 128, lboB = (uint32_t)(N / 8) * 128;
    const uint32_t id = idesc_bf16(kTcRows, N);
    for (int s = 0; s < Kdim / 16; ++s) {
      const uint64_t a = sdesc(saddr(sA) + 2 * s * lboA, lboA, 128);
      const uint64_t b = sdesc(saddr(sB) + 2 * s * lboB, lboB, 128);
      mma_bf16(tmem, a, b, id, (accumulate || s > 0) ? 1u : 0u);
    }
    mma_commit(bar);
  }
  const bool ok = __syncthreads_and(mbar_wait_tc(bar, parity)) != 0;   // uniform across the CTA
  fence_after();
  return ok;
}

// Shared memory: A [128][K] and B [N][K] BF16 tiles (later the FP32 staging of
// the epilogue, `data` bytes in all), an mbarrier and the TMEM slot.
struct TcSmem {
  __nv_bfloat16* A;
  __nv_bfloat16* B;
  float* C;
  unsigned long long* bar;
  uint32_t* slot;
};
__host__ __device__ inline size_t tc_data_bytes(int Kdim, int N, size_t stage_bytes) {
  const size_t ab = ((size_t)kTcRows * Kdim + (size_t)N * Kdim) * 2;
  return ((ab > stage_bytes ? ab : stage_bytes) + 15) & ~(size_t)15;
}
__device__ __forceinline__ TcSmem tc_smem(unsigned char* base, int Kdim, int N, size_t stage_bytes) {
  TcSmem t;
  t.A = reinterpret_cast<__nv_bfloat16*>(base);
  t.B = t.A + (size_t)kTcRows * Kdim;
  t.C = reinterpret_cast<float*>(base);
  unsigned char* tail = base + tc_data_bytes(Kdim, N, stage_bytes);
  t.bar = reinterpret_cast<unsigned long long*>(tail);
  t.slot = reinterpret_cast<uint32_t*>(tail + 8);
  return t;
}
__host__ __device__ inline size_t tc_smem_bytes(int Kdim, int N, size_t stage_bytes) {
  return tc_data_bytes(Kdim, N, stage_bytes) + 16;
}

__device__ __forceinline__ void set_bf16(__nv_bfloat16* tile, uint32_t off, float x) {
  *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(tile) + off) = __float2bfloat16_rn(x);
}

// Failure path: record the timeout and give the MMAs one more bounded wait
// before the tensor memory is freed.
__device__ __forceinline__ void tc_timeout(int* err, unsigned long long* bar, unsigned parity) {
  if (threadIdx.x == 0) {
    atomicExch(err, PNP_ERR_TIMEOUT);
    mbar_wait_tc(bar, parity);
  }
}

// A[r][k] (r < 128, k < Kp) = act(src[r][k]) for r < rows and k < Kd, zero
// elsewhere; src holds rows x Kd FP32 values row after row.  Kd % 8 == 0: one
// float4 load and one 8-byte store per 4 values (consecutive threads read
// consecutive 16-byte chunks), the padding columns in 16-byte stores.
__device__ __forceinline__ void stage_a(__nv_bfloat16* A, const float* __restrict__ src, int rows, int Kd, int Kp,
                                        bool act) {
  const int tid = threadIdx.x;
  unsigned char* a = reinterpret_cast<unsigned char*>(A);
  if ((Kd & 7) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const int nq = kTcRows * Kd / 4;
#pragma unroll 4
    for (int q = tid; q < nq; q += kTcThreads) {
      const int e = 4 * q, r = e / Kd, k = e - r * Kd;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) {
        x = __ldg(s4 + q);
        if (act) {
          x.x = gelu_tc(x.x);
          x.y = gelu_tc(x.y);
          x.z = gelu_tc(x.z);
          x.w = gelu_tc(x.w);
        }
      }
      const __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y), hi = __floats2bfloat162_rn(x.z, x.w);
      uint2 u;
      u.x = *reinterpret_cast<const uint32_t*>(&lo);
      u.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(a + canon(r, k, kTcRows)) = u;
    }
    const int nper = (Kp - Kd) >> 3;
    for (int e = tid; e < kTcRows * nper; e += kTcThreads) {
      const int r = e / nper, k = Kd + 8 * (e - r * nper);
      *reinterpret_cast<uint4*>(a + canon(r, k, kTcRows)) = make_uint4(0u, 0u, 0u, 0u);
    }
  } else {
    for (int e = tid; e < kTcRows * Kp; e += kTcThreads) {
      const int r = e / Kp, k = e - r * Kp;
      float x = 0.f;
      if (r < rows && k < Kd) {
        x = src[(size_t)r * Kd + k];
        if (act) x = gelu_tc(x);
      }
      set_bf16(A, canon(r, k, kTcRows), x);
    }
  }
}

// T[rr][bb] = act(src[bb][rr]) for bb < rows, rr < Rs (the transpose of a chunk
// of rows, for the weight gradient, whose K is the batch), T[ones_at][bb] = 1
// for bb < rows when ones_at >= 0, and zero in columns bb >= rows; rows Rs..R-1
// other than ones_at are left as they are (zero from the start of the kernel).
__device__ __forceinline__ void stage_t(__nv_bfloat16* T, int R, const float* __restrict__ src, int rows, int Rs,
                                        bool act, int ones_at) {
  const int tid = threadIdx.x;
  if ((Rs & 3) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const int nq = rows * Rs / 4;
#pragma unroll 4
    for (int q = tid; q < nq; q += kTcThreads) {
      const int e = 4 * q, bb = e / Rs, rr = e - bb * Rs;
      float4 x = __ldg(s4 + q);
      if (act) {
        x.x = gelu_tc(x.x);
        x.y = gelu_tc(x.y);
        x.z = gelu_tc(x.z);
        x.w = gelu_tc(x.w);
      }
      set_bf16(T, canon(rr, bb, R), x.x);
      set_bf16(T, canon(rr + 1, bb, R), x.y);
      set_bf16(T, canon(rr + 2, bb, R), x.z);
      set_bf16(T, canon(rr + 3, bb, R), x.w);
    }
  } else {
    for (int e = tid; e < rows * Rs; e += kTcThreads) {
      const int bb = e / Rs, rr = e - bb * Rs;
      float x = src[e];
      if (act) x = gelu_tc(x);
      set_bf16(T, canon(rr, bb, R), x);
    }
  }
  if (ones_at >= 0)
    for (int bb = tid; bb < kWgK; bb += kTcThreads) set_bf16(T, canon(ones_at, bb, R), bb < rows ? 1.f : 0.f);
  for (int e = tid; e < (kWgK - rows) * Rs; e += kTcThreads) {
    const int bb = rows + e / Rs, rr = e % Rs;
    set_bf16(T, canon(rr, bb, R), 0.f);
  }
}

// The weight image of a layer (16-byte chunks, already in the shared-memory layout).
__device__ __forceinline__ void copy_image(__nv_bfloat16* Bt, const __nv_bfloat16* __restrict__ img, int n16) {
  const uint4* s = reinterpret_cast<const uint4*>(img);
  uint4* d = reinterpret_cast<uint4*>(Bt);
#pragma unroll 4
  for (int i = threadIdx.x; i < n16; i += kTcThreads) d[i] = __ldg(s + i);
}

// Accumulator columns [0, ncol) of the CTA's 128 rows into C[r][c] (row stride
// ldc floats): warp w reads its lanes 32 (w % 4) .. + 31, the columns 16-wide
// groups alternately with the warp w +- 4 that shares those lanes.
__device__ __forceinline__ void tmem_to_smem(uint32_t tmem, int ncol, float* C, int ldc) {
  const int warp = threadIdx.x >> 5, grp = warp & 3, half = warp >> 2;
  const int r = 32 * grp + (threadIdx.x & 31);
  const uint32_t lane = tmem + ((uint32_t)(32 * grp) << 16);
  for (int c0 = 16 * half; c0 < ncol; c0 += 32) {
    float v[16];
    tmem_ld16(lane + c0, v);
    float4* row = reinterpret_cast<float4*>(C + (size_t)r * ldc + c0);
#pragma unroll
    for (int i = 0; i < 4; ++i) row[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  }
}

}  // namespace

// z[b][n] = sum_k a(b, k) W[n][k] + bias[n] for the CTA's 128 rows; Kp, Np: K, N
// rounded up to 16; Wimg: the layer's forward weight image [Np][Kp].
__global__ void __launch_bounds__(kTcThreads) k_mlp_fwd_tc(const float* __restrict__ in, int K, int act_in,
                                                           const __nv_bfloat16* __restrict__ Wimg,
                                                           const float* __restrict__ bias, int N, int B,
                                                           float* __restrict__ out, int* err) {
  extern __shared__ __align__(128) unsigned char tc_raw[];
  const int Kp = (K + 15) & ~15, Np = (N + 15) & ~15, ldc = Np + 4;
  const TcSmem s = tc_smem(tc_raw, Kp, Np, (size_t)kTcRows * ldc * sizeof(float));
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = tmem_cols(Np);
  if (warp == 0) tmem_alloc(s.slot, ncols);
  if (tid == 0) mbar_init1(s.bar);
  const int b0 = blockIdx.x * kTcRows, rows = min(kTcRows, B - b0);
  stage_a(s.A, in + (size_t)b0 * K, rows, K, Kp, act_in != 0);
  copy_image(s.B, Wimg, Np * Kp / 8);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *s.slot;
  if (mma_tiles(tmem, s.A, s.B, Np, Kp, false, s.bar, 0)) {
    tmem_to_smem(tmem, Np, s.C, ldc);   // the tiles are free: their MMAs have completed
    __syncthreads();
    float* o = out + (size_t)b0 * N;   // the CTA's rows are rows * N consecutive values
    const int n_el = rows * N;
    if ((N & 3) == 0) {
#pragma unroll 4
      for (int e = 4 * tid; e < n_el; e += 4 * kTcThreads) {
        const int r = e / N, n = e - r * N;
        const float4 c = *reinterpret_cast<const float4*>(s.C + (size_t)r * ldc + n);
        const float4 bv = *reinterpret_cast<const float4*>(bias + n);
        *reinterpret_cast<float4*>(o + e) = make_float4(c.x + bv.x, c.y + bv.y, c.z + bv.z, c.w + bv.w);
      }
    } else {
      for (int e = tid; e < n_el; e += kTcThreads) {
        const int r = e / N, n = e - r * N;
        o[e] = s.C[(size_t)r * ldc + n] + bias[n];
      }
    }
  } else {
    tc_timeout(err, s.bar, 0);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// da[b][k] = (sum_n dz[b][n] W[n][k]) GELU'(zprev[b][k]): A = dz [128][Np], B = W^T
// from the layer's backward weight image [Kq][Np].
__global__ void __launch_bounds__(kTcThreads) k_mlp_bwd_data_tc(const float* __restrict__ dz, int N,
                                                                const __nv_bfloat16* __restrict__ WimgT, int K, int B,
                                                                const float* __restrict__ zprev,
                                                                float* __restrict__ out, int* err) {
  extern __shared__ __align__(128) unsigned char tc_raw[];
  const int Np = (N + 15) & ~15, Kq = (K + 15) & ~15, ldc = Kq + 4;
  const TcSmem s = tc_smem(tc_raw, Np, Kq, (size_t)kTcRows * ldc * sizeof(float));
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = tmem_cols(Kq);
  if (warp == 0) tmem_alloc(s.slot, ncols);
  if (tid == 0) mbar_init1(s.bar);
  const int b0 = blockIdx.x * kTcRows, rows = min(kTcRows, B - b0);
  stage_a(s.A, dz + (size_t)b0 * N, rows, N, Np, false);
  copy_image(s.B, WimgT, Kq * Np / 8);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *s.slot;
  if (mma_tiles(tmem, s.A, s.B, Kq, Np, false, s.bar, 0)) {
    tmem_to_smem(tmem, Kq, s.C, ldc);
    __syncthreads();
    const size_t base = (size_t)b0 * K;
    const int n_el = rows * K;
    if ((K & 3) == 0) {
#pragma unroll 4
      for (int e = 4 * tid; e < n_el; e += 4 * kTcThreads) {
        const int r = e / K, k = e - r * K;
        const float4 c = *reinterpret_cast<const float4*>(s.C + (size_t)r * ldc + k);
        const float4 z = __ldg(reinterpret_cast<const float4*>(zprev + base + e));
        *reinterpret_cast<float4*>(out + base + e) =
            make_float4(c.x * gelu_d_tc(z.x), c.y * gelu_d_tc(z.y), c.z * gelu_d_tc(z.z), c.w * gelu_d_tc(z.w));
      }
    } else {
      for (int e = tid; e < n_el; e += kTcThreads) {
        const int r = e / K, k = e - r * K;
        out[base + e] = s.C[(size_t)r * ldc + k] * gelu_d_tc(zprev[base + e]);
      }
    }
  } else {
    tc_timeout(err, s.bar, 0);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Per-CTA partial weight and bias gradients over rows [blk r, min(B, (blk+1) r)):
// D[n][k] = sum_b dz[b][n] a(b, k) (k < K), D[n][K] = sum_b dz[b][n]; the batch
// is the K of the MMAs, in 64-row chunks accumulated in TMEM.  partial[blk] =
// [N][K] weights, then [N] biases.
__global__ void __launch_bounds__(kTcThreads) k_mlp_wgrad_tc(const float* __restrict__ dz, int N,
                                                             const float* __restrict__ in, int K, int act_in, int B,
                                                             int rows_per_block, float* __restrict__ partial,
                                                             int* err) {
  extern __shared__ __align__(128) unsigned char tc_raw[];
  const int Nw = ((K + 1) + 15) & ~15;   // inputs and the ones column of the bias
  const TcSmem s = tc_smem(tc_raw, kWgK, Nw, 0);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = tmem_cols(Nw);
  if (warp == 0) tmem_alloc(s.slot, ncols);
  if (tid == 0) mbar_init1(s.bar);
  {   // rows N.. of A and K+1.. of B stay zero for the whole kernel
    uint4* z = reinterpret_cast<uint4*>(s.A);
    const int n16 = (kTcRows + Nw) * kWgK * 2 / 16;
    for (int i = tid; i < n16; i += kTcThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *s.slot;
  const int r0 = blockIdx.x * rows_per_block, r1 = min(B, r0 + rows_per_block);
  bool ok = true;
  unsigned phase = 0;
  for (int c0 = r0; c0 < r1 && ok; c0 += kWgK, phase ^= 1u) {
    const int rows = min(kWgK, r1 - c0);
    if (c0 > r0) {   // the previous chunk's MMAs read the tiles until their commit arrived
      fence_before();
      __syncthreads();
    }
    stage_t(s.A, kTcRows, dz + (size_t)c0 * N, rows, N, false, -1);
    stage_t(s.B, Nw, in + (size_t)c0 * K, rows, K, act_in != 0, K);
    ok = mma_tiles(tmem, s.A, s.B, Nw, kWgK, c0 > r0, s.bar, phase);
  }
  float* p = partial + (size_t)blockIdx.x * ((size_t)N * K + N);
  if (ok && r0 < r1) {
    const int grp = warp & 3, half = warp >> 2;
    const int n = 32 * grp + (tid & 31);   // this thread's TMEM lane is output row n
    const uint32_t lane = tmem + ((uint32_t)(32 * grp) << 16);
    for (int c0 = 16 * half; c0 < Nw; c0 += 32) {
      float v[16];
      tmem_ld16(lane + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = c0 + i;
        if (n < N && k < K) p[(size_t)n * K + k] = v[i];
        else if (n < N && k == K) p[(size_t)N * K + n] = v[i];
      }
    }
  } else if (!ok) {
    tc_timeout(err, s.bar, phase ^ 1u);
  } else {   // no rows: zero partials
    for (int e = tid; e < N * K + N; e += kTcThreads) p[e] = 0.f;
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// The whole network for inference (the outputs only), one persistent CTA per SM
// looping over 128-row tiles: the five forward weight images stay in shared
// memory for the kernel's life, and each layer's accumulators go from TMEM
// through registers (bias, GELU) straight back into the shared-memory A tile of
// the next layer, so that nothing between the input rows and the five outputs
// touches global memory.  Same arithmetic as the layer-by-layer path: the
// input scaled in FP32, BF16 operands, FP32 accumulation, z + bias in FP32,
// GELU in FP32 rounded to BF16, the output clipped to +-6 standard deviations
// and scaled back.
constexpr float kInferClip = 6.0f;
constexpr int kInferThreads = 512;   // 16 warps: four share each quarter of the TMEM lanes

__global__ void __launch_bounds__(kInferThreads, 1) k_mlp_infer_tc(const float* __restrict__ X, int B,
                                                                const __nv_bfloat16* __restrict__ wimg, MlpImg im,
                                                                MlpDims d, const float* __restrict__ param,
                                                                const float* __restrict__ in_shift,
                                                                const float* __restrict__ in_scale,
                                                                const float* __restrict__ out_shift,
                                                                const float* __restrict__ out_scale,
                                                                int skip_out, int skip_in,
                                                                float* __restrict__ Y, int* err) {
  extern __shared__ __align__(128) unsigned char tc_raw[];
  __nv_bfloat16* W[kMlpLayers];
  size_t off = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    W[l] = reinterpret_cast<__nv_bfloat16*>(tc_raw + off);
    off += (size_t)((d.out[l] + 15) & ~15) * ((d.in[l] + 15) & ~15) * 2;
  }
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(tc_raw + off);   // [128][128] at most
  off += (size_t)kTcRows * kMlpHidden * 2;
  float* nsh = reinterpret_cast<float*>(tc_raw + off);                 // input shift, then scale
  off += 2 * kMlpIn * sizeof(float);
  float* sbias = reinterpret_cast<float*>(tc_raw + off);               // the five layers' biases
  off += (size_t)(4 * kMlpHidden + kMlpOut) * sizeof(float);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(tc_raw + ((off + 15) & ~(size_t)15));
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, grp = warp & 3, quarter = warp >> 2;
  if (warp == 0) tmem_alloc(slot, kMlpHidden);
  if (tid == 0) mbar_init1(bar);
  for (int l = 0; l < kMlpLayers; ++l) {
    const int Kp = (d.in[l] + 15) & ~15, Np = (d.out[l] + 15) & ~15;
    const uint4* src = reinterpret_cast<const uint4*>(wimg + im.fwd[l]);
    uint4* dst = reinterpret_cast<uint4*>(W[l]);
    for (int i = tid; i < Np * Kp / 8; i += kInferThreads) dst[i] = __ldg(src + i);
  }
  for (int k = tid; k < kMlpIn; k += kInferThreads) {
    nsh[k] = in_shift[k];
    nsh[kMlpIn + k] = in_scale[k];
  }
  for (int l = 0, o = 0; l < kMlpLayers; o += d.out[l], ++l)
    for (int n = tid; n < d.out[l]; n += kInferThreads) sbias[o + n] = param[d.boff[l] + n];
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lane = tmem + ((uint32_t)(32 * grp) << 16);
  const int r = 32 * grp + (tid & 31);   // this thread's accumulator row (TMEM lane)
  const int ntiles = (B + kTcRows - 1) / kTcRows;
  unsigned phase = 0;
  bool ok = true;
  unsigned char* a = reinterpret_cast<unsigned char*>(A);
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int b0 = tile * kTcRows, rows = min(kTcRows, B - b0);
    {   // the scaled input rows, BF16, K padded from 40 to 48
      const float4* s4 = reinterpret_cast<const float4*>(X + (size_t)b0 * kMlpIn);
      for (int q = tid; q < kTcRows * kMlpIn / 4; q += kInferThreads) {
        const int e = 4 * q, rr = e / kMlpIn, k = e - rr * kMlpIn;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rr < rows) {
          x = __ldg(s4 + q);
          x.x = (x.x - nsh[k]) * nsh[kMlpIn + k];
          x.y = (x.y - nsh[k + 1]) * nsh[kMlpIn + k + 1];
          x.z = (x.z - nsh[k + 2]) * nsh[kMlpIn + k + 2];
          x.w = (x.w - nsh[k + 3]) * nsh[kMlpIn + k + 3];
        }
        const __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y), hi = __floats2bfloat162_rn(x.z, x.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&lo);
        u.y = *reinterpret_cast<const uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(a + canon(rr, k, kTcRows)) = u;
      }
      for (int rr = tid; rr < kTcRows; rr += kInferThreads)
        *reinterpret_cast<uint4*>(a + canon(rr, kMlpIn, kTcRows)) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int l = 0; l < kMlpLayers && ok; ++l) {
      const int Kp = (d.in[l] + 15) & ~15, Np = (d.out[l] + 15) & ~15;
      ok = mma_tiles(tmem, A, W[l], Np, Kp, false, bar, phase);
      phase ^= 1u;
      if (!ok) break;
      const float* bias = sbias + l * kMlpHidden;
      if (l + 1 < kMlpLayers) {
        // next layer's A: BF16(GELU(z + bias)), 16 columns per load (the four warps on
        // a lane quarter take every fourth group), written as two 16-byte runs of the
        // core-matrix rows (the MMA that read A has completed)
        for (int c0 = 16 * quarter; c0 < Np; c0 += 64) {
          float v[16];
          tmem_ld16(lane + c0, v);
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu_tc(v[2 * i] + bias[c0 + 2 * i]),
                                                            gelu_tc(v[2 * i + 1] + bias[c0 + 2 * i + 1]));
            pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
          }
          *reinterpret_cast<uint4*>(a + canon(r, c0, kTcRows)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(a + canon(r, c0 + 8, kTcRows)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      } else if (quarter == 0) {
        float v[16];
        tmem_ld16(lane, v);
        if (r < rows) {
#pragma unroll
          for (int n = 0; n < kMlpOut; ++n) {
            const float yn = fminf(fmaxf(v[n] + bias[n], -kInferClip), kInferClip);
            const float xs = n == skip_out ? __ldg(X + (size_t)(b0 + r) * kMlpIn + skip_in) : 0.f;
            Y[(size_t)(b0 + r) * kMlpOut + n] = yn / out_scale[n] + out_shift[n] + xs;
          }
        }
      }
    }
  }
  if (!ok) tc_timeout(err, bar, phase ^ 1u);
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kMlpHidden);
}

// Weight images: for every layer, the BF16 weights in the shared-memory layout
// of the forward GEMM's B tile (rows n < Np, columns k < Kp) and of the data
// gradient's (rows k < Kp, columns n < Np), zero in the padding.
MlpImg mlp_images() {
  const MlpDims d = mlp_dims();
  MlpImg im{};
  size_t off = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    const size_t Kp = (size_t)((d.in[l] + 15) & ~15), Np = (size_t)((d.out[l] + 15) & ~15);
    im.fwd[l] = off;
    off += Np * Kp;
    im.bwd[l] = off;
    off += Kp * Np;
  }
  im.total = off;
  return im;
}

__global__ void k_mlp_images(const float* __restrict__ param, __nv_bfloat16* __restrict__ img, MlpDims d, MlpImg im) {
  const int stride = gridDim.x * blockDim.x;
  for (int l = 0; l < kMlpLayers; ++l) {
    const int K = d.in[l], N = d.out[l], Kp = (K + 15) & ~15, Np = (N + 15) & ~15;
    unsigned char* f = reinterpret_cast<unsigned char*>(img + im.fwd[l]);
    unsigned char* b = reinterpret_cast<unsigned char*>(img + im.bwd[l]);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Np * Kp; e += stride) {
      const int n = e / Kp, k = e - n * Kp;
      const __nv_bfloat16 w =
          __float2bfloat16_rn((n < N && k < K) ? param[d.woff[l] + (size_t)n * K + k] : 0.f);
      *reinterpret_cast<__nv_bfloat16*>(f + canon(n, k, Np)) = w;
      *reinterpret_cast<__nv_bfloat16*>(b + canon(k, n, Kp)) = w;
    }
  }
}

cudaError_t mlp_make_images(const float* param, __nv_bfloat16* img, cudaStream_t s) {
  k_mlp_images<<<64, 256, 0, s>>>(param, img, mlp_dims(), mlp_images());
  return cudaGetLastError();
}

// ---- launchers ----
namespace {
uint32_t tmem_cols_host(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// Dynamic shared memory large enough that no more CTAs share an SM than its 512
// tensor-memory columns hold at once, so an allocation never waits.
size_t tc_min_smem(uint32_t ncols) {
  const int fit = 512 / (int)ncols;
  return fit >= 8 ? 0 : (size_t)(228 * 1024) / (size_t)(fit + 1) + 1024;
}

template <typename Kern, typename... Args>
cudaError_t tc_launch(Kern kern, unsigned grid, size_t smem_need, uint32_t ncols, cudaStream_t s, Args... args) {
  if (grid == 0) return cudaSuccess;
  const size_t floor_b = tc_min_smem(ncols);
  const size_t smem = smem_need > floor_b ? smem_need : floor_b;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTcThreads, smem, s>>>(args...);
  return cudaGetLastError();
}
}  // namespace

cudaError_t mlp_fwd_layer_tc(const float* in, int K, bool act_in, const __nv_bfloat16* Wimg, const float* bias, int N,
                             int B, float* out, int* err, cudaStream_t s) {
  if (K > 256 || N > 256) return cudaErrorInvalidValue;
  const int Kp = (K + 15) & ~15, Np = (N + 15) & ~15;
  const size_t smem = tc_smem_bytes(Kp, Np, (size_t)kTcRows * (Np + 4) * sizeof(float));
  return tc_launch(k_mlp_fwd_tc, (unsigned)((B + kTcRows - 1) / kTcRows), smem, tmem_cols_host(Np), s, in, K,
                   act_in ? 1 : 0, Wimg, bias, N, B, out, err);
}

cudaError_t mlp_bwd_data_tc(const float* dz, int N, const __nv_bfloat16* WimgT, int K, int B, const float* zprev,
                            float* out, int* err, cudaStream_t s) {
  if (K > 256 || N > 256) return cudaErrorInvalidValue;
  const int Np = (N + 15) & ~15, Kq = (K + 15) & ~15;
  const size_t smem = tc_smem_bytes(Np, Kq, (size_t)kTcRows * (Kq + 4) * sizeof(float));
  return tc_launch(k_mlp_bwd_data_tc, (unsigned)((B + kTcRows - 1) / kTcRows), smem, tmem_cols_host(Kq), s, dz, N,
                   WimgT, K, B, zprev, out, err);
}

cudaError_t mlp_infer_tc(const float* X, int B, const __nv_bfloat16* wimg, const float* param,
                         const float* in_shift, const float* in_scale, const float* out_shift, const float* out_scale,
                         int skip_out, int skip_in, float* Y, int* err, cudaStream_t s) {
  if (B < 1) return cudaSuccess;
  if (skip_out >= kMlpOut || skip_in >= kMlpIn || (skip_out >= 0 && skip_in < 0)) return cudaErrorInvalidValue;
  const MlpDims d = mlp_dims();
  const MlpImg im = mlp_images();
  size_t smem = 0;
  for (int l = 0; l < kMlpLayers; ++l) smem += (size_t)((d.out[l] + 15) & ~15) * ((d.in[l] + 15) & ~15) * 2;
  smem += (size_t)kTcRows * kMlpHidden * 2 + (2 * kMlpIn + 4 * kMlpHidden + kMlpOut) * sizeof(float);
  smem = ((smem + 15) & ~(size_t)15) + 16;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ntiles = (B + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)std::min(ntiles, std::max(sms, 1));
  k_mlp_infer_tc<<<grid, kInferThreads, smem, s>>>(X, B, wimg, im, d, param, in_shift, in_scale, out_shift, out_scale,
                                                   skip_out, skip_in, Y, err);
  return cudaGetLastError();
}

cudaError_t mlp_wgrad_tc(const float* dz, int N, const float* in, int K, bool act_in, int B, int rows_per_block,
                         int nblk, float* partial, int* err, cudaStream_t s) {
  if (N > kTcRows || K + 1 > 256) return cudaErrorInvalidValue;
  const int Nw = ((K + 1) + 15) & ~15;
  return tc_launch(k_mlp_wgrad_tc, (unsigned)nblk, tc_smem_bytes(kWgK, Nw, 0), tmem_cols_host(Nw), s, dz, N, in, K,
                   act_in ? 1 : 0, B, rows_per_block, partial, err);
}

}  // namespace pnp
