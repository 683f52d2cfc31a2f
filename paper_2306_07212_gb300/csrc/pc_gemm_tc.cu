// Step (1) of Section 4.2 at the start of a hidden or output layer l >= 1:
//   Z_l = W_l a + b_l for every current vertex, a_k = z_k of layer l-1 if the
//   vertex's sign entry for that neuron is + and 0 otherwise (the vertex's own
//   affine piece, Eq. 4 with the stored activation pattern).
// on the fifth-generation tensor cores (tcgen05) as a 3xTF32 product: both
// operands are split into a TF32 head and a TF32 tail, x = x_hi + x_lo, and
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 in tensor memory (the dropped tail x tail term is
// below 2^-22 relative), which keeps the FP32 accuracy of the value arrays.
//
// Shape of one tile: M = 128 vertices (tensor-memory lanes), N = H_l neurons
// padded to a multiple of 16 (columns), K = H_{l-1} inputs in chunks of 32.
// Operands live in shared memory in the K-major 128-byte-swizzle layout: row
// r of a chunk (a vertex for A, a neuron for B) holds 32 values (128 B); the
// 16-byte groups of row r are permuted by XOR with r mod 8; 8-row groups are
// 1024 B apart.  W_l is split and staged once per CTA; activation tiles are
// gathered from the neuron-major value rows (coalesced over vertices), masked
// by the sign words, split, and written by the 128 threads (one vertex each).
// One elected thread issues the MMAs and commits them to an mbarrier; the
// epilogue reads the accumulator rows back with tcgen05.ld (thread t holds
// vertex t), adds b_l and stores the value rows, coalesced over vertices,
// together with the per-vertex FP32 error scale of the layer.
#include <cuda_runtime.h>

#include <cstdint>

#include "pc_ctx.h"
#include "pc_device.cuh"

namespace pc {

constexpr int kTcTileM = 128;    // vertices per tile (tensor-memory lanes)
constexpr int kTcChunkK = 32;    // inputs per 128-byte swizzle row
constexpr int kTcMaxN = 128;     // widest layer on this path
constexpr int kTcMaxK = 128;     // widest input on this path
constexpr int kTcAChunkBytes = kTcTileM * 128;
// B (head and tail of W^T for all of K) + A (head and tail of one chunk) +
// 1024 B for aligning the base + 1024 B of slack behind the operands
constexpr int kTcSmemMax = 2 * (kTcMaxK / kTcChunkK) * kTcMaxN * 128 + 2 * kTcAChunkBytes + 2048;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Byte offset of element (row, k) of a K-major SW128 chunk (1024-B aligned).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  const uint32_t off = static_cast<uint32_t>(row) * 128u + static_cast<uint32_t>(k) * 4u;
  return off ^ (((off >> 7) & 7u) << 4);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;          // leading byte offset (unused here): 16 B
  d |= static_cast<uint64_t>(1024 >> 4) << 32;  // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;          // version
  d |= static_cast<uint64_t>(2) << 61;          // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the MMAs committed to bar (phase parity).  False after
// the limit: the caller records kErrTimeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long spins = 0; spins < (1ll << 22); ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) r[q] = __uint_as_float(u[q]);
}

__global__ void __launch_bounds__(kTcTileM, 1) k_gemm_tc(NetDesc net, State st, int l, int Npad, int Kpad) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ float bias[kTcMaxN];
  __shared__ int fail;
  if (cta_stopped(st)) return;
  const Counters* c = st.cnt + net.off[l];
  const long long nV = c->nV_before + c->nsplit;
  if (nV < 0 || nV > st.Vcap) {  // uniform: every thread reads the same counters
    if (threadIdx.x == 0) report_corrupt(st.g, 1, l, nV, st.Vcap, 0);
    return;
  }
  const int tid = threadIdx.x, warp = tid >> 5;
  const int H = net.w[l + 1], K = net.w[l], KC = Kpad / kTcChunkK;
  const uint32_t chunkB = static_cast<uint32_t>(Npad) * 128u;
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  unsigned char* Bhi = base;
  unsigned char* Blo = Bhi + KC * chunkB;
  unsigned char* Ahi = Blo + KC * chunkB;
  unsigned char* Alo = Ahi + kTcAChunkBytes;

  // W^T (rows: neurons, K-major), split into TF32 head and tail from FP64
  const double* W = net.W64 + net.wofs[l];
  for (int idx = tid; idx < Npad * Kpad; idx += blockDim.x) {
    const int j = idx / Kpad, k = idx % Kpad;
    const double w = (j < H && k < K) ? W[(long long)j * K + k] : 0.0;
    const uint32_t hi = to_tf32(static_cast<float>(w));
    const uint32_t lo = to_tf32(static_cast<float>(w - static_cast<double>(__uint_as_float(hi))));
    const uint32_t off = (k / kTcChunkK) * chunkB + sw128_offset(j, k % kTcChunkK);
    *reinterpret_cast<uint32_t*>(Bhi + off) = hi;
    *reinterpret_cast<uint32_t*>(Blo + off) = lo;
  }
  for (int j = tid; j < kTcMaxN; j += blockDim.x)
    bias[j] = j < H ? static_cast<float>(net.W64[net.bofs[l] + j]) : 0.f;
  if (tid == 0) {
    fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
  }
  int ncols = 32;
  while (ncols < Npad) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tf32_idesc(kTcTileM, Npad);
  const long long Vcap = st.Vcap;
  const float* Zin = static_cast<const float*>(st.Z[l - 1]);
  float* Zout = static_cast<float*>(st.Z[l]);
  const int ebase = net.m + net.off[l - 1];
  uint32_t phase = 0;

  for (long long tile = blockIdx.x; tile * kTcTileM < nV; tile += gridDim.x) {
    const long long v = tile * kTcTileM + tid;
    const bool valid = v < nV;
    float a2 = 0.f;
    for (int q = 0; q < KC; ++q) {
      // gather, mask and split this vertex's 32 inputs of chunk q
      uint64_t word = 0;
      int cw = -1;
#pragma unroll
      for (int g = 0; g < kTcChunkK / 4; ++g) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = q * kTcChunkK + g * 4 + e;
          float a = 0.f;
          if (valid && k < K) {
            const int entry = ebase + k, wi = entry >> 5;
            if (wi != cw) {
              word = st.SIG[(long long)wi * Vcap + v];
              cw = wi;
            }
            if (((word >> (2 * (entry & 31))) & 3ull) == kPlus) a = Zin[(long long)k * Vcap + v];
          }
          a2 = fmaf(a, a, a2);
          hi[e] = to_tf32(a);
          lo[e] = to_tf32(a - __uint_as_float(hi[e]));
        }
        const uint32_t off = sw128_offset(tid, g * 4);
        *reinterpret_cast<uint4*>(Ahi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(Alo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
        const uint32_t bh = smem_u32(Bhi + q * chunkB), bl = smem_u32(Blo + q * chunkB);
#pragma unroll
        for (int kk = 0; kk < kTcChunkK / 8; ++kk) {  // 8 TF32 (32 B) per MMA
          const uint32_t o = kk * 32;
          mma_tf32(tmem, sw128_desc(al + o), sw128_desc(bh + o), idesc, (q > 0 || kk > 0) ? 1 : 0);
          mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1);
          mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bh + o), idesc, 1);
        }
        mma_commit(&bar);
      }
      __syncwarp();
      // the chunk buffers are rewritten next: wait until the MMAs have read them
      if (!mbar_wait(&bar, phase)) fail = 1;
      phase ^= 1u;
      tc_fence_after();
      if (__syncthreads_or(fail)) break;
    }
    if (fail) break;
    // epilogue: accumulator row tid -> value rows of layer l (+ b_l)
    for (int j0 = 0; j0 < Npad; j0 += 16) {
      float r[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(j0), r);
      if (valid) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
          if (j0 + jj < H) Zout[(long long)(j0 + jj) * Vcap + v] = r[jj] + bias[j0 + jj];
      }
    }
    if (valid) {
      // FP32 error scale of the layer's values: u/2 ||a||_2 for the
      // rounding, and the previous layer's scale carried through W_{l-1}
      const float u = 5.9604645e-8f;  // 2^-24
      float rho = 0.5f * u * sqrtf(a2);
      const float inh = net.norms[2 * (l - 1)] * st.esc[v] + 0.5f * u * net.norms[2 * (l - 1) + 1];
      rho = sqrtf(rho * rho + inh * inh);
      st.esc[v] = rho;
    }
    // the next tile's MMAs overwrite the accumulator: all reads done first
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (fail && tid == 0) atomicOr(&st.g->error, kErrTimeout);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace pc

using namespace pc;

// Eligible: a hidden/output layer (l >= 1) with FP32 values and
// H_l, H_{l-1} <= 128.
bool pc_gemm_tc_eligible(const NetDesc& net, int l) {
  return l >= 1 && net.w[l + 1] <= kTcMaxN && net.w[l] <= kTcMaxK;
}

cudaError_t pc_gemm_tc_set_attributes() {
  return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax);
}

cudaError_t pc_gemm_tc_launch(const NetDesc& net, const State& st, int l, long long vcap_tiles, int num_sms,
                              cudaStream_t stream) {
  const int H = net.w[l + 1], K = net.w[l];
  const int Npad = (H + 15) / 16 * 16;
  const int Kpad = (K + kTcChunkK - 1) / kTcChunkK * kTcChunkK;
  const size_t smem = static_cast<size_t>(2 * (Kpad / kTcChunkK) * Npad * 128 + 2 * kTcAChunkBytes + 2048);
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>(num_sms, vcap_tiles)));
  k_gemm_tc<<<grid, kTcTileM, smem, stream>>>(net, st, l, Npad, Kpad);
  return cudaGetLastError();
}
