// Step (1) of Section 4.2 at the start of a hidden or output layer l >= 1:
//   Z_l = W_l a + b_l for every current vertex, a_k = z_k of layer l-1 if the
//   vertex's sign entry for that neuron is + and 0 otherwise (the vertex's own
//   affine piece, Eq. 4 with the stored activation pattern).
// on the fifth-generation tensor cores (tcgen05) as split-TF32 products
// accumulated in FP32 in tensor memory.  Both operands are split into TF32
// pieces, x = x0 + x1 (+ x2), and the products of pieces whose indices sum
// to at most P - 1 are accumulated:
//   P = 2 (3xTF32):  A0 B0 + A0 B1 + A1 B0, about 22 bits per product;
//   P = 3 (default): the six products up to index sum 2; the three-piece
//                    split is exact for an FP32 input, so the product has
//                    the FP32 accuracy that the value arrays and their
//                    error scale assume.
//
// Shape of one tile: M = 128 vertices (tensor-memory lanes), N = H_l neurons
// padded to a multiple of 16 (columns), K = H_{l-1} inputs in chunks of 32.
// Operands live in shared memory in the K-major 128-byte-swizzle layout: row
// r of a chunk (a vertex for A, a neuron for B) holds 32 values (128 B); the
// 16-byte groups of row r are permuted by XOR with r mod 8; 8-row groups are
// 1024 B apart.  The pieces of W_l are split from FP64 and staged once per
// CTA.  Activation chunks are gathered from the neuron-major value rows
// (coalesced over vertices), masked by the sign words and split in registers
// by the 128 threads (one vertex each); each piece goes to one of two
// shared-memory buffers, so the next piece is written while the MMAs of the
// previous one run.  One elected thread issues the MMAs and commits them to
// the buffer's mbarrier; the epilogue reads the accumulator rows back with
// tcgen05.ld (thread t holds vertex t), adds b_l and stores the value rows,
// coalesced over vertices, together with the per-vertex error scale.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pc_ctx.h"
#include "pc_device.cuh"

namespace pc {

constexpr int kTcTileM = 128;    // vertices per tile (tensor-memory lanes)
constexpr int kTcChunkK = 32;    // inputs per 128-byte swizzle row
constexpr int kTcMaxN = 128;     // widest layer on this path
constexpr int kTcMaxK = 128;     // widest input on this path
constexpr int kTcAChunkBytes = kTcTileM * 128;
// W^T pieces for all of K + two activation buffers (one piece of one chunk
// each) + 1024 B for aligning the base + 1024 B of slack behind the operands
__host__ __device__ constexpr int tc_smem_bytes(int pieces, int kc, int npad) {
  return pieces * kc * npad * 128 + 2 * kTcAChunkBytes + 2048;
}
constexpr int kTcSmemMax = tc_smem_bytes(3, kTcMaxK / kTcChunkK, kTcMaxN);

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

// PIECES = 2: the 3xTF32 product (head x head + head x tail + tail x head);
// each product keeps about 22 bits.  PIECES = 3: a three-piece split
// (x = x0 + x1 + x2, which is exact for an FP32 x), with the six products
// whose piece indices sum to at most 2; each product keeps about 33 bits,
// so the result has the FP32 accuracy of the SIMT product.
//
// Accumulation.  The tensor core adds each MMA's result to its FP32
// accumulator with a rounding that does not average out over many adds
// (measured: coordinate errors grew in proportion to the MMAs per
// accumulator).  So every K step (8 inputs) gets its own accumulator while
// tensor memory allows (512 columns: 8 accumulators of 64 columns, 4 of 128),
// the products of a step are issued from the smallest to the largest (tail
// pieces first, head x head last), and the epilogue sums the accumulators
// with FP32 round-to-nearest adds.
template <int PIECES>
__global__ void __launch_bounds__(kTcTileM, 1) k_gemm_tc(NetDesc net, State st, int l, int Npad, int Kpad) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ uint64_t bar[2];
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
  unsigned char* Bp = base;                         // [piece][chunk][Npad rows][128 B]
  unsigned char* Abuf = Bp + PIECES * KC * chunkB;  // two buffers of one chunk piece

  // W^T (rows: neurons, K-major), split into TF32 pieces from FP64
  const double* W = net.W64 + net.wofs[l];
  for (int idx = tid; idx < Npad * Kpad; idx += blockDim.x) {
    const int j = idx / Kpad, k = idx % Kpad;
    double r = (j < H && k < K) ? W[(long long)j * K + k] : 0.0;
    const uint32_t off = (k / kTcChunkK) * chunkB + sw128_offset(j, k % kTcChunkK);
#pragma unroll
    for (int pc = 0; pc < PIECES; ++pc) {
      const uint32_t w = to_tf32(static_cast<float>(r));
      *reinterpret_cast<uint32_t*>(Bp + pc * KC * chunkB + off) = w;
      r -= static_cast<double>(__uint_as_float(w));
    }
  }
  for (int j = tid; j < kTcMaxN; j += blockDim.x)
    bias[j] = j < H ? static_cast<float>(net.W64[net.bofs[l] + j]) : 0.f;
  if (tid == 0) {
    fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])) : "memory");
  }
  int stride = 32;  // columns per accumulator (a power of two >= Npad)
  while (stride < Npad) stride <<= 1;
  const int ksteps = Kpad / 8;
  int nacc = 1;
  while (nacc * 2 <= ksteps && nacc * 2 * stride <= 512) nacc <<= 1;
  const int ncols = nacc * stride;
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
  // buffer b's MMAs: committed (pending[b]) and the parity of their phase
  uint32_t parity[2] = {0u, 0u};
  int pending[2] = {0, 0};
  int stage = 0;  // A buffer to fill next

  for (long long tile = blockIdx.x; tile * kTcTileM < nV; tile += gridDim.x) {
    const long long v = tile * kTcTileM + tid;
    const bool valid = v < nV;
    float a2 = 0.f;
    for (int q = 0; q < KC && !fail; ++q) {
      // this vertex's 32 inputs of chunk q, masked by its activation pattern
      float x[kTcChunkK];
      uint64_t word = 0;
      int cw = -1;
#pragma unroll
      for (int k0 = 0; k0 < kTcChunkK; ++k0) {
        const int k = q * kTcChunkK + k0;
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
        x[k0] = a;
      }
      for (int pa = PIECES - 1; pa >= 0; --pa) {  // tail pieces first
        const int b = stage;
        stage ^= 1;
        // the buffer is free once the MMAs that read it have completed
        if (pending[b]) {
          if (!mbar_wait(&bar[b], parity[b])) fail = 1;
          parity[b] ^= 1u;
          pending[b] = 0;
        }
        unsigned char* A = Abuf + b * kTcAChunkBytes;
#pragma unroll
        for (int g = 0; g < kTcChunkK / 4; ++g) {
          uint32_t u[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {  // piece pa of x: split again from the value
            float r = x[g * 4 + e];
            uint32_t pc = to_tf32(r);
#pragma unroll
            for (int k = 0; k < PIECES - 1; ++k)
              if (k < pa) {
                r -= __uint_as_float(pc);
                pc = to_tf32(r);
              }
            u[e] = pc;
          }
          *reinterpret_cast<uint4*>(A + sw128_offset(tid, g * 4)) = make_uint4(u[0], u[1], u[2], u[3]);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !fail) {
          const uint32_t aa = smem_u32(A);
#pragma unroll
          for (int kk = 0; kk < kTcChunkK / 8; ++kk) {  // 8 TF32 (32 B) per MMA
            const uint32_t o = kk * 32;
            const int s = q * (kTcChunkK / 8) + kk;
            const uint32_t dacc = tmem + static_cast<uint32_t>((s % nacc) * stride);
            for (int pw = PIECES - 1 - pa; pw >= 0; --pw) {  // smallest products first
              // the first product into an accumulator overwrites it
              const bool fresh = s < nacc && pa == PIECES - 1 && pw == 0;
              const uint32_t bb = smem_u32(Bp + (pw * KC + q) * chunkB);
              mma_tf32(dacc, sw128_desc(aa + o), sw128_desc(bb + o), idesc, fresh ? 0 : 1);
            }
          }
          mma_commit(&bar[b]);
        }
        pending[b] = 1;
      }
      if (__syncthreads_or(fail)) break;
    }
    // all of this tile's MMAs complete before the accumulator is read
    for (int b = 0; b < 2; ++b)
      if (pending[b]) {
        if (!mbar_wait(&bar[b], parity[b])) fail = 1;
        parity[b] ^= 1u;
        pending[b] = 0;
      }
    tc_fence_after();
    if (__syncthreads_or(fail)) break;
    // epilogue: accumulator row tid -> value rows of layer l (+ b_l)
    for (int j0 = 0; j0 < Npad; j0 += 16) {
      float r[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(j0), r);
      for (int ia = 1; ia < nacc && ia < ksteps; ++ia) {
        float r2[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(ia * stride + j0), r2);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) r[jj] += r2[jj];
      }
      if (valid) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
          if (j0 + jj < H) Zout[(long long)(j0 + jj) * Vcap + v] = r[jj] + bias[j0 + jj];
      }
    }
    if (valid) {
      // error scale of the layer's values: the rounding of the product
      // (u/2 ||a||_2 for FP32 accuracy; 2^-21 ||a||_2 for 3xTF32, whose
      // products keep about 22 bits) and the previous layer's scale carried
      // through W_{l-1}
      // (several K steps sharing an accumulator add one rounding each)
      const float u = 5.9604645e-8f;  // 2^-24
      const float share = static_cast<float>((ksteps + nacc - 1) / nacc);
      float rho = (PIECES == 2 ? 8.f * u : 0.5f * u * share) * sqrtf(a2);
      const float inh = net.norms[2 * (l - 1)] * st.esc[v] + 0.5f * u * net.norms[2 * (l - 1) + 1];
      rho = sqrtf(rho * rho + inh * inh);
      st.esc[v] = rho;
    }
    // the next tile's MMAs overwrite the accumulator: all reads done first
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // nothing may still read shared memory or write tensor memory at exit
  for (int b = 0; b < 2; ++b)
    if (pending[b] && !mbar_wait(&bar[b], parity[b])) fail = 1;
  if (fail && tid == 0) atomicOr(&st.g->error, kErrTimeout);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}


// The same product, scheduled for overlap and occupancy (layers whose
// operands fit: all pieces of one 32-input chunk get their own buffer).
// Per chunk: the pieces are written, one barrier, one thread issues the
// chunk's MMAs (one accumulator per 8-input K step, tail products first),
// the next chunk is gathered while they run, and the chunk's four
// accumulators are read back into a running FP32 sum in K-step order -- the
// sum the epilogue of k_gemm_tc forms, so the results agree bit for bit
// where k_gemm_tc gives every K step its own accumulator.  Tensor memory
// holds one chunk's accumulators (4 x 64 columns for layers up to 64 wide),
// so two CTAs share an SM.
__device__ __forceinline__ void gather_chunk(const State& st, const float* Zin, long long Vcap, long long v,
                                             bool valid, int q, int K, int ebase, float (&x)[kTcChunkK]) {
  uint64_t word = 0;
  int cw = -1;
#pragma unroll
  for (int k0 = 0; k0 < kTcChunkK; ++k0) {
    const int k = q * kTcChunkK + k0;
    float a = 0.f;
    if (valid && k < K) {
      const int entry = ebase + k, wi = entry >> 5;
      if (wi != cw) {
        word = st.SIG[(long long)wi * Vcap + v];
        cw = wi;
      }
      if (((word >> (2 * (entry & 31))) & 3ull) == kPlus) a = Zin[(long long)k * Vcap + v];
    }
    x[k0] = a;
  }
}

template <int PIECES>
__global__ void __launch_bounds__(kTcTileM, 2) k_gemm_tc2(NetDesc net, State st, int l, int Npad, int Kpad) {
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
  unsigned char* Bp = base;                         // [piece][chunk][Npad rows][128 B]
  unsigned char* Abuf = Bp + PIECES * KC * chunkB;  // one buffer per piece of a chunk
  const double* W = net.W64 + net.wofs[l];
  for (int idx = tid; idx < Npad * Kpad; idx += blockDim.x) {
    const int j = idx / Kpad, k = idx % Kpad;
    double r = (j < H && k < K) ? W[(long long)j * K + k] : 0.0;
    const uint32_t off = (k / kTcChunkK) * chunkB + sw128_offset(j, k % kTcChunkK);
#pragma unroll
    for (int pc = 0; pc < PIECES; ++pc) {
      const uint32_t w = to_tf32(static_cast<float>(r));
      *reinterpret_cast<uint32_t*>(Bp + pc * KC * chunkB + off) = w;
      r -= static_cast<double>(__uint_as_float(w));
    }
  }
  for (int j = tid; j < kTcMaxN; j += blockDim.x)
    bias[j] = j < H ? static_cast<float>(net.W64[net.bofs[l] + j]) : 0.f;
  if (tid == 0) {
    fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
  }
  int stride = 32;  // columns per accumulator (a power of two >= Npad)
  while (stride < Npad) stride <<= 1;
  constexpr int kSteps = kTcChunkK / 8;  // K steps (accumulators) per chunk
  const int ncols = kSteps * stride;
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
  const int ng = Npad / 16;  // 16-column groups of the output
  uint32_t parity = 0u;
  float x[kTcChunkK];  // the chunk being split; the next one is gathered during the MMAs

  for (long long tile = blockIdx.x; tile * kTcTileM < nV; tile += gridDim.x) {
    const long long v = tile * kTcTileM + tid;
    const bool valid = v < nV;
    float acc[kTcMaxN];  // running sum of the K steps' accumulators (row tid)
#pragma unroll
    for (int j = 0; j < kTcMaxN; ++j) acc[j] = 0.f;
    float a2 = 0.f;
    gather_chunk(st, Zin, Vcap, v, valid, 0, K, ebase, x);
    for (int q = 0; q < KC; ++q) {
      // the pieces of this chunk (the previous chunk's MMAs have completed)
#pragma unroll
      for (int k0 = 0; k0 < kTcChunkK; ++k0) a2 = fmaf(x[k0], x[k0], a2);
#pragma unroll
      for (int pa = 0; pa < PIECES; ++pa) {
        unsigned char* A = Abuf + pa * kTcAChunkBytes;
#pragma unroll
        for (int g = 0; g < kTcChunkK / 4; ++g) {
          uint32_t u[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {  // piece pa of x: split again from the value
            float r = x[g * 4 + e];
            uint32_t pc = to_tf32(r);
#pragma unroll
            for (int kk = 0; kk < PIECES - 1; ++kk)
              if (kk < pa) {
                r -= __uint_as_float(pc);
                pc = to_tf32(r);
              }
            u[e] = pc;
          }
          *reinterpret_cast<uint4*>(A + sw128_offset(tid, g * 4)) = make_uint4(u[0], u[1], u[2], u[3]);
        }
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0 && !fail) {
#pragma unroll
        for (int kk = 0; kk < kSteps; ++kk) {  // 8 TF32 (32 B) per MMA
          const uint32_t o = kk * 32;
          const uint32_t dacc = tmem + static_cast<uint32_t>(kk * stride);
          bool fresh = true;  // the first product into an accumulator overwrites it
          for (int pa = PIECES - 1; pa >= 0; --pa)      // tail pieces of the values first,
            for (int pw = PIECES - 1 - pa; pw >= 0; --pw) {  // then smaller products first
              const uint32_t aa = smem_u32(Abuf + pa * kTcAChunkBytes);
              const uint32_t bb = smem_u32(Bp + (pw * KC + q) * chunkB);
              mma_tf32(dacc, sw128_desc(aa + o), sw128_desc(bb + o), idesc, fresh ? 0 : 1);
              fresh = false;
            }
        }
        mma_commit(&bar);
      }
      if (q + 1 < KC) gather_chunk(st, Zin, Vcap, v, valid, q + 1, K, ebase, x);  // while the MMAs run
      if (!mbar_wait(&bar, parity)) fail = 1;
      parity ^= 1u;
      tc_fence_after();
      // this chunk's K steps, in order, into the running sum
#pragma unroll
      for (int kk = 0; kk < kSteps; ++kk) {
#pragma unroll
        for (int g = 0; g < kTcMaxN / 16; ++g) {
          if (g >= ng) break;
          float r[16];
          tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(kk * stride + g * 16), r);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) acc[g * 16 + jj] += r[jj];
        }
      }
      tc_fence_before();
      if (__syncthreads_or(fail)) break;
    }
    if (fail) break;
    if (valid) {
#pragma unroll
      for (int g = 0; g < kTcMaxN / 16; ++g) {
        if (g >= ng) break;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
          if (g * 16 + jj < H) Zout[(long long)(g * 16 + jj) * Vcap + v] = acc[g * 16 + jj] + bias[g * 16 + jj];
      }
      // error scale (as in k_gemm_tc with one accumulator per K step)
      const float u = 5.9604645e-8f;  // 2^-24
      float rho = (PIECES == 2 ? 8.f * u : 0.5f * u) * sqrtf(a2);
      const float inh = net.norms[2 * (l - 1)] * st.esc[v] + 0.5f * u * net.norms[2 * (l - 1) + 1];
      rho = sqrtf(rho * rho + inh * inh);
      st.esc[v] = rho;
    }
  }
  if (fail && tid == 0) atomicOr(&st.g->error, kErrTimeout);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
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

// Shared memory of k_gemm_tc2: W^T pieces for all of K, one buffer per piece
// of a chunk, alignment and slack.
__host__ __device__ constexpr int tc2_smem_bytes(int pieces, int kc, int npad) {
  return pieces * kc * npad * 128 + pieces * kTcAChunkBytes + 2048;
}
constexpr int kTc2SmemMax = 220 * 1024;  // dynamic; the static shared memory comes on top

cudaError_t pc_gemm_tc_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax);
  const cudaError_t e2 = cudaFuncSetAttribute(k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax);
  const cudaError_t e3 = cudaFuncSetAttribute(k_gemm_tc2<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTc2SmemMax);
  const cudaError_t e4 = cudaFuncSetAttribute(k_gemm_tc2<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTc2SmemMax);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  return e3 != cudaSuccess ? e3 : e4;
}

cudaError_t pc_gemm_tc_launch(const NetDesc& net, const State& st, int l, long long vcap_tiles, int num_sms,
                              int pieces, cudaStream_t stream) {
  const int H = net.w[l + 1], K = net.w[l];
  const int Npad = (H + 15) / 16 * 16;
  const int Kpad = (K + kTcChunkK - 1) / kTcChunkK * kTcChunkK;
  const size_t smem2 = static_cast<size_t>(tc2_smem_bytes(pieces, Kpad / kTcChunkK, Npad));
  if (smem2 <= static_cast<size_t>(kTc2SmemMax)) {
    int stride = 32;
    while (stride < Npad) stride <<= 1;
    const int tmem_per_sm = 512 / (4 * stride);
    const int per_sm = std::max(1, std::min({2, tmem_per_sm, static_cast<int>(228 * 1024 / (smem2 + 1024))}));
    const int grid =
        static_cast<int>(std::max<long long>(1, std::min<long long>((long long)num_sms * per_sm, vcap_tiles)));
    if (pieces == 3) k_gemm_tc2<3><<<grid, kTcTileM, smem2, stream>>>(net, st, l, Npad, Kpad);
    else k_gemm_tc2<2><<<grid, kTcTileM, smem2, stream>>>(net, st, l, Npad, Kpad);
    return cudaGetLastError();
  }
  const size_t smem = static_cast<size_t>(tc_smem_bytes(pieces, Kpad / kTcChunkK, Npad));
  // CTAs per SM that shared and tensor memory allow (the kernel allocates
  // accumulators up to 512 columns; a CTA waits in tcgen05.alloc while
  // another CTA on its SM holds the columns)
  int stride = 32;
  while (stride < Npad) stride <<= 1;
  int nacc = 1;
  while (nacc * 2 <= Kpad / 8 && nacc * 2 * stride <= 512) nacc <<= 1;
  const int tmem_per_sm = 512 / (nacc * stride);
  const int per_sm = std::max(1, std::min({4, tmem_per_sm, static_cast<int>(228 * 1024 / (smem + 1024))}));
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>((long long)num_sms * per_sm, vcap_tiles)));
  if (pieces == 3) k_gemm_tc<3><<<grid, kTcTileM, smem, stream>>>(net, st, l, Npad, Kpad);
  else k_gemm_tc<2><<<grid, kTcTileM, smem, stream>>>(net, st, l, Npad, Kpad);
  return cudaGetLastError();
}
