// Device-side data structures and helpers of the edge-subdivision engine.
//
// State layout in HBM (structure of arrays, leading dimension = capacity):
//   X     [D][Vcap]   float64 vertex coordinates
//   Z     [H][Vcap]   current-layer pre-activations (float32, or float64 in
//                     FP64 mode), neuron-major so one neuron's pass reads a
//                     contiguous row; two buffers ping-pong across layers, or
//                     one per layer when the interpolation tape is kept
//   esc   [Vcap]      float32 error scale rho of the vertex's FP32 Z column:
//                     the rms error of z_j is about ||W_j||_2 rho + u/2 |b_j|
//                     (FP32 and mixed precision)
//   exc   [Vcap]      float32 estimate of the vertex's coordinate error
//   SIG   [S][Vcap]   packed sign vectors, 2 bits per entry, word-major
//   EU/EW [Ecap]      int32 edge endpoints (EW = EU + Ecap)
//   list  [2][Ecap]   splitting edges (edge id, V+, V-) of a step, two lists
//                     by neuron parity: one is split while the next neuron's
//                     is built
//   flags [2][Ecap/32] bit e set iff edge e is in the list of that parity
//   table [2][Tcap]   open-addressing hash tables of 2-face keys, by parity
//   cnt   [N+1]       per-neuron counters (slot n+1 belongs to neuron n)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pc {

// Largest input dimension: 8 in libpc.so; the same sources compiled with
// -DPC_MAX_D=10 give libpc_d10.so for D = 9, 10 (its per-vertex Newton
// arrays and shared-memory tiles are sized by it).
#ifndef PC_MAX_D
#define PC_MAX_D 8
#endif
constexpr int kMaxD = PC_MAX_D;
constexpr int kMaxL = 16;
constexpr int kMaxWidth = 256;
constexpr int kMaxEntries = 1024;
constexpr int kMaxWords = kMaxEntries / 32;

constexpr uint64_t kPlus = 1;   // code 01
constexpr uint64_t kMinus = 2;  // code 10
constexpr uint64_t kEvenBits = 0x5555555555555555ull;

constexpr uint64_t kEmpty = ~0ull;       // empty hash slot
constexpr uint64_t kPaired = 1ull << 31; // payload flag: face already paired
constexpr unsigned long long kPaired64 = 1ull << 63;  // same, in the 16-byte slots

constexpr int kBlock = 512;              // threads per CTA in the neuron phases
constexpr int kWarps = kBlock / 32;
constexpr int kMaxGrid = 1024;           // upper bound on CTAs of a phase grid
constexpr int kFilterCap = 2 * kBlock;   // CTA-local list of filtered vertices

// error bits in Global::error
constexpr int kErrPairing = 1;
constexpr int kErrDegenerate = 2;
constexpr int kErrTimeout = 4;
constexpr int kErrProbe = 8;
constexpr int kErrConflict = 16;
constexpr int kErrCorrupt = 32;   // a counter outside its capacity: stop, never index with it
constexpr int kErrVerify = 64;    // a fingerprint pairing failed its exact check (deferred mode)
constexpr int kErrFatal = kErrTimeout | kErrCorrupt;

// halt reasons
constexpr int kHaltV = 1, kHaltE = 2, kHaltT = 4, kHaltTape = 8;

struct NetDesc {
  int L, D, m, N, P, S;
  int precision;         // pc_precision
  int w[kMaxL + 1];      // widths
  int off[kMaxL + 1];    // global index of the first neuron of layer l
  long long wofs[kMaxL]; // offset of W_l in the flat parameter array
  long long bofs[kMaxL]; // offset of b_l
  double lo[kMaxD], hi[kMaxD];
  const double* W64;     // flat parameters, float64 (device copy)
  const float* W32;      // flat parameters rounded to float32
  const float2* WT2;     // per layer W^T (k-major: [K][H]) then b, as (float32 head,
                         // float32 of the remainder): about 48 bits per parameter
  const float* norms;    // per layer: [2l] = max_j ||W_j||_2, [2l+1] = max_j |b_j|
  const float* nrm;      // per neuron n: [3n] = ||W_n||_2, [3n+1] = |b_n|, [3n+2] = 1/||W_n||_2
  float kappa;           // filter factor
  float kappa_sel;       // values with |z| <= kappa_sel x estimate go to FP64: max(kappa, audit band)
  // Polyhedral domain {x : c - A x >= 0} (Section 4.1): facet i of the m
  // entries has the value fc[i] - fA[i, :] x (fA row-major m x D, device).
  // Both null for the box [lo, hi], whose facet 2d is x_d - lo_d and 2d+1
  // is hi_d - x_d.
  const double* fA;
  const double* fc;
  int debug_barrier;     // pc_options.debug_barrier_timeout
  int rd_batch;          // vertices per batch of FP64 re-decisions (rd_batch_size)
};

struct Counters {        // 128 bytes
  long long nV_before, nE_before;
  long long nsplit;      // splitting edges of the step (counted while the previous step runs)
  long long nkeys, npairs;
  long long nfilter, nundecided, ndegenerate;
  long long tsize;
  long long pruned_e1;   // 0, or 1 + the edge count left by pruning after this step
  long long pad[6];
};

struct Global {
  int halted_at;         // -1, or the neuron whose step ran out of capacity
  int halt_reason;
  int error;             // sticky kErr* bits
  int flips;             // FP64 re-decisions that changed the FP32 sign
  int flip_margin_bits;  // largest |z| / (FP32 error estimate) among them (float bits)
  int missed;            // audit band: wrong FP32 signs beyond kappa (not written back)
  int missed_margin_bits;
  unsigned int barrier;  // grid barrier arrival counter (reset per launch)
  unsigned int barrier_extra;  // arrivals a barrier waits for beyond the grid: 0, or 1 to test the timeout path
  long long need_v, need_e, need_t;
  long long polished;
  int diag_site;         // first failed consistency check (1 forward product, 2 classify, 3 split), 0: none
  int diag_n;            // its neuron (layer for the forward product)
  long long diag_a, diag_b, diag_c;  // the values it found
};

// Flags kErrCorrupt and records the first failing check with its values.
__device__ __forceinline__ void report_corrupt(Global* g, int site, int n, long long a, long long b, long long c) {
  if (atomicCAS(&g->diag_site, 0, site) == 0) {
    g->diag_n = n;
    g->diag_a = a;
    g->diag_b = b;
    g->diag_c = c;
  }
  atomicOr(&g->error, kErrCorrupt);
}

struct State {
  long long Vcap, Ecap, Tcap;
  double* X;
  void* Z[kMaxL];        // values of layer l (ping-pong pair unless the tape keeps every layer)
  float* esc;            // FP32 value error estimate per vertex
  float* exc;            // coordinate error estimate per vertex (absolute)
  uint64_t* SIG;
  int32_t* EU;
  int32_t* EW;
  int4* list[2];         // splitting edges (edge, V+, V-, 0) of the steps of each neuron parity
  uint32_t* flags[2];    // bit e of flags[a]: edge e is in list[a]
  uint64_t* table;       // two hash tables of 2 Tcap words each (neuron parity 0, 1); slots of
                         // 16 bytes (fingerprint, payload), or 8 bytes (tag | payload) inline
  int4* vlist;           // per edge: (v_a, v_b, zero ordinals, neuron + 1) of a pairing edge, else 0
  int deferred;          // pairings by 64-bit fingerprint, verified after the extraction
  Counters* cnt;
  Global* g;
  // interpolation tape (optional): parents and t of every created vertex
  int32_t* tape_pq;      // [2][tape_cap] indexed by vertex id
  double* tape_t;        // [tape_cap]
  long long tape_cap;
  int keep_tape;
};

// splitmix64 finalizer (Steele, Lea, Flood 2014) as the per-word mixer of the
// 2-face fingerprint.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// 128-bit compare-and-swap of a 16-byte-aligned slot {lo, hi} (sm_90+).
__device__ __forceinline__ void cas128(unsigned long long* addr, unsigned long long cmp_lo, unsigned long long cmp_hi,
                                       unsigned long long new_lo, unsigned long long new_hi,
                                       unsigned long long& old_lo, unsigned long long& old_hi) {
  asm volatile(
      "{\n\t.reg .b128 c, n, d;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 n, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], c, n;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(old_lo), "=l"(old_hi)
      : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(addr)
      : "memory");
}

__device__ __forceinline__ uint64_t word_hash(int w, uint64_t v) {
  return mix64(v ^ (0x9e3779b97f4a7c15ull * (uint64_t)(w + 1)));
}

// Bit 2r is set iff entry 32w + r is valid (< n_valid) and has code 00.
__device__ __forceinline__ uint64_t zero_mask(uint64_t s, int w, int n_valid) {
  const int cnt = n_valid - 32 * w;
  if (cnt <= 0) return 0;
  const uint64_t valid = cnt >= 32 ? kEvenBits : (((1ull << (2 * cnt)) - 1) & kEvenBits);
  const uint64_t nz = (s | (s >> 1)) & kEvenBits;
  return ~nz & valid;
}

__device__ __forceinline__ uint64_t code_at(const uint64_t* SIG, long long Vcap, long long v, int entry) {
  return (SIG[(long long)(entry >> 5) * Vcap + v] >> (2 * (entry & 31))) & 3ull;
}

__device__ __forceinline__ long long atomic_add_ll(long long* p, long long x) {
  return (long long)atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)x);
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool stopped(const State& st) {
  return *(volatile int*)&st.g->halted_at >= 0 || (*(volatile int*)&st.g->error & kErrFatal);
}

// The stop flags read once per CTA and shared by all its threads.  Another
// CTA of the same launch may raise a flag (a capacity halt, an error) while
// this CTA's warps start; a per-thread read would then let part of the CTA
// return and leave the rest waiting at barriers with partial block data.
__device__ __forceinline__ bool cta_stopped(const State& st) {
  return __syncthreads_or(threadIdx.x == 0 && stopped(st)) != 0;
}

// Grid-wide barrier for cooperative launches.  Bounded: after ~0.5 s of
// waiting it sets kErrTimeout and returns false (the caller then exits).
// With g->barrier_extra = 1 (a test of this path) the target is one arrival
// beyond the grid, which never comes, and the limit is 4096 polls.
__device__ __forceinline__ bool grid_barrier(Global* g, unsigned int& passed) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    passed += 1;
    const unsigned int extra = *(volatile unsigned int*)&g->barrier_extra;
    const unsigned int target = passed * gridDim.x + extra;
    const long long limit = extra ? (1ll << 12) : (1ll << 22);
    __threadfence();
    atomicAdd(&g->barrier, 1u);
    int ok = 1;
    long long spins = 0;
    while (ld_acquire_u32(&g->barrier) < target) {
      if (++spins > limit) {
        atomicOr(&g->error, kErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace pc
