// Optional canonical output order (pc_options.canonical).
//
// The extraction numbers vertices in creation order and emits intersecting
// edges in the order the pairings complete, which varies from run to run.
// With canonical order the result is put in one fixed order after the last
// step: vertices sorted by their packed sign vectors (word 0 most
// significant, each 64-bit word compared as an unsigned number; sign vectors
// are unique under genericity, Section 4.1), edges renumbered to the new
// vertex ids and sorted by (smaller endpoint, larger endpoint).  Two
// extractions of the same network and box then return identical arrays.
//
// Sorting: stable least-significant-digit radix sort of an index
// permutation, one 8-bit digit per pass.  The items are cut into tiles of
// kCanonTile; one thread per tile counts its digits (k_digit_count), one CTA
// turns the counts into exclusive start offsets (bucket-major, so equal
// digits keep tile order; k_scan_counts), and one thread per tile scatters
// its items in order (k_digit_scatter), which keeps every pass stable.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pc_ctx.h"
#include "pc_device.cuh"

namespace pc {

constexpr int kCanonTile = 1024;   // items per counting thread
constexpr int kCanonThreads = 32;  // counting threads per CTA (256 counters each in shared memory)

__global__ void k_iota(int* p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = static_cast<int>(i);
}

// counts[d * ntiles + t] = items of tile t whose digit is d; the key of item
// i is key[perm[i]].
__global__ void __launch_bounds__(kCanonThreads) k_digit_count(const uint64_t* key, const int* perm, long long n,
                                                               int shift, int* counts, int ntiles) {
  __shared__ int c[kCanonThreads][256];
  const int t = blockIdx.x * kCanonThreads + threadIdx.x;
  int* my = c[threadIdx.x];
  for (int d = 0; d < 256; ++d) my[d] = 0;
  if (t < ntiles) {
    const long long i0 = (long long)t * kCanonTile, i1 = n < i0 + kCanonTile ? n : i0 + kCanonTile;
    for (long long i = i0; i < i1; ++i) ++my[(key[perm[i]] >> shift) & 255u];
    for (int d = 0; d < 256; ++d) counts[(long long)d * ntiles + t] = my[d];
  }
}

// Exclusive prefix sum of counts[0..m) in place, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_counts(int* counts, long long m) {
  __shared__ int warp_sum[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long base = 0; base < m; base += 1024) {
    const long long i = base + threadIdx.x;
    const int v = i < m ? counts[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = warp_sum[lane], xx = w;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, xx, o);
        if (lane >= o) xx += y;
      }
      warp_sum[lane] = xx - w;
    }
    __syncthreads();
    const long long excl = carry + warp_sum[warp] + (x - v);
    if (i < m) counts[i] = static_cast<int>(excl);
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kCanonThreads) k_digit_scatter(const uint64_t* key, const int* perm_in, long long n,
                                                                 int shift, const int* offsets, int ntiles,
                                                                 int* perm_out) {
  __shared__ int c[kCanonThreads][256];
  const int t = blockIdx.x * kCanonThreads + threadIdx.x;
  if (t >= ntiles) return;
  int* my = c[threadIdx.x];
  for (int d = 0; d < 256; ++d) my[d] = offsets[(long long)d * ntiles + t];
  const long long i0 = (long long)t * kCanonTile, i1 = n < i0 + kCanonTile ? n : i0 + kCanonTile;
  for (long long i = i0; i < i1; ++i) {
    const int p = perm_in[i];
    perm_out[my[(key[p] >> shift) & 255u]++] = p;
  }
}

__global__ void k_inverse(const int* perm, long long n, int* rank) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    rank[perm[i]] = static_cast<int>(i);
}

// dst[r * n + i] = src[r * ld + perm[i]] for rows r < rows
template <typename T>
__global__ void k_gather_rows(const T* src, long long ld, const int* perm, long long n, int rows, T* dst) {
  const long long total = n * rows;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / n, i = k % n;
    dst[k] = src[r * ld + perm[i]];
  }
}

template <typename T>
__global__ void k_store_rows(const T* src, long long n, int rows, T* dst, long long ld) {
  const long long total = n * rows;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / n, i = k % n;
    dst[r * ld + i] = src[k];
  }
}

__global__ void k_edge_keys(const int32_t* EU, const int32_t* EW, const int* rank, long long nE, uint64_t* K) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    const uint32_t a = static_cast<uint32_t>(rank[EU[e]]), b = static_cast<uint32_t>(rank[EW[e]]);
    K[e] = (static_cast<uint64_t>(a < b ? a : b) << 32) | (a < b ? b : a);
  }
}

__global__ void k_edge_store(const uint64_t* K, const int* perm, long long nE, int32_t* EU, int32_t* EW) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    const uint64_t k = K[perm[e]];
    EU[e] = static_cast<int32_t>(k >> 32);
    EW[e] = static_cast<int32_t>(k & 0xffffffffu);
  }
}

}  // namespace pc

using namespace pc;

namespace {

int grid_for(long long n) { return static_cast<int>(std::max<long long>(1, std::min<long long>(4096, (n + 255) / 256))); }

// Stable radix sort of perm (length n) by key words key_rows[0..words) (row
// 0 most significant), each row indexed by item.  perm and tmp hold n ints;
// counts holds 256 * tiles ints.
void sort_by_words(const uint64_t* const* key_rows, int words, long long n, int* perm, int* tmp, int* counts,
                   cudaStream_t s) {
  const int ntiles = static_cast<int>((n + kCanonTile - 1) / kCanonTile);
  const int cblocks = (ntiles + kCanonThreads - 1) / kCanonThreads;
  int* in = perm;
  int* out = tmp;
  for (int w = words - 1; w >= 0; --w) {
    for (int shift = 0; shift < 64; shift += 8) {
      k_digit_count<<<cblocks, kCanonThreads, 0, s>>>(key_rows[w], in, n, shift, counts, ntiles);
      k_scan_counts<<<1, 1024, 0, s>>>(counts, 256ll * ntiles);
      k_digit_scatter<<<cblocks, kCanonThreads, 0, s>>>(key_rows[w], in, n, shift, counts, ntiles, out);
      std::swap(in, out);
    }
  }
  // 8 passes per word: an even count, so the result is back in perm
}

}  // namespace

// Puts the context's result (coordinates, sign words, last-layer values,
// error estimates, edges) in canonical order.  Throws PcError on failure.
void pc_canonicalize(pc_ctx* c) {
  const long long nV = c->nV, nE = c->nE;
  if (nV <= 0) return;
  cudaStream_t s = c->stream;
  const long long n = std::max(nV, nE);
  const long long ntiles = (n + kCanonTile - 1) / kCanonTile;
  void* perm = ctx_alloc(c, sizeof(int) * n);
  void* tmp = ctx_alloc(c, sizeof(int) * n);
  void* counts = ctx_alloc(c, sizeof(int) * 256 * ntiles);
  void* rank = ctx_alloc(c, sizeof(int) * nV);
  void* keys = ctx_alloc(c, sizeof(uint64_t) * std::max(nE, 1ll));
  const int H = c->net.w[c->net.L];
  const size_t zs = c->net.precision == PC_PREC_FP64 ? 8 : 4;
  const size_t row_bytes = std::max<size_t>({8 * (size_t)c->net.D, 8 * (size_t)c->net.S, zs * H, 8});
  void* gath = ctx_alloc(c, row_bytes * nV);
  auto release = [&]() {
    ctx_free(c, perm);
    ctx_free(c, tmp);
    ctx_free(c, counts);
    ctx_free(c, rank);
    ctx_free(c, keys);
    ctx_free(c, gath);
  };
  if (!perm || !tmp || !counts || !rank || !keys || !gath) {
    release();
    throw PcError(PC_ERR_OOM, "canonical order: device allocation failed");
  }
  auto check = [&]() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      release();
      throw PcError(PC_ERR_CUDA, std::string("canonical order: ") + cudaGetErrorString(e));
    }
  };
  int* P = static_cast<int*>(perm);
  int* R = static_cast<int*>(rank);
  const long long ld = c->Vcap;
  // vertices by sign words
  const uint64_t* SIG = static_cast<const uint64_t*>(c->bufs.SIG);
  const uint64_t* rows[kMaxWords];
  for (int w = 0; w < c->net.S; ++w) rows[w] = SIG + (long long)w * ld;
  k_iota<<<grid_for(nV), 256, 0, s>>>(P, nV);
  sort_by_words(rows, c->net.S, nV, P, static_cast<int*>(tmp), static_cast<int*>(counts), s);
  check();
  k_inverse<<<grid_for(nV), 256, 0, s>>>(P, nV, R);
  // permute the per-vertex rows
  auto permute = [&](void* base, size_t elem, int nrows) {
    if (!base || nrows <= 0) return;
    const int g = grid_for(nV * nrows);
    if (elem == 8) {
      k_gather_rows<uint64_t><<<g, 256, 0, s>>>(static_cast<const uint64_t*>(base), ld, P, nV, nrows,
                                               static_cast<uint64_t*>(gath));
      k_store_rows<uint64_t><<<g, 256, 0, s>>>(static_cast<const uint64_t*>(gath), nV, nrows,
                                              static_cast<uint64_t*>(base), ld);
    } else {
      k_gather_rows<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(base), ld, P, nV, nrows,
                                               static_cast<uint32_t*>(gath));
      k_store_rows<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(gath), nV, nrows,
                                              static_cast<uint32_t*>(base), ld);
    }
  };
  permute(c->bufs.X, 8, c->net.D);
  permute(c->bufs.SIG, 8, c->net.S);
  permute(pc_make_state(c).Z[c->net.L - 1], zs, H);
  if (c->net.precision != PC_PREC_FP64) {
    permute(c->bufs.esc, 4, 1);
    permute(c->bufs.exc, 4, 1);
  }
  check();
  // edges: renumber, then sort by (smaller, larger)
  if (nE > 0) {
    int32_t* EU = static_cast<int32_t*>(c->bufs.E);
    int32_t* EW = EU + c->Ecap;
    uint64_t* K = static_cast<uint64_t*>(keys);
    k_edge_keys<<<grid_for(nE), 256, 0, s>>>(EU, EW, R, nE, K);
    k_iota<<<grid_for(nE), 256, 0, s>>>(P, nE);
    const uint64_t* krow[1] = {K};
    sort_by_words(krow, 1, nE, P, static_cast<int*>(tmp), static_cast<int*>(counts), s);
    k_edge_store<<<grid_for(nE), 256, 0, s>>>(K, P, nE, EU, EW);
    check();
  }
  c->launches += 2 + 24ll * c->net.S + 2 * (3 + 2 * (c->net.precision != PC_PREC_FP64)) + (nE > 0 ? 27 : 0);
  release();
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) throw PcError(PC_ERR_CUDA, std::string("canonical order: ") + cudaGetErrorString(e));
}
