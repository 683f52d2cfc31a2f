// k-cell counts of the extracted complex (pc_cell_counts): the k-faces of
// the polyhedral complex for k = 0..D by perturbation (Section 4.1), from
// which the number of regions (D-cells) and the Euler characteristic follow.
//
// A k-cell is named by its sign vector, which has D - k zeros.  The 1-cells
// are the edges (sign vector = join of the two vertices); the k-cells are
// obtained from the (k-1)-cells by setting one zero to + or - (a box facet's
// zero only to +, the inside), and one k-cell arises from several (k-1)-cells,
// so the candidates are deduplicated: every candidate is keyed by a 64-bit
// fingerprint of its full sign vector (XOR of per-word mixes, updated in O(1)
// for the changed word) and inserted into an open-addressing table with one
// 128-bit CAS of (fingerprint, candidate id); the winners are compacted into
// the next level's cells, and a check pass compares every other candidate's
// full sign vector with its winner's, word by word (a fingerprint collision
// is reported, never counted silently).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "pc_ctx.h"
#include "pc_device.cuh"

namespace pc {

__global__ void __launch_bounds__(1024) k_scan_counts(int* counts, long long m);  // pc_canon.cu

constexpr int kCellBlock = 1024;

// Candidate r of a cell (words c[0..S)): r-th (zero entry, sign) in entry
// order, + before -, a facet's zero only +.  Returns false past the last.
__device__ __forceinline__ bool cell_candidate(const uint64_t* c, int S, int P, int m, int r, int& wj,
                                               uint64_t& neww) {
  int k = 0;
  for (int w = 0; w < S; ++w) {
    uint64_t zm = zero_mask(c[w], w, P);
    while (zm) {
      const int bit = __ffsll((long long)zm) - 1;
      zm &= zm - 1;
      const int entry = 32 * w + bit / 2;
      const int nsg = entry < m ? 1 : 2;
      if (r < k + nsg) {
        wj = w;
        neww = (c[w] & ~(3ull << bit)) | ((r - k == 0 ? kPlus : kMinus) << bit);
        return true;
      }
      k += nsg;
    }
  }
  return false;
}

__device__ __forceinline__ uint64_t cell_hash(const uint64_t* c, int S) {
  uint64_t h = 0;
  for (int w = 0; w < S; ++w) h ^= word_hash(w, c[w]);
  return h;
}

// Level 1: the join of each edge's vertices, as cell words (cell-major).
__global__ void k_edge_cells(const uint64_t* SIG, long long ld, const int32_t* EU, const int32_t* EW, long long nE,
                             int S, uint64_t* cells) {
  const long long total = nE * S;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long e = k / S;
    const int w = static_cast<int>(k % S);
    cells[k] = SIG[(long long)w * ld + EU[e]] | SIG[(long long)w * ld + EW[e]];
  }
}

// Inserts every candidate of every parent cell (R per parent; R = 1 and
// identity = 1: the parent itself).  win[cid] = 1 for the inserted ones.
__global__ void k_cells_insert(const uint64_t* parents, long long np, int S, int P, int m, int R, int identity,
                               unsigned long long* table, long long tmask, int* win, int* err) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    uint64_t c[kMaxWords];
    for (int w = 0; w < S; ++w) c[w] = parents[p * S + w];
    const uint64_t h0 = cell_hash(c, S);
    for (int r = 0; r < R; ++r) {
      uint64_t h = h0;
      if (!identity) {
        int wj;
        uint64_t nw;
        if (!cell_candidate(c, S, P, m, r, wj, nw)) break;
        h = h0 ^ word_hash(wj, c[wj]) ^ word_hash(wj, nw);
      }
      if (h == kEmpty) h = kEmpty - 1;
      const unsigned long long cid = static_cast<unsigned long long>(p) * R + r;
      long long slot = static_cast<long long>(h & static_cast<uint64_t>(tmask));
      for (long long probes = 0;; ++probes) {
        if (probes > tmask) {
          atomicOr(err, 1);
          break;
        }
        unsigned long long ok, ov;
        cas128(table + 2 * slot, kEmpty, kEmpty, h, cid, ok, ov);
        if (ok == kEmpty) {
          win[cid] = 1;
          break;
        }
        if (ok == h) break;  // a duplicate (checked by k_cells_check)
        slot = (slot + 1) & tmask;
      }
    }
    if (!identity) {  // more zeros than R candidates: not a generic complex
      int wj;
      uint64_t nw;
      if (cell_candidate(c, S, P, m, R, wj, nw)) atomicOr(err, 2);
    }
  }
}

__device__ __forceinline__ void cand_words(const uint64_t* parents, int S, int P, int m, int R, int identity,
                                           unsigned long long cid, uint64_t* out) {
  const long long p = static_cast<long long>(cid / R);
  const int r = static_cast<int>(cid % R);
  for (int w = 0; w < S; ++w) out[w] = parents[p * S + w];
  if (!identity) {
    int wj;
    uint64_t nw;
    if (cell_candidate(out, S, P, m, r, wj, nw)) out[wj] = nw;
  }
}

// Every candidate that lost its insert equals its winner exactly.
__global__ void k_cells_check(const uint64_t* parents, long long np, int S, int P, int m, int R, int identity,
                              const unsigned long long* table, long long tmask, const int* win, int* err) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    uint64_t c[kMaxWords], o[kMaxWords];
    for (int w = 0; w < S; ++w) c[w] = parents[p * S + w];
    const uint64_t h0 = cell_hash(c, S);
    for (int r = 0; r < R; ++r) {
      uint64_t h = h0, mine[kMaxWords];
      for (int w = 0; w < S; ++w) mine[w] = c[w];
      if (!identity) {
        int wj;
        uint64_t nw;
        if (!cell_candidate(c, S, P, m, r, wj, nw)) break;
        h = h0 ^ word_hash(wj, c[wj]) ^ word_hash(wj, nw);
        mine[wj] = nw;
      }
      if (h == kEmpty) h = kEmpty - 1;
      const unsigned long long cid = static_cast<unsigned long long>(p) * R + r;
      if (win[cid]) continue;
      long long slot = static_cast<long long>(h & static_cast<uint64_t>(tmask));
      for (long long probes = 0; probes <= tmask; ++probes) {
        const unsigned long long key = table[2 * slot];
        if (key == kEmpty) {  // the winner must be in the table
          atomicOr(err, 4);
          break;
        }
        if (key == h) {
          cand_words(parents, S, P, m, R, identity, table[2 * slot + 1], o);
          for (int w = 0; w < S; ++w)
            if (o[w] != mine[w]) atomicOr(err, 4);
          break;
        }
        slot = (slot + 1) & tmask;
      }
    }
  }
}

__global__ void __launch_bounds__(kCellBlock) k_win_count(const int* win, long long n, int* counts, int nblocks) {
  const long long i = (long long)blockIdx.x * kCellBlock + threadIdx.x;
  const int x = __syncthreads_count(i < n && win[i]);
  if (threadIdx.x == 0) {
    counts[blockIdx.x] = x;
    if (blockIdx.x == 0) counts[nblocks] = 0;
  }
}

__global__ void __launch_bounds__(kCellBlock) k_win_gather(const uint64_t* parents, int S, int P, int m, int R,
                                                           int identity, const int* win, long long n,
                                                           const int* offsets, uint64_t* cells) {
  __shared__ int ws[32];
  const long long i = (long long)blockIdx.x * kCellBlock + threadIdx.x;
  const int f = (i < n && win[i]) ? 1 : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) ws[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    const int w = ws[lane];
    int x = w;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    ws[lane] = x - w;
  }
  __syncthreads();
  if (f) {
    const long long t = offsets[blockIdx.x] + ws[warp] + __popc(bal & ((1u << lane) - 1u));
    uint64_t o[kMaxWords];
    cand_words(parents, S, P, m, R, identity, static_cast<unsigned long long>(i), o);
    for (int w = 0; w < S; ++w) cells[t * S + w] = o[w];
  }
}

}  // namespace pc

using namespace pc;

namespace {

#define PC_CUDA_CELLS(call)                                                           \
  do {                                                                                \
    const cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) throw PcError(PC_ERR_CUDA, std::string("cell counts: ") + cudaGetErrorString(e_)); \
  } while (0)

int cgrid(long long n) { return static_cast<int>(std::max<long long>(1, std::min<long long>(8192, (n + 255) / 256))); }

}  // namespace

extern "C" pc_status pc_cell_counts(pc_ctx* c, int64_t* f_out, int n, int64_t* euler) {
  if (!c || !f_out) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  const int D = c->net.D;
  if (n < D + 1) return c->fail(PC_ERR_INVALID, "f_out needs D + 1 entries");
  const int S = c->net.S, P = c->net.P, m = c->net.m;
  const long long nV = c->nV, nE = c->nE;
  cudaStream_t s = c->stream;
  std::vector<void*> held;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = ctx_alloc(c, std::max<size_t>(bytes, 16));
    if (p) held.push_back(p);
    return p;
  };
  auto release = [&]() {
    for (void*& p : held) ctx_free(c, p);
    held.clear();
  };
  try {
    f_out[0] = nV;
    int64_t chi = nV;
    void* errp = alloc(sizeof(int));
    void* parents = alloc(sizeof(uint64_t) * S * std::max(nE, 1ll));
    if (!errp || !parents) throw PcError(PC_ERR_OOM, "cell counts: device allocation failed");
    PC_CUDA_CELLS(cudaMemsetAsync(errp, 0, sizeof(int), s));
    const int32_t* EU = static_cast<const int32_t*>(c->bufs.E);
    k_edge_cells<<<cgrid(nE * S), 256, 0, s>>>(static_cast<const uint64_t*>(c->bufs.SIG), c->Vcap, EU, EU + c->Ecap,
                                              nE, S, static_cast<uint64_t*>(parents));
    long long np = nE;
    for (int k = 1; k <= D; ++k) {
      const int identity = k == 1 ? 1 : 0;
      const int R = identity ? 1 : 2 * D;
      const long long ncand = std::max(np * R, 1ll);
      long long T = 64;
      while (T < 2 * ncand) T <<= 1;
      const int nblocks = static_cast<int>((ncand + kCellBlock - 1) / kCellBlock);
      void* table = alloc(16 * T);
      void* win = alloc(sizeof(int) * ncand);
      void* counts = alloc(sizeof(int) * (nblocks + 1));
      if (!table || !win || !counts) throw PcError(PC_ERR_OOM, "cell counts: device allocation failed");
      PC_CUDA_CELLS(cudaMemsetAsync(table, 0xff, 16 * T, s));
      PC_CUDA_CELLS(cudaMemsetAsync(win, 0, sizeof(int) * ncand, s));
      const uint64_t* par = static_cast<const uint64_t*>(parents);
      k_cells_insert<<<cgrid(np), 256, 0, s>>>(par, np, S, P, m, R, identity, static_cast<unsigned long long*>(table),
                                              T - 1, static_cast<int*>(win), static_cast<int*>(errp));
      k_cells_check<<<cgrid(np), 256, 0, s>>>(par, np, S, P, m, R, identity,
                                             static_cast<const unsigned long long*>(table), T - 1,
                                             static_cast<const int*>(win), static_cast<int*>(errp));
      k_win_count<<<nblocks, kCellBlock, 0, s>>>(static_cast<const int*>(win), ncand, static_cast<int*>(counts), nblocks);
      k_scan_counts<<<1, 1024, 0, s>>>(static_cast<int*>(counts), nblocks + 1);
      int nk = 0, err = 0;
      PC_CUDA_CELLS(cudaMemcpyAsync(&nk, static_cast<int*>(counts) + nblocks, sizeof(int), cudaMemcpyDeviceToHost, s));
      PC_CUDA_CELLS(cudaMemcpyAsync(&err, errp, sizeof(int), cudaMemcpyDeviceToHost, s));
      PC_CUDA_CELLS(cudaStreamSynchronize(s));
      if (err & 2) throw PcError(PC_ERR_DEGENERATE, "cell counts: a cell has more zeros than a generic complex");
      if (err) throw PcError(PC_ERR_PAIRING, "cell counts: fingerprint table overflow or collision");
      f_out[k] = nk;
      chi += (k % 2 == 0) ? nk : -static_cast<int64_t>(nk);
      if (k < D) {
        void* next = alloc(sizeof(uint64_t) * S * std::max<long long>(nk, 1));
        if (!next) throw PcError(PC_ERR_OOM, "cell counts: device allocation failed");
        k_win_gather<<<nblocks, kCellBlock, 0, s>>>(par, S, P, m, R, identity, static_cast<const int*>(win), ncand,
                                                   static_cast<const int*>(counts), static_cast<uint64_t*>(next));
        PC_CUDA_CELLS(cudaGetLastError());
        // the previous level's buffers are no longer needed
        parents = next;
        np = nk;
      }
      c->launches += 5 + (k < D);
    }
    PC_CUDA_CELLS(cudaStreamSynchronize(s));
    release();
    if (euler) *euler = chi;
    return PC_OK;
  } catch (const PcError& e) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    release();
    return c->fail(e.status, e.what());
  }
}
