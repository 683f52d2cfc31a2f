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

// Every candidate that lost its insert equals its winner exactly.  owner
// (nullable, preset to -1): each candidate's winner id (its own if it won).
__global__ void k_cells_check(const uint64_t* parents, long long np, int S, int P, int m, int R, int identity,
                              const unsigned long long* table, long long tmask, const int* win, int* err,
                              long long* owner) {
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
      if (win[cid]) {
        if (owner) owner[cid] = static_cast<long long>(cid);
        continue;
      }
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
          if (owner) owner[cid] = static_cast<long long>(table[2 * slot + 1]);
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
                                                           const int* offsets, uint64_t* cells, long long* wpos) {
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
    if (wpos) wpos[i] = t;
  }
}

// ---------------------------------------------------------------------------
// Face poset (pc_build_poset): the cells of every level and, for each cell,
// its parents (the cells one level up that contain it) as CSR.

// Level 0: the vertices' sign words, cell-major.
__global__ void k_vertex_cells(const uint64_t* SIG, long long ld, long long nV, int S, uint64_t* cells) {
  const long long total = nV * S;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x)
    cells[k] = SIG[(long long)(k % S) * ld + k / S];
}

// inc[c * R + r] = the parent index of candidate r of cell c (owner -> the
// winner's position in the next level), -1 past the cell's candidates.
__global__ void k_cells_incidence(const long long* owner, const long long* wpos, long long n, long long* inc) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long o = owner[k];
    inc[k] = o >= 0 ? wpos[o] : -1;
  }
}

// Level 0 -> 1: each vertex's perturbations looked up among the edge cells
// (inserted with identity, so a slot's id is the edge index); a
// perturbation that is not an edge is an error (err bit 8).
__global__ void k_vertex_parents(const uint64_t* vcells, long long nV, int S, int P, int m, int R,
                                 const uint64_t* ecells, const unsigned long long* table, long long tmask,
                                 long long* inc, int* err) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nV; v += (long long)gridDim.x * blockDim.x) {
    uint64_t c[kMaxWords];
    for (int w = 0; w < S; ++w) c[w] = vcells[v * S + w];
    const uint64_t h0 = cell_hash(c, S);
    for (int r = 0; r < R; ++r) {
      int wj;
      uint64_t nw;
      inc[v * R + r] = -1;
      if (!cell_candidate(c, S, P, m, r, wj, nw)) continue;
      uint64_t h = h0 ^ word_hash(wj, c[wj]) ^ word_hash(wj, nw);
      if (h == kEmpty) h = kEmpty - 1;
      long long slot = static_cast<long long>(h & static_cast<uint64_t>(tmask));
      bool found = false;
      for (long long probes = 0; probes <= tmask; ++probes) {
        const unsigned long long key = table[2 * slot];
        if (key == kEmpty) break;
        if (key == h) {
          const long long e = static_cast<long long>(table[2 * slot + 1]);
          bool same = true;
          for (int w = 0; w < S; ++w) same = same && ecells[e * S + w] == (w == wj ? nw : c[w]);
          if (same) {
            inc[v * R + r] = e;
            found = true;
            break;
          }
        }
        slot = (slot + 1) & tmask;
      }
      if (!found) atomicOr(err, 8);
    }
  }
}

// CSR from the padded rows (R per cell, valid entries first): row lengths,
// then an exclusive scan in blocks of 1024 rows (block sums scanned by one
// CTA), then the copy.
__global__ void __launch_bounds__(1024) k_row_len(const long long* inc, long long n, int R, long long* rp,
                                                  long long* bsum) {
  __shared__ long long ws[32];
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  long long len = 0;
  if (i < n)
    while (len < R && inc[i * R + len] >= 0) ++len;
  // block-inclusive scan of len
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = len;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = ws[lane], xx = w;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, xx, o);
      if (lane >= o) xx += y;
    }
    ws[lane] = xx - w;
  }
  __syncthreads();
  if (i < n) rp[i + 1] = ws[warp] + x;  // inclusive within the block
  if (threadIdx.x == 1023) bsum[blockIdx.x] = ws[warp] + x;
}

__global__ void __launch_bounds__(1024) k_scan_bsum(long long* bsum, long long nb) {
  if (threadIdx.x != 0) return;
  long long run = 0;
  for (long long b = 0; b < nb; ++b) {
    const long long v = bsum[b];
    bsum[b] = run;
    run += v;
  }
}

__global__ void k_csr_fill(const long long* inc, long long n, int R, long long* rp, const long long* bsum,
                           long long* cols) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long end = rp[i + 1] + bsum[i / 1024];
    long long len = 0;
    while (len < R && inc[i * R + len] >= 0) ++len;
    const long long beg = end - len;
    for (long long q = 0; q < len; ++q) cols[beg + q] = inc[i * R + q];
  }
}

__global__ void k_csr_offsets(long long n, long long* rp, const long long* bsum) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    rp[i + 1] += bsum[i / 1024];
  if (blockIdx.x == 0 && threadIdx.x == 0) rp[0] = 0;
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

// The k-cells of every level by perturbation, deduplicated on the device.
// keep: the cells of every level (cell-major, S words each) and the parents
// of every level below D (CSR) are kept in the context (pc_build_poset).
void build_levels(pc_ctx* c, bool keep, int64_t* f_out, int64_t* euler) {
  const int D = c->net.D;
  const int S = c->net.S, P = c->net.P, m = c->net.m;
  const long long nV = c->nV, nE = c->nE;
  cudaStream_t s = c->stream;
  std::vector<void*> held;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = ctx_alloc(c, std::max<size_t>(bytes, 16));
    if (p) held.push_back(p);
    return p;
  };
  auto keep_alloc = [&](size_t bytes) -> void* {  // owned by the context's poset
    void* p = ctx_alloc(c, std::max<size_t>(bytes, 16));
    if (!p) throw PcError(PC_ERR_OOM, "poset: device allocation failed");
    c->poset_bufs.push_back(p);
    return p;
  };
  struct Release {
    std::vector<void*>& h;
    pc_ctx* c;
    ~Release() {
      for (void*& p : h) ctx_free(c, p);
    }
  } rel{held, c};
  f_out[0] = nV;
  int64_t chi = nV;
  void* errp = alloc(sizeof(int));
  void* parents = keep ? keep_alloc(sizeof(uint64_t) * S * std::max(nE, 1ll)) : alloc(sizeof(uint64_t) * S * std::max(nE, 1ll));
  if (!errp || !parents) throw PcError(PC_ERR_OOM, "cell counts: device allocation failed");
  PC_CUDA_CELLS(cudaMemsetAsync(errp, 0, sizeof(int), s));
  const int32_t* EU = static_cast<const int32_t*>(c->bufs.E);
  k_edge_cells<<<cgrid(nE * S), 256, 0, s>>>(static_cast<const uint64_t*>(c->bufs.SIG), c->Vcap, EU, EU + c->Ecap,
                                            nE, S, static_cast<uint64_t*>(parents));
  void* vcells = nullptr;
  if (keep) {
    vcells = keep_alloc(sizeof(uint64_t) * S * std::max(nV, 1ll));
    k_vertex_cells<<<cgrid(nV * S), 256, 0, s>>>(static_cast<const uint64_t*>(c->bufs.SIG), c->Vcap, nV, S,
                                                static_cast<uint64_t*>(vcells));
    c->poset_cells[0] = vcells;
    c->poset_n[0] = nV;
    c->poset_cells[1] = parents;  // the edges' cells, in edge order
    c->poset_n[1] = nE;
  }
  // CSR of the padded parent rows inc (n x R) of level lev
  auto to_csr = [&](const long long* inc, long long n, int R, int lev) {
    const long long nb = std::max(1ll, (n + 1023) / 1024);
    long long* rp = static_cast<long long*>(keep_alloc(sizeof(long long) * (n + 1)));
    long long* bsum = static_cast<long long*>(alloc(sizeof(long long) * nb));
    if (!bsum) throw PcError(PC_ERR_OOM, "poset: device allocation failed");
    PC_CUDA_CELLS(cudaMemsetAsync(rp, 0, sizeof(long long) * (n + 1), s));
    k_row_len<<<nb, 1024, 0, s>>>(inc, n, R, rp, bsum);
    k_scan_bsum<<<1, 32, 0, s>>>(bsum, nb);
    long long tot_blk = 0, last = 0;
    PC_CUDA_CELLS(cudaMemcpyAsync(&tot_blk, bsum + (nb - 1), sizeof(long long), cudaMemcpyDeviceToHost, s));
    PC_CUDA_CELLS(cudaMemcpyAsync(&last, rp + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    PC_CUDA_CELLS(cudaStreamSynchronize(s));
    const long long nnz = n ? tot_blk + last : 0;
    long long* cols = static_cast<long long*>(keep_alloc(sizeof(long long) * std::max(nnz, 1ll)));
    k_csr_fill<<<cgrid(n), 256, 0, s>>>(inc, n, R, rp, bsum, cols);
    k_csr_offsets<<<cgrid(n), 256, 0, s>>>(n, rp, bsum);
    PC_CUDA_CELLS(cudaGetLastError());
    c->poset_rp[lev] = rp;
    c->poset_cols[lev] = cols;
    c->poset_nnz[lev] = nnz;
    c->launches += 4;
  };
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
    long long* owner = nullptr;
    long long* wpos = nullptr;
    if (keep && !identity) {
      owner = static_cast<long long*>(alloc(sizeof(long long) * ncand));
      wpos = static_cast<long long*>(alloc(sizeof(long long) * ncand));
      if (!owner || !wpos) throw PcError(PC_ERR_OOM, "poset: device allocation failed");
      PC_CUDA_CELLS(cudaMemsetAsync(owner, 0xff, sizeof(long long) * ncand, s));
    }
    PC_CUDA_CELLS(cudaMemsetAsync(table, 0xff, 16 * T, s));
    PC_CUDA_CELLS(cudaMemsetAsync(win, 0, sizeof(int) * ncand, s));
    const uint64_t* par = static_cast<const uint64_t*>(parents);
    k_cells_insert<<<cgrid(np), 256, 0, s>>>(par, np, S, P, m, R, identity, static_cast<unsigned long long*>(table),
                                            T - 1, static_cast<int*>(win), static_cast<int*>(errp));
    k_cells_check<<<cgrid(np), 256, 0, s>>>(par, np, S, P, m, R, identity,
                                           static_cast<const unsigned long long*>(table), T - 1,
                                           static_cast<const int*>(win), static_cast<int*>(errp), owner);
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
    c->launches += 4;
    if (keep && identity) {
      // level 0 -> 1: the vertices' perturbations among the edges (all
      // distinct in a generic complex, so a slot's id is the edge index)
      if (nk != nE) throw PcError(PC_ERR_DEGENERATE, "poset: two edges have the same sign vector");
      const int Rv = 2 * D;
      long long* inc = static_cast<long long*>(alloc(sizeof(long long) * std::max(nV * Rv, 1ll)));
      if (!inc) throw PcError(PC_ERR_OOM, "poset: device allocation failed");
      k_vertex_parents<<<cgrid(nV), 256, 0, s>>>(static_cast<const uint64_t*>(vcells), nV, S, P, m, Rv, par,
                                                static_cast<const unsigned long long*>(table), T - 1, inc,
                                                static_cast<int*>(errp));
      PC_CUDA_CELLS(cudaMemcpyAsync(&err, errp, sizeof(int), cudaMemcpyDeviceToHost, s));
      PC_CUDA_CELLS(cudaStreamSynchronize(s));
      if (err) throw PcError(PC_ERR_PAIRING, "poset: a perturbed vertex is not an edge");
      to_csr(inc, nV, Rv, 0);
      c->launches += 1;
      continue;  // level 1 stays the edges' cells
    }
    if (k < D || keep) {
      void* next = keep ? keep_alloc(sizeof(uint64_t) * S * std::max<long long>(nk, 1))
                        : alloc(sizeof(uint64_t) * S * std::max<long long>(nk, 1));
      if (!next) throw PcError(PC_ERR_OOM, "cell counts: device allocation failed");
      k_win_gather<<<nblocks, kCellBlock, 0, s>>>(par, S, P, m, R, identity, static_cast<const int*>(win), ncand,
                                                 static_cast<const int*>(counts), static_cast<uint64_t*>(next), wpos);
      PC_CUDA_CELLS(cudaGetLastError());
      c->launches += 1;
      if (keep && !identity) {
        long long* inc = static_cast<long long*>(alloc(sizeof(long long) * ncand));
        if (!inc) throw PcError(PC_ERR_OOM, "poset: device allocation failed");
        k_cells_incidence<<<cgrid(ncand), 256, 0, s>>>(owner, wpos, ncand, inc);
        to_csr(inc, np, R, k - 1);
        c->poset_cells[k] = next;
        c->poset_n[k] = nk;
        c->launches += 1;
      }
      parents = next;
      np = nk;
    }
  }
  PC_CUDA_CELLS(cudaStreamSynchronize(s));
  if (euler) *euler = chi;
  if (keep) c->poset_levels = D + 1;
}

}  // namespace

void pc_poset_release(pc_ctx* c) {
  for (void*& p : c->poset_bufs) ctx_free(c, p);
  c->poset_bufs.clear();
  c->poset_levels = 0;
}

extern "C" pc_status pc_cell_counts(pc_ctx* c, int64_t* f_out, int n, int64_t* euler) {
  if (!c || !f_out) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (n < c->net.D + 1) return c->fail(PC_ERR_INVALID, "f_out needs D + 1 entries");
  try {
    build_levels(c, false, f_out, euler);
    return PC_OK;
  } catch (const PcError& e) {
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    return c->fail(e.status, e.what());
  }
}

extern "C" pc_status pc_build_poset(pc_ctx* c) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  pc_poset_release(c);
  int64_t f[kMaxD + 1], chi = 0;
  try {
    build_levels(c, true, f, &chi);
    return PC_OK;
  } catch (const PcError& e) {
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    pc_poset_release(c);
    return c->fail(e.status, e.what());
  }
}

extern "C" pc_status pc_poset_level(pc_ctx* c, int k, int64_t* n_cells, int64_t* n_parents, uint64_t* cells,
                                    int64_t* row_ptr, int64_t* parents) {
  if (!c) return PC_ERR_INVALID;
  if (c->poset_levels == 0 || !c->have_result) return c->fail(PC_ERR_INVALID, "no poset: call pc_build_poset");
  if (k < 0 || k >= c->poset_levels) return c->fail(PC_ERR_INVALID, "level out of range");
  const int D = c->net.D, S = c->net.S;
  const long long n = c->poset_n[k], nnz = k < D ? c->poset_nnz[k] : 0;
  if (n_cells) *n_cells = n;
  if (n_parents) *n_parents = nnz;
  cudaError_t e = cudaSuccess;
  if (cells && n) e = cudaMemcpyAsync(cells, c->poset_cells[k], sizeof(uint64_t) * S * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && row_ptr && k < D)
    e = cudaMemcpyAsync(row_ptr, c->poset_rp[k], sizeof(long long) * (n + 1), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && parents && k < D && nnz)
    e = cudaMemcpyAsync(parents, c->poset_cols[k], sizeof(long long) * nnz, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c->fail(PC_ERR_CUDA, cudaGetErrorString(e));
  return PC_OK;
}
