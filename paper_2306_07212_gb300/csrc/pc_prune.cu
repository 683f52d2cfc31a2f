// Pruning during edge subdivision (Section 5.4.2; pc_options.prune), for
// extracting the level set of the output neuron without the rest of the
// complex.
//
// After each layer l but the last, every current vertex with an edge gets
// its signs w.r.t. all future neurons (layers l+1 .. L-1) from a forward pass
// at its coordinates (float-float, its error far inside the uncertainty band
// below): the stored activation pattern for layers <= l, the ReLU of the
// computed values beyond.  An edge whose two vertices have the same
// future signs is crossed by no future folded hyperplane (along the edge the
// next layer is affine, and so are the later ones while no earlier neuron
// splits it), so it cannot meet the output's zero set: it is dropped.  A
// value within 1e-9 of its sum of |terms| marks its vertex uncertain, and an
// uncertain vertex keeps its edges.  Edges are compacted stably, with their
// pairing records; the per-neuron counters of the next step read the pruned
// edge count.  Vertices stay in place during the extraction (a vertex without
// edges is classified but never split again) and the vertices without an
// edge are dropped once, after the last step (pc_prune_vertices), which gives
// the complex that pruning vertices after every layer would.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pc_ctx.h"
#include "pc_device.cuh"

namespace pc {

constexpr int kPruneWarps = 8;      // vertices in flight per CTA (one per warp)
constexpr int kCompactBlock = 1024; // items per block of the stable compaction

// Exclusive prefix sum of counts[0..m) in place, one CTA of 1024 threads (pc_canon.cu).
__global__ void __launch_bounds__(1024) k_scan_counts(int* counts, long long m);

__device__ __forceinline__ bool g_stopped(const Global* g) {  // once per CTA
  return __syncthreads_or(threadIdx.x == 0 && ((*(volatile const int*)&g->error & kErrFatal) ||
                                                *(volatile const int*)&g->halted_at >= 0)) != 0;
}

// used[v] = 1 for every endpoint of the edges present after layer l.
__global__ void k_mark_edge_ends(NetDesc net, State st, int l, unsigned char* used) {
  if (cta_stopped(st)) return;
  const Counters* c = st.cnt + net.off[l + 1];
  const long long nE = c->nE_before + c->nsplit + c->npairs;
  const long long nV = c->nV_before + c->nsplit;
  if (nE < 0 || nE > st.Ecap) return;  // k_edge_keep reports it
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    const int u = st.EU[e], w = st.EW[e];
    if (u >= 0 && u < nV) used[u] = 1;
    if (w >= 0 && w < nV) used[w] = 1;
  }
}

// Forward pass of vertex v (one per warp) through the rest of the net, for
// the vertices that still have an edge (used; the others are never read),
// in float-float arithmetic (Dot2 as in the polish: exact products by FMA,
// TwoSum of the running sum, error terms in a float; weights as (head,
// remainder) pairs, W^T layout so that the lanes' rows are contiguous).
// fut: Wf 32-bit words per vertex (bit f = 1 iff future neuron f is +);
// unc: 1 if a future value is within 1e-9 of its sum of |terms|.  The
// float-float error, ~(n u)^2 of that sum per layer (u = 2^-24; 1.5e-11 for
// 64 inputs), is far inside the band, so every sign outside it is the exact
// one, and a vertex with a value inside it keeps its edges.
__global__ void __launch_bounds__(32 * kPruneWarps) k_future_signs(NetDesc net, State st, int l, int mw, int Wf,
                                                                   const unsigned char* used, uint32_t* fut,
                                                                   unsigned char* unc) {
  extern __shared__ double psh[];
  if (cta_stopped(st)) return;
  const Counters* c = st.cnt + net.off[l + 1];
  const long long nV = c->nV_before + c->nsplit;
  if (nV < 0 || nV > st.Vcap) {
    if (threadIdx.x == 0) report_corrupt(st.g, 10, l, nV, st.Vcap, 0);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* buf = psh + (long long)warp * (2 * mw + Wf);
  float* fbuf = reinterpret_cast<float*>(buf);                  // a (hi, lo), next (hi, lo): 4 mw floats
  uint32_t* words = reinterpret_cast<uint32_t*>(buf + 2 * mw);  // Wf words (room for 2 Wf)
  const long long Vcap = st.Vcap;
  const int D = net.D, m = net.m, fbase = net.off[l + 1];
  for (long long v = (long long)blockIdx.x * kPruneWarps + warp; v < nV; v += (long long)gridDim.x * kPruneWarps) {
    if (!used[v]) continue;  // warp-uniform
    float* ahi = fbuf;
    float* alo = fbuf + mw;
    float* nhi = fbuf + 2 * mw;
    float* nlo = fbuf + 3 * mw;
    for (int w = lane; w < Wf; w += 32) words[w] = 0u;
    if (lane < D) {
      const double x = st.X[(long long)lane * Vcap + v];
      ahi[lane] = static_cast<float>(x);
      alo[lane] = static_cast<float>(x - static_cast<double>(ahi[lane]));
    }
    __syncwarp();
    int in = D;
    bool uncertain = false;
    for (int k = 0; k < net.L; ++k) {
      const int H = net.w[k + 1];
      const float2* Wt = net.WT2 + net.wofs[k];  // [in][H]
      for (int r = lane; r < H; r += 32) {
        const float2 bj = net.WT2[net.bofs[k] + r];
        float s = bj.x, e = bj.y, sc = fabsf(bj.x);
        for (int q = 0; q < in; ++q) {
          const float2 w = Wt[(long long)q * H + r];
          const float yh = ahi[q], yl = alo[q];
          const float pr = __fmul_rn(w.x, yh);
          float er = fmaf(w.x, yh, -pr);  // exact low part of the product
          er = fmaf(w.x, yl, er);         // cross terms of the low parts
          er = fmaf(w.y, yh, er);
          const float t = __fadd_rn(s, pr);  // TwoSum: t + its error is exact
          const float bb = __fsub_rn(t, s);
          e += __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(pr, bb)) + er;
          s = t;
          sc = fmaf(fabsf(w.x), fabsf(yh), sc);
        }
        const float zh = __fadd_rn(s, e);  // the float-float value zh + zl
        const float zl = __fsub_rn(e, __fsub_rn(zh, s));
        const int entry = m + net.off[k] + r;
        bool act;
        if (k <= l) {
          const uint64_t word = st.SIG[(long long)(entry >> 5) * Vcap + v];
          act = ((word >> (2 * (entry & 31))) & 3ull) == kPlus;
        } else {
          if (fabsf(zh) <= 1e-9f * sc) uncertain = true;
          const int f = net.off[k] + r - fbase;
          act = zh > 0.f;
          if (act) atomicOr(&words[f >> 5], 1u << (f & 31));
        }
        nhi[r] = act ? zh : 0.f;
        nlo[r] = act ? zl : 0.f;
      }
      __syncwarp();
      float* t0 = ahi; ahi = nhi; nhi = t0;
      float* t1 = alo; alo = nlo; nlo = t1;
      in = H;
    }
    const unsigned any_unc = __ballot_sync(0xffffffffu, uncertain);
    for (int w = lane; w < Wf; w += 32) fut[v * Wf + w] = words[w];
    if (lane == 0) unc[v] = any_unc ? 1 : 0;
    __syncwarp();
  }
}

// keep[e] = 1 unless both vertices of edge e have the same (certain) future signs.
__global__ void k_edge_keep(NetDesc net, State st, int l, int Wf, const uint32_t* fut, const unsigned char* unc,
                            int* keep) {
  if (cta_stopped(st)) return;
  const Counters* c = st.cnt + net.off[l + 1];
  const long long nE = c->nE_before + c->nsplit + c->npairs;
  const long long nV = c->nV_before + c->nsplit;
  if (nE < 0 || nE > st.Ecap) {
    if (threadIdx.x == 0) report_corrupt(st.g, 11, l, nE, st.Ecap, 0);
    return;
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    const int u = st.EU[e], w = st.EW[e];
    int k = 1;
    if (u >= 0 && u < nV && w >= 0 && w < nV && !unc[u] && !unc[w]) {
      k = 0;
      for (int q = 0; q < Wf; ++q)
        if (fut[(long long)u * Wf + q] != fut[(long long)w * Wf + q]) {
          k = 1;
          break;
        }
    }
    keep[e] = k;
  }
}

// Stable compaction, block part 1: counts[b] = kept items of block b
// (counts[nblocks] = 0, so the exclusive scan leaves the total there).
__global__ void __launch_bounds__(kCompactBlock) k_block_count(const Global* g, const int* flag, const long long* n_ptr,
                                                               const Counters* cn, int which, int* counts,
                                                               int nblocks) {
  if (g_stopped(g)) return;
  const long long n = which == 0 ? (cn->nE_before + cn->nsplit + cn->npairs) : *n_ptr;
  const long long i = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
  const int f = (i < n && flag[i]) ? 1 : 0;
  const int x = __syncthreads_count(f);
  if (threadIdx.x == 0) {
    counts[blockIdx.x] = x;
    if (blockIdx.x == 0) counts[nblocks] = 0;
  }
}

// Block part 2: item i (flag set) goes to offsets[block] + its rank among the
// block's flagged items, which keeps the order.
__device__ __forceinline__ int block_rank(int f, int* ws) {
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
  return ws[warp] + __popc(bal & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kCompactBlock) k_edge_scatter(State st, const Counters* cn, const int* keep,
                                                                const int* offsets, int32_t* tU, int32_t* tW,
                                                                int4* tL) {
  __shared__ int ws[32];
  if (g_stopped(st.g)) return;
  const long long nE = cn->nE_before + cn->nsplit + cn->npairs;
  const long long i = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
  const int f = (i < nE && keep[i]) ? 1 : 0;
  const int r = block_rank(f, ws);
  if (f) {
    const long long o = offsets[blockIdx.x] + r;
    tU[o] = st.EU[i];
    tW[o] = st.EW[i];
    if (st.deferred) tL[o] = st.vlist[i];
  }
}

// Copies the compacted edges back and records the pruned count for the
// next step (read by phase_classify as the edge count after this layer).
__global__ void k_edge_commit(State st, Counters* cn, const int* total, const int32_t* tU, const int32_t* tW,
                              const int4* tL) {
  if (g_stopped(st.g)) return;
  const long long n = *total;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    st.EU[e] = tU[e];
    st.EW[e] = tW[e];
    if (st.deferred) st.vlist[e] = tL[e];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) cn->pruned_e1 = n + 1;
}

__global__ void k_mark_used(const int32_t* EU, const int32_t* EW, long long nE, long long nV, int* used) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    const int u = EU[e], w = EW[e];
    if (u >= 0 && u < nV) used[u] = 1;
    if (w >= 0 && w < nV) used[w] = 1;
  }
}

__global__ void __launch_bounds__(kCompactBlock) k_vertex_scatter(const int* used, long long nV, const int* offsets,
                                                                  int* order, int* idx) {
  __shared__ int ws[32];
  const long long i = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
  const int f = (i < nV && used[i]) ? 1 : 0;
  const int r = block_rank(f, ws);
  if (f) {
    const long long o = offsets[blockIdx.x] + r;
    order[o] = static_cast<int>(i);
    idx[i] = static_cast<int>(o);
  }
}

template <typename T>
__global__ void k_take_rows(T* base, long long ld, int rows, const int* order, long long n, T* tmp) {
  const long long total = n * rows;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x)
    tmp[k] = base[(k / n) * ld + order[k % n]];
}

template <typename T>
__global__ void k_put_rows(T* base, long long ld, int rows, const T* tmp, long long n) {
  const long long total = n * rows;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x)
    base[(k / n) * ld + k % n] = tmp[k];
}

__global__ void k_remap_edges(int32_t* EU, int32_t* EW, long long nE, const int* idx) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    EU[e] = idx[EU[e]];
    EW[e] = idx[EW[e]];
  }
}

}  // namespace pc

using namespace pc;

namespace {

int grid_of(long long n) { return static_cast<int>(std::max<long long>(1, std::min<long long>(8192, (n + 255) / 256))); }

}  // namespace

// Upper bound of k_future_signs' dynamic shared memory (widths <= kMaxWidth,
// at most kMaxEntries future neurons), set once as its launch attribute.
cudaError_t pc_prune_set_attributes() {
  const int bytes = static_cast<int>(sizeof(double) * kPruneWarps * (2 * kMaxWidth + kMaxEntries / 32));
  return cudaFuncSetAttribute(k_future_signs, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Enqueues the edge pruning after layer l (l < L - 1) on the context's
// stream.  Temporaries are allocated here and freed in stream order.
void pc_prune_edges(pc_ctx* c, const State& st, int l) {
  const NetDesc& net = c->net;
  const int nf = net.N - net.off[l + 1];
  if (nf <= 0) return;
  const int Wf = (nf + 31) / 32;
  const long long V = c->Vcap, E = c->Ecap;
  const int nblocks = static_cast<int>((E + kCompactBlock - 1) / kCompactBlock);
  void* fut = ctx_alloc(c, sizeof(uint32_t) * Wf * V);
  void* unc = ctx_alloc(c, V);
  void* used = ctx_alloc(c, V);
  void* keep = ctx_alloc(c, sizeof(int) * E);
  void* counts = ctx_alloc(c, sizeof(int) * (nblocks + 1));
  void* tU = ctx_alloc(c, sizeof(int32_t) * E);
  void* tW = ctx_alloc(c, sizeof(int32_t) * E);
  void* tL = c->deferred ? ctx_alloc(c, sizeof(int4) * E) : nullptr;
  auto release = [&]() {
    ctx_free(c, fut);
    ctx_free(c, unc);
    ctx_free(c, used);
    ctx_free(c, keep);
    ctx_free(c, counts);
    ctx_free(c, tU);
    ctx_free(c, tW);
    ctx_free(c, tL);
  };
  if (!fut || !unc || !used || !keep || !counts || !tU || !tW || (c->deferred && !tL)) {
    release();
    throw PcError(PC_ERR_OOM, "pruning: device allocation failed");
  }
  cudaStream_t s = c->stream;
  Counters* cn = st.cnt + net.off[l + 1];
  const size_t smem = sizeof(double) * kPruneWarps * (2 * c->mw + Wf);
  const int vgrid = static_cast<int>(std::max<long long>(1, std::min<long long>(4ll * c->num_sms, (V + kPruneWarps - 1) / kPruneWarps)));
  cudaMemsetAsync(used, 0, V, s);
  k_mark_edge_ends<<<grid_of(E), 256, 0, s>>>(net, st, l, static_cast<unsigned char*>(used));
  k_future_signs<<<vgrid, 32 * kPruneWarps, smem, s>>>(net, st, l, c->mw, Wf, static_cast<const unsigned char*>(used),
                                                      static_cast<uint32_t*>(fut), static_cast<unsigned char*>(unc));
  k_edge_keep<<<grid_of(E), 256, 0, s>>>(net, st, l, Wf, static_cast<const uint32_t*>(fut),
                                         static_cast<const unsigned char*>(unc), static_cast<int*>(keep));
  k_block_count<<<nblocks, kCompactBlock, 0, s>>>(st.g, static_cast<const int*>(keep), nullptr, cn, 0,
                                                  static_cast<int*>(counts), nblocks);
  k_scan_counts<<<1, 1024, 0, s>>>(static_cast<int*>(counts), nblocks + 1);
  k_edge_scatter<<<nblocks, kCompactBlock, 0, s>>>(st, cn, static_cast<const int*>(keep),
                                                   static_cast<const int*>(counts), static_cast<int32_t*>(tU),
                                                   static_cast<int32_t*>(tW), static_cast<int4*>(tL));
  k_edge_commit<<<grid_of(E), 256, 0, s>>>(st, cn, static_cast<const int*>(counts) + nblocks,
                                           static_cast<const int32_t*>(tU), static_cast<const int32_t*>(tW),
                                           static_cast<const int4*>(tL));
  const cudaError_t e = cudaGetLastError();
  release();
  if (e != cudaSuccess) throw PcError(PC_ERR_CUDA, std::string("pruning: ") + cudaGetErrorString(e));
  c->launches += 7;
}

// After the last step: drops the vertices without an edge and renumbers the
// edges; coordinates, sign words, last-layer values and error estimates
// follow.  Updates c->nV.  Blocks until done.
void pc_prune_vertices(pc_ctx* c) {
  const long long nV = c->nV, nE = c->nE;
  if (nV <= 0) return;
  cudaStream_t s = c->stream;
  const int nblocks = static_cast<int>((nV + kCompactBlock - 1) / kCompactBlock);
  const int H = c->net.w[c->net.L];
  const size_t zs = c->net.precision == PC_PREC_FP64 ? 8 : 4;
  const size_t row_bytes = std::max<size_t>({8 * (size_t)c->net.D, 8 * (size_t)c->net.S, zs * H, 8});
  void* used = ctx_alloc(c, sizeof(int) * nV);
  void* counts = ctx_alloc(c, sizeof(int) * (nblocks + 1));
  void* order = ctx_alloc(c, sizeof(int) * nV);
  void* idx = ctx_alloc(c, sizeof(int) * nV);
  void* tmp = ctx_alloc(c, row_bytes * nV);
  void* total = ctx_alloc(c, sizeof(long long));
  auto release = [&]() {
    ctx_free(c, used);
    ctx_free(c, counts);
    ctx_free(c, order);
    ctx_free(c, idx);
    ctx_free(c, tmp);
    ctx_free(c, total);
  };
  if (!used || !counts || !order || !idx || !tmp || !total) {
    release();
    throw PcError(PC_ERR_OOM, "pruning: device allocation failed");
  }
  int32_t* EU = static_cast<int32_t*>(c->bufs.E);
  int32_t* EW = EU + c->Ecap;
  const State st = pc_make_state(c);
  cudaMemsetAsync(used, 0, sizeof(int) * nV, s);
  k_mark_used<<<grid_of(nE), 256, 0, s>>>(EU, EW, nE, nV, static_cast<int*>(used));
  // counts via the same block count, with n given directly
  long long hn = nV;
  cudaMemcpyAsync(total, &hn, sizeof(long long), cudaMemcpyHostToDevice, s);
  k_block_count<<<nblocks, kCompactBlock, 0, s>>>(st.g, static_cast<const int*>(used), static_cast<const long long*>(total),
                                                  nullptr, 1, static_cast<int*>(counts), nblocks);
  k_scan_counts<<<1, 1024, 0, s>>>(static_cast<int*>(counts), nblocks + 1);
  k_vertex_scatter<<<nblocks, kCompactBlock, 0, s>>>(static_cast<const int*>(used), nV, static_cast<const int*>(counts),
                                                     static_cast<int*>(order), static_cast<int*>(idx));
  int kept = 0;
  cudaMemcpyAsync(&kept, static_cast<int*>(counts) + nblocks, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    throw PcError(PC_ERR_CUDA, std::string("pruning: ") + cudaGetErrorString(e));
  }
  const long long ld = c->Vcap;
  const int* O = static_cast<const int*>(order);
  auto move = [&](void* base, size_t elem, int rows) {
    if (!base || rows <= 0 || kept <= 0) return;
    const int g = grid_of((long long)kept * rows);
    if (elem == 8) {
      k_take_rows<uint64_t><<<g, 256, 0, s>>>(static_cast<uint64_t*>(base), ld, rows, O, kept, static_cast<uint64_t*>(tmp));
      k_put_rows<uint64_t><<<g, 256, 0, s>>>(static_cast<uint64_t*>(base), ld, rows, static_cast<const uint64_t*>(tmp), kept);
    } else {
      k_take_rows<uint32_t><<<g, 256, 0, s>>>(static_cast<uint32_t*>(base), ld, rows, O, kept, static_cast<uint32_t*>(tmp));
      k_put_rows<uint32_t><<<g, 256, 0, s>>>(static_cast<uint32_t*>(base), ld, rows, static_cast<const uint32_t*>(tmp), kept);
    }
  };
  move(c->bufs.X, 8, c->net.D);
  move(c->bufs.SIG, 8, c->net.S);
  move(st.Z[c->net.L - 1], zs, H);
  if (c->net.precision != PC_PREC_FP64) {
    move(c->bufs.esc, 4, 1);
    move(c->bufs.exc, 4, 1);
  }
  k_remap_edges<<<grid_of(nE), 256, 0, s>>>(EU, EW, nE, static_cast<const int*>(idx));
  e = cudaGetLastError();
  release();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) throw PcError(PC_ERR_CUDA, std::string("pruning: ") + cudaGetErrorString(e));
  c->nV = kept;
  c->launches += 5 + 2 * (3 + 2 * (c->net.precision != PC_PREC_FP64));
}
