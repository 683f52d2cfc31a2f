// The per-neuron steps of edge subdivision (Section 4.2) as device functions.
//
// A layer l (neurons i = 0 .. H-1, global index n = off_l + i, sign entry
// e = m + n) runs as
//
//   phase_decide   (layer start, once) every value z_j of every current
//       vertex gets its final sign: an exact zero is a genericity violation
//       (counted, taken as +); in mixed precision a |z_j| within kappa times
//       its FP32 error estimate is re-decided in FP64 at the exact vertex.
//   phase_scan0    (layer start, once) step (3) for neuron 0: the edges whose
//       endpoints have opposite signs are listed as (edge, V+, V-).
//   phase_step     (once per neuron, one grid-wide synchronisation each)
//       steps (4) + (5) for the listed splitting edges of neuron i: new
//       vertex by interpolation (FP64 t and coordinates), the edge split into
//       E+ and E-, the parent 2-faces paired in a hash table; and, looking
//       ahead, step (3) for neuron i + 1: the warp that splits an edge
//       classifies its two halves and the intersecting edges it creates, the
//       edge scan classifies every other edge.  So each step starts with its
//       splitting edges listed and counted, and the capacity check happens
//       before any write.
//   phase_pack     (layer end, once) the layer's sign codes of every vertex
//       are packed into the sign words from the signs of its values.
//
// During a layer the sign of a vertex w.r.t. a neuron j of the layer is the
// sign of its stored value z_j (0 exactly on the folded hyperplane); the
// values are made consistent with that rule when they are created, so the
// packed codes equal what step (2) decides.  The sign words hold the earlier
// layers' entries; a new vertex's words are written complete (earlier layers
// from its edge's endpoints, this layer from the values) when it is created.
//
// A new vertex whose value for a later neuron of the layer is within the FP32
// filter is re-decided in FP64 by its CTA right after it is created, before
// anything reads that sign (the round's flagged vertices of a CTA together).
#pragma once

#include "pc_device.cuh"
#include "pc_newton.cuh"

namespace pc {

constexpr int kPairCap = 1024;         // intersecting edges a CTA buffers before it appends them
constexpr int kLaCap = 1024;           // look-ahead list entries a CTA buffers
constexpr int kPendCap = 2 * kBlock;   // vertices a CTA queues for an FP64 re-decision

struct Smem {
  long long pend[kPendCap];
  int4 pairs[kPairCap];                // (v_a, v_b, zero ordinals, neuron + 1)
  unsigned char pnext[kPairCap];       // bit 0: v_a is - at the next neuron, bit 1: v_b is -
  int4 la[kLaCap];                     // split halves that split again at the next neuron
  int npairs;
  int npairla;                         // buffered pairs that split at the next neuron
  int nla;
  int cursor;
  int npend;
  int wcnt[kWarps];
  int use_smem;
  long long pbase, lbase, sbase;
  int zlist[kWarps][16];
  float nrl[3 * kMaxWidth];            // the layer's per-neuron norms (NetDesc::nrm)
  int nrl_layer;                       // layer staged in nrl, -1: none
  long long acc[4];
};

template <typename ZT>
__device__ __forceinline__ ZT tiny_value() {
  return ZT(1e-30);
}

// bit 2k of the result = bit k of m
__device__ __forceinline__ uint64_t spread_even(uint32_t m) {
  uint64_t x = m;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

// Bits of word w that hold entries < e_end.
__device__ __forceinline__ uint64_t entries_below(int w, int e_end) {
  const int cnt = e_end - 32 * w;
  if (cnt <= 0) return 0ull;
  if (cnt >= 32) return ~0ull;
  return (1ull << (2 * cnt)) - 1ull;
}

// Vertex and edge counts at the start of step n.
__device__ __forceinline__ bool step_counts(const State& st, int n, long long& nV, long long& nE) {
  const Counters* prev = st.cnt + n;
  nV = prev->nV_before + prev->nsplit;
  nE = prev->pruned_e1 > 0 ? prev->pruned_e1 - 1 : prev->nE_before + prev->nsplit + prev->npairs;
  return nV >= 0 && nV <= st.Vcap && nE >= 0 && nE <= st.Ecap;
}

__device__ __forceinline__ void set_flag(uint32_t* f, long long e) {
  atomicOr(f + (e >> 5), 1u << (e & 31));
}

// Appends this lane's `c` (0..2) list entries with one atomic per warp; all
// lanes must call it.
__device__ __forceinline__ void warp_append(int c, const int4* ent, int4* list, uint32_t* flags, long long* counter) {
  const int lane = threadIdx.x & 31;
  int x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  const int tot = __shfl_sync(0xffffffffu, x, 31);
  if (tot == 0) return;
  long long base = 0;
  if (lane == 31) base = atomic_add_ll(counter, (long long)tot);
  base = __shfl_sync(0xffffffffu, base, 31) + (x - c);
  for (int t = 0; t < c; ++t) {
    list[base + t] = ent[t];
    set_flag(flags, ent[t].x);
  }
}

// ---------------------------------------------------------------------------
// FP64 re-decision of the values z_j, j >= j_from, of layer l that lie within
// the FP32 filter, for a batch of P vertices at once (the CTA's queued new
// vertices).  Each vertex's layer-l values are evaluated at its exact position:
// a forward pass in float64 from its stored coordinates through layers 0..l
// on its own piece (activation pattern = its sign words; gradients in float32,
// forward mode), then one Newton step on its zero set among the entries
// < e_end moves every value to the exact vertex, z + grad . dx (the step is
// small, so the float32 gradient adds only ~1e-7 of it).  Each filtered value
// is written back with its FP64 sign.  The forward pass runs over all
// (vertex, neuron) pairs of the batch together, tpr threads per pair (a
// function of the layer width alone, so results do not depend on how the
// vertices are batched), so the batch costs one chain of per-layer latency
// instead of one per vertex.
// Workspace (dynamic shared memory), rd_layout(P, mw, D, S) bytes:
struct RdLayout {
  size_t a, an, A, gv, dlt, sig, J, Jn, sc, zl, nz, ok, total;
};
__host__ __device__ inline RdLayout rd_layout(int P, int mw, int D, int S) {
  RdLayout r{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) / 16 * 16;
    return at;
  };
  r.a = take((size_t)P * mw * 8);       // activations (float64) [P][mw]
  r.an = take((size_t)P * mw * 8);      // next layer's
  r.A = take((size_t)P * D * D * 8);    // Newton rows [P][D][D]
  r.gv = take((size_t)P * D * 8);       // their values [P][D]
  r.dlt = take((size_t)P * D * 8);      // Newton steps [P][D]
  r.sig = take((size_t)P * S * 8);      // sign words [P][S]
  r.J = take((size_t)P * mw * D * 4);   // gradients (float) [P][mw][D]
  r.Jn = take((size_t)P * mw * D * 4);
  r.sc = take((size_t)P * mw * 4);      // sums of |terms| of layer l [P][mw]
  r.zl = take((size_t)P * D * 4);       // zero entries [P][D]
  r.nz = take((size_t)P * 4);           // zero entries found
  r.ok = take((size_t)P * 4);           // Newton step taken
  r.total = o;
  return r;
}
constexpr int kRdSmemBudget = 48 * 1024;  // shared memory for a batch
constexpr int kRdSmemMax = 64 * 1024;     // launch attribute of the kernels that hold it

// Vertices per batch: all warps' new vertices of a round (kWarps), fewer
// when the workspace would exceed the budget (wide layers, large D).
__host__ inline int rd_batch_size(int mw, int D, int S) {
  int P = kWarps;
  while (P > 1 && rd_layout(P, mw, D, S).total > (size_t)kRdSmemBudget) --P;
  return P;
}

template <typename ZT>
__device__ void redecide_batch(const NetDesc& net, const State& st, const long long* vs, int P, int l,
                                            int e_end, int j_from, int mw, unsigned char* ws) {
  const int D = net.D, S = net.S, m = net.m;
  const long long Vcap = st.Vcap;
  const RdLayout L = rd_layout(P, mw, D, S);
  double* a = reinterpret_cast<double*>(ws + L.a);
  double* an = reinterpret_cast<double*>(ws + L.an);
  double* A = reinterpret_cast<double*>(ws + L.A);
  double* gv = reinterpret_cast<double*>(ws + L.gv);
  double* dlt = reinterpret_cast<double*>(ws + L.dlt);
  uint64_t* sig = reinterpret_cast<uint64_t*>(ws + L.sig);
  float* J = reinterpret_cast<float*>(ws + L.J);
  float* Jn = reinterpret_cast<float*>(ws + L.Jn);
  float* sc = reinterpret_cast<float*>(ws + L.sc);
  int* zl = reinterpret_cast<int*>(ws + L.zl);
  int* nzs = reinterpret_cast<int*>(ws + L.nz);
  int* oks = reinterpret_cast<int*>(ws + L.ok);
  for (int t = threadIdx.x; t < P * S; t += blockDim.x) {
    const int q = t / S, w = t - q * S;
    sig[t] = st.SIG[(long long)w * Vcap + vs[q]];
  }
  for (int t = threadIdx.x; t < P * D; t += blockDim.x) {
    const int q = t / D, d = t - q * D;
    a[q * mw + d] = st.X[(long long)d * Vcap + vs[q]];
    for (int dd = 0; dd < D; ++dd) J[(q * mw + d) * D + dd] = d == dd ? 1.f : 0.f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < P; q += blockDim.x) {  // zero set among the entries < e_end
    int nz = 0;
    for (int w = 0; w < S; ++w) {
      uint64_t zm = zero_mask(sig[q * S + w], w, e_end);
      while (zm) {
        const int bit = __ffsll((long long)zm) - 1;
        if (nz < D) zl[q * D + nz] = w * 32 + bit / 2;
        ++nz;
        zm &= zm - 1;
      }
    }
    nzs[q] = nz;
  }
  __syncthreads();
  int in = D;
  for (int k = 0; k <= l; ++k) {
    const int H = net.w[k + 1];
    const double* W = net.W64 + net.wofs[k];  // [H][in]
    const float* W32 = net.W32 + net.wofs[k];
    const double* b = net.W64 + net.bofs[k];
    // tpr (threads per pair) depends on H only, so each value's summation
    // order, and with it the FP64 result, is the same in any batch
    const int pairs = P * H;
    int tpr = 16;
    while (tpr > 1 && H * tpr > (int)blockDim.x) tpr >>= 1;
    const int per = blockDim.x / tpr;
    for (int p0 = 0; p0 < pairs; p0 += per) {
      const int pr = p0 + threadIdx.x / tpr, s = threadIdx.x % tpr;
      const bool valid = pr < pairs;
      const int q = valid ? pr / H : 0, r = valid ? pr - q * H : 0;
      double acc = 0.0;
      float scl = 0.f, jd[kMaxD];
#pragma unroll
      for (int dd = 0; dd < kMaxD; ++dd) jd[dd] = 0.f;
      if (valid) {
        const double* wr = W + (long long)r * in;
        const float* wr32 = W32 + (long long)r * in;
        const double* aq = a + q * mw;
        const float* Jq = J + q * mw * D;
        for (int c = s; c < in; c += tpr) {
          const double av = aq[c];
          acc = fma(wr[c], av, acc);
          const float w32 = wr32[c];
          scl = fmaf(fabsf(w32), fabsf(static_cast<float>(av)), scl);
#pragma unroll
          for (int dd = 0; dd < kMaxD; ++dd)
            if (dd < D) jd[dd] = fmaf(w32, Jq[c * D + dd], jd[dd]);
        }
      }
      for (int o = tpr >> 1; o > 0; o >>= 1) {  // the tpr lanes of a pair are aligned
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        scl += __shfl_xor_sync(0xffffffffu, scl, o);
#pragma unroll
        for (int dd = 0; dd < kMaxD; ++dd) jd[dd] += __shfl_xor_sync(0xffffffffu, jd[dd], o);
      }
      if (valid && s == 0) {
        const double z = acc + b[r];
        const int entry = m + net.off[k] + r;
        const int nzc = nzs[q] < D ? nzs[q] : D;
        for (int qq = 0; qq < nzc; ++qq)
          if (zl[q * D + qq] == entry) {
            gv[q * D + qq] = z;
            for (int dd = 0; dd < D; ++dd) A[(q * D + qq) * D + dd] = jd[dd];
          }
        if (k < l) {
          const bool act = ((sig[q * S + (entry >> 5)] >> (2 * (entry & 31))) & 3ull) == kPlus;
          an[q * mw + r] = act ? z : 0.0;
          for (int dd = 0; dd < D; ++dd) Jn[(q * mw + r) * D + dd] = act ? jd[dd] : 0.f;
        } else {
          an[q * mw + r] = z;
          sc[q * mw + r] = scl + fabsf(static_cast<float>(b[r]));
          for (int dd = 0; dd < D; ++dd) Jn[(q * mw + r) * D + dd] = jd[dd];
        }
      }
    }
    __syncthreads();
    double* t0 = a; a = an; an = t0;
    float* t1 = J; J = Jn; Jn = t1;
    in = H;
  }
  for (int q = threadIdx.x; q < P; q += blockDim.x) {  // the Newton step of each vertex
    int* zq = zl + q * D;
    const int nzc = nzs[q] < D ? nzs[q] : D;
    if (net.fA != nullptr)
      for (int qq = 0; qq < nzc; ++qq) domain_facet_rows(net, st, vs[q], zq, nzc, qq, A + q * D * D, gv + q * D);
    NewtonOut o{};
    newton_solve(net, st, vs[q], zq, nzs[q], A + q * D * D, gv + q * D, o);
    oks[q] = o.ok;
    for (int d = 0; d < D; ++d) dlt[q * D + d] = o.ok ? o.dlt[d] : 0.0;
  }
  __syncthreads();
  // layer l's values (a), gradients (J) and sums of |terms| (sc): decide
  const int H = net.w[l + 1], n0 = net.off[l];
  ZT* Z = static_cast<ZT*>(st.Z[l]);
  const int nj = H - j_from;
  for (int t = threadIdx.x; t < P * nj; t += blockDim.x) {
    const int q = t / nj, j = j_from + (t - q * nj);
    const long long v = vs[q];
    const float z32 = static_cast<float>(Z[(long long)j * Vcap + v]);
    const float est = net.nrm[3 * (n0 + j)] * st.esc[v] + 2.9802322e-8f * net.nrm[3 * (n0 + j) + 1];
    if (!(fabsf(z32) <= net.kappa_sel * est)) continue;
    double zs = a[q * mw + j];
    if (oks[q])
      for (int d = 0; d < D; ++d) zs += static_cast<double>(J[(q * mw + j) * D + d]) * dlt[q * D + d];
    const bool und = !oks[q] || fabs(zs) <= 1e-12 * sc[q * mw + j];
    const bool minus = zs < 0.0;
    if (!(fabsf(z32) <= net.kappa * est)) {  // audit band: record a wrong FP32 sign, change nothing
      if ((z32 < 0.f) != minus && !und) {
        atomicAdd(&st.g->missed, 1);
        atomicMax(&st.g->missed_margin_bits, __float_as_int(fabsf(z32) / est));
      }
      continue;
    }
    ZT zz = static_cast<ZT>(zs);
    if (!minus && !(zz > ZT(0))) zz = tiny_value<ZT>();
    if (minus && !(zz < ZT(0))) zz = -tiny_value<ZT>();
    Z[(long long)j * Vcap + v] = zz;
    atomic_add_ll(&st.cnt[n0 + j + 1].nfilter, 1ll);
    if (und) atomic_add_ll(&st.cnt[n0 + j + 1].nundecided, 1ll);
    if ((z32 < 0.f) != minus) {  // the FP32 sign was wrong: how close to the filter's edge was it?
      atomicAdd(&st.g->flips, 1);
      atomicMax(&st.g->flip_margin_bits, __float_as_int(est > 0.f ? fabsf(z32) / est : 0.f));
    }
  }
  __syncthreads();
}

// Re-decides the CTA's queued vertices in batches of net.rd_batch and empties
// the queue.
template <typename ZT>
__device__ void drain_pending(const NetDesc& net, const State& st, int l, int e_end, int j_from, int mw, double* ws,
                              Smem& sm) {
  const int np = sm.npend;
  for (int q0 = 0; q0 < np; q0 += net.rd_batch) {
    const int P = np - q0 < net.rd_batch ? np - q0 : net.rd_batch;
    redecide_batch<ZT>(net, st, sm.pend + q0, P, l, e_end, j_from, mw, reinterpret_cast<unsigned char*>(ws));
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.npend = 0;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Layer start, step (2) for every current vertex and every neuron of the
// layer (values from the layer-start product, step (1)).
template <typename ZT, bool MIXED>
__device__ __noinline__ void phase_decide(const NetDesc& net, const State& st, int l, Smem& sm, double* ws, int mw) {
  const int n0 = net.off[l], H = net.w[l + 1];
  long long nV, nE;
  if (!step_counts(st, n0, nV, nE)) {
    if (threadIdx.x == 0) report_corrupt(st.g, 2, n0, nV, nE, st.Vcap);
    return;
  }
  const long long Vcap = st.Vcap;
  ZT* Z = static_cast<ZT*>(st.Z[l]);
  if (threadIdx.x == 0) sm.npend = 0;
  __syncthreads();
  const long long G = gridDim.x;
  for (long long round = 0; round * G * kBlock < nV; ++round) {
    const long long v = (round * G + blockIdx.x) * kBlock + threadIdx.x;
    if (v < nV) {
      bool filt = false;
      const float esc = MIXED ? st.esc[v] : 0.f;
      for (int j = 0; j < H; ++j) {
        ZT z = Z[(long long)j * Vcap + v];
        if (z == ZT(0)) {  // on a folded hyperplane it was not created on: not generic
          z = tiny_value<ZT>();
          Z[(long long)j * Vcap + v] = z;
          atomic_add_ll(&st.cnt[n0 + j + 1].ndegenerate, 1ll);
        }
        if (MIXED)
          filt = filt || fabsf(static_cast<float>(z)) <=
                             net.kappa_sel * (net.nrm[3 * (n0 + j)] * esc + 2.9802322e-8f * net.nrm[3 * (n0 + j) + 1]);
      }
      if (filt) sm.pend[atomicAdd(&sm.npend, 1)] = v;
    }
    if (MIXED) {
      __syncthreads();
      if (sm.npend > kPendCap - kBlock) drain_pending<ZT>(net, st, l, net.m + n0, 0, mw, ws, sm);
    }
  }
  if (MIXED) {
    __syncthreads();
    drain_pending<ZT>(net, st, l, net.m + n0, 0, mw, ws, sm);
  }
}

// ---------------------------------------------------------------------------
// Step (3) for one neuron over the edges [0, nE): an edge splits iff its
// endpoints' values in zrow have opposite signs.  Edges flagged in fcur are
// skipped (they split in the current step, whose warps classify their
// halves); fcur is cleared on the way.  classify = false only clears.  A CTA
// takes 2048 consecutive edges per iteration (one 128-edge tile per warp,
// CTAs round-robin) and reserves its list entries with one atomic.
// The flag word and the four edges (endpoint pairs) of one lane of a tile.
struct ScanTile {
  uint32_t fw;
  int4 eu, ew;
  int nvalid;
};

// nE may be the edge capacity (a load issued before the count is known):
// scan_edges takes the valid edges from the actual count.
__device__ __forceinline__ ScanTile scan_load(const State& st, const uint32_t* fcur, long long idx0, long long nE,
                                              bool classify) {
  ScanTile T;
  T.fw = (fcur != nullptr && idx0 < nE) ? fcur[idx0 >> 5] : 0u;
  T.eu = make_int4(0, 0, 0, 0);
  T.ew = make_int4(0, 0, 0, 0);
  T.nvalid = 0;
  if (classify && idx0 < nE) {
    T.nvalid = nE - idx0 >= 4 ? 4 : int(nE - idx0);
    if (T.nvalid == 4) {
      T.eu = *reinterpret_cast<const int4*>(st.EU + idx0);
      T.ew = *reinterpret_cast<const int4*>(st.EW + idx0);
    } else {
      int* pu = &T.eu.x;
      int* pw = &T.ew.x;
      for (int q = 0; q < T.nvalid; ++q) {
        pu[q] = st.EU[idx0 + q];
        pw[q] = st.EW[idx0 + q];
      }
    }
  }
  return T;
}

__device__ __forceinline__ long long scan_first_idx0() {
  return (long long)blockIdx.x * (4ll * kBlock) + (threadIdx.x >> 5) * 128 + 4 * (threadIdx.x & 31);
}

// first: this lane's part of the CTA's first iteration (scan_load at
// scan_first_idx0()), loaded by the caller early.  The entries go to the
// CTA's look-ahead buffer sm.la while it has room (the caller flushes it),
// else straight to the list with one reservation per CTA iteration.
template <typename ZT>
__device__ void scan_edges(const State& st, const ZT* zrow, long long nE, long long nV, uint32_t* fcur,
                           bool classify, int4* lnext, uint32_t* fnext, long long* counter, int n, Smem& sm,
                           const ScanTile& first) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long G = gridDim.x;
  constexpr long long kSpan = 4ll * kBlock;
  const long long iters = (nE + kSpan * G - 1) / (kSpan * G);
  // the next iteration's flags and endpoints are loaded while this one is classified
  ScanTile nxt = first;
  for (long long it = 0; it < iters; ++it) {
    const long long idx0 = (it * G + blockIdx.x) * kSpan + warp * 128 + 4 * lane;
    const ScanTile T = nxt;
    if (it + 1 < iters) nxt = scan_load(st, fcur, idx0 + kSpan * G, nE, classify);
    const int nvalid = idx0 >= nE ? 0 : (nE - idx0 >= 4 ? 4 : int(nE - idx0));
    const uint32_t skip = (T.fw >> (idx0 & 31)) & 0xFu;
    if (fcur != nullptr) {
      __syncwarp();
      if ((lane & 7) == 0 && idx0 < nE && T.fw) fcur[idx0 >> 5] = 0u;
    }
    if (!classify) continue;  // uniform
    const int* pu = &T.eu.x;
    const int* pw = &T.ew.x;
    int4 ent[4];
    int c = 0;
    uint32_t nib = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= nvalid || ((skip >> q) & 1u)) continue;
      const int u = pu[q], w = pw[q];
      if (u < 0 || u >= nV || w < 0 || w >= nV) {
        report_corrupt(st.g, 6, n, idx0 + q, u, w);  // never index with it
        continue;
      }
      const bool su = zrow[u] < ZT(0), sv = zrow[w] < ZT(0);
      if (su != sv) {
        ent[c++] = make_int4(int(idx0 + q), su ? w : u, su ? u : w, 0);
        nib |= 1u << q;
      }
    }
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.wcnt[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long tot = 0;
      for (int w = 0; w < kWarps; ++w) {
        const int cw = sm.wcnt[w];
        sm.wcnt[w] = int(tot);
        tot += cw;
      }
      if (sm.nla + tot <= kLaCap) {
        sm.use_smem = 1;
        sm.sbase = sm.nla;
        sm.nla += int(tot);
      } else {
        sm.use_smem = 0;
        sm.sbase = atomic_add_ll(counter, tot);
      }
    }
    __syncthreads();
    if (c) {
      const long long base = sm.sbase + sm.wcnt[warp] + (x - c);
      if (sm.use_smem) {
        for (int t = 0; t < c; ++t) sm.la[base + t] = ent[t];  // flagged when flushed
      } else {
        for (int t = 0; t < c; ++t) lnext[base + t] = ent[t];
      }
    }
    if (!sm.use_smem) {
      uint32_t word = nib << (idx0 & 31);  // the 8 lanes of a flag word OR their nibbles
      word |= __shfl_xor_sync(0xffffffffu, word, 1);
      word |= __shfl_xor_sync(0xffffffffu, word, 2);
      word |= __shfl_xor_sync(0xffffffffu, word, 4);
      if ((lane & 7) == 0 && word) atomicOr(fnext + (idx0 >> 5), word);
    }
    __syncthreads();  // sm.use_smem / sbase are reused by the next iteration
  }
}

__device__ void flush_cta(const State& st, Counters* cur, long long* cnext, int4* lnext, uint32_t* fnext,
                          long long ebase, bool ahead, Smem& sm);

// Layer start, step (3) for neuron 0 of layer l.
template <typename ZT>
__device__ void phase_scan0(const NetDesc& net, const State& st, int l, Smem& sm) {
  const int n0 = net.off[l];
  long long nV, nE;
  if (!step_counts(st, n0, nV, nE)) {
    if (threadIdx.x == 0) report_corrupt(st.g, 2, n0, nV, nE, st.Vcap);
    return;
  }
  const ZT* zrow = static_cast<const ZT*>(st.Z[l]);
  if (threadIdx.x == 0) {
    sm.npairs = 0;
    sm.npairla = 0;
    sm.nla = 0;
  }
  __syncthreads();
  const ScanTile first = scan_load(st, nullptr, scan_first_idx0(), nE, true);
  scan_edges<ZT>(st, zrow, nE, nV, nullptr, true, st.list[n0 & 1], st.flags[n0 & 1], &st.cnt[n0 + 1].nsplit, n0, sm,
                 first);
  __syncthreads();
  if (sm.nla) flush_cta(st, nullptr, &st.cnt[n0 + 1].nsplit, st.list[n0 & 1], st.flags[n0 & 1], 0, true, sm);
}

// ---------------------------------------------------------------------------
// Whole-warp check (inline pairing) that the 2-face key of the new vertex
// nV + k2 (payload r2 = 2 * zero ordinal + minus) equals F, where lane w holds word w of this
// splitting edge's sign vector s0 and F is s0 with word wj replaced by Fw.
// The partner's face is rebuilt from its new vertex's sign words, which the
// partner wrote (and fenced) before it inserted its key.  All lanes call it.
__device__ __forceinline__ bool warp_face_matches(const State& st, long long k2, int r2, int e, int S, uint64_t s0,
                                                  int wj, uint64_t Fw, long long nV, long long total, int n) {
  const int lane = threadIdx.x & 31;
  if (k2 < 0 || k2 >= total) {  // a payload that no new vertex of this step wrote
    if (lane == 0) report_corrupt(st.g, 5, n, k2, total, r2);
    return false;
  }
  const long long v2 = nV + k2;
  uint64_t w2 = 0, zm = 0;
  if (lane < S) {
    w2 = __ldcg(st.SIG + (long long)lane * st.Vcap + v2);
    zm = zero_mask(w2, lane, e);
  }
  const int c = __popcll(zm);
  int x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  const int o2 = r2 >> 1;
  int j2 = -1;
  if (o2 >= x - c && o2 < x) {
    uint64_t mm = zm;
    for (int q = x - c; q < o2; ++q) mm &= mm - 1;
    j2 = lane * 32 + (__ffsll((long long)mm) - 1) / 2;
  }
  const unsigned owner = __ballot_sync(0xffffffffu, j2 >= 0);
  if (!owner) return false;
  j2 = __shfl_sync(0xffffffffu, j2, __ffs(owner) - 1);
  if (lane == (j2 >> 5)) {
    const int sj = 2 * (j2 & 31);
    w2 = (w2 & ~(3ull << sj)) | (((r2 & 1) ? kMinus : kPlus) << sj);
  }
  const uint64_t f1 = (lane == wj) ? Fw : s0;
  return __all_sync(0xffffffffu, lane >= S || f1 == w2);
}

// ---------------------------------------------------------------------------
// Appends the CTA's buffered intersecting edges (and those of them that split
// at the next neuron) and buffered look-ahead entries: one atomic each for
// the CTA.  All threads call it after a __syncthreads.
__device__ void flush_cta(const State& st, Counters* cur, long long* cnext, int4* lnext, uint32_t* fnext,
                          long long ebase, bool ahead, Smem& sm) {
  const int np = sm.npairs, nla = sm.nla, npla = sm.npairla;
  if (threadIdx.x == 0) {
    sm.pbase = np ? atomic_add_ll(&cur->npairs, (long long)np) : 0;
    sm.lbase = (ahead && nla + npla) ? atomic_add_ll(cnext, (long long)(nla + npla)) : 0;
    sm.cursor = 0;
  }
  __syncthreads();
  const long long pb = ebase + sm.pbase;
  for (int t = threadIdx.x; t < np; t += kBlock) {
    const int4 rec = sm.pairs[t];
    st.EU[pb + t] = rec.x;
    st.EW[pb + t] = rec.y;
    if (st.deferred) st.vlist[pb + t] = rec;
    const unsigned char nx = sm.pnext[t];
    if (ahead && ((nx ^ (nx >> 1)) & 1)) {  // the new edge splits at the next neuron
      const int j = atomicAdd(&sm.cursor, 1);
      lnext[sm.lbase + nla + j] = (nx & 1) ? make_int4(int(pb + t), rec.y, rec.x, 0)
                                           : make_int4(int(pb + t), rec.x, rec.y, 0);
      set_flag(fnext, pb + t);
    }
  }
  for (int t = threadIdx.x; t < nla; t += kBlock) {
    const int4 ent = sm.la[t];
    lnext[sm.lbase + t] = ent;
    set_flag(fnext, ent.x);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.npairs = 0;
    sm.nla = 0;
    sm.npairla = 0;
  }
  __syncthreads();
}

// One neuron step: steps (4)+(5) for the listed splitting edges, step (3) for
// the next neuron.  Returns true when the step must not run (capacity ran out
// -- nothing has been written -- or a counter is corrupt); the caller exits.
template <typename ZT, bool MIXED>
__device__ bool phase_step(const NetDesc& net, const State& st, int l, int i, Smem& sm, double* ws, int mw) {
  constexpr bool TRACK = sizeof(ZT) == 4;  // FP32 values carry error estimates
  const int n = net.off[l] + i;
  const int H = net.w[l + 1];
  const bool ahead = i + 1 < H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long G = gridDim.x;
  const int4* lcur = st.list[n & 1];
  // this warp's first splitting edge, loaded together with the counters
  const long long k_first = (long long)warp * G + blockIdx.x;
  const int4 sg_first = k_first < st.Ecap ? lcur[k_first] : make_int4(-1, -1, -1, 0);
  Counters* cur = st.cnt + n + 1;
  long long nV, nE;
  if (!step_counts(st, n, nV, nE)) {
    if (threadIdx.x == 0) report_corrupt(st.g, 2, n, nV, nE, st.Vcap);
    return true;
  }
  const long long total = cur->nsplit;
  if (total < 0 || total > nE) {
    if (threadIdx.x == 0) report_corrupt(st.g, 3, n, total, nV, nE);
    return true;
  }
  const int D = net.D, m = net.m, S = net.S;
  const int R = D > 1 ? 2 * (D - 1) : 1;
  const long long kmax = total * (long long)(D - 1) * 2;
  long long tneed = 64;
  while (tneed < 2 * kmax) tneed <<= 1;
  const long long eneed = nE + total * (long long)D;
  const long long vneed = nV + total;
  const bool overV = vneed > st.Vcap || vneed >= (1ll << 31) || total * R >= (1ll << 31);
  const bool overE = eneed > st.Ecap || eneed >= (1ll << 31);
  const bool overT = tneed > st.Tcap;
  const bool overTape = st.keep_tape && vneed > st.tape_cap;
  if (overV || overE || overT || overTape) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      Global* g = st.g;
      if (atomicCAS(&g->halted_at, -1, n) == -1) {
        g->halt_reason = (overV ? kHaltV : 0) | (overE ? kHaltE : 0) | (overT ? kHaltT : 0) | (overTape ? kHaltTape : 0);
        g->need_v = vneed;
        g->need_e = eneed;
        g->need_t = tneed;
      }
    }
    return true;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cur->nV_before = nV;
    cur->nE_before = nE;
    cur->tsize = tneed;
  }
  if (threadIdx.x == 0) {
    sm.npairs = 0;
    sm.npairla = 0;
    sm.nla = 0;
    sm.npend = 0;
    sm.acc[0] = sm.acc[1] = 0;
  }
  if (sm.nrl_layer != l) {  // uniform: set by the previous step of this launch, or -1
    for (int t = threadIdx.x; t < 3 * H; t += kBlock) sm.nrl[t] = net.nrm[3 * net.off[l] + t];
  }
  // the table of the previous step: emptied for the step after this one
  {
    uint64_t* told = st.table + (long long)((n + 1) & 1) * 2 * st.Tcap;
    const long long tprev = 2 * st.cnt[n].tsize;
    for (long long t = (long long)blockIdx.x * kBlock + threadIdx.x; t < tprev; t += G * kBlock) told[t] = kEmpty;
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.nrl_layer = l;
  const long long Vcap = st.Vcap;
  ZT* Z = static_cast<ZT*>(st.Z[l]);
  const int e = m + n;
  const int e0 = m + net.off[l];
  int4* lnext = st.list[(n + 1) & 1];
  uint32_t* fnext = st.flags[(n + 1) & 1];
  long long* cnext = ahead ? &st.cnt[n + 2].nsplit : nullptr;
  uint64_t* table = st.table + (long long)(n & 1) * 2 * st.Tcap;
  const long long tmask = tneed - 1;
  const float* nrl = sm.nrl;
  int* zlist = sm.zlist[warp];
  long long nkeys_w = 0, ndeg_w = 0;
  int err_w = 0;
  unsigned long long paired_seen = 0;  // paired flags found by this lane's second arrivals
  const long long Wt = G * kWarps;
  const long long rounds = (total + Wt - 1) / Wt;
  int4 sg_next = sg_first;
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long k = rd * Wt + k_first;  // splits dealt over the CTAs first
    const int4 sg_this = sg_next;
    if (k + Wt < total) sg_next = lcur[k + Wt];  // the next round's, loaded during this one
    // The round's new vertices are numbered CTA by CTA: CTA b holds entries
    // w G + b of the round (w < n_b = rq + [b < rr]) and gives them the
    // consecutive offsets b rq + min(b, rr) + w, a bijection onto the
    // round's [0, rem), so each CTA writes whole sectors of the value,
    // coordinate and sign rows.
    const long long rem = total - rd * Wt < Wt ? total - rd * Wt : Wt;
    const long long rq = rem / G, rr = rem - rq * G;
    const long long voff = rd * Wt + blockIdx.x * rq + (blockIdx.x < rr ? blockIdx.x : rr) + warp;
    // ---- part A: the new vertex (step (4)) ----
    bool okA = false, pend = false, bad = false;
    int32_t ed = 0, p = 0, q = 0;
    const int32_t v0 = int32_t(nV + voff);
    uint64_t s0 = 0, zm = 0;
    ZT zpn = ZT(0), zqn = ZT(0), z0n = ZT(0);  // values at neuron i + 1
    if (k < total) {
      const int4 sg = sg_this;
      ed = sg.x;
      p = sg.y;  // V+
      q = sg.z;  // V-
      okA = !(ed < 0 || ed >= nE || p < 0 || p >= nV || q < 0 || q >= nV);  // warp-uniform
      if (!okA && lane == 0) report_corrupt(st.g, 4, n, ed, p, q);
    }
    if (okA) {
      // every load of the endpoints is issued before any of them is used
      const ZT za0 = Z[(long long)i * Vcap + p], zb0 = Z[(long long)i * Vcap + q];
      double xp = 0.0, xq = 0.0;
      if (lane < D) {
        xp = st.X[(long long)lane * Vcap + p];
        xq = st.X[(long long)lane * Vcap + q];
      }
      uint64_t sp = 0, sq = 0;
      if (lane < S) {
        sp = st.SIG[(long long)lane * Vcap + p];
        sq = st.SIG[(long long)lane * Vcap + q];
      }
      ZT zp0[2], zq0[2];  // rows lane, lane + 32 of the first 64
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int j = 32 * hh + lane;
        zp0[hh] = j < H ? Z[(long long)j * Vcap + p] : ZT(0);
        zq0[hh] = j < H ? Z[(long long)j * Vcap + q] : ZT(0);
      }
      float rp = 0.f, rq = 0.f, xep = 0.f, xeq = 0.f;
      if (TRACK && lane == 0) {
        rp = st.esc[p];
        rq = st.esc[q];
        xep = st.exc[p];
        xeq = st.exc[q];
      }
      const double a = static_cast<double>(za0);
      const double b = static_cast<double>(zb0);
      // t in float64 on one lane (the FP64 units are few), then broadcast
      double t = 0.0;
      int out_of_range = 0;
      if (lane == 0) {
        t = a / (a - b);
        if (!(t >= 0.0 && t <= 1.0)) {
          t = t < 0.0 ? 0.0 : 1.0;
          out_of_range = 1;
        }
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      out_of_range = __shfl_sync(0xffffffffu, out_of_range, 0);
      bad = !(a > 0.0 && b < 0.0) || out_of_range;
      if (lane < D) st.X[(long long)lane * Vcap + v0] = fma(t, xq - xp, xp);
      const ZT tz = static_cast<ZT>(t);
      // earlier layers' entries: the join of the endpoints' words
      const uint64_t below = lane < S ? entries_below(lane, e0) : 0ull;
      const uint64_t conf = ((sp & kEvenBits) & ((sq >> 1) & kEvenBits)) | ((sq & kEvenBits) & ((sp >> 1) & kEvenBits));
      if (conf & below) err_w |= kErrConflict;
      s0 = (sp | sq) & below;
      float amax = 0.f;
      float zk[2] = {0.f, 0.f};  // this lane's new values of rows lane, lane + 32 (filter)
      for (int c = 0; 64 * c < H; ++c) {
        uint32_t plus2[2], minus2[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int j = 64 * c + 32 * hh + lane;
          ZT zp = zp0[hh], zq = zq0[hh], zj = ZT(0);
          if (c > 0) {
            zp = j < H ? Z[(long long)j * Vcap + p] : ZT(0);
            zq = j < H ? Z[(long long)j * Vcap + q] : ZT(0);
          }
          bool pl = false, mi = false;
          if (j < H) {
            if (j < i) {  // processed: the join of the endpoints' signs, value made consistent
              pl = zp > ZT(0) || zq > ZT(0);
              mi = zp < ZT(0) || zq < ZT(0);
              if (pl && mi) err_w |= kErrConflict;
              zj = zp + tz * (zq - zp);
              if (pl && !(zj > ZT(0))) zj = tiny_value<ZT>();
              if (mi && !(zj < ZT(0))) zj = -tiny_value<ZT>();
              if (!pl && !mi) zj = ZT(0);
            } else if (j > i) {
              zj = zp + tz * (zq - zp);
              if (zj == ZT(0)) {  // on a later folded hyperplane: not generic
                zj = tiny_value<ZT>();
                atomic_add_ll(&st.cnt[net.off[l] + j + 1].ndegenerate, 1ll);
              }
            }
            Z[(long long)j * Vcap + v0] = zj;  // row i: exactly 0
            if (TRACK) amax = fmaxf(amax, fabsf(static_cast<float>(zj)) * nrl[3 * j + 2]);
          }
          if (c == 0) zk[hh] = static_cast<float>(zj);
          plus2[hh] = __ballot_sync(0xffffffffu, pl);
          minus2[hh] = __ballot_sync(0xffffffffu, mi);
          if (ahead && 64 * c + 32 * hh <= i + 1 && i + 1 < 64 * c + 32 * hh + 32) {  // warp-uniform
            const int src = (i + 1) & 31;
            zpn = __shfl_sync(0xffffffffu, zp, src);
            zqn = __shfl_sync(0xffffffffu, zq, src);
            z0n = __shfl_sync(0xffffffffu, zj, src);
          }
        }
        // this chunk's codes (entries e0 + 64c ...) into the lane's word
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const uint64_t il = spread_even(plus2[hh]) | (spread_even(minus2[hh]) << 1);
          if (!il) continue;
          const int ent = e0 + 64 * c + 32 * hh, w = ent >> 5, sft = 2 * (ent & 31);
          if (lane == w) s0 |= il << sft;
          if (sft && lane == w + 1) s0 |= il >> (64 - sft);
        }
      }
      if (TRACK) {
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        float dx = lane < D ? static_cast<float>(fabs(xq - xp)) : 0.f;
        for (int o = 16; o > 0; o >>= 1) dx = fmaxf(dx, __shfl_xor_sync(0xffffffffu, dx, o));
        float esc0 = 0.f;
        if (lane == 0) {
          // rms estimates, independent errors adding in quadrature: the value
          // scale takes the endpoints' (a convex combination does not amplify
          // them) and the interpolation's rounding (u |z_j|, in units of
          // ||W_j||_2); the position takes the endpoints' estimates and the
          // shift along the edge that the errors of a and b cause in t.
          const float rm = fmaxf(rp, rq), rr = 5.9604645e-8f * amax;
          esc0 = sqrtf(rm * rm + rr * rr);
          st.esc[v0] = esc0;
          const float ep = nrl[3 * i] * rp + 2.9802322e-8f * nrl[3 * i + 1];
          const float eq = nrl[3 * i] * rq + 2.9802322e-8f * nrl[3 * i + 1];
          const float shift = static_cast<float>((ep + eq) / (a - b)) * dx;
          const float xe = fmaxf(xep, xeq);
          st.exc[v0] = sqrtf(xe * xe + shift * shift);
        }
        if (MIXED) {  // the later neurons' new values within the filter
          esc0 = __shfl_sync(0xffffffffu, esc0, 0);
          bool f = false;
          for (int j = lane; j < H; j += 32) {
            if (j <= i) continue;
            const float zv = j < 64 ? zk[j >> 5] : static_cast<float>(Z[(long long)j * Vcap + v0]);
            f = f || fabsf(zv) <= net.kappa_sel * (nrl[3 * j] * esc0 + 2.9802322e-8f * nrl[3 * j + 1]);
          }
          pend = __any_sync(0xffffffffu, f);
        }
      }
      if (lane < S) {
        st.SIG[(long long)lane * Vcap + v0] = s0;
        zm = zero_mask(s0, lane, e);
      }
      if (lane == 0) {
        st.EU[ed] = p;
        st.EW[ed] = v0;
        st.EU[nE + k] = q;
        st.EW[nE + k] = v0;
        if (st.deferred) st.vlist[nE + k] = make_int4(0, 0, 0, 0);  // not a pairing edge
        if (st.keep_tape) {
          st.tape_pq[v0] = p;
          st.tape_pq[st.tape_cap + v0] = q;
          st.tape_t[v0] = t;
        }
        if (pend) sm.pend[atomicAdd(&sm.npend, 1)] = v0;
      }
    }
    if (MIXED) {  // FP64 re-decisions of this round's new vertices (uniform per CTA)
      __syncthreads();
      if (sm.npend > 0) drain_pending<ZT>(net, st, l, e + 1, i + 1, mw, ws, sm);
    }
    if (okA) {
      // ---- part B: the parent 2-faces (step (5)) and the look-ahead ----
      if (ahead && pend) z0n = Z[(long long)(i + 1) * Vcap + v0];  // re-decided by this CTA
      const bool m0n = z0n < ZT(0);
      const int c0 = __popcll(zm);
      int x = c0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const int nz = __shfl_sync(0xffffffffu, x, 31);
      {
        int kk = x - c0;
        uint64_t mm = zm;
        while (mm) {
          const int bit = __ffsll((long long)mm) - 1;
          if (kk < 16) zlist[kk] = lane * 32 + bit / 2;
          ++kk;
          mm &= mm - 1;
        }
      }
      uint64_t hb = lane < S ? word_hash(lane, s0) : 0ull;
      for (int o = 16; o > 0; o >>= 1) hb ^= __shfl_xor_sync(0xffffffffu, hb, o);
      __syncwarp();
      if (nz != D - 1) bad = true;
      // this lane's key: zero ordinal lane / 2, sign + (even lane) or - (odd)
      const int o = lane >> 1;
      const bool minus = lane & 1;
      const int jz = (nz == D - 1 && o < nz) ? zlist[o] : 0;
      const int wj = jz >> 5, shj = 2 * (jz & 31);
      const uint64_t s0w = __shfl_sync(0xffffffffu, s0, wj);
      const bool has_key = (nz == D - 1) && (o < nz) && !(minus && jz < m);
      nkeys_w += __popc(__ballot_sync(0xffffffffu, has_key));
      if (bad) ndeg_w += (lane == 0);
      uint64_t Fw = 0, h = 0;
      long long slot = 0;
      if (has_key) {
        Fw = (s0w & ~(3ull << shj)) | ((minus ? kMinus : kPlus) << shj);
        h = hb ^ word_hash(wj, s0w) ^ word_hash(wj, Fw);
        slot = (long long)(h & (uint64_t)tmask);
      }
      if (st.deferred) {
        // Full 64-bit fingerprint and payload in one 16-byte slot: the first
        // arrival inserts both with one 128-bit CAS, the second finds the
        // partner (and its sign at the next neuron, bit 62) in the same
        // atomic and pairs at once; the paired flag it sets is checked at the
        // end.  Every pairing is re-checked exactly after the extraction
        // (k_verify_pairs) from the two new vertices' sign vectors.
        if (has_key) {
          if (h == kEmpty) h = kEmpty - 1;
          const unsigned long long mine = (uint64_t(voff) * R + uint64_t(lane)) | (m0n ? (1ull << 62) : 0ull);
          unsigned long long* tb = reinterpret_cast<unsigned long long*>(table);
          for (long long probes = 0;; ++probes) {
            if (probes > tneed) {
              err_w |= kErrProbe;
              break;
            }
            unsigned long long ok, ov;
            cas128(tb + 2 * slot, kEmpty, kEmpty, h, mine, ok, ov);
            if (ok == kEmpty) break;  // first arrival
            if (ok == h) {
              paired_seen |= atomicOr(tb + 2 * slot + 1, kPaired64);
              const unsigned long long pay = ov & ~(kPaired64 | (1ull << 62));
              const long long k2 = (long long)(pay / R);
              const int r2 = int(pay % R);
              const unsigned char nx = ((ov >> 62) & 1ull ? 1 : 0) | (m0n ? 2 : 0);
              const int slot2 = atomicAdd(&sm.npairs, 1);  // < kPairCap: flushed every round
              sm.pairs[slot2] = make_int4(int(nV + k2), v0, (r2 << 16) | lane, n + 1);
              sm.pnext[slot2] = nx;
              if (ahead && ((nx ^ (nx >> 1)) & 1)) atomicAdd(&sm.npairla, 1);
              break;
            }
            slot = (slot + 1) & tmask;
          }
        }
      } else {
        // Inline: a 32-bit tag; the second arrival compares the full faces
        // before it pairs.  The partner's sign words and value at the next
        // neuron are read from memory, so they are fenced before the insert.
        __threadfence();
        __syncwarp();
        const uint32_t tag = uint32_t(h >> 32);
        const uint64_t mine = has_key ? ((uint64_t(tag) << 32) | (uint64_t(voff) * R + uint64_t(lane))) : 0ull;
        bool active = has_key;
        long long probes = 0;
        while (__any_sync(0xffffffffu, active)) {
          bool cand = false;
          uint64_t old = 0;
          if (active) {
            old = atomicCAS(reinterpret_cast<unsigned long long*>(table + slot), (unsigned long long)kEmpty,
                            (unsigned long long)mine);
            if (old == kEmpty) {
              active = false;  // first arrival: the partner will pair with it
            } else if (uint32_t(old >> 32) == tag) {
              cand = true;
            } else {
              slot = (slot + 1) & tmask;
              if (++probes > tneed) {
                err_w |= kErrProbe;
                active = false;
              }
            }
          }
          __threadfence();
          unsigned cm = __ballot_sync(0xffffffffu, cand);
          while (cm) {
            const int Ld = __ffs(cm) - 1;
            cm &= cm - 1;
            const uint64_t pp = __shfl_sync(0xffffffffu, old, Ld) & 0x7fffffffull;
            const int wjL = __shfl_sync(0xffffffffu, wj, Ld);
            const uint64_t FwL = __shfl_sync(0xffffffffu, Fw, Ld);
            const bool eq =
                warp_face_matches(st, (long long)(pp / R), int(pp % R), e, S, s0, wjL, FwL, nV, total, n);
            if (lane == Ld) {
              if (eq) {
                const uint64_t prev = atomicOr(reinterpret_cast<unsigned long long*>(table + slot),
                                               (unsigned long long)kPaired);
                if (prev & kPaired) {
                  err_w |= kErrPairing;
                } else {
                  const int v2 = int(nV + (long long)(pp / R));
                  const bool m2 = ahead && __ldcg(Z + (long long)(i + 1) * Vcap + v2) < ZT(0);
                  const unsigned char nx = (m2 ? 1 : 0) | (m0n ? 2 : 0);
                  const int slot2 = atomicAdd(&sm.npairs, 1);  // < kPairCap: flushed every round
                  sm.pairs[slot2] = make_int4(v2, v0, 0, 0);
                  sm.pnext[slot2] = nx;
                  if (ahead && ((nx ^ (nx >> 1)) & 1)) atomicAdd(&sm.npairla, 1);
                }
                active = false;
              } else {
                slot = (slot + 1) & tmask;
                if (++probes > tneed) {
                  err_w |= kErrProbe;
                  active = false;
                }
              }
            }
          }
        }
      }
      // look-ahead: the two halves of the split edge at neuron i + 1
      if (ahead && lane == 0) {
        const bool mp = zpn < ZT(0), mq = zqn < ZT(0);
        int4 ent[2];
        int c = 0;
        if (mp != m0n) ent[c++] = mp ? make_int4(ed, v0, p, 0) : make_int4(ed, p, v0, 0);
        if (mq != m0n) ent[c++] = mq ? make_int4(int(nE + k), v0, q, 0) : make_int4(int(nE + k), q, v0, 0);
        if (c) {
          const int b2 = atomicAdd(&sm.nla, c);  // < kLaCap: flushed every round
          for (int t2 = 0; t2 < c; ++t2) sm.la[b2 + t2] = ent[t2];
        }
      }
      __syncwarp();
    }
    // keep the CTA's buffers from filling up in the next round
    __syncthreads();
    if (sm.npairs > kPairCap - kWarps * R || sm.nla > kLaCap - 2 * kWarps)
      flush_cta(st, cur, cnext, lnext, fnext, nE + total, ahead, sm);
  }
  if (paired_seen & kPaired64) err_w |= kErrPairing;  // a third arrival at a 2-face
  err_w = __reduce_or_sync(0xffffffffu, err_w);
  if (lane == 0) {
    if (nkeys_w) atomicAdd(reinterpret_cast<unsigned long long*>(&sm.acc[0]), (unsigned long long)nkeys_w);
    if (ndeg_w) atomicAdd(reinterpret_cast<unsigned long long*>(&sm.acc[1]), (unsigned long long)ndeg_w);
    if (err_w) atomicOr(&st.g->error, err_w);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sm.acc[0]) atomic_add_ll(&cur->nkeys, sm.acc[0]);
    if (sm.acc[1]) atomic_add_ll(&cur->ndegenerate, sm.acc[1]);
  }
  // step (3) for the next neuron over the edges that did not split here
  const ZT* znext = Z + (long long)(ahead ? i + 1 : 0) * Vcap;
  const ScanTile scan_first = scan_load(st, st.flags[n & 1], scan_first_idx0(), nE, ahead);
  scan_edges<ZT>(st, znext, nE, nV, st.flags[n & 1], ahead, lnext, fnext, cnext, n, sm, scan_first);
  __syncthreads();
  if (sm.npairs || sm.nla) flush_cta(st, cur, cnext, lnext, fnext, nE + total, ahead, sm);
  return false;
}

// ---------------------------------------------------------------------------
// Layer end: the codes of the layer's entries of every vertex from the signs
// of its values (+ / - / 0 exactly on the folded hyperplane).
template <typename ZT>
__device__ __noinline__ void phase_pack(const NetDesc& net, const State& st, int l) {
  const int H = net.w[l + 1];
  const Counters* last = st.cnt + net.off[l] + H;
  const long long nV = last->nV_before + last->nsplit;
  if (nV < 0 || nV > st.Vcap) {
    if (threadIdx.x == 0) report_corrupt(st.g, 12, l, nV, st.Vcap, 0);
    return;
  }
  const long long Vcap = st.Vcap;
  const ZT* Z = static_cast<const ZT*>(st.Z[l]);
  const int e0 = net.m + net.off[l], wf = e0 >> 5, wl = (e0 + H - 1) >> 5;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nV; v += (long long)gridDim.x * blockDim.x) {
    for (int w = wf; w <= wl; ++w) {
      uint64_t word = w == wf ? (st.SIG[(long long)w * Vcap + v] & entries_below(w, e0)) : 0ull;
      const int jb = 32 * w - e0 > 0 ? 32 * w - e0 : 0;
      const int je = 32 * w + 32 - e0 < H ? 32 * w + 32 - e0 : H;
      for (int j = jb; j < je; ++j) {
        const ZT z = Z[(long long)j * Vcap + v];
        const uint64_t code = z > ZT(0) ? kPlus : (z < ZT(0) ? kMinus : 0ull);
        word |= code << (2 * ((e0 + j) & 31));
      }
      st.SIG[(long long)w * Vcap + v] = word;
    }
  }
}

}  // namespace pc
