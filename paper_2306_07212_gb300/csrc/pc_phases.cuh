// The per-neuron steps of edge subdivision (Section 4.2) as device functions.
//
// One neuron step is two phases separated by grid-wide synchronisation (a
// kernel boundary in stepwise execution, a grid barrier in the persistent
// per-layer kernel):
//
//   phase_classify  steps (2)+(3).  Every vertex's sign w.r.t. the neuron's
//       folded hyperplane is written into its sign vector; in the same pass
//       every edge is classified from the signs of its endpoints' stored
//       values (splitting iff they differ) and the splitting edges are
//       compacted per CTA range with warp ballots and a block scan, keeping
//       edge order.  In mixed precision a |z| within kappa times its FP32
//       error estimate is re-decided in FP64 at the exact vertex; the edge
//       pass used the FP32 sign, so if a re-decision flips a sign the step is
//       marked and the edges are classified again from the final signs
//       (phase_reclassify) before splitting.
//
//   phase_split  steps (4)+(5).  One warp per splitting edge interpolates the
//       new vertex (FP64 t and coordinates, values in the value type), splits
//       the edge into E+ and E-, and inserts the edge's parent 2-face keys
//       into an open-addressing hash table.  Default: each slot holds the
//       face's 64-bit fingerprint and the first occurrence's payload, written
//       with one 128-bit CAS; the second occurrence pairs in the same atomic
//       and records the pairing, which k_verify_pairs checks exactly after
//       the last step.  Inline mode: the second occurrence compares the full
//       face before it pairs.
#pragma once

#include "pc_device.cuh"
#include "pc_newton.cuh"

namespace pc {

constexpr int kPairCap = 1024;   // intersecting edges a CTA buffers per step

struct Smem {
  long long pref[kMaxGrid + 1];
  long long wsum[kWarps + 1];
  long long flist[kFilterCap];
  int zlist[kWarps][32];
  int4 pairs[kPairCap];   // (v_partner, v_new, zero ordinals, neuron + 1)
  int npairs;
  int fcount;
  int flip;
  int nzl[kMaxD + 2];
  NewtonOut nout;
  long long acc[4];
};

__device__ __forceinline__ long long warp_sum_ll(long long x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Exclusive scan of sm.pref[0..G) in place; sm.pref[G] = total.  G <= kMaxGrid.
__device__ __forceinline__ void block_scan_pref(Smem& sm, int G) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int per = kMaxGrid / kBlock;
  long long loc[per];
  long long s = 0;
#pragma unroll
  for (int q = 0; q < per; ++q) {
    const int idx = t * per + q;
    loc[q] = idx < G ? sm.pref[idx] : 0;
    s += loc[q];
  }
  long long x = s;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm.wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < kWarps ? sm.wsum[lane] : 0;
    long long xx = w;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, xx, o);
      if (lane >= o) xx += y;
    }
    if (lane < kWarps) sm.wsum[lane] = xx - w;
    if (lane == kWarps - 1) sm.wsum[kWarps] = xx;
  }
  __syncthreads();
  long long run = sm.wsum[warp] + (x - s);
#pragma unroll
  for (int q = 0; q < per; ++q) {
    const int idx = t * per + q;
    if (idx < G) sm.pref[idx] = run;
    run += loc[q];
  }
  if (t == 0) sm.pref[G] = sm.wsum[kWarps];
  __syncthreads();
}

// Block-wide exclusive scan of one small count per thread; returns the
// thread's offset and leaves the block total in sm.wsum[kWarps].
__device__ __forceinline__ int block_offsets(Smem& sm, int c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm.wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const long long w = lane < kWarps ? sm.wsum[lane] : 0;
    long long xx = w;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, xx, o);
      if (lane >= o) xx += y;
    }
    if (lane < kWarps) sm.wsum[lane] = xx - w;
    if (lane == kWarps - 1) sm.wsum[kWarps] = xx;
  }
  __syncthreads();
  return int(sm.wsum[warp]) + x - c;
}

// Tag stored beside each CTA's count: identifies the step that wrote it.
__device__ __forceinline__ long long cta_tag(int n, long long nE) { return nE * 65536 + n + 1; }

// Edge range of this CTA in the compaction (a multiple of 4 edges per CTA).
__device__ __forceinline__ void cta_range(long long nE, long long& chunk, long long& begin, long long& end) {
  const long long G = gridDim.x;
  chunk = ((nE + G - 1) / G + 3) & ~3ll;
  begin = blockIdx.x * chunk;
  if (begin > nE) begin = nE;
  end = begin + chunk < nE ? begin + chunk : nE;
}

// Compacts the splitting edges of [begin, end) into stage[begin ...] in edge
// order as (edge, V+, V-).  FROM_CODES: classify from the stored sign codes
// (after every sign is final); otherwise from the sign of the stored value.
template <typename ZT, bool FROM_CODES>
__device__ long long compact_edges(const State& st, const ZT* zrow, int e, long long begin, long long end,
                                   long long nV, int n, Smem& sm) {
  const int sh = 2 * (e & 31);
  const uint64_t* sw = st.SIG + (long long)(e >> 5) * st.Vcap;
  long long count = 0;
  for (long long base = begin; base < end; base += 4 * kBlock) {
    const long long idx0 = base + 4 * threadIdx.x;
    int4 eu = make_int4(0, 0, 0, 0), ew = make_int4(0, 0, 0, 0);
    int nvalid = 0;
    if (idx0 < end) {
      nvalid = end - idx0 >= 4 ? 4 : int(end - idx0);
      if (nvalid == 4) {
        eu = *reinterpret_cast<const int4*>(st.EU + idx0);
        ew = *reinterpret_cast<const int4*>(st.EW + idx0);
      } else {
        int* pu = &eu.x;
        int* pw = &ew.x;
        for (int q = 0; q < nvalid; ++q) {
          pu[q] = st.EU[idx0 + q];
          pw[q] = st.EW[idx0 + q];
        }
      }
    }
    const int* pu = &eu.x;
    const int* pw = &ew.x;
    bool uplus[4], split[4];
    int c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      split[q] = false;
      uplus[q] = true;
      if (q < nvalid && (pu[q] < 0 || pu[q] >= nV || pw[q] < 0 || pw[q] >= nV)) {
        report_corrupt(st.g, 6, n, idx0 + q, pu[q], pw[q]);  // never index with it
      } else if (q < nvalid) {
        bool su, sv;
        if (FROM_CODES) {
          su = ((sw[pu[q]] >> sh) & 3ull) == kMinus;
          sv = ((sw[pw[q]] >> sh) & 3ull) == kMinus;
        } else {
          su = zrow[pu[q]] < ZT(0);
          sv = zrow[pw[q]] < ZT(0);
        }
        split[q] = su != sv;
        uplus[q] = !su;
        c += split[q];
      }
    }
    const int off = block_offsets(sm, c);
    int k = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (split[q]) {
        const int p = uplus[q] ? pu[q] : pw[q];
        const int mq = uplus[q] ? pw[q] : pu[q];
        st.stage[begin + count + off + k] = make_int4(int(idx0 + q), p, mq, 0);
        ++k;
      }
    }
    count += sm.wsum[kWarps];
    __syncthreads();
  }
  return count;
}

// ---------------------------------------------------------------------------
// Steps (2)+(3).
template <typename ZT, bool MIXED>
__device__ void phase_classify(const NetDesc& net, const State& st, int zb, int l, int i, int n,
                               Smem& sm, double* ws, int mw) {
  const Counters* prev = st.cnt + n;
  const long long nV = prev->nV_before + prev->nsplit;
  const long long nE = prev->pruned_e1 > 0 ? prev->pruned_e1 - 1 : prev->nE_before + prev->nsplit + prev->npairs;
  Counters* cur = st.cnt + n + 1;
  if (nV < 0 || nV > st.Vcap || nE < 0 || nE > st.Ecap) {
    if (threadIdx.x == 0) report_corrupt(st.g, 2, n, nV, nE, st.Vcap);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cur->nV_before = nV;
    cur->nE_before = nE;
  }
  const long long Vcap = st.Vcap;
  ZT* Z = static_cast<ZT*>(st.Z[zb]);
  const ZT* zrow = Z + (long long)i * Vcap;
  const int e = net.m + n, sh = 2 * (e & 31);
  uint64_t* sw = st.SIG + (long long)(e >> 5) * Vcap;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    sm.fcount = 0;
    sm.flip = 0;
  }
  __syncthreads();
  long long ndeg = 0;
  int und = 0;
  // FP64 re-decision of the CTA's filtered vertices, one at a time with all
  // threads cooperating (newton_cta).
  auto drain = [&]() {
    const int fc = sm.fcount;
    for (int q = 0; q < fc; ++q) {
      const long long v = sm.flist[q];
      newton_cta(net, st, v, e, l, i, mw, ws, sm.nzl, &sm.nout);
      if (threadIdx.x == 0) {
        const double zs = sm.nout.z;
        if (fabs(zs) <= 1e-12 * sm.nout.scale || !sm.nout.ok) ++und;
        const uint64_t code = zs < 0.0 ? kMinus : kPlus;
        const bool spec_minus = zrow[v] < ZT(0);
        if (spec_minus != (code == kMinus)) sm.flip = 1;
        sw[v] = (sw[v] & ~(3ull << sh)) | (code << sh);
        ZT zz = static_cast<ZT>(zs);
        if (code == kPlus && !(zz > ZT(0))) zz = ZT(1e-30);
        if (code == kMinus && !(zz < ZT(0))) zz = ZT(-1e-30);
        Z[(long long)i * Vcap + v] = zz;
      }
    }
    if (threadIdx.x == 0 && fc > 0) atomic_add_ll(&cur->nfilter, (long long)fc);
    __syncthreads();
    if (threadIdx.x == 0) sm.fcount = 0;
    __syncthreads();
  };
  const float nr_i = net.nrm[3 * n], b_i = 2.9802322e-8f * net.nrm[3 * n + 1];
  // step (2): the signs; 32-vertex tiles are dealt round-robin over the CTAs
  // so that neighbouring vertices (often filtered together) spread out
  const long long G = gridDim.x;
  const int warp = threadIdx.x >> 5;
  for (long long round = 0; round * G * kBlock < nV; ++round) {
    const long long v = ((round * kWarps + warp) * G + blockIdx.x) * 32 + lane;
    if (v < nV) {
      const ZT z = zrow[v];
      bool filt = false;
      if (MIXED) filt = fabsf(static_cast<float>(z)) <= net.kappa * (nr_i * st.esc[v] + b_i);
      if (filt) {
        const int slot = atomicAdd(&sm.fcount, 1);
        sm.flist[slot] = v;
      } else {
        const uint64_t code = (z < ZT(0)) ? kMinus : kPlus;
        ndeg += (z == ZT(0));
        sw[v] = (sw[v] & ~(3ull << sh)) | (code << sh);
      }
    }
    if (MIXED) {
      __syncthreads();
      if (sm.fcount > kFilterCap - kBlock) drain();
    }
  }
  if (MIXED) {
    __syncthreads();
    drain();
    if (threadIdx.x == 0 && sm.flip) atomicMax(&st.g->flip_at, n);
  }
  // the part of the hash table that the previous neuron used
  const long long tprev = 2 * st.cnt[n].tsize;  // 16-byte slots (the inline mode uses the first half)
  for (long long t = (long long)blockIdx.x * kBlock + threadIdx.x; t < tprev; t += (long long)gridDim.x * kBlock)
    st.table[t] = kEmpty;
  // step (3): splitting edges, speculatively from the signs of the values
  long long chunk, begin, end;
  cta_range(nE, chunk, begin, end);
  const long long count = compact_edges<ZT, false>(st, zrow, e, begin, end, nV, n, sm);
  if (threadIdx.x == 0) {
    st.cta_count[blockIdx.x] = count;
    st.cta_count[kMaxGrid + blockIdx.x] = cta_tag(n, nE);
  }
  ndeg = warp_sum_ll(ndeg);
  if (lane == 0 && ndeg) atomic_add_ll(&cur->ndegenerate, ndeg);
  if (MIXED && threadIdx.x == 0 && und) atomic_add_ll(&cur->nundecided, (long long)und);
}

// Step (3) again from the final sign codes, for a step whose FP64 re-decision
// flipped a sign that the speculative pass had used.
__device__ __forceinline__ void phase_reclassify(const NetDesc& net, const State& st, int n, Smem& sm) {
  const long long nV = st.cnt[n + 1].nV_before, nE = st.cnt[n + 1].nE_before;
  long long chunk, begin, end;
  cta_range(nE, chunk, begin, end);
  const long long count = compact_edges<float, true>(st, nullptr, net.m + n, begin, end, nV, n, sm);
  if (threadIdx.x == 0) {
    st.cta_count[blockIdx.x] = count;
    st.cta_count[kMaxGrid + blockIdx.x] = cta_tag(n, nE);
  }
}

// Whole-warp check that the 2-face key of split edge k2 (payload r2 =
// 2 * zero ordinal + minus) equals F, where lane w holds word w of the
// splitting edge's sign vector s0 and F is s0 with word wj replaced by Fw.
// The partner's key is rebuilt from its staged endpoints, which this phase
// does not modify, so no memory fence is needed.  All lanes must call it.
__device__ __forceinline__ bool warp_face_matches(const State& st, const Smem& sm, int G, long long chunk,
                                                  long long k2, int r2, int e, int S, uint64_t s0,
                                                  int wj, uint64_t Fw, long long nV, long long total, int n) {
  const int lane = threadIdx.x & 31;
  if (k2 < 0 || k2 >= total) {  // a payload that no split of this step wrote
    if (lane == 0) report_corrupt(st.g, 5, n, k2, total, r2);
    return false;
  }
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sm.pref[mid] <= k2) lo = mid; else hi = mid - 1;
  }
  const int4 s2 = st.stage[lo * chunk + (k2 - sm.pref[lo])];
  if (s2.y < 0 || s2.y >= nV || s2.z < 0 || s2.z >= nV) {
    if (lane == 0) report_corrupt(st.g, 7, n, k2, s2.y, s2.z);
    return false;
  }
  const long long Vcap = st.Vcap;
  const int wn = e >> 5, sh = 2 * (e & 31);
  uint64_t w2 = 0, zm = 0;
  if (lane < S) {
    w2 = st.SIG[(long long)lane * Vcap + s2.y] | st.SIG[(long long)lane * Vcap + s2.z];
    if (lane == wn) w2 &= ~(3ull << sh);
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
// Steps (4)+(5).  Returns true when capacity ran out (nothing written).
template <typename ZT, bool MIXED>
__device__ bool phase_split(const NetDesc& net, const State& st, int zb, int l, int i, int n, Smem& sm) {
  constexpr bool TRACK = sizeof(ZT) == 4;  // FP32 values carry error estimates
  Counters* cur = st.cnt + n + 1;
  const long long nV = cur->nV_before, nE = cur->nE_before;
  const int G = gridDim.x;
  {
    // every CTA range of this step must carry a count written for this step
    long long chunk0, b0_, b1_;
    cta_range(nE, chunk0, b0_, b1_);
    int bad = 0;
    for (int q = threadIdx.x; q < G; q += kBlock) {
      const long long cq = st.cta_count[q], tq = st.cta_count[kMaxGrid + q];
      sm.pref[q] = cq;
      if (tq != cta_tag(n, nE) || cq < 0 || cq > chunk0) {
        report_corrupt(st.g, 8, n, q, tq, cq);
        bad = 1;
      }
    }
    if (__syncthreads_or(bad)) return true;
  }
  if (threadIdx.x == 0) {
    sm.npairs = 0;
    sm.acc[0] = sm.acc[1] = 0;
  }
  __syncthreads();
  block_scan_pref(sm, G);
  const long long total = sm.pref[G];
  if (total < 0 || total > nE || nV < 0 || nV > st.Vcap || nE > st.Ecap) {
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
    cur->nsplit = total;
    cur->tsize = tneed;
  }
  const long long Vcap = st.Vcap;
  long long chunk, b0, b1;
  cta_range(nE, chunk, b0, b1);
  const int H = net.w[l + 1];
  ZT* Z = static_cast<ZT*>(st.Z[zb]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = m + n, wn = e >> 5, sh = 2 * (e & 31);
  int* zlist = sm.zlist[warp];
  const long long tmask = tneed - 1;
  long long nkeys_w = 0, ndeg_w = 0;
  int err_w = 0;
  for (long long k = (long long)blockIdx.x * kWarps + warp; k < total; k += (long long)G * kWarps) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {  // largest q with pref[q] <= k
      const int mid = (lo + hi + 1) >> 1;
      if (sm.pref[mid] <= k) lo = mid; else hi = mid - 1;
    }
    const int4 sg = st.stage[lo * chunk + (k - sm.pref[lo])];
    const int32_t ed = sg.x, p = sg.y, q = sg.z;  // p: V+, q: V-
    if (ed < 0 || ed >= nE || p < 0 || p >= nV || q < 0 || q >= nV) {  // warp-uniform
      if (lane == 0) report_corrupt(st.g, 4, n, ed, p, q);
      continue;
    }
    // every endpoint load is issued before any of them is used
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
    ZT zpa = ZT(0), zqa = ZT(0), zpb = ZT(0), zqb = ZT(0);  // rows lane and lane + 32 of the first 64
    if (lane < H) {
      zpa = Z[(long long)lane * Vcap + p];
      zqa = Z[(long long)lane * Vcap + q];
    }
    if (lane + 32 < H) {
      zpb = Z[(long long)(lane + 32) * Vcap + p];
      zqb = Z[(long long)(lane + 32) * Vcap + q];
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
    double t = a / (a - b);
    bool bad = !(a > 0.0 && b < 0.0);
    if (!(t >= 0.0 && t <= 1.0)) { t = t < 0.0 ? 0.0 : 1.0; bad = true; }
    const int32_t v0 = int32_t(nV + k);
    if (lane < D) st.X[(long long)lane * Vcap + v0] = fma(t, xq - xp, xp);
    const ZT tz = static_cast<ZT>(t);
    const float* nrl = net.nrm + 3 * net.off[l];
    float amax = 0.f;
    for (int j0 = 0; j0 < H; j0 += 64) {
      const int ja = j0 + lane, jb = ja + 32;
      if (j0 > 0) {
        zpa = zqa = zpb = zqb = ZT(0);
        if (ja < H) {
          zpa = Z[(long long)ja * Vcap + p];
          zqa = Z[(long long)ja * Vcap + q];
        }
        if (jb < H) {
          zpb = Z[(long long)jb * Vcap + p];
          zqb = Z[(long long)jb * Vcap + q];
        }
      }
      const ZT za = (ja == i) ? ZT(0) : zpa + tz * (zqa - zpa);
      const ZT zb2 = (jb == i) ? ZT(0) : zpb + tz * (zqb - zpb);
      if (ja < H) Z[(long long)ja * Vcap + v0] = za;
      if (jb < H) Z[(long long)jb * Vcap + v0] = zb2;
      if (TRACK) {  // the rounding of z_j, in units of ||W_j||_2
        if (ja < H) amax = fmaxf(amax, fabsf(static_cast<float>(za)) * nrl[3 * ja + 2]);
        if (jb < H) amax = fmaxf(amax, fabsf(static_cast<float>(zb2)) * nrl[3 * jb + 2]);
      }
    }
    if (TRACK) {
      // error estimates: values (rounding of the interpolation) and position
      // (a t computed from values carrying the endpoints' estimates)
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      float dx = lane < D ? static_cast<float>(fabs(xq - xp)) : 0.f;
      for (int o = 16; o > 0; o >>= 1) dx = fmaxf(dx, __shfl_xor_sync(0xffffffffu, dx, o));
      if (lane == 0) {
        // rms estimates, independent errors adding in quadrature.  value
        // scale: the endpoints' scales (the convex combination does not
        // amplify them) and the interpolation's rounding (u of |z_j|, in units
        // of ||W_j||_2).
        // position: the shift along the edge that the errors of a and b cause
        // in t = a / (a - b), added in quadrature to the endpoints' position
        // estimates (independent errors; the convex combination does not
        // amplify the endpoints' own errors).
        const float rm = fmaxf(rp, rq), rr = 5.9604645e-8f * amax;
        st.esc[v0] = sqrtf(rm * rm + rr * rr);
        const float ep = nrl[3 * i] * rp + 2.9802322e-8f * nrl[3 * i + 1];
        const float eq = nrl[3 * i] * rq + 2.9802322e-8f * nrl[3 * i + 1];
        const float shift = static_cast<float>((ep + eq) / (a - b)) * dx;
        const float xe = fmaxf(xep, xeq);
        st.exc[v0] = sqrtf(xe * xe + shift * shift);
      }
    }
    // sign vector of the new vertex: join of the endpoints, entry n := 0
    uint64_t s0 = 0, zm = 0;
    if (lane < S) {
      uint64_t conf = ((sp & kEvenBits) & ((sq >> 1) & kEvenBits)) | ((sq & kEvenBits) & ((sp >> 1) & kEvenBits));
      s0 = sp | sq;
      if (lane == wn) {
        conf &= ~(1ull << sh);
        s0 &= ~(3ull << sh);
      }
      if (conf) err_w |= kErrConflict;
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
    }
    // zero entries of the splitting edge (D-1 of them under genericity)
    const int c = __popcll(zm);
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const int nz = __shfl_sync(0xffffffffu, x, 31);
    {
      int kk = x - c;
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
    if (bad) ndeg_w += 1;
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
      // partner in the same atomic and pairs at once.  Every pairing is
      // re-checked exactly after the extraction (k_verify_pairs) from the
      // two new vertices' sign vectors.
      if (has_key) {
        if (h == kEmpty) h = kEmpty - 1;
        const unsigned long long mine = uint64_t(k) * R + uint64_t(lane);
        unsigned long long* tb = reinterpret_cast<unsigned long long*>(st.table);
        for (long long probes = 0;; ++probes) {
          if (probes > tneed) {
            err_w |= kErrProbe;
            break;
          }
          unsigned long long ok, ov;
          cas128(tb + 2 * slot, kEmpty, kEmpty, h, mine, ok, ov);
          if (ok == kEmpty) break;  // first arrival
          if (ok == h) {
            const unsigned long long prev = atomicOr(tb + 2 * slot + 1, kPaired64);
            if (prev & kPaired64) {
              err_w |= kErrPairing;
            } else {
              const long long k2 = (long long)((ov & ~kPaired64) / R);
              const int r2 = int((ov & ~kPaired64) % R);
              const int4 rec = make_int4(int(nV + k2), v0, (r2 << 16) | lane, n + 1);
              const int slot2 = atomicAdd(&sm.npairs, 1);
              if (slot2 < kPairCap) {
                sm.pairs[slot2] = rec;
              } else {
                const long long idx = atomic_add_ll(&cur->npairs, 1ll);
                st.EU[nE + total + idx] = rec.x;
                st.EW[nE + total + idx] = rec.y;
                st.vlist[nE + total + idx] = rec;
              }
            }
            break;
          }
          slot = (slot + 1) & tmask;
        }
      }
    } else {
      const uint32_t tag = uint32_t(h >> 32);
      const uint64_t mine = has_key ? ((uint64_t(tag) << 32) | (uint64_t(k) * R + uint64_t(lane))) : 0ull;
      bool active = has_key;
      long long probes = 0;
      while (__any_sync(0xffffffffu, active)) {
        bool cand = false;
        uint64_t old = 0;
        if (active) {
          old = atomicCAS(reinterpret_cast<unsigned long long*>(st.table + slot), (unsigned long long)kEmpty,
                          (unsigned long long)mine);
          if (old == kEmpty) {
            active = false;  // first arrival: the partner will pair with it
          } else if (uint32_t(old >> 32) == tag) {
            cand = true;
          } else {
            slot = (slot + 1) & tmask;
            if (++probes > tneed) { err_w |= kErrProbe; active = false; }
          }
        }
        unsigned cm = __ballot_sync(0xffffffffu, cand);
        while (cm) {
          const int L = __ffs(cm) - 1;
          cm &= cm - 1;
          const uint64_t pp = __shfl_sync(0xffffffffu, old, L) & 0x7fffffffull;
          const int wjL = __shfl_sync(0xffffffffu, wj, L);
          const uint64_t FwL = __shfl_sync(0xffffffffu, Fw, L);
          const bool eq = warp_face_matches(st, sm, G, chunk, (long long)(pp / R), int(pp % R), e, S, s0, wjL, FwL,
                                            nV, total, n);
          if (lane == L) {
            if (eq) {
              const uint64_t prev = atomicOr(reinterpret_cast<unsigned long long*>(st.table + slot),
                                             (unsigned long long)kPaired);
              if (prev & kPaired) {
                err_w |= kErrPairing;
              } else {
                const int v2 = int(nV + (long long)(pp / R));
                const int slot2 = atomicAdd(&sm.npairs, 1);
                if (slot2 < kPairCap) {
                  sm.pairs[slot2] = make_int4(v2, v0, 0, 0);
                } else {
                  const long long idx = atomic_add_ll(&cur->npairs, 1ll);
                  st.EU[nE + total + idx] = v2;
                  st.EW[nE + total + idx] = v0;
                }
              }
              active = false;
            } else {
              slot = (slot + 1) & tmask;
              if (++probes > tneed) { err_w |= kErrProbe; active = false; }
            }
          }
        }
      }
    }
    __syncwarp();
  }
  err_w = __reduce_or_sync(0xffffffffu, err_w);
  if (lane == 0) {
    if (nkeys_w) atomicAdd(reinterpret_cast<unsigned long long*>(&sm.acc[0]), (unsigned long long)nkeys_w);
    if (ndeg_w) atomicAdd(reinterpret_cast<unsigned long long*>(&sm.acc[1]), (unsigned long long)ndeg_w);
    if (err_w) atomicOr(&st.g->error, err_w);
  }
  __syncthreads();
  // this CTA's intersecting edges: one global allocation
  const int np = sm.npairs < kPairCap ? sm.npairs : kPairCap;
  if (threadIdx.x == 0) {
    sm.acc[2] = np ? atomic_add_ll(&cur->npairs, (long long)np) : 0;
    if (sm.acc[0]) atomic_add_ll(&cur->nkeys, sm.acc[0]);
    if (sm.acc[1]) atomic_add_ll(&cur->ndegenerate, sm.acc[1]);
  }
  __syncthreads();
  const long long base = nE + total + sm.acc[2];
  for (int t = threadIdx.x; t < np; t += kBlock) {
    const int4 rec = sm.pairs[t];
    st.EU[base + t] = rec.x;
    st.EW[base + t] = rec.y;
    if (st.deferred) st.vlist[base + t] = rec;
  }
  return false;
}

}  // namespace pc
