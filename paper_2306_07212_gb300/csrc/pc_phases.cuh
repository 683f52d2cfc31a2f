// The per-neuron steps of edge subdivision (Section 4.2) as device functions.
//
// One neuron step is three phases separated by grid-wide synchronisation
// (a kernel boundary in stepwise execution, a grid barrier in the persistent
// per-layer kernel):
//   phase_sign   step (2): the sign of every vertex w.r.t. the neuron's folded
//                hyperplane, from the stored pre-activation; in mixed precision
//                any |z| within its error bound is re-decided in FP64.
//   phase_edges  step (3): warp-ballot compaction of the splitting edges
//                (endpoint signs differ), order-preserving per CTA range.
//   phase_split  steps (4)+(5): one warp per splitting edge interpolates the
//                new vertex (FP64 t and coordinates, values in the Z type),
//                splits the edge, and inserts the edge's parent 2-face keys
//                into a hash table; the second arrival of a face emits the
//                intersecting edge.
#pragma once

#include "pc_device.cuh"
#include "pc_newton.cuh"

namespace pc {

struct Smem {
  long long pref[kMaxGrid + 1];
  long long wsum[kWarps + 1];
  long long flist[kFilterCap];
  uint64_t s0row[kWarps][kMaxWords];
  int zlist[kWarps][32];
  int fcount;
  int pad;
  int nzl[kMaxD + 2];
  NewtonOut nout;
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

// ---------------------------------------------------------------------------
// Step (2).  In mixed precision a |z| within kappa times the vertex's FP32
// error estimate is re-decided by newton_cta at the exact vertex (FP64); the
// CTA that owns the vertex does it, all threads cooperating.
template <typename ZT, bool MIXED>
__device__ void phase_sign(const NetDesc& net, const State& st, int zb, int l, int i, int n,
                           Smem& sm, double* ws, int mw) {
  const Counters* prev = st.cnt + n;
  const long long nV = prev->nV_before + prev->nsplit;
  const long long nE = prev->nE_before + prev->nsplit + prev->npairs;
  Counters* cur = st.cnt + n + 1;
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
  if (threadIdx.x == 0) sm.fcount = 0;
  __syncthreads();
  long long ndeg = 0;
  int und = 0;
  auto drain = [&]() {
    const int fc = sm.fcount;
    for (int q = 0; q < fc; ++q) {
      const long long v = sm.flist[q];
      newton_cta(net, st, v, e, l, i, mw, ws, sm.nzl, &sm.nout);
      if (threadIdx.x == 0) {
        const double zs = sm.nout.z;
        if (fabs(zs) <= 1e-12 * sm.nout.scale || !sm.nout.ok) ++und;
        const uint64_t code = zs < 0.0 ? kMinus : kPlus;
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
  for (long long base = (long long)blockIdx.x * kBlock; base < nV; base += (long long)gridDim.x * kBlock) {
    const long long v = base + threadIdx.x;
    if (v < nV) {
      const ZT z = zrow[v];
      bool filt = false;
      if (MIXED) filt = fabsf(static_cast<float>(z)) <= net.kappa * st.esc[v];
      if (filt) {
        const int slot = atomicAdd(&sm.fcount, 1);
        sm.flist[slot] = v;
      } else {
        const uint64_t code = (z < ZT(0)) ? kMinus : kPlus;
        ndeg += (z == ZT(0));
        sw[v] = (sw[v] & ~(3ull << sh)) | (code << sh);
      }
    }
    __syncthreads();
    if (sm.fcount > kFilterCap - kBlock) drain();
  }
  if (MIXED) drain();
  ndeg = warp_sum_ll(ndeg);
  if (lane == 0 && ndeg) atomic_add_ll(&cur->ndegenerate, ndeg);
  if (MIXED && threadIdx.x == 0 && und) atomic_add_ll(&cur->nundecided, (long long)und);
}

// ---------------------------------------------------------------------------
// Step (3).
__device__ __forceinline__ void phase_edges(const NetDesc& net, const State& st, int n, Smem& sm) {
  const Counters* cur = st.cnt + n + 1;
  const long long nE = cur->nE_before;
  // clear the part of the hash table that the previous neuron used
  const long long tprev = st.cnt[n].tsize;
  for (long long t = (long long)blockIdx.x * kBlock + threadIdx.x; t < tprev; t += (long long)gridDim.x * kBlock)
    st.table[t] = kEmpty;
  const long long G = gridDim.x;
  const long long chunk = (nE + G - 1) / G;
  const long long begin = blockIdx.x * chunk;
  const long long end = begin + chunk < nE ? begin + chunk : nE;
  const int e = net.m + n, sh = 2 * (e & 31);
  const uint64_t* sw = st.SIG + (long long)(e >> 5) * st.Vcap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long count = 0;
  for (long long base = begin; base < end; base += kBlock) {
    const long long idx = base + threadIdx.x;
    bool split = false;
    if (idx < end) {
      const int32_t u = st.EU[idx], w = st.EW[idx];
      split = ((sw[u] >> sh) & 3ull) != ((sw[w] >> sh) & 3ull);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, split);
    if (lane == 0) sm.wsum[warp] = __popc(mask);
    __syncthreads();
    if (warp == 0) {
      const long long c = lane < kWarps ? sm.wsum[lane] : 0;
      long long x = c;
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane < kWarps) sm.wsum[lane] = x - c;
      if (lane == kWarps - 1) sm.wsum[kWarps] = x;
    }
    __syncthreads();
    if (split) st.stage[begin + count + sm.wsum[warp] + __popc(mask & ((1u << lane) - 1u))] = int32_t(idx);
    count += sm.wsum[kWarps];
    __syncthreads();
  }
  if (threadIdx.x == 0) st.cta_count[blockIdx.x] = count;
}

// ---------------------------------------------------------------------------
// Steps (4)+(5).  Returns true when capacity ran out (nothing written).
template <typename ZT, bool MIXED>
__device__ bool phase_split(const NetDesc& net, const State& st, int zb, int l, int i, int n, Smem& sm) {
  constexpr bool TRACK = sizeof(ZT) == 4;  // FP32 values carry error estimates
  Counters* cur = st.cnt + n + 1;
  const long long nV = cur->nV_before, nE = cur->nE_before;
  const int G = gridDim.x;
  for (int q = threadIdx.x; q < G; q += kBlock) sm.pref[q] = st.cta_count[q];
  __syncthreads();
  block_scan_pref(sm, G);
  const long long total = sm.pref[G];
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
  const long long chunk = (nE + G - 1) / G;
  const int H = net.w[l + 1];
  ZT* Z = static_cast<ZT*>(st.Z[zb]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = m + n, wn = e >> 5, sh = 2 * (e & 31);
  uint64_t* s0row = sm.s0row[warp];
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
    const int32_t ed = st.stage[lo * chunk + (k - sm.pref[lo])];
    const int32_t u = st.EU[ed], w = st.EW[ed];
    const bool u_plus = ((st.SIG[(long long)wn * Vcap + u] >> sh) & 3ull) == kPlus;
    const int32_t p = u_plus ? u : w;   // V+
    const int32_t q = u_plus ? w : u;   // V-
    const double a = static_cast<double>(Z[(long long)i * Vcap + p]);
    const double b = static_cast<double>(Z[(long long)i * Vcap + q]);
    double t = a / (a - b);
    bool bad = !(a > 0.0 && b < 0.0);
    if (!(t >= 0.0 && t <= 1.0)) { t = t < 0.0 ? 0.0 : 1.0; bad = true; }
    const int32_t v0 = int32_t(nV + k);
    if (lane < D) {
      const double xp = st.X[(long long)lane * Vcap + p], xq = st.X[(long long)lane * Vcap + q];
      st.X[(long long)lane * Vcap + v0] = fma(t, xq - xp, xp);
    }
    const ZT tz = static_cast<ZT>(t);
    float amax = 0.f;
    for (int j = lane; j < H; j += 32) {
      const ZT zp = Z[(long long)j * Vcap + p], zq = Z[(long long)j * Vcap + q];
      Z[(long long)j * Vcap + v0] = (j == i) ? ZT(0) : zp + tz * (zq - zp);
      if (TRACK) amax = fmaxf(amax, fabsf(static_cast<float>(zp)) + fabsf(static_cast<float>(zq)));
    }
    if (TRACK) {
      // error estimates: values (rounding of the interpolation) and position
      // (a t computed from values carrying the endpoints' estimates)
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      float dx = 0.f;
      if (lane < D) dx = fabsf(static_cast<float>(st.X[(long long)lane * Vcap + q] - st.X[(long long)lane * Vcap + p]));
      for (int o = 16; o > 0; o >>= 1) dx = fmaxf(dx, __shfl_xor_sync(0xffffffffu, dx, o));
      if (lane == 0) {
        const float ep = st.esc[p], eq = st.esc[q];
        st.esc[v0] = fmaxf(ep, eq) + 2.4e-7f * amax;  // 4 * 2^-24
        st.exc[v0] = fmaxf(st.exc[p], st.exc[q]) + static_cast<float>((ep + eq) / (a - b)) * dx;
      }
    }
    // sign vector of the new vertex: join of the endpoints, entry n := 0
    uint64_t s0 = 0, zm = 0;
    if (lane < S) {
      const uint64_t sp = st.SIG[(long long)lane * Vcap + p], sq = st.SIG[(long long)lane * Vcap + q];
      uint64_t conf = ((sp & kEvenBits) & ((sq >> 1) & kEvenBits)) | ((sq & kEvenBits) & ((sp >> 1) & kEvenBits));
      s0 = sp | sq;
      if (lane == wn) {
        conf &= ~(1ull << sh);
        s0 &= ~(3ull << sh);
      }
      if (conf) err_w |= kErrConflict;
      st.SIG[(long long)lane * Vcap + v0] = s0;
      s0row[lane] = s0;
      zm = zero_mask(s0, lane, e);
    }
    if (lane == 0) {
      st.EU[ed] = p;
      st.EW[ed] = v0;
      st.EU[nE + k] = q;
      st.EW[nE + k] = v0;
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
    // this lane's key: ordinal o = lane / 2 of the zeros, sign + (even) or - (odd)
    const int o = lane >> 1;
    const bool minus = lane & 1;
    const int jz = (nz == D - 1 && o < nz) ? zlist[o] : 0;
    const int wj = jz >> 5, shj = 2 * (jz & 31);
    const uint64_t s0w = __shfl_sync(0xffffffffu, s0, wj);
    const bool has_key = (nz == D - 1) && (o < nz) && !(minus && jz < m);
    const int nk = __popc(__ballot_sync(0xffffffffu, has_key));
    nkeys_w += nk;
    if (bad) ndeg_w += 1;
    __threadfence();  // publish the new vertex before its keys
    if (has_key) {
      const uint64_t Fw = (s0w & ~(3ull << shj)) | ((minus ? kMinus : kPlus) << shj);
      const uint64_t h = hb ^ word_hash(wj, s0w) ^ word_hash(wj, Fw);
      const uint32_t tag = uint32_t(h >> 32);
      const uint64_t payload = uint64_t(k) * R + uint64_t(lane);
      const uint64_t mine = (uint64_t(tag) << 32) | payload;
      long long slot = (long long)(h & (uint64_t)tmask);
      bool done = false;
      for (long long probe = 0; probe < tneed; ++probe) {
        const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(st.table + slot),
                                       (unsigned long long)kEmpty, (unsigned long long)mine);
        if (old == kEmpty) { done = true; break; }
        if (uint32_t(old >> 32) == tag) {
          __threadfence();
          const uint64_t pp = old & 0x7fffffffull;
          const long long k2 = (long long)(pp / R);
          const int r2 = int(pp % R);
          const long long v2 = nV + k2;
          // reconstruct the partner's face and compare word by word
          const int o2 = r2 >> 1;
          const bool minus2 = r2 & 1;
          int seen = 0, j2 = -1;
          bool equal = true;
          uint64_t s2[kMaxWords];
          for (int ww = 0; ww < S; ++ww) {
            s2[ww] = __ldcg(st.SIG + (long long)ww * Vcap + v2);
            uint64_t z2 = zero_mask(s2[ww], ww, e);
            while (z2 && j2 < 0) {
              const int bit = __ffsll((long long)z2) - 1;
              if (seen == o2) j2 = ww * 32 + bit / 2;
              ++seen;
              z2 &= z2 - 1;
            }
          }
          if (j2 < 0) equal = false;
          for (int ww = 0; ww < S && equal; ++ww) {
            uint64_t f1 = s0row[ww];
            if (ww == wj) f1 = Fw;
            uint64_t f2 = s2[ww];
            if (ww == (j2 >> 5)) f2 = (f2 & ~(3ull << (2 * (j2 & 31)))) | ((minus2 ? kMinus : kPlus) << (2 * (j2 & 31)));
            equal = (f1 == f2);
          }
          if (equal) {
            if (old & kPaired) { err_w |= kErrPairing; done = true; break; }
            const uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long*>(st.table + slot),
                                            (unsigned long long)old, (unsigned long long)(old | kPaired));
            if (prev != old) { err_w |= kErrPairing; done = true; break; }
            const long long idx = atomic_add_ll(&cur->npairs, 1ll);
            const long long eo = nE + total + idx;
            st.EU[eo] = int32_t(v2);
            st.EW[eo] = v0;
            done = true;
            break;
          }
        }
        slot = (slot + 1) & tmask;
      }
      if (!done) err_w |= kErrProbe;
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (nkeys_w) atomic_add_ll(&cur->nkeys, nkeys_w);
    if (ndeg_w) atomic_add_ll(&cur->ndegenerate, ndeg_w);
  }
  err_w = __reduce_or_sync(0xffffffffu, err_w);
  if (lane == 0 && err_w) atomicOr(&st.g->error, err_w);
  return false;
}

}  // namespace pc
