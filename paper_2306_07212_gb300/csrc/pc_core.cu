// libpc core: device state management, the set-up kernels, the SIMT
// layer-start product (step (1) of Section 4.2; the tensor-core form is in
// pc_gemm_tc.cu), the per-neuron phase kernels in both execution modes, the
// exact check of fingerprint pairings, the coordinate polish, and the C ABI
// declared in include/pc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pc.h"
#include "pc_ctx.h"
#include "pc_phases.cuh"

namespace pc {

// ---------------------------------------------------------------------------
// Set-up kernels

// The (head, remainder) pairs follow the float32 heads at an even float
// offset, so that every pair is 8-byte aligned.
__host__ __device__ inline long long pairs_offset(long long n_params) { return (n_params + 1) & ~1ll; }

// float32 copy of the parameters, and the norms used by the FP32 error
// estimate: per layer max_j ||W_j||_2 and max_j |b_j|, per neuron ||W_n||_2,
// |b_n| and 1/||W_n||_2 (rounded outward).
__global__ void k_prep(NetDesc net, float* W32, float* norms, long long n_params) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_params;
       t += (long long)gridDim.x * blockDim.x)
  {
    const double w = net.W64[t];
    const float h = static_cast<float>(w);
    W32[t] = h;
    // (head, remainder) pair, weights transposed to [K][H] within their layer
    int l = 0;
    while (l + 1 < net.L && t >= net.wofs[l + 1]) ++l;
    long long dst = t;
    if (t < net.bofs[l]) {
      const long long e = t - net.wofs[l];
      const int K = net.w[l], H = net.w[l + 1];
      dst = net.wofs[l] + (e % K) * H + e / K;
    }
    reinterpret_cast<float2*>(W32 + pairs_offset(n_params))[dst] =
        make_float2(h, static_cast<float>(w - static_cast<double>(h)));
  }
  if (blockIdx.x < net.L) {
    const int l = blockIdx.x, H = net.w[l + 1], K = net.w[l];
    __shared__ double s_w[256], s_b[256];
    double mw = 0.0, mb = 0.0;
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) {
        const double w = net.W64[net.wofs[l] + (long long)j * K + k];
        s += w * w;
      }
      const double bj = fabs(net.W64[net.bofs[l] + j]);
      mw = fmax(mw, sqrt(s));
      mb = fmax(mb, bj);
      float* nr = norms + 2 * kMaxL + 3 * (net.off[l] + j);
      nr[0] = __double2float_ru(sqrt(s) * (1.0 + 1e-6));
      nr[1] = __double2float_ru(bj);
      nr[2] = s > 0.0 ? __double2float_rd(1.0 / (sqrt(s) * (1.0 + 1e-6))) : 0.f;
    }
    s_w[threadIdx.x] = mw;
    s_b[threadIdx.x] = mb;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < blockDim.x; ++q) {
        mw = fmax(mw, s_w[q]);
        mb = fmax(mb, s_b[q]);
      }
      norms[2 * l] = __double2float_ru(mw * (1.0 + 1e-6));
      norms[2 * l + 1] = __double2float_ru(mb);
    }
  }
}

// Step 0: the box's 2^D corners and D 2^(D-1) edges; boundary entries first
// (entry 2d: x_d - lo_d, 2d+1: hi_d - x_d), every neuron entry unprocessed.
__global__ void k_init(NetDesc net, State st) {
  const int D = net.D, nc = 1 << D, ne0 = D << (D - 1);
  const long long Vcap = st.Vcap;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    uint64_t w0 = 0;
    for (int d = 0; d < D; ++d) {
      const bool up = (c >> d) & 1;
      st.X[(long long)d * Vcap + c] = up ? net.hi[d] : net.lo[d];
      if (up) w0 |= kPlus << (2 * (2 * d));
      else w0 |= kPlus << (2 * (2 * d + 1));
    }
    st.SIG[c] = w0;
    for (int w = 1; w < net.S; ++w) st.SIG[(long long)w * Vcap + c] = 0;
    if (st.exc) st.exc[c] = 0.f;
  }
  for (int e = threadIdx.x; e < ne0; e += blockDim.x) {
    const int d = e >> (D - 1), r = e & ((1 << (D - 1)) - 1);
    const int c = ((r >> d) << (d + 1)) | (r & ((1 << d) - 1));
    st.EU[e] = c;
    st.EW[e] = c | (1 << d);
    if (st.deferred) st.vlist[e] = make_int4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    Counters c0{};
    c0.nV_before = nc;
    c0.nE_before = ne0;
    st.cnt[0] = c0;
    Global g{};
    g.halted_at = -1;
    g.barrier_extra = net.debug_barrier ? 1u : 0u;
    *st.g = g;
  }
}

// Step 0 on a polyhedral domain {x : c - A x >= 0} (Section 4.1, bounded
// domains): the caller's 1-skeleton, vertices X0 (row-major nv0 x D) and
// edges E0 (ne0 pairs of vertex indices), checked on the host before the
// launch.  Facet entry i of a vertex is 0 when |c_i - A_i x| <= 1e-12 of
// |c_i| + sum_d |A_id x_d| (the vertex lies on the facet), else +; every
// neuron entry is unprocessed.
__global__ void k_init_domain(NetDesc net, State st, const double* X0, const int32_t* E0, long long nv0,
                              long long ne0) {
  const int D = net.D, m = net.m;
  const long long Vcap = st.Vcap;
  for (long long v = threadIdx.x; v < nv0; v += blockDim.x) {
    const double* x = X0 + v * D;
    for (int d = 0; d < D; ++d) st.X[(long long)d * Vcap + v] = x[d];
    for (int w = 0; w < net.S; ++w) {
      uint64_t word = 0;
      for (int k = 0; k < 32 && 32 * w + k < m; ++k) {
        const int i = 32 * w + k;
        double f = net.fc[i], s = fabs(net.fc[i]);
        for (int d = 0; d < D; ++d) {
          const double t = net.fA[(long long)i * D + d] * x[d];
          f -= t;
          s += fabs(t);
        }
        if (fabs(f) > 1e-12 * s) word |= kPlus << (2 * k);
      }
      st.SIG[(long long)w * Vcap + v] = word;
    }
    if (st.exc) st.exc[v] = 0.f;
  }
  for (long long e = threadIdx.x; e < ne0; e += blockDim.x) {
    st.EU[e] = E0[2 * e];
    st.EW[e] = E0[2 * e + 1];
    if (st.deferred) st.vlist[e] = make_int4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    Counters c0{};
    c0.nV_before = nv0;
    c0.nE_before = ne0;
    st.cnt[0] = c0;
    Global g{};
    g.halted_at = -1;
    g.barrier_extra = net.debug_barrier ? 1u : 0u;
    *st.g = g;
  }
}

// ---------------------------------------------------------------------------
// Step (1) at the start of layer l: Z_l = W_l a + b_l for every vertex, with
// a = x (l = 0) or a_k = z_k of layer l-1 if the vertex's entry is + else 0.
// SIMT version: one thread per vertex and 16 output neurons per block row.
//
// FP32 error estimate (root mean square, FP32 and mixed precision): a K-term
// FP32 dot product accumulated in order has an rms rounding error of about
// u/2 * S with S = sum_k |W_jk a_k| + |b_j| and u = 2^-24 (the running sums
// are a random walk); S <= ||W_j||_2 ||a||_2 + |b_j|.  Errors already in a
// propagate with ||W_j||_2.  Both factor as ||W_j||_2 rho(v) + u/2 |b_j|, so
// one scale rho per vertex serves every neuron of the layer.  Layer 0 is
// evaluated in float64 and rounded once.
template <typename ZT, bool MIXED>
__global__ void __launch_bounds__(128) k_gemm_simt(NetDesc net, State st, int l) {
  constexpr int TJ = 16;
  constexpr bool TRACK = sizeof(ZT) == 4;
  if (cta_stopped(st)) return;
  const Counters* c = st.cnt + net.off[l];
  const long long nV = c->nV_before + c->nsplit;
  if (nV < 0 || nV > st.Vcap) {
    if (threadIdx.x == 0) report_corrupt(st.g, 1, l, nV, st.Vcap, 0);
    return;
  }
  const int H = net.w[l + 1], K = net.w[l];
  const int j0 = blockIdx.y * TJ;
  __shared__ ZT Ws[TJ][kMaxWidth + 1];
  __shared__ double Wd[TJ][kMaxD];
  __shared__ ZT bs[TJ];
  __shared__ double bd[TJ];
  for (int t = threadIdx.x; t < TJ * K; t += blockDim.x) {
    const int jj = t / K, kk = t % K, j = j0 + jj;
    const double wv = j < H ? net.W64[net.wofs[l] + (long long)j * K + kk] : 0.0;
    Ws[jj][kk] = static_cast<ZT>(wv);
    if (kk < kMaxD) Wd[jj][kk] = wv;
  }
  if (threadIdx.x < TJ) {
    const int j = j0 + threadIdx.x;
    const double bv = j < H ? net.W64[net.bofs[l] + j] : 0.0;
    bs[threadIdx.x] = static_cast<ZT>(bv);
    bd[threadIdx.x] = bv;
  }
  __syncthreads();
  const long long Vcap = st.Vcap;
  ZT* Zout = static_cast<ZT*>(st.Z[l]);
  const ZT* Zin = static_cast<const ZT*>(st.Z[l > 0 ? l - 1 : 0]);
  const int ebase = net.m + (l > 0 ? net.off[l - 1] : 0);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nV;
       v += (long long)gridDim.x * blockDim.x) {
    ZT acc[TJ];
    float a2 = 0.f;
    if (l == 0) {
      double dacc[TJ];
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) dacc[jj] = bd[jj];
      for (int d = 0; d < K; ++d) {
        const double x = st.X[(long long)d * Vcap + v];
        a2 += static_cast<float>(x * x);
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj) dacc[jj] = fma(Wd[jj][d], x, dacc[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) acc[jj] = static_cast<ZT>(dacc[jj]);
    } else {
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) acc[jj] = bs[jj];
      uint64_t word = 0;
      int cw = -1;
      for (int kk = 0; kk < K; ++kk) {
        const int entry = ebase + kk, wi = entry >> 5;
        if (wi != cw) {
          word = st.SIG[(long long)wi * Vcap + v];
          cw = wi;
        }
        const bool act = ((word >> (2 * (entry & 31))) & 3ull) == kPlus;
        const ZT a = act ? Zin[(long long)kk * Vcap + v] : ZT(0);
        a2 = fmaf(static_cast<float>(a), static_cast<float>(a), a2);
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj) acc[jj] = fma(Ws[jj][kk], a, acc[jj]);
      }
    }
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj)
      if (j0 + jj < H) Zout[(long long)(j0 + jj) * Vcap + v] = acc[jj];
    if (TRACK && blockIdx.y == 0) {
      // rho_l: u/2 ||a||_2 (rounding: the running sums are bounded by
      // ||W_j||_2 ||a||_2) and the largest input error of the previous layer
      const float u = 5.9604645e-8f;  // 2^-24
      float rho = 0.5f * u * sqrtf(a2);
      if (l > 0) {  // independent of the rounding: add in quadrature
        const float inh = net.norms[2 * (l - 1)] * st.esc[v] + 0.5f * u * net.norms[2 * (l - 1) + 1];
        rho = sqrtf(rho * rho + inh * inh);
      }
      st.esc[v] = rho;
    }
  }
}

// ---------------------------------------------------------------------------
// Neuron phases: stepwise kernels and the persistent per-layer kernel.

template <typename ZT, bool MIXED>
__global__ void __launch_bounds__(kBlock, 2) k_decide(NetDesc net, State st, int l, int mw) {
  extern __shared__ double dsm[];
  __shared__ Smem sm;
  if (cta_stopped(st)) return;
  phase_decide<ZT, MIXED>(net, st, l, sm, dsm, mw);
}

template <typename ZT>
__global__ void __launch_bounds__(kBlock) k_scan0(NetDesc net, State st, int l) {
  __shared__ Smem sm;
  if (cta_stopped(st)) return;
  phase_scan0<ZT>(net, st, l, sm);
}

template <typename ZT, bool MIXED>
__global__ void __launch_bounds__(kBlock, 2) k_step(NetDesc net, State st, int l, int i, int mw) {
  extern __shared__ double dsm[];
  __shared__ Smem sm;
  if (cta_stopped(st)) return;
  if (threadIdx.x == 0) sm.nrl_layer = -1;
  __syncthreads();
  phase_step<ZT, MIXED>(net, st, l, i, sm, dsm, mw);
}

template <typename ZT>
__global__ void __launch_bounds__(kBlock) k_pack(NetDesc net, State st, int l) {
  if (cta_stopped(st)) return;
  phase_pack<ZT>(net, st, l);
}

// The neuron loop of layer l in one cooperative launch: the layer-start
// decisions and first edge scan (prologue = 1; a launch that resumes after a
// capacity halt skips them), one grid barrier per neuron step, and the
// packing of the layer's sign codes.
template <typename ZT, bool MIXED>
__global__ void __launch_bounds__(kBlock, 2) k_layer(NetDesc net, State st, int l, int i_begin, int prologue,
                                                     int mw) {
  extern __shared__ double dsm[];
  __shared__ Smem sm;
  if (cta_stopped(st)) return;
  unsigned int passed = 0;
  const int H = net.w[l + 1];
  if (threadIdx.x == 0) sm.nrl_layer = -1;
  __syncthreads();
  if (prologue) {
    phase_decide<ZT, MIXED>(net, st, l, sm, dsm, mw);
    if (!grid_barrier(st.g, passed)) return;  // uniform per CTA
    if (cta_stopped(st)) return;
    phase_scan0<ZT>(net, st, l, sm);
    if (!grid_barrier(st.g, passed)) return;
    if (cta_stopped(st)) return;
  }
  for (int i = i_begin; i < H; ++i) {
    if (phase_step<ZT, MIXED>(net, st, l, i, sm, dsm, mw)) return;
    if (!grid_barrier(st.g, passed)) return;
    if (cta_stopped(st)) return;
  }
  phase_pack<ZT>(net, st, l);
}

// Exact check of every pairing made by fingerprint (deferred mode), after
// the last step: the two new vertices' sign vectors, restricted to the
// entries before the step's neuron, with the keyed zero set to its sign,
// must be equal (the 2-face of Section 4.2, step 5).  Sign entries below a
// step's neuron never change after the step, so the check can run at the
// end.  One thread per edge; non-pairing edges carry a zero record.
__device__ __forceinline__ void set_keyed_zero(uint64_t& f, uint64_t zm, int& remaining, bool minus) {
  if (remaining < 0) return;
  const int c = __popcll(zm);
  if (remaining >= c) {
    remaining -= c;
    return;
  }
  for (int q = 0; q < remaining; ++q) zm &= zm - 1;
  const int bit = __ffsll((long long)zm) - 1;
  f = (f & ~(3ull << bit)) | ((minus ? kMinus : kPlus) << bit);
  remaining = -1;
}

__global__ void __launch_bounds__(256) k_verify_pairs(NetDesc net, State st) {
  if (cta_stopped(st)) return;
  const Counters* last = st.cnt + net.N;
  const long long nE = last->nE_before + last->nsplit + last->npairs;
  const long long nV = last->nV_before + last->nsplit;
  if (nE < 0 || nE > st.Ecap || nV < 0 || nV > st.Vcap) {
    if (threadIdx.x == 0) report_corrupt(st.g, 9, net.N, nV, nE, 0);
    return;
  }
  const long long Vcap = st.Vcap;
  const int S = net.S, m = net.m;
  int bad = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (long long)gridDim.x * blockDim.x) {
    const int4 r = st.vlist[e];
    if (r.w == 0) continue;
    const int n = r.w - 1;
    if (n < 0 || n >= net.N || r.x < 0 || r.x >= nV || r.y < 0 || r.y >= nV) {
      bad = 1;
      continue;
    }
    const int ent = m + n, ka = r.z >> 16, kb = r.z & 0xffff;
    int oa = ka >> 1, ob = kb >> 1;
    bool same = true;
    for (int w = 0; w < S && 32 * w < ent; ++w) {
      uint64_t fa = st.SIG[(long long)w * Vcap + r.x], fb = st.SIG[(long long)w * Vcap + r.y];
      set_keyed_zero(fa, zero_mask(fa, w, ent), oa, ka & 1);
      set_keyed_zero(fb, zero_mask(fb, w, ent), ob, kb & 1);
      const int cnt = ent - 32 * w;
      const uint64_t valid = cnt >= 32 ? ~0ull : ((1ull << (2 * cnt)) - 1);
      if ((fa ^ fb) & valid) same = false;
    }
    if (!same || oa >= 0 || ob >= 0) bad = 1;  // a keyed zero that does not exist also fails
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st.g->error, kErrVerify);
}

// Coordinate polish: every vertex whose coordinate error estimate (rms)
// exceeds thr is moved to its exact position by a Newton step on its D zero
// entries (all entries are processed at this point), with the values in
// float-float arithmetic (newton_ff_warp).  One warp per vertex; vertices are
// dealt to warps round-robin.  n_stage: parameter pairs copied to shared
// memory (all of them, or 0 when they do not fit; then they are read from
// global memory, coalesced per layer).
template <bool DOMAIN>
__global__ void __launch_bounds__(kBlock) k_polish(NetDesc net, State st, float thr, int mw, long long n_stage) {
  // blockDim.x = 32 x (warps whose workspace fits kPolishSmemMax)
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ int zl[kWarps][kMaxD + 2];
  __shared__ NewtonOut nout[kWarps];
  if (cta_stopped(st)) return;
  const Counters* last = st.cnt + net.N;
  const long long nV = last->nV_before + last->nsplit;
  const long long Vcap = st.Vcap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* Ps = reinterpret_cast<float2*>(psm);
  for (long long t = threadIdx.x; t < n_stage; t += blockDim.x) Ps[t] = net.WT2[t];
  __syncthreads();
  const float2* P = n_stage > 0 ? Ps : net.WT2;
  unsigned char* ws = psm + ((n_stage * 8 + 15) / 16) * 16 + (long long)warp * ff_ws_bytes(mw, net.D);
  long long npol = 0;
  const int wpc = blockDim.x >> 5;
  const long long nwarps = (long long)gridDim.x * wpc;
  for (long long base = ((long long)blockIdx.x * wpc + warp) * 32; base < nV; base += nwarps * 32) {
    const long long v = base + lane;
    unsigned flag = __ballot_sync(0xffffffffu, v < nV && !(st.exc[v] <= thr));
    while (flag) {
      const int L = __ffs(flag) - 1;
      flag &= flag - 1;
      const long long u = base + L;
      newton_ff_warp<DOMAIN>(net, st, P, u, net.P, mw, ws, zl[warp], &nout[warp]);
      if (nout[warp].ok) {
        if (lane < net.D) st.X[(long long)lane * Vcap + u] += nout[warp].dlt[lane];
        npol += (lane == 0);
      }
      __syncwarp();
    }
  }
  if (lane == 0 && npol) atomic_add_ll(&st.g->polished, npol);
}

}  // namespace pc

using namespace pc;

// ---------------------------------------------------------------------------
// Host side.

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void* ctx_alloc(pc_ctx* c, size_t bytes) {
  bytes = round_up(std::max<size_t>(bytes, 256), 256);
  if (c->opt.mem_budget_bytes > 0 && c->allocated + bytes > (size_t)c->opt.mem_budget_bytes) return nullptr;
  void* p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(bytes, c->stream, c->alloc_user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    c->allocated += bytes;
    c->sizes[p] = bytes;
  }
  return p;
}

void ctx_free(pc_ctx* c, void*& p) {
  if (!p) return;
  auto it = c->sizes.find(p);
  const size_t bytes = it != c->sizes.end() ? it->second : 0;
  if (it != c->sizes.end()) c->sizes.erase(it);
  c->allocated -= bytes;
  if (c->free_fn) c->free_fn(p, bytes, c->stream, c->alloc_user);
  else cudaFreeAsync(p, c->stream);
  p = nullptr;
}

#define PC_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      throw PcError(PC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                          \
  } while (0)

static size_t zsize_of(int prec) { return prec == PC_PREC_FP64 ? 8 : 4; }

// (Re)allocates the state for capacities (V, E, T, tape); copies live data.
// Rows come from the context's recorded buffer shape (set when the buffers
// are (re)shaped), which covers every network that runs without reshaping,
// not from the current network (a later, wider one would overrun them).
static void realloc_state(pc_ctx* c, long long V, long long E, long long T, bool copy) {
  // multiples of 64 entries: rows stay 256-byte aligned (vector loads of the
  // second endpoint row need EW = EU + Ecap on a 16-byte boundary)
  V = std::min<long long>((V + 63) & ~63ll, (1ll << 31) - 64);
  E = std::min<long long>((E + 63) & ~63ll, (1ll << 31) - 64);
  const int D = c->shape_D, S = c->shape_S, Hm = c->shape_H;
  const size_t zs = c->shape_zs;
  StateBufs nb;
  auto A = [&](void*& p, size_t bytes) {
    p = ctx_alloc(c, bytes);
    if (!p) {
      nb.release(c);  // nothing half-built survives; the live buffers are untouched
      throw PcError(PC_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
  };
  A(nb.X, sizeof(double) * D * V);
  nb.nz = c->shape_tape ? c->shape_nz : 2;
  for (int k = 0; k < nb.nz; ++k) A(nb.Z[k], zs * Hm * V);
  A(nb.esc, sizeof(float) * V);
  A(nb.exc, sizeof(float) * V);
  A(nb.SIG, sizeof(uint64_t) * S * V);
  A(nb.E, sizeof(int32_t) * 2 * E);
  A(nb.list0, sizeof(int4) * E);
  A(nb.list1, sizeof(int4) * E);
  A(nb.flags, sizeof(uint32_t) * 2 * (E / 32));
  A(nb.vlist, sizeof(int4) * E);
  A(nb.table, 32 * T);
  if (c->opt.keep_tape) {
    A(nb.tape_pq, sizeof(int32_t) * 2 * V);
    A(nb.tape_t, sizeof(double) * V);
  }
  PC_CUDA(cudaMemsetAsync(nb.table, 0xff, 32 * T, c->stream));
  PC_CUDA(cudaMemsetAsync(nb.flags, 0, sizeof(uint32_t) * 2 * (E / 32), c->stream));
  StateBufs& ob = c->bufs;
  if (copy && ob.X) {
    const long long oV = c->Vcap, oE = c->Ecap, nV = std::min(oV, V), nE = std::min(oE, E);
    auto cp2 = [&](void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows) {
      if (rows && width) PC_CUDA(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDeviceToDevice, c->stream));
    };
    cp2(nb.X, 8 * V, ob.X, 8 * oV, 8 * nV, D);
    for (int k = 0; k < nb.nz && k < ob.nz; ++k) cp2(nb.Z[k], zs * V, ob.Z[k], zs * oV, zs * nV, Hm);
    cp2(nb.esc, 4 * V, ob.esc, 4 * oV, 4 * nV, 1);
    cp2(nb.exc, 4 * V, ob.exc, 4 * oV, 4 * nV, 1);
    cp2(nb.SIG, 8 * V, ob.SIG, 8 * oV, 8 * nV, S);
    cp2(nb.E, 4 * E, ob.E, 4 * oE, 4 * nE, 2);
    cp2(nb.vlist, 16 * E, ob.vlist, 16 * oE, 16 * nE, 1);
    // the splitting edges (and their flags) of the step that resumes
    cp2(nb.list0, 16 * E, ob.list0, 16 * oE, 16 * nE, 1);
    cp2(nb.list1, 16 * E, ob.list1, 16 * oE, 16 * nE, 1);
    cp2(nb.flags, 4 * (E / 32), ob.flags, 4 * (oE / 32), 4 * (nE / 32), 2);
    if (c->opt.keep_tape && ob.tape_pq) {
      cp2(nb.tape_pq, 4 * V, ob.tape_pq, 4 * oV, 4 * nV, 2);
      cp2(nb.tape_t, 8 * V, ob.tape_t, 8 * oV, 8 * nV, 1);
    }
  }
  ob.release(c);
  c->bufs = nb;
  c->Vcap = V;
  c->Ecap = E;
  c->Tcap = T;
}

// Counters, status block and per-CTA counts.  A failed allocation leaves the
// context without these buffers (capacity 0), never with a stale capacity.
static void ensure_fixed(pc_ctx* c, int N) {
  const size_t cnt_bytes = sizeof(Counters) * (N + 1);
  if (c->cnt_slots < N + 1 || !c->cnt || !c->h_cnt) {
    c->cnt_slots = 0;
    ctx_free(c, c->cnt);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    c->h_cnt = nullptr;
    c->cnt = ctx_alloc(c, cnt_bytes);
    if (!c->cnt) throw PcError(PC_ERR_OOM, "counter allocation failed");
    if (cudaMallocHost(&c->h_cnt, cnt_bytes) != cudaSuccess) {
      cudaGetLastError();
      c->h_cnt = nullptr;
      throw PcError(PC_ERR_OOM, "pinned counter allocation failed");
    }
    c->cnt_slots = N + 1;
  }
  if (!c->g || !c->h_g) {
    ctx_free(c, c->g);
    c->g = ctx_alloc(c, sizeof(Global));
    if (!c->g) throw PcError(PC_ERR_OOM, "status allocation failed");
    if (!c->h_g && cudaMallocHost(&c->h_g, sizeof(Global)) != cudaSuccess) {
      cudaGetLastError();
      c->h_g = nullptr;
      ctx_free(c, c->g);
      throw PcError(PC_ERR_OOM, "pinned status allocation failed");
    }
  }
}

static State make_state(pc_ctx* c);
State pc_make_state(pc_ctx* c) { return make_state(c); }

static State make_state(pc_ctx* c) {
  State s{};
  s.Vcap = c->Vcap;
  s.Ecap = c->Ecap;
  s.Tcap = c->Tcap;
  s.X = static_cast<double*>(c->bufs.X);
  for (int l = 0; l < kMaxL; ++l) s.Z[l] = c->bufs.Z[c->bufs.nz > 2 ? (l < c->bufs.nz ? l : 0) : (l & 1)];
  s.esc = static_cast<float*>(c->bufs.esc);
  s.exc = static_cast<float*>(c->bufs.exc);
  s.SIG = static_cast<uint64_t*>(c->bufs.SIG);
  s.EU = static_cast<int32_t*>(c->bufs.E);
  s.EW = s.EU + c->Ecap;
  s.list[0] = static_cast<int4*>(c->bufs.list0);
  s.list[1] = static_cast<int4*>(c->bufs.list1);
  s.flags[0] = static_cast<uint32_t*>(c->bufs.flags);
  s.flags[1] = s.flags[0] + (c->Ecap + 31) / 32;
  s.table = static_cast<uint64_t*>(c->bufs.table);
  s.vlist = static_cast<int4*>(c->bufs.vlist);
  s.deferred = c->deferred;
  s.cnt = static_cast<Counters*>(c->cnt);
  s.g = static_cast<Global*>(c->g);
  s.tape_pq = static_cast<int32_t*>(c->bufs.tape_pq);
  s.tape_t = static_cast<double*>(c->bufs.tape_t);
  s.tape_cap = c->opt.keep_tape ? c->Vcap : 0;
  s.keep_tape = c->opt.keep_tape;
  return s;
}

// CUDA events around the kernels of one layer (index 2l: forward product,
// 2l+1: neuron loop), recorded on the extraction's stream when timers are on.
struct TimerScope {
  pc_ctx* c;
  int slot;
  TimerScope(pc_ctx* c_, int s) : c(c_), slot(s) {
    if (c->opt.timers && slot <= pc_ctx::kPolishSlot) {
      if (!c->ev[slot][0]) {
        cudaEventCreate(&c->ev[slot][0]);
        cudaEventCreate(&c->ev[slot][1]);
      }
      cudaEventRecord(c->ev[slot][0], c->stream);
    }
  }
  ~TimerScope() {
    if (c->opt.timers && slot <= pc_ctx::kPolishSlot) {
      cudaEventRecord(c->ev[slot][1], c->stream);
      c->ev_used[slot] = 1;
    }
  }
};

template <typename ZT, bool MIXED>
struct Kernels {
  static void gemm(pc_ctx* c, const State& st, int l) {
    TimerScope ts(c, 2 * l);
    if (sizeof(ZT) == 4 && c->opt.gemm != PC_GEMM_SIMT && pc_gemm_tc_eligible(c->net, l)) {
      const int pieces = c->opt.gemm == PC_GEMM_TENSOR_3XTF32 ? 2 : 3;
      PC_CUDA(pc_gemm_tc_launch(c->net, st, l, (c->Vcap + 127) / 128, c->num_sms, pieces, c->stream));
      c->launches += 1;
      return;
    }
    const int H = c->net.w[l + 1];
    dim3 grid(std::max(1, std::min<int>(c->num_sms * 8, int((c->Vcap + 127) / 128))), (H + 15) / 16);
    k_gemm_simt<ZT, MIXED><<<grid, 128, 0, c->stream>>>(c->net, st, l);
    PC_CUDA(cudaGetLastError());
    c->launches += 1;
  }
  // The neuron loop of layer l from neuron i_begin; prologue: the layer's
  // start (decisions, first edge scan) has not run yet.
  static void layer(pc_ctx* c, const State& st, int l, int i_begin, bool prologue) {
    TimerScope ts(c, 2 * l + 1);
    const int H = c->net.w[l + 1];
    if (c->opt.exec == PC_EXEC_PERSISTENT) {
      PC_CUDA(cudaMemsetAsync(&static_cast<Global*>(c->g)->barrier, 0, sizeof(unsigned int), c->stream));
      auto fn = k_layer<ZT, MIXED>;
      NetDesc net = c->net;
      State s = st;
      int l_ = l, ib = i_begin, pro = prologue ? 1 : 0, mw = c->mw;
      void* args[] = {&net, &s, &l_, &ib, &pro, &mw};
      PC_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(c->grid_persist), dim3(kBlock), args,
                                          c->res_smem, c->stream));
      c->launches += 1;
    } else {
      // grids sized to the edge capacity (2048 edges per CTA of a scan
      // iteration), so that the small extractions of concurrent requests
      // share the GPU; every phase is written for any grid size
      const int gs = int(std::max<long long>(8, std::min<long long>(c->grid_step, c->Ecap / 2048)));
      if (prologue) {
        k_decide<ZT, MIXED><<<gs, kBlock, c->res_smem, c->stream>>>(c->net, st, l, c->mw);
        PC_CUDA(cudaGetLastError());
        k_scan0<ZT><<<gs, kBlock, 0, c->stream>>>(c->net, st, l);
        PC_CUDA(cudaGetLastError());
        c->launches += 2;
      }
      for (int i = i_begin; i < H; ++i) {
        k_step<ZT, MIXED><<<gs, kBlock, c->res_smem, c->stream>>>(c->net, st, l, i, c->mw);
        PC_CUDA(cudaGetLastError());
        c->launches += 1;
      }
      k_pack<ZT><<<gs, kBlock, 0, c->stream>>>(c->net, st, l);
      PC_CUDA(cudaGetLastError());
      c->launches += 1;
    }
  }
  static int occupancy(pc_ctx* c) {
    int nb = 0;
    PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_layer<ZT, MIXED>, kBlock, c->res_smem));
    return nb;
  }
};

template <typename ZT, bool MIXED>
static void enqueue(pc_ctx* c, int l0, int i0, bool gemm_done) {
  const State st = make_state(c);
  for (int l = l0; l < c->net.L; ++l) {
    if (!(l == l0 && gemm_done)) Kernels<ZT, MIXED>::gemm(c, st, l);
    Kernels<ZT, MIXED>::layer(c, st, l, l == l0 ? i0 : 0, !(l == l0 && gemm_done));
    if (c->opt.prune && l + 1 < c->net.L) pc_prune_edges(c, st, l);
  }
}

static void enqueue_any(pc_ctx* c, int l0, int i0, bool gemm_done) {
  switch (c->net.precision) {
    case PC_PREC_FP64: enqueue<double, false>(c, l0, i0, gemm_done); break;
    case PC_PREC_FP32: enqueue<float, false>(c, l0, i0, gemm_done); break;
    default: enqueue<float, true>(c, l0, i0, gemm_done); break;
  }
}

static int occupancy_any(pc_ctx* c) {
  switch (c->net.precision) {
    case PC_PREC_FP64: return Kernels<double, false>::occupancy(c);
    case PC_PREC_FP32: return Kernels<float, false>::occupancy(c);
    default: return Kernels<float, true>::occupancy(c);
  }
}

// Parameter pairs the polish keeps in shared memory: all p (8 B each) when
// they leave room for at least 8 warp workspaces, else none.
static long long polish_stage(long long p, size_t ws) {
  const long long bytes = (p * 8 + 15) / 16 * 16;
  return bytes + 8 * (long long)ws <= kPolishSmemMax ? p : 0;
}

// Thrown when the exact check after a fingerprint-paired extraction fails.
struct NeedsInlinePairing {};

static long long pow2_at_least(long long x) {
  long long p = 64;
  while (p < x) p <<= 1;
  return p;
}

// A polyhedral domain {x : c - A x >= 0} and its 1-skeleton, host arrays.
struct DomainIn {
  int m;
  const double* A;    // m x D, row-major
  const double* c;    // m
  long long nv0;
  const double* X0;   // nv0 x D, row-major
  long long ne0;
  const int32_t* E0;  // ne0 x 2
};

// Checks a domain and its skeleton for edge subdivision: finite values;
// every vertex inside the domain and on exactly D facets (a simple polytope,
// so that every vertex of the complex lies on D hyperplanes); every edge
// joins two distinct vertices that share exactly D - 1 facets, no edge
// twice, D edges at every vertex; a full-dimensional bounding box.  Returns
// "" or the reason; on success lo / hi receive the bounding box.
static std::string check_domain(int D, const DomainIn& d, double* lo, double* hi) {
  if (D < 1 || D > kMaxD) return "input dimension must be in [1, " + std::to_string(kMaxD) + "]";
  if (d.m < D + 1 || d.m > kMaxEntries) return "the number of facets must be in [D + 1, 1024]";
  if (!d.A || !d.c || !d.X0 || !d.E0) return "null domain array";
  if (d.nv0 < D + 1 || d.nv0 > (1ll << 20)) return "the skeleton needs D + 1 to 2^20 vertices";
  if (d.ne0 < 1 || d.ne0 > (1ll << 23)) return "the skeleton needs 1 to 2^23 edges";
  for (long long k = 0; k < (long long)d.m * D; ++k)
    if (!std::isfinite(d.A[k])) return "non-finite facet normal";
  for (int i = 0; i < d.m; ++i)
    if (!std::isfinite(d.c[i])) return "non-finite facet offset";
  const int zw = (d.m + 63) / 64;  // facet-zero bitmask words per vertex
  std::vector<uint64_t> zeros(static_cast<size_t>(d.nv0) * zw, 0);
  for (int k = 0; k < D; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  for (long long v = 0; v < d.nv0; ++v) {
    const double* x = d.X0 + v * D;
    for (int k = 0; k < D; ++k) {
      if (!std::isfinite(x[k])) return "non-finite vertex coordinate";
      lo[k] = std::min(lo[k], x[k]);
      hi[k] = std::max(hi[k], x[k]);
    }
    int nz = 0;
    for (int i = 0; i < d.m; ++i) {
      double f = d.c[i], s = std::fabs(d.c[i]);
      for (int k = 0; k < D; ++k) {
        const double t = d.A[(long long)i * D + k] * x[k];
        f -= t;
        s += std::fabs(t);
      }
      if (std::fabs(f) <= 1e-12 * s) {
        zeros[v * zw + i / 64] |= 1ull << (i % 64);
        ++nz;
      } else if (f < 0) {
        return "vertex " + std::to_string(v) + " lies outside facet " + std::to_string(i);
      }
    }
    if (nz != D)
      return "vertex " + std::to_string(v) + " lies on " + std::to_string(nz) + " facets, not D (a simple polytope is needed)";
  }
  for (int k = 0; k < D; ++k)
    if (!(hi[k] > lo[k])) return "the skeleton is not full-dimensional";
  std::vector<long long> deg(d.nv0, 0);
  std::vector<std::pair<int32_t, int32_t>> pairs(d.ne0);
  for (long long e = 0; e < d.ne0; ++e) {
    const int32_t u = d.E0[2 * e], w = d.E0[2 * e + 1];
    if (u < 0 || w < 0 || u >= d.nv0 || w >= d.nv0 || u == w) return "edge " + std::to_string(e) + " has a bad endpoint";
    int shared = 0;
    for (int q = 0; q < zw; ++q) shared += __builtin_popcountll(zeros[u * zw + q] & zeros[w * zw + q]);
    if (shared != D - 1) return "edge " + std::to_string(e) + " does not lie on D - 1 facets";
    ++deg[u];
    ++deg[w];
    pairs[e] = {std::min(u, w), std::max(u, w)};
  }
  for (long long v = 0; v < d.nv0; ++v)
    if (deg[v] != D) return "vertex " + std::to_string(v) + " has " + std::to_string(deg[v]) + " edges, not D";
  std::sort(pairs.begin(), pairs.end());
  if (std::adjacent_find(pairs.begin(), pairs.end()) != pairs.end()) return "an edge occurs twice";
  return "";
}

static void run_extract(pc_ctx* c, int L, const int32_t* widths, const double* params,
                        const double* lo, const double* hi, bool deferred, const DomainIn* dom = nullptr) {
  c->deferred = deferred ? 1 : 0;
  if (L < 1 || L > kMaxL) throw PcError(PC_ERR_INVALID, "number of layers must be in [1, 16]");
  const int D = widths[0];
  if (D < 1 || D > kMaxD)
    throw PcError(PC_ERR_INVALID, "input dimension must be in [1, " + std::to_string(kMaxD) + "]");
  NetDesc& net = c->net;
  net = NetDesc{};
  net.L = L;
  net.D = D;
  net.m = dom ? dom->m : 2 * D;
  net.precision = c->opt.precision;
  net.kappa = static_cast<float>(c->opt.filter_kappa > 0 ? c->opt.filter_kappa : 2.0);
  net.debug_barrier = c->opt.debug_barrier_timeout ? 1 : 0;
  net.kappa_sel = std::max(net.kappa, static_cast<float>(c->opt.filter_kappa_audit));
  long long p = 0;
  int n = 0, hmax = 0, mw = D;
  for (int l = 0; l <= L; ++l) {
    if (widths[l] < 1 || widths[l] > kMaxWidth) throw PcError(PC_ERR_INVALID, "layer widths must be in [1, 256]");
    net.w[l] = widths[l];
  }
  for (int l = 0; l < L; ++l) {
    net.off[l] = n;
    net.wofs[l] = p;
    p += (long long)widths[l + 1] * widths[l];
    net.bofs[l] = p;
    p += widths[l + 1];
    n += widths[l + 1];
    hmax = std::max(hmax, widths[l + 1]);
    mw = std::max(mw, widths[l + 1]);
  }
  net.off[L] = n;
  net.N = n;
  net.P = net.m + n;
  if (net.P > kMaxEntries) throw PcError(PC_ERR_INVALID, "facets + number of neurons must be <= 1024");
  net.S = (net.P + 31) / 32;
  for (int d = 0; d < D; ++d) {
    net.lo[d] = lo[d];
    net.hi[d] = hi[d];
    if (!(hi[d] > lo[d])) throw PcError(PC_ERR_INVALID, "box must have hi > lo");
  }
  // polyhedral domain: facets and skeleton in one device buffer (A, c, X0
  // as float64, then E0); net.lo / net.hi hold the skeleton's bounding box
  const double* X0dev = nullptr;
  const int32_t* E0dev = nullptr;
  if (dom) {
    const size_t nA = (size_t)dom->m * D, nX = (size_t)dom->nv0 * D;
    const size_t bytes = 8 * (nA + dom->m + nX) + 8 * (size_t)dom->ne0;
    if (c->dom_cap < bytes || !c->dom_buf) {
      c->dom_cap = 0;
      ctx_free(c, c->dom_buf);
      c->dom_buf = ctx_alloc(c, bytes);
      if (!c->dom_buf) throw PcError(PC_ERR_OOM, "domain allocation failed");
      c->dom_cap = bytes;
    }
    double* b = static_cast<double*>(c->dom_buf);
    PC_CUDA(cudaMemcpyAsync(b, dom->A, 8 * nA, cudaMemcpyHostToDevice, c->stream));
    PC_CUDA(cudaMemcpyAsync(b + nA, dom->c, 8 * (size_t)dom->m, cudaMemcpyHostToDevice, c->stream));
    PC_CUDA(cudaMemcpyAsync(b + nA + dom->m, dom->X0, 8 * nX, cudaMemcpyHostToDevice, c->stream));
    PC_CUDA(cudaMemcpyAsync(b + nA + dom->m + nX, dom->E0, 8 * (size_t)dom->ne0, cudaMemcpyHostToDevice, c->stream));
    net.fA = b;
    net.fc = b + nA;
    X0dev = b + nA + dom->m;
    E0dev = reinterpret_cast<const int32_t*>(b + nA + dom->m + nX);
  }
  c->hmax = hmax;
  c->mw = mw;
  c->N = n;

  // parameters: device copies in float64 and float32, per-layer norms
  const size_t pbytes = sizeof(double) * p;
  if (c->params_cap < p || c->norms_cap < n || !c->params64 || !c->params32 || !c->norms) {
    c->params_cap = 0;
    c->norms_cap = 0;
    ctx_free(c, c->params64);
    ctx_free(c, c->params32);
    ctx_free(c, c->norms);
    c->params64 = ctx_alloc(c, pbytes);
    c->params32 = ctx_alloc(c, sizeof(float) * (pairs_offset(p) + 2 * p));  // heads, then (head, remainder) pairs
    c->norms = ctx_alloc(c, sizeof(float) * (2 * kMaxL + 3 * (size_t)n));
    if (!c->params64 || !c->params32 || !c->norms) {
      ctx_free(c, c->params64);
      ctx_free(c, c->params32);
      ctx_free(c, c->norms);
      throw PcError(PC_ERR_OOM, "parameter allocation failed");
    }
    c->params_cap = p;
    c->norms_cap = n;
  }
  PC_CUDA(cudaMemcpyAsync(c->params64, params, pbytes, cudaMemcpyDefault, c->stream));
  net.W64 = static_cast<const double*>(c->params64);
  net.W32 = static_cast<const float*>(c->params32);
  net.WT2 = reinterpret_cast<const float2*>(net.W32 + pairs_offset(p));
  net.norms = static_cast<const float*>(c->norms);
  net.nrm = net.norms + 2 * kMaxL;
  k_prep<<<std::max(L, 64), 256, 0, c->stream>>>(net, static_cast<float*>(c->params32), static_cast<float*>(c->norms), p);
  PC_CUDA(cudaGetLastError());

  // state buffers (kept across extractions when shapes allow)
  ensure_fixed(c, n);
  const size_t zs = zsize_of(net.precision);
  const bool reshape = !c->bufs.X || c->shape_D != D || c->shape_S < net.S || c->shape_H < hmax ||
                       c->shape_zs != zs || c->shape_tape != c->opt.keep_tape ||
                       (c->opt.keep_tape && c->shape_nz < L);
  if (reshape) {
    long long V = std::max<long long>(c->Vcap, std::max<long long>(c->opt.init_vcap, 1 << 14));
    long long E = std::max<long long>(c->Ecap, std::max<long long>(c->opt.init_ecap, (long long)D * V));
    long long T = std::max<long long>(c->Tcap, 1 << 16);
    c->bufs.release(c);
    c->shape_D = D;
    c->shape_S = net.S;
    c->shape_H = hmax;
    c->shape_zs = zs;
    c->shape_tape = c->opt.keep_tape;
    c->shape_nz = L;
    realloc_state(c, V, E, T, false);
  } else {
    // an earlier extraction that stopped early may have left keys and flags
    PC_CUDA(cudaMemsetAsync(c->bufs.table, 0xff, 32 * c->Tcap, c->stream));
    PC_CUDA(cudaMemsetAsync(c->bufs.flags, 0, sizeof(uint32_t) * 2 * (c->Ecap / 32), c->stream));
  }
  if (dom && (c->Vcap < dom->nv0 || c->Ecap < dom->ne0))
    realloc_state(c, std::max(c->Vcap, dom->nv0), std::max(c->Ecap, dom->ne0), c->Tcap, false);
  PC_CUDA(cudaMemsetAsync(c->cnt, 0, sizeof(Counters) * (n + 1), c->stream));

  // launch geometry
  net.rd_batch = rd_batch_size(mw, D, net.S);
  c->res_smem = rd_layout(net.rd_batch, mw, D, net.S).total;
  const int occ = occupancy_any(c);
  if (occ < 1) throw PcError(PC_ERR_INVALID, "persistent kernel does not fit on an SM");
  c->grid_persist = std::min(kMaxGrid, occ * c->num_sms);
  c->grid_step = std::min(kMaxGrid, 2 * c->num_sms);

  for (int k = 0; k <= pc_ctx::kPolishSlot; ++k) c->ev_used[k] = 0;
  if (dom) k_init_domain<<<1, 256, 0, c->stream>>>(net, make_state(c), X0dev, E0dev, dom->nv0, dom->ne0);
  else k_init<<<1, 256, 0, c->stream>>>(net, make_state(c));
  PC_CUDA(cudaGetLastError());
  c->launches += 2;  // k_prep and k_init

  int l0 = 0, i0 = 0;
  bool gemm_done = false;
  for (int attempt = 0;; ++attempt) {
    enqueue_any(c, l0, i0, gemm_done);
    PC_CUDA(cudaMemcpyAsync(c->h_g, c->g, sizeof(Global), cudaMemcpyDeviceToHost, c->stream));
    PC_CUDA(cudaStreamSynchronize(c->stream));
    Global g = *static_cast<Global*>(c->h_g);
    if (g.error & kErrTimeout) throw PcError(PC_ERR_TIMEOUT, "a device-side grid barrier timed out");
    if (g.error & kErrCorrupt)
      throw PcError(PC_ERR_CUDA, "a device counter left its capacity (internal error; check " +
                                     std::to_string(g.diag_site) + " at " + std::to_string(g.diag_n) + ": " +
                                     std::to_string(g.diag_a) + " " + std::to_string(g.diag_b) + " " +
                                     std::to_string(g.diag_c) + ")");
    if (g.halted_at < 0) break;
    if (attempt > 60) throw PcError(PC_ERR_OOM, "capacity growth did not converge");
    // grow what ran out and resume at the halted neuron
    const int hn = g.halted_at;
    int hl = 0;
    while (hl + 1 < L && hn >= net.off[hl + 1]) ++hl;
    long long V = c->Vcap, E = c->Ecap, T = c->Tcap;
    if (g.halt_reason & (kHaltV | kHaltTape)) V = std::max(2 * V, (long long)(g.need_v * 1.3) + 1024);
    if (g.halt_reason & kHaltE) E = std::max(2 * E, (long long)(g.need_e * 1.3) + 1024);
    if (g.halt_reason & kHaltT) T = std::max(2 * T, pow2_at_least(g.need_t));
    V = std::min<long long>(V, (1ll << 31) - 1);
    E = std::min<long long>(E, (1ll << 31) - 1);
    // the halted step wrote nothing: its list of splitting edges (copied with
    // the buffers) and its counters carry over
    realloc_state(c, V, E, T, true);
    Global g0{};
    g0.halted_at = -1;
    g0.error = g.error;
    g0.flips = g.flips;
    g0.flip_margin_bits = g.flip_margin_bits;
    g0.missed = g.missed;
    g0.missed_margin_bits = g.missed_margin_bits;
    g0.barrier_extra = net.debug_barrier ? 1u : 0u;
    *static_cast<Global*>(c->h_g) = g0;
    PC_CUDA(cudaMemcpyAsync(c->g, c->h_g, sizeof(Global), cudaMemcpyHostToDevice, c->stream));
    l0 = hl;
    i0 = hn - net.off[hl];
    gemm_done = true;
    c->grows += 1;
  }
  if (c->deferred) {
    k_verify_pairs<<<c->grid_step, 256, 0, c->stream>>>(net, make_state(c));
    PC_CUDA(cudaGetLastError());
    c->launches += 1;
  }
  const bool polish = c->opt.polish > 0 || (c->opt.polish < 0 && net.precision == PC_PREC_MIXED);
  if (polish && net.precision != PC_PREC_FP64) {
    double diam = 0.0;
    for (int d = 0; d < D; ++d) diam += (hi[d] - lo[d]) * (hi[d] - lo[d]);
    const float thr = static_cast<float>((c->opt.polish_tol > 0 ? c->opt.polish_tol : 1e-6) * std::sqrt(diam));
    const size_t ws = ff_ws_bytes(c->mw, D);
    const long long n_stage = polish_stage(p, ws);
    const size_t stage_b = (n_stage * 8 + 15) / 16 * 16;
    const int wpc = std::max(1, std::min(kWarps, int((kPolishSmemMax - stage_b) / ws)));
    TimerScope ts(c, pc_ctx::kPolishSlot);
    if (pc_polish_tile_eligible(net))
      PC_CUDA(pc_polish_tile_launch(net, make_state(c), thr, c->mw, c->num_sms, dom, c->stream));
    else if (dom)
      k_polish<true><<<c->grid_step, 32 * wpc, stage_b + ws * wpc, c->stream>>>(net, make_state(c), thr, c->mw, n_stage);
    else
      k_polish<false><<<c->grid_step, 32 * wpc, stage_b + ws * wpc, c->stream>>>(net, make_state(c), thr, c->mw, n_stage);
    PC_CUDA(cudaGetLastError());
    c->launches += 1;
  }
  PC_CUDA(cudaMemcpyAsync(c->h_g, c->g, sizeof(Global), cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA(cudaMemcpyAsync(c->h_cnt, c->cnt, sizeof(Counters) * (n + 1), cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA(cudaStreamSynchronize(c->stream));
  c->polished = static_cast<Global*>(c->h_g)->polished;
  c->flips = static_cast<Global*>(c->h_g)->flips;
  c->missed = static_cast<Global*>(c->h_g)->missed;
  {
    int bits = static_cast<Global*>(c->h_g)->flip_margin_bits;
    float f = 0.f;
    std::memcpy(&f, &bits, sizeof(f));
    c->flip_margin = f;
    bits = static_cast<Global*>(c->h_g)->missed_margin_bits;
    std::memcpy(&f, &bits, sizeof(f));
    c->missed_margin = f;
  }
  for (int k = 0; k <= pc_ctx::kPolishSlot; ++k) {
    c->ktime_ms[k] = -1.0;
    if (c->ev_used[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[k][0], c->ev[k][1]) == cudaSuccess) c->ktime_ms[k] = ms;
      else cudaGetLastError();
    }
  }
  const Counters* hc = static_cast<const Counters*>(c->h_cnt);
  const Counters& last = hc[n];
  c->nV = last.nV_before + last.nsplit;
  c->nE = last.nE_before + last.nsplit + last.npairs;
  c->have_result = true;
  const Global g = *static_cast<Global*>(c->h_g);
  if (g.error & kErrCorrupt)
    throw PcError(PC_ERR_CUDA, "a device counter left its capacity (internal error; check " +
                                   std::to_string(g.diag_site) + " at " + std::to_string(g.diag_n) + ")");
  if (g.error & kErrVerify) throw NeedsInlinePairing();
  long long degenerate = 0, undecided = 0;
  bool pairing = (g.error & (kErrPairing | kErrProbe)) != 0;
  int pair_at = -1;
  for (int k = 1; k <= n; ++k) {
    degenerate += hc[k].ndegenerate;
    undecided += hc[k].nundecided;
    if (hc[k].nkeys != 2 * hc[k].npairs && pair_at < 0) pair_at = k - 1;
  }
  pairing = pairing || pair_at >= 0;
  c->degenerate = degenerate;
  c->undecided = undecided;
  if (pairing) {
    std::string where = pair_at >= 0 ? " at neuron " + std::to_string(pair_at) + ": " +
                                           std::to_string(hc[pair_at + 1].nkeys) + " keys, " +
                                           std::to_string(hc[pair_at + 1].npairs) + " pairs"
                                     : "";
    throw PcError(PC_ERR_PAIRING, "a splitting 2-face did not occur exactly twice (non-generic input; error bits " +
                                      std::to_string(g.error) + where + ")");
  }
  if (g.error & kErrConflict) throw PcError(PC_ERR_PAIRING, "edge endpoints disagree on a processed sign entry");
  if (c->opt.strict && (degenerate || undecided))
    throw PcError(PC_ERR_DEGENERATE, "genericity violated: " + std::to_string(degenerate) + " exact zeros, " +
                                          std::to_string(undecided) + " FP64-undecidable signs");
  if (c->opt.prune) pc_prune_vertices(c);
  if (c->opt.canonical) pc_canonicalize(c);
}

void StateBufs::release(pc_ctx* c) {
  ctx_free(c, X);
  for (int k = 0; k < nz; ++k) ctx_free(c, Z[k]);
  nz = 0;
  ctx_free(c, esc);
  ctx_free(c, exc);
  ctx_free(c, SIG);
  ctx_free(c, E);
  ctx_free(c, list0);
  ctx_free(c, list1);
  ctx_free(c, flags);
  ctx_free(c, vlist);
  ctx_free(c, table);
  ctx_free(c, tape_pq);
  ctx_free(c, tape_t);
}

void pc_release_buffers(pc_ctx* c) {
  cudaSetDevice(c->device);
  c->bufs.release(c);
  c->Vcap = c->Ecap = c->Tcap = 0;
  c->shape_D = c->shape_S = c->shape_H = 0;
  c->have_result = false;
  pc_poset_release(c);
  cudaStreamSynchronize(c->stream);
}

// Dynamic shared-memory limits of the kernels, set to constant maxima so that
// every context (in any thread) agrees; a per-network value would race.
void pc_adjoint_set_attributes();
static cudaError_t set_func_attributes_now() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f, int bytes) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = r;
  };
  set((const void*)k_layer<double, false>, kRdSmemMax);
  set((const void*)k_layer<float, false>, kRdSmemMax);
  set((const void*)k_layer<float, true>, kRdSmemMax);
  set((const void*)k_decide<double, false>, kRdSmemMax);
  set((const void*)k_decide<float, false>, kRdSmemMax);
  set((const void*)k_decide<float, true>, kRdSmemMax);
  set((const void*)k_step<double, false>, kRdSmemMax);
  set((const void*)k_step<float, false>, kRdSmemMax);
  set((const void*)k_step<float, true>, kRdSmemMax);
  set((const void*)k_polish<false>, kPolishSmemMax);
  set((const void*)k_polish<true>, kPolishSmemMax);
  {
    const cudaError_t r = pc_gemm_tc_set_attributes();
    if (e == cudaSuccess) e = r;
  }
  {
    const cudaError_t r = pc_polish_tile_set_attributes();
    if (e == cudaSuccess) e = r;
  }
  {
    const cudaError_t r = pc_prune_set_attributes();
    if (e == cudaSuccess) e = r;
  }
  pc_adjoint_set_attributes();
  return e;
}

// Once per device and process, before any launch of these kernels: setting an
// attribute while another thread launches the kernel is not safe.
static cudaError_t set_func_attributes() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  const cudaError_t e = set_func_attributes_now();
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

void pc_default_options(pc_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = PC_PREC_MIXED;
  o->exec = PC_EXEC_PERSISTENT;
  o->filter_kappa = 12.0;
  o->polish = -1;
  o->polish_tol = 1e-6;
}

pc_status pc_create(pc_ctx** out, int device, const pc_options* opt) {
  if (!out) return PC_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PC_ERR_CUDA;
  }
  pc_ctx* c = new pc_ctx();
  c->device = device;
  pc_default_options(&c->opt);
  if (opt) c->opt = *opt;
  if (c->opt.precision < 0 || c->opt.precision > 2 || c->opt.exec < 0 || c->opt.exec > 1 || c->opt.gemm < 0 ||
      c->opt.gemm > 2 || c->opt.pairing < 0 || c->opt.pairing > 1 || (c->opt.canonical && c->opt.keep_tape) ||
      (c->opt.prune && c->opt.keep_tape)) {
    delete c;
    return PC_ERR_INVALID;
  }
  cudaSetDevice(device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (set_func_attributes() != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PC_ERR_CUDA;
  }
  *out = c;
  return PC_OK;
}

pc_status pc_destroy(pc_ctx* c) {
  if (!c) return PC_OK;
  cudaSetDevice(c->device);
  c->bufs.release(c);
  ctx_free(c, c->params64);
  ctx_free(c, c->params32);
  ctx_free(c, c->norms);
  ctx_free(c, c->cnt);
  ctx_free(c, c->g);
  ctx_free(c, c->dom_buf);
  pc_poset_release(c);
  c->release_extra();
  cudaStreamSynchronize(c->stream);
  for (auto& e : c->ev) {
    if (e[0]) cudaEventDestroy(e[0]);
    if (e[1]) cudaEventDestroy(e[1]);
  }
  if (c->h_cnt) cudaFreeHost(c->h_cnt);
  if (c->h_g) cudaFreeHost(c->h_g);
  delete c;
  return PC_OK;
}

pc_status pc_set_allocator(pc_ctx* c, pc_alloc_fn a, pc_free_fn f, void* user) {
  if (!c || (!a) != (!f)) return PC_ERR_INVALID;
  if (c->allocated) return c->fail(PC_ERR_INVALID, "set the allocator before the first extraction");
  c->alloc_fn = a;
  c->free_fn = f;
  c->alloc_user = user;
  return PC_OK;
}

pc_status pc_extract(pc_ctx* c, int L, const int32_t* widths, const double* params, const double* lo,
                     const double* hi, void* stream) {
  if (!c || !widths || !params || !lo || !hi) return PC_ERR_INVALID;
  c->err.clear();
  c->have_result = false;
  pc_poset_release(c);
  try {
    PC_CUDA(cudaSetDevice(c->device));
    c->stream = static_cast<cudaStream_t>(stream);
    try {
      run_extract(c, L, widths, params, lo, hi, c->opt.pairing == PC_PAIR_DEFERRED);
    } catch (const NeedsInlinePairing&) {
      // a 64-bit fingerprint collision paired two different 2-faces: extract
      // again with every pairing verified before it is made
      c->reruns += 1;
      run_extract(c, L, widths, params, lo, hi, false);
    }
    return PC_OK;
  } catch (const PcError& e) {
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    c->have_result = false;
    return c->fail(e.status, e.what());
  } catch (const std::exception& e) {
    c->have_result = false;
    return c->fail(PC_ERR_INVALID, e.what());
  }
}

pc_status pc_check_domain(int D, int m, const double* A, const double* cvec, int64_t nv0, const double* X0,
                          int64_t ne0, const int32_t* E0) {
  double lo[kMaxD], hi[kMaxD];
  const DomainIn dom{m, A, cvec, nv0, X0, ne0, E0};
  return check_domain(D, dom, lo, hi).empty() ? PC_OK : PC_ERR_INVALID;
}

pc_status pc_extract_domain(pc_ctx* c, int L, const int32_t* widths, const double* params, int m, const double* A,
                            const double* cvec, int64_t nv0, const double* X0, int64_t ne0, const int32_t* E0,
                            void* stream) {
  if (!c || !widths || !params || L < 1) return PC_ERR_INVALID;
  c->err.clear();
  c->have_result = false;
  pc_poset_release(c);
  const DomainIn dom{m, A, cvec, nv0, X0, ne0, E0};
  double lo[kMaxD], hi[kMaxD];
  const std::string why = check_domain(widths[0], dom, lo, hi);
  if (!why.empty()) return c->fail(PC_ERR_INVALID, "domain: " + why);
  try {
    PC_CUDA(cudaSetDevice(c->device));
    c->stream = static_cast<cudaStream_t>(stream);
    try {
      run_extract(c, L, widths, params, lo, hi, c->opt.pairing == PC_PAIR_DEFERRED, &dom);
    } catch (const NeedsInlinePairing&) {
      c->reruns += 1;
      run_extract(c, L, widths, params, lo, hi, false, &dom);
    }
    return PC_OK;
  } catch (const PcError& e) {
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    c->have_result = false;
    return c->fail(e.status, e.what());
  } catch (const std::exception& e) {
    c->have_result = false;
    return c->fail(PC_ERR_INVALID, e.what());
  }
}

pc_status pc_counts(pc_ctx* c, int64_t* nv, int64_t* ne, int32_t* sw, int32_t* dim, int32_t* nent) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (nv) *nv = c->nV;
  if (ne) *ne = c->nE;
  if (sw) *sw = c->net.S;
  if (dim) *dim = c->net.D;
  if (nent) *nent = c->net.P;
  return PC_OK;
}

static pc_status copy_rows(pc_ctx* c, void* out, const void* src, size_t elt, long long ld, long long n, int rows) {
  if (!out || n == 0 || rows == 0) return PC_OK;
  cudaError_t e = cudaMemcpy2DAsync(out, elt * n, src, elt * ld, elt * n, rows, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c->fail(PC_ERR_CUDA, cudaGetErrorString(e));
  return PC_OK;
}

pc_status pc_vertices(pc_ctx* c, const double** dev, int64_t* ld, double* out) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (dev) *dev = static_cast<const double*>(c->bufs.X);
  if (ld) *ld = c->Vcap;
  return copy_rows(c, out, c->bufs.X, 8, c->Vcap, c->nV, c->net.D);
}

pc_status pc_edges(pc_ctx* c, const int32_t** dev, int64_t* ld, int32_t* out) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (dev) *dev = static_cast<const int32_t*>(c->bufs.E);
  if (ld) *ld = c->Ecap;
  return copy_rows(c, out, c->bufs.E, 4, c->Ecap, c->nE, 2);
}

pc_status pc_signvectors(pc_ctx* c, const uint64_t** dev, int64_t* ld, uint64_t* out) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (dev) *dev = static_cast<const uint64_t*>(c->bufs.SIG);
  if (ld) *ld = c->Vcap;
  return copy_rows(c, out, c->bufs.SIG, 8, c->Vcap, c->nV, c->net.S);
}

pc_status pc_values(pc_ctx* c, void* out) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  const int L = c->net.L;
  return copy_rows(c, out, pc_make_state(c).Z[L - 1], zsize_of(c->net.precision), c->Vcap, c->nV, c->net.w[L]);
}

pc_status pc_error_estimates(pc_ctx* c, float* value_scale, float* coord_rms) {
  if (!c) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (c->net.precision == PC_PREC_FP64) return c->fail(PC_ERR_INVALID, "no FP32 error estimates in FP64 mode");
  pc_status s = copy_rows(c, value_scale, c->bufs.esc, 4, c->Vcap, c->nV, 1);
  if (s != PC_OK) return s;
  return copy_rows(c, coord_rms, c->bufs.exc, 4, c->Vcap, c->nV, 1);
}

pc_status pc_stats(pc_ctx* c, int64_t* out, int n_neurons) {
  if (!c || !out) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (n_neurons != c->N) return c->fail(PC_ERR_INVALID, "n_neurons does not match the last network");
  const Counters* hc = static_cast<const Counters*>(c->h_cnt);
  for (int k = 0; k < n_neurons; ++k) {
    const Counters& s = hc[k + 1];
    int64_t* o = out + 8 * k;
    o[0] = s.nV_before; o[1] = s.nE_before; o[2] = s.nsplit; o[3] = s.nkeys;
    o[4] = s.npairs; o[5] = s.nfilter; o[6] = s.nundecided; o[7] = s.ndegenerate;
  }
  return PC_OK;
}

pc_status pc_diagnostics(pc_ctx* c, int64_t* out, int n) {
  if (!c || !out) return PC_ERR_INVALID;
  const int64_t v[15] = {c->launches, c->grows, c->polished, c->degenerate, c->undecided, c->Vcap,
                         c->Ecap,    c->Tcap,  (int64_t)c->allocated, c->grid_persist, c->reruns, c->flips,
                         (int64_t)std::ceil(1000.0 * c->flip_margin), c->missed,
                         (int64_t)std::ceil(1000.0 * c->missed_margin)};
  for (int k = 0; k < n && k < 15; ++k) out[k] = v[k];
  return PC_OK;
}

pc_status pc_kernel_times(pc_ctx* c, double* out_ms, int n) {
  if (!c || !out_ms) return PC_ERR_INVALID;
  const int L2 = 2 * c->net.L;
  for (int k = 0; k < n; ++k) out_ms[k] = k < L2 ? c->ktime_ms[k] : (k == L2 ? c->ktime_ms[pc_ctx::kPolishSlot] : -1.0);
  return PC_OK;
}

const char* pc_last_error(pc_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free extraction.
//
// Some callers cannot allocate device memory while they run: code inside a
// custom memory pool or a framework allocator callback, real-time paths that
// forbid cudaMalloc (it can synchronise the device), and hosts that give the
// library a fixed memory reservation.  pc_extract_noalloc serves them: the
// caller passes the parameters and the output arrays, and every other buffer
// the extraction needs (the layer values, error estimates, staged splitting
// edges, the 2-face hash table, counters and the parameter copies) lives in
// one file-scope static device array, g_noalloc_scratch, whose size is fixed
// at compile time.  Every GPU that loads the library holds that array until
// the process exits.  The kernels are the same as pc_extract's, run one
// kernel per step.
namespace {

constexpr long long kNaMaxV = 16384;        // vertices (caller capacity limit)
constexpr long long kNaMaxE = 65536;        // edges
constexpr long long kNaMaxT = 131072;       // 2-face hash slots
constexpr int kNaMaxWidth = 32;             // layer width
constexpr int kNaMaxN = 512;                // neurons
constexpr long long kNaMaxParams = 16384;   // float64 parameters

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kNaOffP64 = 0;
constexpr size_t kNaOffP32 = kNaOffP64 + na_align(8 * kNaMaxParams);
constexpr size_t kNaOffNorm = kNaOffP32 + na_align(12 * kNaMaxParams + 8);
constexpr size_t kNaOffZ0 = kNaOffNorm + na_align(4 * (2 * kMaxL + 3 * kNaMaxN));
constexpr size_t kNaZBytes = na_align(8ull * kNaMaxWidth * kNaMaxV);
constexpr size_t kNaOffZ1 = kNaOffZ0 + kNaZBytes;
constexpr size_t kNaOffEsc = kNaOffZ1 + kNaZBytes;
constexpr size_t kNaOffExc = kNaOffEsc + na_align(4 * kNaMaxV);
constexpr size_t kNaOffList0 = kNaOffExc + na_align(4 * kNaMaxV);
constexpr size_t kNaOffList1 = kNaOffList0 + na_align(16 * kNaMaxE);
constexpr size_t kNaFlagBytes = na_align(4 * 2 * (kNaMaxE / 32));
constexpr size_t kNaOffFlags = kNaOffList1 + na_align(16 * kNaMaxE);
constexpr size_t kNaOffTable = kNaOffFlags + kNaFlagBytes;
constexpr size_t kNaOffCnt = kNaOffTable + na_align(32 * kNaMaxT);
constexpr size_t kNaOffG = kNaOffCnt + na_align(sizeof(Counters) * (kNaMaxN + 1));
constexpr size_t kNaBytes = kNaOffG + na_align(sizeof(Global));

__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch per device (host code cannot use the
// symbol itself as a device pointer).
constexpr int kNaMaxDevices = 64;
void* g_noalloc_addr[kNaMaxDevices] = {};

}  // namespace

extern "C" pc_status pc_extract_noalloc(int L, const int32_t* widths, const double* params, const double* lo,
                                        const double* hi, int precision, double* X, int32_t* E, uint64_t* SIG,
                                        int64_t cap_v, int64_t cap_e, int64_t* n_vertices, int64_t* n_edges,
                                        void* stream) {
  if (!widths || !params || !lo || !hi || !X || !E || !SIG || !n_vertices || !n_edges) return PC_ERR_INVALID;
  if (L < 1 || L > kMaxL || precision < 0 || precision > 2) return PC_ERR_INVALID;
  const int D = widths[0];
  if (D < 1 || D > kMaxD) return PC_ERR_INVALID;
  long long p = 0;
  int n = 0;
  for (int l = 0; l <= L; ++l)
    if (widths[l] < 1 || (l > 0 && widths[l] > kNaMaxWidth)) return PC_ERR_TOO_LARGE;
  for (int l = 0; l < L; ++l) {
    p += (long long)widths[l + 1] * widths[l] + widths[l + 1];
    n += widths[l + 1];
  }
  if (n > kNaMaxN || p > kNaMaxParams || 2 * D + n > kMaxEntries) return PC_ERR_TOO_LARGE;
  if (cap_v > kNaMaxV || cap_e > kNaMaxE) return PC_ERR_TOO_LARGE;
  if (cap_v < (1 << D) || cap_e < (long long)D << (D - 1)) return PC_ERR_INVALID;
  // the edge pass reads four endpoints at a time with 16-byte loads from E and
  // from its second row E + cap_e: both must sit on 16-byte boundaries
  if (cap_e % 4 != 0 || (reinterpret_cast<uintptr_t>(E) & 15) || (reinterpret_cast<uintptr_t>(X) & 7) ||
      (reinterpret_cast<uintptr_t>(SIG) & 7))
    return PC_ERR_INVALID;
  for (int d = 0; d < D; ++d)
    if (!(hi[d] > lo[d])) return PC_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    return PC_ERR_CUDA;
  }
  // once per device, with that device current
  if (!g_noalloc_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) {
      cudaGetLastError();
      return PC_ERR_CUDA;
    }
    g_noalloc_addr[dev] = addr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  if (set_func_attributes() != cudaSuccess) {
    cudaGetLastError();
    return PC_ERR_CUDA;
  }
  pc_ctx c;  // host-side descriptor only: its buffers point into the scratch and the caller's arrays
  c.device = dev;
  cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
  pc_default_options(&c.opt);
  c.opt.precision = precision;
  c.opt.exec = PC_EXEC_STEPWISE;
  c.stream = static_cast<cudaStream_t>(stream);
  try {
    NetDesc& net = c.net;
    net = NetDesc{};
    net.L = L;
    net.D = D;
    net.m = 2 * D;
    net.precision = precision;
    net.kappa = static_cast<float>(c.opt.filter_kappa);
    net.kappa_sel = net.kappa;
    long long q = 0;
    int nn = 0, hmax = 0, mw = D;
    for (int l = 0; l <= L; ++l) net.w[l] = widths[l];
    for (int l = 0; l < L; ++l) {
      net.off[l] = nn;
      net.wofs[l] = q;
      q += (long long)widths[l + 1] * widths[l];
      net.bofs[l] = q;
      q += widths[l + 1];
      nn += widths[l + 1];
      hmax = std::max(hmax, widths[l + 1]);
      mw = std::max(mw, widths[l + 1]);
    }
    net.off[L] = nn;
    net.N = nn;
    net.P = net.m + nn;
    net.S = (net.P + 31) / 32;
    for (int d = 0; d < D; ++d) {
      net.lo[d] = lo[d];
      net.hi[d] = hi[d];
    }
    net.W64 = reinterpret_cast<const double*>(base + kNaOffP64);
    net.W32 = reinterpret_cast<const float*>(base + kNaOffP32);
    net.WT2 = reinterpret_cast<const float2*>(net.W32 + pairs_offset(p));
    net.norms = reinterpret_cast<const float*>(base + kNaOffNorm);
    net.nrm = net.norms + 2 * kMaxL;
    c.hmax = hmax;
    c.mw = mw;
    c.N = nn;
    c.bufs.X = X;
    c.bufs.SIG = SIG;
    c.bufs.E = E;
    c.bufs.Z[0] = base + kNaOffZ0;
    c.bufs.Z[1] = base + kNaOffZ1;
    c.bufs.nz = 2;
    c.bufs.esc = base + kNaOffEsc;
    c.bufs.exc = base + kNaOffExc;
    c.bufs.list0 = base + kNaOffList0;
    c.bufs.list1 = base + kNaOffList1;
    c.bufs.flags = base + kNaOffFlags;
    c.bufs.table = base + kNaOffTable;
    c.cnt = base + kNaOffCnt;
    c.g = base + kNaOffG;
    c.Vcap = cap_v;
    c.Ecap = cap_e;
    c.Tcap = kNaMaxT;
    PC_CUDA(cudaMemcpyAsync(base + kNaOffP64, params, sizeof(double) * p, cudaMemcpyDefault, c.stream));
    k_prep<<<std::max(L, 64), 256, 0, c.stream>>>(net, reinterpret_cast<float*>(base + kNaOffP32),
                                                   reinterpret_cast<float*>(base + kNaOffNorm), p);
    PC_CUDA(cudaGetLastError());
    // the scratch keeps the previous call's contents: reset what must start empty
    PC_CUDA(cudaMemsetAsync(base + kNaOffTable, 0xff, 32 * kNaMaxT, c.stream));
    PC_CUDA(cudaMemsetAsync(base + kNaOffFlags, 0, kNaFlagBytes, c.stream));
    PC_CUDA(cudaMemsetAsync(base + kNaOffCnt, 0, sizeof(Counters) * (nn + 1), c.stream));
    net.rd_batch = rd_batch_size(mw, D, net.S);
    c.res_smem = rd_layout(net.rd_batch, mw, D, net.S).total;
    occupancy_any(&c);
    c.grid_step = std::min(kMaxGrid, 2 * c.num_sms);
    k_init<<<1, 256, 0, c.stream>>>(net, make_state(&c));
    PC_CUDA(cudaGetLastError());
    enqueue_any(&c, 0, 0, false);
    if (precision == PC_PREC_MIXED) {
      double diam = 0.0;
      for (int d = 0; d < D; ++d) diam += (hi[d] - lo[d]) * (hi[d] - lo[d]);
      const float thr = static_cast<float>(c.opt.polish_tol * std::sqrt(diam));
      const size_t ws = ff_ws_bytes(c.mw, D);
      const long long n_stage = polish_stage(p, ws);
      const size_t stage_b = (n_stage * 8 + 15) / 16 * 16;
      const int wpc = std::max(1, std::min(kWarps, int((kPolishSmemMax - stage_b) / ws)));
      if (pc_polish_tile_eligible(net))
        PC_CUDA(pc_polish_tile_launch(net, make_state(&c), thr, c.mw, c.num_sms, false, c.stream));
      else
        k_polish<false><<<c.grid_step, 32 * wpc, stage_b + ws * wpc, c.stream>>>(net, make_state(&c), thr, c.mw, n_stage);
      PC_CUDA(cudaGetLastError());
    }
    Global g{};
    std::vector<Counters> hc(nn + 1);
    PC_CUDA(cudaMemcpyAsync(&g, c.g, sizeof(Global), cudaMemcpyDeviceToHost, c.stream));
    PC_CUDA(cudaMemcpyAsync(hc.data(), c.cnt, sizeof(Counters) * (nn + 1), cudaMemcpyDeviceToHost, c.stream));
    PC_CUDA(cudaStreamSynchronize(c.stream));
    if (g.error & kErrTimeout) return PC_ERR_TIMEOUT;
    if (g.error & kErrCorrupt) return PC_ERR_CUDA;
    if (g.halted_at >= 0) return PC_ERR_OOM;
    bool pairing = (g.error & (kErrPairing | kErrProbe | kErrConflict)) != 0;
    for (int k = 1; k <= nn; ++k)
      if (hc[k].nkeys != 2 * hc[k].npairs) pairing = true;
    if (pairing) return PC_ERR_PAIRING;
    *n_vertices = hc[nn].nV_before + hc[nn].nsplit;
    *n_edges = hc[nn].nE_before + hc[nn].nsplit + hc[nn].npairs;
    return PC_OK;
  } catch (const PcError& e) {
    cudaGetLastError();
    return e.status;
  }
}
