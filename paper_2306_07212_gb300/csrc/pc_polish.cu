// Coordinate polish, tiled: every vertex whose coordinate error estimate
// exceeds the threshold moves to the exact intersection of its D zero sets
// (the vertex of Section 4.2's complex: D entries of its sign vector are
// zero, each affine on the vertex's own piece, Eq. 4 with the stored
// activation pattern).  One Newton step from the stored coordinates solves
// the D x D system A dx = -g, with the values g in float-float and the
// gradients A in float32 (the step is small, so float32 gradients add only
// ~1e-7 of the step; see pc_newton.cuh).
//
// The forward pass over the vertices is a matrix product per layer,
//   a_k[r][v] = sum_c W_k[r][c] a_{k-1}[c][v] + b_k[r]   (masked by v's signs),
// so it runs as one: a CTA owns a tile of TV consecutive vertices (vertices
// are created layer by layer, so a tile's vertices mostly need the same
// layers), keeps the tile's activations (hi, lo) and gradients (D per input)
// neuron-major in shared memory, and each thread accumulates a block of 4
// vertices x kPtRows neurons, so every activation it loads serves kPtRows
// outputs and every weight four.  The dot products follow Ogita-Rump-Oishi Dot2 (exact
// products by FMA, TwoSum of the running sum, error terms summed in a
// float), like newton_ff_warp; the layer's outputs overwrite its inputs
// after a barrier.  D <= kPtMaxD; larger D takes the one-warp-per-vertex
// kernel (k_polish).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pc_ctx.h"
#include "pc_device.cuh"
#include "pc_newton.cuh"

namespace pc {

constexpr int kPtThreads = 256;
constexpr int kPtRows = 2;       // neurons per thread (a thread's block: 4 vertices x kPtRows neurons)
constexpr int kPtMinBlocks = 2;  // CTAs per SM the register allocation is made for
constexpr int kPtMaxD = 5;
constexpr int kPtSmemMax = 200 * 1024;

struct PtLayout {
  int TV, rows;
  size_t A, gv, sig, ahi, alo, J, zl, nz, total;
};

// Shared-memory layout of one tile (byte offsets, each 16-aligned).  rows:
// activation rows held (the widest layer, and D for the coordinates).
__host__ __device__ inline PtLayout pt_layout(int TV, int mw, int S, int D) {
  PtLayout p{};
  p.TV = TV;
  p.rows = mw > D ? mw : D;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) / 16 * 16;
    return at;
  };
  p.A = take((size_t)TV * D * D * 8);
  p.gv = take((size_t)TV * D * 8);
  p.sig = take((size_t)TV * S * 8);
  p.ahi = take((size_t)p.rows * TV * 4);
  p.alo = take((size_t)p.rows * TV * 4);
  p.J = take((size_t)p.rows * D * TV * 4);
  p.zl = take((size_t)TV * D * 4);
  p.nz = take((size_t)TV * 4);
  p.total = o;
  return p;
}

// Vertices per tile: the (vertex, neuron) blocks of the widest layer fill
// the CTA, at most 128 vertices, and the tile fits the shared memory.
static int pt_tile_vertices(int mw, int S, int D) {
  const int nrg = (mw + kPtRows - 1) / kPtRows;
  int TV = std::min(128, 4 * std::max(1, kPtThreads / nrg));
  while (TV > 4 && pt_layout(TV, mw, S, D).total > (size_t)kPtSmemMax) TV -= 4;
  return TV;
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int DT, bool DOMAIN>
__global__ void __launch_bounds__(kPtThreads, kPtMinBlocks) k_polish_tile(NetDesc net, State st, float thr, int mw, int TV) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_lmax;
  __shared__ unsigned long long s_pol;
  if (cta_stopped(st)) return;
  const Counters* last = st.cnt + net.N;
  const long long nV = last->nV_before + last->nsplit;
  const long long Vcap = st.Vcap;
  const int S = net.S, m = net.m;
  const PtLayout lay = pt_layout(TV, mw, S, DT);
  double* sA = reinterpret_cast<double*>(sm + lay.A);
  double* sgv = reinterpret_cast<double*>(sm + lay.gv);
  uint64_t* sig = reinterpret_cast<uint64_t*>(sm + lay.sig);  // [S][TV]
  float* ahi = reinterpret_cast<float*>(sm + lay.ahi);        // [rows][TV]
  float* alo = reinterpret_cast<float*>(sm + lay.alo);
  float* J = reinterpret_cast<float*>(sm + lay.J);            // [rows][DT][TV]
  int* zl = reinterpret_cast<int*>(sm + lay.zl);              // [TV][DT]
  int* nzs = reinterpret_cast<int*>(sm + lay.nz);             // zeros found; -1: not polished
  if (threadIdx.x == 0) s_pol = 0;
  const long long ntiles = (nV + TV - 1) / TV;
  const int nvg = TV >> 2;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long v0 = tile * TV;
    if (threadIdx.x == 0) s_lmax = -1;
    for (int i = threadIdx.x; i < S * TV; i += blockDim.x) {  // coalesced over vertices
      const int w = i / TV, vv = i - w * TV;
      sig[i] = v0 + vv < nV ? st.SIG[(long long)w * Vcap + v0 + vv] : 0ull;
    }
    __syncthreads();
    // per vertex: its zero entries, the highest layer among them, and the
    // coordinates (float-float) with the identity as their gradient
    for (int vv = threadIdx.x; vv < TV; vv += blockDim.x) {
      const long long v = v0 + vv;
      int nz = -1, ll = -1;
      if (v < nV && !(st.exc[v] <= thr)) {
        nz = 0;
        for (int w = 0; w < S; ++w) {
          uint64_t zm = zero_mask(sig[w * TV + vv], w, net.P);
          while (zm) {
            const int bit = __ffsll((long long)zm) - 1;
            if (nz < DT) zl[vv * DT + nz] = w * 32 + bit / 2;
            ++nz;
            zm &= zm - 1;
          }
        }
        if (nz != DT) nz = -1;  // not a vertex of the generic complex: left as it is
        for (int q = 0; nz == DT && q < DT; ++q) {
          const int h = zl[vv * DT + q] - m;
          if (h < 0) continue;
          int l = 0;
          while (l + 1 < net.L && h >= net.off[l + 1]) ++l;
          ll = l > ll ? l : ll;
        }
        if (nz == DT) atomicMax(&s_lmax, ll);
      }
      nzs[vv] = nz;
#pragma unroll
      for (int d = 0; d < DT; ++d) {
        const double x = nz == DT ? st.X[(long long)d * Vcap + v] : 0.0;
        const float h = static_cast<float>(x);
        ahi[d * TV + vv] = h;
        alo[d * TV + vv] = static_cast<float>(x - static_cast<double>(h));
#pragma unroll
        for (int dd = 0; dd < DT; ++dd) J[(d * DT + dd) * TV + vv] = d == dd ? 1.f : 0.f;
      }
    }
    __syncthreads();
    const int lmax = s_lmax;
    int in = DT;
    for (int k = 0; k <= lmax; ++k) {
      const int H = net.w[k + 1];
      const int nrg = (H + kPtRows - 1) / kPtRows;
      const int p = threadIdx.x;
      const bool busy = p < nvg * nrg;
      const int vb = busy ? (p % nvg) * 4 : 0;  // vertex blocks vary fastest in a warp
      const int rb = busy ? (p / nvg) * kPtRows : 0;
      // accumulators of vertex pairs (vb, vb + 1) and (vb + 2, vb + 3): the
      // float-float arithmetic runs on packed FP32 pairs (two lanes of work
      // per instruction, each rounded as the scalar operation)
      float2 s2[2][kPtRows], e2[2][kPtRows], jd2[2][kPtRows][DT];
      if (busy) {
        const float2* Wt = net.WT2 + net.wofs[k];  // [in][H] (head, remainder)
        const float2* bk = net.WT2 + net.bofs[k];
#pragma unroll
        for (int j = 0; j < kPtRows; ++j) {
          const float2 b = rb + j < H ? bk[rb + j] : make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            s2[h][j] = make_float2(b.x, b.x);
            e2[h][j] = make_float2(b.y, b.y);
#pragma unroll
            for (int d = 0; d < DT; ++d) jd2[h][j][d] = make_float2(0.f, 0.f);
          }
        }
#pragma unroll 4
        for (int c = 0; c < in; ++c) {
          const float4 ah = *reinterpret_cast<const float4*>(ahi + c * TV + vb);
          const float4 al = *reinterpret_cast<const float4*>(alo + c * TV + vb);
          float4 jv[DT];
#pragma unroll
          for (int d = 0; d < DT; ++d) jv[d] = *reinterpret_cast<const float4*>(J + (c * DT + d) * TV + vb);
          float2 w[kPtRows];
#pragma unroll
          for (int j = 0; j < kPtRows; ++j) w[j] = rb + j < H ? __ldg(Wt + (long long)c * H + rb + j) : make_float2(0.f, 0.f);
          const float2 yh[2] = {make_float2(ah.x, ah.y), make_float2(ah.z, ah.w)};
          const float2 yl[2] = {make_float2(al.x, al.y), make_float2(al.z, al.w)};
#pragma unroll
          for (int j = 0; j < kPtRows; ++j) {
            const float2 xh = make_float2(w[j].x, w[j].x), xl = make_float2(w[j].y, w[j].y);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float2 pr = __fmul2_rn(xh, yh[h]);
              float2 er = __ffma2_rn(xh, yh[h], neg2(pr));  // exact low part of the product
              er = __ffma2_rn(xh, yl[h], er);                // cross terms of the low parts
              er = __ffma2_rn(xl, yh[h], er);
              const float2 t = __fadd2_rn(s2[h][j], pr);     // TwoSum: t + its error is exact
              const float2 bb = __fadd2_rn(t, neg2(s2[h][j]));
              const float2 ts = __fadd2_rn(s2[h][j], neg2(__fadd2_rn(t, neg2(bb))));
              e2[h][j] = __fadd2_rn(e2[h][j], __fadd2_rn(__fadd2_rn(ts, __fadd2_rn(pr, neg2(bb))), er));
              s2[h][j] = t;
            }
#pragma unroll
            for (int d = 0; d < DT; ++d) {
              jd2[0][j][d] = __ffma2_rn(xh, make_float2(jv[d].x, jv[d].y), jd2[0][j][d]);
              jd2[1][j][d] = __ffma2_rn(xh, make_float2(jv[d].z, jv[d].w), jd2[1][j][d]);
            }
          }
        }
      }
      __syncthreads();  // every input of the layer has been read
      if (busy) {
#pragma unroll
        for (int j = 0; j < kPtRows; ++j) {
          const int r = rb + j;
          if (r >= H) continue;
          const int entry = m + net.off[k] + r;
          float zh[4], zo[4], g[DT][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 sp = s2[i >> 1][j], ep = e2[i >> 1][j];
            const ff z = ff_fast_two_sum((i & 1) ? sp.y : sp.x, (i & 1) ? ep.y : ep.x);
            zh[i] = z.hi;
            zo[i] = z.lo;
#pragma unroll
            for (int d = 0; d < DT; ++d) g[d][i] = (i & 1) ? jd2[i >> 1][j][d].y : jd2[i >> 1][j][d].x;
            const int vv = vb + i;
            const int nz = nzs[vv];
            for (int q = 0; q < nz; ++q)
              if (zl[vv * DT + q] == entry) {
                sgv[vv * DT + q] = static_cast<double>(z.hi) + static_cast<double>(z.lo);
#pragma unroll
                for (int d = 0; d < DT; ++d) sA[(vv * DT + q) * DT + d] = g[d][i];
              }
          }
          if (k < lmax) {
            bool act[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              act[i] = ((sig[(entry >> 5) * TV + vb + i] >> (2 * (entry & 31))) & 3ull) == kPlus;
            *reinterpret_cast<float4*>(ahi + r * TV + vb) = make_float4(act[0] ? zh[0] : 0.f, act[1] ? zh[1] : 0.f,
                                                                       act[2] ? zh[2] : 0.f, act[3] ? zh[3] : 0.f);
            *reinterpret_cast<float4*>(alo + r * TV + vb) = make_float4(act[0] ? zo[0] : 0.f, act[1] ? zo[1] : 0.f,
                                                                       act[2] ? zo[2] : 0.f, act[3] ? zo[3] : 0.f);
#pragma unroll
            for (int d = 0; d < DT; ++d)
              *reinterpret_cast<float4*>(J + (r * DT + d) * TV + vb) =
                  make_float4(act[0] ? g[d][0] : 0.f, act[1] ? g[d][1] : 0.f, act[2] ? g[d][2] : 0.f,
                              act[3] ? g[d][3] : 0.f);
          }
        }
      }
      __syncthreads();
      in = H;
    }
    for (int vv = threadIdx.x; vv < TV; vv += blockDim.x) {
      if (nzs[vv] != DT) continue;
      const long long v = v0 + vv;
      int* zv = zl + vv * DT;
      double* Av = sA + (size_t)vv * DT * DT;
      double* gvv = sgv + (size_t)vv * DT;
      if (DOMAIN)
        for (int q = 0; q < DT; ++q) domain_facet_rows(net, st, v, zv, DT, q, Av, gvv);
      NewtonOut o{};
      newton_solve<float>(net, st, v, zv, DT, Av, gvv, o);
      if (o.ok) {
        for (int d = 0; d < DT; ++d) st.X[(long long)d * Vcap + v] += o.dlt[d];
        atomicAdd(&s_pol, 1ull);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_pol) atomic_add_ll(&st.g->polished, static_cast<long long>(s_pol));
}

template <int DT>
static cudaError_t pt_launch_d(const NetDesc& net, const State& st, float thr, int mw, int num_sms, bool domain,
                               cudaStream_t stream) {
  const int TV = pt_tile_vertices(mw, net.S, DT);
  const size_t smem = pt_layout(TV, mw, net.S, DT).total;
  const void* f = domain ? (const void*)k_polish_tile<DT, true> : (const void*)k_polish_tile<DT, false>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kPtThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, num_sms * std::max(1, per_sm));  // persistent: tiles dealt round-robin
  if (domain) k_polish_tile<DT, true><<<grid, kPtThreads, smem, stream>>>(net, st, thr, mw, TV);
  else k_polish_tile<DT, false><<<grid, kPtThreads, smem, stream>>>(net, st, thr, mw, TV);
  return cudaGetLastError();
}

}  // namespace pc

using namespace pc;

bool pc_polish_tile_eligible(const NetDesc& net) { return net.D >= 1 && net.D <= kPtMaxD; }

cudaError_t pc_polish_tile_set_attributes() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPtSmemMax);
    if (e == cudaSuccess) e = r;
  };
  set((const void*)k_polish_tile<1, false>);
  set((const void*)k_polish_tile<2, false>);
  set((const void*)k_polish_tile<3, false>);
  set((const void*)k_polish_tile<4, false>);
  set((const void*)k_polish_tile<5, false>);
  set((const void*)k_polish_tile<1, true>);
  set((const void*)k_polish_tile<2, true>);
  set((const void*)k_polish_tile<3, true>);
  set((const void*)k_polish_tile<4, true>);
  set((const void*)k_polish_tile<5, true>);
  return e;
}

cudaError_t pc_polish_tile_launch(const NetDesc& net, const State& st, float thr, int mw, int num_sms, bool domain,
                                  cudaStream_t stream) {
  switch (net.D) {
    case 1: return pt_launch_d<1>(net, st, thr, mw, num_sms, domain, stream);
    case 2: return pt_launch_d<2>(net, st, thr, mw, num_sms, domain, stream);
    case 3: return pt_launch_d<3>(net, st, thr, mw, num_sms, domain, stream);
    case 4: return pt_launch_d<4>(net, st, thr, mw, num_sms, domain, stream);
    case 5: return pt_launch_d<5>(net, st, thr, mw, num_sms, domain, stream);
    default: return cudaErrorInvalidValue;
  }
}
