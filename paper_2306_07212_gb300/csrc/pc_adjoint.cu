// Adjoint of the vertex coordinates with respect to the network parameters.
//
// The forward pass (Section 4.2) computes every vertex created at neuron n of
// layer l from its edge's endpoints p (+) and q (-) by
//     t  = a / (a - b),  a = z_i(p), b = z_i(q)
//     x0 = x_p + t (x_q - x_p)
//     z0_j = z_j(p) + t (z_j(q) - z_j(p))  (j != i),  z0_i = 0
// and, at the start of every layer, the values of the vertices present then
//     Z_l = W_l act(Z_{l-1}) + b_l,  act_k = z_k if the vertex's entry is +
// (Z_0 = W_0 x + b_0 at the box corners).  With the interpolation tape
// (p, q, t per created vertex) and the per-layer values kept by the forward
// pass, the adjoint replays these formulas in reverse: neuron steps from the
// last to the first (one warp per created vertex scatters to its two
// parents), and at each layer start the products give dL/dW_l, dL/db_l and
// the previous layer's value adjoint.  Arithmetic is float32 (atomic
// accumulation); the parameter gradient is accumulated in float64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "pc.h"
#include "pc_ctx.h"
#include "pc_device.cuh"

namespace pc {

__global__ void k_adj_init(const double* gx, float* xbar, long long nV, long long Vcap, int D) {
  const long long n = nV * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long d = t / nV, v = t - d * nV;
    xbar[d * Vcap + v] = static_cast<float>(gx[t]);
  }
}

// Reverse of one neuron step: one warp per vertex created at that step.
template <typename ZT>
__global__ void k_adj_split(NetDesc net, State st, float* xbar, float* zbar, int l, int i, long long v_begin,
                            long long count) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long Vcap = st.Vcap;
  const int D = net.D, H = net.w[l + 1];
  const ZT* Z = static_cast<const ZT*>(st.Z[l]);
  for (long long w = w0; w < count; w += nw) {
    const long long v0 = v_begin + w;
    const int p = st.tape_pq[v0], q = st.tape_pq[st.tape_cap + v0];
    const double t = st.tape_t[v0];
    const float tf = static_cast<float>(t);
    float tb = 0.f;
    if (lane < D) {
      const float xb = xbar[(long long)lane * Vcap + v0];
      if (xb != 0.f) {
        atomicAdd(&xbar[(long long)lane * Vcap + p], (1.f - tf) * xb);
        atomicAdd(&xbar[(long long)lane * Vcap + q], tf * xb);
        tb += xb * static_cast<float>(st.X[(long long)lane * Vcap + q] - st.X[(long long)lane * Vcap + p]);
      }
    }
    for (int j = lane; j < H; j += 32) {
      if (j == i) continue;
      const float zb = zbar[(long long)j * Vcap + v0];
      if (zb == 0.f) continue;
      atomicAdd(&zbar[(long long)j * Vcap + p], (1.f - tf) * zb);
      atomicAdd(&zbar[(long long)j * Vcap + q], tf * zb);
      tb += zb * static_cast<float>(static_cast<double>(Z[(long long)j * Vcap + q]) -
                                    static_cast<double>(Z[(long long)j * Vcap + p]));
    }
    for (int o = 16; o > 0; o >>= 1) tb += __shfl_xor_sync(0xffffffffu, tb, o);
    if (lane == 0 && tb != 0.f) {
      const double a = static_cast<double>(Z[(long long)i * Vcap + p]);
      const double b = static_cast<double>(Z[(long long)i * Vcap + q]);
      const double d2 = (a - b) * (a - b);
      atomicAdd(&zbar[(long long)i * Vcap + p], static_cast<float>(tb * (-b) / d2));
      atomicAdd(&zbar[(long long)i * Vcap + q], static_cast<float>(tb * a / d2));
    }
  }
}

// Layer start, parameter part: dW_l[j][k] += sum_v zbar_l[j][v] act_k(v) and
// db_l[j] += sum_v zbar_l[j][v] over the vertices present at the layer start.
// Tiles of 32 vertices are staged in shared memory; each thread owns up to 32
// (j, k) entries; blockIdx.y selects a group of 512 x 32 entries.
template <typename ZT>
__global__ void __launch_bounds__(512) k_adj_wgrad(NetDesc net, State st, const float* zbar, double* gW, int l,
                                                   long long nVl) {
  extern __shared__ float sh[];
  constexpr int EPT = 32, TV = 32;
  const int H = net.w[l + 1], K = net.w[l];
  float* zt = sh;            // [H][TV]
  float* at = sh + H * TV;   // [K][TV]
  const long long Vcap = st.Vcap;
  const ZT* Zin = static_cast<const ZT*>(st.Z[l > 0 ? l - 1 : 0]);
  const int ebase = net.m + (l > 0 ? net.off[l - 1] : 0);
  const int e0 = blockIdx.y * blockDim.x * EPT;
  float acc[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) acc[q] = 0.f;
  float bacc = 0.f;
  for (long long base = (long long)blockIdx.x * TV; base < nVl; base += (long long)gridDim.x * TV) {
    for (int t = threadIdx.x; t < (H + K) * TV; t += blockDim.x) {
      const int r = t / TV, c = t % TV;
      const long long v = base + c;
      float val = 0.f;
      if (v < nVl) {
        if (r < H) {
          val = zbar[(long long)r * Vcap + v];
        } else {
          const int k = r - H;
          if (l == 0) {
            val = static_cast<float>(st.X[(long long)k * Vcap + v]);
          } else {
            const int entry = ebase + k;
            const bool act = ((st.SIG[(long long)(entry >> 5) * Vcap + v] >> (2 * (entry & 31))) & 3ull) == kPlus;
            val = act ? static_cast<float>(Zin[(long long)k * Vcap + v]) : 0.f;
          }
        }
      }
      sh[r * TV + c] = val;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = e0 + q * blockDim.x + threadIdx.x;
      if (e < H * K) {
        const int j = e / K, k = e % K;
        float s = 0.f;
#pragma unroll 8
        for (int c = 0; c < TV; ++c) s = fmaf(zt[j * TV + c], at[k * TV + c], s);
        acc[q] += s;
      }
    }
    if (blockIdx.y == 0 && threadIdx.x < H)
      for (int c = 0; c < TV; ++c) bacc += zt[threadIdx.x * TV + c];
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < H * K && acc[q] != 0.f) atomicAdd(&gW[net.wofs[l] + e], static_cast<double>(acc[q]));
  }
  if (blockIdx.y == 0 && threadIdx.x < H && bacc != 0.f) atomicAdd(&gW[net.bofs[l] + threadIdx.x], (double)bacc);
}

// Layer start, value part: zbar_{l-1}[k][v] = act'_k(v) sum_j W_l[j][k] zbar_l[j][v].
__global__ void k_adj_back(NetDesc net, State st, const float* zbar, float* zprev, int l, long long nVl) {
  const int H = net.w[l + 1], K = net.w[l];
  const long long Vcap = st.Vcap;
  const float* W = net.W32 + net.wofs[l];
  const int k = blockIdx.y;
  const int entry = net.m + net.off[l - 1] + k;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nVl; v += (long long)gridDim.x * blockDim.x) {
    const bool act = ((st.SIG[(long long)(entry >> 5) * Vcap + v] >> (2 * (entry & 31))) & 3ull) == kPlus;
    float s = 0.f;
    if (act)
      for (int j = 0; j < H; ++j) s = fmaf(W[(long long)j * K + k], zbar[(long long)j * Vcap + v], s);
    zprev[(long long)k * Vcap + v] = s;
  }
}

template <typename ZT>
static void run_backward(pc_ctx* c, const State& st, float* xbar, float* zb[2], double* gW) {
  const NetDesc& net = c->net;
  const Counters* hc = static_cast<const Counters*>(c->h_cnt);
  for (int l = net.L - 1; l >= 0; --l) {
    float* zl = zb[l & 1];
    for (int i = net.w[l + 1] - 1; i >= 0; --i) {
      const int n = net.off[l] + i;
      const long long cnt = hc[n + 1].nsplit, vb = hc[n + 1].nV_before;
      if (cnt <= 0) continue;
      const int blocks = int(std::min<long long>((cnt + 7) / 8, 4096));
      k_adj_split<ZT><<<blocks, 256, 0, c->stream>>>(net, st, xbar, zl, l, i, vb, cnt);
      if (cudaPeekAtLastError() != cudaSuccess) return;
    }
    const Counters& s0 = hc[net.off[l]];
    const long long nVl = s0.nV_before + s0.nsplit;
    const int H = net.w[l + 1], K = net.w[l];
    const int gy = (H * K + 512 * 32 - 1) / (512 * 32);
    const size_t smem = sizeof(float) * (H + K) * 32;  // <= kAdjSmemMax (widths <= 256)
    const int gx = int(std::max<long long>(1, std::min<long long>((nVl + 31) / 32, 2 * c->num_sms)));
    k_adj_wgrad<ZT><<<dim3(gx, gy), 512, smem, c->stream>>>(net, st, zl, gW, l, nVl);
    if (l > 0) {
      const int gb = int(std::max<long long>(1, std::min<long long>((nVl + 255) / 256, 4 * c->num_sms)));
      k_adj_back<<<dim3(gb, K), 256, 0, c->stream>>>(net, st, zl, zb[(l - 1) & 1], l, nVl);
    }
  }
}

constexpr int kAdjSmemMax = sizeof(float) * 2 * kMaxWidth * 32;

}  // namespace pc

using namespace pc;

void pc_adjoint_set_attributes() {
  cudaFuncSetAttribute(k_adj_wgrad<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmemMax);
  cudaFuncSetAttribute(k_adj_wgrad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmemMax);
}

extern "C" pc_status pc_backward(pc_ctx* c, const double* grad_x, double* grad_params, void* stream) {
  if (!c || !grad_x || !grad_params) return PC_ERR_INVALID;
  if (!c->have_result) return c->fail(PC_ERR_INVALID, "no extraction result");
  if (!c->opt.keep_tape) return c->fail(PC_ERR_NO_TAPE, "extraction ran without keep_tape");
  cudaSetDevice(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  const NetDesc& net = c->net;
  const int D = net.D;
  const long long Vcap = c->Vcap, nV = c->nV;
  long long np = 0;
  for (int l = 0; l < net.L; ++l) np += (long long)net.w[l + 1] * (net.w[l] + 1);
  const size_t need[4] = {sizeof(float) * D * Vcap, sizeof(float) * c->hmax * Vcap, sizeof(float) * c->hmax * Vcap,
                          sizeof(double) * (np + D * nV)};
  for (int k = 0; k < 4; ++k) {
    if (c->adj_bytes[k] < need[k]) {
      ctx_free(c, c->adj[k]);
      c->adj[k] = ctx_alloc(c, need[k]);
      c->adj_bytes[k] = c->adj[k] ? need[k] : 0;
      if (!c->adj[k]) return c->fail(PC_ERR_OOM, "adjoint buffer allocation failed");
    }
  }
  float* xbar = static_cast<float*>(c->adj[0]);
  float* zb[2] = {static_cast<float*>(c->adj[1]), static_cast<float*>(c->adj[2])};
  double* gW = static_cast<double*>(c->adj[3]);
  double* gx = gW + np;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  ok(cudaMemsetAsync(gW, 0, sizeof(double) * np, c->stream));
  ok(cudaMemsetAsync(xbar, 0, need[0], c->stream));
  ok(cudaMemsetAsync(zb[0], 0, need[1], c->stream));
  ok(cudaMemsetAsync(zb[1], 0, need[2], c->stream));
  ok(cudaMemcpyAsync(gx, grad_x, sizeof(double) * D * nV, cudaMemcpyDefault, c->stream));
  if (e != cudaSuccess) return c->fail(PC_ERR_CUDA, cudaGetErrorString(e));
  k_adj_init<<<std::max<long long>(1, std::min<long long>((D * nV + 255) / 256, 4096)), 256, 0, c->stream>>>(
      gx, xbar, nV, Vcap, D);
  const State st = pc_make_state(c);
  if (net.precision == PC_PREC_FP64) run_backward<double>(c, st, xbar, zb, gW);
  else run_backward<float>(c, st, xbar, zb, gW);
  ok(cudaGetLastError());
  ok(cudaMemcpyAsync(grad_params, gW, sizeof(double) * np, cudaMemcpyDefault, c->stream));
  ok(cudaStreamSynchronize(c->stream));
  if (e != cudaSuccess) return c->fail(PC_ERR_CUDA, cudaGetErrorString(e));
  return PC_OK;
}
