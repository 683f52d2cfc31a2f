// The Newton step to the exact vertex.
//
// A vertex lies on D zero entries (box facets or neuron pre-activations), all
// affine on the vertex's own piece: the activation pattern is its stored sign
// vector (a neuron is active iff its entry is +).  A forward pass from the
// stored coordinates gives the value g and gradient (float32, forward mode,
// D columns) of each zero entry; one Newton step on the D x D system
// A dx = -g lands on the exact vertex: the system is affine, and the step is
// small (the stored coordinates are FP32-accurate), so the float32 gradient
// adds only (1e-7 relative) x (step) to the result.  Used for
//   * the filtered sign predicate, values in float64 (redecide_batch,
//     pc_phases.cuh): the values of layer l at the exact vertex;
//   * the coordinate polish, values in float-float (newton_ff_warp below,
//     and the tiled k_polish_tile): the exact vertex itself.
#pragma once

#include "pc_device.cuh"

namespace pc {

// Upper bound of the dynamic shared memory of the one-warp-per-vertex polish.
constexpr int kPolishSmemMax = 220 * 1024;

struct NewtonOut {
  double z;             // value of the target neuron at the exact vertex
  double scale;         // sum of |terms| of that value (for the FP64 bound)
  double dlt[kMaxD];    // Newton step
  int ok;               // the zero set had D entries and the system was regular
  int nz;               // number of zero entries found
  int l_last;
  int pad;
};

// Added to a polyhedral domain's facet entry in a zero list once its row is
// in A / gv: newton_solve then takes it like a neuron's row.
constexpr int kFacetRow = 1 << 20;

// Rows of a polyhedral domain's facets among the zero entries s_zl[0, nzc)
// of vertex v: facet j has the value c_j - A_j x (x the stored coordinates)
// and the gradient -A_j; they go to the same rows A (q * D + d) and values
// gv[q] as the neurons', and the entry becomes j + kFacetRow (thread q of
// the group handles entry q).
__device__ inline void domain_facet_rows(const NetDesc& net, const State& st, long long v, int* s_zl, int nzc,
                                         int q, double* A, double* gv) {
  if (net.fA == nullptr || q >= nzc) return;
  const int j = s_zl[q];
  if (j >= net.m) return;
  const int D = net.D;
  const double* a = net.fA + (long long)j * D;
  double f = net.fc[j];
  for (int dd = 0; dd < D; ++dd) {
    f -= a[dd] * st.X[(long long)dd * st.Vcap + v];
    A[q * D + dd] = -a[dd];
  }
  gv[q] = f;
  s_zl[q] = j + kFacetRow;
}

// One Newton step on the D zero entries of vertex v: rows are the box
// facets' (+-e_d, value from the stored coordinate) and the neurons' and a
// polyhedral domain's facets' (gradient A,
// value gv); Gaussian elimination with partial pivoting in T.  The residuals
// are formed in float64; the step is small (the stored coordinates are
// FP32-accurate), so solving for it in float32 (the polish) loses only
// ~1e-7 x cond of the step itself, far below the coordinate tolerance.
template <typename T = double>
__device__ inline void newton_solve(const NetDesc& net, const State& st, long long v, const int* s_zl, int nz,
                                    const double* A, const double* gv, NewtonOut& o) {
  const int D = net.D, m = net.m;
  o.ok = 0;
  if (nz != D) return;
  T M[kMaxD][kMaxD + 1];
  for (int q = 0; q < D; ++q) {
    const int j = s_zl[q];
    if (j < m) {
      const int d = j >> 1;
      const double xd = st.X[(long long)d * st.Vcap + v];
      for (int dd = 0; dd < D; ++dd) M[q][dd] = T(0);
      M[q][d] = (j & 1) ? T(-1) : T(1);
      M[q][D] = static_cast<T>(-((j & 1) ? (net.hi[d] - xd) : (xd - net.lo[d])));
    } else {
      for (int dd = 0; dd < D; ++dd) M[q][dd] = static_cast<T>(A[q * D + dd]);
      M[q][D] = static_cast<T>(-gv[q]);
    }
  }
  for (int c = 0; c < D; ++c) {
    int piv = c;
    for (int r = c + 1; r < D; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (M[piv][c] == T(0)) return;
    if (piv != c)
      for (int k2 = 0; k2 <= D; ++k2) {
        const T t = M[c][k2];
        M[c][k2] = M[piv][k2];
        M[piv][k2] = t;
      }
    for (int r = c + 1; r < D; ++r) {
      const T f = M[r][c] / M[c][c];
      for (int k2 = c; k2 <= D; ++k2) M[r][k2] -= f * M[c][k2];
    }
  }
  T dl[kMaxD];
  for (int r = D - 1; r >= 0; --r) {
    T acc = M[r][D];
    for (int k2 = r + 1; k2 < D; ++k2) acc -= M[r][k2] * dl[k2];
    dl[r] = acc / M[r][r];
  }
  for (int r = 0; r < D; ++r) o.dlt[r] = static_cast<double>(dl[r]);
  o.ok = 1;
}

// ---------------------------------------------------------------------------
// Float-float evaluation for the coordinate polish.
//
// A value is the unevaluated sum hi + lo of two floats.  Dot products use
// the compensated scheme of Ogita, Rump and Oishi ("Accurate sum and dot
// product", 2005, Dot2): each product is split exactly with the FMA
// (p = a*b, e = fma(a, b, -p)), each addition of p to the running sum is
// split exactly with Knuth's TwoSum, and the error terms (plus the cross
// terms of the low parts) are summed in a float, which is as accurate as a
// dot product in twice the working precision (about 2^-44 of the sum of
// |terms| here).  Parameters come as (hi = float(w), lo = float(w - hi))
// pairs, inputs as hi = float(x), lo = float(x - hi).  On GB300 the FP32
// pipes run about 64x faster than the FP64 units.
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // Dekker; |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

__host__ __device__ constexpr int ff_ws_bytes(int mw, int D) {
  // a_hi, a_lo, an_hi, an_lo [mw]; J, Jn [mw x D] (float); then A [D x D],
  // gv [D] (double) and the sign words
  return ((4 * mw + 2 * mw * D + 1) / 2 * 2) * 4 + (D * D + D) * 8 + kMaxWords * 8;
}

// One warp: the Newton step of vertex v on its zero set (entries < e_end),
// values in float-float, gradients in float32.  P: the (head, remainder)
// parameters in the WT2 layout, in global or shared memory.  ws:
// ff_ws_bytes(mw, D) bytes of shared memory private to the warp, 8-byte
// aligned; s_zl: kMaxD + 2 ints.
// DOMAIN: the facets are a polyhedral domain's (net.fA), not the box's; a
// separate instantiation, so the box polish compiles as if it had none.
template <bool DOMAIN>
__device__ void newton_ff_warp(const NetDesc& net, const State& st, const float2* P, long long v, int e_end,
                               int mw, unsigned char* ws, int* s_zl, NewtonOut* out) {
  const int lane = threadIdx.x & 31;
  const int D = net.D, m = net.m;
  const long long Vcap = st.Vcap;
  float* ahi = reinterpret_cast<float*>(ws);
  float* alo = ahi + mw;
  float* nhi = alo + mw;
  float* nlo = nhi + mw;
  float* J = nlo + mw;
  float* Jn = J + mw * D;
  double* A = reinterpret_cast<double*>(ws + ((4 * mw + 2 * mw * D + 1) / 2 * 2) * 4);
  double* gv = A + D * D;
  uint64_t* sig = reinterpret_cast<uint64_t*>(gv + D);
  {
    const uint64_t word = lane < net.S ? st.SIG[(long long)lane * Vcap + v] : 0ull;
    if (lane < net.S) sig[lane] = word;
    const uint64_t zm = lane < net.S ? zero_mask(word, lane, e_end) : 0ull;
    const int c = __popcll(zm);
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    int k = x - c;
    uint64_t mm = zm;
    while (mm) {
      const int bit = __ffsll((long long)mm) - 1;
      if (k < kMaxD) s_zl[k] = lane * 32 + bit / 2;
      ++k;
      mm &= mm - 1;
    }
    if (lane == 31) s_zl[kMaxD] = x;
  }
  if (lane < D) {
    const double xd = st.X[(long long)lane * Vcap + v];
    const float h = static_cast<float>(xd);
    ahi[lane] = h;
    alo[lane] = static_cast<float>(xd - static_cast<double>(h));
    for (int dd = 0; dd < D; ++dd) J[lane * D + dd] = (lane == dd) ? 1.f : 0.f;
  }
  __syncwarp();
  const int nz = s_zl[kMaxD];
  const int nzc = nz < D ? nz : D;
  int l_last = -1;  // highest layer among the zero-set neurons
  for (int q = 0; q < nzc; ++q) {
    const int h = s_zl[q] - m;
    if (h < 0) continue;
    int l = 0;
    while (l + 1 < net.L && h >= net.off[l + 1]) ++l;
    if (l > l_last) l_last = l;
  }
  int in = D;
  for (int k = 0; k <= l_last; ++k) {
    const int H = net.w[k + 1];
    const float2* Wt = P + net.wofs[k];  // [in][H]: lanes read consecutive neurons
    for (int r = lane; r < H; r += 32) {
      const int entry = m + net.off[k] + r;
      int zpos = -1;
      for (int q = 0; q < nzc; ++q)
        if (s_zl[q] == entry) zpos = q;
      if (!(k < l_last || zpos >= 0)) continue;
      const float2 bj = P[net.bofs[k] + r];
      float sum = bj.x, err = bj.y;
      float jd[kMaxD];
#pragma unroll
      for (int dd = 0; dd < kMaxD; ++dd) jd[dd] = 0.f;
      for (int c = 0; c < in; ++c) {
        const float2 w = Wt[(long long)c * H + r];
        const float xh = w.x, xl = w.y, yh = ahi[c], yl = alo[c];
        const float p = xh * yh;
        float e = fmaf(xh, yh, -p);  // exact low part of the product
        e = fmaf(xh, yl, e);         // cross terms of the low parts
        e = fmaf(xl, yh, e);
        const float t = sum + p;     // TwoSum(sum, p): t + its error is exact
        const float bb = t - sum;
        err += ((sum - (t - bb)) + (p - bb)) + e;
        sum = t;
#pragma unroll
        for (int dd = 0; dd < kMaxD; ++dd)
          if (dd < D) jd[dd] = fmaf(xh, J[c * D + dd], jd[dd]);
      }
      const ff z = ff_fast_two_sum(sum, err);
      if (zpos >= 0) {
        gv[zpos] = static_cast<double>(z.hi) + static_cast<double>(z.lo);
        for (int dd = 0; dd < D; ++dd) A[zpos * D + dd] = jd[dd];
      }
      if (k < l_last) {
        const bool act = ((sig[entry >> 5] >> (2 * (entry & 31))) & 3ull) == kPlus;
        nhi[r] = act ? z.hi : 0.f;
        nlo[r] = act ? z.lo : 0.f;
        for (int dd = 0; dd < D; ++dd) Jn[r * D + dd] = act ? jd[dd] : 0.f;
      }
    }
    __syncwarp();
    float* t0 = ahi; ahi = nhi; nhi = t0;
    float* t1 = alo; alo = nlo; nlo = t1;
    float* t2 = J; J = Jn; Jn = t2;
    in = H;
  }
  if (DOMAIN) {
    domain_facet_rows(net, st, v, s_zl, nzc, lane, A, gv);
    __syncwarp();
  }
  if (lane == 0) {
    NewtonOut o{};
    o.nz = nz;
    o.l_last = l_last;
    newton_solve<float>(net, st, v, s_zl, nz, A, gv, o);
    *out = o;
  }
  __syncwarp();
}

}  // namespace pc
