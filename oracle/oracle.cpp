// FP64 CPU oracle for edge-subdivision polyhedral-complex extraction.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark load this library.  It is written from the
// paper (Berzins, "Polyhedral Complex Extraction from ReLU Networks using Edge
// Subdivision", ICML 2023) and shares no code, header, table or helper with the
// CUDA path.  Plain, slow and single-threaded on purpose: std::vector state,
// int8 sign vectors with values {-1, 0, +1}, std::map pairing, double
// arithmetic throughout.
//
// Contents
//   orc_extract   edge subdivision, steps (1)-(5) of Section 4.2 per neuron,
//                 repeated for every neuron of every layer.
//   orc_faces     k-cell counts by repeated perturbation (Section 4.1), used
//                 for the Euler-characteristic check.
//   orc_poset     the face poset itself (Section 4.1): every level's cells
//                 and, for each cell, the cells one level up that contain it
//                 (its parents), by perturbing each of its zeros.
//   orc_brute     the complex from its definition (Section 3.3-3.4): every
//                 D-subset of {box facets, neuron zero sets} under every
//                 activation pattern, plus edges by a midpoint test.
//   orc_grad      gradient of a vertex-position loss through the
//                 implicit-function theorem on each vertex's D zero functions.
//   domains       (orc_extract_domain, orc_brute_domain) a bounded polyhedral
//                 domain of m half-spaces c - A x >= 0 (Section 4.1) with
//                 the caller's initial 1-skeleton, e.g. a simplex.
//   pruning       (orc_extract with prune = 1) the pruning during edge
//                 subdivision of Section 5.4.2 for level-set extraction: after
//                 each layer but the last, edges whose two vertices have the
//                 same signs w.r.t. all future neurons are dropped, and so are
//                 the vertices left without an edge.
//
// Readings taken where the paper is silent (same rule on the GPU side):
//   * W[l] is out x in and z = W x + b (the network form of Eq. 4, not the
//     w.x - b hyperplane form of Section 3.1).
//   * Sign-vector order: the m = 2D box facets first (2d: x_d - lo_d >= 0,
//     2d+1: hi_d - x_d >= 0, + meaning inside), then every neuron layer by
//     layer, the output layer included.
//   * Step (1) evaluates the network from the vertex coordinates at the start
//     of each layer, keeping each vertex on its own affine piece by using its
//     stored sign vector as the activation pattern (active iff +); inside a
//     layer the new vertices interpolate coordinates and values (Fig. 3).
//   * A pre-activation that is exactly 0.0 is a genericity violation: it is
//     counted and treated as +.
//   * Edge sign vector = join of its endpoints (entrywise: the nonzero value
//     where one is 0, the common value otherwise).
//
// What pins each function to something other than itself (CPU tests):
//   orc_extract   the brute force on tiny deep nets; the clipped
//                 line-arrangement closed form V = 4 + 2n + I, E = 4 + 3n + 2I;
//                 C(n, D) interior vertices of a generic arrangement; the
//                 clipped-arrangement vertex census; an independent
//                 layer-by-layer breakpoint scan at D = 1; zero counts,
//                 degrees and bookkeeping of Section 4.1; the zero residual
//                 of Section 5.1.1 and a direct D x D solve; invariance under
//                 neuron permutation and positive rescaling; the paper's
//                 printed 2D counts against the line-arrangement identity.
//   orc_faces     the region count of clipped generic arrangements (1 + the
//                 k-subsets whose flat meets the open domain, by a linear
//                 program per flat) and Euler characteristic 1.
//   orc_poset     the perturbed vertices against the independently built
//                 edges; the face relation of polyhedral complexes: every
//                 interval of length two is a diamond (exactly two cells in
//                 between), the boundary of every k-cell is a (k-1)-sphere
//                 (its faces' Euler characteristic is 1 - (-1)^k); and the
//                 geometry: the centroid of a cell's vertices, evaluated by a
//                 forward pass, has the cell's sign vector.
//   orc_brute     the definition itself; it agrees with orc_extract and
//                 with the closed forms above.
//   orc_grad      central finite differences of FP64 extractions.
//   domains       the box as half-spaces reproduces the box bit for bit;
//                 brute force on simplices and a corner-cut cube; the line
//                 arrangement in a triangle; Euler characteristic 1.
//   pruning       a sub-complex of the full extraction with the same level
//                 set, equal to the brute-force level set on tiny nets.
// No function is parity unpinned.  The vertex and edge counts of the
// benchmark workloads themselves are: the paper prints none for them.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

namespace {

struct Net {
  int L = 0;
  std::vector<int> w;                  // widths, w[0] = D
  std::vector<std::vector<double>> W;  // W[l]: w[l+1] x w[l], row-major
  std::vector<std::vector<double>> b;  // b[l]: w[l+1]
  std::vector<int> off;                // first global neuron index of layer l
  int N = 0;                           // total neurons
};

Net make_net(int L, const int32_t* widths, const double* params) {
  Net net;
  net.L = L;
  net.w.assign(widths, widths + L + 1);
  size_t p = 0;
  int n = 0;
  for (int l = 0; l < L; ++l) {
    const int o = net.w[l + 1], i = net.w[l];
    net.W.emplace_back(params + p, params + p + size_t(o) * i);
    p += size_t(o) * i;
    net.b.emplace_back(params + p, params + p + o);
    p += o;
    net.off.push_back(n);
    n += o;
  }
  net.N = n;
  return net;
}

struct Result {
  int D = 0, m = 0, N = 0, P = 0;
  std::vector<double> X;                // nV * D
  std::vector<int8_t> S;                // nV * P
  std::vector<std::array<int32_t, 2>> E;
  std::vector<int64_t> stats;           // per neuron: nsplit, nkeys, npairs, ndegenerate
  std::vector<int64_t> layer_counts;    // per layer: vertices, edges after it (and its pruning)
  int status = 0;                       // 0 ok, 4 degenerate, 5 pairing
  std::string err;
  int64_t nV() const { return int64_t(X.size()) / D; }
};

inline int sgn_of(double z, int64_t& degenerate) {
  if (z > 0.0) return 1;
  if (z < 0.0) return -1;
  ++degenerate;  // exact zero: non-generic arrangement
  return 1;
}

// Pre-activations of layer `l` at point x, with layers < l using the stored
// activation pattern `s` (entry m + off[k] + j active iff it is +).
void layer_preact(const Net& net, int m, int l, const double* x, const int8_t* s,
                  std::vector<double>& z) {
  std::vector<double> a(x, x + net.w[0]);
  for (int k = 0; k <= l; ++k) {
    const int o = net.w[k + 1], in = net.w[k];
    z.assign(o, 0.0);
    for (int r = 0; r < o; ++r) {
      double acc = net.b[k][r];
      for (int c = 0; c < in; ++c) acc += net.W[k][size_t(r) * in + c] * a[c];
      z[r] = acc;
    }
    if (k == l) return;
    a.assign(o, 0.0);
    for (int r = 0; r < o; ++r) a[r] = (s[m + net.off[k] + r] == 1) ? z[r] : 0.0;
  }
}

// Signs of the neurons of layers > l at x: layers <= l use the stored
// activation pattern s (active iff +), later layers the real ReLU of the
// values computed here.  Returns false if a future value is exactly 0.
bool future_signs(const Net& net, int m, int l, const double* x, const int8_t* s, std::vector<int8_t>& fs) {
  std::vector<double> a(x, x + net.w[0]), z;
  fs.clear();
  bool generic = true;
  for (int k = 0; k < net.L; ++k) {
    const int o = net.w[k + 1], in = net.w[k];
    z.assign(o, 0.0);
    for (int r = 0; r < o; ++r) {
      double acc = net.b[k][r];
      for (int c = 0; c < in; ++c) acc += net.W[k][size_t(r) * in + c] * a[c];
      z[r] = acc;
    }
    a.assign(o, 0.0);
    for (int r = 0; r < o; ++r) {
      if (k <= l) {
        a[r] = (s[m + net.off[k] + r] == 1) ? z[r] : 0.0;
      } else {
        if (z[r] == 0.0) generic = false;
        fs.push_back(z[r] > 0.0 ? 1 : (z[r] < 0.0 ? -1 : 0));
        a[r] = z[r] > 0.0 ? z[r] : 0.0;
      }
    }
  }
  return generic;
}

// Pruning during edge subdivision (Section 5.4.2), after layer l: an edge
// whose vertices have the same signs w.r.t. every future neuron is crossed by
// no future folded hyperplane (along the edge each next layer is affine, and
// by induction so are the later ones once no earlier neuron splits it), so it
// cannot meet the zero set of the output; it is dropped, and so is every
// vertex left without an edge.  An exactly zero future value keeps its edges.
void prune_after_layer(const Net& net, int l, Result& R) {
  const int D = R.D, m = R.m, P = R.P;
  const int64_t nV = R.nV();
  std::vector<std::vector<int8_t>> fs(nV);
  std::vector<char> generic(nV);
  for (int64_t v = 0; v < nV; ++v)
    generic[v] = future_signs(net, m, l, &R.X[size_t(v) * D], &R.S[size_t(v) * P], fs[v]);
  std::vector<std::array<int32_t, 2>> kept;
  std::vector<char> used(nV, 0);
  for (const auto& e : R.E) {
    if (generic[e[0]] && generic[e[1]] && fs[e[0]] == fs[e[1]]) continue;
    kept.push_back(e);
    used[e[0]] = used[e[1]] = 1;
  }
  std::vector<int32_t> idx(nV, -1);
  std::vector<double> X;
  std::vector<int8_t> S;
  int32_t k = 0;
  for (int64_t v = 0; v < nV; ++v) {
    if (!used[v]) continue;
    idx[v] = k++;
    X.insert(X.end(), R.X.begin() + size_t(v) * D, R.X.begin() + size_t(v + 1) * D);
    S.insert(S.end(), R.S.begin() + size_t(v) * P, R.S.begin() + size_t(v + 1) * P);
  }
  for (auto& e : kept) e = {idx[e[0]], idx[e[1]]};
  R.X.swap(X);
  R.S.swap(S);
  R.E.swap(kept);
}

void subdivide(const Net& net, int max_neurons, Result& R, bool prune);

// Edge subdivision (Section 4.2) on the box [lo, hi]^D, all neurons in index
// order (or the first `max_neurons` of them when max_neurons >= 0).
void extract(const Net& net, const double* lo, const double* hi, int max_neurons, Result& R, bool prune) {
  const int D = net.w[0], m = 2 * D, N = net.N, P = m + N;
  R.D = D; R.m = m; R.N = N; R.P = P;
  R.stats.assign(size_t(N) * 4, 0);
  // Step 0: the box [lo, hi]^D as the initial 1-skeleton.  Boundary entries
  // come first; a corner lies on exactly one of the two facets of each axis.
  const int nc = 1 << D;
  for (int c = 0; c < nc; ++c) {
    for (int d = 0; d < D; ++d) R.X.push_back(((c >> d) & 1) ? hi[d] : lo[d]);
    std::vector<int8_t> s(P, 0);
    for (int d = 0; d < D; ++d) {
      const bool up = (c >> d) & 1;
      s[2 * d] = up ? 1 : 0;      // x_d - lo_d
      s[2 * d + 1] = up ? 0 : 1;  // hi_d - x_d
    }
    R.S.insert(R.S.end(), s.begin(), s.end());
  }
  for (int d = 0; d < D; ++d)
    for (int c = 0; c < nc; ++c)
      if (!((c >> d) & 1)) R.E.push_back({int32_t(c), int32_t(c | (1 << d))});
  subdivide(net, max_neurons, R, prune);
}

// A bounded polyhedral domain given by m affine half-spaces (Section 4.1):
// facet i is c_i - a_i . x >= 0 (sign entry i, + inside).
struct Domain {
  int m = 0;
  std::vector<double> A;  // m x D, row-major
  std::vector<double> c;  // m
  double value(int i, int D, const double* x) const {
    double v = c[i];
    for (int d = 0; d < D; ++d) v -= A[size_t(i) * D + d] * x[d];
    return v;
  }
  double scale(int i, int D, const double* x) const {
    double s = std::fabs(c[i]);
    for (int d = 0; d < D; ++d) s += std::fabs(A[size_t(i) * D + d] * x[d]);
    return s;
  }
};

// Edge subdivision on a polyhedral domain whose 1-skeleton (nv0 vertices X0,
// ne0 edges E0) the caller gives: the facet entries of each initial vertex are
// 0 on the facet (|value| <= 1e-12 of its scale) and + inside.  The facets'
// zeros are perturbed only toward + in step (5), as for the box.
void extract_domain(const Net& net, const Domain& dom, int64_t nv0, const double* X0, int64_t ne0,
                    const int32_t* E0, int max_neurons, Result& R, bool prune) {
  const int D = net.w[0], m = dom.m, N = net.N, P = m + N;
  R.D = D; R.m = m; R.N = N; R.P = P;
  R.stats.assign(size_t(N) * 4, 0);
  for (int64_t v = 0; v < nv0; ++v) {
    const double* x = X0 + size_t(v) * D;
    R.X.insert(R.X.end(), x, x + D);
    std::vector<int8_t> s(P, 0);
    for (int i = 0; i < m; ++i) {
      const double f = dom.value(i, D, x);
      if (std::fabs(f) <= 1e-12 * dom.scale(i, D, x)) {
        s[i] = 0;
      } else if (f > 0) {
        s[i] = 1;
      } else {
        R.status = 1;
        R.err = "an initial vertex lies outside the domain";
        s[i] = 1;
      }
    }
    R.S.insert(R.S.end(), s.begin(), s.end());
  }
  for (int64_t e = 0; e < ne0; ++e) R.E.push_back({E0[2 * e], E0[2 * e + 1]});
  if (R.status == 0) subdivide(net, max_neurons, R, prune);
}

// The neuron steps of edge subdivision on the current R (Section 4.2).
void subdivide(const Net& net, int max_neurons, Result& R, bool prune) {
  const int D = R.D, m = R.m, P = R.P;
  std::vector<double> Z, zt;  // Z: nV * H values of the current layer
  for (int l = 0; l < net.L; ++l) {
    const int H = net.w[l + 1];
    // Step (1): evaluate the network at all vertices (layer start).
    const int64_t nV0 = R.nV();
    Z.assign(size_t(nV0) * H, 0.0);
    for (int64_t v = 0; v < nV0; ++v) {
      layer_preact(net, m, l, &R.X[size_t(v) * D], &R.S[size_t(v) * P], zt);
      std::copy(zt.begin(), zt.end(), Z.begin() + size_t(v) * H);
    }
    for (int i = 0; i < H; ++i) {
      const int n = net.off[l] + i;
      if (max_neurons >= 0 && n >= max_neurons) return;
      const int e = m + n;  // sign-vector entry of this neuron
      int64_t* st = &R.stats[size_t(n) * 4];
      const int64_t nV = R.nV();
      // Step (2): signs of all vertices w.r.t. the folded hyperplane.
      for (int64_t v = 0; v < nV; ++v) R.S[size_t(v) * P + e] = int8_t(sgn_of(Z[size_t(v) * H + i], st[3]));
      // Step (3): splitting edges have endpoints of opposite sign.
      std::vector<int64_t> split;
      for (size_t k = 0; k < R.E.size(); ++k)
        if (R.S[size_t(R.E[k][0]) * P + e] != R.S[size_t(R.E[k][1]) * P + e]) split.push_back(int64_t(k));
      st[0] = int64_t(split.size());
      // Step (4): new vertex by interpolation; split the edge into E+ and E-.
      std::vector<int32_t> newv(split.size());
      for (size_t k = 0; k < split.size(); ++k) {
        const int32_t u = R.E[split[k]][0], w = R.E[split[k]][1];
        const int32_t p = (R.S[size_t(u) * P + e] == 1) ? u : w;  // V+
        const int32_t q = (p == u) ? w : u;                        // V-
        const double a = Z[size_t(p) * H + i], bq = Z[size_t(q) * H + i];
        const double t = a / (a - bq);
        const int32_t v0 = int32_t(R.nV());
        for (int d = 0; d < D; ++d) {
          const double xp = R.X[size_t(p) * D + d], xq = R.X[size_t(q) * D + d];
          R.X.push_back(xp + t * (xq - xp));
        }
        for (int j = 0; j < H; ++j) {
          const double zp = Z[size_t(p) * H + j], zq = Z[size_t(q) * H + j];
          Z.push_back(j == i ? 0.0 : zp + t * (zq - zp));
        }
        std::vector<int8_t> s0(P, 0);
        for (int j = 0; j < e; ++j) {
          const int8_t sp = R.S[size_t(p) * P + j], sq = R.S[size_t(q) * P + j];
          if (sp != 0 && sq != 0 && sp != sq) {
            R.status = 5;
            R.err = "edge endpoints disagree on a processed entry";
          }
          s0[j] = sp != 0 ? sp : sq;
        }
        s0[e] = 0;
        R.S.insert(R.S.end(), s0.begin(), s0.end());
        R.E[split[k]] = {p, v0};
        R.E.push_back({q, v0});
        newv[k] = v0;
      }
      // Step (5): parent 2-faces of each splitting edge by perturbing each of
      // its zeros (boundary zeros only toward +); each splitting 2-face occurs
      // exactly twice, and its two new vertices form an intersecting edge.
      std::map<std::vector<int8_t>, std::vector<int32_t>> faces;
      for (size_t k = 0; k < split.size(); ++k) {
        const int8_t* s0 = &R.S[size_t(newv[k]) * P];
        std::vector<int8_t> F(s0, s0 + e);  // the splitting edge's sign vector
        for (int j = 0; j < e; ++j) {
          if (F[j] != 0) continue;
          for (int sgn = 1; sgn >= -1; sgn -= 2) {
            if (j < m && sgn < 0) continue;
            F[j] = int8_t(sgn);
            faces[F].push_back(newv[k]);
            ++st[1];
            F[j] = 0;
          }
        }
      }
      for (auto& kv : faces) {
        if (kv.second.size() != 2) {
          R.status = 5;
          R.err = "a splitting 2-face does not occur exactly twice";
          continue;
        }
        R.E.push_back({kv.second[0], kv.second[1]});
        ++st[2];
      }
      if (st[3] != 0 && R.status == 0) {
        R.status = 4;
        R.err = "exact zero pre-activation (non-generic arrangement)";
      }
    }
    if (prune && l + 1 < net.L) prune_after_layer(net, l, R);
    R.layer_counts.push_back(R.nV());
    R.layer_counts.push_back(int64_t(R.E.size()));
  }
}

// ---- k-cells by perturbation (Section 4.1) ---------------------------------

// The face poset: level 0 the vertices' sign vectors, level 1 the edges' (the
// join of their two vertices), level k >= 2 every perturbation of a zero of a
// (k-1)-cell (a box facet's zero only toward +, the inside); each level sorted
// (entries compared as -1 < 0 < +1).  The incidence of level k < D lists for
// each k-cell the (k+1)-cells that contain it: its zeros perturbed one at a
// time in entry order, + before -.  A perturbation of a vertex that is not an
// edge fails the poset (status 5): the vertices' perturbations are checked
// against the edges built from the extraction.
struct Poset {
  int D = 0, P = 0;
  std::vector<std::vector<std::vector<int8_t>>> cells;
  std::vector<std::vector<int64_t>> row_ptr, cols;
  int status = 0;
  std::string err;
};

Poset* build_poset(const Result& R) {
  auto* Q = new Poset;
  const int D = R.D, m = R.m, P = R.P;
  Q->D = D;
  Q->P = P;
  Q->cells.resize(D + 1);
  std::set<std::vector<int8_t>> lev;
  for (int64_t v = 0; v < R.nV(); ++v)
    lev.insert(std::vector<int8_t>(R.S.begin() + v * P, R.S.begin() + (v + 1) * P));
  Q->cells[0].assign(lev.begin(), lev.end());
  lev.clear();
  for (auto& ed : R.E) {
    std::vector<int8_t> s(P);
    for (int j = 0; j < P; ++j) {
      const int8_t a = R.S[size_t(ed[0]) * P + j], b = R.S[size_t(ed[1]) * P + j];
      s[j] = a != 0 ? a : b;
    }
    lev.insert(s);
  }
  if (D >= 1) Q->cells[1].assign(lev.begin(), lev.end());
  for (int k = 2; k <= D; ++k) {
    lev.clear();
    for (auto& c : Q->cells[k - 1]) {
      std::vector<int8_t> s = c;
      for (int j = 0; j < P; ++j) {
        if (c[j] != 0) continue;
        for (int sg = 1; sg >= -1; sg -= 2) {
          if (j < m && sg < 0) continue;
          s[j] = int8_t(sg);
          lev.insert(s);
          s[j] = 0;
        }
      }
    }
    Q->cells[k].assign(lev.begin(), lev.end());
  }
  Q->row_ptr.resize(D);
  Q->cols.resize(D);
  for (int k = 0; k < D; ++k) {
    const auto& up = Q->cells[k + 1];
    auto& rp = Q->row_ptr[k];
    auto& cl = Q->cols[k];
    rp.assign(1, 0);
    for (auto& c : Q->cells[k]) {
      std::vector<int8_t> s = c;
      for (int j = 0; j < P; ++j) {
        if (c[j] != 0) continue;
        for (int sg = 1; sg >= -1; sg -= 2) {
          if (j < m && sg < 0) continue;
          s[j] = int8_t(sg);
          const auto it = std::lower_bound(up.begin(), up.end(), s);
          if (it == up.end() || *it != s) {
            Q->status = 5;
            Q->err = "a perturbation of a " + std::to_string(k) + "-cell is not a " + std::to_string(k + 1) + "-cell";
          } else {
            cl.push_back(int64_t(it - up.begin()));
          }
          s[j] = 0;
        }
      }
      rp.push_back(int64_t(cl.size()));
    }
  }
  return Q;
}

int64_t faces(const Result& R, int64_t* f_out) {
  const int D = R.D, m = R.m, P = R.P;
  std::set<std::vector<int8_t>> cur, nxt;
  f_out[0] = R.nV();
  for (auto& ed : R.E) {
    std::vector<int8_t> s(P);
    for (int j = 0; j < P; ++j) {
      const int8_t a = R.S[size_t(ed[0]) * P + j], b = R.S[size_t(ed[1]) * P + j];
      s[j] = a != 0 ? a : b;
    }
    cur.insert(s);
  }
  f_out[1] = int64_t(cur.size());
  int64_t chi = f_out[0] - f_out[1];
  for (int k = 2; k <= D; ++k) {
    nxt.clear();
    for (auto& c : cur) {
      std::vector<int8_t> s = c;
      for (int j = 0; j < P; ++j) {
        if (c[j] != 0) continue;
        for (int sgn = 1; sgn >= -1; sgn -= 2) {
          if (j < m && sgn < 0) continue;
          s[j] = int8_t(sgn);
          nxt.insert(s);
          s[j] = 0;
        }
      }
    }
    f_out[k] = int64_t(nxt.size());
    chi += (k % 2 == 0) ? f_out[k] : -f_out[k];
    cur.swap(nxt);
  }
  return chi;
}

// ---- brute force from the definition (Sections 3.3-3.4) --------------------

// Real forward pass with ReLU(z) = max(0, z); returns every neuron's value.
void forward_all(const Net& net, const double* x, std::vector<double>& zall) {
  std::vector<double> a(x, x + net.w[0]), z;
  zall.clear();
  for (int l = 0; l < net.L; ++l) {
    const int o = net.w[l + 1], in = net.w[l];
    z.assign(o, 0.0);
    for (int r = 0; r < o; ++r) {
      double acc = net.b[l][r];
      for (int c = 0; c < in; ++c) acc += net.W[l][size_t(r) * in + c] * a[c];
      z[r] = acc;
    }
    zall.insert(zall.end(), z.begin(), z.end());
    a.assign(o, 0.0);
    for (int r = 0; r < o; ++r) a[r] = z[r] > 0 ? z[r] : 0.0;
  }
}

// Solve A x = rhs (n x n, row-major) by Gaussian elimination with partial pivoting.
bool solve(int n, std::vector<double> A, std::vector<double> rhs, std::vector<double>& x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[size_t(r) * n + c]) > std::fabs(A[size_t(piv) * n + c])) piv = r;
    if (std::fabs(A[size_t(piv) * n + c]) < 1e-300) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[size_t(c) * n + k], A[size_t(piv) * n + k]);
      std::swap(rhs[c], rhs[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[size_t(r) * n + c] / A[size_t(c) * n + c];
      for (int k = c; k < n; ++k) A[size_t(r) * n + k] -= f * A[size_t(c) * n + k];
      rhs[r] -= f * rhs[c];
    }
  }
  x.assign(n, 0.0);
  for (int r = n - 1; r >= 0; --r) {
    double acc = rhs[r];
    for (int k = r + 1; k < n; ++k) acc -= A[size_t(r) * n + k] * x[k];
    x[r] = acc / A[size_t(r) * n + r];
  }
  return true;
}

// Value of entry j (facet or neuron) at x given all neuron values zall.
inline double entry_value(int j, int D, const Domain& dom, const double* x, const std::vector<double>& zall) {
  if (j < dom.m) return dom.value(j, D, x);
  return zall[j - dom.m];
}

// The box [lo, hi]^D as half-spaces: 2d: x_d - lo_d >= 0, 2d+1: hi_d - x_d >= 0.
Domain box_domain(int D, const double* lo, const double* hi) {
  Domain dom;
  dom.m = 2 * D;
  dom.A.assign(size_t(2 * D) * D, 0.0);
  dom.c.assign(2 * D, 0.0);
  for (int d = 0; d < D; ++d) {
    dom.A[size_t(2 * d) * D + d] = -1.0;
    dom.c[2 * d] = -lo[d];
    dom.A[size_t(2 * d + 1) * D + d] = 1.0;
    dom.c[2 * d + 1] = hi[d];
  }
  return dom;
}

int brute_domain(const Net& net, const Domain& dom, double tol, Result& R);

int brute(const Net& net, const double* lo, const double* hi, double tol, Result& R) {
  return brute_domain(net, box_domain(net.w[0], lo, hi), tol, R);
}

int brute_domain(const Net& net, const Domain& dom, double tol, Result& R) {
  const int D = net.w[0], m = dom.m, N = net.N, P = m + N;
  R.D = D; R.m = m; R.N = N; R.P = P;
  int Nh = 0;  // neurons whose state changes the affine map: all but the last layer
  for (int l = 0; l + 1 < net.L; ++l) Nh += net.w[l + 1];
  if (Nh > 24 || P > 64) return 1;
  std::map<std::vector<int8_t>, std::vector<double>> verts;
  std::vector<double> G(size_t(P) * D), c(P), zall, x;
  std::vector<int> idx(D);
  for (uint64_t pat = 0; pat < (uint64_t(1) << Nh); ++pat) {
    // Affine map of every entry under activation pattern `pat`; facet i is
    // (-a_i) . x + c_i.
    for (int i = 0; i < m; ++i) {
      for (int k = 0; k < D; ++k) G[size_t(i) * D + k] = -dom.A[size_t(i) * D + k];
      c[i] = dom.c[i];
    }
    std::vector<double> aG(size_t(D) * D, 0.0), ac(D, 0.0);  // input: identity map
    for (int d = 0; d < D; ++d) aG[size_t(d) * D + d] = 1.0;
    int in = D;
    for (int l = 0; l < net.L; ++l) {
      const int o = net.w[l + 1];
      std::vector<double> zG(size_t(o) * D, 0.0), zc(o, 0.0);
      for (int r = 0; r < o; ++r) {
        zc[r] = net.b[l][r];
        for (int q = 0; q < in; ++q) {
          const double wv = net.W[l][size_t(r) * in + q];
          zc[r] += wv * ac[q];
          for (int k = 0; k < D; ++k) zG[size_t(r) * D + k] += wv * aG[size_t(q) * D + k];
        }
        const int j = m + net.off[l] + r;
        for (int k = 0; k < D; ++k) G[size_t(j) * D + k] = zG[size_t(r) * D + k];
        c[j] = zc[r];
      }
      aG.assign(size_t(o) * D, 0.0);
      ac.assign(o, 0.0);
      for (int r = 0; r < o; ++r) {
        const int h = net.off[l] + r;
        if (h < Nh && ((pat >> h) & 1)) {
          for (int k = 0; k < D; ++k) aG[size_t(r) * D + k] = zG[size_t(r) * D + k];
          ac[r] = zc[r];
        }
      }
      in = o;
    }
    // Every D-subset of entries: solve, then check against a real forward pass.
    for (int k = 0; k < D; ++k) idx[k] = k;
    while (true) {
      std::vector<double> A(size_t(D) * D), rhs(D);
      for (int r = 0; r < D; ++r) {
        for (int k = 0; k < D; ++k) A[size_t(r) * D + k] = G[size_t(idx[r]) * D + k];
        rhs[r] = -c[idx[r]];
      }
      if (solve(D, A, rhs, x)) {
        forward_all(net, x.data(), zall);
        bool ok = true;
        std::vector<int8_t> s(P, 0);
        int zi = 0;
        for (int j = 0; j < P && ok; ++j) {
          const double val = entry_value(j, D, dom, x.data(), zall);
          const bool in_set = (zi < D && idx[zi] == j);
          if (in_set) {
            ++zi;
            if (std::fabs(val) > tol) ok = false;
            s[j] = 0;
          } else {
            if (std::fabs(val) <= tol) { ok = false; break; }
            s[j] = val > 0 ? 1 : -1;
            if (j < m && s[j] < 0) ok = false;  // outside the box
            const int h = j - m;
            if (j >= m && h < Nh && (((pat >> h) & 1) != 0) != (s[j] > 0)) ok = false;
          }
        }
        if (ok && !verts.count(s)) verts[s] = x;
      }
      int r = D - 1;
      while (r >= 0 && idx[r] == P - D + r) --r;
      if (r < 0) break;
      ++idx[r];
      for (int k = r + 1; k < D; ++k) idx[k] = idx[k - 1] + 1;
    }
  }
  for (auto& kv : verts) {
    R.X.insert(R.X.end(), kv.second.begin(), kv.second.end());
    R.S.insert(R.S.end(), kv.first.begin(), kv.first.end());
  }
  // Edges: conformal vertex pairs whose join has D-1 zeros and whose midpoint
  // lies in the open cell that the join names.
  const int64_t nV = R.nV();
  std::vector<double> mid(D);
  for (int64_t u = 0; u < nV; ++u) {
    for (int64_t w = u + 1; w < nV; ++w) {
      const int8_t* su = &R.S[size_t(u) * P];
      const int8_t* sw = &R.S[size_t(w) * P];
      std::vector<int8_t> j8(P);
      int zeros = 0;
      bool conformal = true;
      for (int j = 0; j < P; ++j) {
        if (su[j] != 0 && sw[j] != 0 && su[j] != sw[j]) { conformal = false; break; }
        j8[j] = su[j] != 0 ? su[j] : sw[j];
        zeros += (j8[j] == 0);
      }
      if (!conformal || zeros != D - 1) continue;
      for (int d = 0; d < D; ++d) mid[d] = 0.5 * (R.X[size_t(u) * D + d] + R.X[size_t(w) * D + d]);
      forward_all(net, mid.data(), zall);
      bool ok = true;
      for (int j = 0; j < P && ok; ++j) {
        const double val = entry_value(j, D, dom, mid.data(), zall);
        if (j8[j] == 0) ok = std::fabs(val) <= tol;
        else ok = (std::fabs(val) > tol) && ((val > 0) == (j8[j] > 0));
      }
      if (ok) R.E.push_back({int32_t(u), int32_t(w)});
    }
  }
  return 0;
}

// ---- implicit-function gradient ------------------------------------------------
//
// Each vertex x solves g_r(x; theta) = 0 for its D zero entries r, where g_r
// is a box facet (independent of theta) or a neuron pre-activation on the
// vertex's own affine piece.  With A = dg/dx (D x D) and a loss gradient gx:
//   dL/dtheta = -lambda^T dg/dtheta,   A^T lambda = gx.
int grad(const Net& net, const Result& R, const double* gx, double* dtheta) {
  const int D = R.D, m = R.m, P = R.P, L = net.L;
  std::vector<size_t> wofs(L), bofs(L);
  size_t p = 0;
  for (int l = 0; l < L; ++l) {
    wofs[l] = p;
    p += size_t(net.w[l + 1]) * net.w[l];
    bofs[l] = p;
    p += net.w[l + 1];
  }
  std::fill(dtheta, dtheta + p, 0.0);
  const int64_t nV = R.nV();
  for (int64_t v = 0; v < nV; ++v) {
    const double* g = gx + size_t(v) * D;
    bool any = false;
    for (int d = 0; d < D; ++d) any |= (g[d] != 0.0);
    if (!any) continue;
    const double* x = &R.X[size_t(v) * D];
    const int8_t* s = &R.S[size_t(v) * P];
    // Forward with Jacobians under the vertex's pattern.
    std::vector<std::vector<double>> act(L + 1), zG(L);
    act[0].assign(x, x + D);
    std::vector<double> aG(size_t(D) * D, 0.0);
    for (int d = 0; d < D; ++d) aG[size_t(d) * D + d] = 1.0;
    for (int l = 0; l < L; ++l) {
      const int o = net.w[l + 1], in = net.w[l];
      std::vector<double> z(o);
      zG[l].assign(size_t(o) * D, 0.0);
      for (int r = 0; r < o; ++r) {
        double acc = net.b[l][r];
        for (int q = 0; q < in; ++q) {
          const double wv = net.W[l][size_t(r) * in + q];
          acc += wv * act[l][q];
          for (int k = 0; k < D; ++k) zG[l][size_t(r) * D + k] += wv * aG[size_t(q) * D + k];
        }
        z[r] = acc;
      }
      act[l + 1].assign(o, 0.0);
      aG.assign(size_t(o) * D, 0.0);
      for (int r = 0; r < o; ++r) {
        if (s[m + net.off[l] + r] == 1) {
          act[l + 1][r] = z[r];
          for (int k = 0; k < D; ++k) aG[size_t(r) * D + k] = zG[l][size_t(r) * D + k];
        }
      }
    }
    std::vector<int> zs;
    for (int j = 0; j < P; ++j)
      if (s[j] == 0) zs.push_back(j);
    if (int(zs.size()) != D) return 4;
    std::vector<double> AT(size_t(D) * D), lam;
    for (int r = 0; r < D; ++r) {
      const int j = zs[r];
      for (int k = 0; k < D; ++k) {
        double gr;
        if (j < m) gr = (k == j / 2) ? ((j % 2 == 0) ? 1.0 : -1.0) : 0.0;
        else {
          int h = j - m, l = 0;
          while (l + 1 < L && h >= net.off[l + 1]) ++l;
          gr = zG[l][size_t(h - net.off[l]) * D + k];
        }
        AT[size_t(k) * D + r] = gr;  // transpose
      }
    }
    if (!solve(D, AT, std::vector<double>(g, g + D), lam)) return 4;
    // Backpropagate the seeds -lambda_r into the parameters, top layer first.
    std::vector<double> dz;
    for (int l = L - 1; l >= 0; --l) {
      const int o = net.w[l + 1], in = net.w[l];
      std::vector<double> seed(o, 0.0);
      if (!dz.empty()) {  // from layer l+1: dz_l = mask * W_{l+1}^T dz_{l+1}
        const int o2 = net.w[l + 2];
        for (int r = 0; r < o; ++r) {
          if (s[m + net.off[l] + r] != 1) continue;
          double acc = 0.0;
          for (int q = 0; q < o2; ++q) acc += net.W[l + 1][size_t(q) * o + r] * dz[q];
          seed[r] = acc;
        }
      }
      for (int r = 0; r < D; ++r) {
        const int j = zs[r];
        if (j < m) continue;
        const int h = j - m;
        if (h >= net.off[l] && h < net.off[l] + o) seed[h - net.off[l]] -= lam[r];
      }
      for (int r = 0; r < o; ++r) {
        if (seed[r] == 0.0) continue;
        for (int q = 0; q < in; ++q) dtheta[wofs[l] + size_t(r) * in + q] += seed[r] * act[l][q];
        dtheta[bofs[l] + r] += seed[r];
      }
      dz.swap(seed);
    }
  }
  return 0;
}

}  // namespace

// ---- C ABI for the test harness ------------------------------------------------

extern "C" {

void* orc_extract(int L, const int32_t* widths, const double* params, const double* lo,
                  const double* hi, int max_neurons, int prune) {
  Result* R = new Result;
  const Net net = make_net(L, widths, params);
  extract(net, lo, hi, max_neurons, *R, prune != 0);
  return R;
}

// Edge subdivision on the polyhedral domain c - A x >= 0 (m half-spaces,
// A row-major m x D) with the caller's initial 1-skeleton (nv0 vertices X0
// row-major nv0 x D, ne0 edges E0 as pairs).
void* orc_extract_domain(int L, const int32_t* widths, const double* params, int m, const double* A,
                         const double* c, int64_t nv0, const double* X0, int64_t ne0, const int32_t* E0,
                         int max_neurons, int prune) {
  Result* R = new Result;
  const Net net = make_net(L, widths, params);
  Domain dom;
  dom.m = m;
  dom.A.assign(A, A + size_t(m) * widths[0]);
  dom.c.assign(c, c + m);
  extract_domain(net, dom, nv0, X0, ne0, E0, max_neurons, *R, prune != 0);
  return R;
}

void* orc_brute_domain(int L, const int32_t* widths, const double* params, int m, const double* A,
                       const double* c, double tol) {
  Result* R = new Result;
  const Net net = make_net(L, widths, params);
  Domain dom;
  dom.m = m;
  dom.A.assign(A, A + size_t(m) * widths[0]);
  dom.c.assign(c, c + m);
  if (brute_domain(net, dom, tol, *R) != 0) {
    R->status = 1;
    R->err = "network too large for brute force";
  }
  return R;
}

// (vertices, edges) after each completed layer: 2 int64 per layer.
int orc_layer_counts(void* r, int64_t* out) {
  auto* R = static_cast<Result*>(r);
  std::memcpy(out, R->layer_counts.data(), R->layer_counts.size() * sizeof(int64_t));
  return int(R->layer_counts.size() / 2);
}

void* orc_brute(int L, const int32_t* widths, const double* params, const double* lo,
                const double* hi, double tol) {
  Result* R = new Result;
  const Net net = make_net(L, widths, params);
  if (brute(net, lo, hi, tol, *R) != 0) {
    R->status = 1;
    R->err = "network too large for brute force";
  }
  return R;
}

void orc_free(void* r) { delete static_cast<Result*>(r); }

int orc_status(void* r) { return static_cast<Result*>(r)->status; }
const char* orc_error(void* r) { return static_cast<Result*>(r)->err.c_str(); }
int64_t orc_nv(void* r) { return static_cast<Result*>(r)->nV(); }
int64_t orc_ne(void* r) { return int64_t(static_cast<Result*>(r)->E.size()); }
int orc_nsig(void* r) { return static_cast<Result*>(r)->P; }

void orc_vertices(void* r, double* out) {
  auto* R = static_cast<Result*>(r);
  std::memcpy(out, R->X.data(), R->X.size() * sizeof(double));
}
void orc_signs(void* r, int8_t* out) {
  auto* R = static_cast<Result*>(r);
  std::memcpy(out, R->S.data(), R->S.size());
}
void orc_edges(void* r, int32_t* out) {
  auto* R = static_cast<Result*>(r);
  for (size_t k = 0; k < R->E.size(); ++k) {
    out[2 * k] = R->E[k][0];
    out[2 * k + 1] = R->E[k][1];
  }
}
void orc_stats(void* r, int64_t* out) {
  auto* R = static_cast<Result*>(r);
  std::memcpy(out, R->stats.data(), R->stats.size() * sizeof(int64_t));
}

// f_out has D+1 entries (f_0 .. f_D); returns the Euler characteristic.
int64_t orc_faces(void* r, int64_t* f_out) { return faces(*static_cast<Result*>(r), f_out); }

// The face poset of an extraction (build_poset); free with orc_poset_free.
void* orc_poset(void* r) { return build_poset(*static_cast<Result*>(r)); }
int orc_poset_status(void* q) { return static_cast<Poset*>(q)->status; }
const char* orc_poset_error(void* q) { return static_cast<Poset*>(q)->err.c_str(); }
int64_t orc_poset_count(void* q, int k) { return int64_t(static_cast<Poset*>(q)->cells[k].size()); }
// n_k x P sign vectors of level k, sorted
void orc_poset_cells(void* q, int k, int8_t* out) {
  auto* Q = static_cast<Poset*>(q);
  for (size_t i = 0; i < Q->cells[k].size(); ++i) std::memcpy(out + i * Q->P, Q->cells[k][i].data(), Q->P);
}
// parents of level k (k < D) as CSR: row_ptr (n_k + 1), cols (nnz)
int64_t orc_poset_nnz(void* q, int k) { return int64_t(static_cast<Poset*>(q)->cols[k].size()); }
void orc_poset_incidence(void* q, int k, int64_t* row_ptr, int64_t* cols) {
  auto* Q = static_cast<Poset*>(q);
  std::memcpy(row_ptr, Q->row_ptr[k].data(), Q->row_ptr[k].size() * sizeof(int64_t));
  std::memcpy(cols, Q->cols[k].data(), Q->cols[k].size() * sizeof(int64_t));
}
void orc_poset_free(void* q) { delete static_cast<Poset*>(q); }

int orc_grad(void* r, int L, const int32_t* widths, const double* params, const double* gx,
             double* dtheta) {
  const Net net = make_net(L, widths, params);
  return grad(net, *static_cast<Result*>(r), gx, dtheta);
}

}  // extern "C"
