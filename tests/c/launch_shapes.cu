// Host-side check of the launch shapes of the tiled coordinate polish and of
// the batched FP64 re-decision, for every layer width, input dimension and
// sign-word count the library accepts: the busy (vertex, neuron) blocks of
// every layer fit the CTA, tiles hold whole 4-vertex groups, every
// workspace region is 16-byte aligned, and the shared memory stays within
// the launch attribute.  It includes the kernel sources as they are (no GPU
// is needed: nothing is launched).  Prints one line per failure, exits 1 if
// any.
#include <cstdio>

#include "pc_polish.cu"
#include "pc_phases.cuh"

int main() {
  int bad = 0;
  auto fail = [&](const char* what, int mw, int D, int S, long long v) {
    if (bad < 20) std::printf("%s: width %d D %d S %d -> %lld\n", what, mw, D, S, v);
    ++bad;
  };
  for (int mw = 1; mw <= pc::kMaxWidth; ++mw)
    for (int S = 1; S <= pc::kMaxWords; ++S) {
      for (int D = 1; D <= pc::kPtMaxD && D <= mw; ++D) {
        const int TV = pc::pt_tile_vertices(mw, S, D);
        if (TV < 4 || TV % 4 != 0) fail("polish tile not whole 4-vertex groups", mw, D, S, TV);
        const pc::PtLayout L = pc::pt_layout(TV, mw, S, D);
        if (L.total > (size_t)pc::kPtSmemMax) fail("polish shared memory above the attribute", mw, D, S, (long long)L.total);
        if (L.rows < mw || L.rows < D) fail("polish rows", mw, D, S, L.rows);
        for (size_t off : {L.A, L.gv, L.sig, L.ahi, L.alo, L.J, L.zl, L.nz})
          if (off % 16) fail("polish region not 16-byte aligned", mw, D, S, (long long)off);
        for (int H = 1; H <= mw; ++H) {  // any layer of the net, the widest included
          const long long busy = (long long)(TV / 4) * ((H + pc::kPtRows - 1) / pc::kPtRows);
          if (busy > pc::kPtThreads) fail("polish blocks exceed the CTA", mw, D, S, busy);
        }
      }
      for (int D = 1; D <= pc::kMaxD && D <= mw; ++D) {
        const int P = pc::rd_batch_size(mw, D, S);
        if (P < 1 || P > pc::kWarps) fail("re-decision batch size", mw, D, S, P);
        const pc::RdLayout R = pc::rd_layout(P, mw, D, S);
        if (R.total > (size_t)pc::kRdSmemMax) fail("re-decision shared memory above the attribute", mw, D, S,
                                                   (long long)R.total);
        for (size_t off : {R.a, R.an, R.A, R.gv, R.dlt, R.sig, R.J, R.Jn, R.sc, R.zl, R.nz, R.ok})
          if (off % 16) fail("re-decision region not 16-byte aligned", mw, D, S, (long long)off);
      }
    }
  std::printf("%d failures\n", bad);
  return bad ? 1 : 0;
}
