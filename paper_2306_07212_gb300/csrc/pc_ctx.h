// Host-side context of libpc (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "pc.h"
#include "pc_device.cuh"

struct pc_ctx;

void* ctx_alloc(pc_ctx* c, size_t bytes);
void ctx_free(pc_ctx* c, void*& p);
pc::State pc_make_state(pc_ctx* c);

// canonical output order (pc_canon.cu)
void pc_canonicalize(pc_ctx* c);

// face poset (pc_cells.cu)
void pc_poset_release(pc_ctx* c);

// pruning during subdivision (pc_prune.cu)
void pc_prune_edges(pc_ctx* c, const pc::State& st, int l);
void pc_prune_vertices(pc_ctx* c);
cudaError_t pc_prune_set_attributes();

// tcgen05 layer-start product (pc_gemm_tc.cu)
bool pc_gemm_tc_eligible(const pc::NetDesc& net, int l);
cudaError_t pc_gemm_tc_set_attributes();
cudaError_t pc_gemm_tc_launch(const pc::NetDesc& net, const pc::State& st, int l, long long vcap_tiles, int num_sms,
                              int pieces, cudaStream_t stream);

// coordinate polish as a tiled product (pc_polish.cu), D <= 5
bool pc_polish_tile_eligible(const pc::NetDesc& net);
cudaError_t pc_polish_tile_set_attributes();
cudaError_t pc_polish_tile_launch(const pc::NetDesc& net, const pc::State& st, float thr, int mw, int num_sms,
                                  bool domain, cudaStream_t stream);

struct PcError : std::runtime_error {
  pc_status status;
  PcError(pc_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

struct StateBufs {
  void* X = nullptr;
  void* Z[pc::kMaxL] = {};   // nz value buffers (2, or one per layer with the tape)
  int nz = 0;
  void* esc = nullptr;
  void* exc = nullptr;
  void* SIG = nullptr;
  void* E = nullptr;
  void* list0 = nullptr;  // splitting edges of the even / odd neurons' steps
  void* list1 = nullptr;
  void* flags = nullptr;  // two bitmaps of Ecap bits: edge in list0 / list1
  void* vlist = nullptr;
  void* table = nullptr;
  void* tape_pq = nullptr;
  void* tape_t = nullptr;
  void release(pc_ctx* c);
};

struct pc_ctx {
  int device = 0;
  int num_sms = 1;
  pc_options opt{};
  std::string err;
  cudaStream_t stream = nullptr;
  pc_alloc_fn alloc_fn = nullptr;
  pc_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  size_t allocated = 0;
  std::unordered_map<void*, size_t> sizes;

  // network of the last extraction
  pc::NetDesc net{};
  int hmax = 0, mw = 0, N = 0;
  void* params64 = nullptr;
  void* params32 = nullptr;
  void* norms = nullptr;
  long long params_cap = 0;
  int norms_cap = 0;

  // state
  StateBufs bufs;
  long long Vcap = 0, Ecap = 0, Tcap = 0;
  // shape the state buffers were sized for (rows per array); every network
  // that runs without reshaping fits it
  int shape_D = 0, shape_S = 0, shape_H = 0, shape_tape = -1, shape_nz = 0;
  size_t shape_zs = 0;
  void* cnt = nullptr;
  int cnt_slots = 0;
  void* g = nullptr;
  void* h_cnt = nullptr;
  void* h_g = nullptr;

  // polyhedral domain of the last extraction (facets and initial skeleton)
  void* dom_buf = nullptr;
  size_t dom_cap = 0;

  int deferred = 0;  // this extraction pairs by fingerprint (checked after)
  int reruns = 0;    // extractions repeated with inline face verification

  // launch geometry
  int grid_persist = 0, grid_step = 0;
  size_t res_smem = 0;

  // results
  long long nV = 0, nE = 0;
  long long degenerate = 0, undecided = 0;
  long long grows = 0;
  long long polished = 0;
  long long launches = 0;
  long long flips = 0;       // FP64 re-decisions that changed an FP32 sign
  float flip_margin = 0.f;   // largest |z| / estimate among them
  long long missed = 0;      // audit band: wrong FP32 signs beyond kappa
  float missed_margin = 0.f;
  bool have_result = false;

  // per-layer kernel timers (opt.timers)
  static constexpr int kPolishSlot = 2 * pc::kMaxL;
  cudaEvent_t ev[2 * pc::kMaxL + 1][2] = {};
  int ev_used[2 * pc::kMaxL + 1] = {};
  double ktime_ms[2 * pc::kMaxL + 1] = {};

  // face poset of the last result (pc_build_poset): per level the cells
  // (cell-major sign words) and below D the parents as CSR
  std::vector<void*> poset_bufs;
  void* poset_cells[pc::kMaxD + 1] = {};
  long long poset_n[pc::kMaxD + 1] = {};
  void* poset_rp[pc::kMaxD] = {};
  void* poset_cols[pc::kMaxD] = {};
  long long poset_nnz[pc::kMaxD] = {};
  int poset_levels = 0;

  // adjoint scratch (allocated lazily by pc_backward)
  void* adj[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t adj_bytes[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  pc_status fail(pc_status s, const std::string& m) {
    err = m;
    return s;
  }
  void release_extra() {
    for (auto& p : adj) ctx_free(this, p);
  }
};
