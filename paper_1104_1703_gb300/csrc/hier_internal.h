// The hierarchy object behind the mg_hierarchy handle of the C ABI, shared
// by the single-hierarchy driver (mg_capi.cu) and the batched multi-patch
// driver (mg_batch.cu), which owns one hierarchy per patch.
#pragma once

#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"
#include "pass_internal.h"

namespace gbmg {

struct TimedPair {
  cudaEvent_t a, b;
};

// A captured multigrid iteration (plus the residual norm and its copy to the
// pinned host scalar) for one order; replayed once per cycle.
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  int deepest = -2;                // deepest level at capture time
  unsigned long long lists_hash = 0;  // list lengths at capture time (they size the grids)
  unsigned long long nodes = 0;    // kernel launches per replay
  std::vector<TimedPair> events;   // level-0 half-sweep event pairs (timing graphs)
};

}  // namespace gbmg

struct mg_hierarchy {
  using GraphSlot = gbmg::GraphSlot;
  using TimedPair = gbmg::TimedPair;
  using LevelDev = gbmg::LevelDev;
  using FineExtra = gbmg::FineExtra;
  mg_options opt;
  cudaStream_t stream = nullptr;
  cudaStream_t cur = nullptr;          // stream the emitters launch on (stream, or cap_stream while capturing)
  cudaStream_t cap_stream = nullptr;
  GraphSlot graphs[3][2];              // [order][timing]
  std::vector<TimedPair>* cap_events = nullptr;
  size_t cap_events_used = 0;
  bool own_stream = false;
  int device = 0;
  int nlev = 0;
  double h = 0;
  LevelDev L[gbmg::kMaxLevels];
  FineExtra F;
  long long active[3][gbmg::kMaxLevels];
  int deepest[3];
  int hold = 0;
  char* arena = nullptr;
  int8_t* mask_dev = nullptr;
  uint32_t* list_scratch = nullptr;
  // job tables (device, in the arena) of the batched build launches
  gbmg::ListJob* list_jobs = nullptr;
  int n_list_jobs = 0;
  unsigned list_blocks = 0;
  gbmg::ZeroJob* zero_jobs = nullptr;
  int n_zero_jobs = 0;
  bool bc_zero = true;  // the folded boundary terms are all 0
  bool rhsd_valid = false;  // level 0's b / D matches its b
  // the coarsest solve's precomputed map per order (option coarse_matrix):
  // device pointer in the arena, its red / black counts, and whether it
  // matches the current mask
  void* cmat[3] = {nullptr, nullptr, nullptr};
  uint32_t cmat_n[3][2] = {};
  bool cmat_ok[3] = {false, false, false};
  int cmat_prec = 0;
  double* partials = nullptr;
  int max_partials = 0;
  double* dscal = nullptr;             // device scalars
  int* err_flag = nullptr;
  unsigned long long* counts = nullptr;  // [kMaxLevels][2]
  double* hscal = nullptr;               // pinned host scalars
  void* staging = nullptr;
  size_t staging_bytes = 0;
  double r_zero = 0;
  bool r_zero_valid = false;
  bool prepared = false;  // mixed form: rhs32/e32 of level 0 match the current Phi and b
  std::string last_error = "no error";
  bool timing = false;
  std::vector<TimedPair> events;
  size_t events_used = 0;
  long long timed_launches = 0;   // accumulated from graph replays
  double timed_ms = 0;
  // temporal-blocked FP32 smoothing pass of level 0 (mixed form)
  bool pass_on = false;
  float* phi32_alt[2] = {nullptr, nullptr};  // the second FP32 correction buffer of level 0
  uint32_t* pass_flags = nullptr;
  uint32_t* pass_tiles = nullptr;
  uint32_t* pass_ntiles = nullptr;
  gbmg::PassMaps pass_maps;
};

namespace gbmg {
mg_status check_faults(mg_hierarchy* H);  // mg_capi.cu
}  // namespace gbmg
