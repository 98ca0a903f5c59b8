// Host driver of the batched multi-patch solve (mg_batch_* in mg.h): one
// hierarchy per patch (built by mg_create_hierarchy on the batch's stream),
// chunk tables over the compact lists of all patches, the batched cycle as a
// CUDA graph, the per-patch solve loop with the Section 4 order switch, and
// the launch-parameter autotuner.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "batch_internal.h"
#include "hier_internal.h"
#include "mg_internal.h"

namespace gbmg {
void set_thread_error(const char* msg);  // mg_capi.cu
}  // namespace gbmg

using namespace gbmg;

namespace {

struct Table {
  int off = 0;  // first chunk in the chunk array
  int n = 0;    // chunks
};

}  // namespace

struct mg_batch {
  int n = 0;
  std::vector<mg_hierarchy*> P;
  mg_options opt;
  mg_batch_tuning tune;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int sms = 0;  // multiprocessors of the device (resident-block candidates of the autotuner)
  std::string last_error = "no error";

  // per patch and order (index o - 1): bottom start level (0: level 0 is the
  // deepest level) and deepest level
  std::vector<int> lb[2], deepest[2];
  int lmax = 1;  // levels 0 .. lmax-1 run in the chunked kernels

  // chunk tables (device copy in `tables`)
  Table gs[kMaxLevels][2], restr[kMaxLevels], prol[kMaxLevels], norm0;
  std::vector<int> norm_first, norm_count;
  int nchunks = 0;
  size_t bottom_smem = 0;

  // device memory
  char* tables = nullptr;
  Chunk* d_chunks = nullptr;
  PatchLevel* d_pls = nullptr;
  void* d_bottom = nullptr;
  int* d_first = nullptr;
  int* d_count = nullptr;
  double* d_partials = nullptr;
  int* d_state = nullptr;
  double* d_norm2 = nullptr;
  // pinned host memory
  int* h_state = nullptr;
  double* h_norm2 = nullptr;

  cudaGraphExec_t graph = nullptr;
  long long graph_nodes = 0;
  cudaStream_t cap_stream = nullptr;
};

namespace {

mg_status bfail(mg_batch* B, mg_status st, const std::string& msg) {
  if (B) B->last_error = msg;
  set_thread_error(msg.c_str());
  return st;
}

mg_status bcuda(mg_batch* B, cudaError_t e, const char* what) {
  return bfail(B, e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(B, call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return bcuda((B), e_, #call); \
  } while (0)

#define BCKS(call)               \
  do {                           \
    mg_status s_ = (call);       \
    if (s_ != MG_OK) return s_;  \
  } while (0)

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

long long slots(const Geom& g) { return (long long)g.hx * g.ny * g.nz; }

bool valid_tuning(const mg_batch_tuning& t) {
  return (t.threads == 128 || t.threads == 256 || t.threads == 512) && t.persistent_ctas >= 0 &&
         t.persistent_ctas <= (1 << 20) && t.bottom_slots >= 64 && t.bottom_slots <= 16384 && t.n_pre >= 0 &&
         t.n_pre <= 8 && t.n_post >= 0 && t.n_post <= 8 && (t.chunk == 0 || (t.chunk >= 64 && t.chunk <= 65536));
}

// Gauss-Seidel updates of one V-cycle of patch H in `order` (as the
// single-hierarchy count: sweeps x active cells per level, coarse_sweeps on
// the deepest level).
long long cycle_updates(const mg_hierarchy* H, const mg_options& o, int order) {
  const int d = H->deepest[order];
  long long n = 0;
  for (int l = 0; l <= d; ++l) {
    const long long act = l == 0 ? H->active[2][0] : H->active[order][l];
    n += (l == d ? (long long)o.coarse_sweeps : (long long)(o.n_pre + o.n_post)) * act;
  }
  return n;
}

void drop_graph(mg_batch* B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->graph = nullptr;
  B->graph_nodes = 0;
}

void free_tables(mg_batch* B) {
  drop_graph(B);
  if (B->tables) cudaFree(B->tables);
  B->tables = nullptr;
}

// Appends the chunks of one list segment of n entries.
void add_chunks(std::vector<Chunk>& v, uint32_t pl, uint32_t n, int tag, int colour, int chunk) {
  for (uint32_t s = 0; s < n; s += (uint32_t)chunk) {
    Chunk c;
    c.pl = pl;
    c.start = s;
    c.n = (uint16_t)std::min<uint32_t>((uint32_t)chunk, n - s);
    c.tag = (uint8_t)tag;
    c.colour = (uint8_t)colour;
    v.push_back(c);
  }
}

uint32_t list_len(const LevelDev& L, int order, int colour) {
  return L.hcount[(L.level == 0 ? 2 : order) * 2 + colour];
}

// Builds the chunk tables, the patch-level table and the bottom arguments
// for the current tuning and uploads them (one allocation).
mg_status build_tables(mg_batch* B) {
  free_tables(B);
  const mg_batch_tuning& t = B->tune;
  const int chunk = t.chunk > 0 ? t.chunk : 2 * t.threads;
  const int n = B->n;
  for (int o = 0; o < 2; ++o) {
    B->lb[o].assign(n, 0);
    B->deepest[o].assign(n, 0);
  }
  B->lmax = 1;
  for (int p = 0; p < n; ++p) {
    const mg_hierarchy* H = B->P[p];
    for (int o = 1; o <= 2; ++o) {
      const int d = H->deepest[o];
      int lb = 0;
      if (d >= 1) {
        lb = d;
        for (int l = 1; l < d; ++l)
          if (slots(H->L[l].g) <= t.bottom_slots) {
            lb = l;
            break;
          }
      }
      B->lb[o - 1][p] = lb;
      B->deepest[o - 1][p] = d;
      B->lmax = std::max(B->lmax, lb);
    }
  }
  std::vector<Chunk> ch;
  auto begin = [&](Table& T) { T.off = (int)ch.size(); };
  auto end = [&](Table& T) { T.n = (int)ch.size() - T.off; };
  auto pl_of = [](int p, int l) { return (uint32_t)(p * kMaxLevels + l); };
  for (int l = 0; l < kMaxLevels; ++l) {
    B->gs[l][0] = B->gs[l][1] = Table();
    B->restr[l] = B->prol[l] = Table();
  }
  // level 0 (tag 0: every patch whose deepest level is below level 0)
  for (int c = 0; c < 2; ++c) {
    begin(B->gs[0][c]);
    for (int p = 0; p < n; ++p) add_chunks(ch, pl_of(p, 0), list_len(B->P[p]->L[0], 2, c), 0, c, chunk);
    end(B->gs[0][c]);
  }
  begin(B->restr[0]);
  for (int p = 0; p < n; ++p) {
    const mg_hierarchy* H = B->P[p];
    if (H->nlev < 2 || H->deepest[2] < 1) continue;
    for (int c = 0; c < 2; ++c) add_chunks(ch, pl_of(p, 1), list_len(H->L[1], 2, c), 0, c, chunk);
  }
  end(B->restr[0]);
  // prolongation corrects the black unknowns only when a red half-sweep
  // follows (it overwrites the red ones without reading them)
  const int c_prol = t.n_post >= 1 ? 1 : 0;
  begin(B->prol[0]);
  for (int p = 0; p < n; ++p) {
    const mg_hierarchy* H = B->P[p];
    if (H->nlev < 2 || H->deepest[2] < 1) continue;
    for (int c = c_prol; c < 2; ++c) add_chunks(ch, pl_of(p, 0), list_len(H->L[0], 2, c), 0, c, chunk);
  }
  end(B->prol[0]);
  // coarse levels run by the chunked kernels (tag = order)
  for (int l = 1; l < B->lmax; ++l) {
    for (int c = 0; c < 2; ++c) {
      begin(B->gs[l][c]);
      for (int p = 0; p < n; ++p)
        for (int o = 1; o <= 2; ++o)
          if (l < B->lb[o - 1][p]) add_chunks(ch, pl_of(p, l), list_len(B->P[p]->L[l], o, c), o, c, chunk);
      end(B->gs[l][c]);
    }
    begin(B->restr[l]);
    for (int p = 0; p < n; ++p)
      for (int o = 1; o <= 2; ++o)
        if (l + 1 <= B->lb[o - 1][p])
          for (int c = 0; c < 2; ++c) add_chunks(ch, pl_of(p, l + 1), list_len(B->P[p]->L[l + 1], 2, c), o, c, chunk);
    end(B->restr[l]);
    begin(B->prol[l]);
    for (int p = 0; p < n; ++p)
      for (int o = 1; o <= 2; ++o)
        if (l + 1 <= B->lb[o - 1][p])
          for (int c = c_prol; c < 2; ++c) add_chunks(ch, pl_of(p, l), list_len(B->P[p]->L[l], o, c), o, c, chunk);
    end(B->prol[l]);
  }
  // level-0 norm: per patch, red chunks then black chunks (contiguous)
  begin(B->norm0);
  B->norm_first.assign(n, 0);
  B->norm_count.assign(n, 0);
  for (int p = 0; p < n; ++p) {
    B->norm_first[p] = (int)ch.size() - B->norm0.off;
    for (int c = 0; c < 2; ++c) add_chunks(ch, pl_of(p, 0), list_len(B->P[p]->L[0], 2, c), 0, c, chunk);
    B->norm_count[p] = (int)ch.size() - B->norm0.off - B->norm_first[p];
  }
  end(B->norm0);
  B->nchunks = (int)ch.size();

  // patch-level descriptors
  std::vector<PatchLevel> pls((size_t)n * kMaxLevels);
  for (int p = 0; p < n; ++p) {
    const mg_hierarchy* H = B->P[p];
    for (int l = 0; l < H->nlev; ++l) {
      const LevelDev& L = H->L[l];
      PatchLevel& d = pls[(size_t)p * kMaxLevels + l];
      d.g = L.g;
      for (int c = 0; c < 2; ++c) {
        d.phi[c] = L.phi[c];
        d.rhs[c] = L.rhs[c];
        d.invd[c] = L.invd[c];
        d.diag[c] = L.diag[c];
        d.code[c] = L.code[c];
        d.rhsd[c] = L.rhsd[c];
        for (int o = 0; o < 3; ++o) d.list[o][c] = L.list[o][c];
      }
      d.patch = p;
      d.level = l;
    }
  }
  // bottom arguments, slot 2p + (order - 1)
  const size_t bsz = batch_bottom_args_bytes();
  std::vector<char> bot(bsz * 2 * n);
  B->bottom_smem = 0;
  for (int p = 0; p < n; ++p) {
    const mg_hierarchy* H = B->P[p];
    for (int o = 1; o <= 2; ++o) {
      const int d = B->deepest[o - 1][p];
      const int lb = d == 0 ? 0 : B->lb[o - 1][p];
      const size_t sm = batch_fill_bottom(bot.data(), 2 * p + o - 1, H->L, lb, d, o, t.n_pre, t.n_post,
                                          B->opt.coarse_sweeps, p);
      if (sm == kBottomTooDeep)
        return bfail(B, MG_ERR_INVALID_ARG, "patch " + std::to_string(p) + ": too many levels below bottom_slots");
      B->bottom_smem = std::max(B->bottom_smem, sm);
    }
  }
  // one allocation for everything the kernels read
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_ch = 0;
  const size_t o_pl = o_ch + al(sizeof(Chunk) * std::max(1, B->nchunks));
  const size_t o_bot = o_pl + al(sizeof(PatchLevel) * pls.size());
  const size_t o_first = o_bot + al(bot.size());
  const size_t o_count = o_first + al(sizeof(int) * n);
  const size_t o_part = o_count + al(sizeof(int) * n);
  const size_t o_state = o_part + al(sizeof(double) * std::max(1, B->norm0.n));
  const size_t o_norm = o_state + al(sizeof(int) * n);
  const size_t total = o_norm + al(sizeof(double) * n);
  BCK(B, dev_malloc((void**)&B->tables, total));
  B->d_chunks = (Chunk*)(B->tables + o_ch);
  B->d_pls = (PatchLevel*)(B->tables + o_pl);
  B->d_bottom = B->tables + o_bot;
  B->d_first = (int*)(B->tables + o_first);
  B->d_count = (int*)(B->tables + o_count);
  B->d_partials = (double*)(B->tables + o_part);
  B->d_state = (int*)(B->tables + o_state);
  B->d_norm2 = (double*)(B->tables + o_norm);
  cudaStream_t s = B->stream;
  BCK(B, cudaMemsetAsync(B->tables, 0, total, s));
  if (!ch.empty()) BCK(B, cudaMemcpyAsync(B->d_chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice, s));
  BCK(B, cudaMemcpyAsync(B->d_pls, pls.data(), sizeof(PatchLevel) * pls.size(), cudaMemcpyHostToDevice, s));
  BCK(B, cudaMemcpyAsync(B->d_bottom, bot.data(), bot.size(), cudaMemcpyHostToDevice, s));
  BCK(B, cudaMemcpyAsync(B->d_first, B->norm_first.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  BCK(B, cudaMemcpyAsync(B->d_count, B->norm_count.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  BCK(B, cudaStreamSynchronize(s));  // the host vectors above go out of scope
  return MG_OK;
}

mg_status lok(mg_batch* B, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return bcuda(B, e, what);
  return MG_OK;
}

int grid_of(const mg_batch* B, const Table& T) { return batch_grid(T.n, B->tune.threads, B->tune.persistent_ctas); }

mg_status emit_gs(mg_batch* B, int l, int c, cudaStream_t s) {
  const Table& T = B->gs[l][c];
  return lok(B, launch_batch_gs(B->d_chunks + T.off, T.n, B->d_pls, B->d_state, l == 0, B->opt.fp64_sum == 1,
                                B->tune.threads,
                                grid_of(B, T), s),
             "batched half-sweep");
}

mg_status emit_smooth(mg_batch* B, int l, int sweeps, cudaStream_t s) {
  for (int k = 0; k < sweeps; ++k)
    for (int c = 0; c < 2; ++c) BCKS(emit_gs(B, l, c, s));
  return MG_OK;
}

// Sum of squares over the level-0 unknowns of every patch into d_norm2
// (mode 1: residual, 2: right-hand side), then its copy to h_norm2.
mg_status emit_norm(mg_batch* B, int mode, cudaStream_t s) {
  const Table& T = B->norm0;
  BCKS(lok(B, launch_batch_norm(B->d_chunks + T.off, T.n, B->d_pls, B->d_state, mode, B->d_partials,
                                B->tune.threads, grid_of(B, T), s),
           "batched norm"));
  BCKS(lok(B, launch_batch_patch_sums(B->d_partials, B->d_first, B->d_count, B->n, B->d_norm2, s), "patch sums"));
  BCK(B, cudaMemcpyAsync(B->h_norm2, B->d_norm2, sizeof(double) * B->n, cudaMemcpyDeviceToHost, s));
  return MG_OK;
}

// One batched V-cycle (Section 2 recipe on every patch; the per-patch
// state says which patches take part and in which order) and the residual
// norms.  The state is copied from pinned host memory first.
mg_status emit_cycle(mg_batch* B, cudaStream_t s) {
  const mg_batch_tuning& t = B->tune;
  BCK(B, cudaMemcpyAsync(B->d_state, B->h_state, sizeof(int) * B->n, cudaMemcpyHostToDevice, s));
  const bool black_zero = t.n_pre >= 1;
  for (int l = 0; l < B->lmax; ++l) {
    BCKS(emit_smooth(B, l, t.n_pre, s));  // step 1
    const Table& R = B->restr[l];
    BCKS(lok(B, launch_batch_restrict(B->d_chunks + R.off, R.n, B->d_pls, B->d_state, black_zero, t.threads,
                                      grid_of(B, R), s),
             "batched residual and restriction"));  // steps 2-5
  }
  BCKS(lok(B, launch_batch_bottom(B->d_bottom, B->n, B->d_pls, B->d_state, B->bottom_smem, s), "batched bottom"));
  for (int l = B->lmax - 1; l >= 0; --l) {
    const Table& Q = B->prol[l];
    BCKS(lok(B, launch_batch_prolong(B->d_chunks + Q.off, Q.n, B->d_pls, B->d_state, t.threads, grid_of(B, Q), s),
             "batched prolongation"));  // steps 6-7
    BCKS(emit_smooth(B, l, t.n_post, s));  // step 8
  }
  return emit_norm(B, 1, s);
}

mg_status capture(mg_batch* B) {
  drop_graph(B);
  if (!B->cap_stream) BCK(B, cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCK(B, cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
  // launches issued while capturing run only at replay: counted there
  capture_count_begin();
  mg_status st = emit_cycle(B, B->cap_stream);
  const unsigned long long nodes = capture_count_end();
  cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
  if (st != MG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return bcuda(B, e, "batched cycle capture");
  e = cudaGraphInstantiate(&B->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    B->graph = nullptr;
    return bcuda(B, e, "batched cycle instantiate");
  }
  B->graph_nodes = (long long)nodes;
  return MG_OK;
}

// b / D of every patch's level 0 (the scaled sweeps), when some patch's b
// changed since it was last computed.
mg_status ensure_rhsd(mg_batch* B) {
  bool stale = false;
  for (const mg_hierarchy* H : B->P) stale = stale || !H->rhsd_valid;
  if (!stale) return MG_OK;
  for (int c = 0; c < 2; ++c) {
    const Table& T = B->gs[0][c];
    BCKS(lok(B, launch_batch_scale(B->d_chunks + T.off, T.n, B->d_pls, B->tune.threads, grid_of(B, T), B->stream),
             "batched b / D"));
  }
  for (mg_hierarchy* H : B->P) H->rhsd_valid = true;
  return MG_OK;
}

// Replays the batched cycle graph (capturing it first if needed) and waits
// for the norms.
mg_status run_cycle(mg_batch* B) {
  BCKS(ensure_rhsd(B));
  if (!B->graph) BCKS(capture(B));
  BCK(B, cudaGraphLaunch(B->graph, B->stream));
  count_launch((unsigned long long)B->graph_nodes);
  BCK(B, cudaStreamSynchronize(B->stream));
  return MG_OK;
}

int start_order(const mg_hierarchy* H) {
  if (H->opt.order == 1 || H->opt.order == 2) return H->opt.order;
  return H->hold > 0 ? 1 : 2;
}

int state_word(const mg_batch* B, int p, int order) {
  const int d = B->deepest[order - 1][p];
  const bool ends_sweep = d == 0 ? B->opt.coarse_sweeps >= 1 : B->tune.n_post >= 1;
  return order | (d == 0 ? kStDeep0 : 0) | (ends_sweep ? 0 : kStBlackNorm);
}

// r(Phi = 0) and r(current Phi) of every patch, in ||.|| units (unscaled).
mg_status initial_norms(mg_batch* B, std::vector<double>& r_zero, std::vector<double>& r_init) {
  for (int p = 0; p < B->n; ++p) B->h_state[p] = 2 | kStBlackNorm;
  cudaStream_t s = B->stream;
  BCK(B, cudaMemcpyAsync(B->d_state, B->h_state, sizeof(int) * B->n, cudaMemcpyHostToDevice, s));
  BCKS(emit_norm(B, 2, s));
  BCK(B, cudaStreamSynchronize(s));
  r_zero.resize(B->n);
  for (int p = 0; p < B->n; ++p) {
    const double h2 = B->P[p]->h * B->P[p]->h;
    r_zero[p] = std::sqrt(B->h_norm2[p]) / h2;
  }
  BCKS(emit_norm(B, 1, s));
  BCK(B, cudaStreamSynchronize(s));
  r_init.resize(B->n);
  for (int p = 0; p < B->n; ++p) {
    const double h2 = B->P[p]->h * B->P[p]->h;
    r_init[p] = std::sqrt(B->h_norm2[p]) / h2;
  }
  return MG_OK;
}

mg_status copy_phi(mg_batch* B, int p, bool to_save) {
  mg_hierarchy* H = B->P[p];
  const size_t bytes = sizeof(double) * H->L[0].g.total;
  for (int c = 0; c < 2; ++c) {
    void* dst = to_save ? (void*)H->F.save[c] : (void*)H->L[0].phi[c];
    const void* src = to_save ? (const void*)H->L[0].phi[c] : (const void*)H->F.save[c];
    BCK(B, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, B->stream));
  }
  return MG_OK;
}

mg_status set_schedule(mg_batch* B, int n_pre, int n_post) {
  B->tune.n_pre = n_pre;
  B->tune.n_post = n_post;
  B->opt.n_pre = n_pre;
  B->opt.n_post = n_post;
  for (mg_hierarchy* H : B->P) {
    H->opt.n_pre = n_pre;
    H->opt.n_post = n_post;
    for (auto& row : H->graphs)
      for (auto& gs : row) {
        if (gs.exec) cudaGraphExecDestroy(gs.exec);
        gs.exec = nullptr;
        gs.deepest = -2;
      }
  }
  return MG_OK;
}

mg_status solve_impl(mg_batch* B, double tol, int max_cycles, mg_solve_info* infos) {
  const int n = B->n;
  const mg_options& o = B->opt;
  std::vector<int> order(n, 2), active(n, 0), cycles(n, 0), auto_sw(n, 0), switched(n, 0);
  std::vector<mg_status> st(n, MG_ERR_NOT_CONVERGED);
  std::vector<double> r_zero, r_init, r_n(n), r_prev(n), rel(n);
  std::vector<long long> upd(n, 0);
  for (int p = 0; p < n; ++p) {
    mg_hierarchy* H = B->P[p];
    if (o.order == 1 || o.order == 2) {
      order[p] = o.order;
    } else if (H->hold > 0) {
      order[p] = 1;
      H->hold -= 1;
    } else {
      auto_sw[p] = 1;
    }
    if (H->deepest[order[p]] < 0) order[p] = 2;
  }
  BCKS(initial_norms(B, r_zero, r_init));
  for (int p = 0; p < n; ++p) {
    mg_hierarchy* H = B->P[p];
    H->prepared = false;
    r_n[p] = r_init[p];
    rel[p] = r_zero[p] > 0 ? r_init[p] / r_zero[p] : 0.0;
    if (infos) {
      std::memset(&infos[p], 0, sizeof(mg_solve_info));
      infos[p].r_zero = r_zero[p];
      infos[p].r_init = r_init[p];
      infos[p].hist[0] = r_init[p];
    }
    if (!std::isfinite(r_zero[p]) || !std::isfinite(r_init[p])) {
      st[p] = MG_ERR_DIVERGED;
      rel[p] = r_init[p] / r_zero[p];
    } else if (r_zero[p] == 0.0) {
      for (int c = 0; c < 2; ++c)
        BCK(B, cudaMemsetAsync(H->L[0].phi[c], 0, sizeof(double) * H->L[0].g.total, B->stream));
      r_n[p] = 0.0;
      rel[p] = 0.0;
      st[p] = MG_OK;
    } else if (rel[p] < tol) {
      st[p] = MG_OK;
    } else {
      active[p] = 1;
      if (auto_sw[p]) BCKS(copy_phi(B, p, true));
      r_prev[p] = r_init[p];
    }
  }
  for (int cyc = 1; cyc <= max_cycles; ++cyc) {
    bool any = false;
    for (int p = 0; p < n; ++p) {
      B->h_state[p] = active[p] ? state_word(B, p, order[p]) : 0;
      any = any || active[p];
    }
    if (!any) break;
    BCKS(run_cycle(B));
    for (int p = 0; p < n; ++p) {
      if (!active[p]) continue;
      mg_hierarchy* H = B->P[p];
      cycles[p] = cyc;
      upd[p] += cycle_updates(H, o, order[p]);
      r_n[p] = std::sqrt(B->h_norm2[p]) / (H->h * H->h);
      if (infos && cyc <= MG_HIST_MAX) infos[p].hist[cyc] = r_n[p];
      if (!std::isfinite(r_n[p])) {
        st[p] = MG_ERR_DIVERGED;
        active[p] = 0;
        continue;
      }
      rel[p] = r_n[p] / r_zero[p];
      if (rel[p] < tol) {
        st[p] = MG_OK;
        active[p] = 0;
        continue;
      }
      if (auto_sw[p] && !switched[p] && order[p] == 2 && r_n[p] >= 100.0 * DBL_EPSILON * r_zero[p] &&
          r_n[p] / r_prev[p] > o.eta) {
        order[p] = 1;
        switched[p] = 1;
        H->hold = o.hold_solves;
        if (r_n[p] > r_init[p]) {
          BCKS(copy_phi(B, p, false));
          r_n[p] = r_init[p];
        }
      }
      r_prev[p] = r_n[p];
    }
  }
  mg_status worst = MG_OK;
  for (int p = 0; p < n; ++p) {
    if (active[p]) cycles[p] = max_cycles;
    if (infos) {
      infos[p].cycles = cycles[p];
      infos[p].order_used = order[p];
      infos[p].switched = switched[p];
      infos[p].cell_updates = upd[p];
      infos[p].r_final = r_n[p];
      infos[p].rel = rel[p];
      infos[p].status = st[p];
    }
    if (st[p] == MG_ERR_DIVERGED) worst = MG_ERR_DIVERGED;
    else if (st[p] == MG_ERR_NOT_CONVERGED && worst == MG_OK) worst = MG_ERR_NOT_CONVERGED;
  }
  for (int p = 0; p < n; ++p)
    if (check_faults(B->P[p]) != MG_OK) return bfail(B, MG_ERR_INTERNAL, "patch " + std::to_string(p) + ": " +
                                                                          B->P[p]->last_error);
  if (worst == MG_ERR_NOT_CONVERGED) return bfail(B, worst, "a patch did not reach the tolerance within max_cycles");
  if (worst == MG_ERR_DIVERGED) return bfail(B, worst, "a patch's residual norm became non-finite");
  return MG_OK;
}

void destroy_batch(mg_batch* B) {
  if (!B) return;
  Guard guard(B->device);
  if (B->stream) cudaStreamSynchronize(B->stream);
  free_tables(B);
  for (mg_hierarchy* H : B->P)
    if (H) mg_destroy_hierarchy(H);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  if (B->h_state) cudaFreeHost(B->h_state);
  if (B->h_norm2) cudaFreeHost(B->h_norm2);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

}  // namespace

extern "C" {

mg_status mg_batch_create(int n_patches, const int8_t* const* masks, mg_mem where, const int* dims, const double* h,
                          const mg_options* opt, void* cuda_stream, mg_batch** out) {
  if (out) *out = nullptr;
  if (!out || !masks || !dims || !h) return bfail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  if (n_patches < 1 || n_patches > 4096) return bfail(nullptr, MG_ERR_INVALID_ARG, "n_patches must be in 1..4096");
  mg_options o;
  mg_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != 0 || o.n_cycles != 1)
    return bfail(nullptr, MG_ERR_INVALID_ARG, "a batch runs FP64 V-cycles (precision 0, n_cycles 1)");
  mg_batch* B = new mg_batch();
  B->n = n_patches;
  B->opt = o;
  B->tune.threads = 256;
  B->tune.persistent_ctas = 0;
  B->tune.bottom_slots = 4096;
  B->tune.n_pre = o.n_pre;
  B->tune.n_post = o.n_post;
  B->tune.ms_per_cycle = 0;
  B->tune.chunk = 0;
  if (!valid_tuning(B->tune)) {
    delete B;
    return bfail(nullptr, MG_ERR_INVALID_ARG, "invalid options (n_pre, n_post must be in 0..8)");
  }
  if (cudaGetDevice(&B->device) != cudaSuccess) {
    delete B;
    return bfail(nullptr, MG_ERR_CUDA, "no CUDA device");
  }
  B->sms = device_sms();
  if (cuda_stream) {
    B->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreate(&B->stream);
    if (e != cudaSuccess) {
      delete B;
      return bcuda(nullptr, e, "cudaStreamCreate");
    }
    B->own_stream = true;
  }
  mg_status st = MG_OK;
  cudaError_t e = init_batch_kernels();
  if (e != cudaSuccess) st = bcuda(B, e, "batched kernel attributes");
  if (st == MG_OK) {
    e = host_malloc((void**)&B->h_state, sizeof(int) * n_patches);
    if (e == cudaSuccess) e = host_malloc((void**)&B->h_norm2, sizeof(double) * n_patches);
    if (e != cudaSuccess) st = bcuda(B, e, "cudaMallocHost");
  }
  B->P.assign(n_patches, nullptr);
  for (int p = 0; p < n_patches && st == MG_OK; ++p) {
    mg_hierarchy* H = nullptr;
    st = mg_create_hierarchy(masks[p], where, dims[3 * p], dims[3 * p + 1], dims[3 * p + 2], h[p], &o, B->stream, &H);
    if (st != MG_OK) {
      std::string msg = "patch " + std::to_string(p) + ": " + mg_last_error(nullptr);
      st = bfail(B, st, msg);
      break;
    }
    B->P[p] = H;
  }
  if (st == MG_OK) st = build_tables(B);
  if (st != MG_OK) {
    std::string msg = B->last_error;
    destroy_batch(B);
    set_thread_error(msg.c_str());
    return st;
  }
  *out = B;
  return MG_OK;
}

mg_status mg_batch_destroy(mg_batch* B) {
  destroy_batch(B);
  return MG_OK;
}

mg_status mg_batch_patch(mg_batch* B, int p, mg_hierarchy** out) {
  if (!B || !out || p < 0 || p >= B->n) return bfail(B, MG_ERR_INVALID_ARG, "null batch/output or patch out of range");
  *out = B->P[p];
  return MG_OK;
}

mg_status mg_batch_vcycle(mg_batch* B, double* rel_out) {
  if (!B) return bfail(B, MG_ERR_INVALID_ARG, "null batch");
  Guard guard(B->device);
  std::vector<double> r_zero, r_init;
  if (rel_out) BCKS(initial_norms(B, r_zero, r_init));
  for (int p = 0; p < B->n; ++p) {
    B->h_state[p] = state_word(B, p, start_order(B->P[p]));
    B->P[p]->prepared = false;
  }
  BCKS(run_cycle(B));
  for (int p = 0; p < B->n; ++p)
    if (check_faults(B->P[p]) != MG_OK) return bfail(B, MG_ERR_INTERNAL, "patch " + std::to_string(p) + ": " +
                                                                          B->P[p]->last_error);
  if (!rel_out) return MG_OK;
  bool finite = true;
  for (int p = 0; p < B->n; ++p) {
    const double h2 = B->P[p]->h * B->P[p]->h;
    const double r = std::sqrt(B->h_norm2[p]) / h2;
    rel_out[p] = r_zero[p] > 0 ? r / r_zero[p] : 0.0;
    finite = finite && std::isfinite(r);
  }
  if (!finite) return bfail(B, MG_ERR_DIVERGED, "non-finite residual");
  return MG_OK;
}

mg_status mg_batch_solve(mg_batch* B, double tol, int max_cycles, mg_solve_info* infos) {
  if (!B) return bfail(B, MG_ERR_INVALID_ARG, "null batch");
  if (!(tol > 0) || max_cycles < 0) return bfail(B, MG_ERR_INVALID_ARG, "tol must be > 0 and max_cycles >= 0");
  Guard guard(B->device);
  return solve_impl(B, tol, max_cycles, infos);
}

mg_status mg_batch_get_tuning(const mg_batch* B, mg_batch_tuning* out) {
  if (!B || !out) return bfail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  *out = B->tune;
  return MG_OK;
}

mg_status mg_batch_set_tuning(mg_batch* B, const mg_batch_tuning* t) {
  if (!B || !t) return bfail(B, MG_ERR_INVALID_ARG, "null argument");
  if (!valid_tuning(*t)) return bfail(B, MG_ERR_INVALID_ARG, "invalid tuning values");
  Guard guard(B->device);
  const double ms = t->ms_per_cycle;
  B->tune = *t;
  B->tune.ms_per_cycle = ms;
  BCKS(set_schedule(B, t->n_pre, t->n_post));
  return build_tables(B);
}

mg_status mg_batch_autotune(mg_batch* B, int reps, double tol, int max_cycles, int flags, mg_batch_tuning* best) {
  if (!B || reps < 1 || reps > 1000) return bfail(B, MG_ERR_INVALID_ARG, "null batch or reps outside 1..1000");
  if ((flags & MG_TUNE_SCHEDULE) && (!(tol > 0) || max_cycles < 1))
    return bfail(B, MG_ERR_INVALID_ARG, "schedule tuning needs tol > 0 and max_cycles >= 1");
  Guard guard(B->device);
  const int n = B->n;
  cudaStream_t s = B->stream;
  // keep each patch's solution and hold counter
  std::vector<double*> keep(n, nullptr);
  std::vector<int> holds(n);
  mg_status st = MG_OK;
  for (int p = 0; p < n && st == MG_OK; ++p) {
    mg_hierarchy* H = B->P[p];
    holds[p] = H->hold;
    const size_t bytes = sizeof(double) * H->L[0].g.total;
    cudaError_t e = dev_malloc((void**)&keep[p], 2 * bytes);
    if (e != cudaSuccess) {
      keep[p] = nullptr;
      st = bcuda(B, e, "cudaMalloc(autotune backup)");
      break;
    }
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
      e = cudaMemcpyAsync((char*)keep[p] + c * bytes, H->L[0].phi[c], bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = bcuda(B, e, "autotune backup");
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (st == MG_OK && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess))
    st = bfail(B, MG_ERR_CUDA, "cudaEventCreate");
  mg_batch_tuning cur = B->tune, top = B->tune;
  double top_ms = 1e300;
  auto time_cycles = [&](double* ms_out) -> mg_status {
    for (int p = 0; p < n; ++p) B->h_state[p] = state_word(B, p, start_order(B->P[p]));
    BCKS(run_cycle(B));  // capture + warm-up
    BCK(B, cudaEventRecord(ev0, s));
    for (int r = 0; r < reps; ++r) {
      BCK(B, cudaGraphLaunch(B->graph, s));
      count_launch((unsigned long long)B->graph_nodes);
    }
    BCK(B, cudaEventRecord(ev1, s));
    BCK(B, cudaEventSynchronize(ev1));
    float ms = 0;
    BCK(B, cudaEventElapsedTime(&ms, ev0, ev1));
    *ms_out = ms / reps;
    return MG_OK;
  };
  if (st == MG_OK) {
    const int threads[3] = {128, 256, 512};
    const int pers[3] = {0, B->sms * 4, B->sms * 8};
    const int bots[3] = {1024, 2048, 4096};
    for (int a = 0; a < 3 && st == MG_OK; ++a)
      for (int b = 0; b < 3 && st == MG_OK; ++b)
        for (int c = 0; c < 3 && st == MG_OK; ++c) {
          mg_batch_tuning t = cur;
          t.threads = threads[a];
          t.persistent_ctas = pers[b];
          t.bottom_slots = bots[c];
          B->tune = t;
          st = build_tables(B);
          double ms = 0;
          if (st == MG_OK) st = time_cycles(&ms);
          if (st == MG_OK && ms < top_ms) {
            top_ms = ms;
            top = t;
            top.ms_per_cycle = ms;
          }
        }
    // the tile shape: list entries per chunk, with the best launch shape
    const mg_batch_tuning shape = top;
    for (int m = 1; m <= 8 && st == MG_OK; m *= 2) {
      mg_batch_tuning t = shape;
      t.chunk = m * shape.threads;
      B->tune = t;
      st = build_tables(B);
      double ms = 0;
      if (st == MG_OK) st = time_cycles(&ms);
      if (st == MG_OK && ms < top_ms) {
        top_ms = ms;
        top = t;
        top.ms_per_cycle = ms;
      }
    }
  }
  if (st == MG_OK && (flags & MG_TUNE_SCHEDULE)) {
    const int sched[4][2] = {{1, 1}, {2, 1}, {2, 2}, {3, 3}};
    double best_solve = 1e300;
    mg_batch_tuning base = top;
    for (int k = 0; k < 4 && st == MG_OK; ++k) {
      mg_batch_tuning t = base;
      B->tune = t;
      set_schedule(B, sched[k][0], sched[k][1]);
      st = build_tables(B);
      for (int p = 0; p < n && st == MG_OK; ++p) {
        mg_hierarchy* H = B->P[p];
        H->hold = holds[p];
        for (int c = 0; c < 2; ++c)
          if (cudaMemsetAsync(H->L[0].phi[c], 0, sizeof(double) * H->L[0].g.total, s) != cudaSuccess)
            st = bfail(B, MG_ERR_CUDA, "autotune reset");
      }
      if (st != MG_OK) break;
      if (cudaEventRecord(ev0, s) != cudaSuccess) {
        st = bfail(B, MG_ERR_CUDA, "cudaEventRecord");
        break;
      }
      mg_status ss = solve_impl(B, tol, max_cycles, nullptr);
      if (ss != MG_OK && ss != MG_ERR_NOT_CONVERGED && ss != MG_ERR_DIVERGED) {
        st = ss;
        break;
      }
      float ms = 0;
      if (cudaEventRecord(ev1, s) != cudaSuccess || cudaEventSynchronize(ev1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) {
        st = bfail(B, MG_ERR_CUDA, "autotune timing");
        break;
      }
      if (ss == MG_OK && ms < best_solve) {
        best_solve = ms;
        top.n_pre = sched[k][0];
        top.n_post = sched[k][1];
      }
    }
  }
  // restore the solutions and hold counters, apply the best parameters
  for (int p = 0; p < n; ++p) {
    mg_hierarchy* H = B->P[p];
    H->hold = holds[p];
    if (!keep[p]) continue;
    const size_t bytes = sizeof(double) * H->L[0].g.total;
    for (int c = 0; c < 2; ++c)
      cudaMemcpyAsync(H->L[0].phi[c], (char*)keep[p] + c * bytes, bytes, cudaMemcpyDeviceToDevice, s);
  }
  cudaStreamSynchronize(s);
  for (double* k : keep)
    if (k) cudaFree(k);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (st != MG_OK) {
    B->tune = cur;
    set_schedule(B, cur.n_pre, cur.n_post);
    build_tables(B);
    return st;
  }
  B->tune = top;
  set_schedule(B, top.n_pre, top.n_post);
  BCKS(build_tables(B));
  if (best) *best = B->tune;
  return MG_OK;
}

mg_status mg_batch_launches_per_cycle(const mg_batch* B, long long* launches) {
  if (!B || !launches) return bfail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  *launches = B->graph_nodes;
  return MG_OK;
}

const char* mg_batch_last_error(const mg_batch* B) { return B ? B->last_error.c_str() : mg_last_error(nullptr); }

}  // extern "C"
