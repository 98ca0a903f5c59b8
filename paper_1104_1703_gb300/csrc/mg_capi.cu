// Host driver and C ABI of the masked-domain multigrid solver (Guillet &
// Teyssier, arXiv:1104.1703).  Builds the per-level geometry and the device
// arena, issues the kernels of kernels_build.cu / kernels_cycle.cu in the
// order of the Section 2 recipe, and runs the solve loop with the run-time
// reconstruction-order switch of Section 4.
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "hier_internal.h"
#include "mg_internal.h"

namespace gbmg {

static std::atomic<unsigned long long> g_launches{0};
// While a graph is being captured on this thread, launches are counted into
// the graph's node count instead (they run only when the graph is replayed).
static thread_local bool t_capturing = false;
static thread_local unsigned long long t_captured = 0;
void count_launch(unsigned long long n) {
  if (t_capturing) t_captured += n;
  else g_launches.fetch_add(n, std::memory_order_relaxed);
}
void capture_count_begin() {
  t_capturing = true;
  t_captured = 0;
}
unsigned long long capture_count_end() {
  t_capturing = false;
  return t_captured;
}

constexpr int kMaxDevices = 64;
static std::atomic<int> g_sms[kMaxDevices];

int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 152;
  int n = g_sms[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    (void)cudaGetLastError();
    n = 152;
  }
  g_sms[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Allocation-failure test hook: when g_fail_countdown is positive, each
// allocation decrements it and the one that brings it to 0 fails.
static std::atomic<int> g_fail_countdown{0};

static bool alloc_should_fail() {
  int c = g_fail_countdown.load();
  while (c > 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t host_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}

}  // namespace gbmg

extern "C" void mg_debug_fail_alloc(int nth) { gbmg::g_fail_countdown.store(nth > 0 ? nth : 0); }

namespace gbmg {
static std::atomic<int> g_stall_pass{0};
}  // namespace gbmg

extern "C" void mg_debug_stall_pass(int on) { gbmg::g_stall_pass.store(on ? 1 : 0); }

namespace {
thread_local std::string t_last_error = "no error";
}  // namespace

namespace gbmg {
// Sets the message mg_last_error(NULL) returns on this thread.
void set_thread_error(const char* msg) { t_last_error = msg; }

// A caller's MG_MEM_DEVICE pointer is read or written by kernels, so it must
// be device (or managed) memory of `device`; a host pointer or another GPU's
// buffer is refused before any copy or launch.  The query allocates nothing.
bool is_device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();  // leave no error behind for the next check
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}
}  // namespace gbmg

using namespace gbmg;

namespace {

struct Arena {
  size_t used = 0;
  size_t reserve(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    return off;
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

mg_status fail(mg_hierarchy* H, mg_status st, const std::string& msg) {
  if (H) H->last_error = msg;
  t_last_error = msg;
  return st;
}

mg_status cuda_fail(mg_hierarchy* H, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(H, e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA, msg);
}

#define CK(H, call)                                         \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((H), e_, #call); \
  } while (0)

#define CKS(call)                              \
  do {                                         \
    mg_status s_ = (call);                     \
    if (s_ != MG_OK) return s_;                \
  } while (0)

Geom make_geom(int nx, int ny, int nz) {
  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.hx = (nx + 1) / 2;
  g.P = ((g.hx + 1) + 15) & ~15;  // multiple of 16: the byte arrays' rows are valid TMA strides
  g.sz = (long long)(ny + 2) * g.P;
  g.off0 = g.sz + g.P;
  g.total = (long long)(nz + 2) * g.sz;
  g.set_divisors();
  return g;
}

// The lists a level keeps, by order: 1 and 2 on coarse levels; level 0 has
// one active set (order 2, aliased as order 1) and, when the fine level
// sweeps by row segments, its segment lists in slot 0.
std::vector<int> list_orders(int level, bool seg) {
  if (level > 0) return {1, 2};
  if (seg) return {0, 2};
  return {2};
}

bool valid_options(const mg_options& o) {
  return o.n_pre >= 0 && o.n_post >= 0 && o.n_cycles >= 1 && o.n_cycles <= 4 && o.coarse_sweeps >= 1 &&
         o.hold_solves >= 0 && std::isfinite(o.eta) && o.eta > 0 && (o.order == 0 || o.order == 1 || o.order == 2) &&
         (o.precision == 0 || o.precision == 1) && o.inner_cycles >= 1 && o.inner_cycles <= 16 &&
         (o.coarse_cluster == 0 || o.coarse_cluster == 1) && (o.smoother_pass == 0 || o.smoother_pass == 1) &&
         (o.fp64_sum == 0 || o.fp64_sum == 1) && o.fine_segments >= 0 && o.fine_segments <= kSegShiftMax - kSegShiftMin + 2 &&
         (o.coarse_matrix == 0 || o.coarse_matrix == 1);
}

// Number of levels: halve (ceil) until every dimension is at most 2.
int plan_levels(int nx, int ny, int nz, int dims[][3]) {
  int n = 0;
  for (;;) {
    dims[n][0] = nx;
    dims[n][1] = ny;
    dims[n][2] = nz;
    ++n;
    if ((nx <= 2 && ny <= 2 && nz <= 2) || n >= kMaxLevels) break;
    nx = (nx + 1) / 2;
    ny = (ny + 1) / 2;
    nz = (nz + 1) / 2;
  }
  return n;
}

mg_status ensure_staging(mg_hierarchy* H, size_t bytes) {
  if (H->staging_bytes >= bytes) return MG_OK;
  if (H->staging) cudaFree(H->staging);
  H->staging = nullptr;
  H->staging_bytes = 0;
  CK(H, dev_malloc(&H->staging, bytes));
  H->staging_bytes = bytes;
  return MG_OK;
}

// Returns a device pointer holding `bytes` of the caller's data.  Host data
// is copied into the staging buffer at `offset` and the stream synchronised
// so the caller may reuse its buffer on return.
mg_status device_view(mg_hierarchy* H, const void* src, mg_mem where, size_t bytes, size_t offset,
                      const void** out) {
  if (where == MG_MEM_DEVICE) {
    if (!is_device_ptr(src, H->device))
      return fail(H, MG_ERR_INVALID_ARG, "an MG_MEM_DEVICE input is not device memory of the hierarchy's GPU");
    *out = src;
    return MG_OK;
  }
  char* dst = (char*)H->staging + offset;
  CK(H, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, H->stream));
  *out = dst;
  return MG_OK;
}

int kind_order(const mg_hierarchy* H) {
  // order for a bare V-cycle or the start of a solve
  if (H->opt.order == 1 || H->opt.order == 2) return H->opt.order;
  return H->hold > 0 ? 1 : 2;
}

mg_status launch_ok(mg_hierarchy* H, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return cuda_fail(H, e, what);
  return MG_OK;
}

// Brackets the launches that `emit` enqueues with a timing event pair when
// kernel timing is on (inside a capture the records become graph nodes).
template <typename F>
mg_status timed(mg_hierarchy* H, F emit) {
  if (!H->timing) return emit();
  std::vector<TimedPair>& pool = H->cap_events ? *H->cap_events : H->events;
  size_t& used = H->cap_events ? H->cap_events_used : H->events_used;
  if (used == pool.size()) {
    TimedPair p;
    CK(H, cudaEventCreate(&p.a));
    CK(H, cudaEventCreate(&p.b));
    pool.push_back(p);
  }
  TimedPair& p = pool[used++];
  const unsigned flags = H->cap_events ? cudaEventRecordExternal : cudaEventRecordDefault;
  CK(H, cudaEventRecordWithFlags(p.a, H->cur, flags));
  CKS(emit());
  CK(H, cudaEventRecordWithFlags(p.b, H->cur, flags));
  return MG_OK;
}

mg_status half_sweep_on(mg_hierarchy* H, const LevelDev& L, int order, int colour, int prec, bool update) {
  auto emit = [&]() { return launch_ok(H, launch_half_sweep(L, order, colour, prec, update, H->cur), "half-sweep"); };
  if (L.level == 0) return timed(H, emit);
  return emit();
}

mg_status half_sweep(mg_hierarchy* H, int l, int order, int colour, int prec, bool update = false) {
  return half_sweep_on(H, H->L[l], order, colour, prec, update);
}

// Level 0 of the mixed form with the temporal-blocked pass: the FP32
// correction alternates between two buffers (cur = 0: L[0].phi32, 1: the
// second buffer); view0 is level 0 with the current one.
LevelDev view0(const mg_hierarchy* H, int cur) {
  LevelDev v = H->L[0];
  if (cur)
    for (int c = 0; c < 2; ++c) v.phi32[c] = H->phi32_alt[c];
  return v;
}

// One temporal-blocked pass (two red-black sweeps) from buffer cur into the
// other; with update, also Phi += e of the result.
mg_status smooth_pass(mg_hierarchy* H, int& cur, bool update) {
  PassArgs a;
  a.g = H->L[0].g;
  for (int c = 0; c < 2; ++c) {
    a.out[c] = cur ? H->L[0].phi32[c] : H->phi32_alt[c];
    a.phi64[c] = update ? H->L[0].phi[c] : nullptr;
  }
  a.tiles = H->pass_tiles;
  a.ntiles = H->pass_ntiles;
  a.err = H->err_flag + 2;
  a.debug_stall = g_stall_pass.load();
  const int input = cur;
  CKS(timed(H, [&]() {
    return launch_ok(H, launch_smooth_pass(H->pass_maps, input, a, H->cur), "temporal-blocked smoothing pass");
  }));
  cur ^= 1;
  return MG_OK;
}

// `sweeps` FP32 sweeps of level 0: pairs as passes, a remaining single sweep
// as two list half-sweeps on the current buffer.
mg_status smooth0_fp32(mg_hierarchy* H, int order, int sweeps, int& cur, bool update_last) {
  for (; sweeps >= 2; sweeps -= 2) CKS(smooth_pass(H, cur, update_last && sweeps == 2));
  if (sweeps == 1) {
    const LevelDev v = view0(H, cur);
    CKS(half_sweep_on(H, v, order, 0, kFP32, update_last));
    CKS(half_sweep_on(H, v, order, 1, kFP32, update_last));
  }
  return MG_OK;
}

// update_last: the last sweep also applies Phi += e (level 0, mixed form)
mg_status smooth(mg_hierarchy* H, int l, int order, int sweeps, int prec = kFP64, bool update_last = false) {
  if (sweeps <= 0) return MG_OK;
  if (small_level(H->L[l].g))
    return launch_ok(H, launch_smooth_small(H->L[l], order, sweeps, prec, H->cur), "small-level smoother");
  for (int s = 0; s < sweeps; ++s) {
    const bool up = update_last && s == sweeps - 1;
    CKS(half_sweep(H, l, order, 0, prec, up));
    CKS(half_sweep(H, l, order, 1, prec, up));
  }
  return MG_OK;
}

// Section 2 recipe at level l, recursing N_cycles times into level l+1, in
// FP64 or (inner cycles of the mixed form) FP32.
mg_status iteration(mg_hierarchy* H, int l, int order, int prec = kFP64, bool update_last = false) {
  const mg_options& o = H->opt;
  // the coarsest solve's precomputed map, when it matches this solve
  const void* cmat = (H->cmat_ok[order] && H->cmat_prec == prec) ? H->cmat[order] : nullptr;
  // the small coarse levels run as one single-CTA launch, which carries
  // the N_cycles recursion below level l itself
  if (l >= 1 && small_level(H->L[l].g))
    return launch_ok(H, launch_bottom(H->L, l, H->deepest[order], order, o.n_pre, o.n_post, o.coarse_sweeps,
                                      o.n_cycles, prec, cmat, H->cmat_n[order], H->cur),
                     "bottom cycle");
  // the middle levels and the bottom as one launch of a thread-block cluster
  if (l >= 1 && o.n_cycles == 1 && o.coarse_cluster && mid_level(H->L[l].g) && l < H->deepest[order]) {
    int lb = l + 1;
    while (lb < H->deepest[order] && !small_level(H->L[lb].g)) ++lb;
    if (lb - l <= 4)
      return launch_ok(H, launch_mid(H->L, l, lb, H->deepest[order], order, o.n_pre, o.n_post, o.coarse_sweeps,
                                     prec, cmat, H->cmat_n[order], H->cur),
                       "middle levels");
  }
  if (l == H->deepest[order]) return smooth(H, l, order, o.coarse_sweeps, prec, update_last);
  if (l == 0 && prec == kFP32 && H->pass_on) {
    // the same steps with the fine level's sweeps as temporal-blocked passes
    int cur = 0;
    CKS(smooth0_fp32(H, order, o.n_pre, cur, false));  // step 1
    CKS(launch_ok(H, launch_restrict(view0(H, cur), H->L[1], order, o.n_pre >= 1, prec, H->cur),
                  "residual/restriction"));  // steps 2-5
    for (int c = 0; c < o.n_cycles; ++c) CKS(iteration(H, 1, order, prec));  // step 5
    CKS(launch_ok(H, launch_prolong(H->L[1], view0(H, cur), order, prec, o.n_post >= 1, H->cur),
                  "prolongation"));  // steps 6-7
    CKS(smooth0_fp32(H, order, o.n_post, cur, update_last));  // step 8
    if (cur)
      for (int c = 0; c < 2; ++c)
        CK(H, cudaMemcpyAsync(H->L[0].phi32[c], H->phi32_alt[c], sizeof(float) * H->L[0].g.total,
                              cudaMemcpyDeviceToDevice, H->cur));
    return MG_OK;
  }
  CKS(smooth(H, l, order, o.n_pre, prec));                                  // step 1
  CKS(launch_ok(H, launch_restrict(H->L[l], H->L[l + 1], order, o.n_pre >= 1, prec, H->cur),
                "residual/restriction"));                                    // steps 2-5
  for (int c = 0; c < o.n_cycles; ++c) CKS(iteration(H, l + 1, order, prec));  // step 5
  CKS(launch_ok(H, launch_prolong(H->L[l + 1], H->L[l], order, prec, o.n_post >= 1, H->cur),
                "prolongation"));  // steps 6-7
  return smooth(H, l, order, o.n_post, prec, update_last);                  // step 8
}

// Gauss-Seidel updates of active cells in one iteration starting at level l.
long long updates(const mg_hierarchy* H, int l, int order) {
  const mg_options& o = H->opt;
  const long long act = l == 0 ? H->active[2][0] : H->active[order][l];
  if (l == H->deepest[order]) return (long long)o.coarse_sweeps * act;
  return (long long)(o.n_pre + o.n_post) * act + (long long)o.n_cycles * updates(H, l + 1, order);
}

// True when the last operation of an iteration on level 0 was a complete
// red-black sweep (then only red cells carry a residual).
bool ends_with_sweep(const mg_hierarchy* H, int order) {
  return H->deepest[order] == 0 ? H->opt.coarse_sweeps >= 1 : H->opt.n_post >= 1;
}

// Enqueues the residual norm (squared, scaled) and its copy to pinned host
// scalar `slot` on H->cur.
mg_status emit_norm2(mg_hierarchy* H, bool red_only, bool with_phi, int slot = 0) {
  CKS(launch_ok(H, launch_residual_norm2(H->L[0], red_only, with_phi, H->partials, H->max_partials,
                                        H->dscal + slot, H->cur),
                "residual norm"));
  CK(H, cudaMemcpyAsync(H->hscal + slot, H->dscal + slot, sizeof(double), cudaMemcpyDeviceToHost, H->cur));
  return MG_OK;
}

mg_status norm2(mg_hierarchy* H, bool red_only, bool with_phi, double* out) {
  CKS(emit_norm2(H, red_only, with_phi));
  CK(H, cudaStreamSynchronize(H->stream));
  *out = H->hscal[0];
  return MG_OK;
}

unsigned long long lists_hash(const mg_hierarchy* H) {
  unsigned long long x = 1469598103934665603ULL;  // FNV-1a over every list length
  for (int l = 0; l < H->nlev; ++l)
    for (int i = 0; i < 6; ++i) {
      x ^= H->L[l].hcount[i];
      x *= 1099511628211ULL;
    }
  return x;
}

void drop_graph(GraphSlot& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.deepest = -2;
}

// Enqueues the FP64 residual of the mixed form (which also writes the FP32
// right-hand side -r^ and zeroes the FP32 correction) and its norm.
mg_status emit_refine_residual(mg_hierarchy* H) {
  CKS(launch_ok(H, launch_refine_residual(H->L[0], H->partials, H->max_partials, H->dscal, H->cur),
                "refinement residual"));
  CK(H, cudaMemcpyAsync(H->hscal, H->dscal, sizeof(double), cudaMemcpyDeviceToHost, H->cur));
  return MG_OK;
}

// One multigrid iteration and the end-of-cycle residual norm (with its copy
// to the host scalar).  FP64: the Section 2 recipe on Phi.  Mixed: the same
// recipe in FP32 on the error equation (inner_cycles times), Phi += e in
// FP64, then the FP64 residual, which also prepares the next step.
mg_status emit_cycle(mg_hierarchy* H, int order) {
  if (H->opt.precision == 1) {
    // Phi += e rides on the last level-0 sweep when there is one
    const bool fused = !small_level(H->L[0].g) &&
                       (H->deepest[order] == 0 ? H->opt.coarse_sweeps >= 1 : H->opt.n_post >= 1);
    for (int i = 0; i < H->opt.inner_cycles; ++i)
      CKS(iteration(H, 0, order, kFP32, fused && i == H->opt.inner_cycles - 1));
    if (!fused) CKS(launch_ok(H, launch_refine_update(H->L[0], H->cur), "refinement update"));
    if (H->pass_on)
      CK(H, cudaMemcpyAsync(H->hscal + 6, H->err_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, H->cur));
    return emit_refine_residual(H);
  }
  CKS(iteration(H, 0, order));
  return emit_norm2(H, ends_with_sweep(H, order), true);
}

// Captures emit_cycle(order) into a graph.
mg_status capture_cycle(mg_hierarchy* H, int order, GraphSlot& gs) {
  drop_graph(gs);
  if (!H->cap_stream) CK(H, cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
  H->cur = H->cap_stream;
  H->cap_events = H->timing ? &gs.events : nullptr;
  H->cap_events_used = 0;
  t_capturing = true;
  t_captured = 0;
  mg_status st = MG_OK;
  cudaError_t e = cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = emit_cycle(H, order);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(H->cap_stream, &graph);
    if (st == MG_OK && e2 == cudaSuccess) {
      e = cudaGraphInstantiate(&gs.exec, graph, 0);
      if (e != cudaSuccess) gs.exec = nullptr;
    } else if (e2 != cudaSuccess) {
      e = e2;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  t_capturing = false;
  H->cur = H->stream;
  H->cap_events = nullptr;
  if (st != MG_OK) return st;
  if (e != cudaSuccess || !gs.exec) return cuda_fail(H, e, "graph capture");
  gs.deepest = H->deepest[order];
  gs.lists_hash = lists_hash(H);
  gs.nodes = t_captured;
  return MG_OK;
}

// One multigrid iteration of `order` followed by the end-of-cycle residual
// norm, replayed from a CUDA graph when use_graphs is set.  If r_out is
// non-null the stream is synchronised and ||r|| is returned.
// b / D of level 0 for the FP64 sweeps, recomputed after b changed.
mg_status ensure_rhsd(mg_hierarchy* H) {
  if (H->rhsd_valid || !H->L[0].rhsd[0]) return MG_OK;
  CKS(launch_ok(H, launch_scale_rhs(H->L[0], H->stream), "b / D"));
  H->rhsd_valid = true;
  return MG_OK;
}

mg_status run_cycle(mg_hierarchy* H, int order, double* r_out) {
  CKS(ensure_rhsd(H));
  if (H->opt.precision == 1 && !H->prepared) CKS(emit_refine_residual(H));
  H->prepared = true;
  if (!H->opt.use_graphs) {
    CKS(emit_cycle(H, order));
  } else {
    GraphSlot& gs = H->graphs[order][H->timing ? 1 : 0];
    if (!gs.exec || gs.deepest != H->deepest[order] || gs.lists_hash != lists_hash(H))
      CKS(capture_cycle(H, order, gs));
    CK(H, cudaGraphLaunch(gs.exec, H->stream));
    count_launch(gs.nodes);
  }
  if (!r_out) return MG_OK;
  CK(H, cudaStreamSynchronize(H->stream));
  if (H->pass_on) {
    int err = 0;
    std::memcpy(&err, H->hscal + 6, sizeof(int));
    if (err) {
      CK(H, cudaMemsetAsync(H->err_flag + 2, 0, sizeof(int), H->stream));
      CK(H, cudaStreamSynchronize(H->stream));
      std::memset(H->hscal + 6, 0, sizeof(int));
      return fail(H, MG_ERR_INTERNAL, "smoothing pass: a shared-memory copy did not complete in time");
    }
  }
  *r_out = std::sqrt(H->hscal[0]) / (H->h * H->h);
  if (H->opt.use_graphs && H->timing) {
    for (auto& p : H->graphs[order][1].events) {
      float ms = 0;
      CK(H, cudaEventElapsedTime(&ms, p.a, p.b));
      H->timed_ms += ms;
      H->timed_launches += 1;
    }
  }
  return MG_OK;
}

mg_status residual(mg_hierarchy* H, bool red_only, double* out) {
  double s2;
  CKS(norm2(H, red_only, true, &s2));
  *out = std::sqrt(s2) / (H->h * H->h);
  return MG_OK;
}

mg_status residual_zero(mg_hierarchy* H, double* out) {
  if (!H->r_zero_valid) {
    double s2;
    CKS(norm2(H, false, false, &s2));
    H->r_zero = std::sqrt(s2) / (H->h * H->h);
    H->r_zero_valid = true;
  }
  *out = H->r_zero;
  return MG_OK;
}

mg_status zero_split(mg_hierarchy* H, const Geom& g, double* const* a) {
  for (int c = 0; c < 2; ++c) CK(H, cudaMemsetAsync(a[c], 0, sizeof(double) * g.total, H->stream));
  return MG_OK;
}

// Hierarchy build (mask sums, codes, diagonals, counts) from H->mask_dev.
// fine_built: level 0's codes and counts were already built from that mask.
// Level 0's codes (unless fine_built: already built from `mask`), the coarse
// levels, the lists and the coarsest maps from `mask` (the hierarchy's own
// when null); one host synchronisation, for the counts.
mg_status build_levels(mg_hierarchy* H, bool fine_built = false, const int8_t* mask = nullptr) {
  cudaStream_t s = H->stream;
  if (!mask) mask = H->mask_dev;
  if (!fine_built) {
    CK(H, cudaMemsetAsync(H->counts, 0, sizeof(unsigned long long) * 2 * kMaxLevels, s));
    CKS(launch_ok(H, launch_build_fine(H->L[0], mask, H->counts, s), "fine build"));
  } else {
    CK(H, cudaMemsetAsync(H->counts + 2, 0, sizeof(unsigned long long) * 2 * (kMaxLevels - 1), s));
  }
  for (int l = 0; l + 1 < H->nlev; ++l) {
    CKS(launch_ok(H, launch_mask_coarsen(H->L[l], l == 0 ? mask : nullptr, H->L[l + 1], s), "mask R1"));
    CKS(launch_ok(H, launch_coarse_coeffs(H->L[l + 1], H->counts + 2 * (l + 1), s), "coarse coefficients"));
  }
  // compact lists of the unknowns, per order and colour (level 0: one set),
  // all in three launches
  CKS(launch_ok(H, launch_build_lists(H->list_jobs, H->n_list_jobs, H->list_blocks, H->list_scratch, s),
                "active lists"));
  if (H->pass_on)
    CKS(launch_ok(H, launch_pass_tiles(H->L[0].g, H->L[0].code, H->pass_flags, H->pass_tiles, H->pass_ntiles, s),
                  "pass tiles"));
  unsigned long long hc[2 * kMaxLevels];
  CK(H, cudaMemcpyAsync(hc, H->counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
  for (int l = 0; l < H->nlev; ++l)
    CK(H, cudaMemcpyAsync(H->L[l].hcount, H->L[l].count, sizeof(H->L[l].hcount), cudaMemcpyDeviceToHost, s));
  CK(H, cudaStreamSynchronize(s));
  for (int c = 0; c < 2; ++c) H->L[0].hcount[2 + c] = H->L[0].hcount[4 + c];  // level 0: one active set
  for (int l = 0; l < H->nlev; ++l) {
    H->active[2][l] = (long long)hc[2 * l];
    H->active[1][l] = l == 0 ? (long long)hc[0] : (long long)hc[2 * l + 1];
  }
  for (int o = 1; o <= 2; ++o) {
    H->deepest[o] = -1;
    for (int l = 0; l < H->nlev && H->active[o][l] > 0; ++l) H->deepest[o] = l;
  }
  // the coarsest solve's map of each order, for the bottom cycle (one launch)
  const LevelDev* mapped[3] = {nullptr, nullptr, nullptr};
  for (int o = 1; o <= 2; ++o) {
    H->cmat_ok[o] = false;
    const int d = H->deepest[o];
    if (!H->cmat[o] || d < 1 || !small_level(H->L[d].g) || !coarse_map_fits(H->L[d], o)) continue;
    mapped[o] = &H->L[d];
    H->cmat_n[o][0] = H->L[d].hcount[o * 2];
    H->cmat_n[o][1] = H->L[d].hcount[o * 2 + 1];
    H->cmat_ok[o] = true;
  }
  if (mapped[1] || mapped[2])
    CKS(launch_ok(H, launch_coarse_maps(mapped[1], mapped[2], H->opt.coarse_sweeps, H->cmat_prec, H->cmat[1], H->cmat[2],
                                        s),
                  "coarsest-solve maps"));
  return MG_OK;
}

mg_status reset_fields(mg_hierarchy* H) {
  // Phi and b of every level, h^2 rho and the folded boundary terms: one launch
  CKS(launch_ok(H, launch_zero_many(H->zero_jobs, H->n_zero_jobs - (H->bc_zero ? 2 : 0), H->stream),
                "field reset"));
  H->bc_zero = true;
  H->r_zero_valid = false;
  H->rhsd_valid = false;
  H->prepared = false;
  return MG_OK;
}

void destroy(mg_hierarchy* H) {
  if (!H) return;
  DeviceGuard guard(H->device);
  if (H->stream) cudaStreamSynchronize(H->stream);
  for (auto& p : H->events) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto& row : H->graphs)
    for (auto& g : row) {
      drop_graph(g);
      for (auto& p : g.events) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
      }
    }
  if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
  if (H->staging) cudaFree(H->staging);
  if (H->arena) cudaFree(H->arena);
  if (H->hscal) cudaFreeHost(H->hscal);
  if (H->own_stream && H->stream) cudaStreamDestroy(H->stream);
  delete H;
}

}  // namespace

namespace gbmg {
// Bounds-checked builds: MG_ERR_INTERNAL when a kernel of this hierarchy
// recorded a list entry outside its level (the fault word is then cleared);
// MG_OK otherwise and always in normal builds.
mg_status check_faults(mg_hierarchy* H) {
#ifdef MG_CHECKED
  unsigned site = 0;
  CK(H, cudaStreamSynchronize(H->stream));
  CK(H, cudaMemcpy(&site, H->err_flag + 1, sizeof(site), cudaMemcpyDeviceToHost));
  if (site) {
    CK(H, cudaMemset(H->err_flag + 1, 0, sizeof(unsigned)));
    return fail(H, MG_ERR_INTERNAL, "bounds check: a list entry outside its level at kernel site " +
                                        std::to_string(site));
  }
#else
  (void)H;
#endif
  return MG_OK;
}
}  // namespace gbmg

namespace {

mg_status check_level(mg_hierarchy* H, int level) {
  if (!H) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy");
  if (level < 0 || level >= H->nlev) return fail(H, MG_ERR_INVALID_ARG, "level out of range");
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_default_options(mg_options* opt) {
  if (!opt) return;
  opt->n_pre = 2;
  opt->n_post = 2;
  opt->n_cycles = 1;
  opt->coarse_sweeps = 50;
  opt->hold_solves = 10;
  opt->eta = 0.5;
  opt->order = 0;
  opt->use_graphs = 1;
  opt->precision = 0;
  opt->inner_cycles = 1;
  opt->coarse_cluster = 0;
  opt->smoother_pass = 0;
  opt->fp64_sum = 1;
  opt->fine_segments = 3;
  opt->coarse_matrix = 1;
}

const char* mg_status_string(mg_status st) {
  switch (st) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_EMPTY_DOMAIN: return "empty domain";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_DIVERGED: return "diverged";
    case MG_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* mg_last_error(const mg_hierarchy* H) { return H ? H->last_error.c_str() : t_last_error.c_str(); }

unsigned long long mg_launch_count(void) { return g_launches.load(); }

int mg_checked_build(void) {
#ifdef MG_CHECKED
  return 1;
#else
  return 0;
#endif
}

mg_status mg_create_hierarchy(const int8_t* mask, mg_mem where, int nx, int ny, int nz, double h,
                              const mg_options* opt, void* cuda_stream, mg_hierarchy** out) {
  if (out) *out = nullptr;
  if (!out || !mask) return fail(nullptr, MG_ERR_INVALID_ARG, "null mask or output pointer");
  if (where != MG_MEM_HOST && where != MG_MEM_DEVICE) return fail(nullptr, MG_ERR_INVALID_ARG, "bad mg_mem");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 2048 || ny > 2048 || nz > 2048)
    return fail(nullptr, MG_ERR_INVALID_ARG, "dimensions must be in 1..2048");
  if (!(h > 0) || !std::isfinite(h)) return fail(nullptr, MG_ERR_INVALID_ARG, "h must be finite and > 0");
  mg_options o;
  mg_default_options(&o);
  if (opt) o = *opt;
  if (!valid_options(o)) return fail(nullptr, MG_ERR_INVALID_ARG, "invalid options");
  if (where == MG_MEM_DEVICE) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, MG_ERR_CUDA, "no CUDA device");
    if (!is_device_ptr(mask, dev))
      return fail(nullptr, MG_ERR_INVALID_ARG, "the MG_MEM_DEVICE mask is not device memory of the current GPU");
  }

  mg_hierarchy* H = new mg_hierarchy();
  H->opt = o;
  H->h = h;
  if (cudaGetDevice(&H->device) != cudaSuccess) {
    delete H;
    return fail(nullptr, MG_ERR_CUDA, "no CUDA device");
  }
  if (cuda_stream) {
    H->stream = (cudaStream_t)cuda_stream;
  } else {
    // a blocking stream: it orders with the legacy default stream, which
    // callers that pass no stream are most likely using
    cudaError_t e = cudaStreamCreate(&H->stream);
    if (e != cudaSuccess) {
      mg_status st = cuda_fail(nullptr, e, "cudaStreamCreate");
      delete H;
      return st;
    }
    H->own_stream = true;
  }
  H->cur = H->stream;
  {
    cudaError_t e0 = init_cycle_kernels();
    if (e0 != cudaSuccess) {
      mg_status st = cuda_fail(nullptr, e0, "kernel attributes");
      destroy(H);
      return st;
    }
  }
  int dims[kMaxLevels][3];
  H->nlev = plan_levels(nx, ny, nz, dims);
  if (make_geom(nx, ny, nz).total >= (1LL << 31)) {
    destroy(H);
    return fail(nullptr, MG_ERR_INVALID_ARG, "grid too large: padded colour arrays must hold < 2^31 elements");
  }

  // one arena for every level array
  Arena A;
  struct Off {
    size_t phi[2], rhs[2], invd[2], diag[2], code[2], list[3][2], count, S;
    size_t f_phi[2], f_rhs[2], f_invd[2], f_diag[2];
  } off[kMaxLevels];
  const bool mixed = o.precision == 1;
  // fine_segments 1, 2: row segments of 8, 16 slots for the FP32 sweeps;
  // 3: 16-slot segments, two slots per lane
  const bool seg = mixed && o.fine_segments >= 1;
  const int seg_shift = seg ? (o.fine_segments >= 3 ? kSegShiftMax : kSegShiftMin + o.fine_segments - 1) : 0;
  for (int l = 0; l < H->nlev; ++l) {
    Geom g = make_geom(dims[l][0], dims[l][1], dims[l][2]);
    H->L[l].g = g;
    H->L[l].level = l;
    for (int c = 0; c < 2; ++c) {
      off[l].phi[c] = A.reserve(sizeof(double) * g.total);
      off[l].rhs[c] = A.reserve(sizeof(double) * g.total);
      off[l].code[c] = A.reserve(g.total);
      for (int o : list_orders(l, seg))
        off[l].list[o][c] = A.reserve(sizeof(uint32_t) * (size_t)list_job_slots(g, o == 0 ? seg_shift : 0));
      if (mixed) {
        off[l].f_phi[c] = A.reserve(sizeof(float) * g.total);
        off[l].f_rhs[c] = A.reserve(sizeof(float) * g.total);
        if (l > 0) {
          off[l].f_invd[c] = A.reserve(sizeof(float) * g.total);
          off[l].f_diag[c] = A.reserve(sizeof(float) * g.total);
        }
      }
      if (l > 0) {
        off[l].invd[c] = A.reserve(sizeof(double) * g.total);
        off[l].diag[c] = A.reserve(sizeof(double) * g.total);
      }
    }
    if (l > 0) off[l].S = A.reserve(sizeof(int32_t) * g.ncells());
    off[l].count = A.reserve(sizeof(uint32_t) * 6);
  }
  // batched build launches: one scratch word per list block of every list
  std::vector<ListJob> ljobs;
  unsigned lblocks = 0;
  for (int l = 0; l < H->nlev; ++l) {
    const Geom& g = H->L[l].g;
    for (int o : list_orders(l, seg))
      for (int c = 0; c < 2; ++c) {
        ListJob j = {};
        j.g = g;
        j.seg_shift = o == 0 ? seg_shift : 0;
        const unsigned nb = (unsigned)((list_job_chunks(g) + 255) / 256);  // one chunk per thread
        j.block0 = lblocks;
        j.nblocks = nb;
        j.colour = c;
        j.bit = o == 1 ? kActive1 : kActive2;
        ljobs.push_back(j);
        lblocks += nb;
      }
  }
  // the temporal-blocked FP32 pass needs a fine level larger than the
  // one-CTA smoother's and a second FP32 correction buffer
  const bool pass = mixed && o.smoother_pass == 1 && !small_level(H->L[0].g) && H->nlev >= 2;
  const int n_zero = 4 * H->nlev + 4 + (mixed ? 2 * H->nlev : 0) + (pass ? 2 : 0);
  const size_t o_lscr = A.reserve(sizeof(uint32_t) * ((size_t)lblocks + 1));
  const size_t o_ljobs = A.reserve(sizeof(ListJob) * ljobs.size());
  const size_t o_zjobs = A.reserve(sizeof(ZeroJob) * n_zero);
  const Geom& g0 = H->L[0].g;
  size_t o_rhoh2[2], o_bc[2], o_save[2], o_rhsd[2] = {0, 0};
  for (int c = 0; c < 2; ++c) {
    if (!mixed) o_rhsd[c] = A.reserve(sizeof(double) * g0.total);
    o_rhoh2[c] = A.reserve(sizeof(double) * g0.total);
    o_bc[c] = A.reserve(sizeof(double) * g0.total);
    o_save[c] = A.reserve(sizeof(double) * g0.total);
  }
  size_t o_alt[2] = {0, 0}, o_pflags = 0, o_ptiles = 0, o_pn = 0;
  if (pass) {
    int nq, nj, nk;
    pass_tile_grid(g0, &nq, &nj, &nk);
    const size_t ncand = (size_t)nq * nj * nk;
    for (int c = 0; c < 2; ++c) o_alt[c] = A.reserve(sizeof(float) * g0.total);
    o_pflags = A.reserve(sizeof(uint32_t) * ncand);
    o_ptiles = A.reserve(sizeof(uint32_t) * ncand);
    o_pn = A.reserve(sizeof(uint32_t));
  }
  size_t o_mask = A.reserve(g0.ncells());
  H->max_partials = residual_norm_blocks(g0);
  size_t o_part = A.reserve(sizeof(double) * H->max_partials);
  size_t o_scal = A.reserve(sizeof(double) * 8);
  size_t o_err = A.reserve(sizeof(int) * 4);
  // the coarsest solve's maps, in the cycles' precision
  const bool cmaps = o.coarse_matrix == 1;
  const int cprec = mixed ? kFP32 : kFP64;
  size_t o_cmat[3] = {0, 0, 0};
  for (int ord = 1; ord <= 2 && cmaps; ++ord) o_cmat[ord] = A.reserve(coarse_map_bytes(cprec));
  size_t o_cnt = A.reserve(sizeof(unsigned long long) * 2 * kMaxLevels);

  cudaError_t e = dev_malloc((void**)&H->arena, A.used);
  if (e != cudaSuccess) {
    mg_status st = cuda_fail(nullptr, e, "cudaMalloc(arena)");
    H->arena = nullptr;
    destroy(H);
    return st;
  }
  e = host_malloc((void**)&H->hscal, sizeof(double) * 8);
  if (e != cudaSuccess) {
    H->hscal = nullptr;
    mg_status st = cuda_fail(nullptr, e, "cudaMallocHost");
    destroy(H);
    return st;
  }
  char* base = H->arena;
  for (int l = 0; l < H->nlev; ++l) {
    for (int c = 0; c < 2; ++c) {
      H->L[l].phi[c] = (double*)(base + off[l].phi[c]);
      H->L[l].rhs[c] = (double*)(base + off[l].rhs[c]);
      H->L[l].code[c] = (uint8_t*)(base + off[l].code[c]);
      H->L[l].list[0][c] = nullptr;
      for (int o : list_orders(l, seg)) H->L[l].list[o][c] = (uint32_t*)(base + off[l].list[o][c]);
      if (l == 0) H->L[l].list[1][c] = H->L[l].list[2][c];
      LevelDev& Lm = H->L[l];
      Lm.phi32[c] = mixed ? (float*)(base + off[l].f_phi[c]) : nullptr;
      Lm.rhs32[c] = mixed ? (float*)(base + off[l].f_rhs[c]) : nullptr;
      Lm.invd32[c] = (mixed && l > 0) ? (float*)(base + off[l].f_invd[c]) : nullptr;
      Lm.diag32[c] = (mixed && l > 0) ? (float*)(base + off[l].f_diag[c]) : nullptr;
      H->L[l].invd[c] = l > 0 ? (double*)(base + off[l].invd[c]) : nullptr;
      H->L[l].diag[c] = l > 0 ? (double*)(base + off[l].diag[c]) : nullptr;
    }
    H->L[l].S = l > 0 ? (int32_t*)(base + off[l].S) : nullptr;
    H->L[l].count = (uint32_t*)(base + off[l].count);
  }
  H->list_scratch = (uint32_t*)(base + o_lscr);
  H->list_jobs = (ListJob*)(base + o_ljobs);
  H->zero_jobs = (ZeroJob*)(base + o_zjobs);
  H->list_blocks = lblocks;
  for (int l = 0; l < H->nlev; ++l) {
    H->L[l].rhsd[0] = H->L[l].rhsd[1] = nullptr;
    H->L[l].exact_sum = (l == 0 && o.fp64_sum == 1) ? 1 : 0;
    H->L[l].seg_shift = l == 0 ? seg_shift : 0;
    H->L[l].seg_pairs = (l == 0 && seg && o.fine_segments >= 3) ? 1 : 0;
  }
  for (int c = 0; c < 2; ++c) {
    H->L[0].rhsd[c] = mixed ? nullptr : (double*)(base + o_rhsd[c]);
    H->F.rhoh2[c] = (double*)(base + o_rhoh2[c]);
    H->F.bc[c] = (double*)(base + o_bc[c]);
    H->F.save[c] = (double*)(base + o_save[c]);
  }
  H->mask_dev = (int8_t*)(base + o_mask);
  H->F.mask = H->mask_dev;
  H->partials = (double*)(base + o_part);
  H->dscal = (double*)(base + o_scal);
  H->err_flag = (int*)(base + o_err);
  H->cmat_prec = cprec;
  for (int ord = 1; ord <= 2; ++ord) H->cmat[ord] = cmaps ? (void*)(base + o_cmat[ord]) : nullptr;
  for (int l = 0; l < H->nlev; ++l) H->L[l].g.fault = (unsigned*)(H->err_flag + 1);
  H->counts = (unsigned long long*)(base + o_cnt);
  if (pass) {
    for (int c = 0; c < 2; ++c) H->phi32_alt[c] = (float*)(base + o_alt[c]);
    H->pass_flags = (uint32_t*)(base + o_pflags);
    H->pass_tiles = (uint32_t*)(base + o_ptiles);
    H->pass_ntiles = (uint32_t*)(base + o_pn);
    // the pass is used only where its tensor maps and shared-memory size
    // are accepted; otherwise the list half-sweeps run (the same results)
    H->pass_on = init_pass_kernel() == cudaSuccess &&
                 make_pass_maps(&H->pass_maps, g0, H->L[0].phi32, H->phi32_alt, H->L[0].rhs32, H->L[0].code);
    (void)cudaGetLastError();
  }

  mg_status st = MG_OK;
  e = cudaMemsetAsync(H->arena, 0, A.used, H->stream);
  if (e != cudaSuccess) st = cuda_fail(H, e, "cudaMemset(arena)");
  if (st == MG_OK) {
    e = cudaMemcpyAsync(H->mask_dev, mask, g0.ncells(),
                        where == MG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, H->stream);
    if (e != cudaSuccess) st = cuda_fail(H, e, "mask copy");
  }
  // job tables of the batched build launches (after the arena is zeroed)
  if (st == MG_OK) {
    size_t jn = 0;
    for (int l = 0; l < H->nlev; ++l)
      for (int o : list_orders(l, seg))
        for (int c = 0; c < 2; ++c, ++jn) {
          ljobs[jn].code = H->L[l].code[c];
          ljobs[jn].list = H->L[l].list[o][c];
          ljobs[jn].count = H->L[l].count + o * 2 + c;
        }
    std::vector<ZeroJob> zjobs;
    for (int l = 0; l < H->nlev; ++l)
      for (int c = 0; c < 2; ++c) {
        zjobs.push_back({H->L[l].phi[c], H->L[l].g.total});
        zjobs.push_back({H->L[l].rhs[c], H->L[l].g.total});
        // FP32 corrections: cells a new mask makes inactive must read 0
        if (mixed) zjobs.push_back({H->L[l].phi32[c], H->L[l].g.total / 2});
      }
    for (int c = 0; c < 2 && pass; ++c) zjobs.push_back({H->phi32_alt[c], g0.total / 2});
    for (int c = 0; c < 2; ++c) zjobs.push_back({H->F.rhoh2[c], g0.total});
    for (int c = 0; c < 2; ++c) zjobs.push_back({H->F.bc[c], g0.total});  // last: skipped when already 0
    H->n_list_jobs = (int)ljobs.size();
    H->n_zero_jobs = (int)zjobs.size();
    cudaError_t ej = cudaMemcpyAsync(H->list_jobs, ljobs.data(), sizeof(ListJob) * ljobs.size(),
                                     cudaMemcpyHostToDevice, H->stream);
    if (ej == cudaSuccess)
      ej = cudaMemcpyAsync(H->zero_jobs, zjobs.data(), sizeof(ZeroJob) * zjobs.size(), cudaMemcpyHostToDevice,
                           H->stream);
    if (ej == cudaSuccess) ej = cudaStreamSynchronize(H->stream);  // the host tables go out of scope
    if (ej != cudaSuccess) st = cuda_fail(H, ej, "job tables");
  }

  if (st == MG_OK) st = build_levels(H);
  if (st == MG_OK && H->deepest[2] < 0) st = fail(H, MG_ERR_EMPTY_DOMAIN, "the mask has no active cell");
  if (st != MG_OK) {
    t_last_error = H->last_error;
    destroy(H);
    return st;
  }
  *out = H;
  return MG_OK;
}

mg_status mg_destroy_hierarchy(mg_hierarchy* H) {
  destroy(H);
  return MG_OK;
}

mg_status mg_update_mask(mg_hierarchy* H, const int8_t* mask, mg_mem where) {
  if (!H || !mask) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy or mask");
  DeviceGuard guard(H->device);
  if (where == MG_MEM_DEVICE && !is_device_ptr(mask, H->device))
    return fail(H, MG_ERR_INVALID_ARG, "the MG_MEM_DEVICE mask is not device memory of the hierarchy's GPU");
  const Geom& g0 = H->L[0].g;
  // validate on a copy first so that an empty mask leaves the old one in force
  CKS(ensure_staging(H, g0.ncells()));
  CK(H, cudaMemcpyAsync(H->staging, mask, g0.ncells(),
                        where == MG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, H->stream));
  // the whole hierarchy is built from the copy; the old mask stays in force
  // (and is rebuilt) if the new one has no active cell
  CKS(build_levels(H, false, (const int8_t*)H->staging));
  if (H->active[2][0] == 0) {
    CKS(build_levels(H));
    return fail(H, MG_ERR_EMPTY_DOMAIN, "the mask has no active cell");
  }
  CK(H, cudaMemcpyAsync(H->mask_dev, H->staging, g0.ncells(), cudaMemcpyDeviceToDevice, H->stream));
  return reset_fields(H);
}

mg_status mg_set_rhs(mg_hierarchy* H, const double* rho, mg_mem where) {
  if (!H || !rho) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy or rho");
  DeviceGuard guard(H->device);
  const Geom& g0 = H->L[0].g;
  const size_t bytes = sizeof(double) * g0.ncells();
  if (where == MG_MEM_HOST) CKS(ensure_staging(H, bytes));
  const void* src;
  CKS(device_view(H, rho, where, bytes, 0, &src));
  CKS(launch_ok(H, launch_set_rhs(H->L[0], H->F, (const double*)src, H->h * H->h, H->bc_zero, H->stream),
                "rho layout and rhs fold"));
  if (where == MG_MEM_HOST) CK(H, cudaStreamSynchronize(H->stream));
  H->r_zero_valid = false;
  H->rhsd_valid = false;
  H->prepared = false;
  return MG_OK;
}

mg_status mg_set_dirichlet(mg_hierarchy* H, const double* bx, const double* by, const double* bz, mg_mem where) {
  if (!H) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy");
  DeviceGuard guard(H->device);
  const Geom& g = H->L[0].g;
  if (!bx && !by && !bz) {
    // homogeneous Dirichlet values: nothing to fold when the folded terms
    // are already zero
    if (H->bc_zero) return MG_OK;
    CKS(zero_split(H, g, H->F.bc));
    CKS(launch_ok(H, launch_combine_rhs(H->L[0], H->F, H->stream), "rhs fold"));
    H->bc_zero = true;
    H->r_zero_valid = false;
    H->rhsd_valid = false;
    H->prepared = false;
    return MG_OK;
  }
  const size_t nfx = (size_t)(g.nx + 1) * g.ny * g.nz, nfy = (size_t)g.nx * (g.ny + 1) * g.nz,
               nfz = (size_t)g.nx * g.ny * (g.nz + 1);
  const void *dx = nullptr, *dy = nullptr, *dz = nullptr;
  if (where == MG_MEM_HOST && (bx || by || bz)) CKS(ensure_staging(H, sizeof(double) * (nfx + nfy + nfz) + 512));
  size_t o2 = ((sizeof(double) * nfx + 255) & ~(size_t)255);
  size_t o3 = o2 + ((sizeof(double) * nfy + 255) & ~(size_t)255);
  if (bx) CKS(device_view(H, bx, where, sizeof(double) * nfx, 0, &dx));
  if (by) CKS(device_view(H, by, where, sizeof(double) * nfy, o2, &dy));
  if (bz) CKS(device_view(H, bz, where, sizeof(double) * nfz, o3, &dz));
  CKS(launch_ok(H, launch_fold_faces(H->L[0], H->F, (const double*)dx, (const double*)dy, (const double*)dz,
                                    H->stream),
                "face fold"));
  H->bc_zero = false;
  CKS(launch_ok(H, launch_combine_rhs(H->L[0], H->F, H->stream), "rhs fold"));
  if (where == MG_MEM_HOST) CK(H, cudaStreamSynchronize(H->stream));
  H->r_zero_valid = false;
  H->rhsd_valid = false;
  H->prepared = false;
  return MG_OK;
}

mg_status mg_set_dirichlet_from_coarse(mg_hierarchy* H, const double* phi_c, mg_mem where, int cnx, int cny,
                                       int cnz, int ox, int oy, int oz) {
  if (!H || !phi_c) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy or coarse potential");
  if (cnx < 2 || cny < 2 || cnz < 2 || cnx > 4096 || cny > 4096 || cnz > 4096)
    return fail(H, MG_ERR_INVALID_ARG, "coarse dimensions must be in 2..4096");
  DeviceGuard guard(H->device);
  const size_t bytes = sizeof(double) * (size_t)cnx * cny * cnz;
  if (where == MG_MEM_HOST) CKS(ensure_staging(H, bytes));
  const void* src;
  CKS(device_view(H, phi_c, where, bytes, 0, &src));
  CK(H, cudaMemsetAsync(H->err_flag, 0, sizeof(int), H->stream));
  H->bc_zero = false;
  CKS(launch_ok(H, launch_fold_coarse(H->L[0], H->F, (const double*)src, cnx, cny, cnz, ox, oy, oz, H->err_flag,
                                     H->stream),
                "coarse interpolation"));
  int err = 0;
  CK(H, cudaMemcpyAsync(H->hscal, H->err_flag, sizeof(int), cudaMemcpyDeviceToHost, H->stream));
  CK(H, cudaStreamSynchronize(H->stream));
  std::memcpy(&err, H->hscal, sizeof(int));
  if (err) {
    CKS(zero_split(H, H->L[0].g, H->F.bc));
    H->bc_zero = true;
    CKS(launch_ok(H, launch_combine_rhs(H->L[0], H->F, H->stream), "rhs fold"));
    H->r_zero_valid = false;
    H->rhsd_valid = false;
  H->prepared = false;
    return fail(H, MG_ERR_INVALID_ARG,
                "a boundary face lies outside the coarse cell centres; Dirichlet values reset to 0");
  }
  CKS(launch_ok(H, launch_combine_rhs(H->L[0], H->F, H->stream), "rhs fold"));
  H->r_zero_valid = false;
  H->rhsd_valid = false;
  H->prepared = false;
  return MG_OK;
}

mg_status mg_faces_from_coarse(mg_hierarchy* H, const double* phi_c, mg_mem where, int cnx, int cny, int cnz, int ox,
                               int oy, int oz, double* bx, double* by, double* bz) {
  if (!H || !phi_c || !bx || !by || !bz) return fail(H, MG_ERR_INVALID_ARG, "null argument");
  if (cnx < 2 || cny < 2 || cnz < 2 || cnx > 4096 || cny > 4096 || cnz > 4096)
    return fail(H, MG_ERR_INVALID_ARG, "coarse dimensions must be in 2..4096");
  DeviceGuard guard(H->device);
  for (const void* p : {(const void*)bx, (const void*)by, (const void*)bz})
    if (!is_device_ptr(p, H->device))
      return fail(H, MG_ERR_INVALID_ARG, "face arrays must be device memory of the hierarchy's GPU");
  const Geom& g = H->L[0].g;
  const size_t bytes = sizeof(double) * (size_t)cnx * cny * cnz;
  if (where == MG_MEM_HOST) CKS(ensure_staging(H, bytes));
  const void* src;
  CKS(device_view(H, phi_c, where, bytes, 0, &src));
  CK(H, cudaMemsetAsync(bx, 0, sizeof(double) * (size_t)(g.nx + 1) * g.ny * g.nz, H->stream));
  CK(H, cudaMemsetAsync(by, 0, sizeof(double) * (size_t)g.nx * (g.ny + 1) * g.nz, H->stream));
  CK(H, cudaMemsetAsync(bz, 0, sizeof(double) * (size_t)g.nx * g.ny * (g.nz + 1), H->stream));
  CK(H, cudaMemsetAsync(H->err_flag, 0, sizeof(int), H->stream));
  CKS(launch_ok(H, launch_faces_from_coarse(H->L[0], (const double*)src, cnx, cny, cnz, ox, oy, oz, bx, by, bz,
                                            H->err_flag, H->stream),
                "coarse interpolation"));
  int err = 0;
  CK(H, cudaMemcpyAsync(H->hscal, H->err_flag, sizeof(int), cudaMemcpyDeviceToHost, H->stream));
  CK(H, cudaStreamSynchronize(H->stream));
  std::memcpy(&err, H->hscal, sizeof(int));
  if (err) return fail(H, MG_ERR_INVALID_ARG, "a boundary face lies outside the coarse cell centres");
  return MG_OK;
}

mg_status mg_set_solution(mg_hierarchy* H, const double* phi, mg_mem where) {
  if (!H) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy");
  DeviceGuard guard(H->device);
  const Geom& g0 = H->L[0].g;
  H->prepared = false;
  if (!phi) return zero_split(H, g0, H->L[0].phi);
  const size_t bytes = sizeof(double) * g0.ncells();
  if (where == MG_MEM_HOST) CKS(ensure_staging(H, bytes));
  const void* src;
  CKS(device_view(H, phi, where, bytes, 0, &src));
  CKS(launch_ok(H, launch_natural_to_split(g0, (const double*)src, H->L[0].phi[0], H->L[0].phi[1], 1.0,
                                          H->L[0].code, kActive2, H->stream),
                "phi layout"));
  if (where == MG_MEM_HOST) CK(H, cudaStreamSynchronize(H->stream));
  return MG_OK;
}

mg_status mg_get_solution(mg_hierarchy* H, double* phi, mg_mem where) {
  return mg_level_get(H, 0, MG_FIELD_PHI, phi, where);
}

mg_status mg_residual_norm(mg_hierarchy* H, double* norm_out, double* norm_zero_out) {
  if (!H) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy");
  DeviceGuard guard(H->device);
  if (norm_out) CKS(residual(H, false, norm_out));
  if (norm_zero_out) CKS(residual_zero(H, norm_zero_out));
  return check_faults(H);
}

mg_status mg_vcycle(mg_hierarchy* H, double* rel_out) {
  if (!H) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy");
  DeviceGuard guard(H->device);
  const int order = kind_order(H);
  if (!rel_out) {
    CKS(run_cycle(H, order, nullptr));
    return check_faults(H);
  }
  double r, r0;
  CKS(run_cycle(H, order, &r));
  CKS(residual_zero(H, &r0));
  CKS(check_faults(H));
  *rel_out = r0 > 0 ? r / r0 : 0.0;
  if (!std::isfinite(r)) return fail(H, MG_ERR_DIVERGED, "non-finite residual");
  return MG_OK;
}

mg_status mg_solve(mg_hierarchy* H, double tol, int max_cycles, mg_solve_info* info) {
  if (!H) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy");
  if (!(tol > 0) || max_cycles < 0) return fail(H, MG_ERR_INVALID_ARG, "tol must be > 0 and max_cycles >= 0");
  DeviceGuard guard(H->device);
  const mg_options& o = H->opt;
  // Section 4: choose the order for this solve
  int order = 2;
  bool auto_switch = false, switched = false;
  if (o.order == 1 || o.order == 2) {
    order = o.order;
  } else if (H->hold > 0) {
    order = 1;
    H->hold -= 1;
  } else {
    auto_switch = true;
  }
  if (H->deepest[order] < 0) order = 2;
  const Geom& g0 = H->L[0].g;
  double r_zero, r_init;
  // ||r(Phi = 0)|| (unless cached) and ||r(initial guess)||, one wait for both
  const bool need_zero = !H->r_zero_valid;
  if (need_zero) CKS(emit_norm2(H, false, false, 1));
  if (o.precision == 1) {
    // the FP64 residual of the initial guess also prepares the first FP32 step
    CKS(emit_refine_residual(H));
    H->prepared = true;
  } else {
    CKS(emit_norm2(H, false, true, 0));
  }
  CK(H, cudaStreamSynchronize(H->stream));
  if (need_zero) {
    H->r_zero = std::sqrt(H->hscal[1]) / (H->h * H->h);
    H->r_zero_valid = true;
  }
  r_zero = H->r_zero;
  r_init = std::sqrt(H->hscal[0]) / (H->h * H->h);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->r_zero = r_zero;
    info->r_init = r_init;
    info->hist[0] = r_init;
  }
  int cycles = 0;
  long long n_updates = 0;
  double r_n = r_init, rel = r_zero > 0 ? r_init / r_zero : 0.0;
  mg_status st = MG_ERR_NOT_CONVERGED;
  if (!std::isfinite(r_zero) || !std::isfinite(r_init)) {
    st = MG_ERR_DIVERGED;  // non-finite data: nothing to iterate on
    r_n = r_init;
    rel = r_init / r_zero;
  } else if (r_zero == 0.0) {
    CKS(zero_split(H, g0, H->L[0].phi));
    r_n = 0.0;
    rel = 0.0;
    st = MG_OK;
  } else if (rel < tol) {
    st = MG_OK;
  } else {
    if (auto_switch)
      for (int c = 0; c < 2; ++c)
        CK(H, cudaMemcpyAsync(H->F.save[c], H->L[0].phi[c], sizeof(double) * g0.total, cudaMemcpyDeviceToDevice,
                              H->stream));
    double r_prev = r_init;
    // A step of the mixed form runs `inner` multigrid iterations, so the
    // Section 4 test (per-iteration ratio > eta) compares the step's ratio
    // with eta^inner: the geometric mean of the iterations' ratios against eta.
    const int inner = o.precision == 1 ? o.inner_cycles : 1;
    const double eta_step = std::pow(o.eta, (double)inner);
    for (cycles = 1; cycles <= max_cycles; ++cycles) {
      CKS(run_cycle(H, order, &r_n));
      n_updates += updates(H, 0, order) * inner;
      if (info && cycles <= MG_HIST_MAX) info->hist[cycles] = r_n;
      if (!std::isfinite(r_n)) {
        st = MG_ERR_DIVERGED;
        break;
      }
      rel = r_n / r_zero;
      if (rel < tol) {
        st = MG_OK;
        break;
      }
      if (auto_switch && !switched && order == 2 && r_n >= 100.0 * DBL_EPSILON * r_zero && r_n / r_prev > eta_step) {
        order = 1;
        switched = true;
        H->hold = o.hold_solves;
        if (r_n > r_init) {
          for (int c = 0; c < 2; ++c)
            CK(H, cudaMemcpyAsync(H->L[0].phi[c], H->F.save[c], sizeof(double) * g0.total,
                                  cudaMemcpyDeviceToDevice, H->stream));
          H->prepared = false;
          r_n = r_init;
        }
      }
      r_prev = r_n;
    }
    if (cycles > max_cycles) cycles = max_cycles;
  }
  if (info) {
    info->cycles = cycles;
    info->order_used = order;
    info->switched = switched ? 1 : 0;
    info->cell_updates = n_updates;
    info->r_final = r_n;
    info->rel = rel;
    info->status = st;
  }
  CKS(check_faults(H));
  if (st == MG_ERR_NOT_CONVERGED) return fail(H, st, "tolerance not reached within max_cycles");
  if (st == MG_ERR_DIVERGED) return fail(H, st, "non-finite residual norm");
  return st;
}

mg_status mg_get_smoother_pass(const mg_hierarchy* H, int* active) {
  if (!H || !active) return fail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  *active = H->pass_on ? 1 : 0;
  return MG_OK;
}

mg_status mg_get_hold(const mg_hierarchy* H, int* hold) {
  if (!H || !hold) return fail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  *hold = H->hold;
  return MG_OK;
}

mg_status mg_set_hold(mg_hierarchy* H, int hold) {
  if (!H || hold < 0) return fail(H, MG_ERR_INVALID_ARG, "null hierarchy or negative hold");
  H->hold = hold;
  return MG_OK;
}

mg_status mg_num_levels(const mg_hierarchy* H, int* nlev, int* d2, int* d1) {
  if (!H) return fail(nullptr, MG_ERR_INVALID_ARG, "null hierarchy");
  if (nlev) *nlev = H->nlev;
  if (d2) *d2 = H->deepest[2];
  if (d1) *d1 = H->deepest[1];
  return MG_OK;
}

mg_status mg_level_info(const mg_hierarchy* H, int level, int* dims3, long long* a2, long long* a1) {
  if (!H || level < 0 || level >= H->nlev) return fail(nullptr, MG_ERR_INVALID_ARG, "bad hierarchy or level");
  const Geom& g = H->L[level].g;
  if (dims3) {
    dims3[0] = g.nx;
    dims3[1] = g.ny;
    dims3[2] = g.nz;
  }
  if (a2) *a2 = H->active[2][level];
  if (a1) *a1 = H->active[1][level];
  return MG_OK;
}

mg_status mg_level_get(mg_hierarchy* H, int level, int field, void* out, mg_mem where) {
  CKS(check_level(H, level));
  if (!out) return fail(H, MG_ERR_INVALID_ARG, "null output");
  DeviceGuard guard(H->device);
  const LevelDev& L = H->L[level];
  const Geom& g = L.g;
  const size_t n = (size_t)g.ncells();
  const size_t elem = field == MG_FIELD_MASKSUM ? sizeof(int32_t) : sizeof(double);
  if (field == MG_FIELD_INVDIAG && level == 0) return fail(H, MG_ERR_INVALID_ARG, "level 0 has no stored 1/D");
  if (field < 0 || field > 3) return fail(H, MG_ERR_INVALID_ARG, "unknown field");
  void* dst = out;
  if (where == MG_MEM_HOST) {
    CKS(ensure_staging(H, n * elem));
    dst = H->staging;
  } else if (!is_device_ptr(out, H->device)) {
    return fail(H, MG_ERR_INVALID_ARG, "the MG_MEM_DEVICE output is not device memory of the hierarchy's GPU");
  }
  if (field == MG_FIELD_PHI) {
    CKS(launch_ok(H, launch_split_to_natural(g, L.phi, (double*)dst, H->stream), "layout"));
  } else if (field == MG_FIELD_RHS) {
    CKS(launch_ok(H, launch_split_to_natural(g, L.rhs, (double*)dst, H->stream), "layout"));
  } else if (field == MG_FIELD_INVDIAG) {
    CKS(launch_ok(H, launch_split_to_natural(g, L.invd, (double*)dst, H->stream), "layout"));
  } else if (level == 0) {
    CKS(launch_ok(H, launch_u8_split_to_natural_bits(g, L.code, (int32_t*)dst, kActive2, H->stream), "layout"));
  } else {
    CK(H, cudaMemcpyAsync(dst, L.S, n * elem, cudaMemcpyDeviceToDevice, H->stream));
  }
  if (where == MG_MEM_HOST) {
    CK(H, cudaMemcpyAsync(out, dst, n * elem, cudaMemcpyDeviceToHost, H->stream));
    CK(H, cudaStreamSynchronize(H->stream));
  }
  return MG_OK;
}

mg_status mg_level_set(mg_hierarchy* H, int level, int field, const void* in, mg_mem where) {
  CKS(check_level(H, level));
  H->prepared = false;
  if (!in) return fail(H, MG_ERR_INVALID_ARG, "null input");
  if (field != MG_FIELD_PHI && field != MG_FIELD_RHS)
    return fail(H, MG_ERR_INVALID_ARG, "only MG_FIELD_PHI and MG_FIELD_RHS can be set");
  DeviceGuard guard(H->device);
  LevelDev& L = H->L[level];
  const size_t bytes = sizeof(double) * (size_t)L.g.ncells();
  if (where == MG_MEM_HOST) CKS(ensure_staging(H, bytes));
  const void* src;
  CKS(device_view(H, in, where, bytes, 0, &src));
  double** dst = field == MG_FIELD_PHI ? L.phi : L.rhs;
  // values of cells inactive in second order are dropped (they are 0 in every mode)
  CKS(launch_ok(H, launch_natural_to_split(L.g, (const double*)src, dst[0], dst[1], 1.0, L.code, kActive2,
                                          H->stream),
                "layout"));
  if (where == MG_MEM_HOST) CK(H, cudaStreamSynchronize(H->stream));
  if (level == 0 && field == MG_FIELD_RHS) {
    H->r_zero_valid = false;
    H->rhsd_valid = false;
  }
  H->prepared = false;
  return MG_OK;
}

mg_status mg_level_smooth(mg_hierarchy* H, int level, int order, int sweeps) {
  CKS(check_level(H, level));
  H->prepared = false;
  if ((order != 1 && order != 2) || sweeps < 0) return fail(H, MG_ERR_INVALID_ARG, "bad order or sweeps");
  DeviceGuard guard(H->device);
  if (level == 0) CKS(ensure_rhsd(H));
  CKS(smooth(H, level, order, sweeps));
  CK(H, cudaStreamSynchronize(H->stream));
  return check_faults(H);
}

mg_status mg_level_restrict(mg_hierarchy* H, int level, int order) {
  CKS(check_level(H, level));
  H->prepared = false;
  if (level + 1 >= H->nlev || (order != 1 && order != 2)) return fail(H, MG_ERR_INVALID_ARG, "bad level/order");
  DeviceGuard guard(H->device);
  CKS(launch_ok(H, launch_restrict(H->L[level], H->L[level + 1], order, false, kFP64, H->stream, true),
                "restriction"));
  CK(H, cudaStreamSynchronize(H->stream));
  return check_faults(H);
}

mg_status mg_level_prolong(mg_hierarchy* H, int level, int order) {
  CKS(check_level(H, level));
  H->prepared = false;
  if (level + 1 >= H->nlev || (order != 1 && order != 2)) return fail(H, MG_ERR_INVALID_ARG, "bad level/order");
  DeviceGuard guard(H->device);
  CKS(launch_ok(H, launch_prolong(H->L[level + 1], H->L[level], order, kFP64, false, H->stream),
                "prolongation"));
  CK(H, cudaStreamSynchronize(H->stream));
  return check_faults(H);
}

mg_status mg_timing_enable(mg_hierarchy* H, int enable) {
  if (!H) return fail(nullptr, MG_ERR_INVALID_ARG, "null hierarchy");
  H->timing = enable != 0;
  return MG_OK;
}

mg_status mg_timing_read(mg_hierarchy* H, long long* launches, double* total_ms) {
  if (!H) return fail(nullptr, MG_ERR_INVALID_ARG, "null hierarchy");
  DeviceGuard guard(H->device);
  CK(H, cudaStreamSynchronize(H->stream));
  double sum = 0;
  for (size_t i = 0; i < H->events_used; ++i) {
    float ms = 0;
    CK(H, cudaEventElapsedTime(&ms, H->events[i].a, H->events[i].b));
    sum += ms;
  }
  if (launches) *launches = (long long)H->events_used + H->timed_launches;
  if (total_ms) *total_ms = sum + H->timed_ms;
  H->events_used = 0;
  H->timed_launches = 0;
  H->timed_ms = 0;
  return MG_OK;
}

}  // extern "C"
