// Batched multi-patch V-cycle kernels (FP64): the Section 2 recipe on many
// independent patches at once.  Each launch covers one level index of every
// patch; its blocks walk a table of chunks (batch_internal.h), and every
// chunk is a run of consecutive entries of one compact list of one patch
// level, so a block works on one patch at a time with that patch's pitch and
// arrays.  The arithmetic per unknown is that of the single-hierarchy
// kernels (cycle_device.cuh): the same folded operator, GS update, R1 and
// P2, in the same order of operations.
//
// A patch takes part in a chunk's work only when the per-patch state word
// says so: a patch that has converged does nothing, and coarse-level chunks
// run only for patches currently in the chunk's order (Section 4 switches
// the order of each patch on its own).  The small coarse levels of each
// patch run as the one-CTA bottom V-cycle, one CTA per patch.
#include "batch_internal.h"
#include "cycle_device.cuh"

namespace gbmg {

namespace {

constexpr int kPer = 2;              // list entries per thread in a chunk
constexpr int kBatchMaxThreads = 512;

__device__ __forceinline__ bool chunk_runs(const Chunk& C, int st) {
  const int o = st & kStOrder;
  if (o == 0) return false;
  if (C.tag == 0) return !(st & kStDeep0);
  return o == C.tag;
}

__device__ __forceinline__ const uint32_t* chunk_list(const PatchLevel& L, const Chunk& C) {
  return L.list[C.tag ? C.tag : 2][C.colour] + C.start;
}

// One colour of a Gauss-Seidel sweep over the entries of one chunk.  At
// level 0 the right-hand side is b / D and the update one fused
// multiply-add, as in the single-hierarchy FP64 sweep; with EXACT the
// neighbour sum is formed in integer arithmetic as there (option
// fp64_sum).
template <int KIND, bool EXACT = false>
__device__ __forceinline__ void gs_chunk(const PatchLevel& L, const Chunk& C, const double* tab) {
  const int c = C.colour;
  double* __restrict__ self = L.phi[c];
  const double* __restrict__ other = L.phi[c ^ 1];
  const double* __restrict__ rhs = KIND == 0 ? L.rhsd[c] : L.rhs[c];
  const double* __restrict__ invd = L.invd[c];
  const uint8_t* __restrict__ code = L.code[c];
  const uint32_t* __restrict__ list = chunk_list(L, C);
  const int P = L.g.P;
  const long long sz = L.g.sz;
  for (int i0 = 0; i0 < C.n; i0 += kPer * blockDim.x) {
    long long at[kPer];
    double s[kPer], b[kPer], d[kPer];
    bool ok[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int i = i0 + threadIdx.x + u * blockDim.x;
      ok[u] = i < C.n;
      const uint32_t e = ok[u] ? list[i] : 0u;
      at[u] = e & kListAt;
      ok[u] = ok[u] && entry_ok(L.g, at[u], 20);
      if (ok[u]) {
        if constexpr (EXACT)
          s[u] = nbr_sum_exact(other, at[u], (e & kListPlusX) ? 1 : -1, P, sz);
        else
          s[u] = nbr_sum(other, at[u], (e & kListPlusX) ? 1 : -1, P, sz);
        b[u] = rhs[at[u]];
        d[u] = inv_diag<KIND>(KIND == 0 ? code[at[u]] : 0, invd, at[u], tab);
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u)
      if (ok[u]) self[at[u]] = KIND == 0 ? fma(s[u], d[u], -b[u]) : (s[u] - b[u]) * d[u];
  }
}

__global__ void __launch_bounds__(kBatchMaxThreads)
    batch_scale_kernel(const Chunk* __restrict__ chunks, int nchunks, const PatchLevel* __restrict__ pls) {
  pdl_wait();
  __shared__ double tab[16];
  init_tab(tab);
  for (int k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const Chunk C = chunks[k];
    const PatchLevel& L = pls[C.pl];
    const int c = C.colour;
    const uint32_t* __restrict__ list = L.list[2][c] + C.start;
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
      const long long at = list[i] & kListAt;
      if (!entry_ok(L.g, at, 21)) continue;
      L.rhsd[c][at] = L.rhs[c][at] * tab[__popc((unsigned)L.code[c][at] >> kGhostShift)];
    }
  }
}

template <bool FINE, bool EXACT = false>
__global__ void __launch_bounds__(kBatchMaxThreads)
    batch_gs_kernel(const Chunk* __restrict__ chunks, int nchunks, const PatchLevel* __restrict__ pls,
                    const int* __restrict__ state) {
  pdl_wait();
  __shared__ double tab[16];
  if (FINE) init_tab(tab);
  for (int k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const Chunk C = chunks[k];
    const PatchLevel& L = pls[C.pl];
    if (!chunk_runs(C, state[L.patch])) continue;
    if (FINE) gs_chunk<0, EXACT>(L, C, tab);
    else if (C.tag == 2) gs_chunk<1>(L, C, tab);
    else gs_chunk<2>(L, C, tab);
  }
}

// Sum of r^2 over one chunk's entries, r^ = sum_nbr Phi_j - D Phi_i - b the
// scaled residual (MODE 1), or of b^2, the residual of Phi = 0 (MODE 2).
template <int KIND, int MODE>
__device__ __forceinline__ double res_chunk(const PatchLevel& L, const Chunk& C, const double* tab) {
  const int c = C.colour;
  const double* __restrict__ self = L.phi[c];
  const double* __restrict__ other = L.phi[c ^ 1];
  const double* __restrict__ rhs = L.rhs[c];
  const double* __restrict__ diag = L.diag[c];
  const uint8_t* __restrict__ code = L.code[c];
  const uint32_t* __restrict__ list = chunk_list(L, C);
  const int P = L.g.P;
  const long long sz = L.g.sz;
  double acc = 0.0;
  for (int i0 = 0; i0 < C.n; i0 += kPer * blockDim.x) {
    long long at[kPer];
    double r[kPer];
    bool ok[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int i = i0 + threadIdx.x + u * blockDim.x;
      ok[u] = i < C.n;
      const uint32_t e = ok[u] ? list[i] : 0u;
      at[u] = e & kListAt;
      ok[u] = ok[u] && entry_ok(L.g, at[u], 22);
      if (ok[u]) {
        if (MODE == 2) {
          r[u] = -rhs[at[u]];
        } else {
          const double sn = nbr_sum(other, at[u], (e & kListPlusX) ? 1 : -1, P, sz);
          const uint8_t cd = KIND == 0 ? code[at[u]] : 0;
          r[u] = fma(-diag_of<KIND>(cd, diag, at[u], tab), self[at[u]], sn) - rhs[at[u]];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u)
      if (ok[u]) acc = fma(r[u], r[u], acc);
  }
  return acc;
}

// Level-0 norms: one partial sum per chunk (the chunks of a patch are
// contiguous, so the patch sums below add them in a fixed order).
template <int MODE>
__global__ void __launch_bounds__(kBatchMaxThreads)
    batch_norm_kernel(const Chunk* __restrict__ chunks, int nchunks, const PatchLevel* __restrict__ pls,
                      const int* __restrict__ state, double* __restrict__ partials) {
  pdl_wait();
  __shared__ double tab[16];
  init_tab(tab);
  for (int k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const Chunk C = chunks[k];
    const PatchLevel& L = pls[C.pl];
    const int st = state[L.patch];
    const bool run = (st & kStOrder) != 0 && (C.colour == 0 || (st & kStBlackNorm));
    const double acc = run ? res_chunk<0, MODE>(L, C, tab) : 0.0;
    block_reduce_store(acc, partials + k);
    __syncthreads();  // the reduction's shared slots are reused by the next chunk
  }
}

// Residual and R1 in one pass over the entries of a coarse list: each
// coarse cell evaluates the scaled residual of its active children (both
// x-children of coarse cell I sit at fine slot I of the child rows) and
// writes b_c = -1/2 sum r^, dPhi_c = 0 (as restrict_kernel of the single
// hierarchy; only red children when black_zero).
template <int KIND>
__device__ __forceinline__ void restrict_chunk(const PatchLevel& Lc, const PatchLevel& Lf, const Chunk& C,
                                               uint8_t bit, bool black_zero, const double* tab) {
  const int c = C.colour;
  const uint32_t* __restrict__ list = Lc.list[2][c] + C.start;
  const Geom gc = Lc.g, gf = Lf.g;
  const int nsum = black_zero ? 1 : 2;
  for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
    const long long at = list[i] & kListAt;
    if (!entry_ok(gc, at, 23)) continue;
    int Q, J, K;
    gc.slot_of(at, &Q, &J, &K);
    const int I = 2 * Q + ((c ^ J ^ K) & 1);
    double sum = 0.0;
    for (int dk = 0; dk < 2; ++dk) {
      const int kf = 2 * K + dk;
      if (kf >= gf.nz) break;
      for (int dj = 0; dj < 2; ++dj) {
        const int jf = 2 * J + dj;
        if (jf >= gf.ny) break;
        const long long af = gf.at(I, jf, kf);
        for (int cf = 0; cf < nsum; ++cf) {
          const uint8_t cd = Lf.code[cf][af];
          if (!(cd & bit)) continue;
          const double sn = nbr_sum(Lf.phi[cf ^ 1], af, x_offset(cf, jf, kf), gf.P, gf.sz);
          sum += fma(-diag_of<KIND>(cd, Lf.diag[cf], af, tab), Lf.phi[cf][af], sn) - Lf.rhs[cf][af];
        }
      }
    }
    Lc.rhs[c][at] = -0.5 * sum;
    Lc.phi[c][at] = 0.0;
  }
}

__global__ void __launch_bounds__(kBatchMaxThreads)
    batch_restrict_kernel(const Chunk* __restrict__ chunks, int nchunks, const PatchLevel* __restrict__ pls,
                          const int* __restrict__ state, bool black_zero) {
  pdl_wait();
  __shared__ double tab[16];
  init_tab(tab);
  for (int k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const Chunk C = chunks[k];
    const PatchLevel& Lc = pls[C.pl];
    const PatchLevel& Lf = pls[C.pl - 1];
    const int st = state[Lc.patch];
    if (!chunk_runs(C, st)) continue;
    const int o = st & kStOrder;
    if (Lf.level == 0) restrict_chunk<0>(Lc, Lf, C, kActive2, black_zero, tab);
    else if (o == 2) restrict_chunk<1>(Lc, Lf, C, kActive2, black_zero, tab);
    else restrict_chunk<2>(Lc, Lf, C, kActive1, black_zero, tab);
  }
}

// Phi_f += P2(dPhi_c) over the entries of a fine list (27/9/3/1 weights,
// Fig. 3), coarse level = chunk level + 1.
__global__ void __launch_bounds__(kBatchMaxThreads)
    batch_prolong_kernel(const Chunk* __restrict__ chunks, int nchunks, const PatchLevel* __restrict__ pls,
                         const int* __restrict__ state) {
  pdl_wait();
  for (int k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const Chunk C = chunks[k];
    const PatchLevel& Lf = pls[C.pl];
    const PatchLevel& Lc = pls[C.pl + 1];
    if (!chunk_runs(C, state[Lf.patch])) continue;
    const int c = C.colour;
    const uint32_t* __restrict__ list = chunk_list(Lf, C);
    const Geom gf = Lf.g, gc = Lc.g;
    for (int i0 = 0; i0 < C.n; i0 += kPer * blockDim.x) {
      long long at[kPer];
      double w[kPer], old[kPer];
      bool ok[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int i = i0 + threadIdx.x + u * blockDim.x;
        ok[u] = i < C.n;
        if (!ok[u]) continue;
        at[u] = list[i] & kListAt;
        ok[u] = entry_ok(gf, at[u], 24);
        if (!ok[u]) continue;
        int q, j, kk;
        gf.slot_of(at[u], &q, &j, &kk);
        w[u] = p2_sum(gc, (const double*)Lc.phi[0], (const double*)Lc.phi[1], q, j, kk, c, PlainLoad());
        old[u] = Lf.phi[c][at[u]];
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u)
        if (ok[u]) Lf.phi[c][at[u]] = fma(w[u], 1.0 / 64.0, old[u]);
    }
  }
}

// Per-patch, per-order arguments of the bottom launch.
struct BatchBottom {
  BottomArgs<double> a;
  int kind;   // 1: second order, 2: first order, 0: level 0 is the deepest level
  int smem;   // 1: levels staged in shared memory
  uint32_t n0[2];  // kind 0: level-0 unknowns per colour
};

// kind 0: coarse_sweeps red-black sweeps of level 0 inside the CTA.
__device__ void level0_sweeps(const PatchLevel& L, const uint32_t* n, int sweeps, const double* tab) {
  const int P = L.g.P;
  const long long sz = L.g.sz;
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      const uint32_t* list = L.list[2][c];
      for (uint32_t i = threadIdx.x; i < n[c]; i += blockDim.x) {
        const uint32_t e = list[i];
        const long long at = e & kListAt;
        if (!entry_ok(L.g, at, 25)) continue;
        L.phi[c][at] = (nbr_sum(L.phi[c ^ 1], at, (e & kListPlusX) ? 1 : -1, P, sz) - L.rhs[c][at]) *
                       inv_diag<0>(L.code[c][at], (const double*)nullptr, at, tab);
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(kBottomThreads, 1)
    batch_bottom_kernel(const BatchBottom* __restrict__ args, int npatches, const PatchLevel* __restrict__ pls,
                        const int* __restrict__ state) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double tab[16];
  init_tab(tab);
  for (int p = blockIdx.x; p < npatches; p += gridDim.x) {
    const int o = state[p] & kStOrder;
    if (o == 0) continue;
    const BatchBottom& B = args[2 * p + (o - 1)];
    if (B.kind == 0) level0_sweeps(pls[p * kMaxLevels], B.n0, B.a.coarse_sweeps, tab);
    else if (B.kind == 1) {
      if (B.smem) bottom_run<1, double, true>(B.a, smem_raw);
      else bottom_run<1, double, false>(B.a, smem_raw);
    } else {
      if (B.smem) bottom_run<2, double, true>(B.a, smem_raw);
      else bottom_run<2, double, false>(B.a, smem_raw);
    }
    __syncthreads();
  }
}

constexpr int kSumThreads = 256;

__global__ void __launch_bounds__(kSumThreads)
    batch_patch_sums_kernel(const double* __restrict__ partials, const int* __restrict__ first,
                            const int* __restrict__ count, int npatches, double* __restrict__ norm2) {
  pdl_wait();
  for (int p = blockIdx.x; p < npatches; p += gridDim.x) {
    const double* part = partials + first[p];
    const int n = count[p];
    double acc = 0.0;
    for (int e = threadIdx.x; e < n; e += kSumThreads) acc += part[e];
    block_reduce_store(acc, norm2 + p);
    __syncthreads();
  }
}

}  // namespace

size_t batch_bottom_args_bytes() { return sizeof(BatchBottom); }

size_t batch_fill_bottom(void* host_args, int slot, const LevelDev* levels, int lb, int deepest, int order,
                         int n_pre, int n_post, int coarse_sweeps, int patch) {
  (void)patch;
  BatchBottom& B = static_cast<BatchBottom*>(host_args)[slot];
  B = BatchBottom();
  BottomArgs<double>& a = B.a;
  a.n_pre = n_pre;
  a.n_post = n_post;
  a.coarse_sweeps = coarse_sweeps;
  a.n_cycles = 1;  // a batch runs V-cycles
  if (deepest == 0) {
    B.kind = 0;
    B.smem = 0;
    a.nlev = 0;
    B.n0[0] = levels[0].hcount[4];
    B.n0[1] = levels[0].hcount[5];
    return 0;
  }
  B.kind = order == 2 ? 1 : 2;
  a.nlev = deepest - lb + 1;
  if (lb < 1 || a.nlev < 1 || a.nlev > kBottomMaxLevels) return kBottomTooDeep;
  for (int i = 0; i < a.nlev; ++i) {
    const LevelDev& L = levels[lb + i];
    a.L[i].g = L.g;
    for (int c = 0; c < 2; ++c) {
      a.L[i].phi[c] = L.phi[c];
      a.L[i].rhs[c] = L.rhs[c];
      a.L[i].invd[c] = L.invd[c];
      a.L[i].diag[c] = L.diag[c];
      a.L[i].code[c] = L.code[c];
      a.L[i].list[c] = L.list[order][c];
    }
    a.L[i].count = L.count + order * 2;
  }
  a.bit = order == 1 ? kActive1 : kActive2;
  // unknown records of every level, then the deepest levels that fit
  const size_t bytes = plan_bottom_smem(a, levels, lb, order);
  if (bytes > (size_t)kBottomSmemBytes) return kBottomTooDeep;
  B.smem = a.first_smem < a.nlev ? 1 : 0;
  return bytes;
}

cudaError_t init_batch_kernels() {
  return cudaFuncSetAttribute(batch_bottom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottomSmemBytes);
}

int batch_grid(int nchunks, int threads, int persistent_ctas) {
  (void)threads;
  int g = nchunks;
  if (persistent_ctas > 0 && g > persistent_ctas) g = persistent_ctas;
  return g < 1 ? 1 : g;
}

cudaError_t launch_batch_gs(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state, bool fine,
                            bool exact, int threads, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  count_launch();
  if (fine && exact)
    launch_pdl(batch_gs_kernel<true, true>, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state);
  else if (fine) launch_pdl(batch_gs_kernel<true>, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state);
  else launch_pdl(batch_gs_kernel<false>, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state);
  return cudaGetLastError();
}

cudaError_t launch_batch_norm(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state, int mode,
                              double* partials, int threads, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  if (mode != 1 && mode != 2) return cudaErrorInvalidValue;
  count_launch();
  if (mode == 1) launch_pdl(batch_norm_kernel<1>, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state, partials);
  else launch_pdl(batch_norm_kernel<2>, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state, partials);
  return cudaGetLastError();
}

cudaError_t launch_batch_scale(const Chunk* chunks, int nchunks, const PatchLevel* pls, int threads, int grid,
                               cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  count_launch();
  launch_pdl(batch_scale_kernel, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls);
  return cudaGetLastError();
}

cudaError_t launch_batch_restrict(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state,
                                  bool black_zero, int threads, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  count_launch();
  launch_pdl(batch_restrict_kernel, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state, black_zero);
  return cudaGetLastError();
}

cudaError_t launch_batch_prolong(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state,
                                 int threads, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  count_launch();
  launch_pdl(batch_prolong_kernel, dim3(grid), dim3(threads), 0, s, chunks, nchunks, pls, state);
  return cudaGetLastError();
}

cudaError_t launch_batch_bottom(const void* dev_args, int npatches, const PatchLevel* pls, const int* state,
                                size_t smem_bytes, cudaStream_t s) {
  if (npatches <= 0) return cudaSuccess;
  count_launch();
  launch_pdl(batch_bottom_kernel, dim3(npatches), dim3(kBottomThreads), smem_bytes, s, static_cast<const BatchBottom*>(dev_args),
                                                                   npatches, pls, state);
  return cudaGetLastError();
}

cudaError_t launch_batch_patch_sums(const double* partials, const int* first, const int* count, int npatches,
                                    double* norm2, cudaStream_t s) {
  if (npatches <= 0) return cudaSuccess;
  count_launch();
  launch_pdl(batch_patch_sums_kernel, dim3(npatches), dim3(kSumThreads), 0, s, partials, first, count, npatches, norm2);
  return cudaGetLastError();
}

}  // namespace gbmg
