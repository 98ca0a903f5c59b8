// Internal declarations of the batched multi-patch solver: many independent
// AMR patches (each its own masked-domain problem, Section 2 recipe) solved
// together.  Every batched launch sweeps one level index of all patches at
// once: its grid runs over a table of chunks, each chunk a run of at most
// (block size x 2) consecutive entries of one compact list (mg_internal.h)
// of one level of one patch.  A chunk names the patch level through an
// index into a table of PatchLevel descriptors (array pointers and
// geometry), so patches of different shapes share one launch.
#pragma once

#include <cstdint>

#include "mg_internal.h"

namespace gbmg {

// One level of one patch as the batched kernels address it (FP64).
struct PatchLevel {
  Geom g;
  double* phi[2];
  double* rhs[2];
  const double* invd[2];
  const double* diag[2];
  const uint8_t* code[2];
  const uint32_t* list[3][2];  // [order][colour]; level 0: list[2] only
  double* rhsd[2];             // level 0: b / D (the scaled sweep's right-hand side)
  int patch;
  int level;
};

// Entries [start, start + n) of one list of patch level `pl` (an index
// patch * kMaxLevels + level into the PatchLevel table), colour `colour`.
// `tag` is the order a patch must currently be in for the chunk to run (1
// or 2), or 0 for level-0 work, which a patch runs in either order.  The
// list is that of order `tag` (order 2 for tag 0), except for restriction
// chunks, which always run over the second-order list of the coarse level
// (the superset of the first-order one, so that cells of the other order
// are reset too).
struct Chunk {
  uint32_t pl;
  uint32_t start;
  uint16_t n;
  uint8_t tag;
  uint8_t colour;
};

// Per-patch state word, written by the host before each batched cycle.
constexpr int kStOrder = 3;       // 0: the patch does no work; 1 or 2: its current order
constexpr int kStDeep0 = 4;       // its deepest level in that order is level 0
constexpr int kStBlackNorm = 8;   // the end-of-cycle norm needs the black colour too

// Per-patch bottom arguments: the one-CTA V-cycle on the patch's small
// coarse levels (layout owned by kernels_batch.cu; opaque here).
size_t batch_bottom_args_bytes();
// Fills slot (patch, order) of a host copy of the bottom argument array.
// lb..deepest are the levels the CTA runs (lb >= 1), or deepest == 0 for a
// patch whose deepest level is level 0 (the CTA then sweeps level 0
// coarse_sweeps times).  Returns the dynamic shared memory the slot needs
// (0 if it runs from global memory), or kBottomTooDeep when lb..deepest
// holds more levels than the bottom cycle takes.
constexpr size_t kBottomTooDeep = ~(size_t)0;
size_t batch_fill_bottom(void* host_args, int slot, const LevelDev* levels, int lb, int deepest, int order,
                         int n_pre, int n_post, int coarse_sweeps, int patch);

cudaError_t init_batch_kernels();
int batch_grid(int nchunks, int threads, int persistent_ctas);

// Chunked kernels (threads per block = `threads`, chunk size <= 2 * threads).
cudaError_t launch_batch_gs(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state, bool fine,
                            bool exact,
                            int threads, int grid, cudaStream_t s);
// Level-0 chunks: mode 1: per-chunk sum of r^2 into partials[chunk]; 2:
// per-chunk sum of b^2 (the residual of Phi = 0).
cudaError_t launch_batch_norm(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state, int mode,
                              double* partials, int threads, int grid, cudaStream_t s);
// Residual and R1 into the coarse level of each chunk (coarse-list chunks).
// Level-0 chunks: rhsd = b / D of their unknowns (every patch).
cudaError_t launch_batch_scale(const Chunk* chunks, int nchunks, const PatchLevel* pls, int threads, int grid,
                               cudaStream_t s);
cudaError_t launch_batch_restrict(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state,
                                  bool black_zero, int threads, int grid, cudaStream_t s);
cudaError_t launch_batch_prolong(const Chunk* chunks, int nchunks, const PatchLevel* pls, const int* state,
                                 int threads, int grid, cudaStream_t s);
// One CTA per patch: its bottom V-cycle in its current order.
cudaError_t launch_batch_bottom(const void* dev_args, int npatches, const PatchLevel* pls, const int* state,
                                size_t smem_bytes, cudaStream_t s);
// norm2[p] = fixed-order sum of partials[first[p] .. first[p] + count[p]).
cudaError_t launch_batch_patch_sums(const double* partials, const int* first, const int* count, int npatches,
                                    double* norm2, cudaStream_t s);

}  // namespace gbmg
