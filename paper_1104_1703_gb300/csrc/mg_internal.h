// Internal declarations shared by the CUDA kernels and the host driver of
// the masked-domain multigrid solver (Guillet & Teyssier, arXiv:1104.1703).
//
// Device layout ("red/black split"): every cell-centred field of a level is
// stored as two arrays, one per Gauss-Seidel colour (red: (i+j+k) even).
// Cell (i, j, k) has colour c = (i+j+k) & 1 and lives at slot q = i >> 1 of
// row (j, k) of array c.  With this layout a half-sweep of one colour reads
// only the other colour's array plus its own right-hand side and writes its
// own array, every access is unit-stride in q, and no thread idles on a cell
// of the wrong colour.  In row (j, k) the colour-c cells sit at
// i = 2q + (c ^ ((j+k) & 1)), so their x-neighbours of the other colour are
// at slots {q-1, q} when that parity bit is 0 and {q, q+1} when it is 1;
// their y and z neighbours are at slot q of the adjacent rows.
//
// Each colour array has a zero halo: one row above and below in y, one plane
// before and after in z, and in x a row pitch P >= hx + 1 so that slot -1
// of a row is the last (padding) slot of the previous row and slot hx is
// padding.  Halo and padding hold 0 forever, so the stencil needs no bounds
// tests: inactive and out-of-box cells contribute the value 0, which is what
// the folded operators below expect.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace gbmg {

constexpr int kMaxLevels = 12;

// Bits of the per-cell code byte.
constexpr uint8_t kActive2 = 1;  // active in second order (S > 0)
constexpr uint8_t kActive1 = 2;  // active in first order (S == 8^l); level 0: same as kActive2
constexpr int kGhostShift = 2;   // level 0: bits 2..7 flag the faces -x,+x,-y,+y,-z,+z whose
                                 // neighbour is inactive or outside the box (ghost faces)

struct Geom {
  int nx, ny, nz;      // cells per axis
  int hx;              // slots per half-row: (nx + 1) / 2
  int P;               // row pitch in elements (>= hx + 1)
  long long sz;        // plane stride: (ny + 2) * P
  long long off0;      // element offset of slot (0, 0, 0): sz + P
  long long total;     // elements per colour array: (nz + 2) * sz
  // Division of an element offset n (0 <= n < 2^31) by sz and by P without
  // an integer divide: floor(n / d) = (n * m) >> (31 + l) with l = ceil(log2 d)
  // and m = ceil(2^(31+l) / d) (Granlund & Montgomery, PLDI 1994, Thm 4.2:
  // exact when 2^(31+l) <= m d <= 2^(31+l) + 2^l).  Set by set_divisors().
  unsigned long long m_sz, m_P;
  int s_sz, s_P;
  // Bounds-checked builds (MG_CHECKED) record the first list entry that
  // fails slot_in_bounds here (device memory of the owning hierarchy, the
  // site of the failing kernel); unused otherwise.
  unsigned* fault;
  __host__ __device__ long long at(int q, int j, int k) const { return off0 + k * sz + (long long)j * P + q; }
  __host__ __device__ long long ncells() const { return (long long)nx * ny * nz; }
  __host__ __device__ int div_sz(unsigned n) const { return (int)(((unsigned long long)n * m_sz) >> s_sz); }
  __host__ __device__ int div_P(unsigned n) const { return (int)(((unsigned long long)n * m_P) >> s_P); }
  // (q, j, k) of the element at offset `at` of a colour array
  __host__ __device__ void slot_of(long long at, int* q, int* j, int* k) const {
    const unsigned rel = (unsigned)(at - off0);
    *k = div_sz(rel);
    const unsigned rem = rel - (unsigned)(*k) * (unsigned)sz;
    *j = div_P(rem);
    *q = (int)(rem - (unsigned)(*j) * (unsigned)P);
  }
  // True iff `at` is the offset of a slot (q, j, k) with q < hx, j < ny and
  // k < nz.  Then every stencil neighbour at +-1, +-P and +-sz lies inside
  // the colour array [0, total), since off0 = sz + P and sz = (ny + 2) P.
  __host__ __device__ bool slot_in_bounds(long long at) const {
    if (at < off0 || at >= off0 + (long long)nz * sz) return false;
    int q, j, k;
    slot_of(at, &q, &j, &k);
    return q < hx && j < ny && k < nz;
  }
  void set_divisors() {
    auto magic = [](unsigned long long d, unsigned long long* m, int* s) {
      int l = 0;
      while ((1ULL << l) < d) ++l;
      *s = 31 + l;
      *m = ((1ULL << (31 + l)) + d - 1) / d;
    };
    magic((unsigned long long)sz, &m_sz, &s_sz);
    magic((unsigned long long)P, &m_P, &s_P);
  }
};

struct LevelDev {
  Geom g;
  int level;
  double* phi[2];    // level 0: Phi; level >= 1: dPhi
  double* rhs[2];    // b = h_l^2 * (right-hand side), Dirichlet terms folded in at level 0
  double* invd[2];   // level >= 1: 1/D of the second-order operator (0 if inactive)
  double* diag[2];   // level >= 1: D of the second-order operator (0 if inactive)
  uint8_t* code[2];  // kActive2 | kActive1 | ghost-face bits
  int32_t* S;        // level >= 1: mask sums, natural layout nx*ny*nz
  // Compact lists of the unknowns: list[order][colour] holds, in slot order,
  // the element offset of every active cell of that colour (bits 0..30) and
  // in bit 31 whether its non-shared x-neighbour is at +1 (else -1).  Level 0
  // has one active set: list[1] == list[2].  count[order*2 + colour] is the
  // list length (device memory, so captured graphs stay valid when the mask
  // changes).
  // Level 0 also keeps, in list[0][c] and count[c], the row segments of
  // 2^seg_shift slots of colour c that hold an active cell (ListJob with
  // that seg_shift; nullptr and seg_shift 0 when the hierarchy sweeps by
  // cell lists).
  uint32_t* list[3][2];
  uint32_t* count;
  uint32_t hcount[6];  // host copy of count (sizes the launch grids)
  double* rhsd[2];     // level 0 of the FP64 method: b / D (nullptr elsewhere)
  int exact_sum = 0;   // level 0: FP64 neighbour sums in integer arithmetic (exact_sum.cuh)
  int seg_shift = 0;   // level 0: log2 of the row-segment length (0: no segment lists)
  int seg_pairs = 0;   // level 0, 16-slot segments: two slots per lane (gs_seg_pair_kernel)
  // FP32 copies for the inner cycles of the mixed-precision form (nullptr
  // when the hierarchy was created for FP64 only); level 0: phi32 is the
  // correction e, rhs32 is -r^ of the FP64 residual.
  float* phi32[2];
  float* rhs32[2];
  float* invd32[2];
  float* diag32[2];
};

enum { kFP64 = 0, kFP32 = 1 };

constexpr uint32_t kListAt = 0x7fffffffu;
constexpr uint32_t kListPlusX = 0x80000000u;
// Row segments of the fine level: 8 or 16 slots (16 or 32 cells).  A
// segment never reaches past its row's padding: q0 + 2^s = 2^s ceil(hx / 2^s)
// <= P for s <= 4 since P is a multiple of 16 with P >= hx + 1, and padding
// slots hold code 0.
constexpr int kSegShiftMin = 3, kSegShiftMax = 4;

struct FineExtra {
  double* rhoh2[2];  // h^2 rho, split layout
  double* bc[2];     // 2 * sum of Phi_b over the ghost faces, split layout
  double* save[2];   // backup of the initial guess for the order switch
  const int8_t* mask;  // natural-layout mask (device)
};

// Multiprocessors of the current device, read once per device and cached;
// launch grids are sized in multiples of it.
int device_sms();

// Every device and pinned-host allocation of the library goes through these
// two.  mg_debug_fail_alloc (mg.h) can make the n-th of them fail as if the
// device were out of memory, to show that each caller cleans up.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t host_malloc(void** p, size_t bytes);

// Launch-count instrumentation.  Between capture_count_begin and
// capture_count_end (one thread, around a stream capture) launches are
// counted for the graph instead of the process; the graph's replays count
// them with count_launch(nodes).
void count_launch(unsigned long long n = 1);
void capture_count_begin();
unsigned long long capture_count_end();

// ---- hierarchy build (kernels_build.cu) ----
cudaError_t launch_build_fine(const LevelDev& L0, const int8_t* mask, unsigned long long* counts2,
                              cudaStream_t s);
cudaError_t launch_mask_coarsen(const LevelDev& Lf, const int8_t* mask_if_fine, const LevelDev& Lc,
                                cudaStream_t s);
cudaError_t launch_coarse_coeffs(const LevelDev& Lc, unsigned long long* counts2, cudaStream_t s);
// One compact list to build (launch_build_lists builds a table of them in
// three launches).  block0: the job's first block in the launch, nblocks
// its blocks of kListThreads (256) slots; the scratch holds one word per
// block of all jobs.
// With seg_shift > 0 the job lists row segments instead of cells: the
// 2^seg_shift consecutive slots of one colour's half-row starting at slot
// q0 = t 2^seg_shift, for every segment with an active slot, written as the
// offset of slot q0 with the row's x-direction bit (the same entry format).
struct ListJob {
  Geom g;
  const uint8_t* code;
  uint32_t* list;
  uint32_t* count;
  unsigned block0, nblocks;
  int colour;
  uint8_t bit;
  int seg_shift;
};
// list entries a job scans (cells, or row segments with seg_shift > 0)
__host__ __device__ inline long long list_job_slots(const Geom& g, int seg_shift) {
  const long long per_row = seg_shift ? (g.hx + (1 << seg_shift) - 1) >> seg_shift : g.hx;
  return per_row * g.ny * g.nz;
}
// The list build scans a level's rows in chunks of 16 slots, one chunk per
// thread (one 16-byte load of the codes; rows are padded to a multiple of 16
// slots), so a chunk holds 16 cell candidates or 16 >> seg_shift segments.
constexpr int kListChunkShift = 4;
static_assert(kSegShiftMax <= kListChunkShift, "a row segment must fit in one list-build chunk");
__host__ __device__ inline long long list_job_chunks(const Geom& g) {
  return (long long)((g.hx + (1 << kListChunkShift) - 1) >> kListChunkShift) * g.ny * g.nz;
}
cudaError_t launch_build_lists(const ListJob* jobs, int njobs, unsigned total_blocks, uint32_t* scratch,
                               cudaStream_t s);
// Buffers of `words` 8-byte words to zero, many per launch.
struct ZeroJob {
  void* ptr;
  long long words;
};
cudaError_t launch_zero_many(const ZeroJob* jobs, int njobs, cudaStream_t s);

// ---- data movement and boundary data (kernels_build.cu) ----
// natural (nx*ny*nz) <-> split; `scale` multiplies, `mask_bit` zeroes cells
// whose code lacks the bit (0: keep all).
cudaError_t launch_natural_to_split(const Geom& g, const double* nat, double* dst0, double* dst1, double scale,
                                    uint8_t* const* code, uint8_t mask_bit, cudaStream_t s);
cudaError_t launch_split_to_natural(const Geom& g, double* const* src, double* nat, cudaStream_t s);
cudaError_t launch_u8_split_to_natural_bits(const Geom& g, uint8_t* const* code, int32_t* nat, uint8_t bit,
                                            cudaStream_t s);
cudaError_t launch_fold_faces(const LevelDev& L0, const FineExtra& F, const double* bx, const double* by,
                              const double* bz, cudaStream_t s);
cudaError_t launch_fold_coarse(const LevelDev& L0, const FineExtra& F, const double* pc, int cnx, int cny,
                               int cnz, int ox, int oy, int oz, int* err_flag, cudaStream_t s);
cudaError_t launch_combine_rhs(const LevelDev& L0, const FineExtra& F, cudaStream_t s);
// The interpolated values as face arrays (zeroed by the caller; only ghost
// faces of active cells are written).
cudaError_t launch_faces_from_coarse(const LevelDev& L0, const double* pc, int cnx, int cny, int cnz, int ox, int oy,
                                    int oz, double* bx, double* by, double* bz, int* err_flag, cudaStream_t s);
// h^2 rho into F.rhoh2 and the folded b into L0.rhs in one pass.
cudaError_t launch_set_rhs(const LevelDev& L0, const FineExtra& F, const double* rho, double h2, bool bc_zero,
                           cudaStream_t s);

// ---- V-cycle kernels (kernels_cycle.cu) ----
// order: 1 or 2; the level's active bit and diagonal follow from it.
// update: level 0 of the mixed form only: also apply Phi += e (FP64) to the
// colour just smoothed (its last sweep of the refinement step)
cudaError_t launch_half_sweep(const LevelDev& L, int order, int colour, int prec, bool update, cudaStream_t s);
cudaError_t launch_smooth_small(const LevelDev& L, int order, int sweeps, int prec, cudaStream_t s);
bool small_level(const Geom& g);
// One-time kernel attributes (shared-memory opt-in) for the current device.
cudaError_t init_cycle_kernels();
// Residual of level Lf restricted into the rhs of Lc as -R1(r) (scaled), dPhi_c = 0.
// black_zero: the last operation on Lf was a complete red-black sweep, so
// the black residual vanishes and only red cells are evaluated.
// all_cells: write every coarse cell (the level API, which exposes the
// whole coarse right-hand side); otherwise, from level 0, only the coarse
// level's second-order unknowns (the V-cycle).
cudaError_t launch_restrict(const LevelDev& Lf, const LevelDev& Lc, int order, bool black_zero, int prec,
                            cudaStream_t s, bool all_cells = false);
// black_only: correct the black unknowns only (a red half-sweep follows,
// which overwrites the red ones without reading them).
cudaError_t launch_prolong(const LevelDev& Lc, const LevelDev& Lf, int order, int prec, bool black_only,
                           cudaStream_t s);
// Sum of squares of the scaled residual of level 0 into partials[0..nblocks),
// then a fixed-order reduction into out[0].  red_only as black_zero above.
// with_phi = false evaluates the residual of Phi = 0 (i.e. of the rhs alone).
cudaError_t launch_residual_norm2(const LevelDev& L0, bool red_only, bool with_phi, double* partials,
                                  int max_partials, double* out, cudaStream_t s);
// One multigrid iteration with n_cycles coarse iterations per level (1: V,
// 2 or more: W) on levels lb .. deepest in one CTA, for small levels (every
// level lb..deepest satisfies small_level); lb >= 1.
// cmat / cmat_n (nullable): the coarsest solve's precomputed map and its
// red and black unknown counts (launch_coarse_maps builds it)
cudaError_t launch_bottom(const LevelDev* levels, int lb, int deepest, int order, int n_pre, int n_post,
                          int coarse_sweeps, int n_cycles, int prec, const void* cmat, const uint32_t* cmat_n,
                          cudaStream_t s);
// The coarsest solve of level L (order) as a map, for the bottom cycle:
// whether it fits, the bytes of one map, and the build of both orders' maps
// in one launch (L1 / L2: the deepest level of order 1 / 2, null for no map).
bool coarse_map_fits(const LevelDev& L, int order);
size_t coarse_map_bytes(int prec);
cudaError_t launch_coarse_maps(const LevelDev* L1, const LevelDev* L2, int sweeps, int prec, void* out1, void* out2,
                               cudaStream_t s);
int residual_norm_blocks(const Geom& g);
// Middle levels (more than 4096, at most kMidSlots cells per colour): the
// V-cycle from level m (1 <= m < lb) through levels m .. lb-1, and the bottom
// lb .. deepest, in one launch of one thread-block cluster.
constexpr long long kMidSlots = 1 << 17;
bool mid_level(const Geom& g);
cudaError_t launch_mid(const LevelDev* levels, int m, int lb, int deepest, int order, int n_pre, int n_post,
                       int coarse_sweeps, int prec, const void* cmat, const uint32_t* cmat_n, cudaStream_t s);
// Mixed precision: FP64 residual of level 0 over every unknown -> FP32
// right-hand side -r^ and zero FP32 correction, plus the norm (like
// launch_residual_norm2); and Phi += e in FP64.
cudaError_t launch_refine_residual(const LevelDev& L0, double* partials, int max_partials, double* out,
                                   cudaStream_t s);
cudaError_t launch_refine_update(const LevelDev& L0, cudaStream_t s);
// rhsd = b / D over level 0 (no-op when the level has no rhsd).
cudaError_t launch_scale_rhs(const LevelDev& L0, cudaStream_t s);

}  // namespace gbmg
