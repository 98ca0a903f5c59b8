// Device-side building blocks shared by the single-hierarchy cycle kernels
// (kernels_cycle.cu) and the batched multi-patch kernels (kernels_batch.cu):
// the scaled operator of the Section 2 recipe in the red/black split layout
// of mg_internal.h, and the one-CTA V-cycle on small coarse levels.
#pragma once

#include "exact_sum.cuh"
#include "mg_internal.h"

namespace gbmg {
namespace {

constexpr int kBlockX = 32, kBlockY = 4;
constexpr int kListBlock = 256;

// Programmatic dependent launch: the cycle's kernels are launched with
// launch_pdl, so the GPU may schedule a kernel's blocks while the previous
// kernel on the stream drains; each kernel waits here (griddepcontrol.wait,
// a no-op without such a launch) before it reads or writes global memory,
// which keeps the stream order of every memory access.
// After its own wait, a kernel lets the next one be scheduled at once
// (griddepcontrol.launch_dependents): that kernel's blocks become resident
// and wait in their own pdl_wait until this kernel has completed, so the
// next launch costs no gap.  The next kernel cannot start before every block
// of this one has passed its wait, which keeps the chain one kernel deep.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// KIND 0: level 0 (D from the ghost-face count); 1: coarse, second order
// (per-cell D and 1/D); 2: coarse, first order (D = 6).
template <int KIND, typename T>
__device__ __forceinline__ T inv_diag(uint8_t code, const T* __restrict__ invd, uint32_t at, const T* tab) {
  if (KIND == 0) return tab[__popc((unsigned)code >> kGhostShift)];
  if (KIND == 1) return invd[at];
  return T(1) / T(6);
}

// The level-0 diagonal D = 6 + (ghost faces) comes from a table rather than
// an int-to-double conversion, which would run on the FP64 pipe.
template <int KIND, typename T>
__device__ __forceinline__ T diag_of(uint8_t code, const T* __restrict__ diag, uint32_t at, const T* tab) {
  if (KIND == 0) return tab[8 + __popc((unsigned)code >> kGhostShift)];
  if (KIND == 1) return diag[at];
  return T(6);
}

// FP32 <-> FP64 conversions with integer operations only (the conversion
// instructions share the FP64 pipe, the binding resource of the mixed
// form's FP64 kernels).  Narrowing rounds toward zero (it truncates the
// mantissa: relative error below 2^-23; it only feeds the FP32 correction
// problem), so a finite value beyond the float range saturates at +-FLT_MAX
// as round-toward-zero does, and magnitudes below 2^-126 flush to a zero of
// the same sign.  Infinities stay infinite and every NaN stays a NaN.
// Widening is exact (FP32 subnormals, far below any correction, flush to
// zero).
__device__ __forceinline__ float narrow_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned ex = (unsigned)(b >> 52) & 0x7ffu;
  if (ex == 0x7ffu) return __uint_as_float(sign | ((b & 0xfffffffffffffull) ? 0x7fc00000u : 0x7f800000u));
  const int e = (int)ex - 1023 + 127;
  const unsigned mant = (unsigned)((b >> 29) & 0x7fffffu);
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f7fffffu);
  return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

__device__ __forceinline__ double widen_f32(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long mant = (unsigned long long)(b & 0x7fffffu) << 29;
  if (e == 0) return __longlong_as_double((long long)sign);
  if (e == 255) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | mant));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | mant));
}

// Bounds check of a list entry's offset, compiled in only for the
// MG_CHECKED build: an entry outside the level's slots records `site` in
// the geometry's fault word (first failure wins) and is skipped, so the
// host can report MG_ERR_INTERNAL instead of the kernel touching memory
// outside its arrays.  Without MG_CHECKED it is always true and costs
// nothing.
__device__ __forceinline__ bool entry_ok(const Geom& g, long long at, unsigned site) {
#ifdef MG_CHECKED
  if (!g.slot_in_bounds(at)) {
    if (g.fault) atomicCAS(g.fault, 0u, site);
    return false;
  }
#else
  (void)g;
  (void)at;
  (void)site;
#endif
  return true;
}

template <typename T>
__device__ __forceinline__ T nbr_sum(const T* __restrict__ o, long long at, int dx, int P, long long sz) {
  return ((o[at] + o[at + dx]) + (o[at - P] + o[at + P])) + (o[at - sz] + o[at + sz]);
}

// The same six values summed in integer arithmetic (exact_sum.cuh: one
// rounding, no FP64 instruction).
__device__ __forceinline__ double nbr_sum_exact(const double* __restrict__ o, long long at, int dx, int P,
                                                long long sz) {
  const double x[6] = {o[at], o[at + dx], o[at - P], o[at + P], o[at - sz], o[at + sz]};
  return exact_sum(x);
}

// The same sums on 32-bit slot offsets (a colour array holds fewer than
// 2^31 elements, which the hierarchy's constructor checks), so that each
// address is one multiply-add of the offset onto the base pointer rather than
// 64-bit index arithmetic; xo is the offset of the x-neighbour that is not in
// the same slot.  The order of the additions is nbr_sum's.
template <typename T>
__device__ __forceinline__ T nbr_sum32(const T* __restrict__ o, uint32_t at, uint32_t xo, uint32_t P, uint32_t sz) {
  return ((o[at] + o[xo]) + (o[at - P] + o[at + P])) + (o[at - sz] + o[at + sz]);
}

__device__ __forceinline__ double nbr_sum_exact32(const double* __restrict__ o, uint32_t at, uint32_t xo, uint32_t P,
                                                  uint32_t sz) {
  const double x[6] = {o[at], o[xo], o[at - P], o[at + P], o[at - sz], o[at + sz]};
  return exact_sum(x);
}

template <bool EXACT, typename T>
__device__ __forceinline__ T nbr_sum_sel32(const T* __restrict__ o, uint32_t at, uint32_t xo, uint32_t P, uint32_t sz) {
  if constexpr (EXACT && sizeof(T) == 8)
    return nbr_sum_exact32(reinterpret_cast<const double*>(o), at, xo, P, sz);
  else
    return nbr_sum32(o, at, xo, P, sz);
}

// x-neighbour offset of list entry e at offset at
__device__ __forceinline__ uint32_t x_nbr(uint32_t e, uint32_t at) { return (e & kListPlusX) ? at + 1u : at - 1u; }

// nbr_sum, or (EXACT, FP64) nbr_sum_exact
template <bool EXACT, typename T>
__device__ __forceinline__ T nbr_sum_sel(const T* __restrict__ o, long long at, int dx, int P, long long sz) {
  if constexpr (EXACT && sizeof(T) == 8)
    return nbr_sum_exact(reinterpret_cast<const double*>(o), at, dx, P, sz);
  else
    return nbr_sum(o, at, dx, P, sz);
}

// tab[0..7] = 1/(6+n), tab[8..15] = 6+n: the level-0 diagonal and its
// inverse for n ghost faces
template <typename T>
__device__ __forceinline__ void init_tab(T* tab) {
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  if (t < 8) tab[t] = T(1) / (T)(6 + t);
  else if (t < 16) tab[t] = (T)(t - 2);
  __syncthreads();
}

// x offset of the non-shared x-neighbour of a colour-c cell in row (j, k)
__device__ __forceinline__ int x_offset(int c, int j, int k) { return ((c ^ j ^ k) & 1) ? 1 : -1; }

// P2 (Fig. 3) of a fine unknown at slot q of row (j, k), colour c: the
// weighted sum 27 e0 + 9 e1 + 3 e2 + e3 over its 8 nearest coarse cells
// (e0 the parent, e1 / e2 / e3 the corners one, two and three axis steps
// away; divide by 64 for the correction).  The corners are addressed from
// one coarse row base with 32-bit offsets: a step along y or z moves by the
// pitch or the plane stride, and every axis step flips the colour.  `ld`
// loads one coarse value.  Out-of-box corners read the zero halo (the one
// corner that has no halo slot is taken as 0).
struct PlainLoad {
  template <typename T>
  __device__ __forceinline__ T operator()(const T* p) const {
    return *p;
  }
};

template <typename T, typename LD>
__device__ __forceinline__ T p2_sum(const Geom& gc, const T* c0, const T* c1, int q, int j, int k, int c, LD ld) {
  const int ix = 2 * q + ((c ^ j ^ k) & 1);
  const int Xn = q, Xf = q + ((ix & 1) ? 1 : -1);
  const int Yn = j >> 1, Zn = k >> 1;
  const int dY = (j & 1) ? gc.P : -gc.P;
  const int dZ = (k & 1) ? (int)gc.sz : -(int)gc.sz;
  const int row = (int)gc.off0 + Zn * (int)gc.sz + Yn * gc.P;
  const int sn = row + (Xn >> 1), sf = row + (Xf >> 1);
  const bool p = (Xn + Yn + Zn) & 1;
  const T* cp = p ? c1 : c0;  // the parent's colour: corners an even number of steps away
  const T* cq = p ? c0 : c1;  // an odd number of steps away
  const T e0 = ld(cp + sn);
  const T e1 = (ld(cq + sf) + ld(cq + sn + dY)) + ld(cq + sn + dZ);
  const T e2 = (ld(cp + sn + dY + dZ) + ld(cp + sf + dZ)) + ld(cp + sf + dY);
  // the corner three steps away of fine cell (0, 0, 0) is coarse cell
  // (-1, -1, -1), outside the box and, alone of all corners, before the first
  // element of its colour array (offset -1): it holds 0 and is not read
  const int i3 = sf + dY + dZ;
  const T e3 = i3 >= 0 ? ld(cq + i3) : T(0);
  return fma(T(3), e2, fma(T(27), e0, T(9) * e1)) + e3;
}

constexpr int kNormThreads = 256;

__device__ __forceinline__ void block_reduce_store(double acc, double* out) {
  __shared__ double warp_sums[32];
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((t & 31) == 0) warp_sums[t >> 5] = acc;
  __syncthreads();
  if (t < 32) {
    double v = t < nw ? warp_sums[t] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (t == 0) *out = v;
  }
}

// ---------------------------------------------------------------------------
// Bottom of the V-cycle in one CTA
// ---------------------------------------------------------------------------

constexpr int kBottomThreads = 512;
constexpr int kBottomMaxLevels = 8;
constexpr int kBottomSmemBytes = 200 * 1024;

template <typename T>
struct BottomLevel {
  Geom g;
  T* phi[2];             // global copies (read at entry for level lb's b, written at exit)
  T* rhs[2];
  const T* invd[2];
  const T* diag[2];
  const uint8_t* code[2];
  const uint32_t* list[2];   // unknowns of this order, per colour
  const uint32_t* count;     // their numbers (device memory), [colour]
  long long smem_off;    // element offset of this level's staged arrays (phi0, phi1, rhs0, rhs1)
  long long rec_off;     // byte offset of this level's unknown records in shared memory
  uint32_t nrec[2];      // their numbers per colour (the host's copy of count)
};

template <typename T>
struct BottomArgs {
  BottomLevel<T> L[kBottomMaxLevels];
  int nlev;  // levels lb .. deepest
  uint8_t bit;
  int n_pre, n_post, coarse_sweeps;
  int n_cycles;  // coarse iterations per level (Section 5.3): 1 V-cycle, 2 or more W-cycle
  int first_smem;  // levels first_smem .. nlev-1 are staged in shared memory (with SMEM)
  // The coarsest solve as a precomputed map (coarse_matrix_kernel), or
  // nullptr: n_r + n_b rows, n_r + 2 n_b columns (row-major), for the
  // deepest level's n_r red and n_b black unknowns.
  const T* cmat;
  uint32_t cmat_n[2];
};

// Largest coarsest level solved through its precomputed map: unknowns of
// both colours together (the map has at most kCoarseMatMax rows and
// 2 kCoarseMatMax columns; eight of the bottom's 512 threads per row)
constexpr int kCoarseMatMax = 64;

// a level's working arrays: its records (list entries and, second order,
// 1/D per unknown) always in shared memory, its correction and right-hand
// side there when staged
template <typename T>
struct BottomView {
  Geom g;
  T* phi[2];
  T* rhs[2];
  const T* diag[2];
  const uint8_t* code[2];
  uint32_t* list[2];  // shared-memory copies of the lists
  T* rinvd[2];        // 1/D of the listed unknowns, in list order (second order)
  uint32_t n[2];
};

// Shared-memory plan of a bottom launch over levels lb .. lb + a.nlev - 1
// (host side): first the unknown records of every level (read by every
// step: in shared memory they cost no global round trip), then the
// correction and right-hand side of the deepest levels that still fit.
// Returns the dynamic shared memory bytes.
template <typename T>
size_t plan_bottom_smem(BottomArgs<T>& a, const LevelDev* levels, int lb, int order) {
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  size_t off = 0;
  for (int i = 0; i < a.nlev; ++i) {
    const LevelDev& L = levels[lb + i];
    a.L[i].nrec[0] = L.hcount[order * 2];
    a.L[i].nrec[1] = L.hcount[order * 2 + 1];
    const size_t n = (size_t)a.L[i].nrec[0] + a.L[i].nrec[1];
    a.L[i].rec_off = (long long)off;
    off += al(4 * n) + al(sizeof(T) * n);
  }
  a.first_smem = a.nlev;
  size_t staged = 0;
  for (int i = a.nlev - 1; i >= 0; --i) {
    const size_t need = 4 * (size_t)levels[lb + i].g.total * sizeof(T);
    if (off + staged + need > (size_t)kBottomSmemBytes) break;
    staged += need;
    a.first_smem = i;
  }
  long long e = (long long)(off / sizeof(T));
  for (int i = 0; i < a.nlev; ++i) {
    a.L[i].smem_off = e;
    if (i >= a.first_smem) e += 4 * levels[lb + i].g.total;
  }
  return (size_t)e * sizeof(T);
}

// Gauss-Seidel sweeps of one bottom level over its lists of unknowns.  A
// level with at most 64 unknowns per colour is swept by warp 0 alone, with
// warp-level barriers between the half-sweeps (the deepest level of a
// complex domain often has a handful of unknowns and gets 2 * coarse_sweeps
// half-sweeps); otherwise the whole block works and synchronises.  Such a
// sweep is bound by the latency of its dependent chain, so up to two
// unknowns per colour and thread (every level the bottom takes, at 1024
// threads) each thread first loads what stays fixed over the sweeps (slot,
// x-direction, 1/D and b) into registers, and a half-sweep is only the six
// neighbour loads, the update and its store.  (The arithmetic is the list
// kernels', so a level gives the same bits in the bottom as outside it.)
// The hoisted sweeps with K unknowns per colour and thread (K = 1 when a
// colour has at most one unknown per thread, which keeps the loop's state in
// registers under the bottom kernel's 64-register budget).
template <int KIND, typename T, int K>
__device__ __forceinline__ void bottom_sweeps_hoisted(const BottomView<T>& L, int sweeps, unsigned nthr,
                                                      bool one_warp) {
  const Geom& g = L.g;
  T* const phi[2] = {L.phi[0], L.phi[1]};
  const int P = g.P;
  const long long sz = g.sz;
  long long at[2][K];
  int dx[2][K];
  T id[2][K], b[2][K];
  bool has[2][K];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t i = threadIdx.x + k * nthr;
      has[c][k] = i < L.n[c];
      const uint32_t e = has[c][k] ? L.list[c][i] : 0u;
      at[c][k] = e & kListAt;
      has[c][k] = has[c][k] && entry_ok(g, at[c][k], one_warp ? 1 : 2);
      dx[c][k] = (e & kListPlusX) ? 1 : -1;
      id[c][k] = has[c][k] ? (KIND == 1 ? L.rinvd[c][i] : T(1) / T(6)) : T(0);
      b[c][k] = has[c][k] ? L.rhs[c][at[c][k]] : T(0);
    }
  for (int s = 0; s < sweeps; ++s)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (has[c][k]) phi[c][at[c][k]] = (nbr_sum<T>(phi[c ^ 1], at[c][k], dx[c][k], P, sz) - b[c][k]) * id[c][k];
      if (one_warp) __syncwarp();
      else __syncthreads();
    }
}

template <int KIND, typename T>
__device__ void bottom_smooth(const BottomView<T>& L, int sweeps) {
  const Geom& g = L.g;
  const bool one_warp = L.n[0] <= 64 && L.n[1] <= 64;
  const unsigned nthr = one_warp ? 32u : blockDim.x;
  if (threadIdx.x >= nthr) {
    __syncthreads();
    return;
  }
  T* const phi[2] = {L.phi[0], L.phi[1]};
  if (L.n[0] <= nthr && L.n[1] <= nthr) {
    bottom_sweeps_hoisted<KIND, T, 1>(L, sweeps, nthr, one_warp);
  } else if (L.n[0] <= 2 * nthr && L.n[1] <= 2 * nthr) {
    bottom_sweeps_hoisted<KIND, T, 2>(L, sweeps, nthr, one_warp);
  } else {
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 2; ++c) {
        for (uint32_t i = threadIdx.x; i < L.n[c]; i += nthr) {
          const uint32_t e = L.list[c][i];
          const long long at = e & kListAt;
          if (!entry_ok(g, at, 2)) continue;
          phi[c][at] = (nbr_sum<T>(phi[c ^ 1], at, (e & kListPlusX) ? 1 : -1, g.P, g.sz) - L.rhs[c][at]) *
                       (KIND == 1 ? L.rinvd[c][i] : T(1) / T(6));
        }
        if (one_warp) __syncwarp();
        else __syncthreads();
      }
  }
  if (one_warp) __syncthreads();
}

// residual of level f and R1 into level f+1 in one pass over the coarse
// cells (each coarse cell evaluates its own children): b = -1/2 sum r^,
// dPhi = 0.  Children of the black colour carry no residual after a full
// sweep (black_zero).  The children's codes and diagonals (global memory)
// are loaded together, in one round trip, before the residuals, which are
// summed in the order (dk, dj, colour) as restrict_kernel does.  Rows and
// planes past the level's end are its zero halo, whose codes are 0.
template <int KIND, typename T>
__device__ void bottom_restrict(const BottomView<T>& F, const BottomView<T>& C, uint8_t bit, bool black_zero) {
  const Geom g = F.g;
  const Geom gc = C.g;
  const int nc = gc.nx * gc.ny * gc.nz;
  const int ncol = black_zero ? 1 : 2;
  for (int e = threadIdx.x; e < nc; e += blockDim.x) {
    const int I = e % gc.nx, t = e / gc.nx, J = t % gc.ny, K = t / gc.ny;
    long long at[2][2];
    bool act[2][2][2];
    T dg[2][2][2];
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        at[dk][dj] = g.at(I, 2 * J + dj, 2 * K + dk);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          act[dk][dj][c] = c < ncol && (F.code[c][at[dk][dj]] & bit);
          dg[dk][dj][c] = diag_of<KIND>(0, F.diag[c], at[dk][dj], (const T*)nullptr);
        }
      }
    T sum = 0;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          if (act[dk][dj][c]) {
            const long long a = at[dk][dj];
            const T nb = nbr_sum<T>(F.phi[c ^ 1], a, x_offset(c, 2 * J + dj, 2 * K + dk), g.P, g.sz);
            sum += fma(-dg[dk][dj][c], F.phi[c][a], nb) - F.rhs[c][a];
          }
    const int Cc = (I + J + K) & 1;
    const long long atc = gc.at(I >> 1, J, K);
    C.rhs[Cc][atc] = T(-0.5) * sum;
    C.phi[Cc][atc] = T(0);
  }
  __syncthreads();
}


// P2 of level f+1 into the listed unknowns of level f (their records in
// shared memory give the slots, as prolong_list_kernel's lists do)
template <typename T>
__device__ void bottom_prolong(const BottomView<T>& F, const BottomView<T>& C, int first_colour) {
  const Geom& g = F.g;
  for (int c = first_colour; c < 2; ++c)
    for (uint32_t i = threadIdx.x; i < F.n[c]; i += blockDim.x) {
      const long long at = F.list[c][i] & kListAt;
      if (!entry_ok(g, at, 11)) continue;
      int q, j, k;
      g.slot_of(at, &q, &j, &k);
      const T w = p2_sum(C.g, (const T*)C.phi[0], (const T*)C.phi[1], q, j, k, c, PlainLoad());
      F.phi[c][at] = fma(w, T(1) / T(64), F.phi[c][at]);
    }
  __syncthreads();
}

// The coarsest solve through its precomputed map (option coarse_matrix): the
// coarse_sweeps red-black sweeps of level L are an affine map of the
// level's right-hand side b and of its black unknowns' current correction
// (the first red half-sweep overwrites every red one unread),
//   (x_r, x_b)_final = M (b_r, b_b, x_b)_initial,
// which coarse_matrix_kernel has tabulated column by column with the same
// sweeps.  Eight threads form each output row's dot product (partial sums
// strided over the columns, then combined by shuffles).  The result equals
// the sweeps' up to rounding.  Falls back to the sweeps when the level's
// current counts are not the map's.
template <int KIND, typename T>
__device__ void bottom_coarse_map(const BottomView<T>& L, const T* __restrict__ M, const uint32_t* mn, int sweeps,
                                  T* v) {
  const uint32_t nr = mn[0], nb = mn[1];
  if (L.n[0] != nr || L.n[1] != nb || nr + nb > (uint32_t)kCoarseMatMax || blockDim.x < 8 * kCoarseMatMax) {
    bottom_smooth<KIND>(L, sweeps);
    return;
  }
  const uint32_t nt = nr + nb, ncol = nt + nb;
  for (uint32_t j = threadIdx.x; j < ncol; j += blockDim.x) {
    const int c = j < nr ? 0 : (j < nt ? 1 : 2);
    const uint32_t u = c == 0 ? j : (c == 1 ? j - nr : j - nt);
    const long long at = L.list[c == 0 ? 0 : 1][u] & kListAt;
    v[j] = c < 2 ? L.rhs[c][at] : L.phi[1][at];
  }
  __syncthreads();
  constexpr int kParts = 8;
  const uint32_t i = threadIdx.x / kParts, p = threadIdx.x % kParts;
  T acc0 = T(0), acc1 = T(0);
  if (i < nt) {
    const T* row = M + (size_t)i * ncol;
    uint32_t j = p;
    for (; j + kParts < ncol; j += 2 * kParts) {
      acc0 = fma(row[j], v[j], acc0);
      acc1 = fma(row[j + kParts], v[j + kParts], acc1);
    }
    if (j < ncol) acc0 = fma(row[j], v[j], acc0);
  }
  T acc = acc0 + acc1;
#pragma unroll
  for (int off = kParts / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __syncthreads();  // every v read before the corrections are overwritten
  if (i < nt && p == 0) {
    const int c = i < nr ? 0 : 1;
    const uint32_t u = c ? i - nr : i;
    L.phi[c][L.list[c][u] & kListAt] = acc;
  }
  __syncthreads();
}

// The Section 2 recipe with N_cycles coarse iterations per level (Section
// 5.3: 1 is the V-cycle, 2 or more a W-cycle) on the small coarse levels
// lb .. deepest, inside one CTA, from level lb's current state: its
// right-hand side as the restriction left it and its correction (zero on
// the first of a W-cycle's visits, the previous visit's result after that).
// With SMEM the correction and right-hand side of the deepest levels (from
// first_smem on, halo included) live in shared memory for the whole kernel,
// so the many barrier-separated steps (2 * coarse_sweeps of them on each
// visit of the deepest level) read on-chip data that the previous step
// wrote; the results go back to global memory at the end.  Levels above
// first_smem (too large to stage) work in global memory.  Each step is a block-strided loop
// over the level's slots closed by __syncthreads.  This replaces about six
// launches per level visit and the 2 * coarse_sweeps launches of each
// coarsest solve.
template <int KIND, typename T, bool SMEM>
__device__ void bottom_run(const BottomArgs<T>& a, unsigned char* smem_raw, bool wait_after_setup = false) {
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ BottomView<T> V[kBottomMaxLevels];  // one copy per block, read by every thread
  __shared__ T cmat_v[2 * kCoarseMatMax];        // inputs of the coarsest solve's map
  // thread i sets up level i (the list lengths are global loads: made at
  // once rather than one after another)
  if (threadIdx.x < (unsigned)a.nlev) {
    const int i = threadIdx.x;
    {
      const BottomLevel<T>& L = a.L[i];
      V[i].g = L.g;
      const bool st = SMEM && i >= a.first_smem;
      const uint32_t nr = L.nrec[0] + L.nrec[1];
      uint32_t* rl = reinterpret_cast<uint32_t*>(smem_raw + L.rec_off);
      T* ri = reinterpret_cast<T*>(smem_raw + L.rec_off + ((4 * (size_t)nr + 15) & ~(size_t)15));
      for (int c = 0; c < 2; ++c) {
        V[i].phi[c] = st ? sm + L.smem_off + c * L.g.total : L.phi[c];
        V[i].rhs[c] = st ? sm + L.smem_off + (2 + c) * L.g.total : L.rhs[c];
        V[i].diag[c] = L.diag[c];
        V[i].code[c] = L.code[c];
        V[i].list[c] = rl + (c ? L.nrec[0] : 0);
        V[i].rinvd[c] = ri + (c ? L.nrec[0] : 0);
        // the device count, bounded by the records planned for it (the two
        // agree: the host copy is read after every list build)
        const uint32_t n = L.count[c];
        V[i].n[c] = n < L.nrec[c] ? n : L.nrec[c];
      }
    }
  }
  __syncthreads();
  // Staging, as batches of independent global loads (each costs one round
  // trip to L2, far longer than the arithmetic of a small level):
  //  - the unknown records of every level, over one flat index: list
  //    entries, then (second order) 1/D of each listed unknown;
  //  - with SMEM, level lb's b and (W-cycle: later visits start from the
  //    previous one's result) its dPhi; the deeper staged levels are fully
  //    written before they are read except their zero halo, so they are
  //    zeroed.
  __shared__ uint32_t seg_end[2 * kBottomMaxLevels];
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < 2 * a.nlev; ++k) {
      run += V[k >> 1].n[k & 1];
      seg_end[k] = run;
    }
  }
  __syncthreads();
  {
    const uint32_t total = seg_end[2 * a.nlev - 1];
    constexpr int U = 4;
    for (uint32_t r0 = threadIdx.x; r0 < total; r0 += U * blockDim.x) {
      uint32_t ent[U], idx[U];
      int seg[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t r = r0 + u * blockDim.x;
        int k = 0;
        while (k < 2 * a.nlev - 1 && r >= seg_end[k]) ++k;
        seg[u] = k;
        idx[u] = r - (k ? seg_end[k - 1] : 0u);
        ent[u] = r < total ? a.L[k >> 1].list[k & 1][idx[u]] : 0u;
      }
      T iv[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        iv[u] = (KIND == 1 && r0 + u * blockDim.x < total)
                    ? a.L[seg[u] >> 1].invd[seg[u] & 1][ent[u] & kListAt] : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (r0 + u * blockDim.x < total) {
          V[seg[u] >> 1].list[seg[u] & 1][idx[u]] = ent[u];
          if (KIND == 1) V[seg[u] >> 1].rinvd[seg[u] & 1][idx[u]] = iv[u];
        }
    }
  }
  // The level views and the unknown records are built with the mask and do
  // not change during a solve: a kernel of its own stages them before the
  // wait on the previous kernel, which wrote level lb's right-hand side.
  if (wait_after_setup) pdl_wait();
  if (SMEM) {
    const bool keep = a.n_cycles > 1;
    for (int i = a.first_smem > 1 ? a.first_smem : 1; i < a.nlev; ++i) {
      const long long tot = a.L[i].g.total;
      for (int c = 0; c < 2; ++c)
        for (long long e = threadIdx.x; e < tot; e += blockDim.x) V[i].phi[c][e] = V[i].rhs[c][e] = T(0);
    }
    if (a.first_smem == 0) {
      const long long tot = a.L[0].g.total;
      if (keep) {
        constexpr int U = 8;
        for (long long e0 = threadIdx.x; e0 < 2 * tot; e0 += U * (long long)blockDim.x) {
          T r[U], ph[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long e = e0 + u * (long long)blockDim.x;
            const int c = e >= tot;
            const long long o = e - c * tot;
            r[u] = e < 2 * tot ? a.L[0].rhs[c][o] : T(0);
            ph[u] = e < 2 * tot ? a.L[0].phi[c][o] : T(0);
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long e = e0 + u * (long long)blockDim.x;
            const int c = e >= tot;
            const long long o = e - c * tot;
            if (e < 2 * tot) {
              V[0].rhs[c][o] = r[u];
              V[0].phi[c][o] = ph[u];
            }
          }
        }
      } else {
        // b only (dPhi is 0), in batches of 24 loads per thread: the usual
        // 16^3 top level of the bottom in one round trip at 512 threads
        constexpr int U = 24;
        for (long long e0 = threadIdx.x; e0 < 2 * tot; e0 += U * (long long)blockDim.x) {
          T r[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long e = e0 + u * (long long)blockDim.x;
            const int c = e >= tot;
            r[u] = e < 2 * tot ? a.L[0].rhs[c][e - c * tot] : T(0);
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long e = e0 + u * (long long)blockDim.x;
            const int c = e >= tot;
            if (e < 2 * tot) {
              V[0].rhs[c][e - c * tot] = r[u];
              V[0].phi[c][e - c * tot] = T(0);
            }
          }
        }
      }
    }
  }
  __syncthreads();
  // The recursion mg(i) = {smooth n_pre; restrict into i+1; N_cycles times
  // mg(i+1); prolong; smooth n_post}, with mg(deepest) = coarse_sweeps
  // sweeps, unrolled with one counter per level (the same in every thread):
  // owe[i] is the number of visits of level i+1 that level i still owes.
  const int last = a.nlev - 1;
  int owe[kBottomMaxLevels];
  int i = 0;
  for (;;) {
    for (; i < last; ++i) {  // descend: a fresh visit of level i
      bottom_smooth<KIND>(V[i], a.n_pre);
      bottom_restrict<KIND>(V[i], V[i + 1], a.bit, a.n_pre >= 1);
      owe[i] = a.n_cycles;
    }
    if (a.cmat) bottom_coarse_map<KIND>(V[last], a.cmat, a.cmat_n, a.coarse_sweeps, cmat_v);
    else bottom_smooth<KIND>(V[last], a.coarse_sweeps);
    for (i = last - 1; i >= 0; --i) {  // ascend until a level owes a visit
      if (--owe[i] > 0) break;
      bottom_prolong(V[i], V[i + 1], a.n_post >= 1 ? 1 : 0);  // red: see prolong_list_kernel
      bottom_smooth<KIND>(V[i], a.n_post);
    }
    if (i < 0) break;
    ++i;  // visit level i+1 again, from its current correction
  }
  if (SMEM) {
    for (int i = a.first_smem; i < a.nlev; ++i) {
      const long long tot = a.L[i].g.total;
      for (int c = 0; c < 2; ++c)
        for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
          a.L[i].phi[c][e] = V[i].phi[c][e];
          a.L[i].rhs[c][e] = V[i].rhs[c][e];
        }
    }
  }
}

}  // namespace
}  // namespace gbmg
