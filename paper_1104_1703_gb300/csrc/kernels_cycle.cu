// V-cycle kernels of the masked-domain multigrid solver (Guillet & Teyssier,
// arXiv:1104.1703, Section 2 recipe): red-black Gauss-Seidel half-sweeps,
// residual + R1 restriction, P2 prolongation + correction, residual norm,
// and the two FP64 kernels of the mixed-precision refinement step.
//
// All fields are in the red/black split layout described in mg_internal.h.
// Every level stores b = h_l^2 f_l (f_l its right-hand side) and every
// operator is written in that scaled form:
//   scaled residual   r^ = sum_nbr Phi_j - D Phi_i - b      (= h_l^2 r)
//   GS update         Phi_i = (sum_nbr Phi_j - b) / D
// where the neighbour sum runs over all six neighbours (inactive and
// out-of-box cells hold 0) and D is the diagonal of the modified Laplacian:
//   level 0:                 D = 6 + (number of ghost faces)   [theta = 1/2]
//   level >= 1, 2nd order:   D = sum of 1 or 1/theta per face   [Section 3]
//   level >= 1, 1st order:   D = 6 (neighbours with m < 1 hold 0, Section 4)
// The level-0 Dirichlet terms are folded into b once, outside the cycle.
// The coarse right-hand side is b_{l+1} = h_{l+1}^2 (-R1(r_l)) = -1/2 sum of
// the 8 children's r^ (h_{l+1} = 2 h_l, R1 = mean of 8).
//
// Every cycle kernel is a template on the value type T: double for the plain
// FP64 method, float for the inner V-cycle of the mixed-precision form.
//
// On GB300 the FP64 kernels are bound by the FP64 pipe (2 FP64 lane-ops per
// clock per SM), not by HBM, and a warp instruction costs that pipe the same
// whether or not its lanes are predicated off.  So the kernels run over
// compact lists of the unknowns (built once per mask), where every lane holds
// an unknown, and issue as few FP64 instructions as the operator allows.
// Neighbour values come through L1/L2.
#include "cycle_device.cuh"

namespace gbmg {

namespace {

template <typename T>
struct ListArgs {
  Geom g;
  T* self;          // values of the listed colour
  const T* other;   // values of the other colour
  const T* rhs;
  const T* invd;
  const T* diag;
  const uint8_t* code;
  const uint32_t* list;
  const uint32_t* count;
  const T* rhsd;  // level 0 of the FP64 method: b / D (SCALED sweeps)
  double* partials;
  double* phi64;  // level 0 of the mixed form: Phi of the listed colour (fused update)
};

// entries per thread of the list kernels: the FP64 kernels are bound by the
// FP64 pipe, the FP32 ones by load latency, which more entries in flight hide
template <typename T>
struct PerThread {
  static constexpr int value = 2;
};


// K4: one colour of a red-black Gauss-Seidel sweep (Section 2) over the
// compact list of that colour's unknowns: every lane of every warp updates
// an unknown, so no issue slot is spent on a predicated-off lane.  Each
// thread takes PER entries (i, i + stride, ...) and issues every load of
// all of them before any store (the compiler cannot prove that the written
// and the read colour arrays do not alias).  With UPDATE (the last sweep of
// the fine level in a mixed-precision step) the colour's correction e is
// final once written, so Phi += e is applied in FP64 in the same pass.
// With SCALED (level 0 of the FP64 method) the right-hand side comes
// pre-multiplied by 1/D, b/D, so the update (sum - b) / D is one fused
// multiply-add, sum * (1/D) - b/D: 6 FP64 instructions instead of 7 on
// the FP64-pipe-bound sweep.  With EXACT as well the neighbour sum is
// formed in integer arithmetic (nbr_sum_exact), which leaves the fused
// multiply-add as the update's only FP64 instruction.
template <int KIND, typename T, bool UPDATE, bool SCALED = false, bool EXACT = false>
__global__ void __launch_bounds__(kListBlock) gs_list_kernel(ListArgs<T> a) {
  constexpr int PER = PerThread<T>::value;
  __shared__ T tab[16];
  if (KIND == 0) init_tab(tab);
  const uint32_t n = *a.count;
  const uint32_t stride = gridDim.x * kListBlock;
  const uint32_t P = (uint32_t)a.g.P, Z = (uint32_t)a.g.sz;
  uint32_t base = blockIdx.x * kListBlock + threadIdx.x;
  // A round's list entries and diagonals are built with the mask and do
  // not change during a solve: the first round's are loaded before the wait
  // on the previous kernel (their round trip overlaps its end), the next
  // round's while the current one computes.
  uint32_t e[PER];
  T d[PER];
  auto invariants = [&](uint32_t b0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t i = b0 + u * stride;
      e[u] = i < n ? a.list[i] : 0u;
      d[u] = i < n ? inv_diag<KIND>(KIND == 0 ? a.code[e[u] & kListAt] : 0, a.invd, e[u] & kListAt, tab) : T(0);
    }
  };
  invariants(base);
  pdl_wait();
  for (; base < n; base += PER * stride) {
    uint32_t at[PER];
    T s[PER], b[PER], dd[PER];
    bool ok[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      ok[u] = base + u * stride < n;
      at[u] = e[u] & kListAt;
      ok[u] = ok[u] && entry_ok(a.g, at[u], 3);
      dd[u] = d[u];
      if (ok[u]) {
        s[u] = nbr_sum_sel32<EXACT>(a.other, at[u], x_nbr(e[u], at[u]), P, Z);
        b[u] = SCALED ? a.rhsd[at[u]] : a.rhs[at[u]];
      }
    }
    invariants(base + PER * stride);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (!ok[u]) continue;
      const T v = SCALED ? fma(s[u], dd[u], -b[u]) : (s[u] - b[u]) * dd[u];
      a.self[at[u]] = v;
      if (UPDATE) a.phi64[at[u]] += widen_f32(v);
    }
  }
}

// K4 on level 0 of the mixed form's FP32 cycles, over row segments
// (list[0] of level 0): a group of 2^SHIFT lanes takes one segment, lane l
// its slot q0 + l, so that every array is read in runs of consecutive
// slots; PER segments per group are in flight at once.  A lane on an
// inactive or padding slot (code 0) writes 0, the value such a slot always
// holds, so the group writes whole runs.  The grid is persistent (a few
// blocks per SM) and each group loads the segment entries of its next round
// before it works on the current one, which takes the entry load off the
// chain of dependent loads.  The arithmetic per active cell is
// gs_list_kernel's.  (The FP64 sweeps keep the cell lists: their integer
// neighbour sum makes them instruction-bound, and a segment's idle lanes
// would add to that.)
template <typename T, bool UPDATE, int SHIFT>
__global__ void __launch_bounds__(kListBlock) gs_seg_kernel(ListArgs<T> a) {
  constexpr int PER = 2;
  constexpr int GROUPS = 32 >> SHIFT;  // segments per warp and round
  __shared__ T tab[16];
  init_tab(tab);
  const uint32_t n = *a.count;
  const int lane = threadIdx.x & 31;
  const int l = lane & ((1 << SHIFT) - 1);
  const uint32_t group = ((blockIdx.x * kListBlock + threadIdx.x) >> 5) * GROUPS + (lane >> SHIFT);
  const uint32_t ngroups = (gridDim.x * kListBlock >> 5) * GROUPS;
  const uint32_t step = PER * ngroups;
  const uint32_t P = (uint32_t)a.g.P, Z = (uint32_t)a.g.sz;
  uint32_t next[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const uint32_t i = group + u * ngroups;
    next[u] = i < n ? a.list[i] : 0u;
  }
  // the segment entries are constant during a solve: the first ones are
  // loaded before the wait on the previous kernel
  pdl_wait();
  for (uint32_t base = group; base < n; base += step) {
    uint32_t cur[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      cur[u] = next[u];
      const uint32_t i = base + step + u * ngroups;
      next[u] = i < n ? a.list[i] : 0u;
    }
    uint32_t at[PER];
    T s[PER], b[PER], d[PER];
    bool ok[PER], act[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t e = cur[u];
      at[u] = e & kListAt;
      ok[u] = base + u * ngroups < n && entry_ok(a.g, at[u], 9);
      at[u] += (uint32_t)l;
      if (ok[u]) {
        const uint8_t code = a.code[at[u]];
        act[u] = (code & kActive2) != 0;
        s[u] = nbr_sum32(a.other, at[u], x_nbr(e, at[u]), P, Z);
        b[u] = a.rhs[at[u]];
        d[u] = tab[__popc((unsigned)code >> kGhostShift)];
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (!ok[u]) continue;
      const T v = (s[u] - b[u]) * d[u];
      a.self[at[u]] = act[u] ? v : T(0);
      if (UPDATE && act[u]) a.phi64[at[u]] += widen_f32(v);
    }
  }
}

// The same sweep over 16-slot row segments with two consecutive slots per
// lane (8-byte loads and stores): lane l of a group of 8 takes slots
// q0 + 2l and q0 + 2l + 1.  The x-neighbour that is not in the lane's own
// pair is the adjacent lane's (a shuffle within the group) or, for the
// group's first or last lane, one extra load.  Per cell the sum and the
// update are gs_list_kernel's, in the same order, so the results are
// bit-identical.  Groups of a warp run their rounds together (the shuffles
// need every lane); a group without a segment works on slot (0, 0, 0) of the
// level, whose stencil lies inside the arrays, and stores nothing.
template <bool UPDATE>
__global__ void __launch_bounds__(kListBlock) gs_seg_pair_kernel(ListArgs<float> a) {
  constexpr int PER = 1;  // two slots per lane already
  constexpr int GROUPS = 4;  // segments per warp and round
  __shared__ float tab[16];
  init_tab(tab);
  const uint32_t n = *a.count;
  const int lane = threadIdx.x & 31;
  const int l = lane & 7;
  const uint32_t warp_group = ((blockIdx.x * kListBlock + threadIdx.x) >> 5) * GROUPS;
  const uint32_t mine = (uint32_t)(lane >> 3);
  const uint32_t ngroups = (gridDim.x * kListBlock >> 5) * GROUPS;
  const uint32_t step = PER * ngroups;
  const uint32_t P = (uint32_t)a.g.P, Z = (uint32_t)a.g.sz, safe = (uint32_t)a.g.off0;
  uint32_t next[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const uint32_t i = warp_group + mine + u * ngroups;
    next[u] = i < n ? a.list[i] : 0u;
  }
  pdl_wait();
  for (uint32_t wb = warp_group; wb < n; wb += step) {
    uint32_t cur[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      cur[u] = next[u];
      const uint32_t i = wb + step + mine + u * ngroups;
      next[u] = i < n ? a.list[i] : 0u;
    }
    uint32_t at[PER];
    bool ok[PER], plus[PER];
    float2 oh[PER], ym[PER], yp[PER], zm[PER], zp[PER], bb[PER];
    float edge[PER];
    uint16_t cd[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t e = cur[u];
      ok[u] = wb + mine + u * ngroups < n && entry_ok(a.g, e & kListAt, 9);
      plus[u] = ok[u] && (e & kListPlusX) != 0;
      at[u] = (ok[u] ? (e & kListAt) : safe) + 2u * (uint32_t)l;
      oh[u] = *reinterpret_cast<const float2*>(a.other + at[u]);
      ym[u] = *reinterpret_cast<const float2*>(a.other + (at[u] - P));
      yp[u] = *reinterpret_cast<const float2*>(a.other + (at[u] + P));
      zm[u] = *reinterpret_cast<const float2*>(a.other + (at[u] - Z));
      zp[u] = *reinterpret_cast<const float2*>(a.other + (at[u] + Z));
      bb[u] = *reinterpret_cast<const float2*>(a.rhs + at[u]);
      cd[u] = *reinterpret_cast<const uint16_t*>(a.code + at[u]);
      edge[u] = 0.f;
      if (plus[u] ? l == 7 : l == 0) edge[u] = a.other[plus[u] ? at[u] + 2u : at[u] - 1u];
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const float up = __shfl_up_sync(0xffffffffu, oh[u].y, 1, 8);    // o[at - 1]
      const float dn = __shfl_down_sync(0xffffffffu, oh[u].x, 1, 8);  // o[at + 2]
      // x-neighbours of the pair's two cells: dx = +1 (plus) or -1
      const float x0 = plus[u] ? oh[u].y : (l == 0 ? edge[u] : up);
      const float x1 = plus[u] ? (l == 7 ? edge[u] : dn) : oh[u].x;
      const float s0 = ((oh[u].x + x0) + (ym[u].x + yp[u].x)) + (zm[u].x + zp[u].x);
      const float s1 = ((oh[u].y + x1) + (ym[u].y + yp[u].y)) + (zm[u].y + zp[u].y);
      const unsigned c0 = cd[u] & 0xffu, c1 = cd[u] >> 8;
      const bool a0 = (c0 & kActive2) != 0, a1 = (c1 & kActive2) != 0;
      const float v0 = (s0 - bb[u].x) * tab[__popc(c0 >> kGhostShift)];
      const float v1 = (s1 - bb[u].y) * tab[__popc(c1 >> kGhostShift)];
      if (!ok[u]) continue;
      *reinterpret_cast<float2*>(a.self + at[u]) = make_float2(a0 ? v0 : 0.f, a1 ? v1 : 0.f);
      if (UPDATE && (a0 || a1)) {
        double2 ph = *reinterpret_cast<const double2*>(a.phi64 + at[u]);
        if (a0) ph.x += widen_f32(v0);
        if (a1) ph.y += widen_f32(v1);
        *reinterpret_cast<double2*>(a.phi64 + at[u]) = ph;
      }
    }
  }
}

// K9, first pass: the sum of r^2 per block into partials[blockIdx.x], r^ =
// sum_nbr Phi_j - D Phi_i - b the scaled residual of the listed unknowns
// (the grid is fixed per level, so the partials do not depend on scheduling).
template <int KIND, typename T, bool EXACT = false>
__global__ void __launch_bounds__(kListBlock) res_list_kernel(ListArgs<T> a) {
  constexpr int PER = PerThread<T>::value;
  __shared__ T tab[16];
  if (KIND == 0) init_tab(tab);
  const Geom g = a.g;
  const uint32_t n = *a.count;
  const uint32_t stride = gridDim.x * kListBlock;
  uint32_t base = blockIdx.x * kListBlock + threadIdx.x;
  // list entries and diagonals are fixed by the mask: loaded before the wait
  // on the previous kernel (first round) and during the current round (next)
  uint32_t e[PER];
  T d[PER];
  auto invariants = [&](uint32_t b0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t i = b0 + u * stride;
      e[u] = i < n ? a.list[i] : 0u;
      d[u] = i < n ? diag_of<KIND>(KIND == 0 ? a.code[e[u] & kListAt] : 0, a.diag, e[u] & kListAt, tab) : T(0);
    }
  };
  invariants(base);
  pdl_wait();
  double acc = 0.0;
  for (; base < n; base += PER * stride) {
    long long at[PER];
    T r[PER];
    bool ok[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      ok[u] = base + u * stride < n;
      at[u] = e[u] & kListAt;
      ok[u] = ok[u] && entry_ok(g, at[u], 4);
      if (ok[u]) {
        const T s = nbr_sum_sel<EXACT>(a.other, at[u], (e[u] & kListPlusX) ? 1 : -1, g.P, g.sz);
        r[u] = fma(-d[u], a.self[at[u]], s) - a.rhs[at[u]];
      }
    }
    invariants(base + PER * stride);
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (ok[u]) acc = fma((double)r[u], (double)r[u], acc);
  }
  block_reduce_store(acc, a.partials + blockIdx.x);
}

template <typename T>
struct SmallArgs {
  Geom g;
  T* phi0;
  T* phi1;
  const T* rhs0;
  const T* rhs1;
  const T* invd0;
  const T* invd1;
  const uint8_t* code0;
  const uint8_t* code1;
  uint8_t bit;
  int sweeps;
};

constexpr int kSmallThreads = 512;
constexpr int kSmallSmemBytes = 96 * 1024;

// Several full sweeps of a small level inside one CTA (no launch per
// half-sweep); __syncthreads separates the colours.  With SMEM the two
// colour arrays (halo included) are staged in shared memory for the whole
// call, so every neighbour read is an on-chip load.
template <int KIND, bool SMEM, typename T>
__global__ void __launch_bounds__(kSmallThreads) smooth_small_kernel(SmallArgs<T> a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T tab[16];
  if (KIND == 0) init_tab(tab);
  const Geom g = a.g;
  T* p0 = a.phi0;
  T* p1 = a.phi1;
  if (SMEM) {
    T* sm = reinterpret_cast<T*>(smem_raw);
    p0 = sm;
    p1 = sm + g.total;
    for (long long e = threadIdx.x; e < g.total; e += blockDim.x) {
      p0[e] = a.phi0[e];
      p1[e] = a.phi1[e];
    }
    __syncthreads();
  }
  const int n = g.hx * g.ny * g.nz;
  for (int s = 0; s < a.sweeps; ++s) {
    for (int c = 0; c < 2; ++c) {
      T* self = c ? p1 : p0;
      const T* o = c ? p0 : p1;
      const T* rhs = c ? a.rhs1 : a.rhs0;
      const T* invd = c ? a.invd1 : a.invd0;
      const uint8_t* code = c ? a.code1 : a.code0;
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int q = e % g.hx, t = e / g.hx, j = t % g.ny, k = t / g.ny;
        const long long at = g.at(q, j, k);
        const uint8_t cd = code[at];
        if (!(cd & a.bit)) continue;
        self[at] = (nbr_sum(o, at, x_offset(c, j, k), g.P, g.sz) - rhs[at]) * inv_diag<KIND>(cd, invd, at, tab);
      }
      __syncthreads();
    }
  }
  if (SMEM) {
    for (long long e = threadIdx.x; e < g.total; e += blockDim.x) {
      a.phi0[e] = p0[e];
      a.phi1[e] = p1[e];
    }
  }
}

template <typename T>
struct RestrictArgs {
  Geom gf, gc;
  const T* phi[2];   // fine level
  const T* rhs[2];
  const T* diag[2];  // fine level >= 1, second order
  const uint8_t* code[2];
  uint8_t bit;
  T* crhs[2];
  T* cphi[2];
  const uint32_t* clist[2];   // restrict_list_kernel: second-order unknowns of the coarse level
  const uint32_t* ccount[2];
};

// What the mask fixes about the children of coarse cell (I, J, K): their
// offsets, codes and diagonals (loaded before the wait on the previous
// kernel; rows and planes past the fine level's end are its zero halo,
// whose codes are 0).
template <typename T>
struct Children {
  long long at[2][2];
  uint8_t code[2][2][2];
  T diag[2][2][2];
};

template <int KIND, bool BLACK_ZERO, typename T>
__device__ __forceinline__ void child_invariants(const RestrictArgs<T>& a, int I, int J, int K, const T* tab,
                                                 Children<T>& ch) {
  const Geom& gf = a.gf;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      const int j = 2 * J + dj, k = 2 * K + dk;
      const bool in = j < gf.ny && k < gf.nz;
      ch.at[dk][dj] = gf.at(I, j, k);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const bool use = in && (c == 0 || !BLACK_ZERO);
        const uint8_t cd = use ? a.code[c][ch.at[dk][dj]] : 0;
        ch.code[dk][dj][c] = (cd & a.bit) ? cd : 0;
        ch.diag[dk][dj][c] = use ? diag_of<KIND>(cd, a.diag[c], ch.at[dk][dj], tab) : T(0);
      }
    }
}

// Children residuals of coarse cell (I, J, K): the scaled residuals r^ of
// its active children, summed in the order (dk, dj, colour).
template <int KIND, bool BLACK_ZERO, typename T, bool EXACT = false>
__device__ __forceinline__ T child_residual_sum(const RestrictArgs<T>& a, const Children<T>& ch, int J, int K) {
  const Geom& gf = a.gf;
  T sum = 0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int c = 0; c < (BLACK_ZERO ? 1 : 2); ++c) {
        if (!ch.code[dk][dj][c]) continue;
        const long long at = ch.at[dk][dj];
        const T s = nbr_sum_sel<EXACT>(a.phi[c ^ 1], at, x_offset(c, 2 * J + dj, 2 * K + dk), gf.P, gf.sz);
        sum += fma(-ch.diag[dk][dj][c], a.phi[c][at], s) - a.rhs[c][at];
      }
  return sum;
}

// K5: residual and R1 in one pass (Section 2, recipe steps 2-5; Fig. 3).
// Thread (I, J) of coarse plane K evaluates the scaled residual
// r^ = sum_nbr Phi_j - D Phi_i - b of each of its active children and
// writes b_c = -1/2 sum r^ and dPhi_c = 0.  The two x-children of coarse
// cell I are both at fine slot I of the child rows (one per colour), so a
// warp reads consecutive slots of every array it touches.  With BLACK_ZERO
// the last fine operation was a complete red-black sweep, after which every
// black cell satisfies its own equation: only red children carry a
// residual.  Children outside the active set (of this order) count 0.
template <int KIND, bool BLACK_ZERO, typename T>
__global__ void __launch_bounds__(kBlockX * kBlockY) restrict_kernel(RestrictArgs<T> a) {
  __shared__ T tab[16];
  if (KIND == 0) init_tab(tab);
  const Geom gc = a.gc;
  const int I = blockIdx.x * kBlockX + threadIdx.x;
  const int J = blockIdx.y * kBlockY + threadIdx.y;
  const int K = blockIdx.z;
  const bool in = I < gc.nx && J < gc.ny;
  Children<T> ch;
  if (in) child_invariants<KIND, BLACK_ZERO>(a, I, J, K, tab, ch);  // fixed by the mask: before the wait
  pdl_wait();
  if (!in) return;
  const T sum = child_residual_sum<KIND, BLACK_ZERO>(a, ch, J, K);
  const int C = (I + J + K) & 1;
  const long long atc = gc.at(I >> 1, J, K);
  a.crhs[C][atc] = T(-0.5) * sum;
  a.cphi[C][atc] = T(0);
}

// K5 from level 0 in the V-cycle: the same residual + R1, over the
// second-order unknowns of the coarse level only (a superset of the first-order ones, so a switch
// of order leaves no stale correction).  Coarse cells outside that set are
// never written in a cycle: their correction stays the 0 it was reset to,
// and their right-hand side is never read.  Every lane holds a coarse
// unknown, which spares the FP64 pipe the idle lanes of a box-wide grid.
template <int KIND, bool BLACK_ZERO, typename T, bool EXACT = false>
__global__ void __launch_bounds__(kListBlock) restrict_list_kernel(RestrictArgs<T> a) {
  constexpr int PER = 2;
  __shared__ T tab[16];
  if (KIND == 0) init_tab(tab);
  const Geom gc = a.gc;
  const uint32_t n0 = *a.ccount[0], n = n0 + *a.ccount[1];
  const uint32_t stride = gridDim.x * kListBlock;
  uint32_t base = blockIdx.x * kListBlock + threadIdx.x;
  long long atc[PER];
  int cc[PER], JJ[PER], KK[PER];
  bool ok[PER];
  Children<T> ch[PER];
  // the coarse unknowns and their children's codes and diagonals are fixed
  // by the mask: the first round's are loaded before the wait on the
  // previous kernel, the next round's while the current one computes
  auto invariants = [&](uint32_t b0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t i = b0 + u * stride;
      ok[u] = i < n;
      if (!ok[u]) continue;
      const int C = i >= n0;
      cc[u] = C;
      atc[u] = (C ? a.clist[1][i - n0] : a.clist[0][i]) & kListAt;
      ok[u] = entry_ok(gc, atc[u], 5);
      if (!ok[u]) continue;
      int Q;
      gc.slot_of(atc[u], &Q, &JJ[u], &KK[u]);
      child_invariants<KIND, BLACK_ZERO>(a, 2 * Q + ((C ^ JJ[u] ^ KK[u]) & 1), JJ[u], KK[u], tab, ch[u]);
    }
  };
  invariants(base);
  pdl_wait();
  for (; base < n; base += PER * stride) {
    T sum[PER];
    long long at2[PER];
    int c2[PER];
    bool ok2[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      ok2[u] = ok[u];
      at2[u] = atc[u];
      c2[u] = cc[u];
      if (ok[u]) sum[u] = child_residual_sum<KIND, BLACK_ZERO, T, EXACT>(a, ch[u], JJ[u], KK[u]);
    }
    invariants(base + PER * stride);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (!ok2[u]) continue;
      a.crhs[c2[u]][at2[u]] = T(-0.5) * sum[u];
      a.cphi[c2[u]][at2[u]] = T(0);
    }
  }
}

template <typename T>
struct ProlongArgs {
  Geom gf, gc;
  T* phi[2];
  const uint32_t* list[2];
  const uint32_t* count[2];
  const T* cphi[2];
  int skip_red;  // prolong the black unknowns only
};


// K6: Phi_f += P2(dPhi_c) on the unknowns of the fine level (Section 2,
// recipe steps 6-7; Fig. 3).  Per axis a fine cell lies 1/4 of a coarse cell
// from its parent ("near") and 3/4 from the coarse neighbour on its side
// ("far"); P2 weighs them 3/4 and 1/4, so the 8 corner weights are 27, 9, 3
// and 1 (/64) for 0, 1, 2 and 3 far axes.  Grouping the corners by weight
// costs 9 arithmetic instructions per fine cell.  Coarse cells outside
// Omega_c hold 0 and out-of-box coarse indices read the zero halo.
// With skip_red only the black unknowns are corrected: when post-smoothing
// follows, its first (red) half-sweep overwrites every red unknown from its
// black neighbours without reading the red value, so correcting the red
// unknowns first would not change the result.
template <typename T>
__global__ void __launch_bounds__(kListBlock) prolong_list_kernel(ProlongArgs<T> a) {
  constexpr int PER = 2;
  const Geom gf = a.gf;
  const uint32_t n0 = a.skip_red ? 0u : *a.count[0], n = n0 + *a.count[1];
  const uint32_t stride = gridDim.x * kListBlock;
  uint32_t base = blockIdx.x * kListBlock + threadIdx.x;
  // the list entries are constant during a solve: the first round's are
  // loaded before the wait on the previous kernel, the next round's while
  // the current one computes
  uint32_t e[PER];
  auto entries = [&](uint32_t b0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t i = b0 + u * stride;
      e[u] = i < n ? (i >= n0 ? a.list[1][i - n0] : a.list[0][i]) : 0u;
    }
  };
  entries(base);
  pdl_wait();
  for (; base < n; base += PER * stride) {
    uint32_t at[PER];
    int cc[PER];
    T w[PER], old[PER];
    bool ok[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      // every entry's loads are issued; a missing entry reads around slot
      // (0, 0, 0), whose coarse corners lie inside the arrays
      const uint32_t i = base + u * stride;
      const int c = i >= n0;
      cc[u] = c;
      at[u] = e[u] & kListAt;
      ok[u] = i < n && entry_ok(gf, at[u], 6);
      if (!ok[u]) at[u] = (uint32_t)gf.off0;
      int q, j, k;
      gf.slot_of(at[u], &q, &j, &k);
      w[u] = p2_sum(a.gc, a.cphi[0], a.cphi[1], q, j, k, c, PlainLoad());
      old[u] = a.phi[c][at[u]];
    }
    entries(base + PER * stride);
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (ok[u]) a.phi[cc[u]][at[u]] = fma(w[u], T(1) / T(64), old[u]);
  }
}

// The one-CTA bottom V-cycle (bottom_run) as a kernel of its own.
template <int KIND, typename T, bool SMEM>
__global__ void __launch_bounds__(kBottomThreads, 1) bottom_kernel(BottomArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bottom_run<KIND, T, SMEM>(a, smem_raw, true);
}

struct NormArgs {
  Geom g;
  const double* rhs[2];
  const uint8_t* code[2];
  uint8_t bit;
  double* partials;
};

// sum of b^2 over the active cells (the residual of Phi = 0 is -b).  A
// thread takes 16-slot chunks of the colours' rows (rows are padded to a
// multiple of 16 slots): one 16-byte load of the codes, then the right-hand
// side of the chunk's active slots in pairs, summed in slot order.
__global__ void __launch_bounds__(kNormThreads) rhsnorm_kernel(NormArgs a) {
  pdl_wait();
  const Geom g = a.g;
  const unsigned per_row = (unsigned)(g.hx + 15) >> 4;
  const unsigned nch = per_row * (unsigned)g.ny * (unsigned)g.nz;  // chunks per colour
  const int p = a.bit == 1 ? 0 : (a.bit == 2 ? 1 : 31 - __clz((int)a.bit));
  double acc = 0.0;
  for (unsigned x = blockIdx.x * blockDim.x + threadIdx.x; x < 2 * nch; x += gridDim.x * blockDim.x) {
    const int c = x >= nch;
    const unsigned y = x - (c ? nch : 0u);
    const unsigned row = y / per_row;
    const int q0 = (int)(y - row * per_row) << 4;
    const int k = (int)(row / (unsigned)g.ny);
    const int j = (int)(row - (unsigned)k * (unsigned)g.ny);
    const long long at0 = g.at(q0, j, k);
    const uint4 w = *reinterpret_cast<const uint4*>((c ? a.code[1] : a.code[0]) + at0);
    const unsigned word[4] = {w.x, w.y, w.z, w.w};
    unsigned bits = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const unsigned v = (word[i] >> p) & 0x01010101u;
      bits |= ((v & 1u) | ((v >> 7) & 2u) | ((v >> 14) & 4u) | ((v >> 21) & 8u)) << (4 * i);
    }
    const int nv = g.hx - q0;
    if (nv < 16) bits &= (1u << nv) - 1u;
    if (!bits) continue;
    const double2* r2 = reinterpret_cast<const double2*>((c ? a.rhs[1] : a.rhs[0]) + at0);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const unsigned pb = (bits >> (2 * h)) & 3u;
      if (pb) {
        const double2 v = r2[h];
        if (pb & 1u) acc = fma(v.x, v.x, acc);
        if (pb & 2u) acc = fma(v.y, v.y, acc);
      }
    }
  }
  block_reduce_store(acc, a.partials + blockIdx.x);
}

// K9 (second pass): one CTA sums the partials in a fixed order (four
// independent accumulators per thread so that the loads overlap).
constexpr int kFinalThreads = 1024;

__global__ void __launch_bounds__(kFinalThreads) finalize_kernel(const double* __restrict__ partials, int n,
                                                                 double* out) {
  pdl_wait();
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int e = threadIdx.x;
  for (; e + 3 * kFinalThreads < n; e += 4 * kFinalThreads) {
    a0 += partials[e];
    a1 += partials[e + kFinalThreads];
    a2 += partials[e + 2 * kFinalThreads];
    a3 += partials[e + 3 * kFinalThreads];
  }
  for (; e < n; e += kFinalThreads) a0 += partials[e];
  block_reduce_store((a0 + a1) + (a2 + a3), out);
}

// Mixed precision, start of a refinement step: the FP64 scaled residual of
// the fine level, r^ = A Phi - b over both colour lists (every unknown: after
// an FP32 correction the black residual no longer vanishes).  The error
// equation A e = -r^ becomes the FP32 problem: its right-hand side (-r^ in
// float) and its initial correction (0) are written in the same pass, and
// r^2 is summed per block for the FP64 norm.
struct RefineArgs {
  Geom g;
  const double* phi[2];
  const double* rhs[2];
  const uint8_t* code[2];
  const uint32_t* list[2];
  const uint32_t* count[2];
  float* rhs32[2];
  float* e32[2];
  double* partials;
};

template <bool EXACT>
__global__ void __launch_bounds__(kListBlock) refine_residual_kernel(RefineArgs a) {
  constexpr int PER = 2;
  __shared__ double tab[16];
  init_tab(tab);
  const Geom g = a.g;
  const uint32_t n0 = *a.count[0], n = n0 + *a.count[1];
  const uint32_t stride = gridDim.x * kListBlock;
  uint32_t base = blockIdx.x * kListBlock + threadIdx.x;
  // list entries and diagonals are fixed by the mask: the first round's are
  // loaded before the wait on the previous kernel; each next round's
  // entries while the current one computes, its diagonals with its data
  uint32_t e[PER];
  double D[PER];
  auto entry = [&](uint32_t i) { return i < n ? (i >= n0 ? a.list[1][i - n0] : a.list[0][i]) : 0u; };
#pragma unroll
  for (int u = 0; u < PER; ++u) e[u] = entry(base + u * stride);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const uint32_t i = base + u * stride;
    D[u] = i < n ? tab[8 + __popc((unsigned)a.code[i >= n0][e[u] & kListAt] >> kGhostShift)] : 0.0;
  }
  pdl_wait();
  double acc = 0.0;
  for (bool first = true; base < n; base += PER * stride, first = false) {
    long long at[PER];
    int cc[PER];
    double r[PER];
    bool ok[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t i = base + u * stride;
      ok[u] = i < n;
      if (!ok[u]) continue;
      const int c = i >= n0;
      cc[u] = c;
      at[u] = e[u] & kListAt;
      ok[u] = entry_ok(g, at[u], 7);
      if (!ok[u]) continue;
      const double s = nbr_sum_sel<EXACT>(a.phi[1 - c], at[u], (e[u] & kListPlusX) ? 1 : -1, g.P, g.sz);
      const double Du = first ? D[u] : tab[8 + __popc((unsigned)a.code[c][at[u]] >> kGhostShift)];
      r[u] = fma(-Du, a.phi[c][at[u]], s) - a.rhs[c][at[u]];
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) e[u] = entry(base + PER * stride + u * stride);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (!ok[u]) continue;
      a.rhs32[cc[u]][at[u]] = narrow_f64(-r[u]);
      a.e32[cc[u]][at[u]] = 0.0f;
      acc = fma(r[u], r[u], acc);
    }
  }
  block_reduce_store(acc, a.partials + blockIdx.x);
}

// Mixed precision, end of a refinement step: Phi += e in FP64.
struct UpdateArgs {
  Geom g;
  double* phi[2];
  const float* e32[2];
  const uint32_t* list[2];
  const uint32_t* count[2];
};

__global__ void __launch_bounds__(kListBlock) refine_update_kernel(UpdateArgs a) {
  pdl_wait();
  const uint32_t n0 = *a.count[0], n = n0 + *a.count[1];
  for (uint32_t i = blockIdx.x * kListBlock + threadIdx.x; i < n; i += gridDim.x * kListBlock) {
    const int c = i >= n0;
    const long long at = (c ? a.list[1][i - n0] : a.list[0][i]) & kListAt;
    if (!entry_ok(a.g, at, 8)) continue;
    a.phi[c][at] += widen_f32(a.e32[c][at]);
  }
}


int kind_of(int level, int order) { return level == 0 ? 0 : (order == 1 ? 2 : 1); }
uint8_t bit_of(int level, int order) { return (level >= 1 && order == 1) ? kActive1 : kActive2; }

// fixed grid of the norm kernels of a level: enough blocks for every slot of
// one colour, at most 16 per SM (grid-stride beyond that)
int list_grid(const Geom& g) {
  const long long n = (long long)g.hx * g.ny * g.nz;
  long long b = (n + kListBlock - 1) / kListBlock;
  const long long cap = 16LL * device_sms();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// grid for n list entries: `per` entries per thread for long lists, one
// entry per thread for short ones (so that short lists still spread over
// all SMs); the kernels loop over their entries up to n either way
int exact_grid(uint32_t n, int per) {
  if ((long long)n < 4LL * device_sms() * kListBlock * per) per = 1;
  const long long b = ((long long)n + (long long)kListBlock * per - 1) / ((long long)kListBlock * per);
  return b < 1 ? 1 : (int)b;
}

// grid for n row segments of 2^shift slots (one lane per slot), at most
// the blocks that stay resident together (8 per SM at 256 threads), which
// then loop
int seg_grid(uint32_t n, int shift) {
  const long long groups_per_block = (long long)kListBlock >> shift;
  long long b = ((long long)n + groups_per_block - 1) / groups_per_block;
  const long long cap = 8LL * device_sms();
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

template <typename T>
bool small_smem(const Geom& g) {
  return 2 * g.total * (long long)sizeof(T) <= kSmallSmemBytes;
}

// level 0 has a single active set, stored under order 2
int list_order(const LevelDev& L, int order) { return L.level == 0 ? 2 : order; }

template <typename T>
struct Fields {
  T* const* phi;
  T* const* rhs;
  T* const* invd;
  T* const* diag;
};

Fields<double> fields(const LevelDev& L, double) { return {L.phi, L.rhs, L.invd, L.diag}; }
Fields<float> fields(const LevelDev& L, float) { return {L.phi32, L.rhs32, L.invd32, L.diag32}; }

template <typename T>
ListArgs<T> list_args(const LevelDev& L, int order, int colour) {
  const Fields<T> f = fields(L, T());
  ListArgs<T> a;
  a.g = L.g;
  a.self = f.phi[colour];
  a.other = f.phi[colour ^ 1];
  a.rhs = f.rhs[colour];
  a.invd = L.level ? f.invd[colour] : nullptr;
  a.diag = L.level ? f.diag[colour] : nullptr;
  a.code = L.code[colour];
  a.list = L.list[list_order(L, order)][colour];
  a.count = L.count + list_order(L, order) * 2 + colour;
  a.rhsd = nullptr;
  a.partials = nullptr;
  a.phi64 = nullptr;
  return a;
}

// level 0 of the FP32 cycles by row segments (gs_seg_kernel), when the
// hierarchy keeps them
template <int SHIFT>
cudaError_t half_sweep_seg(const LevelDev& L, int colour, bool update, cudaStream_t s) {
  ListArgs<float> a = list_args<float>(L, 2, colour);
  a.phi64 = L.phi[colour];
  a.list = L.list[0][colour];
  a.count = L.count + colour;
  if (SHIFT == 4 && L.seg_pairs) {  // 8 lanes per 16-slot segment: the grid of 8-slot segments
    const int grid = seg_grid(L.hcount[colour], 3);
    count_launch();
    if (update) launch_pdl(gs_seg_pair_kernel<true>, dim3(grid), dim3(kListBlock), 0, s, a);
    else launch_pdl(gs_seg_pair_kernel<false>, dim3(grid), dim3(kListBlock), 0, s, a);
    return cudaGetLastError();
  }
  const int grid = seg_grid(L.hcount[colour], SHIFT);
  count_launch();
  if (update)
    launch_pdl(gs_seg_kernel<float, true, SHIFT>, dim3(grid), dim3(kListBlock), 0, s, a);
  else
    launch_pdl(gs_seg_kernel<float, false, SHIFT>, dim3(grid), dim3(kListBlock), 0, s, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t half_sweep_t(const LevelDev& L, int order, int colour, bool update, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (L.level == 0 && L.seg_shift == 3) return half_sweep_seg<3>(L, colour, update, s);
    if (L.level == 0 && L.seg_shift == 4) return half_sweep_seg<4>(L, colour, update, s);
  }
  ListArgs<T> a = list_args<T>(L, order, colour);
  a.phi64 = L.phi[colour];
  const int grid = exact_grid(L.hcount[list_order(L, order) * 2 + colour], PerThread<T>::value);
  count_launch();
  if (update) {
    if (L.level != 0 || sizeof(T) != 4) return cudaErrorInvalidValue;
    launch_pdl(gs_list_kernel<0, T, true>, dim3(grid), dim3(kListBlock), 0, s, a);
    return cudaGetLastError();
  }
  if (L.level == 0 && sizeof(T) == 8 && L.rhsd[0]) {
    a.rhsd = (const T*)L.rhsd[colour];
    if constexpr (sizeof(T) == 8) {
      if (L.exact_sum) {
        launch_pdl(gs_list_kernel<0, T, false, true, true>, dim3(grid), dim3(kListBlock), 0, s, a);
        return cudaGetLastError();
      }
    }
    launch_pdl(gs_list_kernel<0, T, false, true>, dim3(grid), dim3(kListBlock), 0, s, a);
    return cudaGetLastError();
  }
  switch (kind_of(L.level, order)) {
    case 0: launch_pdl(gs_list_kernel<0, T, false>, dim3(grid), dim3(kListBlock), 0, s, a); break;
    case 1: launch_pdl(gs_list_kernel<1, T, false>, dim3(grid), dim3(kListBlock), 0, s, a); break;
    default: launch_pdl(gs_list_kernel<2, T, false>, dim3(grid), dim3(kListBlock), 0, s, a); break;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t smooth_small_t(const LevelDev& L, int order, int sweeps, cudaStream_t s) {
  const Fields<T> f = fields(L, T());
  SmallArgs<T> a;
  a.g = L.g;
  a.phi0 = f.phi[0];
  a.phi1 = f.phi[1];
  a.rhs0 = f.rhs[0];
  a.rhs1 = f.rhs[1];
  a.invd0 = L.level ? f.invd[0] : nullptr;
  a.invd1 = L.level ? f.invd[1] : nullptr;
  a.code0 = L.code[0];
  a.code1 = L.code[1];
  a.bit = bit_of(L.level, order);
  a.sweeps = sweeps;
  const bool sm = small_smem<T>(L.g);
  const size_t bytes = sm ? 2 * L.g.total * sizeof(T) : 0;
  count_launch();
#define GBMG_SMALL(K)                                                         \
  if (sm) launch_pdl(smooth_small_kernel<K, true, T>, dim3(1), dim3(kSmallThreads), bytes, s, a); \
  else launch_pdl(smooth_small_kernel<K, false, T>, dim3(1), dim3(kSmallThreads), 0, s, a);
  switch (kind_of(L.level, order)) {
    case 0: GBMG_SMALL(0) break;
    case 1: GBMG_SMALL(1) break;
    default: GBMG_SMALL(2) break;
  }
#undef GBMG_SMALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t restrict_t(const LevelDev& Lf, const LevelDev& Lc, int order, bool black_zero, bool all_cells,
                       cudaStream_t s) {
  const Fields<T> ff = fields(Lf, T()), fc = fields(Lc, T());
  RestrictArgs<T> a;
  a.gf = Lf.g;
  a.gc = Lc.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = ff.phi[c];
    a.rhs[c] = ff.rhs[c];
    a.diag[c] = Lf.level ? ff.diag[c] : nullptr;
    a.code[c] = Lf.code[c];
    a.crhs[c] = fc.rhs[c];
    a.cphi[c] = fc.phi[c];
  }
  a.bit = bit_of(Lf.level, order);
  for (int c = 0; c < 2; ++c) {
    a.clist[c] = Lc.list[2][c];
    a.ccount[c] = Lc.count + 4 + c;
  }
  // over the coarse unknowns from level 0 (FP64: no idle lanes on the FP64
  // pipe; FP32: fewer threads); from a coarse level the box-wide grid, whose
  // extra warps hide more latency, is faster
  if (!all_cells && Lf.level == 0) {
    const int lgrid = exact_grid(Lc.hcount[4] + Lc.hcount[5], 2);
    count_launch();
    if (sizeof(T) == 8 && Lf.exact_sum) {  // level 0, FP64: the residuals with the integer neighbour sum
      if (black_zero) launch_pdl(restrict_list_kernel<0, true, T, true>, dim3(lgrid), dim3(kListBlock), 0, s, a);
      else launch_pdl(restrict_list_kernel<0, false, T, true>, dim3(lgrid), dim3(kListBlock), 0, s, a);
      return cudaGetLastError();
    }
#define GBMG_RESTRICT_LIST(K)                                                                            \
  if (black_zero) launch_pdl(restrict_list_kernel<K, true, T>, dim3(lgrid), dim3(kListBlock), 0, s, a); \
  else launch_pdl(restrict_list_kernel<K, false, T>, dim3(lgrid), dim3(kListBlock), 0, s, a);
    switch (kind_of(Lf.level, order)) {
      case 0: GBMG_RESTRICT_LIST(0) break;
      case 1: GBMG_RESTRICT_LIST(1) break;
      default: GBMG_RESTRICT_LIST(2) break;
    }
#undef GBMG_RESTRICT_LIST
    return cudaGetLastError();
  }
  const dim3 grid((Lc.g.nx + kBlockX - 1) / kBlockX, (Lc.g.ny + kBlockY - 1) / kBlockY, Lc.g.nz);
  const dim3 block(kBlockX, kBlockY);
  count_launch();
#define GBMG_RESTRICT(K)                                                  \
  if (black_zero) launch_pdl(restrict_kernel<K, true, T>, dim3(grid), dim3(block), 0, s, a); \
  else launch_pdl(restrict_kernel<K, false, T>, dim3(grid), dim3(block), 0, s, a);
  switch (kind_of(Lf.level, order)) {
    case 0: GBMG_RESTRICT(0) break;
    case 1: GBMG_RESTRICT(1) break;
    default: GBMG_RESTRICT(2) break;
  }
#undef GBMG_RESTRICT
  return cudaGetLastError();
}

template <typename T>
cudaError_t prolong_t(const LevelDev& Lc, const LevelDev& Lf, int order, bool black_only, cudaStream_t s) {
  const Fields<T> ff = fields(Lf, T()), fc = fields(Lc, T());
  ProlongArgs<T> a;
  a.gf = Lf.g;
  a.gc = Lc.g;
  const int lo = list_order(Lf, order);
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = ff.phi[c];
    a.list[c] = Lf.list[lo][c];
    a.count[c] = Lf.count + lo * 2 + c;
    a.cphi[c] = fc.phi[c];
  }
  a.skip_red = black_only ? 1 : 0;
  const uint32_t n = (black_only ? 0u : Lf.hcount[lo * 2]) + Lf.hcount[lo * 2 + 1];
  count_launch();
  launch_pdl(prolong_list_kernel<T>, dim3(exact_grid(n, 2)), dim3(kListBlock), 0, s, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Middle levels in one thread-block cluster
// ---------------------------------------------------------------------------
//
// The levels between the large ones (one launch per step, the whole GPU)
// and the small ones (the one-CTA bottom) have from a few thousand to about
// a hundred thousand unknowns per colour: too few to fill the GPU, so each
// launch costs more in latency than in work.  mid_kernel runs them, and the
// bottom after them, as one launch of one cluster of kMidCluster CTAs: the
// steps of the Section 2 recipe are loops over the level's lists strided
// over the cluster's threads, separated by hardware cluster barriers.  The
// data stay in global memory (L2-resident at these sizes); values written by
// another CTA of the cluster are read with ld.global.cg (L2, not the SM's
// L1) after a __threadfence and the barrier.

constexpr int kMidCluster = 8;
constexpr int kMidThreads = 1024;
constexpr int kMidMaxLevels = 4;
constexpr int kMidPer = 4;  // list entries in flight per thread

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

struct CgLoad {
  template <typename T>
  __device__ __forceinline__ T operator()(const T* p) const {
    return __ldcg(p);
  }
};

template <typename T>
__device__ __forceinline__ T nbr_sum_cg(const T* o, long long at, int dx, int P, long long sz) {
  return ((ldcg(o + at) + ldcg(o + at + dx)) + (ldcg(o + at - P) + ldcg(o + at + P))) +
         (ldcg(o + at - sz) + ldcg(o + at + sz));
}

__device__ __forceinline__ void cluster_barrier() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename T>
struct MidLevel {
  Geom g;
  T* phi[2];
  T* rhs[2];
  const T* invd[2];
  const T* diag[2];
  const uint8_t* code[2];
  const uint32_t* list[2];  // unknowns of this order, per colour
  const uint32_t* count;    // [colour], device memory
};

template <typename T>
struct MidArgs {
  MidLevel<T> L[kMidMaxLevels + 1];  // the middle levels m .. lb-1, then level lb
  int nmid;
  uint8_t bit;
  int n_pre, n_post;
  BottomArgs<T> bottom;  // levels lb .. deepest
};

// Gauss-Seidel sweeps of one middle level (as gs_list_kernel).
template <int KIND, typename T>
__device__ void mid_smooth(const MidLevel<T>& L, int sweeps, unsigned tid, unsigned nthr) {
  const int P = L.g.P;
  const long long sz = L.g.sz;
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      const uint32_t n = L.count[c];
      const uint32_t* list = L.list[c];
      for (uint32_t base = tid; base < n; base += kMidPer * nthr) {
        long long at[kMidPer];
        T v[kMidPer];
        bool ok[kMidPer];
#pragma unroll
        for (int u = 0; u < kMidPer; ++u) {
          const uint32_t i = base + u * nthr;
          ok[u] = i < n;
          const uint32_t e = ok[u] ? list[i] : 0u;
          at[u] = e & kListAt;
          ok[u] = ok[u] && entry_ok(L.g, at[u], 9);
          if (ok[u])
            v[u] = (nbr_sum_cg(L.phi[c ^ 1], at[u], (e & kListPlusX) ? 1 : -1, P, sz) - ldcg(L.rhs[c] + at[u])) *
                   inv_diag<KIND>(0, L.invd[c], at[u], (const T*)nullptr);
        }
#pragma unroll
        for (int u = 0; u < kMidPer; ++u)
          if (ok[u]) L.phi[c][at[u]] = v[u];
      }
      cluster_barrier();
    }
}

// Residual and R1 into the next level (as restrict_kernel), strided over
// the coarse cells.
template <int KIND, typename T>
__device__ void mid_restrict(const MidLevel<T>& F, const MidLevel<T>& C, uint8_t bit, bool black_zero,
                             unsigned tid, unsigned nthr) {
  const Geom& g = F.g;
  const Geom& gc = C.g;
  const unsigned nc = (unsigned)(gc.nx * gc.ny * gc.nz);
  for (unsigned e = tid; e < nc; e += nthr) {
    const int I = (int)(e % gc.nx), t = (int)(e / gc.nx), J = t % gc.ny, K = t / gc.ny;
    T sum = 0;
    for (int dk = 0; dk < 2; ++dk) {
      const int k = 2 * K + dk;
      if (k >= g.nz) break;
      for (int dj = 0; dj < 2; ++dj) {
        const int j = 2 * J + dj;
        if (j >= g.ny) break;
        const long long at = g.at(I, j, k);
        for (int c = 0; c < (black_zero ? 1 : 2); ++c) {
          if (!(F.code[c][at] & bit)) continue;
          const T nb = nbr_sum_cg(F.phi[c ^ 1], at, x_offset(c, j, k), g.P, g.sz);
          sum += fma(-diag_of<KIND>(0, F.diag[c], at, (const T*)nullptr), ldcg(F.phi[c] + at), nb) -
                 ldcg(F.rhs[c] + at);
        }
      }
    }
    const int Cc = (I + J + K) & 1;
    const long long atc = gc.at(I >> 1, J, K);
    C.rhs[Cc][atc] = T(-0.5) * sum;
    C.phi[Cc][atc] = T(0);
  }
  cluster_barrier();
}

// P2 of level C into the listed unknowns of level F (as prolong_list_kernel).
template <typename T>
__device__ void mid_prolong(const MidLevel<T>& F, const MidLevel<T>& C, int first_colour, unsigned tid,
                            unsigned nthr) {
  const Geom& gf = F.g;
  const Geom& gc = C.g;
  for (int c = first_colour; c < 2; ++c) {
    const uint32_t n = F.count[c];
    for (uint32_t i = tid; i < n; i += nthr) {
      const long long at = F.list[c][i] & kListAt;
      if (!entry_ok(gf, at, 10)) continue;
      int q, j, k;
      gf.slot_of(at, &q, &j, &k);
      const T w = p2_sum(gc, (const T*)C.phi[0], (const T*)C.phi[1], q, j, k, c, CgLoad());
      F.phi[c][at] = fma(w, T(1) / T(64), ldcg(F.phi[c] + at));
    }
  }
  cluster_barrier();
}

// The Section 2 recipe (V-cycle) from level m, whose right-hand side the
// restriction from level m-1 has set, down through the middle levels, the
// bottom (run by CTA 0 of the cluster, from shared memory when SMEM), and
// back up to level m.  Launched as a single cluster of kMidCluster CTAs.
template <int KIND, typename T, bool SMEM>
__global__ void __launch_bounds__(kMidThreads, 1) mid_kernel(MidArgs<T> a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const unsigned nthr = kMidCluster * blockDim.x;
  const unsigned tid = rank * blockDim.x + threadIdx.x;
  for (int i = 0; i < a.nmid; ++i) {
    mid_smooth<KIND>(a.L[i], a.n_pre, tid, nthr);                              // step 1
    mid_restrict<KIND>(a.L[i], a.L[i + 1], a.bit, a.n_pre >= 1, tid, nthr);  // steps 2-5
  }
  if (rank == 0) bottom_run<KIND, T, SMEM>(a.bottom, smem_raw);
  cluster_barrier();
  for (int i = a.nmid - 1; i >= 0; --i) {
    mid_prolong(a.L[i], a.L[i + 1], a.n_post >= 1 ? 1 : 0, tid, nthr);  // steps 6-7
    mid_smooth<KIND>(a.L[i], a.n_post, tid, nthr);                       // step 8
  }
}

// The coarsest solve's map for bottom_coarse_map: column j of M
// is the result (x_r, x_b) of `sweeps` red-black sweeps of the deepest level
// started from a unit input, b = e_j for j < n_r + n_b with a zero initial
// correction, or the initial black correction e_(j - n_r - n_b) with b = 0.
// One warp per column, kCmWarps columns per CTA.  Each CTA first indexes the
// level's unknowns: slot -> position in its colour's list, then per unknown
// the positions of its six neighbours of the other colour (-1 for a slot
// that is not an unknown: it holds 0).  The sweeps then run on the unknowns'
// values alone, in per-warp shared-memory vectors, with the operator's own
// arithmetic and summation order: (sum of the six neighbours - b) * (1/D).
constexpr int kCmWarps = 16;
constexpr long long kCmMaxSlots = 8192;  // slots per colour array of a level the map is built for

template <typename T>
struct CoarseMatArgs {
  Geom g;
  const uint32_t* list[2];
  const T* invd[2];
  uint32_t n[2];
  int sweeps;
  T* out;
};

template <typename T>
struct CoarseMatSmem {
  int8_t map[2][kCmMaxSlots];
  int8_t nbr[2][kCoarseMatMax][6];
  T id[2][kCoarseMatMax];
  T xs[kCmWarps][2][kCoarseMatMax];
};

template <int KIND, typename T>
__device__ void coarse_matrix_body(const CoarseMatArgs<T>& a, CoarseMatSmem<T>& sm) {
  auto& map = sm.map;
  auto& nbr = sm.nbr;
  auto& id = sm.id;
  auto& xs = sm.xs;
  const Geom& g = a.g;
  const uint32_t nr = a.n[0], nb = a.n[1], nt = nr + nb, ncol = nt + nb;
  if (g.total > kCmMaxSlots || nt > (uint32_t)kCoarseMatMax) return;
  if (blockIdx.x * kCmWarps >= ncol) return;  // the other order's map needs more CTAs
  for (long long e = threadIdx.x; e < 2 * g.total; e += blockDim.x) map[e >= g.total][e % g.total] = -1;
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < nt; e += blockDim.x) {
    const int c = e >= nr;
    const uint32_t u = c ? e - nr : e;
    const long long at = a.list[c][u] & kListAt;
    if (entry_ok(g, at, 12)) map[c][at] = (int8_t)u;
  }
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < nt; e += blockDim.x) {
    const int c = e >= nr;
    const uint32_t u = c ? e - nr : e;
    const uint32_t ent = a.list[c][u];
    long long at = ent & kListAt;
    if (!entry_ok(g, at, 12)) at = g.off0;
    const long long dx = (ent & kListPlusX) ? 1 : -1;
    const long long off[6] = {0, dx, -(long long)g.P, (long long)g.P, -g.sz, g.sz};
    for (int k = 0; k < 6; ++k) nbr[c][u][k] = map[c ^ 1][at + off[k]];
    id[c][u] = KIND == 1 ? a.invd[c][at] : T(1) / T(6);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t j = blockIdx.x * kCmWarps + w;
  if (j >= ncol) return;
  T(*x)[kCoarseMatMax] = xs[w];
  for (uint32_t u = lane; u < (uint32_t)kCoarseMatMax; u += 32) {
    x[0][u] = T(0);
    x[1][u] = (j >= nt && u == j - nt) ? T(1) : T(0);
  }
  __syncwarp();
  const int bc = j < nr ? 0 : (j < nt ? 1 : -1);  // the colour of the unit right-hand side
  const uint32_t bu = bc == 0 ? j : j - nr;
  for (int s = 0; s < a.sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      for (uint32_t u = lane; u < a.n[c]; u += 32) {
        T v[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = nbr[c][u][k] >= 0 ? x[c ^ 1][nbr[c][u][k]] : T(0);
        const T sum = ((v[0] + v[1]) + (v[2] + v[3])) + (v[4] + v[5]);
        x[c][u] = (sum - ((bc == c && bu == u) ? T(1) : T(0))) * id[c][u];
      }
      __syncwarp();
    }
  for (uint32_t i = lane; i < nt; i += 32) a.out[(size_t)i * ncol + j] = i < nr ? x[0][i] : x[1][i - nr];
}

// Both orders' maps in one launch: blockIdx.y = 0 builds order 1's (the
// first-order operator, D = 6), 1 order 2's; an order with no map has no
// columns.
template <typename T>
__global__ void __launch_bounds__(kCmWarps * 32) coarse_matrix_kernel(CoarseMatArgs<T> a1, CoarseMatArgs<T> a2) {
  __shared__ CoarseMatSmem<T> sm;
  if (blockIdx.y == 0) coarse_matrix_body<2, T>(a1, sm);
  else coarse_matrix_body<1, T>(a2, sm);
}

// b / D of the level-0 unknowns (D = 6 + ghost faces), for SCALED sweeps;
// 0 on inactive cells.
__global__ void scale_rhs_kernel(long long total, const double* __restrict__ r0, const double* __restrict__ r1,
                                 const uint8_t* __restrict__ c0, const uint8_t* __restrict__ c1, double* __restrict__ o0,
                                 double* __restrict__ o1) {
  pdl_wait();
  __shared__ double tab[16];
  init_tab(tab);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    o0[e] = (c0[e] & kActive2) ? r0[e] * tab[__popc((unsigned)c0[e] >> kGhostShift)] : 0.0;
    o1[e] = (c1[e] & kActive2) ? r1[e] * tab[__popc((unsigned)c1[e] >> kGhostShift)] : 0.0;
  }
}

}  // namespace

bool small_level(const Geom& g) { return (long long)g.hx * g.ny * g.nz <= 4096; }

cudaError_t init_cycle_kernels() {
  cudaError_t e = cudaSuccess;
#define GBMG_SMEM_ATTR(K, T)                                                                                \
  if (e == cudaSuccess)                                                                                     \
    e = cudaFuncSetAttribute(smooth_small_kernel<K, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             kSmallSmemBytes);
  GBMG_SMEM_ATTR(0, double)
  GBMG_SMEM_ATTR(1, double)
  GBMG_SMEM_ATTR(2, double)
  GBMG_SMEM_ATTR(0, float)
  GBMG_SMEM_ATTR(1, float)
  GBMG_SMEM_ATTR(2, float)
#undef GBMG_SMEM_ATTR
#define GBMG_BOTTOM_ATTR(K, T)                                                                          \
  if (e == cudaSuccess)                                                                                 \
    e = cudaFuncSetAttribute(bottom_kernel<K, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             kBottomSmemBytes);                                                         \
  if (e == cudaSuccess)                                                                                 \
    e = cudaFuncSetAttribute(bottom_kernel<K, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             kBottomSmemBytes);
  GBMG_BOTTOM_ATTR(1, double)
  GBMG_BOTTOM_ATTR(2, double)
  GBMG_BOTTOM_ATTR(1, float)
  GBMG_BOTTOM_ATTR(2, float)
#undef GBMG_BOTTOM_ATTR
#define GBMG_MID_ATTR(K, T)                                                                                     \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(mid_kernel<K, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottomSmemBytes); \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(mid_kernel<K, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottomSmemBytes);
  GBMG_MID_ATTR(1, double)
  GBMG_MID_ATTR(2, double)
  GBMG_MID_ATTR(1, float)
  GBMG_MID_ATTR(2, float)
#undef GBMG_MID_ATTR
  return e;
}

cudaError_t launch_half_sweep(const LevelDev& L, int order, int colour, int prec, bool update, cudaStream_t s) {
  return prec == kFP32 ? half_sweep_t<float>(L, order, colour, update, s)
                       : half_sweep_t<double>(L, order, colour, update, s);
}

cudaError_t launch_smooth_small(const LevelDev& L, int order, int sweeps, int prec, cudaStream_t s) {
  return prec == kFP32 ? smooth_small_t<float>(L, order, sweeps, s) : smooth_small_t<double>(L, order, sweeps, s);
}

cudaError_t launch_restrict(const LevelDev& Lf, const LevelDev& Lc, int order, bool black_zero, int prec,
                            cudaStream_t s, bool all_cells) {
  return prec == kFP32 ? restrict_t<float>(Lf, Lc, order, black_zero, all_cells, s)
                       : restrict_t<double>(Lf, Lc, order, black_zero, all_cells, s);
}

cudaError_t launch_prolong(const LevelDev& Lc, const LevelDev& Lf, int order, int prec, bool black_only,
                           cudaStream_t s) {
  return prec == kFP32 ? prolong_t<float>(Lc, Lf, order, black_only, s)
                       : prolong_t<double>(Lc, Lf, order, black_only, s);
}


// Fills the bottom arguments for levels lb .. deepest and their shared
// memory plan (plan_bottom_smem): the returned bytes hold the unknown
// records of every level and the staged levels (first_smem on).
template <typename T>
bool fill_bottom(const LevelDev* levels, int lb, int deepest, int order, int n_pre, int n_post, int coarse_sweeps,
                 int n_cycles, BottomArgs<T>& a, size_t* smem_bytes) {
  a.nlev = deepest - lb + 1;
  if (lb < 1 || a.nlev < 1 || a.nlev > kBottomMaxLevels) return false;
  for (int i = 0; i < a.nlev; ++i) {
    const LevelDev& L = levels[lb + i];
    const Fields<T> f = fields(L, T());
    a.L[i].g = L.g;
    for (int c = 0; c < 2; ++c) {
      a.L[i].phi[c] = f.phi[c];
      a.L[i].rhs[c] = f.rhs[c];
      a.L[i].invd[c] = f.invd[c];
      a.L[i].diag[c] = f.diag[c];
      a.L[i].code[c] = L.code[c];
      a.L[i].list[c] = L.list[order][c];
    }
    a.L[i].count = L.count + order * 2;
  }
  a.bit = bit_of(lb, order);
  a.n_pre = n_pre;
  a.n_post = n_post;
  a.coarse_sweeps = coarse_sweeps;
  a.n_cycles = n_cycles;
  a.cmat = nullptr;
  a.cmat_n[0] = a.cmat_n[1] = 0;
  *smem_bytes = plan_bottom_smem(a, levels, lb, order);
  return *smem_bytes <= (size_t)kBottomSmemBytes;
}

template <typename T>
cudaError_t bottom_t(const LevelDev* levels, int lb, int deepest, int order, int n_pre, int n_post, int coarse_sweeps,
                     int n_cycles, const T* cmat, const uint32_t* cmat_n, cudaStream_t s) {
  BottomArgs<T> a;
  size_t bytes = 0;
  if (!fill_bottom(levels, lb, deepest, order, n_pre, n_post, coarse_sweeps, n_cycles, a, &bytes))
    return cudaErrorInvalidValue;
  if (cmat && cmat_n) {  // the coarsest solve through its precomputed map
    a.cmat = cmat;
    a.cmat_n[0] = cmat_n[0];
    a.cmat_n[1] = cmat_n[1];
  }
  const bool sm = a.first_smem < a.nlev;  // some level's correction staged
  count_launch();
  if (order == 1) {
    if (sm) launch_pdl(bottom_kernel<2, T, true>, dim3(1), dim3(kBottomThreads), bytes, s, a);
    else launch_pdl(bottom_kernel<2, T, false>, dim3(1), dim3(kBottomThreads), bytes, s, a);
  } else {
    if (sm) launch_pdl(bottom_kernel<1, T, true>, dim3(1), dim3(kBottomThreads), bytes, s, a);
    else launch_pdl(bottom_kernel<1, T, false>, dim3(1), dim3(kBottomThreads), bytes, s, a);
  }
  return cudaGetLastError();
}

template <int KIND, typename T, bool SMEM>
cudaError_t launch_mid_cluster(const MidArgs<T>& a, size_t bytes, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kMidCluster, 1, 1);
  cfg.blockDim = dim3(kMidThreads, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kMidCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mid_kernel<KIND, T, SMEM>, a);
}

template <typename T>
cudaError_t mid_t(const LevelDev* levels, int m, int lb, int deepest, int order, int n_pre, int n_post,
                  int coarse_sweeps, const T* cmat, const uint32_t* cmat_n, cudaStream_t s) {
  MidArgs<T> a;
  a.nmid = lb - m;
  if (m < 1 || a.nmid < 1 || a.nmid > kMidMaxLevels) return cudaErrorInvalidValue;
  for (int i = 0; i <= a.nmid; ++i) {
    const LevelDev& L = levels[m + i];
    const Fields<T> f = fields(L, T());
    a.L[i].g = L.g;
    for (int c = 0; c < 2; ++c) {
      a.L[i].phi[c] = f.phi[c];
      a.L[i].rhs[c] = f.rhs[c];
      a.L[i].invd[c] = f.invd[c];
      a.L[i].diag[c] = f.diag[c];
      a.L[i].code[c] = L.code[c];
      a.L[i].list[c] = L.list[order][c];
    }
    a.L[i].count = L.count + order * 2;
  }
  a.bit = bit_of(m, order);
  a.n_pre = n_pre;
  a.n_post = n_post;
  size_t bytes = 0;
  if (!fill_bottom(levels, lb, deepest, order, n_pre, n_post, coarse_sweeps, 1, a.bottom, &bytes))
    return cudaErrorInvalidValue;
  if (cmat && cmat_n) {
    a.bottom.cmat = cmat;
    a.bottom.cmat_n[0] = cmat_n[0];
    a.bottom.cmat_n[1] = cmat_n[1];
  }
  count_launch();
  const bool sm = a.bottom.first_smem < a.bottom.nlev;
  if (order == 1) return sm ? launch_mid_cluster<2, T, true>(a, bytes, s) : launch_mid_cluster<2, T, false>(a, bytes, s);
  return sm ? launch_mid_cluster<1, T, true>(a, bytes, s) : launch_mid_cluster<1, T, false>(a, bytes, s);
}

cudaError_t launch_bottom(const LevelDev* levels, int lb, int deepest, int order, int n_pre, int n_post,
                          int coarse_sweeps, int n_cycles, int prec, const void* cmat, const uint32_t* cmat_n,
                          cudaStream_t s) {
  return prec == kFP32 ? bottom_t<float>(levels, lb, deepest, order, n_pre, n_post, coarse_sweeps, n_cycles,
                                         static_cast<const float*>(cmat), cmat_n, s)
                       : bottom_t<double>(levels, lb, deepest, order, n_pre, n_post, coarse_sweeps, n_cycles,
                                          static_cast<const double*>(cmat), cmat_n, s);
}

bool coarse_map_fits(const LevelDev& L, int order) {
  return L.level >= 1 && L.g.total <= kCmMaxSlots &&
         (long long)L.hcount[order * 2] + L.hcount[order * 2 + 1] <= kCoarseMatMax;
}

size_t coarse_map_bytes(int prec) {
  return (size_t)kCoarseMatMax * 2 * kCoarseMatMax * (prec == kFP32 ? sizeof(float) : sizeof(double));
}

template <typename T>
CoarseMatArgs<T> coarse_map_args(const LevelDev* L, int order, int sweeps, T* out) {
  CoarseMatArgs<T> a = {};
  a.sweeps = sweeps;
  a.out = out;
  if (!L) return a;  // no map for this order: no columns
  const Fields<T> f = fields(*L, T());
  a.g = L->g;
  for (int c = 0; c < 2; ++c) {
    a.list[c] = L->list[order][c];
    a.invd[c] = f.invd[c];
    a.n[c] = L->hcount[order * 2 + c];
  }
  return a;
}

template <typename T>
cudaError_t coarse_maps_t(const LevelDev* L1, const LevelDev* L2, int sweeps, T* out1, T* out2, cudaStream_t s) {
  const CoarseMatArgs<T> a1 = coarse_map_args(L1, 1, sweeps, out1), a2 = coarse_map_args(L2, 2, sweeps, out2);
  const uint32_t n1 = a1.n[0] + 2 * a1.n[1], n2 = a2.n[0] + 2 * a2.n[1];
  const unsigned grid = ((n1 > n2 ? n1 : n2) + kCmWarps - 1) / kCmWarps;
  if (grid == 0) return cudaSuccess;
  count_launch();
  coarse_matrix_kernel<T><<<dim3(grid, 2), kCmWarps * 32, 0, s>>>(a1, a2);
  return cudaGetLastError();
}

cudaError_t launch_coarse_maps(const LevelDev* L1, const LevelDev* L2, int sweeps, int prec, void* out1, void* out2,
                               cudaStream_t s) {
  return prec == kFP32 ? coarse_maps_t<float>(L1, L2, sweeps, static_cast<float*>(out1), static_cast<float*>(out2), s)
                       : coarse_maps_t<double>(L1, L2, sweeps, static_cast<double*>(out1),
                                               static_cast<double*>(out2), s);
}

bool mid_level(const Geom& g) { return (long long)g.hx * g.ny * g.nz <= kMidSlots; }

cudaError_t launch_mid(const LevelDev* levels, int m, int lb, int deepest, int order, int n_pre, int n_post,
                       int coarse_sweeps, int prec, const void* cmat, const uint32_t* cmat_n, cudaStream_t s) {
  return prec == kFP32 ? mid_t<float>(levels, m, lb, deepest, order, n_pre, n_post, coarse_sweeps,
                                      static_cast<const float*>(cmat), cmat_n, s)
                       : mid_t<double>(levels, m, lb, deepest, order, n_pre, n_post, coarse_sweeps,
                                       static_cast<const double*>(cmat), cmat_n, s);
}

cudaError_t launch_scale_rhs(const LevelDev& L0, cudaStream_t s) {
  if (!L0.rhsd[0]) return cudaSuccess;
  long long b = (L0.g.total + 255) / 256;
  if (b > 16LL * device_sms()) b = 16LL * device_sms();
  count_launch();
  launch_pdl(scale_rhs_kernel, dim3((unsigned)b), dim3(256), 0, s, L0.g.total, (const double*)L0.rhs[0],
             (const double*)L0.rhs[1], (const uint8_t*)L0.code[0], (const uint8_t*)L0.code[1], L0.rhsd[0], L0.rhsd[1]);
  return cudaGetLastError();
}

int residual_norm_blocks(const Geom& g) {
  const int plain = device_sms() * 8;
  const int lists = 2 * list_grid(g);
  return lists > plain ? lists : plain;
}

cudaError_t launch_residual_norm2(const LevelDev& L0, bool red_only, bool with_phi, double* partials,
                                  int max_partials, double* out, cudaStream_t s) {
  int blocks;
  if (!with_phi) {
    NormArgs a;
    a.g = L0.g;
    for (int c = 0; c < 2; ++c) {
      a.rhs[c] = L0.rhs[c];
      a.code[c] = L0.code[c];
    }
    a.bit = kActive2;
    a.partials = partials;
    blocks = device_sms() * 8;
    count_launch();
    launch_pdl(rhsnorm_kernel, dim3(blocks), dim3(kNormThreads), 0, s, a);
  } else {
    const int grid = list_grid(L0.g);
    blocks = red_only ? grid : 2 * grid;
    if (blocks > max_partials) return cudaErrorInvalidValue;
    for (int c = 0; c < (red_only ? 1 : 2); ++c) {
      ListArgs<double> a = list_args<double>(L0, 2, c);
      a.partials = partials + c * grid;
      count_launch();
      if (L0.exact_sum) launch_pdl(res_list_kernel<0, double, true>, dim3(grid), dim3(kListBlock), 0, s, a);
      else launch_pdl(res_list_kernel<0, double>, dim3(grid), dim3(kListBlock), 0, s, a);
    }
  }
  count_launch();
  launch_pdl(finalize_kernel, dim3(1), dim3(kFinalThreads), 0, s, partials, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_refine_residual(const LevelDev& L0, double* partials, int max_partials, double* out,
                                   cudaStream_t s) {
  RefineArgs a;
  a.g = L0.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = L0.phi[c];
    a.rhs[c] = L0.rhs[c];
    a.code[c] = L0.code[c];
    a.list[c] = L0.list[2][c];
    a.count[c] = L0.count + 4 + c;
    a.rhs32[c] = L0.rhs32[c];
    a.e32[c] = L0.phi32[c];
  }
  a.partials = partials;
  const int blocks = 2 * list_grid(L0.g);
  if (blocks > max_partials) return cudaErrorInvalidValue;
  count_launch(2);
  if (L0.exact_sum) launch_pdl(refine_residual_kernel<true>, dim3(blocks), dim3(kListBlock), 0, s, a);
  else launch_pdl(refine_residual_kernel<false>, dim3(blocks), dim3(kListBlock), 0, s, a);
  launch_pdl(finalize_kernel, dim3(1), dim3(kFinalThreads), 0, s, partials, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_refine_update(const LevelDev& L0, cudaStream_t s) {
  UpdateArgs a;
  a.g = L0.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = L0.phi[c];
    a.e32[c] = L0.phi32[c];
    a.list[c] = L0.list[2][c];
    a.count[c] = L0.count + 4 + c;
  }
  count_launch();
  launch_pdl(refine_update_kernel, dim3(exact_grid(L0.hcount[4] + L0.hcount[5], 1)), dim3(kListBlock), 0, s, a);
  return cudaGetLastError();
}



}  // namespace gbmg
