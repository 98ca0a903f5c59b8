// V-cycle kernels of the masked-domain multigrid solver (Guillet & Teyssier,
// arXiv:1104.1703, Section 2 recipe): red-black Gauss-Seidel half-sweeps,
// residual + R1 restriction, P2 prolongation + correction, residual norm.
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
// On GB300 every one of these kernels is bound by the FP64 pipe (2 FP64
// lane-operations per clock per SM), not by HBM, and a warp instruction
// costs the pipe the same whether or not its lanes are predicated off.  So
// the kernels run over compact lists of the unknowns (built once per mask),
// where every lane holds an unknown, and issue as few FP64 instructions as
// the operator allows.  Neighbour values come through L1/L2.

#include "mg_internal.h"

namespace gbmg {

namespace {

constexpr int kBlockX = 32, kBlockY = 4;

// KIND 0: level 0 (D from the ghost-face count); 1: coarse, second order
// (per-cell D and 1/D); 2: coarse, first order (D = 6).
template <int KIND>
__device__ __forceinline__ double inv_diag(uint8_t code, const double* __restrict__ invd, long long at,
                                           const double* tab) {
  if (KIND == 0) return tab[__popc((unsigned)code >> kGhostShift)];
  if (KIND == 1) return invd[at];
  return 1.0 / 6.0;
}

template <int KIND>
__device__ __forceinline__ double diag_of(uint8_t code, const double* __restrict__ diag, long long at) {
  if (KIND == 0) return (double)(6 + __popc((unsigned)code >> kGhostShift));
  if (KIND == 1) return diag[at];
  return 6.0;
}

__device__ __forceinline__ double nbr_sum(const double* __restrict__ o, long long at, int dx, int P,
                                          long long sz) {
  return ((o[at] + o[at + dx]) + (o[at - P] + o[at + P])) + (o[at - sz] + o[at + sz]);
}

__device__ __forceinline__ void init_tab(double* tab) {
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  if (t < 8) tab[t] = 1.0 / (double)(6 + t);
  __syncthreads();
}

// x offset of the non-shared x-neighbour of a colour-c cell in row (j, k)
__device__ __forceinline__ int x_offset(int c, int j, int k) { return ((c ^ j ^ k) & 1) ? 1 : -1; }

constexpr int kListBlock = 256;

struct ListArgs {
  Geom g;
  double* self;          // Phi of the listed colour
  const double* other;   // Phi of the other colour
  const double* rhs;
  const double* invd;
  const double* diag;
  const uint8_t* code;
  const uint32_t* list;
  const uint32_t* count;
  double* res;
  double* partials;
};

// K4: one colour of a red-black Gauss-Seidel sweep (Section 2) over the
// compact list of that colour's unknowns: every lane of every warp updates
// an unknown, so no FP64 issue slot is spent on a predicated-off lane.
template <int KIND>
__global__ void __launch_bounds__(kListBlock) gs_list_kernel(ListArgs a) {
  __shared__ double tab[8];
  if (KIND == 0) init_tab(tab);
  const Geom g = a.g;
  const uint32_t n = *a.count;
  for (uint32_t i = blockIdx.x * kListBlock + threadIdx.x; i < n; i += gridDim.x * kListBlock) {
    const uint32_t e = a.list[i];
    const long long at = e & kListAt;
    const double s = nbr_sum(a.other, at, (e & kListPlusX) ? 1 : -1, g.P, g.sz);
    const uint8_t code = KIND == 0 ? a.code[at] : 0;
    a.self[at] = (s - a.rhs[at]) * inv_diag<KIND>(code, a.invd, at, tab);
  }
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

// Scaled residual r^ = sum_nbr Phi_j - D Phi_i - b of the listed unknowns
// (Section 2, recipe step 2).  NORM = false stores it for the restriction;
// NORM = true sums r^2 per block into partials[blockIdx.x] (K9, first pass;
// the grid is fixed per level, so the partials do not depend on scheduling).
template <int KIND, bool NORM>
__global__ void __launch_bounds__(kListBlock) res_list_kernel(ListArgs a) {
  const Geom g = a.g;
  const uint32_t n = *a.count;
  double acc = 0.0;
  for (uint32_t i = blockIdx.x * kListBlock + threadIdx.x; i < n; i += gridDim.x * kListBlock) {
    const uint32_t e = a.list[i];
    const long long at = e & kListAt;
    const double s = nbr_sum(a.other, at, (e & kListPlusX) ? 1 : -1, g.P, g.sz);
    const uint8_t code = KIND == 0 ? a.code[at] : 0;
    const double r = fma(-diag_of<KIND>(code, a.diag, at), a.self[at], s) - a.rhs[at];
    if (NORM)
      acc = fma(r, r, acc);
    else
      a.res[at] = r;
  }
  if (NORM) block_reduce_store(acc, a.partials + blockIdx.x);
}

struct SmallArgs {
  Geom g;
  double* phi0;
  double* phi1;
  const double* rhs0;
  const double* rhs1;
  const double* invd0;
  const double* invd1;
  const uint8_t* code0;
  const uint8_t* code1;
  uint8_t bit;
  int sweeps;
};

constexpr int kSmallThreads = 512;
constexpr int kSmallSmemBytes = 96 * 1024;

// Several full sweeps of a small level inside one CTA (no launch per
// half-sweep); __syncthreads separates the colours.  With SMEM the two
// colour arrays of Phi (halo included) are staged in shared memory for the
// whole call, so every neighbour read is an on-chip load.
template <int KIND, bool SMEM>
__global__ void __launch_bounds__(kSmallThreads) smooth_small_kernel(SmallArgs a) {
  extern __shared__ double sm[];
  __shared__ double tab[8];
  if (KIND == 0) init_tab(tab);
  const Geom g = a.g;
  double* p0 = a.phi0;
  double* p1 = a.phi1;
  if (SMEM) {
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
      double* self = c ? p1 : p0;
      const double* o = c ? p0 : p1;
      const double* rhs = c ? a.rhs1 : a.rhs0;
      const double* invd = c ? a.invd1 : a.invd0;
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

struct RestrictArgs {
  Geom gf, gc;
  const double* res[2];
  const uint8_t* code[2];
  uint8_t bit;
  double* crhs[2];
  double* cphi[2];
};

// K5 (second half): R1 of the stored fine residuals into the coarse
// right-hand side, b_c = -1/2 sum of the children's r^ (Section 2, recipe
// steps 3-5; Fig. 3), and dPhi_c = 0.  Thread (I, J) of coarse plane K; the
// two x-children of coarse cell I are both at fine slot I of the child rows.
// With BLACK_ZERO the last fine operation was a full red-black sweep, after
// which every black cell satisfies its own equation, so only red children
// carry a residual.  Children outside the active set (of this order) count 0.
template <bool BLACK_ZERO>
__global__ void __launch_bounds__(kBlockX * kBlockY) restrict_sum_kernel(RestrictArgs a) {
  const Geom gf = a.gf, gc = a.gc;
  const int I = blockIdx.x * kBlockX + threadIdx.x;
  const int J = blockIdx.y * kBlockY + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= gc.nx || J >= gc.ny) return;
  double sum = 0.0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk) {
    const int k = 2 * K + dk;
    if (k >= gf.nz) break;
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      const int j = 2 * J + dj;
      if (j >= gf.ny) break;
      const long long at = gf.at(I, j, k);
#pragma unroll
      for (int c = 0; c < (BLACK_ZERO ? 1 : 2); ++c)
        if (a.code[c][at] & a.bit) sum += a.res[c][at];
    }
  }
  const int C = (I + J + K) & 1;
  const long long atc = gc.at(I >> 1, J, K);
  a.crhs[C][atc] = -0.5 * sum;
  a.cphi[C][atc] = 0.0;
}

struct ProlongArgs {
  Geom gf, gc;
  double* phi[2];
  const uint32_t* list[2];
  const uint32_t* count[2];
  const double* cphi[2];
};

__device__ __forceinline__ double coarse_at(const ProlongArgs& a, int X, int Y, int Z) {
  return a.cphi[(X + Y + Z) & 1][a.gc.at(X >> 1, Y, Z)];
}

// K6: Phi_f += P2(dPhi_c) on the unknowns of the fine level (Section 2,
// recipe steps 6-7; Fig. 3).  Per axis a fine cell lies 1/4 of a coarse cell
// from its parent ("near") and 3/4 from the coarse neighbour on its side
// ("far"); P2 weighs them 3/4 and 1/4, so the 8 corner weights are 27, 9, 3
// and 1 (/64) for 0, 1, 2 and 3 far axes.  Grouping the corners by weight
// costs 9 FP64 instructions per fine cell.  Coarse cells outside Omega_c
// hold 0 and out-of-box coarse indices read the zero halo.
__global__ void __launch_bounds__(kListBlock) prolong_list_kernel(ProlongArgs a) {
  const Geom gf = a.gf;
  const uint32_t n0 = *a.count[0], n = n0 + *a.count[1];
  for (uint32_t i = blockIdx.x * kListBlock + threadIdx.x; i < n; i += gridDim.x * kListBlock) {
    const int c = i >= n0;
    const uint32_t e = c ? a.list[1][i - n0] : a.list[0][i];
    const long long at = e & kListAt;
    const int rel = (int)(at - gf.off0);
    const int k = rel / (int)gf.sz;
    const int rem = rel - k * (int)gf.sz;
    const int j = rem / gf.P;
    const int q = rem - j * gf.P;
    const int ix = 2 * q + ((c ^ j ^ k) & 1);
    const int Xn = q, Xf = q + ((ix & 1) ? 1 : -1);
    const int Yn = j >> 1, Yf = Yn + ((j & 1) ? 1 : -1);
    const int Zn = k >> 1, Zf = Zn + ((k & 1) ? 1 : -1);
    const double e0 = coarse_at(a, Xn, Yn, Zn);
    const double e1 = (coarse_at(a, Xf, Yn, Zn) + coarse_at(a, Xn, Yf, Zn)) + coarse_at(a, Xn, Yn, Zf);
    const double e2 = (coarse_at(a, Xn, Yf, Zf) + coarse_at(a, Xf, Yn, Zf)) + coarse_at(a, Xf, Yf, Zn);
    const double e3 = coarse_at(a, Xf, Yf, Zf);
    const double w = fma(3.0, e2, fma(27.0, e0, 9.0 * e1)) + e3;
    a.phi[c][at] = fma(w, 1.0 / 64.0, a.phi[c][at]);
  }
}

struct NormArgs {
  Geom g;
  const double* rhs[2];
  const uint8_t* code[2];
  uint8_t bit;
  double* partials;
};

// sum of b^2 over the active cells (the residual of Phi = 0 is -b)
__global__ void __launch_bounds__(kNormThreads) rhsnorm_kernel(NormArgs a) {
  const Geom g = a.g;
  const long long per_colour = (long long)g.hx * g.ny * g.nz;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * per_colour;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = e >= per_colour;
    const long long r = e - c * per_colour;
    const int q = (int)(r % g.hx);
    const long long t = r / g.hx;
    const long long at = g.at(q, (int)(t % g.ny), (int)(t / g.ny));
    if (a.code[c][at] & a.bit) acc = fma(a.rhs[c][at], a.rhs[c][at], acc);
  }
  block_reduce_store(acc, a.partials + blockIdx.x);
}

// K9 (second pass): one CTA sums the partials in a fixed order.
__global__ void __launch_bounds__(kNormThreads) finalize_kernel(const double* __restrict__ partials, int n,
                                                                double* out) {
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc += partials[e];
  __shared__ double sm[kNormThreads];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kNormThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

int kind_of(int level, int order) { return level == 0 ? 0 : (order == 1 ? 2 : 1); }
uint8_t bit_of(int level, int order) { return (level >= 1 && order == 1) ? kActive1 : kActive2; }

// fixed grid of the list kernels of a level: enough blocks for every slot of
// one colour, at most 16 per SM (grid-stride beyond that)
int list_grid(const Geom& g) {
  const long long n = (long long)g.hx * g.ny * g.nz;
  long long b = (n + kListBlock - 1) / kListBlock;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

bool small_smem(const Geom& g) { return 2 * g.total * (long long)sizeof(double) <= kSmallSmemBytes; }

// level 0 has a single active set, stored under order 2
int list_order(const LevelDev& L, int order) { return L.level == 0 ? 2 : order; }

ListArgs list_args(const LevelDev& L, int order, int colour) {
  ListArgs a;
  a.g = L.g;
  a.self = L.phi[colour];
  a.other = L.phi[colour ^ 1];
  a.rhs = L.rhs[colour];
  a.invd = L.level ? L.invd[colour] : nullptr;
  a.diag = L.level ? L.diag[colour] : nullptr;
  a.code = L.code[colour];
  a.list = L.list[list_order(L, order)][colour];
  a.count = L.count + list_order(L, order) * 2 + colour;
  a.res = L.res[colour];
  a.partials = nullptr;
  return a;
}

}  // namespace

bool small_level(const Geom& g) { return (long long)g.hx * g.ny * g.nz <= 4096; }

cudaError_t init_cycle_kernels() {
  cudaError_t e = cudaSuccess;
#define GBMG_SMEM_ATTR(K)                                                                                \
  if (e == cudaSuccess)                                                                                  \
    e = cudaFuncSetAttribute(smooth_small_kernel<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             kSmallSmemBytes);
  GBMG_SMEM_ATTR(0)
  GBMG_SMEM_ATTR(1)
  GBMG_SMEM_ATTR(2)
#undef GBMG_SMEM_ATTR
  return e;
}

cudaError_t launch_half_sweep(const LevelDev& L, int order, int colour, cudaStream_t s) {
  const ListArgs a = list_args(L, order, colour);
  const int grid = list_grid(L.g);
  count_launch();
  switch (kind_of(L.level, order)) {
    case 0: gs_list_kernel<0><<<grid, kListBlock, 0, s>>>(a); break;
    case 1: gs_list_kernel<1><<<grid, kListBlock, 0, s>>>(a); break;
    default: gs_list_kernel<2><<<grid, kListBlock, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_smooth_small(const LevelDev& L, int order, int sweeps, cudaStream_t s) {
  SmallArgs a;
  a.g = L.g;
  a.phi0 = L.phi[0];
  a.phi1 = L.phi[1];
  a.rhs0 = L.rhs[0];
  a.rhs1 = L.rhs[1];
  a.invd0 = L.level ? L.invd[0] : nullptr;
  a.invd1 = L.level ? L.invd[1] : nullptr;
  a.code0 = L.code[0];
  a.code1 = L.code[1];
  a.bit = bit_of(L.level, order);
  a.sweeps = sweeps;
  const bool sm = small_smem(L.g);
  const size_t bytes = sm ? 2 * L.g.total * sizeof(double) : 0;
  count_launch();
#define GBMG_SMALL(K)                                                      \
  if (sm) smooth_small_kernel<K, true><<<1, kSmallThreads, bytes, s>>>(a); \
  else smooth_small_kernel<K, false><<<1, kSmallThreads, 0, s>>>(a);
  switch (kind_of(L.level, order)) {
    case 0: GBMG_SMALL(0) break;
    case 1: GBMG_SMALL(1) break;
    default: GBMG_SMALL(2) break;
  }
#undef GBMG_SMALL
  return cudaGetLastError();
}

// residual of the listed unknowns of one colour into L.res (NORM = false)
static cudaError_t launch_residual(const LevelDev& L, int order, int colour, cudaStream_t s) {
  const ListArgs a = list_args(L, order, colour);
  const int grid = list_grid(L.g);
  count_launch();
  switch (kind_of(L.level, order)) {
    case 0: res_list_kernel<0, false><<<grid, kListBlock, 0, s>>>(a); break;
    case 1: res_list_kernel<1, false><<<grid, kListBlock, 0, s>>>(a); break;
    default: res_list_kernel<2, false><<<grid, kListBlock, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_restrict(const LevelDev& Lf, const LevelDev& Lc, int order, bool black_zero, cudaStream_t s) {
  cudaError_t e = launch_residual(Lf, order, 0, s);
  if (e == cudaSuccess && !black_zero) e = launch_residual(Lf, order, 1, s);
  if (e != cudaSuccess) return e;
  RestrictArgs a;
  a.gf = Lf.g;
  a.gc = Lc.g;
  for (int c = 0; c < 2; ++c) {
    a.res[c] = Lf.res[c];
    a.code[c] = Lf.code[c];
    a.crhs[c] = Lc.rhs[c];
    a.cphi[c] = Lc.phi[c];
  }
  a.bit = bit_of(Lf.level, order);
  const dim3 grid((Lc.g.nx + kBlockX - 1) / kBlockX, (Lc.g.ny + kBlockY - 1) / kBlockY, Lc.g.nz);
  const dim3 block(kBlockX, kBlockY);
  count_launch();
  if (black_zero)
    restrict_sum_kernel<true><<<grid, block, 0, s>>>(a);
  else
    restrict_sum_kernel<false><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const LevelDev& Lc, const LevelDev& Lf, int order, cudaStream_t s) {
  ProlongArgs a;
  a.gf = Lf.g;
  a.gc = Lc.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = Lf.phi[c];
    a.list[c] = Lf.list[list_order(Lf, order)][c];
    a.count[c] = Lf.count + list_order(Lf, order) * 2 + c;
    a.cphi[c] = Lc.phi[c];
  }
  count_launch();
  prolong_list_kernel<<<list_grid(Lf.g), kListBlock, 0, s>>>(a);
  return cudaGetLastError();
}

int residual_norm_blocks(const Geom& g) {
  const int plain = 152 * 8;
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
    blocks = 152 * 8;
    count_launch();
    rhsnorm_kernel<<<blocks, kNormThreads, 0, s>>>(a);
  } else {
    const int grid = list_grid(L0.g);
    blocks = red_only ? grid : 2 * grid;
    if (blocks > max_partials) return cudaErrorInvalidValue;
    for (int c = 0; c < (red_only ? 1 : 2); ++c) {
      ListArgs a = list_args(L0, 2, c);
      a.partials = partials + c * grid;
      count_launch();
      res_list_kernel<0, true><<<grid, kListBlock, 0, s>>>(a);
    }
  }
  count_launch();
  finalize_kernel<<<1, kNormThreads, 0, s>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace gbmg
