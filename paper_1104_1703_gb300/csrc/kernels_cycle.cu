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
#include "mg_internal.h"

namespace gbmg {

namespace {

// P2 weights (Section 2, Fig. 3): per axis a fine cell takes 3/4 of its
// parent and 1/4 of the coarse neighbour on its side.  kWyz[py*2+pz][b*2+e]
// is the y-z weight of coarse rows Ya+b, Za+e for a fine cell whose y and z
// parities are py, pz (Ya = (j-1)>>1, Za = (k-1)>>1).
__constant__ double kWyz[4][4] = {
    {0.0625, 0.1875, 0.1875, 0.5625},  // py=0 (0.25,0.75) x pz=0 (0.25,0.75)
    {0.1875, 0.0625, 0.5625, 0.1875},  // py=0 x pz=1 (0.75,0.25)
    {0.1875, 0.5625, 0.0625, 0.1875},  // py=1 x pz=0
    {0.5625, 0.1875, 0.1875, 0.0625},  // py=1 x pz=1
};

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

struct SweepArgs {
  Geom g;
  double* self;
  const double* other;
  const double* rhs;
  const double* invd;
  const uint8_t* code;
  int colour;
  uint8_t bit;
  int kchunk;
};

// K4: one colour of a red-black Gauss-Seidel sweep (Section 2).  A thread
// owns slot (q, j) and marches through kchunk planes keeping the z
// neighbours in registers; the same-slot value of the other colour is one of
// the two x-neighbours.
template <int KIND>
__global__ void __launch_bounds__(128) half_sweep_kernel(SweepArgs a) {
  __shared__ double tab[8];
  if (KIND == 0) init_tab(tab);
  const Geom g = a.g;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * a.kchunk;
  if (q >= g.hx || j >= g.ny || k0 >= g.nz) return;
  const int k1 = min(g.nz, k0 + a.kchunk);
  const double* __restrict__ o = a.other;
  long long at = g.at(q, j, k0);
  double zm = o[at - g.sz], z0 = o[at];
  for (int k = k0; k < k1; ++k, at += g.sz) {
    const double zp = o[at + g.sz];
    const uint8_t code = a.code[at];
    if (code & a.bit) {
      const int dx = ((a.colour ^ j ^ k) & 1) ? 1 : -1;
      const double s = ((z0 + o[at + dx]) + (o[at - g.P] + o[at + g.P])) + (zm + zp);
      a.self[at] = (s - a.rhs[at]) * inv_diag<KIND>(code, a.invd, at, tab);
    }
    zm = z0;
    z0 = zp;
  }
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

// Several full sweeps of a small level inside one CTA (no launch per
// half-sweep); __syncthreads separates the colours.
template <int KIND>
__global__ void __launch_bounds__(512) smooth_small_kernel(SmallArgs a) {
  __shared__ double tab[8];
  if (KIND == 0) init_tab(tab);
  const Geom g = a.g;
  const int n = g.hx * g.ny * g.nz;
  for (int s = 0; s < a.sweeps; ++s) {
    for (int c = 0; c < 2; ++c) {
      double* self = c ? a.phi1 : a.phi0;
      const double* o = c ? a.phi0 : a.phi1;
      const double* rhs = c ? a.rhs1 : a.rhs0;
      const double* invd = c ? a.invd1 : a.invd0;
      const uint8_t* code = c ? a.code1 : a.code0;
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int q = e % g.hx, t = e / g.hx, j = t % g.ny, k = t / g.ny;
        const long long at = g.at(q, j, k);
        const uint8_t cd = code[at];
        if (!(cd & a.bit)) continue;
        const int dx = ((c ^ j ^ k) & 1) ? 1 : -1;
        self[at] = (nbr_sum(o, at, dx, g.P, g.sz) - rhs[at]) * inv_diag<KIND>(cd, invd, at, tab);
      }
      __syncthreads();
    }
  }
}

struct RestrictArgs {
  Geom gf, gc;
  const double* phi[2];
  const double* rhs[2];
  const double* diag[2];
  const uint8_t* code[2];
  uint8_t bit;
  double* crhs[2];
  double* cphi[2];
};

// K5: scaled residual of the fine level, R1 into the coarse right-hand side
// (b_c = -1/2 sum of the children's r^), dPhi_c = 0 (Section 2, recipe steps
// 2-5).  One thread per coarse cell; its children in x are both at slot I of
// the four child rows.  With BLACK_ZERO the last fine operation was a full
// red-black sweep, after which every black cell satisfies its own equation,
// so only the red children are evaluated.
template <int KIND, bool BLACK_ZERO>
__global__ void restrict_kernel(RestrictArgs a) {
  const Geom gf = a.gf, gc = a.gc;
  const long long n = gc.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(idx % gc.nx);
    const long long t = idx / gc.nx;
    const int J = (int)(t % gc.ny), K = (int)(t / gc.ny);
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
        for (int c = 0; c < (BLACK_ZERO ? 1 : 2); ++c) {
          const uint8_t code = a.code[c][at];
          if (!(code & a.bit)) continue;
          const int dx = ((c ^ j ^ k) & 1) ? 1 : -1;
          const double s = nbr_sum(a.phi[1 - c], at, dx, gf.P, gf.sz);
          const double D = diag_of<KIND>(code, a.diag[c], at);
          sum += fma(-D, a.phi[c][at], s) - a.rhs[c][at];
        }
      }
    }
    const int C = (I + J + K) & 1;
    const long long atc = gc.at(I >> 1, J, K);
    a.crhs[C][atc] = -0.5 * sum;
    a.cphi[C][atc] = 0.0;
  }
}

struct ProlongArgs {
  Geom gf, gc;
  double* phi[2];
  const uint8_t* code[2];
  const double* cphi[2];
  uint8_t bit;
};

__device__ __forceinline__ double coarse_at(const ProlongArgs& a, int X, int Y, int Z) {
  return a.cphi[(X + Y + Z) & 1][a.gc.at(X >> 1, Y, Z)];
}

// K6: Phi_f += P2(dPhi_c) on active fine cells (Section 2, recipe steps 6-7;
// Fig. 3).  A thread owns fine slot (q, j, k), i.e. the two x-children
// i = 2q and 2q+1 of coarse column q, which share the coarse planes
// Ya..Ya+1, Za..Za+1 and the coarse columns q-1..q+1.  Coarse cells outside
// Omega_c hold 0 and out-of-box coarse indices read the zero halo.
__global__ void __launch_bounds__(128) prolong_kernel(ProlongArgs a) {
  const Geom gf = a.gf;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (q >= gf.hx || j >= gf.ny || k >= gf.nz) return;
  const long long at = gf.at(q, j, k);
  const int c0 = (j + k) & 1;  // colour of i = 2q
  const bool act0 = a.code[c0][at] & a.bit;
  const bool act1 = a.code[c0 ^ 1][at] & a.bit;
  if (!act0 && !act1) return;
  const int Ya = (j - 1) >> 1, Za = (k - 1) >> 1;
  const double* w = kWyz[((j & 1) << 1) | (k & 1)];
  double t[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const int X = q - 1 + x;
    t[x] = w[0] * coarse_at(a, X, Ya, Za);
    t[x] = fma(w[1], coarse_at(a, X, Ya, Za + 1), t[x]);
    t[x] = fma(w[2], coarse_at(a, X, Ya + 1, Za), t[x]);
    t[x] = fma(w[3], coarse_at(a, X, Ya + 1, Za + 1), t[x]);
  }
  if (act0) a.phi[c0][at] += fma(0.25, t[0], 0.75 * t[1]);
  if (act1) a.phi[c0 ^ 1][at] += fma(0.75, t[1], 0.25 * t[2]);
}

struct NormArgs {
  Geom g;
  const double* phi[2];
  const double* rhs[2];
  const double* diag[2];
  const uint8_t* code[2];
  uint8_t bit;
  double* partials;
};

constexpr int kNormThreads = 256;

// K9 (first pass): per-block sums of r^2 over the active cells (only red
// cells with RED_ONLY, see BLACK_ZERO above; WITH_PHI false gives the
// residual of Phi = 0, i.e. -b).  Warp shuffles, then a fixed tree across
// the block's warps, so the partial of each block is reproducible.
template <int KIND, bool RED_ONLY, bool WITH_PHI>
__global__ void __launch_bounds__(kNormThreads) resnorm_kernel(NormArgs a) {
  const Geom g = a.g;
  const long long per_colour = (long long)g.hx * g.ny * g.nz;
  const long long n = RED_ONLY ? per_colour : 2 * per_colour;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / per_colour);
    const long long r = e - c * per_colour;
    const int q = (int)(r % g.hx);
    const long long t = r / g.hx;
    const int j = (int)(t % g.ny), k = (int)(t / g.ny);
    const long long at = g.at(q, j, k);
    const uint8_t code = a.code[c][at];
    if (!(code & a.bit)) continue;
    double res;
    if (WITH_PHI) {
      const int dx = ((c ^ j ^ k) & 1) ? 1 : -1;
      const double s = nbr_sum(a.phi[1 - c], at, dx, g.P, g.sz);
      res = fma(-diag_of<KIND>(code, a.diag[c], at), a.phi[c][at], s) - a.rhs[c][at];
    } else {
      res = a.rhs[c][at];
    }
    acc = fma(res, res, acc);
  }
  __shared__ double warp_sums[kNormThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kNormThreads / 32 ? warp_sums[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = v;
  }
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

int kchunk_for(const Geom& g) {
  const long long cols = (long long)g.hx * g.ny;
  const long long target = 152LL * 2048 * 2;  // resident threads x 2
  long long chunk = (cols * g.nz + target - 1) / target;
  if (chunk < 1) chunk = 1;
  if (chunk > g.nz) chunk = g.nz;
  return (int)chunk;
}

}  // namespace

bool small_level(const Geom& g) { return (long long)g.hx * g.ny * g.nz <= 4096; }

cudaError_t launch_half_sweep(const LevelDev& L, int order, int colour, cudaStream_t s) {
  SweepArgs a;
  a.g = L.g;
  a.self = L.phi[colour];
  a.other = L.phi[colour ^ 1];
  a.rhs = L.rhs[colour];
  a.invd = L.level ? L.invd[colour] : nullptr;
  a.code = L.code[colour];
  a.colour = colour;
  a.bit = bit_of(L.level, order);
  a.kchunk = kchunk_for(L.g);
  dim3 block(32, 4);
  dim3 grid((L.g.hx + 31) / 32, (L.g.ny + 3) / 4, (L.g.nz + a.kchunk - 1) / a.kchunk);
  count_launch();
  switch (kind_of(L.level, order)) {
    case 0: half_sweep_kernel<0><<<grid, block, 0, s>>>(a); break;
    case 1: half_sweep_kernel<1><<<grid, block, 0, s>>>(a); break;
    default: half_sweep_kernel<2><<<grid, block, 0, s>>>(a); break;
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
  count_launch();
  switch (kind_of(L.level, order)) {
    case 0: smooth_small_kernel<0><<<1, 512, 0, s>>>(a); break;
    case 1: smooth_small_kernel<1><<<1, 512, 0, s>>>(a); break;
    default: smooth_small_kernel<2><<<1, 512, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_restrict(const LevelDev& Lf, const LevelDev& Lc, int order, bool black_zero, cudaStream_t s) {
  RestrictArgs a;
  a.gf = Lf.g;
  a.gc = Lc.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = Lf.phi[c];
    a.rhs[c] = Lf.rhs[c];
    a.diag[c] = Lf.level ? Lf.diag[c] : nullptr;
    a.code[c] = Lf.code[c];
    a.crhs[c] = Lc.rhs[c];
    a.cphi[c] = Lc.phi[c];
  }
  a.bit = bit_of(Lf.level, order);
  long long n = Lc.g.ncells();
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  const int kind = kind_of(Lf.level, order);
#define GBMG_RESTRICT(K)                                                    \
  if (black_zero) restrict_kernel<K, true><<<blocks, 256, 0, s>>>(a);       \
  else restrict_kernel<K, false><<<blocks, 256, 0, s>>>(a);
  if (kind == 0) { GBMG_RESTRICT(0) }
  else if (kind == 1) { GBMG_RESTRICT(1) }
  else { GBMG_RESTRICT(2) }
#undef GBMG_RESTRICT
  return cudaGetLastError();
}

cudaError_t launch_prolong(const LevelDev& Lc, const LevelDev& Lf, int order, cudaStream_t s) {
  ProlongArgs a;
  a.gf = Lf.g;
  a.gc = Lc.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = Lf.phi[c];
    a.code[c] = Lf.code[c];
    a.cphi[c] = Lc.phi[c];
  }
  a.bit = bit_of(Lf.level, order);
  dim3 block(32, 4);
  dim3 grid((Lf.g.hx + 31) / 32, (Lf.g.ny + 3) / 4, Lf.g.nz);
  count_launch();
  prolong_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

int residual_norm_blocks(const Geom& g) {
  long long n = 2LL * g.hx * g.ny * g.nz;
  long long b = (n + kNormThreads - 1) / kNormThreads;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_residual_norm2(const LevelDev& L0, bool red_only, bool with_phi, double* partials,
                                  int max_partials, double* out, cudaStream_t s) {
  NormArgs a;
  a.g = L0.g;
  for (int c = 0; c < 2; ++c) {
    a.phi[c] = L0.phi[c];
    a.rhs[c] = L0.rhs[c];
    a.diag[c] = L0.level ? L0.diag[c] : nullptr;
    a.code[c] = L0.code[c];
  }
  a.bit = kActive2;
  a.partials = partials;
  int blocks = residual_norm_blocks(L0.g);
  if (blocks > max_partials) return cudaErrorInvalidValue;
  count_launch(2);
  if (!with_phi) resnorm_kernel<0, false, false><<<blocks, kNormThreads, 0, s>>>(a);
  else if (red_only) resnorm_kernel<0, true, true><<<blocks, kNormThreads, 0, s>>>(a);
  else resnorm_kernel<0, false, true><<<blocks, kNormThreads, 0, s>>>(a);
  finalize_kernel<<<1, kNormThreads, 0, s>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace gbmg
