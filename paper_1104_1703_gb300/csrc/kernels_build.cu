// Hierarchy construction, layout conversion and boundary-data kernels.
//
// Guillet & Teyssier, arXiv:1104.1703:
//  - Section 3: the mask is +1 on active and -1 on inactive fine cells and is
//    averaged (R1) level by level; Omega^l = {m^l > 0}.  We keep the exact
//    integer sums S_l (m_l = S_l / 8^l).
//  - Section 3, Fig. 5: across a boundary the neighbour value is replaced by
//    a ghost extrapolated through Phi_b at distance theta = m_i / (m_i - m_j).
//    Solving a cell's row for Phi_i turns each ghost face into a diagonal
//    contribution 1/theta and a right-hand-side contribution Phi_b/theta.
//    At level 0 theta = 1/2 (the boundary is on the face); at coarse levels
//    Phi_b = 0, so only the diagonal changes.
//  - Section 4: first-order coarse levels keep as unknowns only the cells
//    with m = 1 (S = 8^l); every other cell holds 0, so D = 6.
//  - Section 1 / Fig. 1: the fine Dirichlet values sit on the boundary faces
//    and come from the coarser AMR level by linear interpolation.
#include "mg_internal.h"

namespace gbmg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int colour_of(int i, int j, int k) { return (i + j + k) & 1; }

// (i, j, k) of natural index idx; grids hold fewer than 2^32 cells (a colour
// array, about half of them, is limited to 2^31 elements), so 32-bit
// division suffices.
__device__ __forceinline__ void natural_coords(long long idx, int nx, int ny, int& i, int& j, int& k) {
  const unsigned u = (unsigned)idx;
  const unsigned t = u / (unsigned)nx;
  i = (int)(u - t * (unsigned)nx);
  k = (int)(t / (unsigned)ny);
  j = (int)(t - (unsigned)k * (unsigned)ny);
}

__device__ __forceinline__ long long pow8(int l) { return 1LL << (3 * l); }

// Adds every thread's count into *ctr with one atomic per block (all
// threads of the block call it, after their loop).
__device__ void block_count_add(unsigned long long* ctr, unsigned n) {
  __shared__ unsigned warp_n[32];
  for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(0xffffffffu, n, off);
  if ((threadIdx.x & 31) == 0) warp_n[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned v = threadIdx.x < (blockDim.x >> 5) ? warp_n[threadIdx.x] : 0u;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0 && v) atomicAdd(ctr, (unsigned long long)v);
  }
  __syncthreads();
}

// Level 0: code byte (active bits and ghost-face flags) from the int8 mask,
// and the active-cell count.  A warp takes one row (j, k) at a time, 32
// cells per round (no division per cell); the x-neighbours come from the
// adjacent lanes (the round's two edge cells load theirs), and only active
// cells load their y- and z-neighbours.
__global__ void build_fine_kernel(LevelDev L, const int8_t* __restrict__ mask, unsigned long long* counts2) {
  const Geom g = L.g;
  const unsigned rows = (unsigned)g.ny * (unsigned)g.nz;
  const int lane = threadIdx.x & 31;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  unsigned n_act = 0;
  for (unsigned row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nw) {
    const int k = (int)(row / (unsigned)g.ny);
    const int j = (int)(row - (unsigned)k * (unsigned)g.ny);
    const int8_t* __restrict__ m = mask + (long long)row * g.nx;
    // even i has colour (j + k) & 1
    uint8_t* const even = L.code[(j + k) & 1] + g.at(0, j, k);
    uint8_t* const odd = L.code[(j + k + 1) & 1] + g.at(0, j, k);
    const bool ylo = j > 0, yhi = j + 1 < g.ny, zlo = k > 0, zhi = k + 1 < g.nz;
    for (int i0 = 0; i0 < g.nx; i0 += 32) {
      const int i = i0 + lane;
      const bool in = i < g.nx;
      const int c = in ? (int)m[i] : 0;
      const bool act = c > 0;
      int xm = __shfl_up_sync(0xffffffffu, c, 1);
      int xp = __shfl_down_sync(0xffffffffu, c, 1);
      if (lane == 0) xm = i > 0 && in ? (int)m[i - 1] : 0;
      if (lane == 31) xp = i + 1 < g.nx ? (int)m[i + 1] : 0;
      uint8_t code = 0;
      if (act) {
        const bool nb[6] = {xm > 0, i + 1 < g.nx && xp > 0, ylo && m[i - sy] > 0, yhi && m[i + sy] > 0,
                            zlo && m[i - sz] > 0, zhi && m[i + sz] > 0};
        code = kActive2 | kActive1;
#pragma unroll
        for (int d = 0; d < 6; ++d)
          if (!nb[d]) code |= (uint8_t)(1u << (kGhostShift + d));
      }
      n_act += act;
      if (in) ((i & 1) ? odd : even)[i >> 1] = code;
    }
  }
  block_count_add(&counts2[0], n_act);
}

// K1: S_c = sum of the 8 children (missing children of an odd dimension are
// outside the box: -8^l each).  Level 0 children are read from the mask.
__global__ void mask_coarsen_kernel(Geom gf, int level_f, const int8_t* __restrict__ mask,
                                    const int32_t* __restrict__ Sf, Geom gc, int32_t* __restrict__ Sc) {
  const long long n = gc.ncells();
  const int out_val = -(int)pow8(level_f);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int I, J, K;
    natural_coords(idx, gc.nx, gc.ny, I, J, K);
    int sum = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
      if (i < gf.nx && j < gf.ny && k < gf.nz) {
        long long f = ((long long)k * gf.ny + j) * gf.nx + i;
        sum += mask ? (mask[f] > 0 ? 1 : -1) : Sf[f];
      } else {
        sum += out_val;
      }
    }
    Sc[idx] = sum;
  }
}

// K2 for a coarse level: active bits, D and 1/D of the second-order operator.
// D = sum over faces of 1 (active neighbour) or 1/theta = (S_i - S_j)/S_i
// (inactive or out-of-box neighbour, S_j = -8^l), computed exactly in integer
// form D = N / S_i, so 1/D = S_i / N and D = N / S_i each round once.
__global__ void coarse_coeffs_kernel(LevelDev L, unsigned long long* counts2) {
  const Geom g = L.g;
  const long long n = g.ncells();
  const long long p8 = pow8(L.level);
  unsigned n2 = 0, n1 = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    bool a2 = false, a1 = false;
    {
      int i, j, k;
      natural_coords(idx, g.nx, g.ny, i, j, k);
      const long long Si = L.S[idx];
      a2 = Si > 0;
      a1 = Si == p8;
      uint8_t code = (a2 ? kActive2 : 0) | (a1 ? kActive1 : 0);
      double invd = 0.0, diag = 0.0;
      if (a2) {
        const long long sy = g.nx, sz = (long long)g.nx * g.ny;
        long long Sj[6] = {i > 0 ? L.S[idx - 1] : -p8, i + 1 < g.nx ? L.S[idx + 1] : -p8,
                           j > 0 ? L.S[idx - sy] : -p8, j + 1 < g.ny ? L.S[idx + sy] : -p8,
                           k > 0 ? L.S[idx - sz] : -p8, k + 1 < g.nz ? L.S[idx + sz] : -p8};
        long long N = 0;
        for (int d = 0; d < 6; ++d) N += Sj[d] > 0 ? Si : Si - Sj[d];
        invd = (double)Si / (double)N;
        diag = (double)N / (double)Si;
      }
      const int c = colour_of(i, j, k);
      const long long at = g.at(i >> 1, j, k);
      L.code[c][at] = code;
      L.invd[c][at] = invd;
      L.diag[c][at] = diag;
      if (L.invd32[0]) {  // the mixed form's FP32 copies (round to nearest)
        L.invd32[c][at] = (float)invd;
        L.diag32[c][at] = (float)diag;
      }
    }
    n2 += a2;
    n1 += a1;
  }
  block_count_add(&counts2[0], n2);
  block_count_add(&counts2[1], n1);
}

__global__ void natural_to_split_kernel(Geom g, const double* __restrict__ nat, double* dst0, double* dst1,
                                        double scale, const uint8_t* code0, const uint8_t* code1,
                                        uint8_t mask_bit) {
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    const int c = colour_of(i, j, k);
    const long long at = g.at(i >> 1, j, k);
    bool keep = true;
    if (mask_bit) keep = ((c ? code1 : code0)[at] & mask_bit) != 0;
    (c ? dst1 : dst0)[at] = keep ? scale * nat[idx] : 0.0;
  }
}

// rho (natural layout) -> h^2 rho on the active cells (split layout) and the
// folded right-hand side b = h^2 rho - (boundary terms) in the same pass
// (bc null: the boundary terms are all zero).
__global__ void set_rhs_kernel(Geom g, const double* __restrict__ rho, double h2, const uint8_t* code0,
                               const uint8_t* code1, double* rh0, double* rh1, const double* __restrict__ bc0,
                               const double* __restrict__ bc1, double* b0, double* b1) {
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    const int c = colour_of(i, j, k);
    const long long at = g.at(i >> 1, j, k);
    const double v = ((c ? code1 : code0)[at] & kActive2) ? h2 * rho[idx] : 0.0;
    (c ? rh1 : rh0)[at] = v;
    (c ? b1 : b0)[at] = bc0 ? v - (c ? bc1 : bc0)[at] : v;
  }
}

__global__ void split_to_natural_kernel(Geom g, const double* __restrict__ s0, const double* __restrict__ s1,
                                        double* __restrict__ nat) {
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    nat[idx] = (colour_of(i, j, k) ? s1 : s0)[g.at(i >> 1, j, k)];
  }
}

__global__ void code_bits_to_natural_kernel(Geom g, const uint8_t* c0, const uint8_t* c1, int32_t* nat,
                                            uint8_t bit) {
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    nat[idx] = ((colour_of(i, j, k) ? c1 : c0)[g.at(i >> 1, j, k)] & bit) ? 1 : -1;
  }
}

// K3 (face form): bc = 2 * sum of Phi_b over the ghost faces of each active
// fine cell (theta = 1/2 at level 0, so Phi_b/theta = 2 Phi_b).
__global__ void fold_faces_kernel(LevelDev L, FineExtra F, const double* __restrict__ bx,
                                  const double* __restrict__ by, const double* __restrict__ bz) {
  const Geom g = L.g;
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    const int c = colour_of(i, j, k);
    const long long at = g.at(i >> 1, j, k);
    const uint8_t code = L.code[c][at];
    double acc = 0.0;
    if (code & kActive2) {
      const int gh = code >> kGhostShift;
      const long long fx = ((long long)k * g.ny + j) * (g.nx + 1) + i;
      const long long fy = ((long long)k * (g.ny + 1) + j) * g.nx + i;
      const long long fz = ((long long)k * g.ny + j) * g.nx + i;
      const long long nxy = (long long)g.nx * g.ny;
      if ((gh & 1) && bx) acc += bx[fx];
      if ((gh & 2) && bx) acc += bx[fx + 1];
      if ((gh & 4) && by) acc += by[fy];
      if ((gh & 8) && by) acc += by[fy + g.nx];
      if ((gh & 16) && bz) acc += bz[fz];
      if ((gh & 32) && bz) acc += bz[fz + nxy];
    }
    F.bc[c][at] = 2.0 * acc;
  }
}

// Trilinear interpolation of the coarse AMR potential at a point given in
// fine-cell units; coarse cell (I,J,K) is centred at o + 2I + 1.
__device__ __forceinline__ bool coarse_sample(const double* __restrict__ pc, int cnx, int cny, int cnz, int ox,
                                              int oy, int oz, double px, double py, double pz, double& out) {
  const double u = (px - ox) * 0.5 - 0.5, v = (py - oy) * 0.5 - 0.5, w = (pz - oz) * 0.5 - 0.5;
  const double fu = floor(u), fv = floor(v), fw = floor(w);
  const int I = (int)fu, J = (int)fv, K = (int)fw;
  if (I < 0 || J < 0 || K < 0 || I + 1 >= cnx || J + 1 >= cny || K + 1 >= cnz) return false;
  const double tu = u - fu, tv = v - fv, tw = w - fw;
  const long long sy = cnx, sz = (long long)cnx * cny;
  const double* p = pc + K * sz + (long long)J * sy + I;
  const double c00 = (1.0 - tu) * p[0] + tu * p[1];
  const double c10 = (1.0 - tu) * p[sy] + tu * p[sy + 1];
  const double c01 = (1.0 - tu) * p[sz] + tu * p[sz + 1];
  const double c11 = (1.0 - tu) * p[sz + sy] + tu * p[sz + sy + 1];
  const double c0 = (1.0 - tv) * c00 + tv * c10;
  const double c1 = (1.0 - tv) * c01 + tv * c11;
  out = (1.0 - tw) * c0 + tw * c1;
  return true;
}

// K7 + K3: Dirichlet values interpolated from the coarser AMR level at the
// centre of each ghost face, folded into bc.
__global__ void fold_coarse_kernel(LevelDev L, FineExtra F, const double* __restrict__ pc, int cnx, int cny,
                                   int cnz, int ox, int oy, int oz, int* err_flag) {
  const Geom g = L.g;
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    const int c = colour_of(i, j, k);
    const long long at = g.at(i >> 1, j, k);
    const uint8_t code = L.code[c][at];
    double acc = 0.0;
    if (code & kActive2) {
      const int gh = code >> kGhostShift;
      const double x = i + 0.5, y = j + 0.5, z = k + 0.5;
      const double fx[6] = {(double)i, (double)(i + 1), x, x, x, x};
      const double fy[6] = {y, y, (double)j, (double)(j + 1), y, y};
      const double fz[6] = {z, z, z, z, (double)k, (double)(k + 1)};
      for (int d = 0; d < 6; ++d) {
        if (!(gh & (1 << d))) continue;
        double v;
        if (coarse_sample(pc, cnx, cny, cnz, ox, oy, oz, fx[d], fy[d], fz[d], v))
          acc += v;
        else
          atomicExch(err_flag, 1);
      }
    }
    F.bc[c][at] = 2.0 * acc;
  }
}

// The same interpolated values as face arrays (mg_set_dirichlet's layout):
// each ghost face of an active cell gets the coarse potential sampled at its
// centre (a ghost face has one active cell, so one thread writes it); the
// arrays were zeroed before.
__global__ void faces_from_coarse_kernel(LevelDev L, const double* __restrict__ pc, int cnx, int cny, int cnz, int ox,
                                         int oy, int oz, double* __restrict__ bx, double* __restrict__ by,
                                         double* __restrict__ bz, int* err_flag) {
  const Geom g = L.g;
  const long long n = g.ncells();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    natural_coords(idx, g.nx, g.ny, i, j, k);
    const int c = colour_of(i, j, k);
    const uint8_t code = L.code[c][g.at(i >> 1, j, k)];
    if (!(code & kActive2)) continue;
    const int gh = code >> kGhostShift;
    if (!gh) continue;
    const double x = i + 0.5, y = j + 0.5, z = k + 0.5;
    const double fx[6] = {(double)i, (double)(i + 1), x, x, x, x};
    const double fy[6] = {y, y, (double)j, (double)(j + 1), y, y};
    const double fz[6] = {z, z, z, z, (double)k, (double)(k + 1)};
    const long long nx1 = g.nx + 1, ny1 = g.ny + 1;
    double* const dst[6] = {bx + ((long long)k * g.ny + j) * nx1 + i, bx + ((long long)k * g.ny + j) * nx1 + i + 1,
                            by + ((long long)k * ny1 + j) * g.nx + i, by + ((long long)k * ny1 + j + 1) * g.nx + i,
                            bz + ((long long)k * g.ny + j) * g.nx + i, bz + ((long long)(k + 1) * g.ny + j) * g.nx + i};
    for (int d = 0; d < 6; ++d) {
      if (!(gh & (1 << d))) continue;
      double v;
      if (coarse_sample(pc, cnx, cny, cnz, ox, oy, oz, fx[d], fy[d], fz[d], v)) *dst[d] = v;
      else atomicExch(err_flag, 1);
    }
  }
}

// b = h^2 rho - bc over whole colour arrays (halo and padding stay 0).
__global__ void combine_rhs_kernel(long long total, const double* __restrict__ r0, const double* __restrict__ r1,
                                   const double* __restrict__ b0, const double* __restrict__ b1, double* __restrict__ o0,
                                   double* __restrict__ o1) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    o0[e] = r0[e] - b0[e];
    o1[e] = r1[e] - b1[e];
  }
}

// Stream compaction of the active cells (or row segments) of one colour, in
// slot order (k, j, q), in three passes: per-block counts, one-block
// exclusive scan, per-block ordered writes.  A thread scans one 16-slot chunk
// of a row.
constexpr int kListThreads = 256;

// Chunk x of a list job: the 16 slots (q0 .. q0 + 15) of one row of one
// colour, x = row * chunks_per_row + q0 / 16, rows in (k, j) order.  Returns
// the membership bits of the chunk's candidates (bit c: cell q0 + c, or row
// segment c of 2^seg_shift slots, holds a slot whose code has `bit`), with the
// offset of slot q0 and the x-neighbour flag of the row.  Slots at q >= hx
// are masked off whatever the padding holds.
__device__ __forceinline__ unsigned list_chunk(const ListJob& J, unsigned x, long long& at0, uint32_t& flag) {
  const Geom& g = J.g;
  const unsigned per_row = (unsigned)(g.hx + (1 << kListChunkShift) - 1) >> kListChunkShift;
  const unsigned rows = (unsigned)g.ny * (unsigned)g.nz;
  if (x >= per_row * rows) return 0u;
  const unsigned row = x / per_row;
  const int q0 = (int)(x - row * per_row) << kListChunkShift;
  const int k = (int)(row / (unsigned)g.ny);
  const int j = (int)(row - (unsigned)k * (unsigned)g.ny);
  at0 = g.at(q0, j, k);
  flag = ((J.colour ^ j ^ k) & 1) ? kListPlusX : 0u;
  const uint4 w = *reinterpret_cast<const uint4*>(J.code + at0);
  const int p = J.bit == 1 ? 0 : (J.bit == 2 ? 1 : 31 - __clz((int)J.bit));
  const unsigned word[4] = {w.x, w.y, w.z, w.w};
  unsigned slots = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned y = (word[i] >> p) & 0x01010101u;  // byte b: 1 if slot 4i + b has the bit
    slots |= ((y & 1u) | ((y >> 7) & 2u) | ((y >> 14) & 4u) | ((y >> 21) & 8u)) << (4 * i);
  }
  const int nv = g.hx - q0;  // slots of this row in the chunk (>= 1)
  if (nv < 16) slots &= (1u << nv) - 1u;
  const int sh = J.seg_shift;
  if (sh == 0) return slots;
  unsigned m = 0;
  const int per = 1 << sh;
  for (int c = 0; c < (16 >> sh); ++c)
    if ((slots >> (c * per)) & ((1u << per) - 1u)) m |= 1u << c;
  return m;
}

// exclusive scan of nb block counts in place (one block of 1024 threads);
// the total goes to *count
__device__ void list_scan_block(uint32_t* block_counts, int nb, uint32_t* count) {
  __shared__ uint32_t part[1024];
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  uint32_t sum = 0;
  for (int b = b0; b < b1; ++b) sum += block_counts[b];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (int b = b0; b < b1; ++b) {
    const uint32_t c = block_counts[b];
    block_counts[b] = run;
    run += c;
  }
  if (threadIdx.x == 1023) *count = part[1023];
}

// All the lists of a hierarchy in three launches: the same three passes,
// with every block of a launch belonging to one list (a job) of the table.
// Job b0 is the first global block of the job; the scratch holds one count
// (then one offset) per global block.
__device__ int find_job(const ListJob* jobs, int njobs, unsigned b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kListThreads) list_count_all_kernel(const ListJob* __restrict__ jobs, int njobs,
                                                                      uint32_t* scratch) {
  __shared__ int js;
  __shared__ unsigned warp_n[kListThreads / 32];
  if (threadIdx.x == 0) js = find_job(jobs, njobs, blockIdx.x);
  __syncthreads();
  const ListJob& J = jobs[js];
  long long at0 = 0;
  uint32_t flag = 0;
  unsigned n = __popc(list_chunk(J, (blockIdx.x - J.block0) * kListThreads + threadIdx.x, at0, flag));
  for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(0xffffffffu, n, off);
  if ((threadIdx.x & 31) == 0) warp_n[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < kListThreads / 32; ++w) t += warp_n[w];
    scratch[blockIdx.x] = t;
  }
}

// one block per job: exclusive scan of the job's block counts in place; the
// job's total goes to *count
__global__ void __launch_bounds__(1024) list_scan_all_kernel(const ListJob* __restrict__ jobs, uint32_t* scratch) {
  const ListJob& J = jobs[blockIdx.x];
  list_scan_block(scratch + J.block0, (int)J.nblocks, J.count);
}

// The block's entries in slot order: each thread places its chunk's members
// at its exclusive prefix in shared memory, then the block writes them out
// contiguously from the block's offset in the list.
__global__ void __launch_bounds__(kListThreads) list_write_all_kernel(const ListJob* __restrict__ jobs, int njobs,
                                                                      const uint32_t* __restrict__ scratch) {
  __shared__ int js;
  __shared__ unsigned warp_base[kListThreads / 32 + 1];
  __shared__ uint32_t stage[kListThreads << kListChunkShift];
  if (threadIdx.x == 0) js = find_job(jobs, njobs, blockIdx.x);
  __syncthreads();
  const ListJob& J = jobs[js];
  long long at0 = 0;
  uint32_t flag = 0;
  unsigned m = list_chunk(J, (blockIdx.x - J.block0) * kListThreads + threadIdx.x, at0, flag);
  const unsigned cnt = __popc(m);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned incl = cnt;
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) warp_base[w] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int i = 0; i < kListThreads / 32; ++i) {
      const unsigned c = warp_base[i];
      warp_base[i] = run;
      run += c;
    }
    warp_base[kListThreads / 32] = run;
  }
  __syncthreads();
  unsigned pos = warp_base[w] + incl - cnt;
  const int sh = J.seg_shift;
  while (m) {
    const int c = __ffs((int)m) - 1;
    m &= m - 1u;
    stage[pos++] = (uint32_t)(at0 + (c << sh)) | flag;
  }
  __syncthreads();
  const unsigned total = warp_base[kListThreads / 32];
  uint32_t* out = J.list + scratch[blockIdx.x];
  for (unsigned i = threadIdx.x; i < total; i += kListThreads) out[i] = stage[i];
}

// Many device buffers zeroed in one launch: blockIdx.y selects the buffer.
__global__ void zero_many_kernel(const ZeroJob* __restrict__ jobs) {
  const ZeroJob J = jobs[blockIdx.y];
  unsigned long long* p = (unsigned long long*)J.ptr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < J.words; e += (long long)gridDim.x * blockDim.x)
    p[e] = 0ull;
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 32LL * device_sms()) b = 32LL * device_sms();
  return (int)b;
}

}  // namespace

cudaError_t launch_build_fine(const LevelDev& L0, const int8_t* mask, unsigned long long* counts2,
                              cudaStream_t s) {
  count_launch();
  build_fine_kernel<<<grid_for(L0.g.ncells()), kThreads, 0, s>>>(L0, mask, counts2);
  return cudaGetLastError();
}

cudaError_t launch_mask_coarsen(const LevelDev& Lf, const int8_t* mask_if_fine, const LevelDev& Lc,
                                cudaStream_t s) {
  count_launch();
  mask_coarsen_kernel<<<grid_for(Lc.g.ncells()), kThreads, 0, s>>>(Lf.g, Lf.level, mask_if_fine, Lf.S, Lc.g,
                                                                    Lc.S);
  return cudaGetLastError();
}

cudaError_t launch_coarse_coeffs(const LevelDev& Lc, unsigned long long* counts2, cudaStream_t s) {
  count_launch();
  coarse_coeffs_kernel<<<grid_for(Lc.g.ncells()), kThreads, 0, s>>>(Lc, counts2);
  return cudaGetLastError();
}

cudaError_t launch_build_lists(const ListJob* jobs, int njobs, unsigned total_blocks, uint32_t* scratch,
                               cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  count_launch(3);
  list_count_all_kernel<<<total_blocks, kListThreads, 0, s>>>(jobs, njobs, scratch);
  list_scan_all_kernel<<<njobs, 1024, 0, s>>>(jobs, scratch);
  list_write_all_kernel<<<total_blocks, kListThreads, 0, s>>>(jobs, njobs, scratch);
  return cudaGetLastError();
}

cudaError_t launch_zero_many(const ZeroJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  count_launch();
  zero_many_kernel<<<dim3(device_sms() * 2, njobs), 256, 0, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_natural_to_split(const Geom& g, const double* nat, double* dst0, double* dst1, double scale,
                                    uint8_t* const* code, uint8_t mask_bit, cudaStream_t s) {
  count_launch();
  natural_to_split_kernel<<<grid_for(g.ncells()), kThreads, 0, s>>>(g, nat, dst0, dst1, scale, code[0], code[1],
                                                                     mask_bit);
  return cudaGetLastError();
}

cudaError_t launch_set_rhs(const LevelDev& L0, const FineExtra& F, const double* rho, double h2, bool bc_zero,
                           cudaStream_t s) {
  count_launch();
  set_rhs_kernel<<<grid_for(L0.g.ncells()), kThreads, 0, s>>>(L0.g, rho, h2, L0.code[0], L0.code[1], F.rhoh2[0],
                                                               F.rhoh2[1], bc_zero ? nullptr : F.bc[0],
                                                               bc_zero ? nullptr : F.bc[1], L0.rhs[0], L0.rhs[1]);
  return cudaGetLastError();
}

cudaError_t launch_split_to_natural(const Geom& g, double* const* src, double* nat, cudaStream_t s) {
  count_launch();
  split_to_natural_kernel<<<grid_for(g.ncells()), kThreads, 0, s>>>(g, src[0], src[1], nat);
  return cudaGetLastError();
}

cudaError_t launch_u8_split_to_natural_bits(const Geom& g, uint8_t* const* code, int32_t* nat, uint8_t bit,
                                            cudaStream_t s) {
  count_launch();
  code_bits_to_natural_kernel<<<grid_for(g.ncells()), kThreads, 0, s>>>(g, code[0], code[1], nat, bit);
  return cudaGetLastError();
}

cudaError_t launch_fold_faces(const LevelDev& L0, const FineExtra& F, const double* bx, const double* by,
                              const double* bz, cudaStream_t s) {
  count_launch();
  fold_faces_kernel<<<grid_for(L0.g.ncells()), kThreads, 0, s>>>(L0, F, bx, by, bz);
  return cudaGetLastError();
}

cudaError_t launch_fold_coarse(const LevelDev& L0, const FineExtra& F, const double* pc, int cnx, int cny,
                               int cnz, int ox, int oy, int oz, int* err_flag, cudaStream_t s) {
  count_launch();
  fold_coarse_kernel<<<grid_for(L0.g.ncells()), kThreads, 0, s>>>(L0, F, pc, cnx, cny, cnz, ox, oy, oz,
                                                                   err_flag);
  return cudaGetLastError();
}

cudaError_t launch_faces_from_coarse(const LevelDev& L0, const double* pc, int cnx, int cny, int cnz, int ox, int oy,
                                    int oz, double* bx, double* by, double* bz, int* err_flag, cudaStream_t s) {
  count_launch();
  faces_from_coarse_kernel<<<grid_for(L0.g.ncells()), kThreads, 0, s>>>(L0, pc, cnx, cny, cnz, ox, oy, oz, bx, by, bz,
                                                                         err_flag);
  return cudaGetLastError();
}

cudaError_t launch_combine_rhs(const LevelDev& L0, const FineExtra& F, cudaStream_t s) {
  count_launch();
  combine_rhs_kernel<<<grid_for(L0.g.total), kThreads, 0, s>>>(L0.g.total, F.rhoh2[0], F.rhoh2[1], F.bc[0],
                                                                F.bc[1], L0.rhs[0], L0.rhs[1]);
  return cudaGetLastError();
}

}  // namespace gbmg
