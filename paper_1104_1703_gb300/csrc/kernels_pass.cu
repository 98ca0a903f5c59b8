// Temporal-blocked FP32 smoothing of the fine level (the mixed form's inner
// V-cycle): both red-black Gauss-Seidel sweeps of a pre- or post-smoothing
// step (Section 2 recipe, steps 1 and 8, with N_pre = N_post = 2) in one pass
// over the level, instead of four list half-sweeps that each read and write
// the whole level.
//
// Schedule.  The four half-sweeps are the stages S1 (red), S2 (black), S3
// (red), S4 (black).  A CTA owns a tile of TQ x TJ slots of the red/black
// split layout (mg_internal.h) and a z-segment of Z planes, and walks z with
// a wavefront: at step t it runs S1 on plane t+3, S2 on t+2, S3 on t+1 and
// S4 on t, in that order, each stage reading only values the previous stages
// left in shared memory.  A stage at plane p reads the other colour at planes
// p-1, p, p+1, which the wavefront has brought to exactly the state the
// sequential half-sweeps would see.  In x and y a stage reaches one slot (or
// row) into the other colour, so the stages run on rings of 3, 2, 1 and 0
// slots around the tile (S4 on the tile itself), and the same in z around the
// segment (the step loop starts six planes before it).  Neighbouring tiles
// compute the ring values themselves from the pass's input, so no CTA waits
// on another: the pass reads the correction from one buffer and writes the
// tile interiors to the other (the hierarchy keeps two FP32 copies of the
// fine correction and alternates them).  Every update is the list kernel's
// arithmetic in the list kernel's order, so the pass is bit-identical to
// four sequential half-sweeps.
//
// Red values before the pass are never read (S1 overwrites every red value
// from black neighbours), so a plane's loads are the black correction, the
// right-hand side of both colours and the cell codes of both colours.  Each
// is one TMA tile copy (cp.async.bulk.tensor) of the padded plane region into
// shared memory, completed on an mbarrier; the next plane's copies are issued
// two steps ahead.  Planes sit in rings of shared-memory slots (7 for the
// black correction, 6 for the right-hand side and codes, 5 for the red
// correction, which is never copied in).  One thread waits on each copy's
// mbarrier and the others wait at the block barrier after it, so that no
// warp spins on the copies.  The wait is bounded by time: a copy that has not
// landed after a second makes every thread of the CTA leave the pass, after
// thread 0 has waited (again bounded) for the CTA's copies in flight, with an
// error word set for the host.
//
// Only tiles with an active cell are walked (a list built with the mask).
// With the mixed form's last post-smoothing pass, the write-back also adds
// the final correction to Phi in FP64 (Phi += e).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "async_copy.cuh"
#include "cycle_device.cuh"
#include "pass_internal.h"

namespace gbmg {

namespace {

constexpr int kR = kPassHalo;                   // loaded halo: slots and rows around the tile
constexpr int kWQ = kPassTQ + 2 * kR;           // float region width (slots)
constexpr int kWJ = kPassTJ + 2 * kR;           // region height (rows)
constexpr int kWQC = kPassCodeWidth;            // code region width (bytes), x start aligned to 16
constexpr int kCodeShift = kPassCodeShift;      // code index of float region column 0
// Ring slots: a black plane's copy is issued two steps before S1 first reads
// it and the plane stays until its write-back (7 slots); right-hand side and
// codes likewise (6); red planes are written by S1 and read until S4 of the
// plane above (5).
constexpr int kAhead = 2;
constexpr int kRedSlots = 5;
constexpr int kPhiSlots = 5 + kAhead;
constexpr int kBcSlots = 4 + kAhead;
constexpr int kPlaneF = kWQ * kWJ;              // floats per plane region
constexpr int kPlaneC = kWQC * kWJ;             // code bytes per plane region
constexpr unsigned kPhiBytes = kPlaneF * 4;
constexpr unsigned kBcBytes = 2 * kPlaneF * 4 + 2 * kPlaneC;

struct __align__(128) PassSmem {
  float red[kRedSlots][kPlaneF];
  float black[kPhiSlots][kPlaneF];
  float b[kBcSlots][2][kPlaneF];
  uint8_t code[kBcSlots][2][kPlaneC];
  unsigned long long bar_phi[kPhiSlots];
  unsigned long long bar_bc[kBcSlots];
  unsigned long long bar_dbg;
  float tab[8];
  int abort;
};

// One stage of the wavefront: colour c's Gauss-Seidel update on one plane
// region, rows [J0, J1) and quads [Q0, Q1) of 4 slots (columns 4 Q .. 4 Q + 3).
// `om`, `o0`, `op` are the other colour's planes below, at and above; `self`
// is this colour's plane; b and code the plane's right-hand side and codes.
// A thread takes one quad of one row at a time: its 4 values of the other
// colour in the row, the rows above and below and the planes below and
// above are 128-bit shared loads, plus the two scalars on either side; the
// codes are one 32-bit load.  Every update is the list kernel's
//   ((o[q] + o[q + dx]) + (o[row - 1] + o[row + 1])) + (o[plane - 1] + o[plane + 1])
// then (s - b) * (1 / D), in the same order.  Each slot of the quad is written,
// 0 where the cell is inactive (those hold 0 anyway, and S1 thereby clears
// the stale red values of a reused slot).  A stage's quads span the whole
// region width (ring 4 in x), wider than its ring; the values it computes
// beyond its ring read stale or outside neighbours and are wrong, but each
// ring's values are read only by later stages inside their own, narrower
// rings, and S1 reads black values no later stage has touched, so no wrong
// value reaches the tile.
template <int J0, int J1, int Q0, int Q1>
__device__ __forceinline__ void stage(int c, int j_base, int k, const float* __restrict__ om,
                                      const float* __restrict__ o0, const float* __restrict__ op, float* self,
                                      const float* __restrict__ b, const uint8_t* __restrict__ code,
                                      const float* tab) {
  constexpr int NQ = Q1 - Q0;
  constexpr int N = (J1 - J0) * NQ;
  const int par = (c ^ j_base ^ k) & 1;  // row jj has dx = +1 iff (par ^ jj) & 1
  for (int t = threadIdx.x; t < N; t += kPassThreads) {
    const int jj = J0 + t / NQ;
    const int idx = jj * kWQ + 4 * (Q0 + t % NQ);
    const float4 v = *reinterpret_cast<const float4*>(o0 + idx);
    const float vl = o0[idx - 1], vr = o0[idx + 4];
    const float4 ym = *reinterpret_cast<const float4*>(o0 + idx - kWQ);
    const float4 yp = *reinterpret_cast<const float4*>(o0 + idx + kWQ);
    const float4 zm = *reinterpret_cast<const float4*>(om + idx);
    const float4 zp = *reinterpret_cast<const float4*>(op + idx);
    const float4 bb = *reinterpret_cast<const float4*>(b + idx);
    const unsigned cd = *reinterpret_cast<const unsigned*>(code + jj * kWQC + (idx - jj * kWQ) + kCodeShift);
    const bool plus = (par ^ jj) & 1;
    const float x0 = plus ? v.y : vl, x1 = plus ? v.z : v.x, x2 = plus ? v.w : v.y, x3 = plus ? vr : v.z;
    const float s0 = ((v.x + x0) + (ym.x + yp.x)) + (zm.x + zp.x);
    const float s1 = ((v.y + x1) + (ym.y + yp.y)) + (zm.y + zp.y);
    const float s2 = ((v.z + x2) + (ym.z + yp.z)) + (zm.z + zp.z);
    const float s3 = ((v.w + x3) + (ym.w + yp.w)) + (zm.w + zp.w);
    const unsigned c0 = cd & 0xffu, c1 = (cd >> 8) & 0xffu, c2 = (cd >> 16) & 0xffu, c3 = cd >> 24;
    float4 out;
    out.x = (c0 & kActive2) ? (s0 - bb.x) * tab[__popc(c0 >> kGhostShift)] : 0.0f;
    out.y = (c1 & kActive2) ? (s1 - bb.y) * tab[__popc(c1 >> kGhostShift)] : 0.0f;
    out.z = (c2 & kActive2) ? (s2 - bb.z) * tab[__popc(c2 >> kGhostShift)] : 0.0f;
    out.w = (c3 & kActive2) ? (s3 - bb.w) * tab[__popc(c3 >> kGhostShift)] : 0.0f;
    *reinterpret_cast<float4*>(self + idx) = out;
  }
}

}  // namespace

__global__ void __launch_bounds__(kPassThreads, 2)
    smooth_pass_kernel(const __grid_constant__ CUtensorMap map_black, const __grid_constant__ CUtensorMap map_b0,
                       const __grid_constant__ CUtensorMap map_b1, const __grid_constant__ CUtensorMap map_c0,
                       const __grid_constant__ CUtensorMap map_c1, PassArgs a) {
  pdl_wait();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PassSmem& S = *reinterpret_cast<PassSmem*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < kPhiSlots; ++i) mbar_init(&S.bar_phi[i], 1);
    for (int i = 0; i < kBcSlots; ++i) mbar_init(&S.bar_bc[i], 1);
    mbar_init(&S.bar_dbg, 1);
    S.abort = 0;
    mbar_init_fence();
  }
  if (tid < 8) S.tab[tid] = 1.0f / (float)(6 + tid);
  __syncthreads();
  const Geom g = a.g;
  const uint32_t ntiles = *a.ntiles;
  unsigned ph_phi = 0, ph_bc = 0;  // parity of each slot's next completion
  unsigned issued_phi = 0, issued_bc = 0;  // slots with a copy in flight (thread 0's view)
  constexpr unsigned long long kLimitNs = 1000000000ull;
  bool stall = a.debug_stall && blockIdx.x == 0;
  for (uint32_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const uint32_t code_t = a.tiles[ti];
    const int q0 = (int)(code_t & 1023u) * kPassTQ;
    const int j0 = (int)((code_t >> 10) & 1023u) * kPassTJ;
    const int k0 = (int)(code_t >> 20) * kPassZ;
    const int x0 = q0 - kR;             // float region: slots q0-4 .. q0+TQ+3
    const int xc = x0 - kCodeShift;     // code region: 16-byte aligned start
    const int y0 = j0 - kR + 1;         // tensor row of region row 0 (the padded layout's row -1 is row 0)
    const int pbase = k0 - kR;          // plane of relative index 0
    const int nsteps = kPassZ + 6;
    // copies: the black correction of plane r (relative), and the right-hand
    // side and codes of plane r (b/c slot (r-1) % 5, used from r = 1)
    auto issue_phi = [&](int r) {
      const int sl = r % kPhiSlots;
      fence_proxy_async();
      mbar_expect_tx(&S.bar_phi[sl], kPhiBytes);
      tma_load_3d(S.black[sl], &map_black, x0, y0, pbase + r + 1, &S.bar_phi[sl]);
      issued_phi |= 1u << sl;
    };
    auto issue_bc = [&](int r) {
      const int sl = (r - 1) % kBcSlots;
      fence_proxy_async();
      mbar_expect_tx(&S.bar_bc[sl], kBcBytes);
      tma_load_3d(S.b[sl][0], &map_b0, x0, y0, pbase + r + 1, &S.bar_bc[sl]);
      tma_load_3d(S.b[sl][1], &map_b1, x0, y0, pbase + r + 1, &S.bar_bc[sl]);
      tma_load_3d(S.code[sl][0], &map_c0, xc, y0, pbase + r + 1, &S.bar_bc[sl]);
      tma_load_3d(S.code[sl][1], &map_c1, xc, y0, pbase + r + 1, &S.bar_bc[sl]);
      issued_bc |= 1u << sl;
    };
    if (tid == 0) {
      for (int r = 0; r < 2 + kAhead; ++r) issue_phi(r);
      for (int r = 1; r < 1 + kAhead; ++r) issue_bc(r);
    }
    {
      // black planes 0 and 1 (plane 2 is waited for in step 0)
      if (tid == 0) {
        bool ok = true;
        for (int r = 0; r < 2 && ok; ++r) ok = stall || mbar_wait_bounded(&S.bar_phi[r], (ph_phi >> r) & 1u, kLimitNs);
        if (!ok) S.abort = 1;
        if (!stall) {
          ph_phi ^= 3u;
          issued_phi &= ~3u;
        }
      }
      __syncthreads();
      if (S.abort) goto abort;
    }
    for (int s = 0; s < nsteps; ++s) {
      // prefetch: black plane s+2+kAhead and the right-hand side and codes of
      // plane s+1+kAhead (S1 reads them kAhead steps from now)
      if (tid == 0) {
        if (s + 2 + kAhead < kPassZ + 8) issue_phi(s + 2 + kAhead);
        if (s + 1 + kAhead < kPassZ + 7) issue_bc(s + 1 + kAhead);
      }
      // wait (thread 0; the others at the barrier): black plane s+2 and the
      // right-hand side and codes of plane s+1, which S1 needs now
      if (tid == 0) {
        const int sp = (s + 2) % kPhiSlots, sb = s % kBcSlots;
        bool ok;
        if (stall) {
          ok = mbar_wait_bounded(&S.bar_dbg, 0, kLimitNs);  // never completes: the timeout path
        } else {
          ok = mbar_wait_bounded(&S.bar_phi[sp], (ph_phi >> sp) & 1u, kLimitNs) &&
               mbar_wait_bounded(&S.bar_bc[sb], (ph_bc >> sb) & 1u, kLimitNs);
        }
        if (!ok) {
          S.abort = 1;
        } else {
          ph_phi ^= 1u << sp;
          ph_bc ^= 1u << sb;
          issued_phi &= ~(1u << sp);
          issued_bc &= ~(1u << sb);
        }
      }
      __syncthreads();
      if (S.abort) goto abort;
      {
        // S1: red on plane r1 = s+1
        const int r1 = s + 1;
        stage<1, kWJ - 1, 0, kWQ / 4>(0, j0 - kR, pbase + r1, S.black[(r1 + kPhiSlots - 1) % kPhiSlots], S.black[r1 % kPhiSlots],
                       S.black[(r1 + 1) % kPhiSlots], S.red[r1 % kRedSlots], S.b[(r1 - 1) % kBcSlots][0],
                       S.code[(r1 - 1) % kBcSlots][0], S.tab);
        __syncthreads();
        if (s >= 2) {  // S2: black on plane s
          const int r2 = s;
          stage<2, kWJ - 2, 0, kWQ / 4>(1, j0 - kR, pbase + r2, S.red[(r2 + kRedSlots - 1) % kRedSlots], S.red[r2 % kRedSlots],
                          S.red[(r2 + 1) % kRedSlots], S.black[r2 % kPhiSlots], S.b[(r2 - 1) % kBcSlots][1],
                          S.code[(r2 - 1) % kBcSlots][1], S.tab);
        }
        __syncthreads();
        if (s >= 4) {  // S3: red on plane s-1
          const int r3 = s - 1;
          stage<3, kWJ - 3, 0, kWQ / 4>(0, j0 - kR, pbase + r3, S.black[(r3 + kPhiSlots - 1) % kPhiSlots],
                          S.black[r3 % kPhiSlots], S.black[(r3 + 1) % kPhiSlots], S.red[r3 % kRedSlots],
                          S.b[(r3 - 1) % kBcSlots][0], S.code[(r3 - 1) % kBcSlots][0], S.tab);
        }
        __syncthreads();
        if (s >= 6) {  // S4: black on plane s-2, then the plane's write-back
          const int r4 = s - 2;
          stage<4, kWJ - 4, 1, kWQ / 4 - 1>(1, j0 - kR, pbase + r4, S.red[(r4 + kRedSlots - 1) % kRedSlots], S.red[r4 % kRedSlots],
                          S.red[(r4 + 1) % kRedSlots], S.black[r4 % kPhiSlots], S.b[(r4 - 1) % kBcSlots][1],
                          S.code[(r4 - 1) % kBcSlots][1], S.tab);
          __syncthreads();
          const int k = pbase + r4;
          if (k < g.nz) {
            const float* src[2] = {S.red[r4 % kRedSlots], S.black[r4 % kPhiSlots]};
            const uint8_t* cds[2] = {S.code[(r4 - 1) % kBcSlots][0], S.code[(r4 - 1) % kBcSlots][1]};
            constexpr int NQ = kPassTQ / 4;
            for (int e = tid; e < 2 * kPassTJ * NQ; e += kPassThreads) {
              const int c = e / (kPassTJ * NQ);
              const int rem = e - c * (kPassTJ * NQ);
              const int jj = rem / NQ, qq = 4 * (rem - jj * NQ);
              const int q = q0 + qq, j = j0 + jj;
              // quads are 4-aligned and the pitch is a multiple of 16, so a
              // quad lies inside the row or wholly in its padding (whose
              // values are 0: nothing there is active)
              if (q >= g.P || j >= g.ny) continue;
              const int idx = (jj + kR) * kWQ + qq + kR;
              const long long at = g.at(q, j, k);
              const float4 v = *reinterpret_cast<const float4*>(src[c] + idx);
              *reinterpret_cast<float4*>(a.out[c] + at) = v;
              if (a.phi64[c]) {
                const unsigned cd = *reinterpret_cast<const unsigned*>(cds[c] + (jj + kR) * kWQC + qq + kR + kCodeShift);
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  if ((cd >> (8 * u)) & kActive2) a.phi64[c][at + u] += widen_f32(vv[u]);
              }
            }
          }
        }
        __syncthreads();
      }
    }
  }
  return;
abort:
  // leave the pass: record the error and wait (bounded) for this CTA's copies
  // still in flight, so that none lands in shared memory after the CTA exits
  if (tid == 0) {
    atomicExch(a.err, 1);
    for (int sl = 0; sl < kPhiSlots; ++sl)
      if (issued_phi & (1u << sl)) mbar_wait_bounded(&S.bar_phi[sl], (ph_phi >> sl) & 1u, kLimitNs);
    for (int sl = 0; sl < kBcSlots; ++sl)
      if (issued_bc & (1u << sl)) mbar_wait_bounded(&S.bar_bc[sl], (ph_bc >> sl) & 1u, kLimitNs);
  }
  __syncthreads();
}

// One flag per candidate tile: does its interior hold an active cell (either
// colour)?
__global__ void pass_tile_flags_kernel(Geom g, const uint8_t* __restrict__ c0, const uint8_t* __restrict__ c1,
                                       int nq, int nj, uint32_t* flags) {
  const int t = blockIdx.x;
  const int mq = t % nq, rest = t / nq, mj = rest % nj, mk = rest / nj;
  const int q0 = mq * kPassTQ, j0 = mj * kPassTJ, k0 = mk * kPassZ;
  int any = 0;
  for (int e = threadIdx.x; e < kPassTQ * kPassTJ * kPassZ; e += blockDim.x) {
    const int qq = e % kPassTQ, r = e / kPassTQ, jj = r % kPassTJ, kk = r / kPassTJ;
    const int q = q0 + qq, j = j0 + jj, k = k0 + kk;
    if (q >= g.hx || j >= g.ny || k >= g.nz) continue;
    const long long at = g.at(q, j, k);
    any |= (c0[at] | c1[at]) & kActive2;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) flags[t] = any ? 1u : 0u;
}

// Ordered compaction of the flags into the tile list (one CTA): entry =
// mq | mj << 10 | mk << 20, in candidate order (x fastest, then y, then z),
// so that CTAs running at the same time work on neighbouring tiles.
__global__ void __launch_bounds__(1024) pass_tile_list_kernel(const uint32_t* __restrict__ flags, int ncand, int nq,
                                                             int nj, uint32_t* tiles, uint32_t* count) {
  __shared__ uint32_t part[1024];
  const int per = (ncand + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(ncand, lo + per);
  uint32_t n = 0;
  for (int t = lo; t < hi; ++t) n += flags[t];
  part[threadIdx.x] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < 1024; ++i) {
      const uint32_t v = part[i];
      part[i] = acc;
      acc += v;
    }
    *count = acc;
  }
  __syncthreads();
  uint32_t o = part[threadIdx.x];
  for (int t = lo; t < hi; ++t)
    if (flags[t]) {
      const uint32_t mq = (uint32_t)(t % nq), r = (uint32_t)(t / nq), mj = r % (uint32_t)nj, mk = r / (uint32_t)nj;
      tiles[o++] = mq | (mj << 10) | (mk << 20);
    }
}

size_t pass_smem_bytes() { return sizeof(PassSmem); }

cudaError_t init_pass_kernel() {
  return cudaFuncSetAttribute(smooth_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PassSmem));
}

cudaError_t launch_pass_tiles(const Geom& g, uint8_t* const* code, uint32_t* flags, uint32_t* tiles, uint32_t* count,
                              cudaStream_t s) {
  int nq, nj, nk;
  pass_tile_grid(g, &nq, &nj, &nk);
  const int ncand = nq * nj * nk;
  count_launch(2);
  pass_tile_flags_kernel<<<ncand, 256, 0, s>>>(g, code[0], code[1], nq, nj, flags);
  pass_tile_list_kernel<<<1, 1024, 0, s>>>(flags, ncand, nq, nj, tiles, count);
  return cudaGetLastError();
}

cudaError_t launch_smooth_pass(const PassMaps& m, int input, const PassArgs& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * device_sms()));
  cfg.blockDim = dim3(kPassThreads);
  cfg.dynamicSmemBytes = sizeof(PassSmem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, smooth_pass_kernel, m.black[input], m.b[0], m.b[1], m.code[0], m.code[1], a);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool encode(CUtensorMap* map, const Geom& g, void* base, bool bytes) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t esz = bytes ? 1 : 4;
  const cuuint64_t dims[3] = {(cuuint64_t)g.P, (cuuint64_t)(g.ny + 2), (cuuint64_t)(g.nz + 2)};
  const cuuint64_t strides[2] = {(cuuint64_t)g.P * esz, (cuuint64_t)g.sz * esz};
  const cuuint32_t box[3] = {bytes ? (cuuint32_t)kWQC : (cuuint32_t)kWQ, (cuuint32_t)kWJ, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

bool make_pass_maps(PassMaps* m, const Geom& g, float* const* phi_a, float* const* phi_b, float* const* rhs,
                    uint8_t* const* code) {
  return encode(&m->black[0], g, phi_a[1], false) && encode(&m->black[1], g, phi_b[1], false) &&
         encode(&m->b[0], g, rhs[0], false) && encode(&m->b[1], g, rhs[1], false) &&
         encode(&m->code[0], g, code[0], true) && encode(&m->code[1], g, code[1], true);
}

}  // namespace gbmg
