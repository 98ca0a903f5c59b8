// Kernels of the learned initial guess's network: the 3x3x3 convolution as a
// tcgen05 implicit GEMM, and the packing of its weights.
//
// Convolution.  An output tile is 128 voxels (a box of bx x by x bz) by cout
// channels, accumulated in tensor memory (TMEM) in FP32 over K = 27 taps x
// cin input channels.  For each tap the input tile is the output tile's box
// shifted by the tap's offset: one TMA copy of a 5-D view of the
// channels-last input, (8 channels, x, y, z, channel chunk), lands it in
// shared memory as [chunk][voxel][8 channels], which is the canonical
// K-major layout of the MMA's A operand (8-row x 16-byte core matrices,
// 128 bytes apart along M and 2048 bytes apart along K).  Voxels outside the
// grid read 0 (the convolution's zero padding).  The weights of the tap come
// from a packed [27][cin / 8][cout][8] array by one bulk copy, in the same
// layout for the B operand.  Per 16 input channels one tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32, M = 128, N = cout) accumulates.
//
// Roles: warp 0's lane 0 issues the copies into a ring of 4 stages, warp 1
// allocates TMEM and its lane 0 issues the MMAs (each stage is released by a
// tcgen05.commit when its MMAs have read it), warps 2-5 read the two
// accumulator buffers back (tcgen05.ld, one TMEM lane quarter per warp),
// add the bias, apply ReLU and the optional mask, and store BF16.  Tiles are
// distributed over persistent CTAs; the two accumulators let the next tile's
// MMAs run while the last one drains.  Every wait is bounded by time and by a
// shared abort flag: a wait that runs out sets the error word, every role
// leaves its loop, the copy and MMA threads wait (bounded) for their
// operations in flight, and TMEM is released.
#include <cudaTypedefs.h>

#include "async_copy.cuh"
#include "mg_internal.h"
#include "unet_internal.h"

namespace gbmg {

namespace {

constexpr unsigned long long kConvLimitNs = 1000000000ull;

struct ConvSmemHeader {
  unsigned long long full[kConvStages];
  unsigned long long empty[kConvStages];
  unsigned long long accf[2];
  unsigned long long acce[2];
  uint32_t tmem;
  int abort;
  int consumed;  // units the MMA thread has waited for (the copies still in flight at an abort are after it)
};

__device__ __forceinline__ int conv_units(const ConvArgs& a) { return 27 * (a.cin / (8 * a.kc)); }

__global__ void __launch_bounds__(kConvThreads, 1)
    conv_kernel(const __grid_constant__ CUtensorMap map, ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  ConvSmemHeader& S = *reinterpret_cast<ConvSmemHeader*>(smem_raw);
  unsigned char* stage_a = smem_raw + 1024;
  const unsigned a_bytes = (unsigned)a.kc * 2048u;
  const unsigned b_bytes = (unsigned)a.kc * (unsigned)a.cout * 16u;
  unsigned char* stage_b = stage_a + kConvStages * a_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = a.ntx * a.nty * a.ntz;
  const int units = conv_units(a);
  const int upt = a.cin / (8 * a.kc);
  const uint32_t acc_cols = (uint32_t)a.cout;
  const uint32_t tcols = acc_cols * 2 <= 32 ? 32u : (acc_cols * 2 <= 64 ? 64u : (acc_cols * 2 <= 128 ? 128u : 256u));
  if (threadIdx.x == 0) {
    for (int i = 0; i < kConvStages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.accf[i], 1);
      mbar_init(&S.acce[i], 128);
    }
    S.abort = 0;
    S.consumed = 0;
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(&S.tmem, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  volatile int* abort = &S.abort;

  if (warp == 0) {
    if (lane == 0) {
      // ---- copies ----
      int it = 0;
      const bool stall = a.debug_stall && blockIdx.x == 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        const int tx = t % a.ntx, r = t / a.ntx, ty = r % a.nty, tz = r / a.nty;
        const int x0 = tx * a.bx, y0 = ty * a.by, z0 = tz * a.bz;
        for (int u = 0; u < units; ++u, ++it) {
          const int st = it % kConvStages, n = it / kConvStages;
          if (n > 0 && !mbar_wait_bounded(&S.empty[st], (n - 1) & 1, kConvLimitNs, abort)) {
            atomicExch(a.err, 1);
            *abort = 1;
            break;
          }
          if (stall && it >= kConvStages) {  // stop issuing: the MMA thread's wait runs out
            --it;
            break;
          }
          const int tap = u / upt, kq = u % upt;
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          fence_proxy_async();
          mbar_expect_tx(&S.full[st], a_bytes + b_bytes);
          tma_load_5d(stage_a + st * a_bytes, &map, 0, x0 + dx - 1, y0 + dy - 1, z0 + dz - 1, kq * a.kc, &S.full[st]);
          bulk_load(stage_b + st * b_bytes, a.w + ((size_t)tap * (a.cin / 8) + (size_t)kq * a.kc) * a.cout * 8, b_bytes,
                    &S.full[st]);
        }
        if (stall) break;
      }
      // at an abort, let the copies still in flight land before the CTA exits
      if (*abort) {
        __threadfence_block();
        for (int j = S.consumed; j < it; ++j)
          mbar_wait_bounded(&S.full[j % kConvStages], (j / kConvStages) & 1, kConvLimitNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMAs ----
      const uint32_t idesc = idesc_bf16_f32(kConvTileM, a.cout);
      int it = 0, tc = 0;
      bool issued = false;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++tc) {
        const int b = tc & 1, n = tc >> 1;
        if (n > 0 && !mbar_wait_bounded(&S.acce[b], (n - 1) & 1, kConvLimitNs, abort)) {
          atomicExch(a.err, 1);
          *abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)b * acc_cols;
        bool ok = true;
        for (int u = 0; u < units; ++u, ++it) {
          const int st = it % kConvStages;
          if (!mbar_wait_bounded(&S.full[st], (it / kConvStages) & 1, kConvLimitNs, abort)) {
            atomicExch(a.err, 1);
            *abort = 1;
            ok = false;
            break;
          }
          S.consumed = it + 1;
          tc_fence_after();
          const unsigned char* A = stage_a + st * a_bytes;
          const unsigned char* Bm = stage_b + st * b_bytes;
          for (int ks = 0; ks < a.kc / 2; ++ks) {
            const uint64_t ad = smem_desc_kmajor(A + ks * 2 * 2048, 2048, 128);
            const uint64_t bd = smem_desc_kmajor(Bm + ks * 2 * a.cout * 16, (uint32_t)a.cout * 16, 128);
            tc_mma_f16(d, ad, bd, idesc, (u > 0 || ks > 0) ? 1u : 0u);
          }
          tc_commit(&S.empty[st]);
          issued = true;
        }
        if (!ok) break;
        tc_commit(&S.accf[b]);
      }
      // at an abort, wait for the MMAs in flight before TMEM is released
      if (*abort && issued) {
        for (int j = (it > kConvStages ? it - kConvStages : 0); j < it; ++j)
          mbar_wait_bounded(&S.empty[j % kConvStages], (j / kConvStages) & 1, kConvLimitNs);
      }
    }
  } else {
    // ---- epilogue: warps 2..5 own TMEM lane quarters 2, 3, 0, 1 ----
    const int q = warp & 3;
    const int m = 32 * q + lane;
    const int mx = m % a.bx, my = (m / a.bx) % a.by, mz = m / (a.bx * a.by);
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
      const int b = tc & 1, n = tc >> 1;
      // lane 0 waits and the warp follows its verdict, so that the
      // warp-collective TMEM loads below run in every lane or in none
      int ok = 1;
      if (lane == 0) ok = mbar_wait_bounded(&S.accf[b], n & 1, kConvLimitNs, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          if (!*abort) atomicExch(a.err, 1);
          *abort = 1;
        }
        break;
      }
      __syncwarp();
      tc_fence_after();
      const int tx = t % a.ntx, r = t / a.ntx, ty = r % a.nty, tz = r / a.nty;
      const int x = tx * a.bx + mx, y = ty * a.by + my, z = tz * a.bz + mz;
      const bool in = x < a.W && y < a.H && z < a.D;
      const size_t v = ((size_t)z * a.H + y) * a.W + x;
      for (int c0 = 0; c0 < a.cout; c0 += 16) {
        float val[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * acc_cols + (uint32_t)c0, val);
        if (!in) continue;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float f = val[i];
          if (a.bias) f += a.bias[c0 + i];
          if (a.relu) f = fmaxf(f, 0.0f);
          val[i] = f;
        }
        if (a.mask) {
          const __nv_bfloat16* mk = a.mask + v * a.mask_stride + a.mask_off + c0;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (!(__bfloat162float(mk[i]) > 0.0f)) val[i] = 0.0f;
        }
        if (a.out_f32) {
          float* o = a.out_f32 + v * a.cout + c0;
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] = val[i];
        }
        __align__(16) __nv_bfloat16 h[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(val[i]);
        uint4* dst = reinterpret_cast<uint4*>(a.out + v * a.out_stride + a.out_off + c0);
        dst[0] = reinterpret_cast<const uint4*>(h)[0];
        dst[1] = reinterpret_cast<const uint4*>(h)[1];
      }
      tc_fence_before();
      mbar_arrive(&S.acce[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, tcols);
}

__global__ void pack_weights_kernel(const float* __restrict__ w, int cout, int cin, int cin_pad, int backward,
                                    __nv_bfloat16* __restrict__ out) {
  const long long n = 27LL * cout * cin_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    // forward: e enumerates [tap][cin_pad / 8][cout][8]
    // backward: [tap][cout / 8][cin_pad][8] (rows = forward input channels)
    const int j = (int)(e % 8);
    long long r = e / 8;
    int tap, kc, row;
    if (!backward) {
      row = (int)(r % cout);
      r /= cout;
      kc = (int)(r % (cin_pad / 8));
      tap = (int)(r / (cin_pad / 8));
      const int o = row, i = kc * 8 + j;
      out[e] = __float2bfloat16_rn(i < cin ? w[((size_t)o * cin + i) * 27 + tap] : 0.0f);
    } else {
      row = (int)(r % cin_pad);
      r /= cin_pad;
      kc = (int)(r % (cout / 8));
      tap = (int)(r / (cout / 8));
      const int i = row, o = kc * 8 + j;
      out[e] = __float2bfloat16_rn(i < cin ? w[((size_t)o * cin + i) * 27 + (26 - tap)] : 0.0f);
    }
  }
}

}  // namespace

int conv_kc(int cin) {
  const int chunks = cin / 8;
  for (int k = 8; k >= 2; k -= 2)
    if (chunks % k == 0) return k;
  return 2;
}

// The stages plus 32 KB of slack after them: every operand address the
// MMAs form stays inside the allocation even for a descriptor whose two
// core-matrix strides were read the other way round (at most 15 x 2048 +
// 255 bytes past an operand's start).
size_t conv_smem_bytes(int cin, int cout, int kc) {
  (void)cin;
  return 1024 + (size_t)kConvStages * ((size_t)kc * 2048 + (size_t)kc * cout * 16) + 32768;
}

uint32_t conv_tmem_cols(int cout) {
  const int c = 2 * cout;
  return c <= 32 ? 32u : (c <= 64 ? 64u : (c <= 128 ? 128u : 256u));
}

cudaError_t init_conv_kernel(size_t smem_bytes) {
  return cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

// The output tile's box: powers of two with bx * by * bz = 128 exactly (the
// copy of a tile must deliver the 128 rows the MMA and the barrier's byte
// count expect; rows beyond the grid read 0 and are not stored).
void conv_tile_box(int W, int H, int D, int* bx, int* by, int* bz) {
  auto pow2_at_most = [](int n, int cap) {
    int p = 1;
    while (2 * p <= n && 2 * p <= cap) p *= 2;
    return p;
  };
  *bx = pow2_at_most(W, 128);
  *by = pow2_at_most(H, 128 / *bx);
  *bz = 128 / (*bx * *by);
  (void)D;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 conv_encode_fn() {
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
}  // namespace

bool make_conv_input_map(CUtensorMap* map, const __nv_bfloat16* x, int W, int H, int D, int cin, int bx, int by,
                         int bz, int kc) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = conv_encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)(cin / 8)};
  const cuuint64_t strides[4] = {(cuuint64_t)cin * 2, (cuuint64_t)W * cin * 2, (cuuint64_t)H * W * cin * 2, 16};
  const cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)kc};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)x, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int conv_grid(const ConvArgs& a, size_t smem_bytes) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_kernel, kConvThreads, smem_bytes) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  const int by_tmem = (int)(512 / conv_tmem_cols(a.cout));
  if (per_sm > by_tmem) per_sm = by_tmem;
  const int tiles = a.ntx * a.nty * a.ntz;
  const int g = per_sm * device_sms();
  return tiles < g ? tiles : g;
}

cudaError_t launch_conv(const CUtensorMap& map, const ConvArgs& a, int grid, cudaStream_t s) {
  count_launch();
  conv_kernel<<<grid, kConvThreads, conv_smem_bytes(a.cin, a.cout, a.kc), s>>>(map, a);
  return cudaGetLastError();
}

cudaError_t launch_pack_weights(const float* w, int cout, int cin, int cin_pad, bool backward, __nv_bfloat16* out,
                                cudaStream_t s) {
  const long long n = 27LL * cout * cin_pad;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  pack_weights_kernel<<<(int)blocks, 256, 0, s>>>(w, cout, cin, cin_pad, backward ? 1 : 0, out);
  return cudaGetLastError();
}

}  // namespace gbmg

// ---------------------------------------------------------------------------
// Element-wise kernels of the network (channels-last BF16 tensors)
// ---------------------------------------------------------------------------

namespace gbmg {

namespace {

// x[c][z][y][x] (FP32, natural layout, c < 3) -> X0[v][16] BF16 (channels 3..15 zero)
__global__ void input_to_bf16_kernel(const float* __restrict__ x, long long V, __nv_bfloat16* __restrict__ out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = __float2bfloat16_rn(c < 3 ? x[c * V + v] : 0.0f);
    uint4* d = reinterpret_cast<uint4*>(out + v * 16);
    d[0] = reinterpret_cast<const uint4*>(h)[0];
    d[1] = reinterpret_cast<const uint4*>(h)[1];
  }
}

// 2x2x2 mean of src (level size 2W x 2H x 2D, channel stride ss, offset so)
// into dst (W x H x D, c channels, stride ds, offset do); one thread per
// output voxel and group of 8 channels
__global__ void avg_pool_kernel(const __nv_bfloat16* __restrict__ src, int ss, int so, int W, int H, int D, int c,
                                __nv_bfloat16* __restrict__ dst, int ds, int dofs) {
  const long long n = (long long)W * H * D * (c / 8);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(e % (c / 8));
    const long long v = e / (c / 8);
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((long long)W * H));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const long long vs = ((long long)(2 * z + dz) * (2 * H) + (2 * y + dy)) * (2 * W) + (2 * x + dx);
          const uint4 raw = *reinterpret_cast<const uint4*>(src + vs * ss + so + 8 * g);
          const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] += __bfloat162float(h[i]);
        }
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16_rn(acc[i] * 0.125f);
    *reinterpret_cast<uint4*>(dst + v * ds + dofs + 8 * g) = *reinterpret_cast<const uint4*>(o);
  }
}

// nearest-neighbour upsampling by 2 of src (W x H x D, c channels, stride ss,
// offset so) into dst (2W x 2H x 2D, stride ds, offset do)
__global__ void upsample_kernel(const __nv_bfloat16* __restrict__ src, int ss, int so, int W, int H, int D, int c,
                                __nv_bfloat16* __restrict__ dst, int ds, int dofs) {
  const long long n = 8LL * W * H * D * (c / 8);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(e % (c / 8));
    const long long v = e / (c / 8);
    const int X = 2 * W, Y = 2 * H;
    const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((long long)X * Y));
    const long long vs = ((long long)(z >> 1) * H + (y >> 1)) * W + (x >> 1);
    *reinterpret_cast<uint4*>(dst + v * ds + dofs + 8 * g) = *reinterpret_cast<const uint4*>(src + vs * ss + so + 8 * g);
  }
}

// the head: pred[v] = (b + sum_i w[i] u[v][i]) * (active ? 1 : 0), FP32;
// active from the input's mask channel (channel 1 of X0 > 0)
__global__ void head_kernel(const __nv_bfloat16* __restrict__ u, int c, const float* __restrict__ w,
                            const float* __restrict__ b, const __nv_bfloat16* __restrict__ x0, long long V,
                            float* __restrict__ pred) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    float acc = b[0];
    for (int i = 0; i < c; ++i) acc = fmaf(w[i], __bfloat162float(u[v * c + i]), acc);
    pred[v] = __bfloat162float(x0[v * 16 + 1]) > 0.0f ? acc : 0.0f;
  }
}

// channels [off, off + c) of a channels-last tensor -> FP32 natural [c][V]
__global__ void tensor_to_natural_kernel(const __nv_bfloat16* __restrict__ t, int stride, int off, int c, long long V,
                                         float* __restrict__ out) {
  const long long n = (long long)c * V;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(e / V);
    const long long v = e - (long long)ch * V;
    out[e] = __bfloat162float(t[v * stride + off + ch]);
  }
}

int ew_grid(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 32LL * device_sms();
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_input_to_bf16(const float* x, long long V, __nv_bfloat16* out, cudaStream_t s) {
  count_launch();
  input_to_bf16_kernel<<<ew_grid(V), 256, 0, s>>>(x, V, out);
  return cudaGetLastError();
}

cudaError_t launch_avg_pool(const __nv_bfloat16* src, int ss, int so, int W, int H, int D, int c, __nv_bfloat16* dst,
                            int ds, int dofs, cudaStream_t s) {
  count_launch();
  avg_pool_kernel<<<ew_grid((long long)W * H * D * (c / 8)), 256, 0, s>>>(src, ss, so, W, H, D, c, dst, ds, dofs);
  return cudaGetLastError();
}

cudaError_t launch_upsample(const __nv_bfloat16* src, int ss, int so, int W, int H, int D, int c, __nv_bfloat16* dst,
                            int ds, int dofs, cudaStream_t s) {
  count_launch();
  upsample_kernel<<<ew_grid(8LL * W * H * D * (c / 8)), 256, 0, s>>>(src, ss, so, W, H, D, c, dst, ds, dofs);
  return cudaGetLastError();
}

cudaError_t launch_head(const __nv_bfloat16* u, int c, const float* w, const float* b, const __nv_bfloat16* x0,
                        long long V, float* pred, cudaStream_t s) {
  count_launch();
  head_kernel<<<ew_grid(V), 256, 0, s>>>(u, c, w, b, x0, V, pred);
  return cudaGetLastError();
}

cudaError_t launch_tensor_to_natural(const __nv_bfloat16* t, int stride, int off, int c, long long V, float* out,
                                     cudaStream_t s) {
  count_launch();
  tensor_to_natural_kernel<<<ew_grid((long long)c * V), 256, 0, s>>>(t, stride, off, c, V, out);
  return cudaGetLastError();
}

}  // namespace gbmg
