// Kernels of the learned initial guess's network: the 3x3x3 convolution as a
// tcgen05 implicit GEMM, its weight gradients, and the packing of weights.
//
// Convolution.  An output tile is 128 voxels (a box of bx x by x bz) by cout
// channels, accumulated in tensor memory (TMEM) in FP32 over K = 27 taps x
// cin input channels.  Per 16 input channels one tcgen05.mma (kind::f16,
// BF16 x BF16 -> FP32, M = 128, N = cout) accumulates.  The A operand comes
// from the channels-last input by TMA copies of a 5-D view of it,
// (8 channels, x, y, z, channel chunk), landing in shared memory in the
// canonical K-major layout (8-row x 16-byte core matrices); voxels outside
// the grid read 0 (the convolution's zero padding).  Two ways to stage it:
//  - halo rows (a tile that is one whole row of 128 voxels): one copy per 16
//    input channels of the box (130 x 3 x 3) around the row; each of the 27
//    taps is then a view of it, offset by (dz * 3 + dy) * 130 + dx rows, so
//    the input is read once instead of 27 times;
//  - tap tiles (other shapes): one copy per tap and channel chunk of the
//    tile's box shifted by the tap.
// The B operand (the weights, packed [27][cin / 8][cout][8]) stays resident
// in shared memory for the whole launch when it fits (up to 72 KB), loaded
// once per CTA by one bulk copy; otherwise it is staged with each tap.  The
// pipeline depth is as many stages as fit in the shared-memory budget.
//
// Roles: warp 0's lane 0 issues the copies into the ring of stages, warp 1
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
  unsigned long long full[kConvMaxStages];
  unsigned long long empty[kConvMaxStages];
  unsigned long long accf[2];
  unsigned long long acce[2];
  unsigned long long wbar;
  uint32_t tmem;
  int abort;
  int consumed;  // units the MMA thread has waited for (the copies still in flight at an abort are after it)
};

}  // namespace

// Shared-memory layout of one convolution launch: per pipeline unit the
// input bytes (a halo row box of 16 channels, or one tap's tile of kc
// chunks) and the weight bytes staged with it (0 when the layer's weights
// are resident: w_bytes, loaded once per CTA).
__host__ __device__ ConvLayout conv_layout(const ConvArgs& a) {
  ConvLayout l;
  const unsigned wall = 27u * (unsigned)a.cin * (unsigned)a.cout * 2u;
  l.w_load = a.wres ? wall : 0u;
  l.w_bytes = a.wres ? (wall + 1023u) / 1024u * 1024u : 0u;
  if (a.halo) {
    l.a_bytes = 2u * 9u * 130u * 16u;
    l.b_bytes = 0;
    l.units = a.cin / 16;
  } else {
    l.a_bytes = (unsigned)a.kc * 2048u;
    l.b_bytes = a.wres ? 0u : (unsigned)a.kc * (unsigned)a.cout * 16u;
    l.units = 27 * (a.cin / (8 * a.kc));
  }
  // a TMA copy's shared-memory destination must be 128-byte aligned: the
  // stages are laid out at a stride rounded up to 128 bytes (the weight
  // stages' size, a multiple of 256, already is)
  l.a_stride = (l.a_bytes + 127u) / 128u * 128u;
  return l;
}

size_t conv_smem_bytes(const ConvArgs& a) {
  const ConvLayout l = conv_layout(a);
  return 1024 + (size_t)l.w_bytes + (size_t)a.stages * (l.a_stride + l.b_bytes);
}

// Pipeline depth, resident weights and the halo path of a convolution: a
// tile that is one full row of 128 voxels takes its input once with a halo
// (box 130 x 3 x 3, every tap a view of it; this needs the weights
// resident); weights up to 72 KB stay resident; as many stages as fit in
// about 110 KB (two CTAs per multiprocessor) or, for halo stages, 220 KB.
void conv_plan(ConvArgs& a) {
  const unsigned wall = 27u * (unsigned)a.cin * (unsigned)a.cout * 2u;
  a.wres = wall <= 72u * 1024u ? 1 : 0;
  a.halo = (a.bx == 128 && a.wres) ? 1 : 0;
  a.stages = 1;
  const ConvLayout l = conv_layout(a);
  const size_t per = l.a_stride + l.b_bytes;
  const size_t budget = per > 12 * 1024 ? 220 * 1024 : 110 * 1024;
  long long n = ((long long)budget - 1024 - (long long)l.w_bytes) / (long long)per;
  if (n > kConvMaxStages) n = kConvMaxStages;
  if (n < 2) n = 2;
  a.stages = (int)n;
}

// TMEM columns of a convolution CTA: two FP32 accumulators of cout columns,
// rounded up to the power of two the allocator takes.
__host__ __device__ uint32_t conv_tmem_cols(int cout) {
  const int c = 2 * cout;
  return c <= 32 ? 32u : (c <= 64 ? 64u : (c <= 128 ? 128u : (c <= 256 ? 256u : 512u)));
}

namespace {

__global__ void __launch_bounds__(kConvThreads, 1)
    conv_kernel(const __grid_constant__ CUtensorMap map, ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  ConvSmemHeader& S = *reinterpret_cast<ConvSmemHeader*>(smem_raw);
  const ConvLayout lay = conv_layout(a);
  unsigned char* wres = smem_raw + 1024;  // resident weights (when lay.w_bytes > 0)
  unsigned char* stage_a = wres + lay.w_bytes;
  unsigned char* stage_b = stage_a + a.stages * lay.a_stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = a.ntx * a.nty * a.ntz;
  const int units = lay.units;
  const int upt = a.cin / (8 * a.kc);
  const int NS = a.stages;
  const uint32_t acc_cols = (uint32_t)a.cout;
  const uint32_t tcols = conv_tmem_cols(a.cout);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.accf[i], 1);
      mbar_init(&S.acce[i], 128);
    }
    mbar_init(&S.wbar, 1);
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
      if (lay.w_bytes) {  // the whole layer's weights, once per CTA
        mbar_expect_tx(&S.wbar, lay.w_load);
        bulk_load(wres, a.w, lay.w_load, &S.wbar);
      }
      int it = 0;
      const bool stall = a.debug_stall && blockIdx.x == 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        const int tx = t % a.ntx, r = t / a.ntx, ty = r % a.nty, tz = r / a.nty;
        const int x0 = tx * a.bx, y0 = ty * a.by, z0 = tz * a.bz;
        for (int u = 0; u < units; ++u, ++it) {
          const int st = it % NS, n = it / NS;
          if (n > 0 && !mbar_wait_bounded(&S.empty[st], (n - 1) & 1, kConvLimitNs, abort)) {
            atomicExch(a.err, 1);
            *abort = 1;
            break;
          }
          if (stall && it >= NS) {  // stop issuing: the MMA thread's wait runs out
            --it;
            break;
          }
          fence_proxy_async();
          mbar_expect_tx(&S.full[st], lay.a_bytes + lay.b_bytes);
          if (a.halo) {
            // the row of 128 output voxels with a one-voxel halo in x, y and
            // z, 16 input channels: every tap is a view of it
            tma_load_5d(stage_a + st * lay.a_stride, &map, 0, x0 - 1, y0 - 1, z0 - 1, 2 * u, &S.full[st]);
          } else {
            const int tap = u / upt, kq = u % upt;
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            tma_load_5d(stage_a + st * lay.a_stride, &map, 0, x0 + dx - 1, y0 + dy - 1, z0 + dz - 1, kq * a.kc,
                        &S.full[st]);
            if (lay.b_bytes)
              bulk_load(stage_b + st * lay.b_bytes,
                        a.w + ((size_t)tap * (a.cin / 8) + (size_t)kq * a.kc) * a.cout * 8, lay.b_bytes, &S.full[st]);
          }
        }
        if (stall) break;
      }
      // at an abort, let the copies still in flight land before the CTA exits
      if (*abort) {
        __threadfence_block();
        for (int j = S.consumed; j < it; ++j) mbar_wait_bounded(&S.full[j % NS], (j / NS) & 1, kConvLimitNs);
        if (lay.w_bytes) mbar_wait_bounded(&S.wbar, 0, kConvLimitNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMAs ----
      const uint32_t idesc = idesc_bf16_f32(kConvTileM, a.cout);
      const uint32_t wchunk = (uint32_t)a.cout * 16u;  // bytes of one 8-channel chunk of one tap's weights
      int it = 0, tc = 0;
      bool issued = false;
      if (lay.w_bytes && !mbar_wait_bounded(&S.wbar, 0, kConvLimitNs, abort)) {
        atomicExch(a.err, 1);
        *abort = 1;
      }
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
          const int st = it % NS;
          if (!mbar_wait_bounded(&S.full[st], (it / NS) & 1, kConvLimitNs, abort)) {
            atomicExch(a.err, 1);
            *abort = 1;
            ok = false;
            break;
          }
          S.consumed = it + 1;
          tc_fence_after();
          const unsigned char* A = stage_a + st * lay.a_stride;
          if (a.halo) {
            // channels 16u .. 16u + 15 of the 27 taps: each tap's 128 rows
            // start (dz, dy, dx) rows into the halo box; the box's rows are
            // 16 bytes apart and its two 8-channel chunks 9 x 130 rows apart
            for (int tap = 0; tap < 27; ++tap) {
              const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
              const uint64_t ad = smem_desc_kmajor(A + ((dz * 3 + dy) * 130 + dx) * 16, 9u * 130u * 16u, 128);
              const uint64_t bd = smem_desc_kmajor(wres + ((size_t)tap * (a.cin / 8) + 2 * u) * wchunk, wchunk, 128);
              tc_mma_f16(d, ad, bd, idesc, (u > 0 || tap > 0) ? 1u : 0u);
            }
          } else {
            const int tap = u / upt, kq = u % upt;
            const unsigned char* Bm = lay.w_bytes ? wres + ((size_t)tap * (a.cin / 8) + (size_t)kq * a.kc) * wchunk
                                                  : stage_b + st * lay.b_bytes;
            for (int ks = 0; ks < a.kc / 2; ++ks) {
              const uint64_t ad = smem_desc_kmajor(A + ks * 2 * 2048, 2048, 128);
              const uint64_t bd = smem_desc_kmajor(Bm + ks * 2 * wchunk, wchunk, 128);
              tc_mma_f16(d, ad, bd, idesc, (u > 0 || ks > 0) ? 1u : 0u);
            }
          }
          tc_commit(&S.empty[st]);
          issued = true;
        }
        if (!ok) break;
        tc_commit(&S.accf[b]);
      }
      // at an abort, wait for the MMAs in flight before TMEM is released
      if (*abort && issued) {
        for (int j = (it > NS ? it - NS : 0); j < it; ++j)
          mbar_wait_bounded(&S.empty[j % NS], (j / NS) & 1, kConvLimitNs);
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
  conv_kernel<<<grid, kConvThreads, conv_smem_bytes(a), s>>>(map, a);
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

// ---------------------------------------------------------------------------
// Backward pass: weight gradients on the tensor cores, and the element-wise
// and reduction kernels
// ---------------------------------------------------------------------------
//
// Weight gradient of a convolution: dW[o][i][tap] = sum over voxels v of
// g[v][o] x[v + offset(tap)][i], with g the gradient of the pre-activation
// and x the layer's input (zero outside the grid).  As a GEMM: rows (tap, i)
// of the tap-major row space (27 x cin rows), columns o, K = the voxels.  A
// CTA takes 128 rows and a range of voxel tiles: per tile, the 16 channel
// octets of its rows are 16 TMA copies of the input tile shifted by each
// octet's tap (box 8 channels x the tile), landing as [octet][voxel][8],
// and g's tile is one copy, [o-octet][voxel][8]; both are the canonical
// MN-major layout (8 voxels x 8 channels per 128-byte core matrix, 128 bytes
// apart along K = voxels, 2048 bytes apart along M or N), so the MMA reads
// them as they land.  The 128 x cout FP32 accumulator stays in TMEM over the
// CTA's voxel range and is written once as the CTA's partial sum; a second
// kernel adds the partials in a fixed order.

namespace gbmg {

namespace {

constexpr int kWgStages = 3;

struct WgSmemHeader {
  unsigned long long full[kWgStages];
  unsigned long long empty[kWgStages];
  unsigned long long accf;
  uint32_t tmem;
  int abort;
  int consumed;
};

__global__ void __launch_bounds__(kConvThreads, 1)
    wgrad_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_g, WgradArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WgSmemHeader& S = *reinterpret_cast<WgSmemHeader*>(smem_raw);
  const unsigned a_bytes = 16u * 2048u;
  const unsigned b_bytes = (unsigned)a.cout * 256u;
  unsigned char* stage_a = smem_raw + 1024;
  unsigned char* stage_b = stage_a + kWgStages * a_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mb = blockIdx.x % a.nmblk, sp = blockIdx.x / a.nmblk;
  const int T = a.ntx * a.nty * a.ntz;
  const int t_lo = (int)((long long)T * sp / a.nsplit), t_hi = (int)((long long)T * (sp + 1) / a.nsplit);
  const uint32_t tcols = a.cout <= 32 ? 32u : (a.cout <= 64 ? 64u : 128u);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kWgStages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    mbar_init(&S.accf, 1);
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
  const int octets = a.cin / 8;
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int t = t_lo; t < t_hi; ++t, ++it) {
        const int st = it % kWgStages, n = it / kWgStages;
        if (n > 0 && !mbar_wait_bounded(&S.empty[st], (n - 1) & 1, kConvLimitNs, abort)) {
          atomicExch(a.err, 1);
          *abort = 1;
          break;
        }
        const int tx = t % a.ntx, r = t / a.ntx, ty = r % a.nty, tz = r / a.nty;
        const int x0 = tx * a.bx, y0 = ty * a.by, z0 = tz * a.bz;
        fence_proxy_async();
        mbar_expect_tx(&S.full[st], a_bytes + b_bytes);
        for (int g = 0; g < 16; ++g) {
          int R = mb * 16 + g;  // row octet in the tap-major row space
          if (R >= 27 * octets) R = 27 * octets - 1;  // padding rows: any valid octet (their sums are not used)
          const int tap = R / octets, ic = R % octets;
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          tma_load_5d(stage_a + st * a_bytes + g * 2048, &map_x, 0, x0 + dx - 1, y0 + dy - 1, z0 + dz - 1, ic,
                      &S.full[st]);
        }
        tma_load_5d(stage_b + st * b_bytes, &map_g, 0, x0, y0, z0, 0, &S.full[st]);
      }
      if (*abort) {
        for (int j = S.consumed; j < it; ++j) mbar_wait_bounded(&S.full[j % kWgStages], (j / kWgStages) & 1, kConvLimitNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(kConvTileM, a.cout, true);
      int it = 0;
      bool issued = false;
      for (int t = t_lo; t < t_hi && !*abort; ++t, ++it) {
        const int st = it % kWgStages;
        if (!mbar_wait_bounded(&S.full[st], (it / kWgStages) & 1, kConvLimitNs, abort)) {
          atomicExch(a.err, 1);
          *abort = 1;
          break;
        }
        S.consumed = it + 1;
        tc_fence_after();
        const unsigned char* A = stage_a + st * a_bytes;
        const unsigned char* Bm = stage_b + st * b_bytes;
        for (int ks = 0; ks < 8; ++ks) {
          const uint64_t ad = smem_desc_mnmajor(A + ks * 256, 128, 2048);
          const uint64_t bd = smem_desc_mnmajor(Bm + ks * 256, 128, 2048);
          tc_mma_f16(tmem, ad, bd, idesc, (t > t_lo || ks > 0) ? 1u : 0u);
        }
        tc_commit(&S.empty[st]);
        issued = true;
      }
      if (!*abort) tc_commit(&S.accf);
      else if (issued)
        for (int j = (it > kWgStages ? it - kWgStages : 0); j < it; ++j)
          mbar_wait_bounded(&S.empty[j % kWgStages], (j / kWgStages) & 1, kConvLimitNs);
    }
  } else {
    const int q = warp & 3;
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(&S.accf, 0, kConvLimitNs, abort) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      __syncwarp();
      tc_fence_after();
      const int row = mb * 128 + 32 * q + lane;
      float* dst = a.partial + ((size_t)sp * a.nmblk * 128 + row) * a.cout;
      for (int c0 = 0; c0 < a.cout; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[c0 + i] = v[i];
      }
    } else if (lane == 0) {
      if (!*abort) atomicExch(a.err, 1);
      *abort = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, tcols);
}

// dW[o][i][tap] (+)= sum over splits of partial[split][tap * cin_pad + i][o],
// in split order; i < cin (the real input channels).
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int nsplit, int rows, int cin_pad, int cin,
                                    int cout, float* __restrict__ dw) {
  const long long n = (long long)cout * cin * 27;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int tap = (int)(e % 27);
    const long long r = e / 27;
    const int i = (int)(r % cin), o = (int)(r / cin);
    const size_t row = (size_t)tap * cin_pad + i;
    float acc = 0.0f;
    for (int s = 0; s < nsplit; ++s) acc += partial[((size_t)s * rows + row) * cout + o];
    dw[e] = acc;
  }
}

// Per-block partial sums over voxels of g[v][o] (bias gradient), one row of
// partials per block; then a fixed-order reduction.
__global__ void channel_sum_kernel(const __nv_bfloat16* __restrict__ g, int c, long long V, float* __restrict__ part) {
  extern __shared__ float sh[];
  for (int o = threadIdx.x; o < c; o += blockDim.x) sh[o] = 0.0f;
  __syncthreads();
  const long long per = (V + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(V, lo + per);
  // each thread owns one channel and a stride of voxels
  const int lanes = blockDim.x / c;
  const int o = threadIdx.x % c, l = threadIdx.x / c;
  float acc = 0.0f;
  if (l < lanes)
    for (long long v = lo + l; v < hi; v += lanes) acc += __bfloat162float(g[v * c + o]);
  if (l < lanes) atomicAdd(&sh[o], acc);  // within the block only
  __syncthreads();
  for (int k = threadIdx.x; k < c; k += blockDim.x) part[(size_t)blockIdx.x * c + k] = sh[k];
}

__global__ void partial_rows_sum_kernel(const float* __restrict__ part, int nrows, int c, float* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int r = 0; r < nrows; ++r) acc += part[(size_t)r * c + k];
    out[k] = acc;
  }
}

// Head backward.  g_pred (FP32, dL/dpred), act = input channel 1 > 0:
// gz[v][i] = (top[v][i] > 0) w[i] g act (BF16), and per-block partial sums
// of g act top[v][i] (head weights) and g act (head bias).
__global__ void head_backward_kernel(const float* __restrict__ gp, const __nv_bfloat16* __restrict__ x0,
                                     const __nv_bfloat16* __restrict__ top, int c, const float* __restrict__ w,
                                     long long V, __nv_bfloat16* __restrict__ gz, float* __restrict__ part) {
  extern __shared__ float sh[];  // [c + 1]
  for (int k = threadIdx.x; k <= c; k += blockDim.x) sh[k] = 0.0f;
  __syncthreads();
  float acc_b = 0.0f;
  float acc_w[64];
  for (int i = 0; i < c && i < 64; ++i) acc_w[i] = 0.0f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const float g = __bfloat162float(x0[v * 16 + 1]) > 0.0f ? gp[v] : 0.0f;
    acc_b += g;
    for (int i = 0; i < c; ++i) {
      const float t = __bfloat162float(top[v * c + i]);
      acc_w[i] += g * t;
      gz[v * c + i] = __float2bfloat16_rn(t > 0.0f ? w[i] * g : 0.0f);
    }
  }
  for (int i = 0; i < c; ++i) atomicAdd(&sh[i], acc_w[i]);
  atomicAdd(&sh[c], acc_b);
  __syncthreads();
  for (int k = threadIdx.x; k <= c; k += blockDim.x) part[(size_t)blockIdx.x * (c + 1) + k] = sh[k];
}

// Gradient through nearest upsampling: dst[v][i] = sum over the 8 children of
// src[child][so + i] (src at twice the size), FP32 sum rounded to BF16.
__global__ void upsample_backward_kernel(const __nv_bfloat16* __restrict__ src, int ss, int so, int W, int H, int D,
                                         int c, __nv_bfloat16* __restrict__ dst) {
  const long long n = (long long)W * H * D * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % c);
    const long long v = e / c;
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((long long)W * H));
    float acc = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const long long vs = ((long long)(2 * z + dz) * (2 * H) + (2 * y + dy)) * (2 * W) + (2 * x + dx);
          acc += __bfloat162float(src[vs * ss + so + i]);
        }
    dst[e] = __float2bfloat16_rn(acc);
  }
}

// Gradient of a down level's second convolution output that feeds both the
// concatenation (skip, already masked) and the pooling of the level below:
// gz[v][i] = skip[v][i] + (act[v][i] > 0) gpool[parent][i] / 8.
__global__ void skip_pool_combine_kernel(const __nv_bfloat16* __restrict__ skip, int ss,
                                         const __nv_bfloat16* __restrict__ act, int as,
                                         const __nv_bfloat16* __restrict__ gpool, int W, int H, int D, int c,
                                         __nv_bfloat16* __restrict__ gz) {
  const long long n = (long long)W * H * D * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % c);
    const long long v = e / c;
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((long long)W * H));
    const long long vp = ((long long)(z >> 1) * (H / 2) + (y >> 1)) * (W / 2) + (x >> 1);
    const float a = __bfloat162float(act[v * as + i]);
    const float gpv = a > 0.0f ? 0.125f * __bfloat162float(gpool[vp * c + i]) : 0.0f;
    gz[e] = __float2bfloat16_rn(__bfloat162float(skip[v * ss + i]) + gpv);
  }
}

// Loss and its gradient (relative squared error over the active cells):
// per-block partials of sum act y^2 and sum act (p - y)^2 ...
__global__ void loss_partials_kernel(const float* __restrict__ p, const float* __restrict__ y,
                                     const __nv_bfloat16* __restrict__ x0, long long V, double* __restrict__ part) {
  double den = 0.0, num = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    if (!(__bfloat162float(x0[v * 16 + 1]) > 0.0f)) continue;
    const double yy = y[v], d = (double)p[v] - yy;
    den += yy * yy;
    num += d * d;
  }
  __shared__ double sd[256], sn[256];
  sd[threadIdx.x] = den;
  sn[threadIdx.x] = num;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sd[threadIdx.x] += sd[threadIdx.x + w];
      sn[threadIdx.x] += sn[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sd[0];
    part[2 * blockIdx.x + 1] = sn[0];
  }
}

// ... summed in a fixed order: out[0] = den, out[1] = num
__global__ void loss_finalize_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double d = 0.0, n = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      d += part[2 * b];
      n += part[2 * b + 1];
    }
    out[0] = d;
    out[1] = n;
  }
}

// g[v] = 2 act (p - y) / den
__global__ void loss_grad_kernel(const float* __restrict__ p, const float* __restrict__ y,
                                 const __nv_bfloat16* __restrict__ x0, long long V, const double* __restrict__ sums,
                                 float* __restrict__ g) {
  const double den = sums[0];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const bool act = __bfloat162float(x0[v * 16 + 1]) > 0.0f;
    g[v] = act && den > 0.0 ? (float)(2.0 * ((double)p[v] - (double)y[v]) / den) : 0.0f;
  }
}

// Adam (Kingma & Ba, Algorithm 1) on the flat FP32 parameters; bc1 = 1 -
// beta1^t, bc2 = 1 - beta2^t.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  }
}

}  // namespace

size_t wgrad_smem_bytes(int cout) { return 1024 + (size_t)kWgStages * (16 * 2048 + (size_t)cout * 256); }

cudaError_t init_wgrad_kernel(size_t smem_bytes) {
  return cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_wgrad(const CUtensorMap& mx, const CUtensorMap& mg, const WgradArgs& a, cudaStream_t s) {
  count_launch();
  wgrad_kernel<<<a.nmblk * a.nsplit, kConvThreads, wgrad_smem_bytes(a.cout), s>>>(mx, mg, a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad_reduce(const float* partial, int nsplit, int rows, int cin_pad, int cin, int cout, float* dw,
                                cudaStream_t s) {
  count_launch();
  wgrad_reduce_kernel<<<ew_grid((long long)cout * cin * 27), 256, 0, s>>>(partial, nsplit, rows, cin_pad, cin, cout, dw);
  return cudaGetLastError();
}

cudaError_t launch_bias_grad(const __nv_bfloat16* g, int c, long long V, float* part, int nblocks, float* db,
                             cudaStream_t s) {
  count_launch(2);
  channel_sum_kernel<<<nblocks, 256, sizeof(float) * c, s>>>(g, c, V, part);
  partial_rows_sum_kernel<<<1, 256, 0, s>>>(part, nblocks, c, db);
  return cudaGetLastError();
}

cudaError_t launch_head_backward(const float* gp, const __nv_bfloat16* x0, const __nv_bfloat16* top, int c,
                                 const float* w, long long V, __nv_bfloat16* gz, float* part, int nblocks, float* dwb,
                                 cudaStream_t s) {
  count_launch(2);
  head_backward_kernel<<<nblocks, 256, sizeof(float) * (c + 1), s>>>(gp, x0, top, c, w, V, gz, part);
  partial_rows_sum_kernel<<<1, 256, 0, s>>>(part, nblocks, c + 1, dwb);
  return cudaGetLastError();
}

cudaError_t launch_upsample_backward(const __nv_bfloat16* src, int ss, int so, int W, int H, int D, int c,
                                     __nv_bfloat16* dst, cudaStream_t s) {
  count_launch();
  upsample_backward_kernel<<<ew_grid((long long)W * H * D * c), 256, 0, s>>>(src, ss, so, W, H, D, c, dst);
  return cudaGetLastError();
}

cudaError_t launch_skip_pool_combine(const __nv_bfloat16* skip, int ss, const __nv_bfloat16* act, int as,
                                     const __nv_bfloat16* gpool, int W, int H, int D, int c, __nv_bfloat16* gz,
                                     cudaStream_t s) {
  count_launch();
  skip_pool_combine_kernel<<<ew_grid((long long)W * H * D * c), 256, 0, s>>>(skip, ss, act, as, gpool, W, H, D, c, gz);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* p, const float* y, const __nv_bfloat16* x0, long long V, double* part, int nblocks,
                        double* sums, float* g, cudaStream_t s) {
  count_launch(3);
  loss_partials_kernel<<<nblocks, 256, 0, s>>>(p, y, x0, V, part);
  loss_finalize_kernel<<<1, 32, 0, s>>>(part, nblocks, sums);
  loss_grad_kernel<<<ew_grid(V), 256, 0, s>>>(p, y, x0, V, sums, g);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, cudaStream_t s) {
  count_launch();
  adam_kernel<<<ew_grid(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace gbmg

// ---------------------------------------------------------------------------
// The network's input channels from one patch's data (device buffers in the
// C ABI's natural layout), and the scale that maps its output back to Phi
// ---------------------------------------------------------------------------

namespace gbmg {

namespace {

struct CellFaces {
  int n;        // ghost faces
  double sum;   // sum of their Dirichlet values
  double sq;    // sum of their squares
};

__device__ __forceinline__ CellFaces ghost_faces(const int8_t* __restrict__ mask, const double* __restrict__ bx,
                                                 const double* __restrict__ by, const double* __restrict__ bz, int nx,
                                                 int ny, int nz, long long v) {
  const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((long long)nx * ny));
  const long long sy = nx, sz = (long long)nx * ny;
  const bool in[6] = {i > 0, i + 1 < nx, j > 0, j + 1 < ny, k > 0, k + 1 < nz};
  const long long off[6] = {-1, 1, -sy, sy, -sz, sz};
  const long long nx1 = nx + 1, ny1 = ny + 1;
  const long long fi[6] = {((long long)k * ny + j) * nx1 + i, ((long long)k * ny + j) * nx1 + i + 1,
                           ((long long)k * ny1 + j) * nx + i, ((long long)k * ny1 + j + 1) * nx + i,
                           ((long long)k * ny + j) * nx + i, ((long long)(k + 1) * ny + j) * nx + i};
  const double* fb[6] = {bx, bx, by, by, bz, bz};
  CellFaces r = {0, 0.0, 0.0};
  for (int d = 0; d < 6; ++d) {
    if (in[d] && mask[v + off[d]] > 0) continue;
    const double f = fb[d] ? fb[d][fi[d]] : 0.0;
    r.n += 1;
    r.sum += f;
    r.sq += f * f;
  }
  return r;
}

// per-block partial sums: [0] sum of src^2 over active cells, [1] active
// cells, [2] sum of ghost-face values squared, [3] ghost faces
__global__ void features_partials_kernel(const int8_t* __restrict__ mask, const double* __restrict__ rho,
                                         const double* __restrict__ bx, const double* __restrict__ by,
                                         const double* __restrict__ bz, int nx, int ny, int nz, double h2n2,
                                         double* __restrict__ part) {
  const long long V = (long long)nx * ny * nz;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    if (mask[v] <= 0) continue;
    const double src = h2n2 * rho[v];
    a[0] += src * src;
    a[1] += 1.0;
    const CellFaces f = ghost_faces(mask, bx, by, bz, nx, ny, nz, v);
    a[2] += f.sq;
    a[3] += f.n;
  }
  __shared__ double sh[4][256];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// s = sqrt(mean src^2 + mean face^2) (1 when that is not positive), in a
// fixed order over the blocks
__global__ void features_scale_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ s_out) {
  if (threadIdx.x || blockIdx.x) return;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 4; ++q) a[q] += part[4 * b + q];
  const double ms = (a[1] > 0 ? a[0] / a[1] : 0.0) + (a[3] > 0 ? a[2] / a[3] : 0.0);
  const double s = sqrt(ms);
  *s_out = s > 0.0 ? s : 1.0;
}

// xin[0] = src / s on active cells; xin[1] = +1 active, -1 inactive; xin[2] =
// mean ghost-face value / s where the cell has ghost faces
__global__ void features_write_kernel(const int8_t* __restrict__ mask, const double* __restrict__ rho,
                                      const double* __restrict__ bx, const double* __restrict__ by,
                                      const double* __restrict__ bz, int nx, int ny, int nz, double h2n2,
                                      const double* __restrict__ s_dev, float* __restrict__ xin) {
  const long long V = (long long)nx * ny * nz;
  const double s = *s_dev;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const bool act = mask[v] > 0;
    double f0 = 0.0, f2 = 0.0;
    if (act) {
      f0 = h2n2 * rho[v] / s;
      const CellFaces f = ghost_faces(mask, bx, by, bz, nx, ny, nz, v);
      if (f.n) f2 = f.sum / f.n / s;
    }
    xin[v] = (float)f0;
    xin[V + v] = act ? 1.0f : -1.0f;
    xin[2 * V + v] = (float)f2;
  }
}

// phi[v] = s pred[v] (FP64)
__global__ void scale_prediction_kernel(const float* __restrict__ pred, long long V, const double* __restrict__ s_dev,
                                        double* __restrict__ phi) {
  const double s = *s_dev;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
    phi[v] = s * (double)pred[v];
}

// y[v] = phi[v] / s (the training target of a solved patch)
__global__ void scale_target_kernel(const double* __restrict__ phi, long long V, const double* __restrict__ s_dev,
                                    float* __restrict__ y) {
  const double s = *s_dev;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
    y[v] = (float)(phi[v] / s);
}

}  // namespace

cudaError_t launch_features(const int8_t* mask, const double* rho, const double* bx, const double* by,
                            const double* bz, int nx, int ny, int nz, double h, double* part, int nblocks,
                            double* s_dev, float* xin, cudaStream_t s) {
  const int n = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
  const double h2n2 = h * h * (double)n * (double)n;
  count_launch(3);
  features_partials_kernel<<<nblocks, 256, 0, s>>>(mask, rho, bx, by, bz, nx, ny, nz, h2n2, part);
  features_scale_kernel<<<1, 32, 0, s>>>(part, nblocks, s_dev);
  features_write_kernel<<<ew_grid((long long)nx * ny * nz), 256, 0, s>>>(mask, rho, bx, by, bz, nx, ny, nz, h2n2, s_dev,
                                                                        xin);
  return cudaGetLastError();
}

cudaError_t launch_scale_prediction(const float* pred, long long V, const double* s_dev, double* phi, cudaStream_t s) {
  count_launch();
  scale_prediction_kernel<<<ew_grid(V), 256, 0, s>>>(pred, V, s_dev, phi);
  return cudaGetLastError();
}

cudaError_t launch_scale_target(const double* phi, long long V, const double* s_dev, float* y, cudaStream_t s) {
  count_launch();
  scale_target_kernel<<<ew_grid(V), 256, 0, s>>>(phi, V, s_dev, y);
  return cudaGetLastError();
}

}  // namespace gbmg
