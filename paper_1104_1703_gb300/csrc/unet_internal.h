// Internal declarations of the learned initial guess's network (a 3D U-Net,
// BF16 weights and activations, FP32 accumulation): the tcgen05 convolution
// and the element-wise kernels of kernels_unet.cu, driven by mg_unet.cu.
//
// Activations are channels-last BF16 tensors [z][y][x][channel] of one grid
// level; a tensor may be a channel range of a wider buffer (the
// concatenation of a skip connection and an upsampled tensor), given by a
// channel stride and offset.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

namespace gbmg {

constexpr int kConvThreads = 192;  // warp 0 copies, warp 1 issues the MMAs, warps 2-5 drain the accumulators
constexpr int kConvMaxStages = 16;
constexpr int kConvTileM = 128;    // voxels per output tile (the MMA's M)

// One 3x3x3 convolution (zero padding 1) as an implicit GEMM: output tile of
// 128 voxels x cout channels, K = 27 taps x cin channels.  The pipeline's
// unit is one tap and `kc` 8-channel chunks of the input.
struct ConvArgs {
  int W, H, D;           // spatial size of input and output
  int cin, cout;         // channels, multiples of 16; cout <= 256
  int kc;                // 8-channel chunks per unit (even, divides cin / 8, <= 8)
  int bx, by, bz;        // the output tile's box (bx * by * bz = 128)
  int ntx, nty, ntz;     // tiles per axis
  const __nv_bfloat16* w;  // packed weights [27][cin / 8][cout][8]
  const float* bias;       // nullable, [cout]
  int relu;                // apply max(0, .) after the bias
  const __nv_bfloat16* mask;  // nullable: out *= (mask[v][mask_off + o] > 0)
  int mask_stride, mask_off;
  __nv_bfloat16* out;         // out[v][out_off + o], channel stride out_stride
  int out_stride, out_off;
  float* out_f32;             // nullable: also out_f32[v][o] (FP32, before rounding)
  int* err;                   // set to 1 when a wait runs out
  int debug_stall;            // test hook: the copy thread of CTA 0 stops issuing
  // pipeline (conv_plan): stages in flight, the layer's weights resident in
  // shared memory, and the halo path (a tile is one row of 128 voxels whose
  // input is copied once with a one-voxel halo; needs resident weights)
  int stages;
  int wres;
  int halo;
};

struct ConvLayout {
  unsigned w_load;   // bytes of the packed weights copied in once (a multiple of 16)
  unsigned w_bytes;  // their shared-memory footprint, rounded to 1 KB (0: staged per unit)
  unsigned a_bytes;  // input bytes per unit (the copy's size)
  unsigned a_stride; // their shared-memory stride, a multiple of 128 bytes
  unsigned b_bytes;  // weight bytes per unit
  int units;         // units per tile
};
__host__ __device__ ConvLayout conv_layout(const ConvArgs& a);
void conv_plan(ConvArgs& a);
size_t conv_smem_bytes(const ConvArgs& a);

__host__ __device__ uint32_t conv_tmem_cols(int cout);
int conv_kc(int cin);
cudaError_t init_conv_kernel(size_t smem_bytes);
// `map` describes the input tensor: dims (8, W, H, D, cin / 8), box
// (8, bx, by, bz, kc), BF16; for the halo path box (8, 130, 3, 3, 2).
bool make_conv_input_map(CUtensorMap* map, const __nv_bfloat16* x, int W, int H, int D, int cin, int bx, int by,
                         int bz, int kc);
void conv_tile_box(int W, int H, int D, int* bx, int* by, int* bz);
cudaError_t launch_conv(const CUtensorMap& map, const ConvArgs& a, int grid, cudaStream_t s);
int conv_grid(const ConvArgs& a, size_t smem_bytes);

// Packs FP32 weights w[o][i][27] (the network's [cout][cin][3][3][3]) into the
// BF16 layout of the forward convolution, [27][cin_pad / 8][cout][8] (input
// channels cin .. cin_pad - 1 zero), or, with `backward`, of the
// backward-data convolution: taps mirrored and the roles of input and output
// channels exchanged, [27][cout / 8][cin_pad][8].
cudaError_t launch_pack_weights(const float* w, int cout, int cin, int cin_pad, bool backward, __nv_bfloat16* out,
                                cudaStream_t s);

// Weight gradient of one convolution (see kernels_unet.cu): CTA
// (mblock, split) sums the voxel tiles [T split / nsplit, T (split+1) /
// nsplit) into partial[split][mblock * 128 + row][o], rows (tap, i) of the
// tap-major row space of cin (padded) input channels.
struct WgradArgs {
  int W, H, D;
  int cin;     // padded input channels (the input tensor's channels), multiple of 16
  int cout;    // output channels, multiple of 16, <= 128
  int bx, by, bz, ntx, nty, ntz;
  int nmblk;   // ceil(27 cin / 128)
  int nsplit;  // <= the number of voxel tiles
  float* partial;
  int* err;
};
size_t wgrad_smem_bytes(int cout);
cudaError_t init_wgrad_kernel(size_t smem_bytes);
// mx: the input tensor with box (8, bx, by, bz, 1); mg: the gradient tensor
// (cout channels) with box (8, bx, by, bz, cout / 8)
cudaError_t launch_wgrad(const CUtensorMap& mx, const CUtensorMap& mg, const WgradArgs& a, cudaStream_t s);
cudaError_t launch_wgrad_reduce(const float* partial, int nsplit, int rows, int cin_pad, int cin, int cout, float* dw,
                                cudaStream_t s);
cudaError_t launch_bias_grad(const __nv_bfloat16* g, int c, long long V, float* part, int nblocks, float* db,
                             cudaStream_t s);
cudaError_t launch_head_backward(const float* gp, const __nv_bfloat16* x0, const __nv_bfloat16* top, int c,
                                 const float* w, long long V, __nv_bfloat16* gz, float* part, int nblocks, float* dwb,
                                 cudaStream_t s);
cudaError_t launch_upsample_backward(const __nv_bfloat16* src, int ss, int so, int W, int H, int D, int c,
                                     __nv_bfloat16* dst, cudaStream_t s);
cudaError_t launch_skip_pool_combine(const __nv_bfloat16* skip, int ss, const __nv_bfloat16* act, int as,
                                     const __nv_bfloat16* gpool, int W, int H, int D, int c, __nv_bfloat16* gz,
                                     cudaStream_t s);
cudaError_t launch_loss(const float* p, const float* y, const __nv_bfloat16* x0, long long V, double* part, int nblocks,
                        double* sums, float* g, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, cudaStream_t s);

// The three input channels (FP32 [3][V]) of a patch and its scale s (device
// scalar), from device mask, rho and face arrays (faces nullable = 0).
cudaError_t launch_features(const int8_t* mask, const double* rho, const double* bx, const double* by,
                            const double* bz, int nx, int ny, int nz, double h, double* part, int nblocks,
                            double* s_dev, float* xin, cudaStream_t s);
cudaError_t launch_scale_prediction(const float* pred, long long V, const double* s_dev, double* phi, cudaStream_t s);
cudaError_t launch_scale_target(const double* phi, long long V, const double* s_dev, float* y, cudaStream_t s);

cudaError_t launch_input_to_bf16(const float* x, long long V, __nv_bfloat16* out, cudaStream_t s);
cudaError_t launch_avg_pool(const __nv_bfloat16* src, int ss, int so, int W, int H, int D, int c, __nv_bfloat16* dst,
                            int ds, int dofs, cudaStream_t s);
cudaError_t launch_upsample(const __nv_bfloat16* src, int ss, int so, int W, int H, int D, int c, __nv_bfloat16* dst,
                            int ds, int dofs, cudaStream_t s);
cudaError_t launch_head(const __nv_bfloat16* u, int c, const float* w, const float* b, const __nv_bfloat16* x0,
                        long long V, float* pred, cudaStream_t s);
cudaError_t launch_tensor_to_natural(const __nv_bfloat16* t, int stride, int off, int c, long long V, float* out,
                                     cudaStream_t s);

}  // namespace gbmg
