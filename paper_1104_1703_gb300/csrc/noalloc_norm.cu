// Residual norm of the fine-level operator computed from caller buffers
// without any device allocation (mg_residual_norm_noalloc in mg.h).
//
// Some callers cannot allocate device memory when they need this norm: AMR
// codes and frameworks that reserve the GPU's memory up front in their own
// pool (a cudaMalloc outside the pool can fail on a device they have filled),
// and host code that must not block on the allocator, since cudaMalloc and
// cudaFree can wait for work in flight.  They still need the convergence
// measure of their own Phi, rho and boundary values, without building a
// hierarchy (whose arena is allocated).
//
// The per-block partial sums, the only scratch this computation needs, live
// in a file-scope __device__ array of fixed size.  Host code cannot use the
// array's name as a device address, so every call obtains the address with
// cudaGetSymbolAddress, with the caller's device current, and passes it to
// the kernels.  The lookup allocates nothing and is cheap; doing it on every
// call rather than caching it keeps the address right when the module is
// loaded again at another address (after cudaDeviceReset, or in another
// context of the same device).  The first call on a device also loads this
// file's kernels and the array.
#include <cmath>

#include "../../include/mg.h"
#include "mg_internal.h"

namespace gbmg {

void set_thread_error(const char* msg);        // mg_capi.cu
bool is_device_ptr(const void* p, int device);  // mg_capi.cu

namespace {

constexpr int kNoAllocMaxPartials = 4096;  // 32 KB of scratch on each device
constexpr int kNoAllocThreads = 256;

// One partial sum of squares per block of the first kernel.  Every call on a
// device uses the same array; each slot the second kernel reads is written by
// the first kernel of the same call, so nothing needs clearing between calls.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

// Residual r^ = h^2 (Laplacian Phi - rho) of every active cell, with the
// modified stencil of Section 3 at level 0 (ghost at theta = 1/2 through the
// face value Phi_b, Fig. 5): r^ = sum_active Phi_j + 2 sum_ghost Phi_b
// - (6 + #ghost) Phi_i - h^2 rho_i.  Block sums of r^2 go to partials.
__global__ void __launch_bounds__(kNoAllocThreads)
noalloc_resnorm_kernel(const int8_t* __restrict__ mask, const double* __restrict__ phi,
                       const double* __restrict__ rho, const double* __restrict__ bx,
                       const double* __restrict__ by, const double* __restrict__ bz, int nx, int ny, int nz,
                       double h2, double* partials) {
  const long long n = (long long)nx * ny * nz;
  const long long sy = nx, sz = (long long)nx * ny;
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    if (mask[idx] <= 0) continue;
    const int i = (int)(idx % nx);
    const long long t = idx / nx;
    const int j = (int)(t % ny), k = (int)(t / ny);
    const long long fx = ((long long)k * ny + j) * (nx + 1) + i;
    const long long fy = ((long long)k * (ny + 1) + j) * nx + i;
    const long long fz = idx;
    const bool in[6] = {i > 0, i + 1 < nx, j > 0, j + 1 < ny, k > 0, k + 1 < nz};
    const long long off[6] = {-1, 1, -sy, sy, -sz, sz};
    const double* fb[6] = {bx, bx, by, by, bz, bz};
    const long long fi[6] = {fx, fx + 1, fy, fy + nx, fz, fz + sz};
    double s = 0.0;
    int ghosts = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (in[d] && mask[idx + off[d]] > 0) {
        s += phi[idx + off[d]];
      } else {
        ++ghosts;
        if (fb[d]) s += 2.0 * fb[d][fi[d]];
      }
    }
    const double r = fma(-(double)(6 + ghosts), phi[idx], s) - h2 * rho[idx];
    acc = fma(r, r, acc);
  }
  __shared__ double warp_sums[kNoAllocThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kNoAllocThreads / 32 ? warp_sums[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// Sums the partials in a fixed order and writes ||r|| = sqrt(sum) / h^2.
__global__ void __launch_bounds__(kNoAllocThreads)
noalloc_finalize_kernel(const double* __restrict__ partials, int nblocks, double h2, double* out) {
  double acc = 0.0;
  for (int e = threadIdx.x; e < nblocks; e += blockDim.x) acc += partials[e];
  __shared__ double sm[kNoAllocThreads];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(sm[0]) / h2;
}

}  // namespace
}  // namespace gbmg

extern "C" mg_status mg_residual_norm_noalloc(const int8_t* mask, const double* phi, const double* rho,
                                              const double* bx, const double* by, const double* bz, int nx,
                                              int ny, int nz, double h, double* norm_out, void* cuda_stream) {
  using namespace gbmg;
  if (!mask || !phi || !rho || !norm_out) {
    set_thread_error("mg_residual_norm_noalloc: null mask, phi, rho or output");
    return MG_ERR_INVALID_ARG;
  }
  if (nx < 1 || ny < 1 || nz < 1 || nx > 2048 || ny > 2048 || nz > 2048) {
    set_thread_error("mg_residual_norm_noalloc: dimensions must be in 1..2048");
    return MG_ERR_INVALID_ARG;
  }
  if (!(h > 0) || !std::isfinite(h)) {
    set_thread_error("mg_residual_norm_noalloc: h must be finite and > 0");
    return MG_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    set_thread_error("mg_residual_norm_noalloc: no usable current CUDA device");
    return MG_ERR_CUDA;
  }
  const void* const bufs[] = {mask, phi, rho, bx, by, bz, norm_out};
  for (const void* p : bufs)
    if (p && !is_device_ptr(p, dev)) {
      set_thread_error("mg_residual_norm_noalloc: a buffer is not device memory of the current GPU");
      return MG_ERR_INVALID_ARG;
    }
  void* scratch = nullptr;
  cudaError_t es = cudaGetSymbolAddress(&scratch, g_noalloc_partials);
  if (es != cudaSuccess || !scratch) {
    (void)cudaGetLastError();
    set_thread_error("mg_residual_norm_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return MG_ERR_CUDA;
  }
  const long long n = (long long)nx * ny * nz;
  long long blocks = (n + kNoAllocThreads - 1) / kNoAllocThreads;
  if (blocks > kNoAllocMaxPartials) blocks = kNoAllocMaxPartials;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const double h2 = h * h;
  count_launch(2);
  noalloc_resnorm_kernel<<<(int)blocks, kNoAllocThreads, 0, s>>>(mask, phi, rho, bx, by, bz, nx, ny, nz, h2,
                                                                  (double*)scratch);
  noalloc_finalize_kernel<<<1, kNoAllocThreads, 0, s>>>((const double*)scratch, (int)blocks, h2, norm_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}
