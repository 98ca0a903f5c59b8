// Synthetic AMR patches generated on the GPU (mg_generate_blob_patch in
// mg.h): the input recipe of the blob-patch workload, for the learned
// guess's thousands of training and evaluation patches.  This file holds
// none of the method's arithmetic.
//
// Recipe (the same streams as the host generator in workloads.py):
//  - SplitMix64 with the patch's seed; element n (n >= 1) of the stream is
//    the SplitMix64 output of seed + n * 0x9e3779b97f4a7c15, a 53-bit
//    uniform is that output >> 11 times 2^-53;
//  - white noise: normal v = sqrt(-2 log(1 - u1)) cos(2 pi u2) with u1 =
//    element v + 1 and u2 = element V + v + 1 (V cells);
//  - the noise smoothed by a periodic Gaussian of `corr_cells` cells (a
//    separable real-space convolution over 4 corr_cells on each side, where
//    the host generator filters with the Gaussian's transfer function), and
//    thresholded at 0: mask = 1 where positive;
//  - rho = -1 + 2 u with u = element 2V + v + 1;
//  - coarse potential on ((nz+1)/2 + 2, (ny+1)/2 + 2, (nx+1)/2 + 2) cells
//    (one coarse ghost cell on every side, origin -2 in fine-cell units):
//    the sum of 6 modes a cos(2 pi w_z Z + p_z) cos(2 pi w_y Y + p_y)
//    cos(2 pi w_x X + p_x) at coarse centres X = (I + 1/2) / cnx etc., with
//    the stream of seed + 1000003: amplitudes normal (elements 1..12), wave
//    numbers 1 + floor(3 u) (elements 13..30), phases 2 pi u (elements
//    31..48).
#include <cmath>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"

namespace gbmg {
void set_thread_error(const char* msg);        // mg_capi.cu
bool is_device_ptr(const void* p, int device);  // mg_capi.cu
}  // namespace gbmg

using namespace gbmg;

namespace {

constexpr unsigned long long kGolden = 0x9e3779b97f4a7c15ull;

__host__ __device__ __forceinline__ unsigned long long splitmix_at(unsigned long long seed, unsigned long long n) {
  unsigned long long z = seed + n * kGolden;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ double uniform_at(unsigned long long seed, unsigned long long n) {
  return (double)(splitmix_at(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void noise_kernel(unsigned long long seed, long long V, float* __restrict__ out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const double u1 = uniform_at(seed, (unsigned long long)v + 1);
    const double u2 = uniform_at(seed, (unsigned long long)(V + v) + 1);
    out[v] = (float)(sqrt(-2.0 * log1p(-u1)) * cos(2.0 * 3.14159265358979323846 * u2));
  }
}

// periodic 1-D Gaussian smoothing along axis `axis` (0 = x, 1 = y, 2 = z)
__global__ void blur_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, int axis,
                            const float* __restrict__ w, int radius) {
  const long long V = (long long)nx * ny * nz;
  const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int i = (int)((v / stride) % n);
    const long long base = v - (long long)i * stride;
    float acc = 0.0f;
    for (int d = -radius; d <= radius; ++d) {
      int t = (i + d) % n;
      if (t < 0) t += n;
      acc += w[d + radius] * in[base + (long long)t * stride];
    }
    out[v] = acc;
  }
}

__global__ void threshold_kernel(const float* __restrict__ f, unsigned long long seed, long long V,
                                 int8_t* __restrict__ mask, double* __restrict__ rho) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    mask[v] = f[v] > 0.0f ? 1 : 0;
    rho[v] = -1.0 + 2.0 * uniform_at(seed, (unsigned long long)(2 * V + v) + 1);
  }
}

struct Modes {
  double a[6], w[6][3], p[6][3];
};

__global__ void coarse_potential_kernel(Modes m, int cnx, int cny, int cnz, double* __restrict__ out) {
  const long long n = (long long)cnx * cny * cnz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(e % cnx), J = (int)((e / cnx) % cny), K = (int)(e / ((long long)cnx * cny));
    const double X = (I + 0.5) / cnx, Y = (J + 0.5) / cny, Z = (K + 0.5) / cnz;
    const double tp = 2.0 * 3.14159265358979323846;
    double acc = 0.0;
    for (int k = 0; k < 6; ++k)
      acc += m.a[k] * cos(tp * m.w[k][2] * Z + m.p[k][2]) * cos(tp * m.w[k][1] * Y + m.p[k][1]) *
             cos(tp * m.w[k][0] * X + m.p[k][0]);
    out[e] = acc;
  }
}

int gen_grid(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 32LL * device_sms();
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

extern "C" mg_status mg_generate_blob_patch(unsigned long long seed, int nx, int ny, int nz, double corr_cells,
                                           float* scratch, int8_t* mask, double* rho, double* phi_c,
                                           void* cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > 2048 || ny > 2048 || nz > 2048 || !(corr_cells > 0) || corr_cells > 64) {
    set_thread_error("mg_generate_blob_patch: sizes must be in 1..2048 and corr_cells in (0, 64]");
    return MG_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_thread_error("mg_generate_blob_patch: no CUDA device");
    return MG_ERR_CUDA;
  }
  for (const void* p : {(const void*)scratch, (const void*)mask, (const void*)rho, (const void*)phi_c})
    if (!p || !is_device_ptr(p, dev)) {
      set_thread_error("mg_generate_blob_patch: every buffer must be device memory of the current GPU");
      return MG_ERR_INVALID_ARG;
    }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long V = (long long)nx * ny * nz;
  // Gaussian weights (their normalisation does not change the sign)
  const int radius = (int)std::ceil(4.0 * corr_cells);
  std::vector<float> w(2 * radius + 1);
  for (int d = -radius; d <= radius; ++d) w[d + radius] = (float)std::exp(-0.5 * d * d / (corr_cells * corr_cells));
  // the weights ride in the tail of the scratch buffer (2 V + 2 radius + 1 floats)
  float* a = scratch;
  float* b = scratch + V;
  float* wd = scratch + 2 * V;
  cudaError_t e = cudaMemcpyAsync(wd, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, s);
  count_launch(5);
  noise_kernel<<<gen_grid(V), 256, 0, s>>>(seed, V, a);
  blur_kernel<<<gen_grid(V), 256, 0, s>>>(a, b, nx, ny, nz, 0, wd, radius);
  blur_kernel<<<gen_grid(V), 256, 0, s>>>(b, a, nx, ny, nz, 1, wd, radius);
  blur_kernel<<<gen_grid(V), 256, 0, s>>>(a, b, nx, ny, nz, 2, wd, radius);
  threshold_kernel<<<gen_grid(V), 256, 0, s>>>(b, seed, V, mask, rho);
  // coarse potential
  Modes m;
  const unsigned long long cs = seed + 1000003ull;
  for (int k = 0; k < 6; ++k) {
    const double u1 = uniform_at(cs, (unsigned long long)k + 1), u2 = uniform_at(cs, (unsigned long long)k + 7);
    m.a[k] = std::sqrt(-2.0 * std::log1p(-u1)) * std::cos(2.0 * M_PI * u2);
    for (int d = 0; d < 3; ++d) {
      m.w[k][d] = 1.0 + std::floor(uniform_at(cs, 13 + 3 * k + d) * 3.0);
      m.p[k][d] = 2.0 * M_PI * uniform_at(cs, 31 + 3 * k + d);
    }
  }
  const int cnx = (nx + 1) / 2 + 2, cny = (ny + 1) / 2 + 2, cnz = (nz + 1) / 2 + 2;
  count_launch();
  coarse_potential_kernel<<<gen_grid((long long)cnx * cny * cnz), 256, 0, s>>>(m, cnx, cny, cnz, phi_c);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}
