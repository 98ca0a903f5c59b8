// Runs exact_sum<6> (exact_sum.cuh) on sets of six doubles, on the host or
// on the GPU, for tests/test_exact_sum.py and tests/test_gpu_exact_sum.py.
//   exact_sum_check host|device IN OUT
// IN: an int64 count n, then n * 6 doubles; OUT: the n sums (doubles).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../paper_1104_1703_gb300/csrc/exact_sum.cuh"

__global__ void sum_kernel(const double* in, long long n, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[6];
  for (int j = 0; j < 6; ++j) x[j] = in[6 * i + j];
  out[i] = gbmg::exact_sum(x);
}

int main(int argc, char** argv) {
  if (argc != 4) {
    std::fprintf(stderr, "usage: %s host|device IN OUT\n", argv[0]);
    return 2;
  }
  FILE* f = std::fopen(argv[2], "rb");
  if (!f) return 2;
  long long n = 0;
  if (std::fread(&n, 8, 1, f) != 1 || n < 0 || n > (1LL << 26)) return 2;
  std::vector<double> in(6 * n), out(n);
  if (std::fread(in.data(), 8, 6 * n, f) != (size_t)(6 * n)) return 2;
  std::fclose(f);
  if (!std::strcmp(argv[1], "host")) {
    for (long long i = 0; i < n; ++i) {
      double x[6];
      for (int j = 0; j < 6; ++j) x[j] = in[6 * i + j];
      out[i] = gbmg::exact_sum(x);
    }
  } else {
    double *din = nullptr, *dout = nullptr;
    if (cudaMalloc(&din, 8 * in.size() + 8) != cudaSuccess || cudaMalloc(&dout, 8 * out.size() + 8) != cudaSuccess)
      return 3;
    cudaMemcpy(din, in.data(), 8 * in.size(), cudaMemcpyHostToDevice);
    if (n) sum_kernel<<<(unsigned)((n + 255) / 256), 256>>>(din, n, dout);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    cudaMemcpy(out.data(), dout, 8 * out.size(), cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
  }
  f = std::fopen(argv[3], "wb");
  if (!f) return 2;
  std::fwrite(out.data(), 8, n, f);
  std::fclose(f);
  return 0;
}
