// Device check of the integer-only FP64 -> FP32 narrowing and FP32 -> FP64
// widening of cycle_device.cuh against CUDA's own conversions:
//  - narrow_f64(x) equals __double2float_rz(x) (round toward zero) bit for
//    bit wherever the result is a normal float or an overflow (which round
//    toward zero saturates at +-FLT_MAX), is a zero of x's sign where the
//    exact result is below 2^-126 (documented flush), keeps infinities and
//    maps every NaN to a NaN;
//  - widen_f32(f) equals (double)f for every normal, zero, infinite and NaN
//    float, and a zero of f's sign for subnormals.
// Inputs: hand-picked edge values around each boundary plus a fixed
// pseudo-random sweep of bit patterns.  Prints "ok" or the first mismatch.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_1104_1703_gb300/csrc/cycle_device.cuh"

using gbmg::narrow_f64;
using gbmg::widen_f32;

__global__ void convert_kernel(const double* in, int n, float* mine, float* rz, const float* fin, int nf,
                               double* wide) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    mine[i] = narrow_f64(in[i]);
    rz[i] = __double2float_rz(in[i]);
  }
  if (i < nf) wide[i] = widen_f32(fin[i]);
}

static unsigned long long splitmix(unsigned long long* s) {
  unsigned long long z = (*s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static double bits_d(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}
static unsigned long long d_bits(double d) {
  unsigned long long b;
  std::memcpy(&b, &d, 8);
  return b;
}
static unsigned f_bits(float f) {
  unsigned b;
  std::memcpy(&b, &f, 4);
  return b;
}
static float bits_f(unsigned b) {
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

#define CK(x)                                                          \
  do {                                                                 \
    cudaError_t e_ = (x);                                              \
    if (e_ != cudaSuccess) {                                           \
      std::printf("cuda error %s at %s\n", cudaGetErrorString(e_), #x); \
      return 2;                                                        \
    }                                                                  \
  } while (0)

int main() {
  std::vector<double> in;
  const unsigned long long exps[] = {0x000, 0x001, 0x200, 0x380, 0x381, 0x382, 0x3ff, 0x47e, 0x47f, 0x480,
                                     0x481, 0x7fe, 0x7ff};
  const unsigned long long mants[] = {0ull, 1ull, 0x1fffffffull, 0x20000000ull, 0xfffffe0000000ull,
                                      0xfffffffffffffull, 0x8000000000000ull, 0x0000000000001ull << 28,
                                      0x123456789abcdull};
  for (unsigned long long e : exps)
    for (unsigned long long m : mants)
      for (int s = 0; s < 2; ++s) in.push_back(bits_d(((unsigned long long)s << 63) | (e << 52) | m));
  const double named[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 3.402823669209385e38,
                          1e39, -1e39, 1e300, -1e300, 1.1754943508222875e-38, 1.1754942e-38, 1e-40, -1e-40, 1e-310};
  for (double d : named) in.push_back(d);
  unsigned long long st = 12345;
  for (int i = 0; i < 200000; ++i) {
    unsigned long long b = splitmix(&st);
    if (i & 1) {  // mostly values inside or near the float range
      const unsigned long long e = 0x370 + (splitmix(&st) % 0x120);
      b = (b & 0x800fffffffffffffull) | (e << 52);
    }
    in.push_back(bits_d(b));
  }
  std::vector<float> fin;
  const unsigned fexps[] = {0x00, 0x01, 0x7f, 0xfe, 0xff};
  const unsigned fmants[] = {0u, 1u, 0x400000u, 0x7fffffu, 0x123456u};
  for (unsigned e : fexps)
    for (unsigned m : fmants)
      for (unsigned s = 0; s < 2; ++s) fin.push_back(bits_f((s << 31) | (e << 23) | m));
  for (int i = 0; i < 100000; ++i) fin.push_back(bits_f((unsigned)splitmix(&st)));

  const int n = (int)in.size(), nf = (int)fin.size();
  double *d_in, *d_wide;
  float *d_mine, *d_rz, *d_fin;
  CK(cudaMalloc(&d_in, sizeof(double) * n));
  CK(cudaMalloc(&d_mine, sizeof(float) * n));
  CK(cudaMalloc(&d_rz, sizeof(float) * n));
  CK(cudaMalloc(&d_fin, sizeof(float) * nf));
  CK(cudaMalloc(&d_wide, sizeof(double) * nf));
  CK(cudaMemcpy(d_in, in.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_fin, fin.data(), sizeof(float) * nf, cudaMemcpyHostToDevice));
  const int m = n > nf ? n : nf;
  convert_kernel<<<(m + 255) / 256, 256>>>(d_in, n, d_mine, d_rz, d_fin, nf, d_wide);
  CK(cudaGetLastError());
  std::vector<float> mine(n), rz(n);
  std::vector<double> wide(nf);
  CK(cudaMemcpy(mine.data(), d_mine, sizeof(float) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(rz.data(), d_rz, sizeof(float) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(wide.data(), d_wide, sizeof(double) * nf, cudaMemcpyDeviceToHost));
  long long checked_rz = 0, flushed = 0, saturated = 0;
  for (int i = 0; i < n; ++i) {
    const unsigned long long b = d_bits(in[i]);
    const unsigned ex = (unsigned)(b >> 52) & 0x7ffu;
    const unsigned sign = (unsigned)(b >> 63);
    const unsigned got = f_bits(mine[i]), want = f_bits(rz[i]);
    const bool got_nan = (got & 0x7f800000u) == 0x7f800000u && (got & 0x7fffffu);
    if (ex == 0x7ff && (b & 0xfffffffffffffull)) {  // NaN
      if (!got_nan) {
        std::printf("mismatch: NaN %016llx -> %08x\n", b, got);
        return 1;
      }
      continue;
    }
    if (got_nan) {
      std::printf("mismatch: NaN from a non-NaN %016llx\n", b);
      return 1;
    }
    const unsigned wexp = (want >> 23) & 0xffu;
    if (ex != 0x7ff && wexp == 0) {  // exact result below 2^-126: flushed
      if (got != (sign << 31)) {
        std::printf("mismatch: flush %016llx -> %08x\n", b, got);
        return 1;
      }
      ++flushed;
      continue;
    }
    if (got != want) {
      std::printf("mismatch: %016llx -> %08x, round toward zero %08x\n", b, got, want);
      return 1;
    }
    ++checked_rz;
    if ((want & 0x7fffffffu) == 0x7f7fffffu && ex != 0x7ff) ++saturated;
  }
  for (int i = 0; i < nf; ++i) {
    const unsigned b = f_bits(fin[i]);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long got = d_bits(wide[i]);
    if (e == 0xff && (b & 0x7fffffu)) {
      if (!((got >> 52 & 0x7ff) == 0x7ff && (got & 0xfffffffffffffull))) {
        std::printf("mismatch: widen NaN %08x -> %016llx\n", b, got);
        return 1;
      }
      continue;
    }
    const unsigned long long want = e == 0 ? (unsigned long long)(b >> 31) << 63 : d_bits((double)fin[i]);
    if (got != want) {
      std::printf("mismatch: widen %08x -> %016llx, want %016llx\n", b, got, want);
      return 1;
    }
  }
  if (saturated == 0 || flushed == 0 || checked_rz < 100000) {
    std::printf("too few cases: rz %lld flushed %lld saturated %lld\n", checked_rz, flushed, saturated);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
