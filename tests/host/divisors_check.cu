// Host check of Geom::div_sz / div_P / slot_of (mg_internal.h) against
// integer division, for the geometries of many grid shapes: every element
// offset of small grids, and offsets next to every multiple of the divisor
// plus random offsets for large ones; and of Geom::slot_in_bounds, the
// checked build's bounds test.  Prints "ok" or the first mismatch.
#include <cstdio>
#include <cstdlib>

#include "../../paper_1104_1703_gb300/csrc/mg_internal.h"

using gbmg::Geom;

static Geom geom(int nx, int ny, int nz) {
  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.hx = (nx + 1) / 2;
  g.P = ((g.hx + 1) + 7) & ~7;
  g.sz = (long long)(ny + 2) * g.P;
  g.off0 = g.sz + g.P;
  g.total = (long long)(nz + 2) * g.sz;
  g.set_divisors();
  return g;
}

static bool check(const Geom& g, unsigned n) {
  const unsigned k = n / (unsigned)g.sz, r = n % (unsigned)g.sz;
  if (g.div_sz(n) != (int)k) return false;
  if (g.div_P(r) != (int)(r / (unsigned)g.P)) return false;
  int q, j, kk;
  g.slot_of(g.off0 + n, &q, &j, &kk);
  return kk == (int)k && j == (int)(r / (unsigned)g.P) && q == (int)(r % (unsigned)g.P);
}

int main() {
  unsigned long long x = 88172645463325252ULL;
  auto rnd = [&]() {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return x;
  };
  const int dims[][3] = {{1, 1, 1}, {2, 3, 5}, {17, 12, 10}, {48, 32, 40}, {64, 64, 64}, {127, 255, 3},
                         {256, 256, 256}, {512, 512, 512}, {2048, 2048, 500}, {1000, 3, 2048}, {2047, 2047, 2}};
  for (const auto& d : dims) {
    const Geom g = geom(d[0], d[1], d[2]);
    const long long lim = g.total - g.off0;
    if (lim <= (1LL << 22)) {
      for (long long n = 0; n < lim; ++n)
        if (!check(g, (unsigned)n)) {
          std::printf("mismatch %dx%dx%d n=%lld\n", d[0], d[1], d[2], n);
          return 1;
        }
    } else {
      for (long long m = g.sz; m < lim; m += g.sz)
        for (int e = -1; e <= 1; ++e)
          if (!check(g, (unsigned)(m + e))) {
            std::printf("mismatch %dx%dx%d n=%lld\n", d[0], d[1], d[2], m + e);
            return 1;
          }
      for (int t = 0; t < 2000000; ++t) {
        const unsigned n = (unsigned)(rnd() % (unsigned long long)lim);
        if (!check(g, n)) {
          std::printf("mismatch %dx%dx%d n=%u\n", d[0], d[1], d[2], n);
          return 1;
        }
      }
    }
  }
  // the bounds test of the checked build (Geom::slot_in_bounds): true
  // exactly on the slots (q < hx, j < ny, k < nz) of every offset of small
  // grids, and every stencil neighbour of a slot lies inside the array
  const int small[][3] = {{1, 1, 1}, {2, 3, 5}, {3, 1, 2}, {17, 12, 10}, {9, 16, 7}, {48, 32, 40}};
  for (const auto& d : small) {
    const Geom g = geom(d[0], d[1], d[2]);
    for (long long at = -g.sz; at < g.total + g.sz; ++at) {
      bool slot = false;
      if (at >= g.off0) {
        const long long rel = at - g.off0;
        const long long k = rel / g.sz, r = rel % g.sz, j = r / g.P, q = r % g.P;
        slot = k < g.nz && j < g.ny && q < g.hx;
      }
      if (g.slot_in_bounds(at) != slot) {
        std::printf("bounds mismatch %dx%dx%d at=%lld\n", d[0], d[1], d[2], at);
        return 1;
      }
      if (slot) {
        const long long nb[6] = {at - 1, at + 1, at - g.P, at + g.P, at - g.sz, at + g.sz};
        for (long long b : nb)
          if (b < 0 || b >= g.total) {
            std::printf("neighbour outside %dx%dx%d at=%lld\n", d[0], d[1], d[2], at);
            return 1;
          }
      }
    }
  }
  // the divisor formula itself over every divisor up to 2^16 and dividends
  // next to its multiples up to 2^31
  for (unsigned long long dv = 1; dv <= 65536; ++dv) {
    Geom g = geom(1, 1, 1);
    g.sz = (long long)dv;
    g.P = (int)dv;
    g.set_divisors();
    for (int t = 0; t < 64; ++t) {
      const unsigned long long qm = rnd() % ((1ULL << 31) / dv);
      for (long long e = -1; e <= 1; ++e) {
        const long long n = (long long)(qm * dv) + e;
        if (n < 0 || n >= (1LL << 31)) continue;
        if (g.div_sz((unsigned)n) != (int)((unsigned long long)n / dv)) {
          std::printf("mismatch d=%llu n=%lld\n", dv, n);
          return 1;
        }
      }
    }
  }
  std::printf("ok\n");
  return 0;
}
