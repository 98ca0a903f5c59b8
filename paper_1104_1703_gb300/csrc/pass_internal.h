// Internal declarations of the temporal-blocked FP32 smoothing pass of the
// fine level (kernels_pass.cu).
#pragma once

#include <cuda.h>

#include "mg_internal.h"

namespace gbmg {

constexpr int kPassTQ = 32;        // tile width in slots (64 cells in x)
constexpr int kPassTJ = 16;        // tile height in rows
constexpr int kPassZ = 16;         // planes per z-segment
constexpr int kPassHalo = 4;       // loaded halo around the tile, slots and rows
constexpr int kPassCodeWidth = 64; // code region width in bytes (TMA x start aligned to 16 bytes)
constexpr int kPassCodeShift = 12; // code column of float column 0 (the float region starts at q0 - 4)
constexpr int kPassThreads = 512;

// Tensor maps of one hierarchy's fine level: the black FP32 correction of
// each of the two correction buffers (the pass input), the FP32 right-hand
// side and the codes of both colours.
struct PassMaps {
  CUtensorMap black[2];
  CUtensorMap b[2];
  CUtensorMap code[2];
};

struct PassArgs {
  Geom g;
  float* out[2];         // the other correction buffer (both colours), tile interiors written
  double* phi64[2];      // non-null: Phi += e of the written values (the mixed form's last pass)
  const uint32_t* tiles; // non-empty tiles: mq | mj << 10 | mk << 20
  const uint32_t* ntiles;
  int* err;              // set to 1 when a copy did not land in time
  int debug_stall;       // test hook: CTA 0 waits on a barrier that never completes
};

// candidate tiles per axis
inline void pass_tile_grid(const Geom& g, int* nq, int* nj, int* nk) {
  *nq = (g.hx + kPassTQ - 1) / kPassTQ;
  *nj = (g.ny + kPassTJ - 1) / kPassTJ;
  *nk = (g.nz + kPassZ - 1) / kPassZ;
}

size_t pass_smem_bytes();
cudaError_t init_pass_kernel();
bool make_pass_maps(PassMaps* m, const Geom& g, float* const* phi_a, float* const* phi_b, float* const* rhs,
                    uint8_t* const* code);
// flags: one word per candidate tile; tiles: up to nq*nj*nk entries
cudaError_t launch_pass_tiles(const Geom& g, uint8_t* const* code, uint32_t* flags, uint32_t* tiles, uint32_t* count,
                              cudaStream_t s);
// input: which correction buffer the pass reads (0: a, 1: b)
cudaError_t launch_smooth_pass(const PassMaps& m, int input, const PassArgs& a, cudaStream_t s);

}  // namespace gbmg
