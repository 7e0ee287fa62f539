// Tensor maps (TMA descriptors) of the pipelined 2D half steps: one per
// array the half step stages, built once per context on the host.
#pragma once
#include <cuda.h>

namespace fw2 {

constexpr int kPipeMaps = 17;

// velocity: 0 p (136 x 15 halo box), 1 rho (132 x 9; tissue-index form: the
//   uint8 index, 144 x 9), 2 v_x, 3 v_y, 4 psi1_x (128 x 8 x N), 5 psi1_y,
//   6 1/kappa1, 7 a1 (128 x 8 x N), 8 b1, 9 K (132 x 9, float maps with the
//   literal nonlinear system)
// pressure: 0 v_x (136 x 10 halo box), 1 v_y (136 x 15), 2 p, 3 psi2_x,
//   4 psi2_y, 5 1/kappa2 (tissue-index form: the uint8 index), 6 K, 7 chi,
//   8 a2, 9 b2
// (boxes 128 x 8 unless stated; unused slots stay zero)
struct PipeMaps {
  CUtensorMap m[kPipeMaps];
};

// 3D pipelined half steps (bf16 maps):
// velocity: 0 p halo plane (136 x 15 x 1), 2 rho bf16 (136 x 9 x 2), 3 v
//   (128 x 8 x 1 x 3), 5 1/kappa1 bf16, 6 a1 bf16 (128 x 8 x 1 x N), 7 b1,
//   10 and 11 the x C-PML strip's a1, b1 (L x 8 x 1 x N of the [N][z][y][2L]
//   strip arrays; L a multiple of 8, at most 64), 12 K bf16 (136 x 9 x 2,
//   literal nonlinear system), 13 and 14 the y strip's a1, b1 (128 x 8 x 1 x
//   N of [N][z][2L][x]), 15 and 16 the z strip's (128 x 8 x 1 x N of
//   [N][2L][y][x])
// pressure: 0 v_x (136 x 8 x 1; with cross taps 136 x 10 x 1), 1 v_y
//   (128 x 15 x 1; with cross taps 136 x 15 x 1), 2 v_z plane (128 x 8 x 1;
//   with cross taps 136 x 10 x 1), 3 p, 5 1/kappa2, 6 K, 7 chi, 8 a2, 9 b2
//   (bf16), 10 and 11 the x strip's a2, b2, 13 to 16 the y and z strips'
// Encode a tiled tensor map (host): element size 1, 2 or 4 bytes (uint8,
// bf16, float), rank 2..4, dims[0] innermost, strides in bytes of dims 1..;
// cells outside the tensor read as zero.  False when the driver entry point
// is missing or rejects the map.
bool encode_tensor_map(CUtensorMap *m, const void *base, int elem_bytes, int rank, const unsigned long long *dims,
                       const unsigned long long *strides_bytes, const unsigned *box);

}  // namespace fw2
