// Tensor maps (TMA descriptors) of the pipelined 2D half steps: one per
// array the half step stages, built once per context on the host.
#pragma once
#include <cuda.h>

namespace fw2 {

constexpr int kPipeMaps = 10;

// velocity: 0 p (136 x 15 halo box), 1 rho (132 x 9; tissue-index form: the
//   uint8 index, 144 x 9), 2 v_x, 3 v_y, 4 psi1_x (128 x 8 x N), 5 psi1_y,
//   6 1/kappa1, 7 a1 (128 x 8 x N), 8 b1
// pressure: 0 v_x (136 x 10 halo box), 1 v_y (136 x 15), 2 p, 3 psi2_x,
//   4 psi2_y, 5 1/kappa2 (tissue-index form: the uint8 index), 6 K, 7 chi,
//   8 a2, 9 b2
// (boxes 128 x 8 unless stated; unused slots stay zero)
struct PipeMaps {
  CUtensorMap m[kPipeMaps];
};

}  // namespace fw2
