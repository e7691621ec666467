// Persistent Horner-filter kernel (horner_grid.cuh) for double-float sweeps: the shapes (tile bits
// NB, register bits RB, column bits C, L = 2 NB - C) offered to the autotuner per chain length.
#include <algorithm>

#include "horner_grid.cuh"

namespace fq {

template <> std::vector<HornerGridShape<dfloat>> horner_grid_shapes<dfloat>(int L) {
  switch (L) {
    case 13: return {{launch_horner_grid_shape<dfloat, 8, 2, 3>, 8, 2, 3}};
    case 14: return {{launch_horner_grid_shape<dfloat, 8, 2, 2>, 8, 2, 2}};
    case 15: return {{launch_horner_grid_shape<dfloat, 9, 2, 3>, 9, 2, 3}};
    case 16: return {{launch_horner_grid_shape<dfloat, 9, 2, 2>, 9, 2, 2}, {launch_horner_grid_shape<dfloat, 8, 2, 0>, 8, 2, 0}};
    case 17: return {{launch_horner_grid_shape<dfloat, 10, 3, 3>, 10, 3, 3}};
    case 18: return {{launch_horner_grid_shape<dfloat, 10, 3, 2>, 10, 3, 2}, {launch_horner_grid_shape<dfloat, 10, 2, 2>, 10, 2, 2}, {launch_horner_grid_shape<dfloat, 9, 3, 0>, 9, 3, 0}};
    case 19: return {{launch_horner_grid_shape<dfloat, 11, 3, 3>, 11, 3, 3}};
    case 20: return {{launch_horner_grid_shape<dfloat, 11, 3, 2>, 11, 3, 2}, {launch_horner_grid_shape<dfloat, 11, 2, 2>, 11, 2, 2}, {launch_horner_grid_shape<dfloat, 12, 3, 4>, 12, 3, 4}, {launch_horner_grid_shape<dfloat, 10, 3, 0>, 10, 3, 0}};
    case 21: return {{launch_horner_grid_shape<dfloat, 12, 3, 3>, 12, 3, 3}};
    case 22: return {{launch_horner_grid_shape<dfloat, 12, 3, 2>, 12, 3, 2}};
  }
  return {};
}

}  // namespace fq
