// Persistent Horner-filter kernel (horner_grid.cuh) for complex64 sweeps: the shapes (tile bits
// NB, register bits RB, column bits C, L = 2 NB - C) offered to the autotuner per chain length.
#include <algorithm>

#include "horner_grid.cuh"

namespace fq {

template <> std::vector<HornerGridShape<float>> horner_grid_shapes<float>(int L) {
  switch (L) {
    case 13: return {{launch_horner_grid_shape<float, 8, 2, 3>, 8, 2, 3}};
    case 14: return {{launch_horner_grid_shape<float, 8, 2, 2>, 8, 2, 2}};
    case 15: return {{launch_horner_grid_shape<float, 9, 3, 3>, 9, 3, 3}};
    case 16: return {{launch_horner_grid_shape<float, 9, 3, 2>, 9, 3, 2}, {launch_horner_grid_shape<float, 10, 4, 4>, 10, 4, 4}};
    case 17: return {{launch_horner_grid_shape<float, 10, 3, 3>, 10, 3, 3}, {launch_horner_grid_shape<float, 10, 4, 3>, 10, 4, 3}};
    case 18: return {{launch_horner_grid_shape<float, 10, 3, 2>, 10, 3, 2}, {launch_horner_grid_shape<float, 10, 4, 2>, 10, 4, 2}, {launch_horner_grid_shape<float, 11, 4, 4>, 11, 4, 4}, {launch_horner_grid_shape<float, 9, 3, 0>, 9, 3, 0}};
    case 19: return {{launch_horner_grid_shape<float, 11, 3, 3>, 11, 3, 3}, {launch_horner_grid_shape<float, 11, 4, 3>, 11, 4, 3}};
    case 20: return {{launch_horner_grid_shape<float, 11, 3, 2>, 11, 3, 2}, {launch_horner_grid_shape<float, 11, 4, 2>, 11, 4, 2}, {launch_horner_grid_shape<float, 12, 4, 4>, 12, 4, 4}, {launch_horner_grid_shape<float, 10, 3, 0>, 10, 3, 0}};
    case 21: return {{launch_horner_grid_shape<float, 12, 3, 3>, 12, 3, 3}, {launch_horner_grid_shape<float, 12, 4, 3>, 12, 4, 3}};
    case 22: return {{launch_horner_grid_shape<float, 12, 3, 2>, 12, 3, 2}, {launch_horner_grid_shape<float, 12, 4, 2>, 12, 4, 2}};
  }
  return {};
}

}  // namespace fq
