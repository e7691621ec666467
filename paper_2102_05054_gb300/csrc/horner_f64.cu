// Persistent Horner-filter kernel (horner_grid.cuh) for complex128 sweeps: the shapes (tile bits
// NB, register bits RB, column bits C, L = 2 NB - C) offered to the autotuner per chain length.
#include <algorithm>

#include "horner_grid.cuh"

namespace fq {

template <> std::vector<HornerGridShape<double>> horner_grid_shapes<double>(int L) {
  switch (L) {
    case 13: return {{launch_horner_grid_shape<double, 8, 2, 3>, 8, 2, 3}};
    case 14: return {{launch_horner_grid_shape<double, 8, 2, 2>, 8, 2, 2}};
    case 15: return {{launch_horner_grid_shape<double, 9, 2, 3>, 9, 2, 3}};
    case 16: return {{launch_horner_grid_shape<double, 9, 2, 2>, 9, 2, 2}};
    case 17: return {{launch_horner_grid_shape<double, 10, 3, 3>, 10, 3, 3}};
    case 18: return {{launch_horner_grid_shape<double, 10, 3, 2>, 10, 3, 2}};
    case 19: return {{launch_horner_grid_shape<double, 11, 3, 3>, 11, 3, 3}};
    case 20: return {{launch_horner_grid_shape<double, 11, 3, 2>, 11, 3, 2}, {launch_horner_grid_shape<double, 10, 3, 0>, 10, 3, 0}};
    case 21: return {{launch_horner_grid_shape<double, 12, 3, 3>, 12, 3, 3}};
    case 22: return {{launch_horner_grid_shape<double, 12, 3, 2>, 12, 3, 2}};
  }
  return {};
}

}  // namespace fq
