// Geometry and workspace of a split sum (shared by host plans and kernels).
#pragma once

#include <cstdint>

namespace gb {

// S partial sums per output row, combined in groups of G consecutive
// splits (level 1) and then across the NG = ceil(S / G) groups (level 2,
// skipped when NG == 1).  Workspace layout, in this order:
//   tickets  [items][NG + 1] unsigned (level-1 counters, then level 2),
//            padded to 256 bytes
//   part     [S][m]  double           level-1 inputs
//   part2    [NG][m] double           level-2 inputs (NG > 1)
struct Split {
  int S, G, NG;
  int64_t m;
  double* part;
  double* part2;
  unsigned* tickets;
};

}  // namespace gb
