// Fused emission kernels for 4 species (see emission_fused.cuh).
#include "emission_fused.cuh"

namespace bartem {
template FusedLauncher fused_launcher<4>(int, bool, int, int);
}  // namespace bartem
