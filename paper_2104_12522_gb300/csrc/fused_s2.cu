// Fused emission kernels for 2 species (see emission_fused.cuh).
#include "emission_fused.cuh"

namespace bartem {
template FusedLauncher fused_launcher<2>(int, bool, int, int);
}  // namespace bartem
