// Fused emission kernels for 3 species (see emission_fused.cuh).
#include "emission_fused.cuh"

namespace bartem {
template FusedLauncher fused_launcher<3>(int, bool, int, int);
}  // namespace bartem
