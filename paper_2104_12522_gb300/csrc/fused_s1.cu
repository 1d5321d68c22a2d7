// Fused emission kernels for 1 species (see emission_fused.cuh).
#include "emission_fused.cuh"

namespace bartem {
template FusedLauncher fused_launcher<1>(int, bool, int, int);
}  // namespace bartem
