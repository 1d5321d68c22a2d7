// Transmission (transit) geometry of the forward model.  Filled in by the
// transit-depth kernel; until then the geometry is reported as unsupported.
#include "bart_internal.cuh"

bart_status bart_transmission_batch(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                    const bart_batch* b, float* spectra, const bart_filters* f, float* bands) {
  (void)g; (void)c; (void)b; (void)spectra; (void)f; (void)bands;
  return bart_fail(ctx, BART_EUNSUPPORTED, "transmission geometry is not built yet");
}
