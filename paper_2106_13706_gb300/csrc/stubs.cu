// stubs.cu -- entry points whose kernels are not built yet report
// DDKS_EUNSUPPORTED instead of computing anything on the host.
#include "ddks_host.h"
#include "ddks_internal.cuh"

int ddks_submit(ddks_ctx*, const void*, int64_t, const void*, int64_t, int32_t, int32_t, uint64_t*) {
  return DDKS_EUNSUPPORTED;
}
int ddks_poll(ddks_ctx*, uint64_t, int32_t, ddks_result*) { return DDKS_EUNSUPPORTED; }
void ddks_serve_shutdown(ddks_ctx*) {}
void ddks_serve_fill_stats(ddks_ctx*, ddks_stats* out) {
  out->submitted = out->admitted = out->completed = out->rejected = 0;
  out->batches = out->bytes_resident = out->bytes_resident_peak = 0;
}
