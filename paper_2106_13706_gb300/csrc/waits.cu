// waits.cu -- the bound on device-side waits, and a self-test of it.
//
// The kernels that stream their inputs with bulk asynchronous copies wait on
// shared-memory mbarriers for each copy.  Every such wait gives up after the
// context's bound (ddks_set_device_wait_limit; the config's wait_limit_ms, or
// 1 s), sets the timeout flag, waits (bounded) for its own copies still in
// flight and returns, so the call reports DDKS_ETIMEOUT and the context stays
// usable.  ddks_wait_selftest runs that same wait on a phase that never
// completes: nothing faults, traps or hangs.
#include "../../include/ddks.h"
#include "bulk_copy.cuh"
#include "ddks_host.h"

namespace {

// One thread arms an mbarrier for 16 transaction bytes and issues no copy;
// the wait must give up after wait_ns.  flags |= kFlagTimeout when it does
// (or kFlagBounds if the phase completed, which cannot happen).
__global__ void k_wait_selftest(unsigned* __restrict__ flags, unsigned long long wait_ns,
                                unsigned long long* __restrict__ waited_ns) {
  namespace bk = ddks::bulk;
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(&bar);
  bk::mbar_init(bar_s, 1);
  bk::mbar_init_fence();
  bk::mbar_expect(bar_s, 16u);  // the arrival happens, the 16 bytes never do
  const unsigned long long t0 = bk::global_ns();
  const bool ok = bk::wait(bar_s, 0u, wait_ns);
  *waited_ns = bk::global_ns() - t0;
  atomicOr(flags, ok ? ddks::kFlagBounds : ddks::kFlagTimeout);
}

}  // namespace

int ddks_set_device_wait_limit(ddks_ctx* ctx, uint64_t limit_ns) {
  if (!ctx) return DDKS_EINVAL;
  ctx->dev_wait_ns = limit_ns ? limit_ns : ctx->dev_wait_cfg_ns;
  return DDKS_OK;
}

int ddks_wait_selftest(ddks_ctx* ctx, void* stream, uint64_t* waited_ns) {
  if (!ctx) return DDKS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  int rc = ctx->flags.reserve(ctx, 64);
  if (rc) return rc;
  unsigned* flags = (unsigned*)ctx->flags.ptr;
  unsigned long long* dwaited = (unsigned long long*)((char*)ctx->flags.ptr + 32);
  e = cudaMemsetAsync(flags, 0, 64, st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 1, 0, st>>>(flags, ctx->dev_wait_ns, dwaited);
    e = cudaGetLastError();
    ++ctx->launches;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_out, flags, 64, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "wait self-test");
  const unsigned f = (unsigned)(ctx->h_out[0] & 0xFFFFFFFFull);
  if (waited_ns) *waited_ns = ctx->h_out[4];
  if (f & ddks::kFlagTimeout) return DDKS_ETIMEOUT;
  return DDKS_ECUDA;  // the phase completed without its bytes: not expected
}
