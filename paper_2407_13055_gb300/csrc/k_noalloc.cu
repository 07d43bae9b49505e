// Rescale without any allocation: the same three rescale kernels as
// ckks_rescale, with their scratch in a fixed device array that the library
// owns for the life of the process.
//
// Who needs this: callers that must not allocate device memory while they
// run, for example a serving loop with a latency budget (cudaMalloc can
// synchronize the whole device and can fail when memory is tight) or code
// running where the CUDA allocator is off limits. They pass device buffers
// for the input and the output; the scratch comes from g_noalloc_scratch.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchWords = CKKS_NOALLOC_SCRATCH_WORDS;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps whatever the last call wrote.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

std::mutex g_mu;
uint32_t* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch for the current device. The array's name in
// host code is only a host-side handle, so the address is looked up once per
// device with that device current.
cudaError_t scratch_on_current_device(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int ckks_rescale_noalloc(ckks_ctx* ctx, const uint32_t* in_dev, int level, uint32_t* out_dev) {
  if (!ctx || !in_dev || !out_dev) return CKKS_EINVAL;
  if (level < 1 || level >= ctx->dp.L) {
    ctx->err = "rescale_noalloc: level must be in [1, n_q - 1]";
    return CKKS_ELEVEL;
  }
  if (ctx->windowed) {
    ctx->err = "rescale_noalloc: single-rescaling levels only";
    return CKKS_EINVAL;
  }
  const size_t limb = (size_t)1 << ctx->dp.log_n;
  const size_t need = (2 + 2 * (size_t)level) * limb;  // top limb of both polys + level limbs of both
  if (need > kScratchWords) {
    ctx->err = "rescale_noalloc: (2 + 2 * level) * N = " + std::to_string(need) +
               " scratch words exceed the fixed maximum of " + std::to_string(kScratchWords);
    return CKKS_EINVAL;
  }
  // the array's address is per device: look it up on the context's device,
  // which must be the current one (its stream and buffers live there)
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device) {
    ctx->err = "rescale_noalloc: the current device (" + std::to_string(dev) + ") is not the context's device (" +
               std::to_string(ctx->device) + "); make the context's device current first";
    return CKKS_EINVAL;
  }
  uint32_t* base = nullptr;
  const cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) {
    ctx->err = std::string("rescale_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return CKKS_ECUDA;
  }
  // Every scratch word the kernels read is written earlier in the same call,
  // so nothing has to be cleared first.
  ckks::Scratch sc{};
  sc.S = base;
  sc.T = base + 2 * limb;
  const int n = level + 1;
  ckks::launch_rescale(ctx->dp, sc, in_dev, (size_t)n * limb, n, out_dev, (size_t)level * limb, ctx->stream);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    ctx->err = std::string("rescale_noalloc: ") + cudaGetErrorString(le);
    return CKKS_ECUDA;
  }
  return CKKS_OK;
}
