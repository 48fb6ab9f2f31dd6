// noalloc.cu -- mafp_build_stencils_noalloc: the stencil build without a
// context, for callers that cannot allocate device memory.
//
// Its only scratch (the queue of particles redone in FP64 and a few counters)
// lives in one file-scope __device__ array of fixed size, which exists on
// every GPU that loads this library until the process exits.
#include <math.h>
#include <string.h>

#include <atomic>

#include "internal.cuh"

namespace mafp {
int build_stencils(mafp_ctx *, int64_t, int32_t, const void *, const uint8_t *, const void *,
                   const int64_t *, const int32_t *, void *, uint8_t *, float *, cudaStream_t);
}  // namespace mafp

using namespace mafp;

namespace {

constexpr int64_t kNoAllocMaxParticles = MAFP_NOALLOC_MAX_PARTICLES;

struct NoAllocScratch {
  DevStatus status;                        // counters; the queue length lives here
  int32_t queue[kNoAllocMaxParticles];     // particles whose stencil is redone in FP64
};

// The scratch.  In host code this name is only a stand-in for the device
// object: its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::atomic<NoAllocScratch *> g_scratch_addr[kMaxDevices];

// Device address of the scratch on the current device (looked up once per
// device, with that device current).  Returns nullptr on failure.
NoAllocScratch *scratch_on_current_device(int *dev_out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  *dev_out = dev;
  NoAllocScratch *p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (p) return p;
  void *addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr)
    return nullptr;
  p = static_cast<NoAllocScratch *>(addr);
  g_scratch_addr[dev].store(p, std::memory_order_release);
  return p;
}

}  // namespace

extern "C" int mafp_build_stencils_noalloc(int64_t n, int32_t dtype, const mafp_params *params,
                                           const void *pos_h, const uint8_t *model,
                                           const void *frame, const int64_t *row_ptr,
                                           const int32_t *col, void *coef, uint8_t *status,
                                           float *cond, void *stream) {
  if (dtype != MAFP_F32_REFINED && dtype != MAFP_F32_PLAIN && dtype != MAFP_F64)
    return MAFP_EINVAL;
  if (n < 0) return MAFP_EINVAL;
  if (n > kNoAllocMaxParticles) return MAFP_ECAPACITY;
  if (n == 0) return MAFP_OK;
  if (!pos_h || !model || !frame || !row_ptr || !col || !coef || !status || !cond)
    return MAFP_EINVAL;
  int dev = 0;
  NoAllocScratch *scr = scratch_on_current_device(&dev);
  if (!scr) return MAFP_ECUDA;
  // A context on the stack whose only scratch pointers lead into the static
  // array; nothing here allocates.
  mafp_ctx c;
  memset(&c, 0, sizeof(c));
  if (params) c.prm = *params; else mafp_default_params(&c.prm);
  default_tuning(&c.tune);
  c.cap_particles = kNoAllocMaxParticles;
  c.device = dev;
  c.fallback = scr->queue;
  c.d_status = &scr->status;
  return build_stencils(&c, n, dtype, pos_h, model, frame, row_ptr, col, coef, status, cond,
                        (cudaStream_t)stream);
}
