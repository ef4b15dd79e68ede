// Serving: expands an admission's compact split references into the decode
// kernel's descriptors on the device. The serving loop keeps every pool
// stream's descriptors resident (built and uploaded once before the run); an
// admission sends one 16-byte reference per kept split (which descriptor, the
// owned low end the combine gave it, the request's place in the launch)
// instead of the 288-byte descriptor itself, so the host writes and the link
// carries 18 times less per split.
#include "recoil_internal.h"

namespace recoil {
namespace {

static_assert(sizeof(DevEntry) == 18 * 16, "a descriptor is 18 16-byte words");
static_assert(offsetof(DevEntry, lo) == 8 && offsetof(DevEntry, stream) == 17 * 16,
              "the patched fields sit in the first and the last 16-byte word");

// One warp per descriptor: lanes 0..17 copy its 16-byte words, patching the
// owned low end (word 0) and the stream index (word 17).
__global__ void __launch_bounds__(256) expand_entries_kernel(const DevEntry* __restrict__ pool,
                                                             const EntryRef* __restrict__ refs,
                                                             DevEntry* __restrict__ out, uint32_t n) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (w >= n || lane >= 18) return;
  const EntryRef r = refs[w];
  uint4 v = reinterpret_cast<const uint4*>(pool + r.src)[lane];
  if (lane == 0) v.z = r.lo;
  if (lane == 17) v.x = r.stream;
  reinterpret_cast<uint4*>(out + w)[lane] = v;
}

}  // namespace

cudaError_t launch_expand_entries(const DevEntry* pool, const EntryRef* refs, DevEntry* out, uint32_t n,
                                  cudaStream_t s) {
  if (!n) return cudaSuccess;
  const unsigned blocks = (unsigned)(((uint64_t)n * 32 + 255) / 256);
  expand_entries_kernel<<<blocks, 256, 0, s>>>(pool, refs, out, n);
  return cudaGetLastError();
}

}  // namespace recoil
