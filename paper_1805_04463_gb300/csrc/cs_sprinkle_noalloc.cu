// cs_sprinkle_noalloc.cu -- cs_sprinkle for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they sprinkle: code
// running while a stream is being captured into a CUDA graph (allocation
// calls are not allowed there), plugins that may only use memory handed to
// them by a host application, or real-time loops that must not touch the
// allocator.  This entry point takes only the output buffer: its scratch
// (random keys, ranks, bucket tables -- what cs_sprinkle keeps in the caller's
// workspace) lives in one file-scope device array of fixed size, which every
// GPU that loads the library holds until the process exits.
//
// Limits and sharing: n is at most CS_SPRINKLE_NOALLOC_MAX_N.  All calls on a
// device share the one array; each call clears the parts that must start at
// zero, and the array keeps the last call's contents afterwards.  Two calls
// whose work overlaps on the GPU (different streams without ordering between
// them) race on the array and may corrupt each other's result.  The first
// call on a device looks up the array's device address (and, for the de
// Sitter slab, uploads that kind's constant table); make that first call
// before any stream capture begins.  The in-kernel status word (set only if
// a 3D or 4D element exhausts its 16384 rejection attempts, which has
// probability below 1e-900) lands in the array and is not reported by this
// entry point.
#include <mutex>

#include "cs_kernels.cuh"

namespace cs {
namespace {

constexpr int kMaxDevices = 64;
// Scratch for n <= CS_SPRINKLE_NOALLOC_MAX_N (the same layout cs_sprinkle
// uses in a caller's workspace).
constexpr size_t kScratchBytes = size_t(12) << 20;

static __device__ __align__(256) uint8_t g_sprinkle_scratch[kScratchBytes];

// Device address of g_sprinkle_scratch, looked up once per device with that
// device current (in host code the symbol's name is only a host-side
// stand-in, not a device address).
void* g_scratch_ptr[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

cudaError_t scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_scratch_once[dev], [dev] {
        void* p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_sprinkle_scratch);
        g_scratch_ptr[dev] = g_scratch_err[dev] == cudaSuccess ? p : nullptr;
    });
    if (g_scratch_err[dev] != cudaSuccess) return g_scratch_err[dev];
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" int cs_sprinkle_noalloc(int kind, int64_t n, uint64_t seed, int32_t* coords_dev, void* stream) {
    CS_TRACE("cs_sprinkle_noalloc");
    if (cs_dim(kind) == 0 || n < 1 || n > CS_SPRINKLE_NOALLOC_MAX_N || !coords_dev ||
        (reinterpret_cast<uintptr_t>(coords_dev) % 4) != 0)
        return CS_EINVAL;
    static_assert(CS_SPRINKLE_NOALLOC_MAX_N <= kMaxN, "limit within the ABI's range");
    if (sprinkle_workspace_bytes(CS_SPRINKLE_NOALLOC_MAX_N) > kScratchBytes) return CS_ENOMEM;
    void* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return CS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(&static_cast<WsHeader*>(scratch)->status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_sprinkle(kind, n, seed, coords_dev, scratch, st);
    return e == cudaSuccess ? CS_OK : CS_ECUDA;
}
