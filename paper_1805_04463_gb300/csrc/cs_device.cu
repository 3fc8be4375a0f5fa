// cs_device.cu -- per-device properties and TMA descriptor encoding.
#include <cudaTypedefs.h>

#include <mutex>

#include "cs_kernels.cuh"

namespace cs {

namespace {

struct DevProps {
    int sm_count = 0;
    int major = 0, minor = 0;
    size_t total_mem = 0;
    bool valid = false;
};

DevProps g_props[64];
std::mutex g_mu;

const DevProps& props() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    DevProps& p = g_props[dev];
    if (!p.valid) {
        cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&p.major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&p.minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (p.sm_count < 1) p.sm_count = 1;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) p.total_mem = total_b;
        p.valid = true;
    }
    return p;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

}  // namespace

int device_sm_count() { return props().sm_count; }

size_t device_total_memory() { return props().total_mem; }

// The kernels are built for sm_103a only; tcgen05 is present on compute
// capability 10.x.
bool device_has_tcgen05() {
    const DevProps& p = props();
    return p.major == 10 && p.minor == 3;
}

CUresult encode_tensor_map_2d(CUtensorMap* map, CUtensorMapDataType type, void* base, uint64_t dim0,
                              uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                              CUtensorMapSwizzle swizzle) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return CUDA_ERROR_NOT_FOUND;
    const cuuint64_t dims[2] = {dim0, dim1};
    const cuuint64_t strides[1] = {stride1_bytes};
    const cuuint32_t box[2] = {box0, box1};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(map, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace cs
