// cs_kernels.cuh -- launchers shared between the translation units of the library.
#pragma once

#include "cs_internal.cuh"

namespace cs {

// cs_sprinkle.cu
size_t sprinkle_workspace_bytes(int64_t n);
cudaError_t launch_sprinkle(int kind, int64_t n, uint64_t seed, int32_t* coords, void* workspace,
                            cudaStream_t st);

// cs_relate.cu
cudaError_t launch_relate(int kind, int64_t n, const int32_t* coords, uint64_t* bits, int64_t row_words,
                          cudaStream_t st);

// cs_count_popc.cu
size_t popc_workspace_bytes(int64_t n);
cudaError_t launch_count_popc(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist,
                              void* workspace, cudaStream_t st);

// cs_count_mma.cu
size_t mma_workspace_bytes(int64_t n);
cudaError_t launch_count_mma(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist,
                             void* workspace, cudaStream_t st);

// Path chosen for CS_PATH_AUTO at size n.
int resolve_path(int64_t n, int path);

// cs_action.cu
int action_host(int dim, int64_t n, const int64_t* hist, int64_t len, double eps, double* out,
                int64_t* bracket);
size_t action_workspace_bytes();
cudaError_t launch_action_device(int dim, int64_t n, const int64_t* hist, int64_t len, const double* eps,
                                 int n_eps, double* out, int64_t* bracket, void* workspace, cudaStream_t st);

// Device properties cached per device.
int device_sm_count();
bool device_has_tcgen05();

// cuTensorMapEncodeTiled, resolved once through the runtime's driver entry point.
CUresult encode_tensor_map_2d(CUtensorMap* map, CUtensorMapDataType type, void* base, uint64_t dim0,
                              uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                              CUtensorMapSwizzle swizzle);

}  // namespace cs
