// cs_selftest.cu -- failure-detection checks that need no GPU fault.
//
// cs_selftest_wait launches one warp that waits on an mbarrier nothing will
// complete, through the same bounded-wait code path the pipelines use but
// with a caller-chosen short limit; the wait gives up, records CS_ETIMEOUT in
// the workspace status word and the kernel returns normally, so the context
// stays usable.  cs_inject_fault makes chosen host-side steps of the library
// fail as if the CUDA call behind them had failed, to test error propagation.
#include <atomic>

#include "cs_kernels.cuh"

namespace cs {

namespace {

std::atomic<int> g_fault_mask{0};
std::atomic<int> g_fault_count{0};

__global__ void k_wait_probe(WsHeader* hdr, unsigned long long limit_ns, int complete) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (complete && threadIdx.x == 0) mbar_arrive(&bar);
    __syncwarp();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = global_timer_ns();
        mbar_wait_bounded(&bar, 0, hdr, limit_ns);  // records CS_ETIMEOUT on expiry
        hdr->aux[0] = global_timer_ns() - t0;       // time spent waiting
    }
}

}  // namespace

bool fault_injected(int where) {
    if (!(g_fault_mask.load() & where)) return false;
    if (g_fault_count.fetch_sub(1) <= 0) {
        g_fault_count.store(0);
        return false;
    }
    return true;
}

}  // namespace cs

using namespace cs;

extern "C" int cs_selftest_wait(void* workspace_dev, double limit_s, int complete, void* stream) {
    if (!workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) % 256) != 0 || !(limit_s > 0.0) ||
        limit_s > 10.0)
        return CS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader* hdr = static_cast<WsHeader*>(workspace_dev);
    if (cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st) != cudaSuccess) return CS_ECUDA;
    k_wait_probe<<<1, 32, 0, st>>>(hdr, static_cast<unsigned long long>(limit_s * 1e9), complete ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? CS_OK : CS_ECUDA;
}

extern "C" int cs_inject_fault(int where, int count) {
    if (where < 0 || count < 0) return CS_EINVAL;
    g_fault_count.store(count);
    g_fault_mask.store(count > 0 ? where : 0);
    return CS_OK;
}
