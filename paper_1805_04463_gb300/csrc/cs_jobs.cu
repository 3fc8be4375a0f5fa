// cs_jobs.cu -- counting slices of several causal sets in one launch.
//
// A set's interval count is a fixed list of work items (POPC tiles, FP8
// tensor-core tile slots, or FP4 pair supertile slots); cs_count_jobs runs
// any slice [item_begin, item_end)
// of any number of sets in one persistent launch and adds the counts into
// each set's histogram.  A scheduler can therefore advance many sets a
// little at a time, and sets that arrive later join the next launch: the
// counts are integer additions, so a set's final histogram does not depend
// on how its items were sliced or what they shared a launch with.
#include <cstring>

#include "cs_kernels.cuh"

using namespace cs;

namespace {

int jobs_path(int path) { return path == CS_PATH_AUTO ? batch_auto_path() : path; }

bool tensor_path(int path) { return path == CS_PATH_MMA || path == CS_PATH_MMA4; }

size_t entry_bytes(int path) { return tensor_path(path) ? sizeof(MmaSetEntry) : sizeof(PopcSetEntry); }

bool valid_path(int path) { return path >= CS_PATH_AUTO && path <= CS_PATH_MMA4; }

}  // namespace

extern "C" {

int64_t cs_count_items(int64_t n, int path) {
    if (n < 1 || n > kMaxN || !valid_path(path)) return -1;
    const int p = jobs_path(path);
    return p == CS_PATH_MMA ? mma_items(n) : p == CS_PATH_MMA4 ? mma4_units(n) : popc_tiles(n);
}

size_t cs_operands_bytes(int64_t n, int path) {
    if (n < 1 || n > kMaxN || !valid_path(path)) return 0;
    const int p = jobs_path(path);
    if (!tensor_path(p)) return 0;
    const bool fp4 = p == CS_PATH_MMA4;
    return align_up(mma_operand_bytes(n, fp4, 0), 1024) + mma_operand_bytes(n, fp4, 1);
}

int cs_prepare_operands(int64_t n, int path, const uint64_t* bits_dev, int64_t row_words, void* operands_dev,
                        size_t operands_bytes, void* stream) {
    CS_TRACE("cs_prepare_operands");
    if (n < 1 || n > kMaxN || !valid_path(path) || !tensor_path(jobs_path(path)) || !bits_dev ||
        row_words < cs_row_words(n) || row_words % 16 != 0 || !operands_dev ||
        (reinterpret_cast<uintptr_t>(operands_dev) % 1024) != 0)
        return CS_EINVAL;
    const bool fp4 = jobs_path(path) == CS_PATH_MMA4;
    if (operands_bytes < cs_operands_bytes(n, path)) return CS_ENOMEM;
    MmaSetEntry e;
    std::memset(static_cast<void*>(&e), 0, sizeof(e));
    e.bits = bits_dev;
    e.n = n;
    e.row_words = row_words;
    e.kpad = mma_kpad(n, fp4);
    e.op0 = static_cast<uint8_t*>(operands_dev);
    e.op1 = e.op0 + align_up(mma_operand_bytes(n, fp4, 0), 1024);
    return launch_expand_single(&e, static_cast<cudaStream_t>(stream), fp4) == cudaSuccess ? CS_OK : CS_ECUDA;
}

size_t cs_count_jobs_table_bytes(int n_jobs, int path) {
    if (n_jobs < 1 || !valid_path(path)) return 0;
    return entry_bytes(jobs_path(path)) * size_t(n_jobs);
}

size_t cs_count_jobs_workspace_bytes(int n_jobs, int path) {
    const size_t t = cs_count_jobs_table_bytes(n_jobs, path);
    return t ? sizeof(WsHeader) + t : 0;
}

int cs_count_jobs(const cs_count_job* jobs, int n_jobs, int path, void* table_host, void* workspace_dev,
                  size_t workspace_bytes, void* stream) {
    CS_TRACE("cs_count_jobs");
    if (!jobs || n_jobs < 1 || !valid_path(path) || !table_host || !workspace_dev ||
        (reinterpret_cast<uintptr_t>(workspace_dev) % 256) != 0 || (reinterpret_cast<uintptr_t>(table_host) % 128) != 0)
        return CS_EINVAL;
    const int p = jobs_path(path);
    if (tensor_path(p) && !device_has_tcgen05()) return CS_EUNSUPPORTED;
    if (workspace_bytes < cs_count_jobs_workspace_bytes(n_jobs, p)) return CS_ENOMEM;
    int64_t items = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const cs_count_job& b = jobs[j];
        const int64_t total = cs_count_items(b.n, p);
        if (b.n < 1 || b.n > kMaxN || !b.bits || b.row_words < cs_row_words(b.n) || b.row_words % 16 != 0 ||
            !b.hist || (reinterpret_cast<uintptr_t>(b.hist) % 8) != 0 || b.item_begin < 0 ||
            b.item_end < b.item_begin || b.item_end > total ||
            (tensor_path(p) && (!b.operands || (reinterpret_cast<uintptr_t>(b.operands) % 1024) != 0)))
            return CS_EINVAL;
        if (tensor_path(p)) {
            const bool fp4 = p == CS_PATH_MMA4;
            MmaSetEntry& e = static_cast<MmaSetEntry*>(table_host)[j];
            std::memset(static_cast<void*>(&e), 0, sizeof(e));
            uint8_t* op0 = static_cast<uint8_t*>(b.operands);
            uint8_t* op1 = op0 + align_up(mma_operand_bytes(b.n, fp4, 0), 1024);
            if (mma_fill_entry(&e, b.bits, b.n, b.row_words, op0, op1, fp4) != CUDA_SUCCESS) return CS_ECUDA;
            e.item_begin = items;
            e.item_offset = b.item_begin;
            e.hist_off = int64_t(reinterpret_cast<uintptr_t>(b.hist));
        } else {
            PopcSetEntry& e = static_cast<PopcSetEntry*>(table_host)[j];
            std::memset(static_cast<void*>(&e), 0, sizeof(e));
            popc_fill_entry(&e, b.bits, b.n, b.row_words);
            if (popc_encode_map(&e.map, b.bits, b.n, b.row_words) != CUDA_SUCCESS) return CS_ECUDA;
            e.item_begin = items;
            e.item_offset = b.item_begin;
            e.hist_off = int64_t(reinterpret_cast<uintptr_t>(b.hist));
        }
        items += b.item_end - b.item_begin;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader* hdr = static_cast<WsHeader*>(workspace_dev);
    void* table_dev = static_cast<uint8_t*>(workspace_dev) + sizeof(WsHeader);
    cudaError_t e = cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(table_dev, table_host, entry_bytes(p) * size_t(n_jobs), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return CS_ECUDA;
    if (items == 0) return CS_OK;
    // Entries with empty slices stay in the table; the item search skips them.
    if (p == CS_PATH_MMA)
        e = launch_count_mma_multi(static_cast<const MmaSetEntry*>(table_dev), n_jobs, items, 0, hdr, 0, st);
    else if (p == CS_PATH_MMA4)
        e = launch_count_mma4_multi(static_cast<const MmaSetEntry*>(table_dev), n_jobs, items, 0, hdr, st);
    else
        e = launch_count_popc_multi(static_cast<const PopcSetEntry*>(table_dev), n_jobs, items, 0, hdr, 0, st);
    return e == cudaSuccess ? CS_OK : CS_ECUDA;
}

}  // extern "C"
