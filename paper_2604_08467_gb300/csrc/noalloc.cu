// ptn_sample_block_noalloc: the NBS sampling step of ptn_sample_block with its
// scratch memory in a fixed, statically allocated device array instead of
// memory the library allocates at run time.
//
// Some callers cannot allocate device memory while they run this step: code
// that executes inside a pre-reserved memory budget (a serving process that
// carved the GPU up at start-up and forbids later cudaMalloc/cudaFree, which
// also synchronise the device), or code holding a caching allocator that must
// not be bypassed.  This entry point touches only the caller's inputs and
// outputs plus the array below, which every GPU that loads the library holds
// until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {
void clear_error();
namespace {

// Scratch shared by every call (any stream) on a device.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device with that device
// current (in host code the symbol name only stands in for it).  The lookup
// runs under a mutex; later calls read the published pointer atomically.
constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int dev, void** out) {
    void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lk(g_scratch_mutex);
        p = g_scratch_ptr[dev].load(std::memory_order_relaxed);
        if (!p) {
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            if (!p) return cudaErrorInvalidSymbol;
            g_scratch_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return cudaSuccess;
}

// Checks that parents are grouped by (non-decreasing) trajectory and finds the
// largest trajectory index; out[0] = max index, out[1] = 1 if unsorted or negative.
__global__ void k_check_parents(const int32_t* __restrict__ traj, int64_t n, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = traj[i];
        atomicMax(&out[0], t);
        if (t < 0 || (i > 0 && traj[i - 1] > t)) atomicExch(&out[1], 1);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace ptn

using namespace ptn;

extern "C" ptn_status ptn_sample_block_noalloc(const float* marg, int32_t b, int32_t start,
                                               const int32_t* parent_traj, const uint64_t* parent_prefix,
                                               const int64_t* parent_count, int64_t n_parent, uint64_t seed,
                                               int32_t circuit_id, int32_t block, int32_t* child_traj,
                                               uint64_t* child_prefix, int64_t* child_count, int64_t child_cap,
                                               int64_t* n_child, ptn_stream stream) {
    clear_error();
    if (!n_child || b < 1 || b > 14 || start < 0 || start + b > 64 || n_parent < 0 || child_cap < 0)
        return set_error(PTN_ERR_INVALID_ARG, "bad sampling arguments (b must be 1..14)");
    *n_child = 0;
    if (n_parent == 0) return PTN_OK;
    if (!marg || !parent_traj || !parent_prefix || !parent_count || !child_traj || !child_prefix || !child_count)
        return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    // The array used is the one of the current device, which must also be the
    // device the stream belongs to.
    int dev = 0, sdev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(PTN_ERR_UNSUPPORTED, "device index %d", dev);
    if (s) {
        e = cudaStreamGetDevice(s, &sdev);
        if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "cudaStreamGetDevice: %s", cudaGetErrorString(e));
        if (sdev != dev)
            return set_error(PTN_ERR_INVALID_ARG, "stream belongs to device %d but device %d is current", sdev, dev);
    }
    void* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    unsigned char* base = static_cast<unsigned char*>(scratch);

    // Layout of the scratch for this call; everything must fit the fixed array.
    const size_t np = sizeof(int64_t) * (size_t)n_parent;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_check = take(2 * sizeof(int32_t));
    const size_t o_cap = take(np), o_tmp_off = take(np), o_rank0 = take(np), o_excl = take(np);
    const size_t o_ndist = take(np), o_out_off = take(np);
    const size_t o_scan = take(sizeof(int64_t) * (size_t)scan_tmp_elems(n_parent));
    const size_t fixed = off;
    if (fixed > kNoAllocScratchBytes)
        return set_error(PTN_ERR_TOO_LARGE, "ptn_sample_block_noalloc: %lld parents exceed the %zu-byte scratch",
                         (long long)n_parent, kNoAllocScratchBytes);

    // Validate the parent list on the device; the result comes back through a
    // host variable of this function (no allocation).
    int32_t* chk = reinterpret_cast<int32_t*>(base + o_check);
    int32_t h_chk[2] = {0, 0};
    e = cudaMemsetAsync(chk, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) {
        int64_t blocks = (n_parent + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        count_launches(K_MISC);
        k_check_parents<<<(unsigned)blocks, 256, 0, s>>>(parent_traj, n_parent, chk);
        e = cudaMemcpyAsync(h_chk, chk, sizeof h_chk, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "parent check: %s", cudaGetErrorString(e));
    if (h_chk[1]) return set_error(PTN_ERR_INVALID_ARG, "parents must be grouped by non-negative trajectory");
    const int64_t n_traj = (int64_t)h_chk[0] + 1;

    const size_t o_first = take(sizeof(int64_t) * (size_t)n_traj);
    const size_t o_tmp_x = take(sizeof(int32_t) * (size_t)child_cap);
    const size_t o_tmp_c = take(sizeof(int64_t) * (size_t)child_cap);
    if (off > kNoAllocScratchBytes)
        return set_error(PTN_ERR_TOO_LARGE,
                         "ptn_sample_block_noalloc: %lld parents, %lld trajectories and %lld child slots need %zu "
                         "bytes of scratch, more than the %zu-byte maximum",
                         (long long)n_parent, (long long)n_traj, (long long)child_cap, off, kNoAllocScratchBytes);

    SampleScratch sc;
    sc.cap = reinterpret_cast<int64_t*>(base + o_cap);
    sc.tmp_off = reinterpret_cast<int64_t*>(base + o_tmp_off);
    sc.rank0 = reinterpret_cast<int64_t*>(base + o_rank0);
    sc.excl = reinterpret_cast<int64_t*>(base + o_excl);
    sc.first = reinterpret_cast<int64_t*>(base + o_first);
    sc.ndist = reinterpret_cast<int64_t*>(base + o_ndist);
    sc.out_off = reinterpret_cast<int64_t*>(base + o_out_off);
    sc.tmp_x = reinterpret_cast<int32_t*>(base + o_tmp_x);
    sc.tmp_c = reinterpret_cast<int64_t*>(base + o_tmp_c);
    sc.scan_tmp = reinterpret_cast<int64_t*>(base + o_scan);
    int64_t host_tmp[4] = {0, 0, 0, 0};   // sizes read back by the sampling step
    ptn_status st;
    const int64_t nc = run_sample_block(marg, b, start, parent_traj, parent_prefix, parent_count, n_parent, n_traj,
                                        seed, circuit_id, block, child_traj, child_prefix, child_count, child_cap, sc,
                                        host_tmp, s, &st);
    if (st != PTN_OK) return st;
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "sampling: %s", cudaGetErrorString(e));
    *n_child = nc;
    return PTN_OK;
}
