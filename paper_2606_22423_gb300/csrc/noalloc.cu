// Allocation-free scan entry point.
//
// Some callers cannot call cudaMalloc at scan time: latency-critical serving
// loops that must not take the allocator's implicit device synchronisation,
// engines that own a fixed memory budget and hand out memory only through
// their own sub-allocator, and plug-ins hosted by a process whose device
// memory belongs to another runtime.  For them this file keeps the full
// scan's grid-reduction scratch (one (count, sum) pair per CTA plus the
// last-CTA ticket) in a statically sized device array instead of a per-column
// workspace.
//
// The array lives at file scope, so every GPU that loads the library holds it
// until the process exits.  Host code cannot use its name as a device
// address; the entry point looks the address up with cudaGetSymbolAddress
// once per device (on its first call there, with that device current) and
// passes the looked-up pointer to the kernel.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/gbscan.h"
#include "scan_kernels.cuh"

#include "internal.h"

namespace {

// Scratch for at most kNoAllocMaxCtas CTAs: 64-byte header (ticket) plus two
// 64-bit words per CTA = 16 KiB + 64 B.  The scan uses one CTA per SM.
constexpr int kNoAllocMaxCtas = 1024;
constexpr size_t kNoAllocHeader = 64;
constexpr size_t kNoAllocBytes = kNoAllocHeader + 16 * kNoAllocMaxCtas;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

scan_status noalloc_fail(scan_status s, const char* msg)
{
    gb_set_last_error(msg);  // reported by scan_last_error()
    return s;
}

// Once per device: the scratch array's device address and the SM count.
scan_status setup_device(int dev, void** scratch, int* sms)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return noalloc_fail(SCAN_ECUDA, "cudaGetSymbolAddress(scratch) failed");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || n <= 0) return noalloc_fail(SCAN_ECUDA, "cannot read the SM count");
        g_sms[dev] = n;
        g_scratch_addr[dev] = p;
    }
    *scratch = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return SCAN_OK;
}

}  // namespace

extern "C" scan_status scan_run_packed_noalloc(const uint32_t* dev_packed, uint64_t n, uint32_t b,
                                               uint32_t base, scan_pred pred, scan_strategy strategy,
                                               void* stream, scan_result* dev_out, uint32_t* dev_status)
{
    gb_set_last_error("");
    if (!dev_out || !dev_status) return noalloc_fail(SCAN_EINVAL, "dev_out and dev_status are required");
    // the kernel stores 64-bit words to dev_out and a 32-bit word to dev_status:
    // a misaligned pointer would fault on the device, so refuse it here
    if (reinterpret_cast<uintptr_t>(dev_out) & 7u)
        return noalloc_fail(SCAN_EINVAL, "dev_out must be 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(dev_status) & 3u)
        return noalloc_fail(SCAN_EINVAL, "dev_status must be 4-byte aligned");
    if (b < 1 || b > 32 || static_cast<uint64_t>(base) + ((1ull << b) - 1ull) > 0xffffffffull)
        return noalloc_fail(SCAN_EINVAL, "bad width or frame-of-reference base");
    if (n > (1ull << 31)) return noalloc_fail(SCAN_EINVAL, "n exceeds the 2^31-value maximum");
    if (n && !dev_packed) return noalloc_fail(SCAN_EINVAL, "dev_packed is NULL");
    if (reinterpret_cast<uintptr_t>(dev_packed) & 15u)
        return noalloc_fail(SCAN_EINVAL, "dev_packed must be 16-byte aligned");
    int op;
    if (strategy == SCAN_AUTO || strategy == SCAN_BRANCHFREE) op = gb::kOpFullBF;
    else if (strategy == SCAN_BRANCHY) op = gb::kOpFullBR;
    else return noalloc_fail(SCAN_EINVAL, "only full-scan strategies run without allocation");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SCAN_ECUDA, "no usable current device");
    void* scratch = nullptr;
    int sms = 0;
    scan_status s = setup_device(dev, &scratch, &sms);
    if (s != SCAN_OK) return s;
    if (sms > kNoAllocMaxCtas)
        return noalloc_fail(SCAN_EINVAL, "this GPU needs more CTAs than the static scratch holds (1024)");

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(dev_status, 0, sizeof(uint32_t), st) != cudaSuccess)
        return noalloc_fail(SCAN_ECUDA, "cudaMemsetAsync(dev_status) failed");

    // predicate on decoded values -> code space; an empty range never launches
    const int64_t lo_v = static_cast<int64_t>(base);
    const int64_t hi_v = lo_v + (1ll << b);
    const int64_t lo = pred.lo > lo_v ? pred.lo : lo_v;
    const int64_t hi = pred.hi < hi_v ? pred.hi : hi_v;
    if (n == 0 || lo >= hi) {
        if (cudaMemsetAsync(dev_out, 0, sizeof(scan_result), st) != cudaSuccess)
            return noalloc_fail(SCAN_ECUDA, "cudaMemsetAsync(dev_out) failed");
        return SCAN_OK;
    }
    // the ticket must start at zero; a call that stopped early could leave it set
    if (cudaMemsetAsync(scratch, 0, kNoAllocHeader, st) != cudaSuccess)
        return noalloc_fail(SCAN_ECUDA, "cudaMemsetAsync(scratch) failed");

    gb::ScanParams p{};
    p.packed = dev_packed;
    p.n = n;
    p.base = base;
    p.lo = static_cast<uint32_t>(lo - lo_v);
    p.wm1 = static_cast<uint32_t>(hi - lo - 1);
    p.zlo = static_cast<uint64_t>(lo);
    p.zhi = static_cast<uint64_t>(hi);
    p.done = reinterpret_cast<unsigned int*>(scratch);
    p.partials = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(scratch) + kNoAllocHeader);
    p.status = dev_status;
    p.result = reinterpret_cast<long long*>(dev_out);
    const cudaError_t e = gb_launch(static_cast<int>(b), op, p, gb_shape_for(static_cast<int>(b), op), sms, st);
    if (e != cudaSuccess) return noalloc_fail(SCAN_ECUDA, cudaGetErrorString(e));
    return SCAN_OK;
}
