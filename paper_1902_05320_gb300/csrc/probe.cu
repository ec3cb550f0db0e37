// probe.cu -- diagnostics beside the hashing path:
//
// * the integer-issue microbenchmark behind the ALU roofline: each thread
//   keeps eight 32-bit values and, per round, computes eight new ones, each
//   from three values of the previous round with one instruction of the kind
//   measured (LOP3 with the chi table 0xD2, a funnel shift whose amount comes
//   from a register, PRMT with a register selector, or a three-input add).
//   Every output depends on three loop-carried inputs and no two rounds can
//   be merged into one instruction (chi is not linear; the shift amount and
//   selector change every round), so the compiler issues exactly one
//   instruction per output, which ncu's smsp__inst_executed confirms.  Every
//   block of a one-wave grid reads its SM's clock before and after, and the
//   SM's span is its earliest start to its latest end: the blocks of an SM do
//   not finish together (the lower hardware warp slots issue first), so an
//   average of per-block durations would undercount the cycles.  Lanes per
//   clock per SM = (thread-instructions issued on the SM) / its span;
// * the bounded mbarrier wait of the staging kernel, run on a barrier whose
//   phase nothing completes, so that its give-up path (KB_DEV_TIMEOUT in the
//   device status word, then return) is exercised without a fault.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "runtime.cuh"
#include "tma.cuh"

namespace kb {
namespace {

constexpr int kProbeThreads = 256;

template <int OP>
__device__ __forceinline__ uint32_t probe_op(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    if constexpr (OP == 0) asm volatile("lop3.b32 %0, %1, %2, %3, 0xD2;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    else if constexpr (OP == 1) asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    else if constexpr (OP == 2) asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    else asm volatile("add.u32 %0, %1, %2;\n\tadd.u32 %0, %0, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads)
    k_int_probe(uint32_t iters, uint32_t seed, uint32_t *sink, long long *stamps) {
    uint32_t a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed * (threadIdx.x + 1) + 0x9E3779B9u * (j + 1) + blockIdx.x;
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 4
    for (uint32_t i = 0; i < iters; ++i) {
        uint32_t b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = probe_op<OP>(a[j], a[(j + 1) & 7], a[(j + 3) & 7]);
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = b[j];
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x ^= a[j];
    if (x == 0x12345678u) sink[blockIdx.x] = x;  // keeps the chains live
    if (threadIdx.x == 0) {
        unsigned smid;
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        stamps[3 * blockIdx.x + 0] = t0;
        stamps[3 * blockIdx.x + 1] = t1;
        stamps[3 * blockIdx.x + 2] = smid;
    }
}

template <int OP>
int run_probe(uint32_t iters, double *lanes_per_clk, cudaStream_t stream, const DeviceInfo &dev) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_int_probe<OP>, kProbeThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return KB_ERR_CUDA;
    const int grid = per_sm * dev.sm_count;
    uint32_t *sink = nullptr;
    long long *stamps = nullptr;
    if (cudaMalloc(&sink, sizeof(uint32_t) * grid) != cudaSuccess) return KB_ERR_NOMEM;
    if (cudaMalloc(&stamps, 3 * sizeof(long long) * grid) != cudaSuccess) {
        cudaFree(sink);
        return KB_ERR_NOMEM;
    }
    k_int_probe<OP><<<grid, kProbeThreads, 0, stream>>>(iters, 12345u, sink, stamps);
    std::vector<long long> h(3 * size_t(grid));
    int rc = cuda_status(cudaGetLastError());
    if (rc == KB_OK) rc = cuda_status(cudaMemcpyAsync(h.data(), stamps, 3 * sizeof(long long) * grid,
                                                      cudaMemcpyDeviceToHost, stream));
    if (rc == KB_OK) rc = cuda_status(cudaStreamSynchronize(stream));
    cudaFree(sink);
    cudaFree(stamps);
    if (rc != KB_OK) return rc;
    // Per SM: its blocks' thread-instructions over its earliest start to latest end.
    std::map<long long, std::tuple<long long, long long, double>> sms;  // smid -> (first, last, instructions)
    const double per_block = double(iters) * 8.0 * kProbeThreads;
    for (int b = 0; b < grid; ++b) {
        const long long t0 = h[3 * b], t1 = h[3 * b + 1], sm = h[3 * b + 2];
        auto it = sms.find(sm);
        if (it == sms.end()) {
            sms[sm] = std::make_tuple(t0, t1, per_block);
        } else {
            auto &[first, last, instr] = it->second;
            first = std::min(first, t0);
            last = std::max(last, t1);
            instr += per_block;
        }
    }
    double sum = 0;
    for (const auto &kv : sms) {
        const auto &[first, last, instr] = kv.second;
        sum += instr / double(std::max<long long>(1, last - first));
    }
    *lanes_per_clk = sms.empty() ? 0.0 : sum / double(sms.size());
    return KB_OK;
}

// One thread initialises a shared-memory mbarrier for one arrival.  With
// arrive == 0 nothing ever arrives, so phase 0 never completes and the
// staging kernel's bounded wait gives up after limit_ns; with arrive == 1 the
// thread arrives first and the wait returns at once.  No copy or other
// asynchronous operation is in flight either way, so returning is safe.
__global__ void k_wait_probe(uint64_t limit_ns, int arrive, unsigned int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_barrier_init();
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(status, KB_DEV_TIMEOUT);
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" int sha3gb_wait_timeout_probe(uint64_t limit_ns, int arrive, void *stream) {
    if (limit_ns == 0 || limit_ns > 2000000000ull || (arrive != 0 && arrive != 1)) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    k_wait_probe<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns, arrive, dev->d_status);
    return cuda_status(cudaGetLastError());
}

extern "C" int sha3gb_int_issue_probe(int op, uint32_t iters, double *lanes_per_clk_per_sm, void *stream) {
    if (!lanes_per_clk_per_sm || op < 0 || op > 3 || iters == 0) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (op) {
        case 0: return run_probe<0>(iters, lanes_per_clk_per_sm, s, *dev);
        case 1: return run_probe<1>(iters, lanes_per_clk_per_sm, s, *dev);
        case 2: return run_probe<2>(iters, lanes_per_clk_per_sm, s, *dev);
        default: return run_probe<3>(iters, lanes_per_clk_per_sm, s, *dev);
    }
}
