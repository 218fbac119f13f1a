// Uniform sample of k distinct nodes on the device (section 2: "sample k
// points uniformly at random"; Algorithm 1, first step): node v is keyed by
// splitmix64 output number v of the stream `seed` (Steele, Lea and Flood
// 2014) and the sample is the k nodes with the smallest (key, v), in that
// order -- bottom-k sampling, uniform without replacement.
//
// Selection: every node whose key is below a threshold chosen to admit
// about 2k + 64 candidates is appended to a candidate buffer; one CTA sorts
// the candidates with a shared-memory bitonic network and keeps the first k.
// The host widens or narrows the threshold and retries if the candidate count
// falls outside [k, capacity].
#include <cmath>
#include <cstdint>

#include "cc_internal.h"

namespace ccg {

namespace {

constexpr int kCap = 8192;        // candidate capacity (power of two)
constexpr int kSortThreads = 1024;

struct Cand {
    uint64_t key;
    uint32_t v;
    uint32_t pad_;
};

__global__ void k_candidates(int64_t n, uint64_t seed, uint64_t thr, Cand *buf,
                             unsigned *count)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = splitmix64_out(seed, (uint64_t)v);
        if (key <= thr) {
            const unsigned pos = atomicAdd(count, 1u);
            if (pos < (unsigned)kCap) buf[pos] = Cand{key, (uint32_t)v, 0u};
        }
    }
}

__device__ __forceinline__ bool cand_less(const Cand &a, const Cand &b)
{
    return a.key < b.key || (a.key == b.key && a.v < b.v);
}

__global__ void __launch_bounds__(kSortThreads)
k_sort_take(const Cand *buf, const unsigned *count, int k, int32_t *out)
{
    extern __shared__ Cand s[];
    const unsigned m = min(*count, (unsigned)kCap);
    int P = 1;
    while (P < (int)m) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        s[i] = i < (int)m ? buf[i] : Cand{~0ull, 0xFFFFFFFFu, 0u};
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const bool swap = up ? cand_less(s[j], s[i]) : cand_less(s[i], s[j]);
                    if (swap) { const Cand t = s[i]; s[i] = s[j]; s[j] = t; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) out[i] = (int32_t)s[i].v;
}

}  // namespace

size_t sample_candidate_bytes() { return sizeof(Cand) * kCap; }

int choose_sample_ws(int64_t n, int k, uint64_t seed, int32_t *host_out, void *cand_buf,
                     unsigned *cnt, int32_t *dout, cudaStream_t st)
{
    Cand *buf = static_cast<Cand *>(cand_buf);
    int rc = CC_ERR_TOO_LARGE;  // until a selection succeeds
    // Expected candidates: n * thr / 2^64.
    double frac = (2.0 * k + 64.0) / (double)n;
    for (int attempt = 0; attempt < 64; ++attempt) {
        const uint64_t thr = frac >= 1.0 ? ~0ull : (uint64_t)std::ldexp(frac, 64);
        if (cudaMemsetAsync(cnt, 0, 4, st) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
        int64_t grid = (n + 255) / 256;
        if (grid > 152 * 16) grid = 152 * 16;
        k_candidates<<<(int)grid, 256, 0, st>>>(n, seed, thr, buf, cnt);
        unsigned c = 0;
        if (cudaMemcpyAsync(&c, cnt, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = CC_ERR_CUDA;
            break;
        }
        if (c < (unsigned)k) {
            if (frac >= 1.0) { rc = CC_ERR_ARG; break; }
            frac = std::min(1.0, frac * 2.0);
            continue;
        }
        if (c > (unsigned)kCap) {
            frac *= 0.5 * (double)kCap / (double)c;
            continue;
        }
        int P = 1;
        while (P < (int)c) P <<= 1;
        const size_t smem = sizeof(Cand) * (size_t)P;
        if (cudaFuncSetAttribute(k_sort_take, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(Cand) * kCap)) != cudaSuccess) {
            rc = CC_ERR_CUDA;
            break;
        }
        k_sort_take<<<1, kSortThreads, smem, st>>>(buf, cnt, k, dout);
        rc = cudaMemcpyAsync(host_out, dout, (size_t)k * 4, cudaMemcpyDeviceToHost, st) ==
                             cudaSuccess &&
                     cudaStreamSynchronize(st) == cudaSuccess
                 ? CC_OK
                 : CC_ERR_CUDA;
        break;
    }
    cudaGetLastError();
    return rc;
}

int choose_sample_device(int64_t n, int k, uint64_t seed, int32_t *host_out)
{
    Cand *buf = nullptr;
    unsigned *cnt = nullptr;
    int32_t *dout = nullptr;
    if (cudaMalloc(&buf, sizeof(Cand) * kCap) != cudaSuccess ||
        cudaMalloc(&cnt, 4) != cudaSuccess || cudaMalloc(&dout, (size_t)k * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf); cudaFree(cnt); cudaFree(dout);
        return CC_ERR_OOM;
    }
    const int rc = choose_sample_ws(n, k, seed, host_out, buf, cnt, dout, 0);
    cudaFree(buf);
    cudaFree(cnt);
    cudaFree(dout);
    return rc;
}

}  // namespace ccg

extern "C" int cc_sample_choose(cc_graph_t g, int32_t k, uint64_t seed, int32_t *sample_out)
{
    int64_t n = 0;
    if (!g || !sample_out || cc_graph_info(g, &n, nullptr, nullptr, nullptr) != CC_OK)
        return CC_ERR_ARG;
    if (k < 1 || k > CC_MAX_K || k > n) return CC_ERR_ARG;
    return ccg::choose_sample_device(n, k, seed, sample_out);
}
