// Sampling and pivot statistics without any allocation.
//
// Some callers cannot allocate device memory: code running inside a
// framework whose memory pool owns the whole device, or a process under a
// strict memory budget where a cudaMalloc/cudaFree pair would synchronise the
// device or fail at an unpredictable moment.  For them this entry point runs
// the first traversal pass of cc_estimate (sums of distances, pivots, Delta,
// exact S of the sampled nodes) with every working buffer carved out of one
// fixed device array declared in this file.  The caller passes the graph and
// the outputs as device memory it already owns and the sample as host memory.
//
// The array costs kNoAllocScratchBytes of device memory on every GPU that
// loads the library, held until the process exits.  All calls share it and
// it keeps the contents of the last call: every region a call needs zeroed is
// cleared by that call.  Two calls that overlap on the GPU (different streams
// or threads, in flight at the same time) race on the array and must not be
// issued.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "cc_internal.h"
#include "estimate.h"

namespace ccg {
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kNoAllocHistLevels = 2048;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// is only a host-side stand-in; the real address comes from
// cudaGetSymbolAddress with that device current.
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CC_ERR_NO_DEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) return CC_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CC_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return CC_OK;
}

// Checks the caller's CSR before any traversal touches it.
__global__ void k_check_csr(int64_t n, const int64_t *rp, const int32_t *col, int64_t arcs,
                            int *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t v = t; v < n; v += stride)
        if (rp[v] > rp[v + 1] || rp[v] < 0 || rp[v + 1] > arcs) atomicExch(err, CC_ERR_GRAPH);
    for (int64_t e = t; e < arcs; e += stride)
        if (col[e] < 0 || col[e] >= n) atomicExch(err, CC_ERR_GRAPH);
}

// In-degrees (indeg zeroed by the caller); out-of-range columns are left to
// k_check_csr's report.
__global__ void k_in_degree(int64_t n, const int32_t *col, int64_t arcs, int32_t *indeg)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < arcs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = col[e];
        if (c >= 0 && c < n) atomicAdd(&indeg[c], 1);
    }
}

// A symmetric CSR has every node's in-degree equal to its out-degree (a
// necessary condition only: it catches a directed CSR, not every error).
__global__ void k_degree_match(int64_t n, const int64_t *rp, const int32_t *indeg, int *err)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (rp[v + 1] - rp[v] != (int64_t)indeg[v]) atomicExch(err, CC_ERR_GRAPH);
}

__global__ void k_iota(int32_t *p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

// sample index per node; a repeated node sets CC_ERR_ARG.
__global__ void k_sidx_checked(int32_t *sidx, const int32_t *src, int k, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k && atomicCAS(&sidx[src[i]], -1, i) != -1) atomicExch(err, CC_ERR_ARG);
}

__global__ void k_take_sum(const uint64_t *sum2, uint64_t *out, int64_t n)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = sum2[2 * v];
}

struct Carve {
    unsigned char *base;
    size_t off = 0;
    template <class T> T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

int grid_of(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace ccg

using namespace ccg;

extern "C" int cc_sampling_pivots_noalloc(int64_t n, const int64_t *d_row_ptr,
                                          const int32_t *d_col, const int32_t *sample,
                                          int32_t k, uint64_t *d_sample_sum,
                                          int32_t *d_pivot, uint32_t *d_delta,
                                          uint64_t *d_S_sampled, void *stream)
{
    if (n < 2 || !d_row_ptr || !d_col || !sample || !d_sample_sum || !d_pivot ||
        !d_delta || !d_S_sampled)
        return CC_ERR_ARG;
    if (k < 1 || k > CC_MAX_K || k > n) return CC_ERR_ARG;
    for (int i = 0; i < k; ++i)
        if (sample[i] < 0 || sample[i] >= n) return CC_ERR_ARG;
    int W = 1;
    while (W * 64 < k) W <<= 1;
    const int hist_cap = (int)(n + 1 < kNoAllocHistLevels ? n + 1 : kNoAllocHistLevels);

    // Size check first: nothing is touched when the call does not fit.
    {
        Carve c{nullptr};
        for (int i = 0; i < 4; ++i) c.take<uint64_t>((size_t)n * W);
        for (int i = 0; i < 9; ++i) c.take<int32_t>((size_t)n);
        c.take<uint64_t>((size_t)n * 2);
        c.take<uint32_t>((size_t)k * k);
        c.take<uint32_t>((size_t)hist_cap * k);
        c.take<int32_t>((size_t)k);
        c.take<Ctl>(1);
        c.take<int>(1);
        if (c.off > kNoAllocScratchBytes) return CC_ERR_TOO_LARGE;
    }
    unsigned char *base = nullptr;
    const int rc0 = scratch_on_current_device(&base);
    if (rc0 != CC_OK) return rc0;
    cudaStream_t st = (cudaStream_t)stream;

    Carve c{base};
    uint64_t *vis = c.take<uint64_t>((size_t)n * W);
    uint64_t *F0 = c.take<uint64_t>((size_t)n * W);
    uint64_t *F1 = c.take<uint64_t>((size_t)n * W);
    uint64_t *nxt = c.take<uint64_t>((size_t)n * W);
    int32_t *Q0 = c.take<int32_t>((size_t)n);
    int32_t *Q1 = c.take<int32_t>((size_t)n);
    int32_t *T = c.take<int32_t>((size_t)n);
    unsigned *tflag = c.take<unsigned>((size_t)n);
    int32_t *sidx = c.take<int32_t>((size_t)n);
    int32_t *Llist = c.take<int32_t>((size_t)n);
    int32_t *AL0 = c.take<int32_t>((size_t)n);
    int32_t *AL1 = c.take<int32_t>((size_t)n);
    uint32_t *fstamp = c.take<uint32_t>((size_t)n);
    uint64_t *sum2 = c.take<uint64_t>((size_t)n * 2);
    uint32_t *dcc = c.take<uint32_t>((size_t)k * k);
    uint32_t *hist = c.take<uint32_t>((size_t)hist_cap * k);
    int32_t *src = c.take<int32_t>((size_t)k);
    Ctl *ctl = c.take<Ctl>(1);
    int *err = c.take<int>(1);

#define NA_CK(x)                                     \
    do {                                             \
        if ((x) != cudaSuccess) {                    \
            cudaGetLastError();                      \
            return CC_ERR_CUDA;                      \
        }                                            \
    } while (0)

    int64_t arcs = 0;
    NA_CK(cudaMemcpyAsync(&arcs, d_row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (arcs < 1 || arcs > 0x7FFFFFFFLL) return CC_ERR_GRAPH;

    NA_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    k_check_csr<<<grid_of(arcs), 256, 0, st>>>(n, d_row_ptr, d_col, arcs, err);
    // T (the traversal's queue, overwritten by it) holds the in-degrees.
    NA_CK(cudaMemsetAsync(T, 0, (size_t)n * 4, st));
    k_in_degree<<<grid_of(arcs), 256, 0, st>>>(n, d_col, arcs, T);
    k_degree_match<<<grid_of(n), 256, 0, st>>>(n, d_row_ptr, T, err);
    NA_CK(cudaMemcpyAsync(src, sample, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    run_fill_i32(sidx, n, -1, st);
    k_sidx_checked<<<(k + 255) / 256, 256, 0, st>>>(sidx, src, k, err);
    k_iota<<<grid_of(n), 256, 0, st>>>(Llist, n);
    NA_CK(cudaMemsetAsync(sum2, 0, (size_t)n * 16, st));
    NA_CK(cudaMemsetAsync(dcc, 0, (size_t)k * k * 4, st));
    NA_CK(cudaMemsetAsync(hist, 0, (size_t)hist_cap * k * 4, st));
    NA_CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
    int herr = 0;
    NA_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (herr != 0) return herr;

    // The traversal kernel of cc_estimate's first pass, every node scanned
    // one thread per (node, word).
    BfsJob j;
    memset(&j, 0, sizeof(j));
    j.n = n;
    j.arcs = arcs;
    j.rp = d_row_ptr;
    j.col = d_col;
    j.prp = d_row_ptr;
    j.pcol = d_col;
    j.k = k;
    j.sources = src;
    j.sidx = sidx;
    j.Llist = Llist;
    j.nL = n;
    j.vis = vis; j.F0 = F0; j.F1 = F1; j.nxt = nxt;
    j.Q0 = Q0; j.Q1 = Q1; j.T = T; j.tflag = tflag;
    j.AL0 = AL0; j.AL1 = AL1;
    j.fstamp = fstamp;
    j.red = RED_SUM | RED_PIVOT | RED_DCC | RED_HIST;
    j.sum2 = sum2;
    j.pivot = d_pivot;
    j.delta = d_delta;
    j.dcc = dcc;
    j.dcc_k = k;
    j.hist = hist;
    j.hist_cap = hist_cap;
    j.ctl = ctl;
    j.timeout_ns = 10ull * 1000 * 1000 * 1000;
    j.alpha = default_alpha(W, j.n, j.arcs);
    const int rc = launch_msbfs(W, j, st, nullptr);
    if (rc != CC_OK) return rc;
    Ctl h;
    NA_CK(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (h.err < 0) return h.err;
    if (h.err == 1) return CC_ERR_TOO_LARGE;  // more levels than the fixed histogram
    if (h.ninc_final != 0) return CC_ERR_DISCONNECTED;
    run_S_sampled(hist, DevCount{nullptr, h.levels}, k, dcc, d_S_sampled, st);
    k_take_sum<<<grid_of(n), 256, 0, st>>>(sum2, d_sample_sum, n);
    NA_CK(cudaStreamSynchronize(st));
    NA_CK(cudaGetLastError());
#undef NA_CK
    return CC_OK;
}
