// Bit-packed multi-source BFS with fused per-node reductions (sm_103a).
//
// One persistent cooperative kernel runs every level of one traversal pass.
// k sources are packed 64 per uint64 word, W words per node (W a power of
// two).  Per level l every node v gets new = (OR of its neighbours' frontier
// words) & ~visited(v) -- the nodes at distance exactly l from the sources
// whose bits are set -- and the pass reduces it on the fly (section 3: the
// per-node running sums, the running minimum Delta(v) and pivot c(v)):
//   RED_SUM    sum[v] += l * popc(new), sumsq[v] += l^2 * popc(new)
//   RED_PIVOT  on the first level with new bits: Delta(v) = l and c(v) =
//              the lowest set bit (smallest sample index among the nearest)
//   RED_DCC    v sampled with index j: dcc[i][j] = l for each new bit i
//   RED_HIST   v not sampled: hist[l][i] += 1 for each new bit i
//   RED_LC     v not sampled: lc[v] += l, l^2 times popc(new & Lmask(v))
// so the k x n distance matrix never exists.
//
// Direction per level (same decision in every CTA, from the previous level's
// counters): top-down pushes the frontier words of the queued frontier nodes
// into their neighbours with atomicOr; bottom-up pulls, per node and word,
// the OR of the neighbours' frontier words with early exit once every
// missing bit has arrived.  Bottom-up splits nodes by degree: <= 32 a thread
// per (node, word), <= 256 a warp per node, larger nodes in 256-entry warp
// tasks that OR into a scratch word finalised after the barrier.
//
// Every wait is bounded: the grid barrier gives up after timeout_ns, records
// CC_ERR_TIMEOUT and every CTA returns.
#include <cstdint>


#include "msbfs_dev.cuh"

namespace ccg {

namespace {

// Resident CTAs per SM the register allocation must allow, for W <= 4 and
// for W >= 8 words per node (build-time tunables).
#ifndef CC_MSBFS_MIN_CTAS_NARROW
#define CC_MSBFS_MIN_CTAS_NARROW 4
#endif
#ifndef CC_MSBFS_MIN_CTAS_WIDE
#define CC_MSBFS_MIN_CTAS_WIDE 4
#endif

template <int W>
__global__ void __launch_bounds__(kBlock, W >= 8 ? CC_MSBFS_MIN_CTAS_WIDE
                                                 : CC_MSBFS_MIN_CTAS_NARROW)
    msbfs_kernel(BfsJob J)
{
    extern __shared__ unsigned s_hist[];  // W * 64 counters
    bfs_pass<W>(J, blockIdx.x, gridDim.x, J.ctl, s_hist);
}

__global__ void barrier_selftest_kernel(Ctl *ctl, uint64_t timeout_ns)
{
    // A team of two CTAs of which only one is launched: the barrier cannot
    // complete and must give up after timeout_ns.
    grid_sync(ctl, 0u, 2u, timeout_ns);
}

template <int W>
int launch_w(const BfsJob &job, cudaStream_t st, int *grid_used)
{
    static int blocks_per_sm = -1, sms = 0;
    const size_t smem = (size_t)W * 64 * sizeof(unsigned);
    if (blocks_per_sm < 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return CC_ERR_CUDA;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return CC_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm,
                                                          msbfs_kernel<W>, kBlock,
                                                          smem) != cudaSuccess)
            return CC_ERR_CUDA;
        if (blocks_per_sm < 1) return CC_ERR_CUDA;
    }
    int grid = blocks_per_sm * sms;
    if (job.max_ctas > 0 && job.max_ctas < grid) grid = job.max_ctas;
    if (grid_used) *grid_used = grid;
    BfsJob j = job;
    void *args[] = {&j};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)msbfs_kernel<W>,
                                                      dim3(grid), dim3(kBlock), args,
                                                      smem, st);
    return e == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace

int launch_msbfs(int W, const BfsJob &job, cudaStream_t st, int *grid_used)
{
    switch (W) {
    case 1: return launch_w<1>(job, st, grid_used);
    case 2: return launch_w<2>(job, st, grid_used);
    case 4: return launch_w<4>(job, st, grid_used);
    case 8: return launch_w<8>(job, st, grid_used);
    case 16: return launch_w<16>(job, st, grid_used);
    case 32: return launch_w<32>(job, st, grid_used);
    default: return CC_ERR_ARG;
    }
}

// One shared-memory carveout for every traversal variant: an SM runs CTAs of
// different kernels side by side only when they agree on the L1/shared split,
// so persistent grids that share the GPU must not ask for different splits.
void msbfs_set_carveout(int percent)
{
    const void *fns[] = {(const void *)msbfs_kernel<1>, (const void *)msbfs_kernel<2>,
                         (const void *)msbfs_kernel<4>, (const void *)msbfs_kernel<8>,
                         (const void *)msbfs_kernel<16>, (const void *)msbfs_kernel<32>};
    for (const void *f : fns)
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, percent);
    cudaGetLastError();
}

// Smallest number of co-resident CTAs per SM over every traversal variant.
int msbfs_min_blocks_per_sm()
{
    int m = 1 << 30, b = 0;
    const size_t kSmem[] = {64, 128, 256, 512, 1024, 2048};
    const void *fns[] = {(const void *)msbfs_kernel<1>, (const void *)msbfs_kernel<2>,
                         (const void *)msbfs_kernel<4>, (const void *)msbfs_kernel<8>,
                         (const void *)msbfs_kernel<16>, (const void *)msbfs_kernel<32>};
    for (int i = 0; i < 6; ++i) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fns[i], kBlock,
                                                          kSmem[i] * sizeof(unsigned)) !=
            cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        m = b < m ? b : m;
    }
    return m < 1 ? 1 : m;
}

int launch_barrier_selftest(uint64_t timeout_ns, int *err_out)
{
    Ctl *d = nullptr;
    if (cudaMalloc(&d, sizeof(Ctl)) != cudaSuccess) return CC_ERR_OOM;
    cudaMemset(d, 0, sizeof(Ctl));
    barrier_selftest_kernel<<<1, 32>>>(d, timeout_ns);
    Ctl h;
    cudaError_t e = cudaMemcpy(&h, d, sizeof(Ctl), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return CC_ERR_CUDA;
    *err_out = h.err;
    return CC_OK;
}

}  // namespace ccg
