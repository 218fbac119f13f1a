// Graph to CSR on the device (graph_gpu.cu).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace ccg {

struct DeviceCSR {
    int64_t n = 0, arcs = 0;
    void *rp = nullptr, *col = nullptr, *w = nullptr;  // device, caller frees
    std::vector<int64_t> rp_host;
    std::vector<int32_t> old_id;
};

int build_csr_device(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
                     const uint32_t *w, bool keep_component, DeviceCSR &out);

// Directed graph to CSR on the device: arcs one way, merged, G in F and G^T
// in R (same numbering).  With keep_component, only the largest strongly
// connected component (ties to the one holding the smallest id) is kept,
// found by trimming and forward-backward searches confined to ever smaller
// parts of the graph.
int build_csr_device_directed(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
                              const uint32_t *w, bool keep_component, DeviceCSR &F,
                              DeviceCSR &R);

// Exclusive scan of n uint64 values (in -> out, may alias); *total = the sum.
// Synchronises the stream.
int device_scan_u64(const uint64_t *in, uint64_t *out, int64_t n, uint64_t *total,
                    cudaStream_t st);

// Stable LSD radix sort of (keys, vals) by the low `bits` bits of the keys,
// 8 bits a round through the scratch tk / tv (n each); *in_tmp tells whether
// the result ended in tk / tv.  Synchronises the stream.
int device_radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, int bits, uint64_t *tk,
                      uint32_t *tv, cudaStream_t st, bool *in_tmp);

}  // namespace ccg
