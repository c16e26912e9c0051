// Device-side helpers shared by the CUDA translation units of librpq.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "rpq_internal.h"

#define RPQ_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess)                                                              \
            return ::rpq::fail(_e == cudaErrorMemoryAllocation ? RPQ_ERR_OOM : RPQ_ERR_CUDA, \
                               "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),      \
                               __FILE__, __LINE__);                                         \
    } while (0)

namespace rpq {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One adjacency structure: the rows of G^a (CSR, out-edges) or of (G^a)^T
// (CSC, in-edges) for one label a.
enum AdjFormat : int32_t { ADJ_EMPTY = 0, ADJ_DENSE = 1, ADJ_HYPER = 2 };

struct DevAdj {
    int32_t fmt;
    int32_t nrows;         // hyper: number of non-empty rows; dense: n
    int64_t nnz;
    const int32_t *rows;   // hyper: sorted ids of the non-empty rows
    const int32_t *off;    // dense: [n+1]; hyper: [nrows+1]; relative to nbr
    const int32_t *nbr;    // neighbour ids, sorted within each row
};

// Row v of an adjacency as [b, e) into nbr.
__device__ __forceinline__ void adj_row(const DevAdj &A, int32_t v, int32_t &b, int32_t &e) {
    if (A.fmt == ADJ_DENSE) {
        b = __ldg(A.off + v);
        e = __ldg(A.off + v + 1);
    } else if (A.fmt == ADJ_HYPER) {
        int32_t lo = 0, hi = A.nrows;  // first index with rows[idx] >= v
        while (lo < hi) {
            int32_t mid = (lo + hi) >> 1;
            if (__ldg(A.rows + mid) < v) lo = mid + 1; else hi = mid;
        }
        if (lo < A.nrows && __ldg(A.rows + lo) == v) {
            b = __ldg(A.off + lo);
            e = __ldg(A.off + lo + 1);
        } else {
            b = e = 0;
        }
    } else {
        b = e = 0;
    }
}

}  // namespace rpq
