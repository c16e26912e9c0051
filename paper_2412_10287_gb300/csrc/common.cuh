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
    // hyper: bucket b holds the ids [b << bbits, (b+1) << bbits); bkt[b] is
    // the first row index with an id in it or after it (about 4 rows a bucket)
    const int32_t *bkt;
    int32_t bbits, pad;
};

// Row v of an adjacency as [b, e) into nbr.
__device__ __forceinline__ void adj_row(const DevAdj &A, int32_t v, int32_t &b, int32_t &e) {
    if (A.fmt == ADJ_DENSE) {
        b = __ldg(A.off + v);
        e = __ldg(A.off + v + 1);
    } else if (A.fmt == ADJ_HYPER) {
        // v's bucket, then v among the bucket's few row ids
        const int32_t bi = v >> A.bbits;
        int32_t lo = __ldg(A.bkt + bi), hi = __ldg(A.bkt + bi + 1);
        int32_t at = -1;
        if (hi - lo <= 8) {
            int32_t x[8];
#pragma unroll
            for (int r = 0; r < 8; r++) x[r] = lo + r < hi ? __ldg(A.rows + lo + r) : -1;
#pragma unroll
            for (int r = 0; r < 8; r++)
                if (x[r] == v) at = lo + r;
        } else {
            while (lo < hi) {  // first index with rows[idx] >= v
                const int32_t mid = (lo + hi) >> 1;
                if (__ldg(A.rows + mid) < v) lo = mid + 1; else hi = mid;
            }
            if (lo < A.nrows && __ldg(A.rows + lo) == v) at = lo;
        }
        if (at >= 0) {
            b = __ldg(A.off + at);
            e = __ldg(A.off + at + 1);
        } else {
            b = e = 0;
        }
    } else {
        b = e = 0;
    }
}

}  // namespace rpq
