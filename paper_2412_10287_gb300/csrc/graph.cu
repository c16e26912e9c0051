// Graph residency (section 3: Boolean decomposition {G^a}; section 5: CSR and
// CSC both kept in memory).  Built on the device from host COO triples:
//   1. copy (label, src, dst) to the device and check every id;
//   2. LSD radix sort by (label, src, dst) -- own kernels, 8-bit digits, a
//      stable rank inside each tile by warp match + per-warp digit counts;
//   3. drop duplicate triples (Boolean matrices);
//   4. per label, pick dense offsets (n+1 entries) or hypersparse rows
//      (sorted non-empty row ids + offsets) and fill them;
//   5. repeat 2-4 with (label, dst, src) for the CSC.
#include <algorithm>
#include <cstring>

#include "graph.h"

namespace rpq {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; *total gets the block sum.
template <class T>
__device__ T block_exclusive_scan(T v, T *total) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ T warp_sums[kWarps + 1];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T s = (int)lane < kWarps ? warp_sums[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, si, o);
            if ((int)lane >= o) si += y;
        }
        if ((int)lane < kWarps) warp_sums[lane] = si - s;
        if ((int)lane == kWarps - 1) warp_sums[kWarps] = si;
    }
    __syncthreads();
    const T res = warp_sums[wid] + incl - v;
    *total = warp_sums[kWarps];
    __syncthreads();
    return res;
}

template <class T>
__global__ void scan_tiles_kernel(const T *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                                  int64_t *__restrict__ partials) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t vals[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        vals[k] = i < n ? (int64_t)in[i] : 0;
        sum += vals[k];
    }
    int64_t total = 0;
    int64_t run = block_exclusive_scan<int64_t>(sum, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += vals[k];
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t n,
                                const int64_t *__restrict__ offs) {
    int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    const int64_t add = offs[blockIdx.x];
    for (int k = 0; k < kScanItems; k++, i += kScanThreads)
        if (i < n) out[i] += add;
}

__global__ void copy_total_kernel(const int64_t *scan, const int64_t *partials, int64_t nb,
                                  int64_t *total) {
    // total = scanned offset of the last tile + the last tile's sum
    (void)scan;
    *total = partials[nb];
}

}  // namespace

// Exclusive scan of n values into out (int64); the sum goes to *total_dev.
template <class T>
rpq_status device_exclusive_scan(const T *in, int64_t *out, int64_t n, int64_t *total_dev,
                                 cudaStream_t st) {
    const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    DevBuf part, part_scan;
    if (!part.alloc(sizeof(int64_t) * (nb + 1)) || !part_scan.alloc(sizeof(int64_t) * (nb + 1)))
        return fail(RPQ_ERR_OOM, "scan temporaries");
    scan_tiles_kernel<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, part.as<int64_t>());
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    // scan the tile sums (recursively) into part_scan[0..nb], part_scan[nb] = total
    if (nb == 1) {
        RPQ_CUDA_TRY(cudaMemsetAsync(part_scan.p, 0, sizeof(int64_t), st));
        RPQ_CUDA_TRY(cudaMemcpyAsync(part_scan.as<int64_t>() + 1, part.p, sizeof(int64_t),
                                     cudaMemcpyDeviceToDevice, st));
    } else {
        rpq_status s = device_exclusive_scan<int64_t>(part.as<int64_t>(), part_scan.as<int64_t>(),
                                                      nb, part_scan.as<int64_t>() + nb, st);
        if (s != RPQ_OK) return s;
        scan_add_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, part_scan.as<int64_t>());
        note_launch();
        RPQ_CUDA_TRY(cudaGetLastError());
    }
    copy_total_kernel<<<1, 1, 0, st>>>(out, part_scan.as<int64_t>(), nb, total_dev);
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    // temporaries are freed when this returns: make sure the kernels are done
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    return RPQ_OK;
}

template rpq_status device_exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, int64_t *,
                                                   cudaStream_t);
template rpq_status device_exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *,
                                                   cudaStream_t);

namespace {

// ----------------------------------------------------------- radix sort --
constexpr int kSortThreads = 256;
constexpr int kSortChunks = 16;
constexpr int kSortTile = kSortThreads * kSortChunks;

__global__ void radix_hist_kernel(const int32_t *__restrict__ key, int64_t m, int shift, int64_t nb,
                                  int32_t *__restrict__ hist) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortChunks; c++) {
        int64_t i = base + (int64_t)c * kSortThreads + threadIdx.x;
        if (i < m) atomicAdd(&h[((uint32_t)key[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const int32_t *__restrict__ key, int shift, int64_t m,
                                     int64_t nb, const int64_t *__restrict__ offs,
                                     const int32_t *__restrict__ a0, const int32_t *__restrict__ a1,
                                     const int32_t *__restrict__ a2, int32_t *__restrict__ b0,
                                     int32_t *__restrict__ b1, int32_t *__restrict__ b2) {
    __shared__ int64_t base[256];
    __shared__ int32_t wcnt[kSortThreads / 32][256];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
    for (int w = 0; w < kSortThreads / 32; w++) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortChunks; c++) {
        const int64_t i = tile + (int64_t)c * kSortThreads + threadIdx.x;
        const bool valid = i < m;
        const unsigned d = valid ? (((uint32_t)key[i] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = base[d] + rank;
            for (unsigned w = 0; w < wid; w++) pos += wcnt[w][d];
            b0[pos] = a0[i];
            b1[pos] = a1[i];
            b2[pos] = a2[i];
        }
        __syncthreads();
        {
            int32_t s = 0;
            for (int w = 0; w < kSortThreads / 32; w++) {
                s += wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = 0;
            }
            base[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ checks -----
__global__ void check_ids_kernel(const int32_t *src, const int32_t *dst, const int32_t *lab,
                                 int64_t m, int32_t n, int32_t L, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if ((uint32_t)src[i] >= (uint32_t)n || (uint32_t)dst[i] >= (uint32_t)n ||
            (uint32_t)lab[i] >= (uint32_t)L)
            atomicExch(bad, 1);
    }
}

// unique flag of sorted triples (lab, major, minor); row flag = first edge of a (lab, major) row
__global__ void flags_kernel(const int32_t *lab, const int32_t *maj, const int32_t *mnr, int64_t m,
                             int32_t *uniq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t f = 1;
        if (i > 0 && lab[i] == lab[i - 1] && maj[i] == maj[i - 1] && mnr[i] == mnr[i - 1]) f = 0;
        uniq[i] = f;
    }
}

__global__ void compact_kernel(const int32_t *lab, const int32_t *maj, const int32_t *mnr,
                               int64_t m, const int32_t *uniq, const int64_t *pos, int32_t *olab,
                               int32_t *omaj, int32_t *omnr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (uniq[i]) {
            int64_t p = pos[i];
            olab[p] = lab[i];
            omaj[p] = maj[i];
            omnr[p] = mnr[i];
        }
    }
}

__global__ void row_flags_kernel(const int32_t *lab, const int32_t *maj, int64_t m, int32_t *rf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        rf[i] = (i == 0 || lab[i] != lab[i - 1] || maj[i] != maj[i - 1]) ? 1 : 0;
}

// label_start[a] = first unique index with label >= a, for a in [0, L]
__global__ void label_start_kernel(const int32_t *lab, int64_t m, int32_t L, int64_t *start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = (i == 0) ? 0 : lab[i - 1] + 1;
        int32_t hi = (i == m) ? L : lab[i];
        for (int32_t a = lo; a <= hi; a++) start[a] = i;
    }
}

// dense offsets of one label segment [s, e) of majors sorted ascending
__global__ void dense_offsets_kernel(const int32_t *maj, int64_t s, int64_t e, int32_t n,
                                     int32_t *off) {
    const int64_t cnt = e - s;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= cnt;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t prev = (k == 0) ? -1 : maj[s + k - 1];
        int32_t cur = (k == cnt) ? n : maj[s + k];
        for (int32_t v = prev + 1; v <= cur; v++) off[v] = (int32_t)k;
    }
}

// hypersparse rows of one label segment
// bkt[b] = first index of rows (sorted ids, nrows of them) with id >= b << bbits,
// for b in [0, nb]; bkt[nb] = nrows.
__global__ void bucket_index_kernel(const int32_t *rows, int32_t nrows, int32_t bbits, int64_t nb,
                                    int32_t *bkt) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nb;
         b += (int64_t)gridDim.x * blockDim.x) {
        if (b == nb) {
            bkt[b] = nrows;
            continue;
        }
        const int64_t v0 = b << bbits;
        int32_t lo = 0, hi = nrows;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if ((int64_t)rows[mid] < v0) lo = mid + 1; else hi = mid;
        }
        bkt[b] = lo;
    }
}

__global__ void hyper_rows_kernel(const int32_t *maj, const int32_t *rf, const int64_t *rscan,
                                  int64_t s, int64_t e, int32_t *rows, int32_t *off) {
    const int64_t cnt = e - s;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (rf[s + k]) {
            int64_t r = rscan[s + k] - rscan[s];
            rows[r] = maj[s + k];
            off[r] = (int32_t)k;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t nr = (e > s) ? (rscan[e - 1] - rscan[s] + rf[e - 1]) : 0;
        off[nr] = (int32_t)cnt;
    }
}

// non-empty rows per label from the row-flag scan
__global__ void rows_per_label_kernel(const int64_t *rscan, const int32_t *rf, const int64_t *start,
                                      int32_t L, int64_t *rows) {
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
        const int64_t s = start[a], e = start[a + 1];
        rows[a] = e > s ? rscan[e - 1] - rscan[s] + rf[e - 1] : 0;
    }
}

// rows of at least `minlen` edges and their chunk count, for one adjacency
// Per direction: rows of >= minlen edges, their chunks, and the non-empty
// rows shorter than that.
__global__ void long_rows_kernel(DevAdj A, int32_t minlen, int32_t chunk,
                                 unsigned long long *out /* [3] */) {
    const int64_t rows = A.fmt == ADJ_EMPTY ? 0 : A.nrows;
    unsigned long long nr = 0, nc = 0, ns = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t deg = A.off[r + 1] - A.off[r];
        if (deg >= minlen) {
            nr++;
            // chunks start on 16-byte boundaries: up to 3 ids before the row
            nc += (unsigned long long)((deg + 3 + chunk - 1) / chunk);
        } else if (deg > 0) {
            ns++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nr += __shfl_down_sync(kFull, nr, o);
        nc += __shfl_down_sync(kFull, nc, o);
        ns += __shfl_down_sync(kFull, ns, o);
    }
    if ((threadIdx.x & 31) == 0 && (nr || nc || ns)) {
        atomicAdd(out, nr);
        atomicAdd(out + 1, nc);
        atomicAdd(out + 2, ns);
    }
}

unsigned grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

int bits_for(int64_t maxval) {
    int b = 0;
    while (b < 31 && (int64_t(1) << b) <= maxval) b++;
    return b;
}

// Sorts (k0, k1, k2) ascending by the tuple (k0, k1, k2); ping-pongs with (t0, t1, t2).
// Returns in *which (0 = result in k*, 1 = result in t*).
rpq_status radix_sort3(int32_t *k[3], int32_t *t[3], const int bits[3], int64_t m, cudaStream_t st,
                       int *which) {
    const int64_t nb = std::max<int64_t>(1, (m + kSortTile - 1) / kSortTile);
    DevBuf hist, offs, total;
    if (!hist.alloc(sizeof(int32_t) * 256 * nb) || !offs.alloc(sizeof(int64_t) * 256 * nb) ||
        !total.alloc(sizeof(int64_t)))
        return fail(RPQ_ERR_OOM, "radix sort temporaries");
    int32_t *cur[3] = {k[0], k[1], k[2]};
    int32_t *alt[3] = {t[0], t[1], t[2]};
    int flips = 0;
    for (int a = 2; a >= 0; a--) {  // least significant array first
        for (int shift = 0; shift < bits[a]; shift += 8) {
            radix_hist_kernel<<<(unsigned)nb, kSortThreads, 0, st>>>(cur[a], m, shift, nb,
                                                                    hist.as<int32_t>());
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
            rpq_status s = device_exclusive_scan<int32_t>(hist.as<int32_t>(), offs.as<int64_t>(),
                                                          256 * nb, total.as<int64_t>(), st);
            if (s != RPQ_OK) return s;
            radix_scatter_kernel<<<(unsigned)nb, kSortThreads, 0, st>>>(
                cur[a], shift, m, nb, offs.as<int64_t>(), cur[0], cur[1], cur[2], alt[0], alt[1],
                alt[2]);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
            std::swap(cur[0], alt[0]);
            std::swap(cur[1], alt[1]);
            std::swap(cur[2], alt[2]);
            flips ^= 1;
        }
    }
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    *which = flips;
    return RPQ_OK;
}

struct Side {
    int32_t *nbr;                  // unique minors (owned by the graph)
    std::vector<int64_t> start;    // label_start, L+1
    std::vector<int64_t> rows;     // non-empty rows per label
};

// Builds one side (CSR if major = src) from sorted unique triples.
rpq_status build_side(rpq_graph *g, bool csc, int32_t *lab, int32_t *maj, int32_t *mnr, int64_t m,
                      cudaStream_t st) {
    const int32_t n = g->n, L = g->L;
    const int dir0 = csc ? L : 0;
    // row flags and their scan
    DevBuf rf, rscan, rtot, lstart;
    if (!rf.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1)) ||
        !rscan.alloc(sizeof(int64_t) * std::max<int64_t>(m, 1)) || !rtot.alloc(sizeof(int64_t)) ||
        !lstart.alloc(sizeof(int64_t) * (L + 1)))
        return fail(RPQ_ERR_OOM, "graph build temporaries");
    if (m > 0) {
        row_flags_kernel<<<grid_for(m), 256, 0, st>>>(lab, maj, m, rf.as<int32_t>());
        note_launch();
        RPQ_CUDA_TRY(cudaGetLastError());
        rpq_status s = device_exclusive_scan<int32_t>(rf.as<int32_t>(), rscan.as<int64_t>(), m,
                                                      rtot.as<int64_t>(), st);
        if (s != RPQ_OK) return s;
    }
    label_start_kernel<<<grid_for(m + 1), 256, 0, st>>>(lab, m, L, lstart.as<int64_t>());
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> start(L + 1);
    RPQ_CUDA_TRY(cudaMemcpyAsync(start.data(), lstart.p, sizeof(int64_t) * (L + 1),
                                 cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> rows(L, 0);
    if (m > 0) {
        DevBuf drows;
        if (!drows.alloc(sizeof(int64_t) * L)) return fail(RPQ_ERR_OOM, "rows per label");
        rows_per_label_kernel<<<grid_for(L), 256, 0, st>>>(rscan.as<int64_t>(), rf.as<int32_t>(),
                                                           lstart.as<int64_t>(), L,
                                                           drows.as<int64_t>());
        note_launch();
        RPQ_CUDA_TRY(cudaGetLastError());
        RPQ_CUDA_TRY(cudaMemcpyAsync(rows.data(), drows.p, sizeof(int64_t) * L,
                                     cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // formats: dense offsets (n + 1) when at least n/16 rows are non-empty,
    // when n is small, or when the label holds at least dense_edges edges,
    // by default n/16 (a row is then found in one lookup instead of the
    // bucket index's three; the offsets cost 4 (n + 1) bytes per direction,
    // at most 64 bytes per edge of such a label); hypersparse otherwise.
    // RPQ_DENSE_EDGES overrides the edge threshold (0: rows only).
    const char *de = getenv("RPQ_DENSE_EDGES");
    const int64_t dense_edges = de ? (int64_t)atoll(de) : std::max<int64_t>(1, n / 16);
    int64_t dense_words = 0, hyper_rows_total = 0, hyper_off_total = 0, bucket_total = 0;
    std::vector<int32_t> fmt(L), bbits(L, 0);
    for (int32_t a = 0; a < L; a++) {
        const int64_t nnz = start[a + 1] - start[a];
        if (nnz >= (int64_t(1) << 31)) return fail(RPQ_ERR_INVALID, "label %d has >= 2^31 edges", a);
        if (nnz == 0) fmt[a] = ADJ_EMPTY;
        else if (rows[a] * 16 >= (int64_t)n || n <= 65536 || (dense_edges > 0 && nnz >= dense_edges))
            fmt[a] = ADJ_DENSE;
        else fmt[a] = ADJ_HYPER;
        if (fmt[a] == ADJ_DENSE) dense_words += (int64_t)n + 1;
        if (fmt[a] == ADJ_HYPER) {
            hyper_rows_total += rows[a];
            hyper_off_total += rows[a] + 1;
            // largest bucket width with at most ~4 non-empty rows a bucket on average
            while (bbits[a] < 30 && (int64_t(2) << bbits[a]) * rows[a] <= 4 * (int64_t)n)
                bbits[a]++;
            bucket_total += (((int64_t)n - 1) >> bbits[a]) + 2;
        }
    }
    std::unique_ptr<DevBuf> dense_p(new DevBuf()), hrows_p(new DevBuf()), hoff_p(new DevBuf()),
        bkt_p(new DevBuf());
    DevBuf &dense_buf = *dense_p, &hrows_buf = *hrows_p, &hoff_buf = *hoff_p, &bkt_buf = *bkt_p;
    if (!dense_buf.alloc(sizeof(int32_t) * std::max<int64_t>(dense_words, 1)) ||
        !hrows_buf.alloc(sizeof(int32_t) * std::max<int64_t>(hyper_rows_total, 1)) ||
        !hoff_buf.alloc(sizeof(int32_t) * std::max<int64_t>(hyper_off_total, 1)) ||
        !bkt_buf.alloc(sizeof(int32_t) * std::max<int64_t>(bucket_total, 1)))
        return fail(RPQ_ERR_OOM, "graph offsets");
    int64_t dpos = 0, hrpos = 0, hopos = 0, bpos = 0;
    for (int32_t a = 0; a < L; a++) {
        DevAdj A{};
        A.fmt = fmt[a];
        A.nnz = start[a + 1] - start[a];
        A.nbr = mnr + start[a];
        if (fmt[a] == ADJ_DENSE) {
            int32_t *off = dense_buf.as<int32_t>() + dpos;
            dense_offsets_kernel<<<grid_for(A.nnz + 1), 256, 0, st>>>(maj, start[a], start[a + 1],
                                                                     n, off);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
            A.off = off;
            A.nrows = n;
            dpos += (int64_t)n + 1;
        } else if (fmt[a] == ADJ_HYPER) {
            int32_t *rw = hrows_buf.as<int32_t>() + hrpos;
            int32_t *off = hoff_buf.as<int32_t>() + hopos;
            hyper_rows_kernel<<<grid_for(A.nnz), 256, 0, st>>>(maj, rf.as<int32_t>(),
                                                              rscan.as<int64_t>(), start[a],
                                                              start[a + 1], rw, off);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
            A.rows = rw;
            A.off = off;
            A.nrows = (int32_t)rows[a];
            const int64_t nb = (((int64_t)n - 1) >> bbits[a]) + 1;
            int32_t *bk = bkt_buf.as<int32_t>() + bpos;
            bucket_index_kernel<<<grid_for(nb + 1), 256, 0, st>>>(rw, A.nrows, bbits[a], nb, bk);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
            A.bkt = bk;
            A.bbits = bbits[a];
            hrpos += rows[a];
            hopos += rows[a] + 1;
            bpos += nb + 1;
        }
        g->adj[dir0 + a] = A;
    }
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    g->owned.push_back(std::move(dense_p));
    g->owned.push_back(std::move(hrows_p));
    g->owned.push_back(std::move(hoff_p));
    g->owned.push_back(std::move(bkt_p));
    if (!csc) {
        g->nnz.assign(L, 0);
        for (int32_t a = 0; a < L; a++) g->nnz[a] = start[a + 1] - start[a];
    }
    return RPQ_OK;
}

}  // namespace
}  // namespace rpq

using namespace rpq;

extern "C" rpq_status rpq_graph_load(int32_t n_vertices, int32_t n_labels, int64_t n_edges,
                                     const int32_t *src, const int32_t *dst, const int32_t *label,
                                     void *stream, rpq_graph **out) {
    clear_error();
    if (!out) return fail(RPQ_ERR_INVALID, "out is null");
    *out = nullptr;
    if (n_vertices <= 0 || n_labels <= 0 || n_edges < 0)
        return fail(RPQ_ERR_INVALID, "sizes must be positive (n=%d, L=%d, m=%lld)", n_vertices,
                    n_labels, (long long)n_edges);
    if (n_labels > (1 << 20)) return fail(RPQ_ERR_INVALID, "at most 2^20 labels");
    if (n_edges >= (int64_t(1) << 31)) return fail(RPQ_ERR_INVALID, "n_edges must be < 2^31");
    if (n_edges > 0 && (!src || !dst || !label)) return fail(RPQ_ERR_INVALID, "null edge array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    std::unique_ptr<rpq_graph> g(new rpq_graph());
    g->n = n_vertices;
    g->L = n_labels;
    g->m_input = n_edges;
    RPQ_CUDA_TRY(cudaGetDevice(&g->device));
    g->adj.assign(2 * (size_t)n_labels, DevAdj{});

    const int64_t m = n_edges;
    const size_t mb = sizeof(int32_t) * std::max<int64_t>(m, 1);
    DevBuf k0, k1, k2, t0, t1, t2, bad;
    if (!k0.alloc(mb) || !k1.alloc(mb) || !k2.alloc(mb) || !t0.alloc(mb) || !t1.alloc(mb) ||
        !t2.alloc(mb) || !bad.alloc(sizeof(int32_t)))
        return fail(RPQ_ERR_OOM, "graph build buffers for %lld edges", (long long)m);
    if (m > 0) {
        RPQ_CUDA_TRY(cudaMemcpyAsync(k0.p, label, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        RPQ_CUDA_TRY(cudaMemcpyAsync(k1.p, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        RPQ_CUDA_TRY(cudaMemcpyAsync(k2.p, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    }
    RPQ_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), st));
    if (m > 0) {
        check_ids_kernel<<<grid_for(m), 256, 0, st>>>(k1.as<int32_t>(), k2.as<int32_t>(),
                                                     k0.as<int32_t>(), m, n_vertices, n_labels,
                                                     bad.as<int32_t>());
        note_launch();
        RPQ_CUDA_TRY(cudaGetLastError());
    }
    int32_t h_bad = 0;
    RPQ_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_bad) return fail(RPQ_ERR_INVALID, "edge id or label out of range");

    // keep an untouched copy of the COO for the second side
    DevBuf c0, c1, c2;
    if (!c0.alloc(mb) || !c1.alloc(mb) || !c2.alloc(mb))
        return fail(RPQ_ERR_OOM, "graph build buffers");
    if (m > 0) {
        RPQ_CUDA_TRY(cudaMemcpyAsync(c0.p, k0.p, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
        RPQ_CUDA_TRY(cudaMemcpyAsync(c1.p, k1.p, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
        RPQ_CUDA_TRY(cudaMemcpyAsync(c2.p, k2.p, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
    }
    const int bits_l = bits_for(n_labels - 1), bits_v = bits_for(n_vertices - 1);

    for (int side = 0; side < 2; side++) {
        // side 0: (label, src, dst) -> CSR; side 1: (label, dst, src) -> CSC
        int32_t *k[3], *t[3];
        if (side == 0) { k[0] = k0.as<int32_t>(); k[1] = k1.as<int32_t>(); k[2] = k2.as<int32_t>(); }
        else { k[0] = c0.as<int32_t>(); k[1] = c2.as<int32_t>(); k[2] = c1.as<int32_t>(); }
        t[0] = t0.as<int32_t>(); t[1] = t1.as<int32_t>(); t[2] = t2.as<int32_t>();
        const int bits[3] = {bits_l, bits_v, bits_v};
        int which = 0;
        if (m > 0) {
            rpq_status s = radix_sort3(k, t, bits, m, st, &which);
            if (s != RPQ_OK) return s;
        }
        int32_t **r = which ? t : k;   // sorted arrays
        int32_t **o = which ? k : t;   // free arrays (for the compacted result)
        // dedup: flags in o[0] (as int32), positions in a scan buffer
        DevBuf pos, tot;
        if (!pos.alloc(sizeof(int64_t) * std::max<int64_t>(m, 1)) || !tot.alloc(sizeof(int64_t)))
            return fail(RPQ_ERR_OOM, "dedup buffers");
        int64_t mu = 0;
        if (m > 0) {
            flags_kernel<<<grid_for(m), 256, 0, st>>>(r[0], r[1], r[2], m, o[0]);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
            rpq_status s = device_exclusive_scan<int32_t>(o[0], pos.as<int64_t>(), m,
                                                          tot.as<int64_t>(), st);
            if (s != RPQ_OK) return s;
            RPQ_CUDA_TRY(cudaMemcpy(&mu, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost));
        }
        // compacted triples: label -> o[1], major -> o[2], minor -> owned neighbour buffer
        DevBuf *nb = side == 0 ? &g->csr_nbr : &g->csc_nbr;
        // 4 ids of padding: a 16-byte load of the last ids never leaves the buffer
        if (!nb->alloc(sizeof(int32_t) * (std::max<int64_t>(mu, 1) + 4)))
            return fail(RPQ_ERR_OOM, "neighbour array");
        if (m > 0) {
            compact_kernel<<<grid_for(m), 256, 0, st>>>(r[0], r[1], r[2], m, o[0],
                                                        pos.as<int64_t>(), o[1], o[2],
                                                        nb->as<int32_t>());
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
        }
        g->m_unique = mu;
        rpq_status s = build_side(g.get(), side == 1, o[1], o[2], nb->as<int32_t>(), mu, st);
        if (s != RPQ_OK) return s;
    }
    // long- and short-row statistics per direction
    {
        DevBuf lr;
        const size_t nd = g->adj.size();
        if (!lr.alloc(sizeof(unsigned long long) * 3 * nd)) return fail(RPQ_ERR_OOM, "row statistics");
        RPQ_CUDA_TRY(cudaMemsetAsync(lr.p, 0, sizeof(unsigned long long) * 3 * nd, st));
        for (size_t d = 0; d < nd; d++) {
            const DevAdj &A = g->adj[d];
            if (A.fmt == ADJ_EMPTY) continue;
            long_rows_kernel<<<grid_for(A.nrows), 256, 0, st>>>(
                A, rpq_graph::kLongRow, rpq_graph::kLongChunk, lr.as<unsigned long long>() + 3 * d);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
        }
        std::vector<unsigned long long> h(3 * nd);
        RPQ_CUDA_TRY(cudaMemcpyAsync(h.data(), lr.p, sizeof(unsigned long long) * 3 * nd,
                                     cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
        g->long_rows.assign(nd, 0);
        g->long_chunks.assign(nd, 0);
        g->short_rows.assign(nd, 0);
        for (size_t d = 0; d < nd; d++) {
            g->long_rows[d] = (int64_t)h[3 * d];
            g->long_chunks[d] = (int64_t)h[3 * d + 1];
            g->short_rows[d] = (int64_t)h[3 * d + 2];
        }
    }
    if (!g->d_adj.alloc(sizeof(DevAdj) * g->adj.size())) return fail(RPQ_ERR_OOM, "adjacency table");
    RPQ_CUDA_TRY(cudaMemcpyAsync(g->d_adj.p, g->adj.data(), sizeof(DevAdj) * g->adj.size(),
                                 cudaMemcpyHostToDevice, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    *out = g.release();
    return RPQ_OK;
}

extern "C" void rpq_graph_free(rpq_graph *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    delete g;
}

extern "C" rpq_status rpq_graph_info(const rpq_graph *g, int32_t label, int32_t *n_vertices,
                                     int32_t *n_labels, int64_t *n_edges) {
    clear_error();
    if (!g) return fail(RPQ_ERR_INVALID, "graph is null");
    if (label >= g->L) return fail(RPQ_ERR_INVALID, "label %d out of range", label);
    if (n_vertices) *n_vertices = g->n;
    if (n_labels) *n_labels = g->L;
    if (n_edges) *n_edges = label < 0 ? g->m_unique : g->nnz[label];
    return RPQ_OK;
}

namespace rpq {
namespace {
__global__ void export_dense_kernel(DevAdj A, int32_t n, int64_t *off) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = 0;
        if (A.fmt == ADJ_DENSE) o = A.off[v];
        else if (A.fmt == ADJ_HYPER) {
            int32_t lo = 0, hi = A.nrows;  // rows with id < v
            while (lo < hi) {
                int32_t mid = (lo + hi) >> 1;
                if (A.rows[mid] < v) lo = mid + 1; else hi = mid;
            }
            o = A.off[lo];
        }
        off[v] = o;
    }
}
}  // namespace
}  // namespace rpq

extern "C" rpq_status rpq_graph_export(const rpq_graph *g, int32_t label, int32_t inverse,
                                       int64_t *offsets, int32_t *neighbours, int64_t capacity) {
    clear_error();
    if (!g || !offsets) return fail(RPQ_ERR_INVALID, "null argument");
    if (label < 0 || label >= g->L) return fail(RPQ_ERR_INVALID, "label %d out of range", label);
    const DevAdj &A = g->adj[(inverse ? g->L : 0) + label];
    DevBuf d;
    if (!d.alloc(sizeof(int64_t) * ((size_t)g->n + 1))) return fail(RPQ_ERR_OOM, "export buffer");
    export_dense_kernel<<<grid_for((int64_t)g->n + 1), 256>>>(A, g->n, d.as<int64_t>());
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    RPQ_CUDA_TRY(cudaMemcpy(offsets, d.p, sizeof(int64_t) * ((size_t)g->n + 1),
                            cudaMemcpyDeviceToHost));
    if (neighbours) {
        if (capacity < A.nnz) return fail(RPQ_ERR_CAPACITY, "need %lld entries", (long long)A.nnz);
        if (A.nnz > 0)
            RPQ_CUDA_TRY(cudaMemcpy(neighbours, A.nbr, sizeof(int32_t) * A.nnz,
                                    cudaMemcpyDeviceToHost));
    }
    return RPQ_OK;
}
