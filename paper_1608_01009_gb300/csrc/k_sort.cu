// Supercell counting sort of a species' particle store.
//
// arXiv:1608.01009 Sec. 3 stores particles per cell and Sec. 4.3 processes them
// by supercells of S^3 cells.  On the GPU the store is one structure of arrays
// kept ordered by supercell ("bins"); every K steps (K * max(dt/d) < 1, so a
// particle never leaves its supercell's one-cell slack in between) it is
// re-binned by a counting sort (the order inside a bin is unspecified):
//   k_sort_count   : key = supercell of each active particle, histogram with
//                    warp-aggregated atomics (one atomic per distinct key per warp)
//   k_sort_scan    : one CTA: exclusive scan of the histogram -> bin starts and
//                    scatter cursors, new particle count, and the chunk table the
//                    particle kernel walks (each bin cut into near-equal chunks
//                    of at most CHUNK particles)
//   k_sort_scatter : every active particle copied to its slot in the other
//                    buffer; deactivated particles are dropped (compaction)
#include "pic_internal.cuh"

namespace picgb {

constexpr int SORT_NT = 256;
constexpr int SCAN_NT = 1024;

__device__ __forceinline__ int bin_of(const GridDev& g, int cp) {
    const int bx = cell_x(cp) / g.S, by = cell_y(cp) / g.S, bz = cell_z(cp) / g.S;
    return bx + g.nsc[0] * (by + g.nsc[1] * bz);
}

template <class R>
__global__ void __launch_bounds__(SORT_NT) k_sort_count(PStore<R> ps, const long long* __restrict__ n_cur, GridDev g,
                                                       int* __restrict__ keys, int* __restrict__ counts) {
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * SORT_NT;
    for (long long base = (long long)blockIdx.x * SORT_NT + (threadIdx.x & ~31); base < N; base += stride) {
        const long long p = base + lane;
        int key = -1;
        if (p < N) {
            const int cp = ps.cell[p];
            key = cp < 0 ? -1 : bin_of(g, cp);
            keys[p] = key;
        }
        warp_agg_slot(counts, key);
    }
}

__global__ void __launch_bounds__(SCAN_NT) k_sort_scan(int* __restrict__ counts, int nbins, int* __restrict__ bin_start,
                                                      int* __restrict__ cursor, long long* __restrict__ n_next,
                                                      Chunk* __restrict__ chunks, int* __restrict__ nchunks) {
    __shared__ long long s_cnt[SCAN_NT];
    __shared__ int s_nch[SCAN_NT];
    const int per = (nbins + SCAN_NT - 1) / SCAN_NT;
    const int b0 = threadIdx.x * per, b1 = min(nbins, b0 + per);
    long long cnt = 0;
    int nch = 0;
    for (int b = b0; b < b1; ++b) {
        const int c = counts[b];
        cnt += c;
        nch += (c + CHUNK - 1) / CHUNK;
    }
    s_cnt[threadIdx.x] = cnt;
    s_nch[threadIdx.x] = nch;
    __syncthreads();
    // inclusive Hillis-Steele scan over the per-thread sums
    for (int off = 1; off < SCAN_NT; off <<= 1) {
        long long vc = threadIdx.x >= off ? s_cnt[threadIdx.x - off] : 0;
        int vn = threadIdx.x >= off ? s_nch[threadIdx.x - off] : 0;
        __syncthreads();
        s_cnt[threadIdx.x] += vc;
        s_nch[threadIdx.x] += vn;
        __syncthreads();
    }
    long long start = s_cnt[threadIdx.x] - cnt;
    int ch = s_nch[threadIdx.x] - nch;
    for (int b = b0; b < b1; ++b) {
        const int c = counts[b];
        bin_start[b] = (int)start;
        cursor[b] = (int)start;
        const int k = (c + CHUNK - 1) / CHUNK;
        if (k > 0) {
            const int base = c / k, rem = c % k;
            for (int q = 0; q < k; ++q) {
                Chunk e;
                e.sc = b;
                e.start = (int)start + q * base + min(q, rem);
                e.count = base + (q < rem ? 1 : 0);
                e.pad = 0;
                chunks[ch + q] = e;
            }
        }
        ch += k;
        start += c;
        counts[b] = 0;  // ready for the next sort
    }
    if (threadIdx.x == SCAN_NT - 1) {
        bin_start[nbins] = (int)s_cnt[SCAN_NT - 1];
        *n_next = s_cnt[SCAN_NT - 1];
        *nchunks = s_nch[SCAN_NT - 1];
    }
}

template <class R>
__global__ void __launch_bounds__(SORT_NT) k_sort_scatter(PStore<R> src, PStore<R> dst, const long long* __restrict__ n_cur,
                                                         const int* __restrict__ keys, int* __restrict__ cursor) {
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * SORT_NT;
    for (long long base = (long long)blockIdx.x * SORT_NT + (threadIdx.x & ~31); base < N; base += stride) {
        const long long p = base + lane;
        const int key = p < N ? keys[p] : -1;
        const int q = warp_agg_slot(cursor, key);
        if (q >= 0) {
            dst.cell[q] = src.cell[p];
            for (int a = 0; a < 3; ++a) {
                dst.off[a][q] = src.off[a][p];
                dst.u[a][q] = src.u[a][p];
            }
            dst.w[q] = src.w[p];
            dst.id[q] = src.id[p];
        }
    }
}

int sort_grid(int nsm) { return nsm * 8; }

template <class R>
cudaError_t sort_launch(cudaStream_t st, int nsm, const GridDev& g, PStore<R> src, PStore<R> dst,
                        const long long* n_cur, long long* n_next, int* keys, int* counts, int* cursor, int* bin_start,
                        Chunk* chunks, int* nchunks) {
    k_sort_count<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, n_cur, g, keys, counts);
    k_sort_scan<<<1, SCAN_NT, 0, st>>>(counts, g.nbins, bin_start, cursor, n_next, chunks, nchunks);
    k_sort_scatter<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, dst, n_cur, keys, cursor);
    return cudaGetLastError();
}

template cudaError_t sort_launch<double>(cudaStream_t, int, const GridDev&, PStore<double>, PStore<double>,
                                         const long long*, long long*, int*, int*, int*, int*, Chunk*, int*);
template cudaError_t sort_launch<float>(cudaStream_t, int, const GridDev&, PStore<float>, PStore<float>,
                                        const long long*, long long*, int*, int*, int*, int*, Chunk*, int*);

}  // namespace picgb
