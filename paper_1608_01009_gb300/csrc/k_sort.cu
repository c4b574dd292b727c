// Supercell counting sort of a species' particle store.
//
// arXiv:1608.01009 Sec. 3 stores particles per cell and Sec. 4.3 processes them
// by supercells of S^3 cells.  On the GPU the store is one structure of arrays
// ordered by supercell and, inside a supercell, by cell.  Every K steps
// (K * max(dt/d) < 1, so a particle never leaves its supercell's one-cell slack
// in between) it is re-sorted by a counting sort over cell keys
//   key = supercell * S^3 + local cell,
// so that each supercell is a contiguous run of cell runs (the particle kernel
// relies on the cell order: warp lanes that share a cell share their gather
// loads and sum their currents before the shared-memory atomics):
//   k_sort_count  : histogram of keys, warp-aggregated atomics (one atomic per
//                   distinct key per warp); deactivated particles get no key
//   k_scan_tiles  : per tile of SCAN_TILE keys, exclusive prefix into cursor[]
//                   and the tile total
//   k_scan_top    : one CTA: scan of the tile totals, new particle count, the
//                   supercell bin starts and the chunk table the particle
//                   kernel walks (each bin cut into near-equal chunks of at
//                   most CHUNK particles)
//   k_scan_add    : cursor[] += tile offset; the histogram is cleared
//   k_sort_scatter: every active particle copied to its slot in the other
//                   buffer (order inside a cell unspecified); deactivated
//                   particles are dropped (compaction).  It recomputes each
//                   key from the cell it copies anyway, so no per-particle
//                   key array is written or read.
#include "pic_internal.cuh"

namespace picgb {

constexpr int SORT_NT = 256;
constexpr int SCAN_NT = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_NT * SCAN_PER;  // keys per tile; a multiple of every S^3

__device__ __forceinline__ int cell_key(const GridDev& g, int cp) {
    const int sh = g.Sshift, m = g.S - 1;
    const int ix = cell_x(cp), iy = cell_y(cp), iz = cell_z(cp);
    const int sc = (ix >> sh) + g.nsc[0] * ((iy >> sh) + g.nsc[1] * (iz >> sh));
    return (((sc << sh) + (iz & m)) << (2 * sh)) + ((iy & m) << sh) + (ix & m);
}

// U independent warp-aggregated slot claims: every lane's U match/atomic
// chains are issued before the first result is needed, so U atomics per lane
// are in flight at once (one atomic per distinct key per warp and group).
template <int U>
__device__ __forceinline__ void warp_agg_slots(int* counters, const int (&key)[U], int (&slot)[U]) {
    const int lane = threadIdx.x & 31;
    unsigned peers[U];
    int leader[U], base[U];
#pragma unroll
    for (int i = 0; i < U; ++i) {
        peers[i] = __match_any_sync(0xffffffffu, key[i]);
        leader[i] = __ffs(peers[i]) - 1;
    }
#pragma unroll
    for (int i = 0; i < U; ++i)
        base[i] = (lane == leader[i] && key[i] >= 0) ? atomicAdd(&counters[key[i]], __popc(peers[i])) : 0;
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const int b = __shfl_sync(0xffffffffu, base[i], leader[i]);
        slot[i] = key[i] >= 0 ? b + __popc(peers[i] & ((1u << lane) - 1u)) : -1;
    }
}

// Lane-interleaved groups of U x 32 particles per warp and iteration.
constexpr int COUNT_U = 4;

template <class R>
__global__ void __launch_bounds__(SORT_NT) k_sort_count(PStore<R> ps, const long long* __restrict__ n_cur, GridDev g,
                                                       int* __restrict__ counts) {
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * SORT_NT * COUNT_U;
    for (long long base = ((long long)blockIdx.x * SORT_NT + (threadIdx.x & ~31)) * COUNT_U; base < N;
         base += stride) {
        int key[COUNT_U], slot[COUNT_U];
#pragma unroll
        for (int i = 0; i < COUNT_U; ++i) {
            const long long p = base + i * 32 + lane;
            const int cp = p < N ? ps.cell[p] : INACTIVE;
            key[i] = cp < 0 ? -1 : cell_key(g, cp);
        }
        warp_agg_slots<COUNT_U>(counts, key, slot);
    }
}

// Exclusive block scan of one value per thread (SCAN_NT threads).
__device__ int block_exclusive_scan(int v, int* s, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = s[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s[lane] = t;
    }
    __syncthreads();
    const int before = (w > 0 ? s[w - 1] : 0) + x - v;
    *total = s[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_tiles(const int* __restrict__ counts, long long nkeys,
                                                       int* __restrict__ cursor, int* __restrict__ tile_sum) {
    __shared__ int s[32];
    const long long k0 = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER;
    int c[SCAN_PER];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        c[i] = k0 + i < nkeys ? counts[k0 + i] : 0;
        sum += c[i];
    }
    int total;
    int run = block_exclusive_scan(sum, s, &total);
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        if (k0 + i < nkeys) cursor[k0 + i] = run;
        run += c[i];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// One CTA: tile offsets, bin starts, chunk table, new particle count.
__global__ void __launch_bounds__(SCAN_NT) k_scan_top(int* __restrict__ tile_sum, int ntiles,
                                                     const int* __restrict__ cursor, long long nkeys, int keys_per_bin,
                                                     int nbins, int* __restrict__ bin_start, long long* __restrict__ n_next,
                                                     Chunk* __restrict__ chunks, int* __restrict__ nchunks) {
    __shared__ int s[32];
    __shared__ int s_total;
    // exclusive scan of the tile totals, in place (tiles <= SCAN_NT * per)
    const int per_t = (ntiles + SCAN_NT - 1) / SCAN_NT;
    const int t0 = threadIdx.x * per_t, t1 = min(ntiles, t0 + per_t);
    int sum = 0;
    for (int t = t0; t < t1; ++t) sum += tile_sum[t];
    int total;
    int run = block_exclusive_scan(sum, s, &total);
    for (int t = t0; t < t1; ++t) {
        const int v = tile_sum[t];
        tile_sum[t] = run;
        run += v;
    }
    if (threadIdx.x == 0) s_total = total;
    __syncthreads();
    // bin starts = key prefix at each bin's first key
    const int per_b = (nbins + SCAN_NT - 1) / SCAN_NT;
    const int b0 = threadIdx.x * per_b, b1 = min(nbins, b0 + per_b);
    auto start_of = [&](int b) -> int {
        if (b >= nbins) return s_total;
        const long long k = (long long)b * keys_per_bin;
        return tile_sum[k / SCAN_TILE] + cursor[k];
    };
    int nch = 0;
    for (int b = b0; b < b1; ++b) {
        const int cnt = start_of(b + 1) - start_of(b);
        nch += (cnt + CHUNK - 1) / CHUNK;
    }
    int nch_total;
    int ch = block_exclusive_scan(nch, s, &nch_total);
    for (int b = b0; b < b1; ++b) {
        const int st = start_of(b);
        const int cnt = start_of(b + 1) - st;
        bin_start[b] = st;
        const int k = (cnt + CHUNK - 1) / CHUNK;
        if (k > 0) {
            const int base = cnt / k, rem = cnt % k;
            for (int q = 0; q < k; ++q) {
                Chunk e;
                e.sc = b;
                e.start = st + q * base + min(q, rem);
                e.count = base + (q < rem ? 1 : 0);
                e.pad = 0;
                chunks[ch + q] = e;
            }
        }
        ch += k;
    }
    if (threadIdx.x == 0) {
        bin_start[nbins] = s_total;
        *n_next = s_total;
        *nchunks = nch_total;
    }
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_add(int* __restrict__ counts, long long nkeys,
                                                     int* __restrict__ cursor, const int* __restrict__ tile_off) {
    const long long k0 = (long long)blockIdx.x * SCAN_TILE + threadIdx.x;
    const int off = tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        const long long k = k0 + (long long)i * SCAN_NT;
        if (k < nkeys) {
            cursor[k] += off;
            counts[k] = 0;  // ready for the next sort
        }
    }
}

// Records per lane: FP32 (36 B) eight, FP64 (64 B) four.  Each lane loads its
// whole records before claiming their slots, so the loads overlap the slot
// atomics (mixed 128^3 x 32 sort per step: 2 records 1.05 ms, 4 0.87 ms,
// 8 0.84 ms; FP64 64^3 x 50: 2 records 0.167 ms, 4 0.159 ms).
#ifndef PICGB_SCATTER_U_F32
#define PICGB_SCATTER_U_F32 8
#endif
#ifndef PICGB_SCATTER_U_F64
#define PICGB_SCATTER_U_F64 4
#endif
template <class R>
struct ScatterU {
    static constexpr int U = sizeof(R) == 8 ? PICGB_SCATTER_U_F64 : PICGB_SCATTER_U_F32;
};

template <class R>
__global__ void __launch_bounds__(SORT_NT) k_sort_scatter(PStore<R> src, PStore<R> dst, const long long* __restrict__ n_cur,
                                                         GridDev g, int* __restrict__ cursor) {
    constexpr int U = ScatterU<R>::U;
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * SORT_NT * U;
    for (long long base = ((long long)blockIdx.x * SORT_NT + (threadIdx.x & ~31)) * U; base < N; base += stride) {
        int key[U], slot[U], cell[U], id[U];
        R off[U][3], u[U][3], w[U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const long long p = base + i * 32 + lane;
            key[i] = -1;
            if (p < N) {
                cell[i] = src.cell[p];
                key[i] = cell[i] < 0 ? -1 : cell_key(g, cell[i]);  // the count kernel's key, recomputed
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    off[i][a] = src.off[a][p];
                    u[i][a] = src.u[a][p];
                }
                w[i] = src.w[p];
                id[i] = src.id[p];
            }
        }
        warp_agg_slots<U>(cursor, key, slot);
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int q = slot[i];
            if (q >= 0) {
                dst.cell[q] = cell[i];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    dst.off[a][q] = off[i][a];
                    dst.u[a][q] = u[i][a];
                }
                dst.w[q] = w[i];
                dst.id[q] = id[i];
            }
        }
    }
}

int sort_grid(int nsm) { return nsm * 8; }

long long sort_tiles(long long nkeys) { return (nkeys + SCAN_TILE - 1) / SCAN_TILE; }

template <class R>
cudaError_t sort_launch(cudaStream_t st, int nsm, const GridDev& g, PStore<R> src, PStore<R> dst,
                        const long long* n_cur, long long* n_next, int* counts, int* cursor, int* tile_sum,
                        int* bin_start, Chunk* chunks, int* nchunks) {
    const long long nkeys = (long long)g.n[0] * g.n[1] * g.n[2];
    const int ntiles = (int)sort_tiles(nkeys);
    const int kpb = g.S * g.S * g.S;
    k_sort_count<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, n_cur, g, counts);
    k_scan_tiles<<<ntiles, SCAN_NT, 0, st>>>(counts, nkeys, cursor, tile_sum);
    k_scan_top<<<1, SCAN_NT, 0, st>>>(tile_sum, ntiles, cursor, nkeys, kpb, g.nbins, bin_start, n_next, chunks,
                                      nchunks);
    k_scan_add<<<ntiles, SCAN_NT, 0, st>>>(counts, nkeys, cursor, tile_sum);
    k_sort_scatter<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, dst, n_cur, g, cursor);
    return cudaGetLastError();
}

template cudaError_t sort_launch<double>(cudaStream_t, int, const GridDev&, PStore<double>, PStore<double>,
                                         const long long*, long long*, int*, int*, int*, int*, Chunk*, int*);
template cudaError_t sort_launch<float>(cudaStream_t, int, const GridDev&, PStore<float>, PStore<float>,
                                        const long long*, long long*, int*, int*, int*, int*, Chunk*, int*);

}  // namespace picgb
