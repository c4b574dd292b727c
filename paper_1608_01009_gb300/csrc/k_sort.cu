// Supercell counting sort of a species' particle store.
//
// arXiv:1608.01009 Sec. 3 stores particles per cell and Sec. 4.3 processes them
// by supercells of S^3 cells.  On the GPU the store is one structure of arrays
// ordered by supercell and, inside a supercell, by cell.  Before a particle
// could leave its supercell's one-cell slack (a fixed interval K with
// K * max(dt/d) < 1, or the displacement bound of the host's schedule) it is
// re-sorted by a counting sort over cell keys
//   key = supercell * S^3 + local cell,
// so that each supercell is a contiguous run of cell runs (the particle kernel
// relies on the cell order: warp lanes that share a cell share their gather
// loads and sum their currents before the shared-memory atomics):
//   k_sort_count  : histogram of keys, one atomic per run of equal keys in
//                   consecutive lanes; deactivated particles get no key
//   k_scan_tiles  : per tile of SCAN_TILE keys (whole bins), exclusive prefix
//                   into cursor[], the tile total, its bins' tile-local starts
//                   and the number of chunks they need
//   k_scan_top    : one CTA: scans of the per-tile particle and chunk totals,
//                   new particle count and chunk count
//   k_scan_add    : per tile: cursor[] += tile offset, the histogram cleared,
//                   the bin starts made global and the tile's part of the
//                   chunk table the particle kernel walks written (each bin cut
//                   into near-equal chunks of at most CHUNK particles)
//   k_sort_scatter_pipe: every active particle copied to its slot in the
//                   other buffer (order inside a cell unspecified), through
//                   shared-memory tiles loaded one tile ahead and written back
//                   in destination order; deactivated particles are dropped
//                   (compaction).  It recomputes each key from the cell it
//                   copies anyway, so no per-particle key array is written or
//                   read.
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

// Lane-interleaved groups of U x 32 particles per warp and iteration (U
// independent loads and atomics in flight per lane).
#ifndef PICGB_COUNT_U
#define PICGB_COUNT_U 4
#endif
#ifndef PICGB_RANK_U
#define PICGB_RANK_U 4
#endif
constexpr int COUNT_U = PICGB_COUNT_U, RANK_U = PICGB_RANK_U;

// Runs of equal keys in consecutive lanes (the store is sorted by key up to
// the particles that changed cell since the last sort): `head` is the first
// lane of this lane's run and `len` the run's length.  Equal keys in separate
// runs make separate runs, each claiming its own slots.
__device__ __forceinline__ void key_run(int key, int lane, int& head, int& len) {
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    const unsigned le = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;  // lanes 0..lane
    head = 31 - __clz(heads & le);
    const unsigned after = heads & ~le;
    len = (after ? __ffs(after) - 1 : 32) - head;
}

template <class R>
__global__ void __launch_bounds__(SORT_NT) k_sort_count(PStore<R> ps, const long long* __restrict__ n_cur, GridDev g,
                                                       int* __restrict__ counts) {
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * SORT_NT * COUNT_U;
    for (long long base = ((long long)blockIdx.x * SORT_NT + (threadIdx.x & ~31)) * COUNT_U; base < N;
         base += stride) {
        int key[COUNT_U];
#pragma unroll
        for (int i = 0; i < COUNT_U; ++i) {
            const long long p = base + i * 32 + lane;
            const int cp = p < N ? ps.cell[p] : INACTIVE;
            key[i] = cp < 0 ? -1 : cell_key(g, cp);
            if (key[i] >= 0 && !in_range(key[i], (long long)g.n[0] * g.n[1] * g.n[2])) key[i] = -1;  // debug build only
        }
#pragma unroll
        for (int i = 0; i < COUNT_U; ++i) {
            int head, len;
            key_run(key[i], lane, head, len);
            if (lane == head && key[i] >= 0) atomicAdd(&counts[key[i]], len);
        }
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

// Per tile of SCAN_TILE keys (whole bins: SCAN_TILE is a multiple of every
// S^3): tile-local exclusive prefix of the counts into cursor[], the tile's
// particle total, the tile-local start of each of its bins (into bin_start,
// made global by k_scan_add) and the number of chunks its bins need.
__global__ void __launch_bounds__(SCAN_NT) k_scan_tiles(const int* __restrict__ counts, long long nkeys,
                                                       int* __restrict__ cursor, int* __restrict__ tile_sum,
                                                       int keys_per_bin, int* __restrict__ bin_start,
                                                       int* __restrict__ tile_nch) {
    __shared__ int s[32];
    __shared__ int s_loc[SCAN_TILE / 8];  // tile-local bin starts (bins of >= 8 keys)
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    const long long k0 = base + (long long)threadIdx.x * SCAN_PER;
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
        const long long k = k0 + i;
        if (k < nkeys) {
            cursor[k] = run;
            const int kl = (int)(k - base);
            if (kl % keys_per_bin == 0) {
                s_loc[kl / keys_per_bin] = run;
                bin_start[k / keys_per_bin] = run;
            }
        }
        run += c[i];
    }
    __syncthreads();
    const long long left = nkeys - base;
    const int nb = (int)((left < SCAN_TILE ? left : SCAN_TILE) / keys_per_bin);
    int nch = 0;
    if ((int)threadIdx.x < nb) {
        const int t = threadIdx.x;
        const int cnt = (t + 1 < nb ? s_loc[t + 1] : total) - s_loc[t];
        nch = (cnt + CHUNK - 1) / CHUNK;
    }
    int nch_total;
    block_exclusive_scan(nch, s, &nch_total);
    if (threadIdx.x == 0) {
        tile_sum[blockIdx.x] = total;
        tile_nch[blockIdx.x] = nch_total;
    }
}

// In-place exclusive scan of v[0..n) by one CTA; returns the total.
__device__ int block_scan_inplace(int* v, int n, int* s) {
    const int per = (n + SCAN_NT - 1) / SCAN_NT;
    const int t0 = threadIdx.x * per, t1 = min(n, t0 + per);
    int sum = 0;
    for (int t = t0; t < t1; ++t) sum += v[t];
    int total;
    int run = block_exclusive_scan(sum, s, &total);
    for (int t = t0; t < t1; ++t) {
        const int x = v[t];
        v[t] = run;
        run += x;
    }
    return total;
}

// One CTA: tile particle offsets and tile chunk offsets (exclusive scans of
// the per-tile totals), the new particle count and the chunk count.
__global__ void __launch_bounds__(SCAN_NT) k_scan_top(int* __restrict__ tile_sum, int* __restrict__ tile_nch,
                                                     int ntiles, int nbins, int* __restrict__ bin_start,
                                                     long long* __restrict__ n_next, int* __restrict__ nchunks) {
    __shared__ int s[32];
    const int total = block_scan_inplace(tile_sum, ntiles, s);
    const int nch_total = block_scan_inplace(tile_nch, ntiles, s);
    if (threadIdx.x == 0) {
        bin_start[nbins] = total;
        *n_next = total;
        *nchunks = nch_total;
    }
}

// Per tile: cursor[] += tile offset (the histogram is cleared for the next
// sort); the tile's bin starts made global and its bins' chunks written (each
// bin cut into near-equal chunks of at most CHUNK particles).
__global__ void __launch_bounds__(SCAN_NT) k_scan_add(int* __restrict__ counts, long long nkeys,
                                                     int* __restrict__ cursor, const int* __restrict__ tile_off,
                                                     const int* __restrict__ tile_choff, int ntiles,
                                                     const long long* __restrict__ n_total, int keys_per_bin,
                                                     int* __restrict__ bin_start, Chunk* __restrict__ chunks) {
    __shared__ int s[32];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    const int off = tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        const long long k = base + threadIdx.x + (long long)i * SCAN_NT;
        if (k < nkeys) {
            cursor[k] += off;
            counts[k] = 0;  // ready for the next sort
        }
    }
    const long long left = nkeys - base;
    const int nb = (int)((left < SCAN_TILE ? left : SCAN_TILE) / keys_per_bin);
    const int b0 = (int)(base / keys_per_bin);
    const int tile_total = (blockIdx.x + 1 < ntiles ? tile_off[blockIdx.x + 1] : (int)*n_total) - off;
    const int t = threadIdx.x;
    int ls = 0, cnt = 0;
    if (t < nb) {
        ls = bin_start[b0 + t];  // tile-local starts (k_scan_tiles); read all before any is rewritten
        cnt = (t + 1 < nb ? bin_start[b0 + t + 1] : tile_total) - ls;
    }
    const int nch = (cnt + CHUNK - 1) / CHUNK;
    int nch_total;
    const int ch = tile_choff[blockIdx.x] + block_exclusive_scan(nch, s, &nch_total);  // (synchronises)
    if (t < nb) {
        const int st = off + ls;
        bin_start[b0 + t] = st;
        if (nch > 0) {
            const int q0 = cnt / nch, rem = cnt % nch;
            for (int q = 0; q < nch; ++q) {
                Chunk e;
                e.sc = b0 + t;
                e.start = st + q * q0 + min(q, rem);
                e.count = q0 + (q < rem ? 1 : 0);
                e.pad = 0;
                chunks[ch + q] = e;
            }
        }
    }
}

constexpr int SW = 1024;  // keys per window of the scatter

#ifndef PICGB_PIPE_TILE32
#define PICGB_PIPE_TILE32 1024
#endif
#ifndef PICGB_PIPE_TILE64
#define PICGB_PIPE_TILE64 256
#endif
#ifndef PICGB_PIPE_NT
#define PICGB_PIPE_NT 256
#endif
constexpr int PIPE_NT = PICGB_PIPE_NT;  // threads of the pipelined scatter
// Pipelined tiled scatter.  A scatter that claims slots per warp writes every
// cell run in pieces claimed by different warps at different times, and a
// piece's ends leave 32-byte sectors partly written (DRAM writes 31% above the
// moved bytes on a 96^3 x 32 FP32 capture).  Here each CTA takes tiles of
// consecutive records:
//   * keys inside a window of SW keys from a quarter window below the tile's
//     first key take their rank within the tile from shared-memory counters
//     (one claim per run of equal keys), the window is scanned, and each key
//     present claims one contiguous slot range of the destination with one
//     global atomic;
//   * keys outside the window (moves into far supercells) claim their slots
//     from the global cursor and are stored directly;
//   * the window's records are written out through a permutation (s_src: the
//     stage position of each destination-ordered slot), so consecutive threads
//     write consecutive slots of each cell run.
// The records are not held in registers: each CTA keeps two tile stages in
// shared memory, filled by bulk asynchronous copies (one per array) while the
// previous tile is ranked and written (tile t + gridDim loads during tile t).
template <class R>
struct PipeScatter {
    static constexpr int TILE = sizeof(R) == 8 ? PICGB_PIPE_TILE64 : PICGB_PIPE_TILE32;  // records per tile
    static constexpr int TR = TILE / PIPE_NT;
    static_assert(TR * PIPE_NT == TILE && TILE % 4 == 0, "tile: whole records per thread, 16-byte copies");
    // stage: 3 offsets, 3 momenta, weight (R), then cell and id (int)
    static constexpr size_t STAGE = (size_t)TILE * (7 * sizeof(R) + 2 * sizeof(int));
    // two stages, destination slot and stage position of each ordered record, window counts and claims
    static constexpr size_t SMEM = 2 * STAGE + (size_t)TILE * 2 * sizeof(int) + 2 * SW * sizeof(int) + 32 * sizeof(int);
};

template <class R>
__global__ void __launch_bounds__(PIPE_NT) k_sort_scatter_pipe(PStore<R> src, PStore<R> dst,
                                                              const long long* __restrict__ n_cur, GridDev g,
                                                              int* __restrict__ cursor, int* __restrict__ err) {
    using PS = PipeScatter<R>;
    constexpr int TILE = PS::TILE, TR = PS::TR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* s_slot = reinterpret_cast<int*>(smem_raw + 2 * PS::STAGE);  // TILE
    int* s_src = s_slot + TILE;                                        // TILE
    int* s_cnt = s_src + TILE;                                         // SW: counts, then tile positions
    int* s_gb = s_cnt + SW;                                            // SW: first slot of each key's claim
    int* s_scan = s_gb + SW;                                           // 32 warp totals of the block scan
    __shared__ uint64_t bar[2];
    __shared__ int s_kb, s_nw;
    const long long N = *n_cur;
    const long long ntile = (N + TILE - 1) / TILE;
    const int lane = threadIdx.x & 31;
    const auto stR = [&](int st) { return reinterpret_cast<R*>(smem_raw + st * PS::STAGE); };
    const auto stI = [&](int st) { return reinterpret_cast<int*>(smem_raw + st * PS::STAGE + 7 * TILE * sizeof(R)); };
    // the copies of tile t into stage st (thread 0): every array of the store is
    // allocated to a multiple of 4 records, so rounding the last tile's copies
    // up to 16 bytes stays inside it
    const auto issue = [&](long long t, int st) {
        const long long base = t * TILE;
        const long long nrec = min((long long)TILE, N - base);
        const uint32_t nR = (uint32_t)((nrec * sizeof(R) + 15) & ~15ll), nI = (uint32_t)((nrec * 4 + 15) & ~15ll);
        R* sr = stR(st);
        int* si = stI(st);
        fence_proxy_async();
        mbar_expect_tx(&bar[st], 7 * nR + 2 * nI);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bulk_load(sr + a * TILE, src.off[a] + base, nR, &bar[st]);
            bulk_load(sr + (3 + a) * TILE, src.u[a] + base, nR, &bar[st]);
        }
        bulk_load(sr + 6 * TILE, src.w + base, nR, &bar[st]);
        bulk_load(si, src.cell + base, nI, &bar[st]);
        bulk_load(si + TILE, src.id + base, nI, &bar[st]);
    };
    const long long nkeys = (long long)g.n[0] * g.n[1] * g.n[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < SW; i += PIPE_NT) s_cnt[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < ntile) issue(blockIdx.x, 0);
    uint32_t phase = 0;  // bit st: parity of stage st's next completion
    int st = 0;
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x, st ^= 1) {
        const long long tn = t + gridDim.x;
        // the other stage was released by the barrier that ended the previous tile
        if (threadIdx.x == 0 && tn < ntile) issue(tn, st ^ 1);
        const bool ok = mbar_wait_bounded(&bar[st], (phase >> st) & 1u, WAIT_LIMIT, WAIT_LIMIT_NS);
        phase ^= 1u << st;
        if (__syncthreads_or(!ok)) {
            // leave only once the copy already issued into the other stage has landed
            if (tn < ntile) mbar_wait_bounded(&bar[st ^ 1], (phase >> (st ^ 1)) & 1u, WAIT_LIMIT, WAIT_LIMIT_NS);
            if (threadIdx.x == 0) atomicOr(err, ERRBIT_TIMEOUT);
            return;
        }
        const long long base = t * TILE;
        const R* sr = stR(st);
        const int* si = stI(st);
        // window: from a quarter window below the first active key of the tile's first 32 records
        if (threadIdx.x < 32) {
            // the block scan reads 32 warp totals (8 warps write theirs) and leaves its
            // running total in all 32: cleared for every tile
            s_scan[threadIdx.x] = 0;
            const int cp = base + lane < N ? si[lane] : INACTIVE;
            const unsigned act = __ballot_sync(0xffffffffu, cp >= 0);
            const int k = cp >= 0 ? cell_key(g, cp) : 0;
            const int k0 = __shfl_sync(0xffffffffu, k, act ? __ffs(act) - 1 : 0);
            if (lane == 0) s_kb = act ? max(0, k0 - SW / 4) : 0;
        }
        __syncthreads();
        const int kb = s_kb;
        int key[TR], rank[TR];
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const int r = i * PIPE_NT + threadIdx.x;
            key[i] = -1;
            if (base + r < N) {
                const int cp = si[r];
                key[i] = cp < 0 ? -1 : cell_key(g, cp);
                if (key[i] >= 0 && !in_range(key[i], nkeys)) key[i] = -1;  // debug build only
            }
            const bool inw = key[i] >= kb && key[i] < kb + SW;
            // a run of one key claims its ranks with one atomic: in-window keys from
            // the shared counters, the others from the global cursor
            int head, len;
            key_run(key[i], lane, head, len);
            int b = 0;
            if (lane == head) {
                if (inw) b = atomicAdd(&s_cnt[key[i] - kb], len);
                else if (key[i] >= 0) b = atomicAdd(&cursor[key[i]], len);
            }
            b = __shfl_sync(0xffffffffu, b, head);
            rank[i] = key[i] >= 0 ? b + lane - head : -1;
        }
        __syncthreads();
        // exclusive scan of the window counts (tile positions); one global claim per key present
        {
            constexpr int PER = SW / PIPE_NT;
            int c[PER], sum = 0;
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                c[j] = s_cnt[threadIdx.x * PER + j];
                sum += c[j];
            }
            int total;
            int run = block_exclusive_scan(sum, s_scan, &total);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int k = threadIdx.x * PER + j;
                s_cnt[k] = run;
                s_gb[k] = c[j] && in_range(kb + k, nkeys) ? atomicAdd(&cursor[kb + k], c[j]) : 0;
                run += c[j];
            }
            if (threadIdx.x == 0) s_nw = total;
        }
        __syncthreads();
        // window records: their destination-ordered position; the others are stored directly
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            if (key[i] < 0) continue;
            const int r = i * PIPE_NT + threadIdx.x;
            if (key[i] >= kb && key[i] < kb + SW) {
                const int tp = s_cnt[key[i] - kb] + rank[i];
                if (!in_range(tp, TILE)) continue;  // debug build only
                s_slot[tp] = s_gb[key[i] - kb] + rank[i];
                s_src[tp] = r;
            } else {
                const int q = rank[i];
                if (!in_range(q, N)) continue;  // debug build only
                dst.cell[q] = si[r];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    dst.off[a][q] = sr[a * TILE + r];
                    dst.u[a][q] = sr[(3 + a) * TILE + r];
                }
                dst.w[q] = sr[6 * TILE + r];
                dst.id[q] = si[TILE + r];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < SW; i += PIPE_NT) s_cnt[i] = 0;  // positions read above; counts of the next tile
        const int nw = in_range(s_nw, TILE + 1) ? s_nw : 0;  // the check: debug build only
        for (int tp = threadIdx.x; tp < nw; tp += PIPE_NT) {
            const int q = s_slot[tp], r = s_src[tp];
            if (!in_range(q, N) || !in_range(r, TILE)) continue;  // debug build only
            dst.cell[q] = si[r];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dst.off[a][q] = sr[a * TILE + r];
                dst.u[a][q] = sr[(3 + a) * TILE + r];
            }
            dst.w[q] = sr[6 * TILE + r];
            dst.id[q] = si[TILE + r];
        }
        __syncthreads();
    }
}

// Ranks only: each active particle's destination slot, as perm[slot] = its
// index in the current store (one atomic per run of equal keys in consecutive
// lanes).  The particle kernel then reads particle perm[i] and writes it to
// slot i of the other buffer, so the particles move once per step instead of
// twice (scatter, then push in place).
template <class R>
__global__ void __launch_bounds__(SORT_NT) k_sort_rank(PStore<R> ps, const long long* __restrict__ n_cur,
                                                      const long long* __restrict__ n_next, GridDev g,
                                                      int* __restrict__ cursor, int* __restrict__ perm) {
    const long long N = *n_cur, M = *n_next;
    const long long nkeys = (long long)g.n[0] * g.n[1] * g.n[2];
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * SORT_NT * RANK_U;
    for (long long b = ((long long)blockIdx.x * SORT_NT + (threadIdx.x & ~31)) * RANK_U; b < N; b += stride) {
        int key[RANK_U], head[RANK_U], len[RANK_U], s0[RANK_U];
#pragma unroll
        for (int i = 0; i < RANK_U; ++i) {
            const long long p = b + i * 32 + lane;
            const int cp = p < N ? ps.cell[p] : INACTIVE;
            key[i] = cp < 0 ? -1 : cell_key(g, cp);
            if (key[i] >= 0 && !in_range(key[i], nkeys)) key[i] = -1;  // debug build only
        }
#pragma unroll
        for (int i = 0; i < RANK_U; ++i) {
            key_run(key[i], lane, head[i], len[i]);
            s0[i] = lane == head[i] && key[i] >= 0 ? atomicAdd(&cursor[key[i]], len[i]) : 0;
        }
#pragma unroll
        for (int i = 0; i < RANK_U; ++i) {
            const int base = __shfl_sync(0xffffffffu, s0[i], head[i]);
            const long long slot = (long long)base + (lane - head[i]);
            if (key[i] >= 0 && in_range(slot, M)) perm[slot] = (int)(b + i * 32 + lane);
        }
    }
}

// Apply a pending permutation without a particle step: slot i of dst gets
// particle perm[i] of src, every field (for callers that read or replace the
// store before the next particle kernel would have moved it).
template <class R>
__global__ void __launch_bounds__(SORT_NT) k_apply_perm(PStore<R> src, PStore<R> dst, const long long* __restrict__ n,
                                                       const int* __restrict__ perm) {
    const long long N = *n;
    for (long long i = (long long)blockIdx.x * SORT_NT + threadIdx.x; i < N; i += (long long)gridDim.x * SORT_NT) {
        const int q = perm[i];
        dst.cell[i] = src.cell[q];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dst.off[a][i] = src.off[a][q];
            dst.u[a][i] = src.u[a][q];
        }
        dst.w[i] = src.w[q];
        dst.id[i] = src.id[q];
    }
}

template <class R>
cudaError_t apply_perm_launch(cudaStream_t st, int nsm, PStore<R> src, PStore<R> dst, const long long* n,
                              const int* perm) {
    k_apply_perm<R><<<nsm * 8, SORT_NT, 0, st>>>(src, dst, n, perm);
    return cudaGetLastError();
}
template cudaError_t apply_perm_launch<double>(cudaStream_t, int, PStore<double>, PStore<double>, const long long*,
                                               const int*);
template cudaError_t apply_perm_launch<float>(cudaStream_t, int, PStore<float>, PStore<float>, const long long*,
                                              const int*);

int sort_grid(int nsm) { return nsm * 8; }

long long sort_tiles(long long nkeys) { return (nkeys + SCAN_TILE - 1) / SCAN_TILE; }

// Size of the per-tile scratch (particle and chunk totals) the sort needs.
long long sort_tile_scratch(long long nkeys) { return 2 * sort_tiles(nkeys); }

template <class R>
cudaError_t sort_launch(cudaStream_t st, int nsm, const GridDev& g, PStore<R> src, PStore<R> dst,
                        const long long* n_cur, long long* n_next, int* counts, int* cursor, int* tile_sum,
                        int* bin_start, Chunk* chunks, int* nchunks, int* err) {
    const long long nkeys = (long long)g.n[0] * g.n[1] * g.n[2];
    const int ntiles = (int)sort_tiles(nkeys);
    const int kpb = g.S * g.S * g.S;
    int* tile_nch = tile_sum + ntiles;
    k_sort_count<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, n_cur, g, counts);
    k_scan_tiles<<<ntiles, SCAN_NT, 0, st>>>(counts, nkeys, cursor, tile_sum, kpb, bin_start, tile_nch);
    k_scan_top<<<1, SCAN_NT, 0, st>>>(tile_sum, tile_nch, ntiles, g.nbins, bin_start, n_next, nchunks);
    k_scan_add<<<ntiles, SCAN_NT, 0, st>>>(counts, nkeys, cursor, tile_sum, tile_nch, ntiles, n_next, kpb, bin_start,
                                           chunks);
    constexpr int sm = (int)PipeScatter<R>::SMEM;
    const cudaError_t e = cudaFuncSetAttribute(k_sort_scatter_pipe<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_scatter_pipe<R>, PIPE_NT, sm);
    k_sort_scatter_pipe<R><<<nsm * (per_sm > 0 ? per_sm : 1), PIPE_NT, sm, st>>>(src, dst, n_cur, g, cursor, err);
    return cudaGetLastError();
}

// The sort without its data movement: count, scans, chunk table, and the
// destination permutation of the current store (see k_sort_rank).
template <class R>
cudaError_t sort_rank_launch(cudaStream_t st, int nsm, const GridDev& g, PStore<R> src, const long long* n_cur,
                             long long* n_next, int* counts, int* cursor, int* tile_sum, int* bin_start,
                             Chunk* chunks, int* nchunks, int* perm) {
    const long long nkeys = (long long)g.n[0] * g.n[1] * g.n[2];
    const int ntiles = (int)sort_tiles(nkeys);
    const int kpb = g.S * g.S * g.S;
    int* tile_nch = tile_sum + ntiles;
    k_sort_count<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, n_cur, g, counts);
    k_scan_tiles<<<ntiles, SCAN_NT, 0, st>>>(counts, nkeys, cursor, tile_sum, kpb, bin_start, tile_nch);
    k_scan_top<<<1, SCAN_NT, 0, st>>>(tile_sum, tile_nch, ntiles, g.nbins, bin_start, n_next, nchunks);
    k_scan_add<<<ntiles, SCAN_NT, 0, st>>>(counts, nkeys, cursor, tile_sum, tile_nch, ntiles, n_next, kpb, bin_start,
                                           chunks);
    k_sort_rank<R><<<sort_grid(nsm), SORT_NT, 0, st>>>(src, n_cur, n_next, g, cursor, perm);
    return cudaGetLastError();
}

template cudaError_t sort_rank_launch<double>(cudaStream_t, int, const GridDev&, PStore<double>, const long long*,
                                              long long*, int*, int*, int*, int*, Chunk*, int*, int*);
template cudaError_t sort_rank_launch<float>(cudaStream_t, int, const GridDev&, PStore<float>, const long long*,
                                             long long*, int*, int*, int*, int*, Chunk*, int*, int*);

template cudaError_t sort_launch<double>(cudaStream_t, int, const GridDev&, PStore<double>, PStore<double>,
                                         const long long*, long long*, int*, int*, int*, int*, Chunk*, int*, int*);
template cudaError_t sort_launch<float>(cudaStream_t, int, const GridDev&, PStore<float>, PStore<float>,
                                        const long long*, long long*, int*, int*, int*, int*, Chunk*, int*, int*);

PICGB_INDEX_FLAG_READER(sort_index_flags)

}  // namespace picgb
