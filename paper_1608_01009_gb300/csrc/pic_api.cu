// C ABI of libpicgb (declared in include/pic.h): context, species stores,
// step scheduling, diagnostics and error reporting.  Every compute step runs
// in the CUDA kernels of this library; there is no host fallback.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace picgb {

// launchers defined in the kernel translation units
cudaError_t fdtd_b_launch(cudaStream_t, double*, const GridDev&, double, int, float*, double*);
cudaError_t fdtd_e_launch(cudaStream_t, double*, double*, double*, const GridDev&);
cudaError_t refresh_launch(cudaStream_t, double*, const GridDev&, float*);
cudaError_t damp_table_launch(cudaStream_t, const GridDev&, double*);
cudaError_t field_energy_launch(cudaStream_t, const double*, const GridDev&, double*);
int fdtd_blocks(const GridDev&);
template <class R>
cudaError_t sort_launch(cudaStream_t, int, const GridDev&, PStore<R>, PStore<R>, const long long*, long long*, int*,
                        int*, int*, int*, Chunk*, int*, int*);
template <class R>
cudaError_t sort_rank_launch(cudaStream_t, int, const GridDev&, PStore<R>, const long long*, long long*, int*, int*,
                             int*, int*, Chunk*, int*, int*);
template <class R>
cudaError_t apply_perm_launch(cudaStream_t, int, PStore<R>, PStore<R>, const long long*, const int*);
long long sort_tiles(long long nkeys);
long long sort_tile_scratch(long long nkeys);
template <class R>
cudaError_t load_launch(cudaStream_t, long long, const double* const*, const PStore<R>&, const GridDev&);
template <class R>
cudaError_t unload_launch(cudaStream_t, int, const PStore<R>&, const long long*, const GridDev&, int*, long long,
                          long long*, double* const*);
template <class R>
cudaError_t count_launch(cudaStream_t, int, const PStore<R>&, const long long*, int*);
template <class R>
cudaError_t kinetic_launch(cudaStream_t, int, const PStore<R>&, const long long*, double, double*);
cudaError_t energy_finalize_launch(cudaStream_t, const double*, int, const double*, int, double, double*);
cudaError_t tsc_launch(int, cudaStream_t, const PushParams&, const PStore<double>&, const long long*, const double*,
                       double*, double*);
cudaError_t wait_probe_launch(cudaStream_t, int*, uint64_t);

// rows of the per-push displacement record: the longest run between two sorts
// under the displacement-bounded schedule
constexpr int DRIFT_ROWS = 64;

// differentiable path (k_adjoint.cu)
cudaError_t tape_step_launch(cudaStream_t, const TapeDev&, long long, const StepParams&, const double*, double*);
cudaError_t tape_move_launch(cudaStream_t, const TapeDev&, const TapeDev&, long long, const StepParams&);
cudaError_t tape_seed_launch(cudaStream_t, const TapeDev&, const LamDev&, long long, double, double);
cudaError_t tape_adjoint_launch(cudaStream_t, const TapeDev&, const LamDev&, long long, const StepParams&,
                                const double*, const double*, double*);
cudaError_t tape_kinetic_launch(cudaStream_t, int, const TapeDev&, long long, double, double*);
template <class R>
cudaError_t tape_from_store_launch(cudaStream_t, int, const PStore<R>&, const long long*, const TapeDev&, double*,
                                   long long);
cudaError_t tape_to_phys_launch(cudaStream_t, const TapeDev&, long long, const GridDev&, double* const*);
cudaError_t lam_to_phys_launch(cudaStream_t, const LamDev&, long long, const GridDev&, double* const*);
cudaError_t adj_fields_launch(cudaStream_t, double*, double*, const GridDev&);
cudaError_t adj_fold_add_launch(cudaStream_t, double*, double*, const GridDev&);

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <class R>
struct Store {
    PStore<R> buf[2];
    int cur = 0;
    PStore<R>& a() { return buf[cur]; }
    PStore<R>& b() { return buf[cur ^ 1]; }
};

struct Species {
    double q = 0, m = 1;
    // destination permutation of the last ranks-only sort (cap ints); the next
    // particle kernel moves the store through it into the other buffer
    int* d_perm = nullptr;
    bool perm_pending = false;
    bool immobile = false;         // neutralising background: no particles stored
    long long cap = 0;
    Store<double> s64;
    Store<float> s32;
    long long* d_n = nullptr;      // d_n[0] current count, d_n[1] count after the pending sort
    int* d_bin_start = nullptr;
    Chunk* d_chunks = nullptr;
    int* d_nchunks = nullptr;
    double* d_ek = nullptr;        // kinetic-energy partials of the last push (push_grid entries)
    float* d_wmax = nullptr;       // mixed: largest |w| of the store (scale of the fixed-point current)
    double* d_stage = nullptr;     // 7 x cap FP64 staging area for host uploads (allocated on first use)
    // asynchronous upload (pic_upload_particles): 7 x up_cap FP64 arrays filled on
    // the copy stream; up_n >= 0 while an upload waits to be consumed.  Not part
    // of `allocs`: a re-allocation of the store leaves a pending upload intact.
    double* d_up = nullptr;
    long long up_cap = 0, up_n = -1;
    cudaEvent_t up_done = nullptr;  // recorded on the copy stream after the copy
    cudaEvent_t up_free = nullptr;  // recorded on the stream after the load that read the area
    long long nid = 0;             // ids 0..nid-1 were given at the last load
    std::vector<void*> allocs;
};

// Recorded differentiable run: id-ordered FP64 particle states of every
// species, full checkpoints every K steps, and for the segment being reversed
// the momentum of every step plus the positions and active flags of every
// B-th step (B = ceil(sqrt(K))).  The positions of the other steps of a block
// of B are rebuilt once, when the reverse sweep enters the block, by the
// forward's own move (k_tape_move), bit for bit.  A step's record costs
// 24 B per particle instead of the 52 B of a whole state, so the same memory
// keeps about twice as many steps without a replay.
struct TapeSpecies {
    long long n = 0;
    double* w = nullptr;
    TapeDev cur{};
    LamDev lam{};
    std::vector<TapeDev> ck;  // whole states at the segment starts (a one-segment tape keeps none)
    std::vector<TapeDev> us;  // u^{m-1/2} of step m of the segment (u only)
    std::vector<TapeDev> xs;  // x^m and flags of steps m = 0, B, 2B, ... (xi and act only)
    std::vector<TapeDev> xw;  // x^{m0 + j} and flags, j = 1..B-1, of the block rebuilt last
    int blk = -1;             // first step m0 of that block (-1: none)
};

struct Tape {
    bool ready = false;
    int nsteps = 0, K = 1, B = 1;
    int snap_seg = -1;  // checkpoint segment whose per-step records `us`, `xs`, `snapEB` hold (-1: none)
    std::vector<TapeSpecies> sp;
    std::vector<double*> ckEB, snapEB;
    double* finalEB = nullptr;
    double* L = nullptr;     // cotangents of E, B (6 padded components)
    double* LJ = nullptr;    // cotangent of J (3 padded components, ghosts filled)
    double* scat = nullptr;  // gather cotangents scattered by the particles (6 padded)
    std::vector<void*> allocs;
    void release() {
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
        sp.clear();
        ckEB.clear();
        snapEB.clear();
        finalEB = L = LJ = scat = nullptr;
        ready = false;
        snap_seg = -1;
    }
};

}  // namespace picgb

using namespace picgb;

struct pic_ctx {
    pic_grid_desc desc{};
    GridDev g{};
    cudaStream_t st = nullptr;
    cudaStream_t cst = nullptr;  // copy stream of asynchronous uploads (created on first use)
    int dev = 0, nsm = 0;
    bool mixed = false;
    int K = 1, since_sort = 0;
    long long steps = 0;
    // Displacement-bounded sort schedule (mixed precision with sort_interval 0):
    // the particle kernel records the largest gamma^2 of each push in row
    // since_sort of d_drift, that is the largest speed v_i = sqrt(1 - 1/gamma^2)
    // (units of c) of push i, and a sort is due once (sum_i v_i + 1) dt/d_a --
    // the displacement bound since the last sort plus one more step at the
    // speed of light -- could reach the one-cell slack of the supercell tile.
    bool adaptive = false;
    unsigned* d_drift = nullptr;  // DRIFT_ROWS float bit patterns, zero after each sort
    double vsum0 = 0.0;           // speeds summed before row 0 (a restored state), zero after each sort
    double dtd[3] = {0, 0, 0};    // dt / d_a: a step's largest displacement at speed c (cells)
    cudaEvent_t ev_push = nullptr;
    cudaStream_t xst = nullptr;   // reads of d_drift (non-blocking: they do not wait for the field kernels)
    double* EB = nullptr;
    double* J = nullptr;
    double* Jlast = nullptr;
    float* EB32 = nullptr;
    CUtensorMap tm64{}, tm32{};
    int push_grid = 0;
    XQueue<double> xq64{};  // crossing-move queues of the particle kernel (push_grid x CHUNK entries)
    XQueue<float> xq32{};
    std::vector<Species> sp;
    int* d_err = nullptr;
    int* d_counts = nullptr;    // per-cell histogram of the sort (ncell)
    int* d_cursor = nullptr;    // per-cell scatter cursor (ncell)
    int* d_tile_sum = nullptr;  // per-tile totals of the sort's scan
    int* d_counter = nullptr;
    double* d_wf = nullptr;     // field-energy partials (fdtd blocks)
    double* d_ekall = nullptr;  // kinetic partials, contiguous over species
    double* d_energy = nullptr; // [wf, wk] of the last finalize
    bool energy_fresh = false;  // d_energy describes the current state
    std::string err;
    long long launches = 0;
    bool timing = false;
    double stage_ms[4] = {0, 0, 0, 0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
    std::vector<void*> allocs;
    Tape tape;
};

namespace {

int fail(pic_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CUDA_TRY(c, call)                                                                             \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail((c), PIC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int dalloc(pic_ctx* c, std::vector<void*>& list, T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PIC_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    list.push_back(q);
    *p = static_cast<T*>(q);
    return PIC_OK;
}

int validate(const pic_grid_desc* g, pic_ctx* c) {
    if (!g) return fail(c, PIC_ERR_ARG, "null descriptor");
    int S = g->supercell;
    if (g->precision != PIC_FP64 && g->precision != PIC_MIXED) return fail(c, PIC_ERR_ARG, "bad precision");
    if (!(S == 4 || S == 8 || (S == 2 && g->precision == PIC_FP64)))
        return fail(c, PIC_ERR_ARG, "supercell must be 4 or 8 (2 for FP64 only), got %d", S);
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] < 4 || g->n[a] > 1024) return fail(c, PIC_ERR_ARG, "n[%d]=%d outside 4..1024", a, g->n[a]);
        if (g->n[a] % S) return fail(c, PIC_ERR_ARG, "n[%d]=%d not a multiple of supercell %d", a, g->n[a], S);
        if (!(g->d[a] > 0) || !std::isfinite(g->d[a])) return fail(c, PIC_ERR_ARG, "cell size d[%d] must be > 0", a);
        if (g->bc[a] != PIC_BC_PERIODIC && g->bc[a] != PIC_BC_ABSORBING) return fail(c, PIC_ERR_ARG, "bad bc[%d]", a);
        if (g->bc[a] == PIC_BC_ABSORBING && 2 * g->absorb_cells > g->n[a])
            return fail(c, PIC_ERR_ARG, "absorbing layer wider than half the axis %d", a);
    }
    if (!(g->dt > 0) || !std::isfinite(g->dt)) return fail(c, PIC_ERR_ARG, "dt must be > 0");
    if (g->absorb_cells < 0 || !(g->absorb_sigma >= 0 && g->absorb_sigma <= 1))
        return fail(c, PIC_ERR_ARG, "absorbing layer: cells >= 0 and 0 <= sigma <= 1 required");
    if ((long long)g->n[0] * g->n[1] * g->n[2] > (1LL << 30)) return fail(c, PIC_ERR_ARG, "grid too large");
    double s = 0, dmax = 0;
    for (int a = 0; a < 3; ++a) {
        s += 1.0 / (g->d[a] * g->d[a]);
        dmax = std::fmax(dmax, g->dt / g->d[a]);
    }
    double courant = g->dt * std::sqrt(s);
    if (!(courant < 1.0)) return fail(c, PIC_ERR_CFL, "Courant number %.6f >= 1", courant);
    if (g->sort_interval < 0) return fail(c, PIC_ERR_ARG, "sort_interval < 0");
    if (g->sort_interval > 0 && !(g->sort_interval * dmax < 1.0))
        return fail(c, PIC_ERR_CFL, "sort_interval %d * max(dt/d) = %.4f must be < 1 (supercell slack is one cell)",
                    g->sort_interval, g->sort_interval * dmax);
    if (g->precision == PIC_MIXED && S % 4) return fail(c, PIC_ERR_ARG, "mixed precision needs supercell 4 or 8");
    if (g->form_factor < 0 || g->form_factor > 2) return fail(c, PIC_ERR_ARG, "form_factor must be 0, 1 or 2");
    if (g->form_factor == 2 && g->precision != PIC_FP64)
        return fail(c, PIC_ERR_ARG, "the second-order form factor runs in FP64 only");
    return PIC_OK;
}

int encode_tmap(pic_ctx* c, CUtensorMap* map, void* base, bool fp32) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        CUDA_TRY(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !f) return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    const GridDev& g = c->g;
    const size_t es = fp32 ? 4 : 8;
    const cuuint32_t T = (cuuint32_t)(g.S + 4);
    cuuint64_t dims[4] = {(cuuint64_t)g.np[0], (cuuint64_t)g.np[1], (cuuint64_t)g.np[2], 6};
    cuuint64_t strides[3] = {(cuuint64_t)g.np[0] * es, (cuuint64_t)g.np[0] * g.np[1] * es, (cuuint64_t)g.P * es};
    cuuint32_t box[4] = {T, T, T, 6};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PIC_OK;
}

template <class R>
int push_dispatch_setup(pic_ctx* c, int S, int* bps) {
    cudaError_t e = cudaErrorInvalidValue;
    if constexpr (sizeof(R) == 4) {
        if (S == 4) e = push32_setup<4>(bps);
        if (S == 8) e = push32_setup<8>(bps);
    } else {
        if (S == 2) e = push_setup<double, 2>(bps);
        if (S == 4) e = push_setup<double, 4>(bps);
        if (S == 8) e = push_setup<double, 8>(bps);
    }
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "push kernel setup: %s", cudaGetErrorString(e));
    return PIC_OK;
}

PushParams make_params(const pic_ctx* c, const Species& s) {
    PushParams pp;
    pp.g = c->g;
    pp.qdt2m = 0.5 * s.q * c->g.dt / s.m;
    for (int a = 0; a < 3; ++a) {
        pp.dtd[a] = c->g.dt / c->g.d[a];
        pp.cq[a] = s.q / (c->g.dt * c->g.d[(a + 1) % 3] * c->g.d[(a + 2) % 3]);
    }
    pp.mass = s.m;
    pp.wmax = s.d_wmax;
    pp.drift = nullptr;
    pp.qdt2m_f = (float)pp.qdt2m;
    for (int a = 0; a < 3; ++a) {
        pp.dtd_f[a] = (float)pp.dtd[a];
        pp.cq_f[a] = (float)pp.cq[a];
    }
    return pp;
}

void stage_begin(pic_ctx* c, int stage, cudaEvent_t* e0) {
    if (!c->timing) return;
    cudaEventCreate(e0);
    cudaEventRecord(*e0, c->st);
    (void)stage;
}

void stage_end(pic_ctx* c, int stage, cudaEvent_t e0) {
    if (!c->timing) return;
    cudaEvent_t e1;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, c->st);
    c->ev[stage].push_back({e0, e1});
}

template <class R>
Store<R>& store_of(Species& s);
template <>
Store<double>& store_of<double>(Species& s) { return s.s64; }
template <>
Store<float>& store_of<float>(Species& s) { return s.s32; }

template <class R>
int sort_species(pic_ctx* c, Species& s) {
    Store<R>& st = store_of<R>(s);
    cudaError_t e = sort_launch<R>(c->st, c->nsm, c->g, st.a(), st.b(), s.d_n, s.d_n + 1, c->d_counts,
                                   c->d_cursor, c->d_tile_sum, s.d_bin_start, s.d_chunks, s.d_nchunks, c->d_err);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "sort launch: %s", cudaGetErrorString(e));
    c->launches += 5;
    st.cur ^= 1;
    CUDA_TRY(c, cudaMemcpyAsync(s.d_n, s.d_n + 1, sizeof(long long), cudaMemcpyDeviceToDevice, c->st));
    return PIC_OK;
}

// The cloud-in-cell paths' sort (before a step, and after a load): ranks only
// (count, scans, chunk table, destination permutation); the next particle
// kernel launch moves the particles through the permutation into the other
// buffer, or materialize() does when another entry point needs them first.
template <class R>
int sort_species_ranks(pic_ctx* c, Species& s) {
    Store<R>& st = store_of<R>(s);
    const cudaError_t e = sort_rank_launch<R>(c->st, c->nsm, c->g, st.a(), s.d_n, s.d_n + 1, c->d_counts, c->d_cursor,
                                              c->d_tile_sum, s.d_bin_start, s.d_chunks, s.d_nchunks, s.d_perm);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "sort launch: %s", cudaGetErrorString(e));
    return PIC_OK;
}

int sort_all_ranks(pic_ctx* c) {
    for (auto& s : c->sp) {
        if (s.immobile) continue;
        const int r = c->mixed ? sort_species_ranks<float>(c, s) : sort_species_ranks<double>(c, s);
        if (r) return r;
        c->launches += 5;
        s.perm_pending = true;
        CUDA_TRY(c, cudaMemcpyAsync(s.d_n, s.d_n + 1, sizeof(long long), cudaMemcpyDeviceToDevice, c->st));
    }
    c->since_sort = 0;
    c->vsum0 = 0.0;
    if (c->d_drift) CUDA_TRY(c, cudaMemsetAsync(c->d_drift, 0, DRIFT_ROWS * sizeof(unsigned), c->st));
    return PIC_OK;
}

// Move the records of every species with a pending permutation into sorted
// order now (for the entry points that read, sort or replace the store before
// a particle step would have moved them).
int materialize(pic_ctx* c) {
    for (auto& s : c->sp) {
        if (!s.perm_pending) continue;
        cudaError_t e;
        if (c->mixed) {
            e = apply_perm_launch<float>(c->st, c->nsm, s.s32.a(), s.s32.b(), s.d_n, s.d_perm);
            if (e == cudaSuccess) s.s32.cur ^= 1;
        } else {
            e = apply_perm_launch<double>(c->st, c->nsm, s.s64.a(), s.s64.b(), s.d_n, s.d_perm);
            if (e == cudaSuccess) s.s64.cur ^= 1;
        }
        if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "permutation: %s", cudaGetErrorString(e));
        c->launches += 1;
        s.perm_pending = false;
    }
    return PIC_OK;
}

int sort_all(pic_ctx* c) {
    int rm = materialize(c);  // a full sort reads the current buffer: no permutation may be pending
    if (rm) return rm;
    for (auto& s : c->sp) {
        if (s.immobile) continue;  // empty store, never pushed
        int r = c->mixed ? sort_species<float>(c, s) : sort_species<double>(c, s);
        if (r) return r;
    }
    c->since_sort = 0;
    c->vsum0 = 0.0;
    if (c->d_drift) CUDA_TRY(c, cudaMemsetAsync(c->d_drift, 0, DRIFT_ROWS * sizeof(unsigned), c->st));
    return PIC_OK;
}

// D_a = dt/d_a times the sum over the pushes since the last sort of their
// largest speed: an upper bound of any particle's displacement along a (cells)
// since it was binned.  Waits for the last push only (not for the field
// kernels queued behind it).
int drift_sum(pic_ctx* c, double D[3]) {
    D[0] = D[1] = D[2] = 0.0;
    if (!c->adaptive || c->since_sort <= 0) return PIC_OK;
    unsigned rows[DRIFT_ROWS];
    const int n = std::min(c->since_sort, DRIFT_ROWS);
    CUDA_TRY(c, cudaStreamWaitEvent(c->xst, c->ev_push, 0));
    CUDA_TRY(c, cudaMemcpyAsync(rows, c->d_drift, n * sizeof(unsigned), cudaMemcpyDeviceToHost, c->xst));
    CUDA_TRY(c, cudaStreamSynchronize(c->xst));
    double vsum = c->vsum0;
    for (int i = 0; i < n; ++i) {
        float g2;
        memcpy(&g2, &rows[i], sizeof g2);
        vsum += g2 > 1.0f ? std::sqrt(1.0 - 1.0 / (double)g2) : 0.0;
    }
    for (int a = 0; a < 3; ++a) D[a] = vsum * c->dtd[a];
    return PIC_OK;
}

// Whether the next step must be preceded by a sort.
int sort_due(pic_ctx* c, bool* due) {
    if (!c->adaptive) {
        *due = c->since_sort >= c->K;
        return PIC_OK;
    }
    constexpr double MARGIN = 1e-4;  // FP32 offsets round their positions
    const double wc = std::max(c->dtd[0], std::max(c->dtd[1], c->dtd[2]));
    *due = false;
    if (c->since_sort >= DRIFT_ROWS) {
        *due = true;
    } else if (c->since_sort > 0 && !((c->since_sort + 1) * wc < 1.0 - MARGIN)) {
        // not ruled out by the speed-of-light bound alone: read the recorded maxima
        double D[3];
        int r = drift_sum(c, D);
        if (r) return r;
        for (int a = 0; a < 3; ++a) *due = *due || !(D[a] + c->dtd[a] < 1.0 - MARGIN);
    }
    return PIC_OK;
}

template <class R>
XQueue<R>& xqueue_of(pic_ctx* c);
template <>
XQueue<double>& xqueue_of<double>(pic_ctx* c) { return c->xq64; }
template <>
XQueue<float>& xqueue_of<float>(pic_ctx* c) { return c->xq32; }

template <class R>
int alloc_xqueue(pic_ctx* c) {
    XQueue<R>& q = xqueue_of<R>(c);
    const size_t n = (size_t)c->push_grid * CHUNK;
    int r = dalloc(c, c->allocs, &q.key, n);
    for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, c->allocs, &q.a[a], n);
    for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, c->allocs, &q.d[a], n);
    if (!r) r = dalloc(c, c->allocs, &q.w, n);
    return r;
}

template <class R>
int push_species(pic_ctx* c, Species& s) {
    PushParams pp = make_params(c, s);
    const XQueue<R>& xq = xqueue_of<R>(c);
    const CUtensorMap& tm = c->mixed ? c->tm32 : c->tm64;
    cudaError_t e = cudaErrorInvalidValue;
    PStore<R>& ps = store_of<R>(s).a();
    const int S = c->g.S;
    if constexpr (sizeof(R) == 8) {
        // after a ranks-only sort: read the current buffer through the permutation, write the other
        const bool g = s.perm_pending;
        PStore<R>& out = g ? store_of<R>(s).b() : ps;
        const int* perm = g ? s.d_perm : nullptr;
        if (S == 2)
            e = push_launch<double, 2>(c->push_grid, c->st, tm, pp, out, ps, perm, xq, s.d_chunks, s.d_nchunks, c->J,
                                       s.d_ek, c->d_err);
        if (S == 4)
            e = push_launch<double, 4>(c->push_grid, c->st, tm, pp, out, ps, perm, xq, s.d_chunks, s.d_nchunks, c->J,
                                       s.d_ek, c->d_err);
        if (S == 8)
            e = push_launch<double, 8>(c->push_grid, c->st, tm, pp, out, ps, perm, xq, s.d_chunks, s.d_nchunks, c->J,
                                       s.d_ek, c->d_err);
        if (g && e == cudaSuccess) {
            store_of<R>(s).cur ^= 1;
            s.perm_pending = false;
        }
    } else {
        if (c->adaptive) pp.drift = c->d_drift + std::min(c->since_sort, DRIFT_ROWS - 1);
        const bool g = s.perm_pending;
        PStore<R>& out = g ? store_of<R>(s).b() : ps;
        const int* perm = g ? s.d_perm : nullptr;
        if (S == 4)
            e = push32_launch<4>(c->push_grid, c->st, tm, pp, out, ps, perm, xq, s.d_chunks, s.d_nchunks, c->J, s.d_ek,
                                 c->d_err);
        if (S == 8)
            e = push32_launch<8>(c->push_grid, c->st, tm, pp, out, ps, perm, xq, s.d_chunks, s.d_nchunks, c->J, s.d_ek,
                                 c->d_err);
        if (g && e == cudaSuccess) {
            store_of<R>(s).cur ^= 1;
            s.perm_pending = false;
        }
    }
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "push launch: %s", cudaGetErrorString(e));
    c->launches += 1;
    return PIC_OK;
}

// Second-order form factor: gather, push, move and Esirkepov current of one
// species (FP64 only; validated at create).
int push_species_tsc(pic_ctx* c, Species& s) {
    PushParams pp = make_params(c, s);
    cudaError_t e = tsc_launch(c->push_grid, c->st, pp, s.s64.a(), s.d_n, c->EB, c->J, s.d_ek);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "push launch: %s", cudaGetErrorString(e));
    c->launches += 1;
    return PIC_OK;
}

template <class R>
int alloc_store(pic_ctx* c, Species& s, Store<R>& st, long long cap) {
    // the FP32 particle kernel reads and writes four particles at a time with
    // 16-byte accesses: every array holds a whole number of such groups
    cap = (cap + 3) & ~3LL;
    for (int b = 0; b < 2; ++b) {
        PStore<R>& p = st.buf[b];
        int r = dalloc(c, s.allocs, &p.cell, cap);
        for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, s.allocs, &p.off[a], cap);
        for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, s.allocs, &p.u[a], cap);
        if (!r) r = dalloc(c, s.allocs, &p.w, cap);
        if (!r) r = dalloc(c, s.allocs, &p.id, cap);
        if (r) return r;
    }
    {
        int r = dalloc(c, s.allocs, &s.d_perm, cap);
        if (r) return r;
    }
    s.perm_pending = false;
    st.cur = 0;
    return PIC_OK;
}

void free_species(Species& s) {
    for (void* p : s.allocs) cudaFree(p);
    s.allocs.clear();
    // every device pointer of the species came from `allocs`: none may outlive it
    // (the staging area in particular is re-allocated on first use only when null)
    s.s64 = Store<double>{};
    s.s32 = Store<float>{};
    s.d_n = nullptr;
    s.d_bin_start = nullptr;
    s.d_chunks = nullptr;
    s.d_nchunks = nullptr;
    s.d_stage = nullptr;
    s.d_wmax = nullptr;
    s.d_perm = nullptr;
    s.perm_pending = false;
}

// Device address of a page-locked host array (cudaHostAlloc / cudaHostRegister,
// e.g. pinned torch tensors), or null for pageable memory.
const double* mapped_view(const double* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<const double*>(a.devicePointer) : nullptr;
}

// (Re)allocate the store and bin tables of species s for n particles.
int alloc_species(pic_ctx* c, Species& s, long long n) {
    cudaStreamSynchronize(c->st);
    free_species(s);
    long long cap = n > 0 ? n : 1;
    s.cap = cap;
    int r = dalloc(c, s.allocs, &s.d_n, 2);
    if (!r) r = dalloc(c, s.allocs, &s.d_bin_start, (size_t)c->g.nbins + 1);
    if (!r) r = dalloc(c, s.allocs, &s.d_chunks, (size_t)(c->g.nbins + cap / CHUNK + 1));
    if (!r) r = dalloc(c, s.allocs, &s.d_nchunks, 1);
    if (!r) r = dalloc(c, s.allocs, &s.d_wmax, 1);
    if (!r) r = c->mixed ? alloc_store(c, s, s.s32, cap) : alloc_store(c, s, s.s64, cap);
    if (r) return r;
    CUDA_TRY(c, cudaMemsetAsync(s.d_wmax, 0, sizeof(float), c->st));
    CUDA_TRY(c, cudaMemsetAsync(s.d_nchunks, 0, sizeof(int), c->st));
    // an immobile species is never sorted: its (empty) bins stay at 0
    CUDA_TRY(c, cudaMemsetAsync(s.d_bin_start, 0, ((size_t)c->g.nbins + 1) * sizeof(int), c->st));
    return PIC_OK;
}

// Largest |w| of a mixed-precision store (the fixed-point current's scale).
int refresh_wmax(pic_ctx* c, Species& s) {
    if (!c->mixed || !s.d_wmax) return PIC_OK;
    cudaError_t e = wmax_launch(c->st, c->nsm, s.s32.a().w, s.d_n, s.d_wmax);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "wmax: %s", cudaGetErrorString(e));
    return PIC_OK;
}

// (Re)load the particles of species s from FP64 arrays (host or device).
int load_particles(pic_ctx* c, Species& s, long long n, const double* const* src, bool device) {
    {
        const int rm = materialize(c);  // the other species are re-sorted below
        if (rm) return rm;
    }
    if (n < 0 || n >= (1LL << 31) - 1) return fail(c, PIC_ERR_ARG, "particle count %lld out of range", n);
    for (int k = 0; k < 7 && n > 0; ++k)
        if (!src[k]) return fail(c, PIC_ERR_ARG, "null particle array %d", k);
    if (!s.d_n || n > s.cap) {
        int r = alloc_species(c, s, n);
        if (r) return r;
    }
    int r = PIC_OK;
    // host inputs: page-locked arrays the device can address are read in place
    // by the load kernel (over the CPU-GPU link); the others are staged
    const double* dsrc[7];
    if (!device && n > 0) {
        for (int k = 0; k < 7; ++k) {
            dsrc[k] = mapped_view(src[k]);
            if (dsrc[k]) continue;
            if (!s.d_stage && (r = dalloc(c, s.allocs, &s.d_stage, (size_t)7 * s.cap))) return r;
            double* d = s.d_stage + (size_t)k * s.cap;
            CUDA_TRY(c, cudaMemcpyAsync(d, src[k], n * sizeof(double), cudaMemcpyHostToDevice, c->st));
            dsrc[k] = d;
        }
    } else {
        for (int k = 0; k < 7; ++k) dsrc[k] = src[k];
    }
    long long nn = n;
    s.nid = n;
    CUDA_TRY(c, cudaMemcpyAsync(s.d_n, &nn, sizeof(long long), cudaMemcpyHostToDevice, c->st));
    cudaError_t e = c->mixed ? load_launch<float>(c->st, n, dsrc, s.s32.a(), c->g)
                             : load_launch<double>(c->st, n, dsrc, s.s64.a(), c->g);
    c->launches += n > 0 ? 1 : 0;
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "load: %s", cudaGetErrorString(e));
    // bin the new particles; the other species are re-sorted too, so that every
    // species starts the next sort interval together.  On the cloud-in-cell paths
    // ranks only: the next particle step moves the records (every other reader
    // of the store applies the permutation first, see materialize)
    r = refresh_wmax(c, s);
    if (!r) r = c->desc.form_factor != 2 ? sort_all_ranks(c) : sort_all(c);
    c->energy_fresh = false;
    return r;
}

// The kinetic-energy partials of all species, contiguous (push_grid slots
// per species), zeroed.
int rebuild_ek(pic_ctx* c) {
    if (c->d_ekall) {
        cudaStreamSynchronize(c->st);
        cudaFree(c->d_ekall);
        for (auto& p : c->allocs)
            if (p == c->d_ekall) p = nullptr;
        c->d_ekall = nullptr;
    }
    if (c->sp.empty()) return PIC_OK;
    int r = dalloc(c, c->allocs, &c->d_ekall, (size_t)c->push_grid * c->sp.size());
    if (r) return r;
    CUDA_TRY(c, cudaMemsetAsync(c->d_ekall, 0, sizeof(double) * c->push_grid * c->sp.size(), c->st));
    for (size_t i = 0; i < c->sp.size(); ++i) c->sp[i].d_ek = c->d_ekall + i * c->push_grid;
    return PIC_OK;
}

int add_species_impl(pic_ctx* c, const pic_species_desc* d, int64_t n, const double* const* src, bool device,
                     int* id) {
    if (!c) return PIC_ERR_ARG;
    if (!d || !id) return fail(c, PIC_ERR_ARG, "null argument");
    if (!(d->m > 0) || !std::isfinite(d->q)) return fail(c, PIC_ERR_ARG, "species mass must be > 0");
    if ((int)c->sp.size() >= MAX_SPECIES) return fail(c, PIC_ERR_ARG, "too many species");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    c->sp.emplace_back();
    Species& s = c->sp.back();
    s.q = d->q;
    s.m = d->m;
    s.immobile = d->immobile != 0;
    if (n < 0) {
        c->sp.pop_back();
        return fail(c, PIC_ERR_ARG, "particle count %lld out of range", (long long)n);
    }
    // an immobile background keeps an empty store
    int r = load_particles(c, s, s.immobile ? 0 : n, src, device);
    if (r) {
        free_species(s);
        c->sp.pop_back();
        return r;
    }
    if ((r = rebuild_ek(c))) return r;
    *id = (int)c->sp.size() - 1;
    if (!device) CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return PIC_OK;
}

// 3-D copies between the unpadded ABI layout and a padded component.
cudaMemcpy3DParms copy_params(const GridDev& g, void* padded, void* flat, bool to_padded) {
    cudaMemcpy3DParms p;
    memset(&p, 0, sizeof p);
    cudaPitchedPtr pp = make_cudaPitchedPtr(padded, g.np[0] * sizeof(double), g.np[0], g.np[1]);
    cudaPitchedPtr fp = make_cudaPitchedPtr(flat, g.n[0] * sizeof(double), g.n[0], g.n[1]);
    if (to_padded) {
        p.srcPtr = fp;
        p.dstPtr = pp;
        p.dstPos = make_cudaPos(PAD * sizeof(double), PAD, PAD);
    } else {
        p.srcPtr = pp;
        p.srcPos = make_cudaPos(PAD * sizeof(double), PAD, PAD);
        p.dstPtr = fp;
    }
    p.extent = make_cudaExtent(g.n[0] * sizeof(double), g.n[1], g.n[2]);
    p.kind = cudaMemcpyDefault;
    return p;
}

int set_fields_impl(pic_ctx* c, const double* const E[3], const double* const B[3], bool device) {
    if (!c) return PIC_ERR_ARG;
    if (!E || !B) return fail(c, PIC_ERR_ARG, "null field array");
    for (int k = 0; k < 3; ++k)
        if (!E[k] || !B[k]) return fail(c, PIC_ERR_ARG, "null field component");
    for (int k = 0; k < 6; ++k) {
        const double* src = k < 3 ? E[k] : B[k - 3];
        cudaMemcpy3DParms p = copy_params(c->g, c->EB + k * c->g.P, const_cast<double*>(src), true);
        CUDA_TRY(c, cudaMemcpy3DAsync(&p, c->st));
    }
    CUDA_TRY(c, refresh_launch(c->st, c->EB, c->g, c->EB32));
    c->launches += 1;
    c->energy_fresh = false;
    if (!device) CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int get_fields_impl(pic_ctx* c, double* const E[3], double* const B[3], bool device) {
    if (!c) return PIC_ERR_ARG;
    if (!E || !B) return fail(c, PIC_ERR_ARG, "null field array");
    for (int k = 0; k < 6; ++k) {
        double* dst = k < 3 ? E[k] : B[k - 3];
        if (!dst) return fail(c, PIC_ERR_ARG, "null field component");
        cudaMemcpy3DParms p = copy_params(c->g, c->EB + k * c->g.P, dst, false);
        CUDA_TRY(c, cudaMemcpy3DAsync(&p, c->st));
    }
    if (!device) CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int get_current_impl(pic_ctx* c, double* const J[3], bool device) {
    if (!c) return PIC_ERR_ARG;
    if (!J) return fail(c, PIC_ERR_ARG, "null current array");
    const long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
    for (int k = 0; k < 3; ++k) {
        if (!J[k]) return fail(c, PIC_ERR_ARG, "null current component");
        CUDA_TRY(c, cudaMemcpyAsync(J[k], c->Jlast + k * ncell, ncell * sizeof(double), cudaMemcpyDefault, c->st));
    }
    if (!device) CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int device_status(pic_ctx* c) {
    int flags = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&flags, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
#if PICGB_DEBUG
    // the index flags of the checking units, kept sticky in this context's flag word
    const int idx = push_index_flags() | push32_index_flags() | tsc_index_flags() | tape_index_flags() |
                    sort_index_flags();
    if (idx && !(flags & ERRBIT_INDEX)) {
        flags |= ERRBIT_INDEX;
        CUDA_TRY(c, cudaMemcpyAsync(c->d_err, &flags, sizeof(int), cudaMemcpyHostToDevice, c->st));
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
#endif
    if (flags & ERRBIT_INDEX)
        return fail(c, PIC_ERR_INDEX, "a kernel index fell outside its array (debug build check; the access was skipped)");
    if (flags & ERRBIT_TIMEOUT) return fail(c, PIC_ERR_TIMEOUT, "a bounded TMA/mbarrier wait expired in a kernel");
    if (flags & ERRBIT_DRIFT)
        return fail(c, PIC_ERR_BIN_OVERFLOW, "a particle left its supercell slack between sorts");
    if (flags & ERRBIT_NAN) return fail(c, PIC_ERR_NAN, "non-finite value");
    return PIC_OK;
}

template <class R>
int get_particles_impl(pic_ctx* c, int species, int64_t cap, int64_t* n, int64_t* id, double* const* dst,
                       bool device) {
    {
        const int rm = materialize(c);
        if (rm) return rm;
    }
    Species& s = c->sp[species];
    PStore<R>& ps = store_of<R>(s).a();
    CUDA_TRY(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->st));
    long long* did = reinterpret_cast<long long*>(id);
    double* ddst[7];
    std::vector<void*> tmp;
    if (!device) {
        // stage on the device, then copy back
        long long m = cap > 0 ? cap : 1;
        void* q = nullptr;
        if (cudaMalloc(&q, m * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PIC_ERR_OOM, "staging");
        }
        tmp.push_back(q);
        did = (long long*)q;
        for (int k = 0; k < 7; ++k) {
            if (cudaMalloc(&q, m * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                for (void* t : tmp) cudaFree(t);
                return fail(c, PIC_ERR_OOM, "staging");
            }
            tmp.push_back(q);
            ddst[k] = (double*)q;
        }
    } else {
        for (int k = 0; k < 7; ++k) ddst[k] = dst[k];
    }
    cudaError_t e = unload_launch<R>(c->st, c->nsm, ps, s.d_n, c->g, c->d_counter, cap, did, ddst);
    c->launches += 1;
    int cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, c->d_counter, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess && !device && cnt > 0) {
        long long m = cnt < cap ? cnt : cap;
        cudaMemcpyAsync(id, did, m * sizeof(long long), cudaMemcpyDeviceToHost, c->st);
        for (int k = 0; k < 7; ++k)
            cudaMemcpyAsync(dst[k], ddst[k], m * sizeof(double), cudaMemcpyDeviceToHost, c->st);
        e = cudaStreamSynchronize(c->st);
    }
    for (void* t : tmp) cudaFree(t);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "get_particles: %s", cudaGetErrorString(e));
    *n = cnt;
    if (cnt > cap) return fail(c, PIC_ERR_ARG, "cap %lld < %d active particles", (long long)cap, cnt);
    return PIC_OK;
}

int finalize_energy(pic_ctx* c, int nwf) {
    const int nek = c->push_grid * (int)c->sp.size();
    cudaError_t e = energy_finalize_launch(c->st, c->d_wf, nwf, c->d_ekall, nek,
                                           0.5 * c->g.d[0] * c->g.d[1] * c->g.d[2], c->d_energy);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "energy finalize: %s", cudaGetErrorString(e));
    return PIC_OK;
}


// ---------------------------------------------------------------- differentiable runs
StepParams step_params(const pic_ctx* c, const Species& s) {
    StepParams sp;
    sp.g = c->g;
    sp.qdt2m = 0.5 * s.q * c->g.dt / s.m;
    for (int a = 0; a < 3; ++a) {
        sp.dtd[a] = c->g.dt / c->g.d[a];
        sp.cq[a] = s.q / (c->g.dt * c->g.d[(a + 1) % 3] * c->g.d[(a + 2) % 3]);
    }
    sp.mass = s.m;
    return sp;
}

int alloc_tape_dev(pic_ctx* c, Tape& t, TapeDev& d, long long n, const double* w) {
    int r = PIC_OK;
    for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, t.allocs, &d.xi[a], (size_t)n);
    for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, t.allocs, &d.u[a], (size_t)n);
    if (!r) r = dalloc(c, t.allocs, &d.act, (size_t)n);
    d.w = w;
    return r;
}

int alloc_tape_u(pic_ctx* c, Tape& t, TapeDev& d, long long n) {
    int r = PIC_OK;
    for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, t.allocs, &d.u[a], (size_t)n);
    return r;
}

int alloc_tape_x(pic_ctx* c, Tape& t, TapeDev& d, long long n, const double* w) {
    int r = PIC_OK;
    for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, t.allocs, &d.xi[a], (size_t)n);
    if (!r) r = dalloc(c, t.allocs, &d.act, (size_t)n);
    d.w = w;
    return r;
}

int copy_tape_u(pic_ctx* c, const TapeDev& dst, const TapeDev& src, long long n) {
    if (n <= 0) return PIC_OK;
    for (int a = 0; a < 3; ++a)
        CUDA_TRY(c, cudaMemcpyAsync(dst.u[a], src.u[a], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return PIC_OK;
}

int copy_tape_x(pic_ctx* c, const TapeDev& dst, const TapeDev& src, long long n) {
    if (n <= 0) return PIC_OK;
    for (int a = 0; a < 3; ++a)
        CUDA_TRY(c, cudaMemcpyAsync(dst.xi[a], src.xi[a], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    CUDA_TRY(c, cudaMemcpyAsync(dst.act, src.act, n * sizeof(int), cudaMemcpyDeviceToDevice, c->st));
    return PIC_OK;
}

int copy_tape_dev(pic_ctx* c, const TapeDev& dst, const TapeDev& src, long long n) {
    if (n <= 0) return PIC_OK;
    for (int a = 0; a < 3; ++a) {
        CUDA_TRY(c, cudaMemcpyAsync(dst.xi[a], src.xi[a], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CUDA_TRY(c, cudaMemcpyAsync(dst.u[a], src.u[a], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    }
    CUDA_TRY(c, cudaMemcpyAsync(dst.act, src.act, n * sizeof(int), cudaMemcpyDeviceToDevice, c->st));
    return PIC_OK;
}

int copy_EB(pic_ctx* c, double* dst, const double* src) {
    CUDA_TRY(c, cudaMemcpyAsync(dst, src, 6 * c->g.P * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return PIC_OK;
}

// One whole step of the differentiable path on the context's fields.
int tape_step(pic_ctx* c) {
    Tape& t = c->tape;
    for (size_t i = 0; i < c->sp.size(); ++i) {
        const StepParams sp = step_params(c, c->sp[i]);
        CUDA_TRY(c, tape_step_launch(c->st, t.sp[i].cur, t.sp[i].n, sp, c->EB, c->J));
        c->launches += t.sp[i].n > 0 ? 1 : 0;
    }
    const double h = 0.5 * c->g.dt;
    CUDA_TRY(c, fdtd_b_launch(c->st, c->EB, c->g, h, 0, nullptr, nullptr));
    CUDA_TRY(c, fdtd_e_launch(c->st, c->EB, c->J, c->Jlast, c->g));
    CUDA_TRY(c, fdtd_b_launch(c->st, c->EB, c->g, h, 1, c->EB32, c->d_wf));
    c->launches += 3;
    return PIC_OK;
}

// Records step m of the segment from the current state: its momentum, its
// positions and flags when m is a multiple of B, and its fields.
int tape_record(pic_ctx* c, int m) {
    Tape& t = c->tape;
    int r;
    for (auto& ts : t.sp) {
        ts.blk = -1;
        if ((r = copy_tape_u(c, ts.us[m], ts.cur, ts.n))) return r;
        if (m % t.B == 0 && (r = copy_tape_x(c, ts.xs[m / t.B], ts.cur, ts.n))) return r;
    }
    return copy_EB(c, t.snapEB[m], c->EB);
}

// The recorded state (x^m, u^{m-1/2}, flags) of step m of a segment of `len`
// steps for species i.  Positions of a multiple m0 of B are read where they
// were recorded; on entering the block m0 .. m0 + B - 1 (the reverse sweep
// meets its last step first) the positions of its other steps are rebuilt
// into xw by moving with the recorded momenta, x^{j+1} from x^j and u^{j+1/2}.
int tape_state_at(pic_ctx* c, size_t i, int m, int len, TapeDev& T) {
    Tape& t = c->tape;
    TapeSpecies& ts = t.sp[i];
    const int b = m / t.B, m0 = b * t.B, j = m - m0;
    if (j > 0 && ts.blk != m0) {
        const StepParams sp = step_params(c, c->sp[i]);
        const int last = std::min(t.B - 1, len - 1 - m0);
        for (int k = 1; k <= last; ++k) {
            TapeDev src = k == 1 ? ts.xs[b] : ts.xw[k - 1];
            for (int a = 0; a < 3; ++a) src.u[a] = ts.us[m0 + k].u[a];
            CUDA_TRY(c, tape_move_launch(c->st, src, ts.xw[k], ts.n, sp));
            c->launches += ts.n > 0 ? 1 : 0;
        }
        ts.blk = m0;
    }
    T = j == 0 ? ts.xs[b] : ts.xw[j];
    for (int a = 0; a < 3; ++a) T.u[a] = ts.us[m].u[a];
    T.w = ts.w;
    return PIC_OK;
}

int tape_forward_impl(pic_ctx* c, int nsteps, int K, double* wk) {
    if (nsteps < 1 || K < 1) return fail(c, PIC_ERR_ARG, "nsteps and ckpt_every must be >= 1");
    if (c->desc.form_factor == 2)
        return fail(c, PIC_ERR_STATE, "the differentiable path implements the cloud-in-cell form factor only");
    {
        const int rm = materialize(c);  // the tape starts from the store in sorted order
        if (rm) return rm;
    }
    Tape& t = c->tape;
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    t.release();
    t.nsteps = nsteps;
    t.K = K;
    const int nck = (nsteps + K - 1) / K;
    const int nsnap = K < nsteps ? K : nsteps;
    int B = 1;
    while (B * B < nsnap) ++B;
    t.B = B;
    const int nxs = (nsnap + B - 1) / B;
    const long long P6 = 6 * c->g.P;
    int r = PIC_OK;
    long long nmax = 1;
    t.sp.resize(c->sp.size());
    for (size_t i = 0; i < c->sp.size() && !r; ++i) {
        TapeSpecies& ts = t.sp[i];
        Species& s = c->sp[i];
        ts.n = s.nid;
        nmax = ts.n > nmax ? ts.n : nmax;
        r = dalloc(c, t.allocs, &ts.w, (size_t)(ts.n > 0 ? ts.n : 1));
        if (!r) r = alloc_tape_dev(c, t, ts.cur, ts.n, ts.w);
        for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, t.allocs, &ts.lam.xi[a], (size_t)ts.n);
        for (int a = 0; a < 3 && !r; ++a) r = dalloc(c, t.allocs, &ts.lam.u[a], (size_t)ts.n);
        // a one-segment tape never replays, so it keeps no checkpoint (its records start
        // with the whole initial state); with several, the last one serves a second backward
        ts.ck.resize(nck > 1 ? nck : 0);
        ts.us.resize(nsnap);
        ts.xs.resize(nxs);
        ts.xw.resize(B);
        for (size_t k = 0; k < ts.ck.size() && !r; ++k) r = alloc_tape_dev(c, t, ts.ck[k], ts.n, ts.w);
        for (int k = 0; k < nsnap && !r; ++k) r = alloc_tape_u(c, t, ts.us[k], ts.n);
        for (int k = 0; k < nxs && !r; ++k) r = alloc_tape_x(c, t, ts.xs[k], ts.n, ts.w);
        for (int k = 1; k < B && !r; ++k) r = alloc_tape_x(c, t, ts.xw[k], ts.n, ts.w);
        if (r) break;
        // the current (binned) store -> id order
        if (ts.n > 0) {
            CUDA_TRY(c, cudaMemsetAsync(ts.cur.act, 0, ts.n * sizeof(int), c->st));
            CUDA_TRY(c, cudaMemsetAsync(ts.w, 0, ts.n * sizeof(double), c->st));
            for (int a = 0; a < 3; ++a) {
                CUDA_TRY(c, cudaMemsetAsync(ts.cur.xi[a], 0, ts.n * sizeof(double), c->st));
                CUDA_TRY(c, cudaMemsetAsync(ts.cur.u[a], 0, ts.n * sizeof(double), c->st));
            }
            cudaError_t e = c->mixed ? tape_from_store_launch<float>(c->st, c->nsm, s.s32.a(), s.d_n, ts.cur, ts.w, ts.n)
                                     : tape_from_store_launch<double>(c->st, c->nsm, s.s64.a(), s.d_n, ts.cur, ts.w,
                                                                      ts.n);
            c->launches += 1;
            if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "tape load: %s", cudaGetErrorString(e));
        }
    }
    t.ckEB.resize(nck > 1 ? nck : 0);
    t.snapEB.resize(nsnap);
    for (size_t k = 0; k < t.ckEB.size() && !r; ++k) r = dalloc(c, t.allocs, &t.ckEB[k], (size_t)P6);
    for (int k = 0; k < nsnap && !r; ++k) r = dalloc(c, t.allocs, &t.snapEB[k], (size_t)P6);
    if (!r) r = dalloc(c, t.allocs, &t.finalEB, (size_t)P6);
    if (!r) r = dalloc(c, t.allocs, &t.L, (size_t)P6);
    if (!r) r = dalloc(c, t.allocs, &t.LJ, (size_t)(3 * c->g.P));
    if (!r) r = dalloc(c, t.allocs, &t.scat, (size_t)P6);
    if (r) {
        t.release();
        return r;
    }
    // staging for the re-load of the store after the last step, taken before the first
    // step (so that the tape fails before it starts) and freed on return: the backward
    // does not hold it
    double* stage = nullptr;
    {
        const cudaError_t e = cudaMalloc(&stage, (size_t)7 * nmax * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            t.release();
            return fail(c, PIC_ERR_OOM, "tape re-load staging of %lld particles", nmax);
        }
    }
    struct StageFree {
        double* p;
        ~StageFree() { cudaFree(p); }  // cudaFree waits for the device work that reads it
    } stage_free{stage};
    for (int n = 0; n < nsteps; ++n) {
        if (n % K == 0 && nck > 1) {
            const int k = n / K;
            for (auto& ts : t.sp)
                if ((r = copy_tape_dev(c, ts.ck[k], ts.cur, ts.n))) return r;
            if ((r = copy_EB(c, t.ckEB[k], c->EB))) return r;
        }
        // the last segment's steps are recorded: the backward starts there without a replay
        if (n / K == nck - 1 && (r = tape_record(c, n - (nck - 1) * K))) return r;
        if ((r = tape_step(c))) return r;
    }
    t.snap_seg = nck - 1;
    if ((r = copy_EB(c, t.finalEB, c->EB))) return r;
    // final kinetic energy (and field energy, from the last B half step)
    for (size_t i = 0; i < c->sp.size(); ++i)
        CUDA_TRY(c, tape_kinetic_launch(c->st, c->push_grid, t.sp[i].cur, t.sp[i].n, c->sp[i].m, c->sp[i].d_ek));
    c->launches += c->sp.size();
    if ((r = finalize_energy(c, fdtd_blocks(c->g)))) return r;
    double out[2];
    CUDA_TRY(c, cudaMemcpyAsync(out, c->d_energy, sizeof out, cudaMemcpyDeviceToHost, c->st));
    // the context continues from the final state: re-load the binned store
    for (size_t i = 0; i < c->sp.size(); ++i) {
        TapeSpecies& ts = t.sp[i];
        if (ts.n == 0) continue;
        double* dst[7];
        for (int k = 0; k < 7; ++k) dst[k] = stage + (size_t)k * ts.n;
        double** ddst = nullptr;
        CUDA_TRY(c, cudaMalloc(&ddst, sizeof dst));
        cudaError_t e = cudaMemcpyAsync(ddst, dst, sizeof dst, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = tape_to_phys_launch(c->st, ts.cur, ts.n, c->g, ddst);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        cudaFree(ddst);
        if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "tape write-back: %s", cudaGetErrorString(e));
        c->launches += 1;
        const double* src[7] = {dst[0], dst[1], dst[2], dst[3], dst[4], dst[5], dst[6]};
        if ((r = load_particles(c, c->sp[i], ts.n, src, true))) return r;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    c->energy_fresh = false;
    c->since_sort = 0;
    c->steps += nsteps;
    t.ready = true;
    if (wk) *wk = out[1];
    return device_status(c);
}

int tape_backward_impl(pic_ctx* c, double wk_weight, const double* const gE[3], const double* const gB[3],
                       double* const dE0[3], double* const dB0[3]) {
    Tape& t = c->tape;
    if (!t.ready) return fail(c, PIC_ERR_STATE, "no tape recorded (call pic_tape_forward first)");
    const long long P6 = 6 * c->g.P;
    CUDA_TRY(c, cudaMemsetAsync(t.L, 0, P6 * sizeof(double), c->st));
    CUDA_TRY(c, cudaMemsetAsync(t.LJ, 0, 3 * c->g.P * sizeof(double), c->st));
    CUDA_TRY(c, cudaMemsetAsync(t.scat, 0, P6 * sizeof(double), c->st));
    for (int k = 0; k < 6; ++k) {
        const double* src = k < 3 ? (gE ? gE[k] : nullptr) : (gB ? gB[k - 3] : nullptr);
        if (!src) continue;
        cudaMemcpy3DParms p = copy_params(c->g, t.L + k * c->g.P, const_cast<double*>(src), true);
        CUDA_TRY(c, cudaMemcpy3DAsync(&p, c->st));
    }
    const int nck = (t.nsteps + t.K - 1) / t.K;
    int r;
    if (t.snap_seg != nck - 1) {
        // an earlier backward replayed the first segments over the final state: replay the
        // last segment from its checkpoint, recording its steps, to bring that state back
        const int n0 = (nck - 1) * t.K, len = t.nsteps - n0;
        for (auto& ts : t.sp)
            if ((r = copy_tape_dev(c, ts.cur, ts.ck[nck - 1], ts.n))) return r;
        if ((r = copy_EB(c, c->EB, t.ckEB[nck - 1]))) return r;
        for (int m = 0; m < len; ++m) {
            if ((r = tape_record(c, m))) return r;
            if ((r = tape_step(c))) return r;
        }
        t.snap_seg = nck - 1;
    }
    // seed: cotangent of the final kinetic energy
    for (size_t i = 0; i < c->sp.size(); ++i) {
        CUDA_TRY(c, tape_seed_launch(c->st, t.sp[i].cur, t.sp[i].lam, t.sp[i].n, c->sp[i].m, wk_weight));
        c->launches += 1;
    }
    for (int k = nck - 1; k >= 0; --k) {
        const int n0 = k * t.K, n1 = n0 + t.K < t.nsteps ? n0 + t.K : t.nsteps;
        if (t.snap_seg != k) {
            // restore the checkpoint and replay the segment, recording each step
            for (auto& ts : t.sp)
                if ((r = copy_tape_dev(c, ts.cur, ts.ck[k], ts.n))) return r;
            if ((r = copy_EB(c, c->EB, t.ckEB[k]))) return r;
            for (int m = 0; m < n1 - n0; ++m) {
                if ((r = tape_record(c, m))) return r;
                if (m + 1 < n1 - n0 && (r = tape_step(c))) return r;
            }
            t.snap_seg = k;
        }
        // adjoint steps, last to first
        for (int m = n1 - n0 - 1; m >= 0; --m) {
            CUDA_TRY(c, adj_fields_launch(c->st, t.L, t.LJ, c->g));
            c->launches += 6;
            for (size_t i = 0; i < c->sp.size(); ++i) {
                const StepParams sp = step_params(c, c->sp[i]);
                TapeDev T;
                if ((r = tape_state_at(c, i, m, n1 - n0, T))) return r;
                CUDA_TRY(c, tape_adjoint_launch(c->st, T, t.sp[i].lam, t.sp[i].n, sp, t.snapEB[m], t.LJ, t.scat));
                c->launches += 1;
            }
            CUDA_TRY(c, adj_fold_add_launch(c->st, t.L, t.scat, c->g));
            c->launches += 1;
        }
    }
    for (int k = 0; k < 6; ++k) {
        double* dst = k < 3 ? (dE0 ? dE0[k] : nullptr) : (dB0 ? dB0[k - 3] : nullptr);
        if (!dst) continue;
        cudaMemcpy3DParms p = copy_params(c->g, t.L + k * c->g.P, dst, false);
        CUDA_TRY(c, cudaMemcpy3DAsync(&p, c->st));
    }
    // the context's fields return to the end of the tape
    if ((r = copy_EB(c, c->EB, t.finalEB))) return r;
    CUDA_TRY(c, refresh_launch(c->st, c->EB, c->g, c->EB32));
    c->launches += 1;
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return device_status(c);
}

}  // namespace

// ====================================================================== ABI
// ---------------------------------------------------------------- state blob
namespace {

const char STATE_MAGIC[8] = {'P', 'I', 'C', 'G', 'B', 'S', 'T', '3'};

// chunk: the build's CHUNK (most particles of one chunk), which bounds every
// chunk of the blob's table and the particle kernel's per-CTA queue slots.
struct StateHeader {
    char magic[8];
    int32_t precision, supercell, sort_interval, absorb_cells;
    int32_t n[3], bc[3];
    int32_t nspecies, form_factor;
    int32_t chunk, reserved;
    double d[3], dt, absorb_sigma;
    double drift[3];  // displacement bound since the last sort (displacement-bounded schedule; else 0)
    int64_t steps, since_sort;
};

struct SpeciesHeader {
    double q, m;
    int64_t n, nid;
    int32_t immobile, nchunks;
};

size_t pad8(size_t x) { return (x + 7) & ~size_t(7); }

// Store and bin-table bytes of one species with n particles and nch chunks.
size_t species_payload(const pic_ctx* c, long long n, int nch) {
    const size_t rs = c->mixed ? sizeof(float) : sizeof(double);
    return pad8(n * sizeof(int)) * 2 + 7 * pad8(n * rs) + pad8(((size_t)c->g.nbins + 1) * sizeof(int)) +
           pad8((size_t)nch * sizeof(Chunk));
}

size_t grid_payload(const pic_ctx* c) {
    const long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
    return (size_t)(9 * c->g.P + 3 * ncell) * sizeof(double);
}

// Host-side cursor over the blob; every access is bounds-checked.
struct Cursor {
    unsigned char* p;
    size_t left;
    bool take(size_t n, unsigned char** at) {
        if (n > left) return false;
        *at = p;
        p += pad8(n) <= left ? pad8(n) : n;
        left -= pad8(n) <= left ? pad8(n) : left;
        return true;
    }
};

// Every index the kernels take from a blob is checked before use: active
// particles' cells inside the grid; bin starts non-decreasing from 0 to n;
// every chunk inside its own bin's range and at most CHUNK particles long
// (the particle kernel gives each particle of a chunk one of CHUNK per-CTA
// queue slots).  A cell far from its chunk's supercell is legal here: the
// particle kernel flags it as outside the supercell slack and skips it.
bool species_payload_valid(const pic_ctx* c, const unsigned char* p, long long n, int nch) {
    const size_t rs = c->mixed ? sizeof(float) : sizeof(double);
    const int* cell = reinterpret_cast<const int*>(p);
    for (long long i = 0; i < n; ++i) {
        const int cp = cell[i];
        if (cp >= 0 && (cell_x(cp) >= c->g.n[0] || cell_y(cp) >= c->g.n[1] || cell_z(cp) >= c->g.n[2])) return false;
    }
    const size_t bin_off = pad8(n * sizeof(int)) * 2 + 7 * pad8(n * rs);
    const int* bs = reinterpret_cast<const int*>(p + bin_off);
    const int nb = c->g.nbins;
    for (int b = 0; b <= nb; ++b) {
        int v, prev = 0;
        memcpy(&v, bs + b, sizeof v);
        if (b > 0) memcpy(&prev, bs + b - 1, sizeof prev);
        if (v < prev || v > n || (b == 0 && v != 0) || (b == nb && v != n)) return false;
    }
    const size_t chunk_off = bin_off + pad8(((size_t)nb + 1) * sizeof(int));
    const Chunk* ch = reinterpret_cast<const Chunk*>(p + chunk_off);
    for (int k = 0; k < nch; ++k) {
        Chunk e;
        memcpy(&e, ch + k, sizeof e);
        if (e.sc < 0 || e.sc >= nb || e.start < 0 || e.count < 0 || e.count > CHUNK ||
            (long long)e.start + e.count > n)
            return false;
        int b0, b1;
        memcpy(&b0, bs + e.sc, sizeof b0);
        memcpy(&b1, bs + e.sc + 1, sizeof b1);
        if (e.start < b0 || e.start + e.count > b1) return false;
    }
    return true;
}

bool same_desc(const StateHeader& h, const pic_grid_desc& d) {
    bool ok = h.chunk == CHUNK && h.precision == d.precision && h.supercell == d.supercell && h.sort_interval == d.sort_interval &&
              (h.form_factor == 2) == (d.form_factor == 2) &&
              h.absorb_cells == d.absorb_cells && h.dt == d.dt && h.absorb_sigma == d.absorb_sigma;
    for (int a = 0; a < 3; ++a) ok = ok && h.n[a] == d.n[a] && h.bc[a] == d.bc[a] && h.d[a] == d.d[a];
    return ok;
}

template <class R>
int copy_store(pic_ctx* c, Species& s, long long n, Cursor& cur, bool to_blob) {
    PStore<R>& ps = store_of<R>(s).a();
    void* dev[9] = {ps.cell, ps.off[0], ps.off[1], ps.off[2], ps.u[0], ps.u[1], ps.u[2], ps.w, ps.id};
    const size_t es[9] = {sizeof(int), sizeof(R), sizeof(R), sizeof(R), sizeof(R), sizeof(R), sizeof(R), sizeof(R),
                          sizeof(int)};
    for (int k = 0; k < 9; ++k) {
        unsigned char* at;
        if (!cur.take(n * es[k], &at)) return fail(c, PIC_ERR_ARG, "state blob too small");
        if (n > 0)
            CUDA_TRY(c, to_blob ? cudaMemcpyAsync(at, dev[k], n * es[k], cudaMemcpyDeviceToHost, c->st)
                                : cudaMemcpyAsync(dev[k], at, n * es[k], cudaMemcpyHostToDevice, c->st));
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_create(const pic_grid_desc* gd, pic_ctx** out) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    pic_ctx tmp;
    int r = validate(gd, &tmp);
    if (r) {
        fprintf(stderr, "pic_create: %s\n", tmp.err.c_str());
        return r;
    }
    pic_ctx* c = new pic_ctx();
    c->desc = *gd;
    c->dev = gd->device;
    c->st = reinterpret_cast<cudaStream_t>(gd->stream);
    c->mixed = gd->precision == PIC_MIXED;
    GridDev& g = c->g;
    double dmax = 0;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = gd->n[a];
        g.np[a] = gd->n[a] + 2 * PAD;
        g.d[a] = gd->d[a];
        g.rd[a] = 1.0 / gd->d[a];
        g.bc[a] = gd->bc[a];
        g.nsc[a] = gd->n[a] / gd->supercell;
        dmax = std::fmax(dmax, gd->dt / gd->d[a]);
    }
    g.P = (long long)g.np[0] * g.np[1] * g.np[2];
    g.dt = gd->dt;
    g.S = gd->supercell;
    g.Sshift = g.S == 2 ? 1 : (g.S == 4 ? 2 : 3);
    g.nbins = g.nsc[0] * g.nsc[1] * g.nsc[2];
    g.absorb_cells = gd->absorb_cells;
    g.absorb_sigma = gd->absorb_sigma;
    g.absorb_rL = gd->absorb_cells > 0 ? 1.0 / gd->absorb_cells : 0.0;
    g.damp = nullptr;
    g.damp_off[0] = 0;
    g.damp_off[1] = 2 * g.n[0];
    g.damp_off[2] = 2 * (g.n[0] + g.n[1]);
    // the default interval (sort_interval 0), measured on the 64^3 x 50 FP64, 128^3 x 32 mixed and
    // laser-ramp workloads: the FP64 cloud-in-cell kernel runs 13% faster on particles sorted
    // every step, which outweighs the sorts; the second-order kernel (one thread per particle,
    // no tile) gains nothing from fresher order and takes the largest fixed interval; the mixed
    // kernel takes the displacement-bounded schedule
    const int kmax = (int)std::floor((1.0 - 1e-9) / dmax);
    if (gd->sort_interval > 0) c->K = gd->sort_interval;
    else c->K = (gd->precision == PIC_FP64 && gd->form_factor != 2) ? 1 : kmax;
    if (c->K < 1) c->K = 1;
    for (int a = 0; a < 3; ++a) c->dtd[a] = gd->dt / gd->d[a];
    c->adaptive = c->mixed && gd->sort_interval == 0;
    if (c->adaptive) c->K = DRIFT_ROWS;  // the longest run between sorts
    auto bail = [&](int code) {
        pic_destroy(c);
        return code;
    };
    cudaError_t e = cudaSetDevice(c->dev);
    if (e != cudaSuccess) {
        fprintf(stderr, "pic_create: cudaSetDevice(%d): %s\n", c->dev, cudaGetErrorString(e));
        delete c;
        return PIC_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev);
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    if ((r = dalloc(c, c->allocs, &c->EB, 6 * g.P))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->J, 3 * g.P))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->Jlast, 3 * ncell))) return bail(r);
    if (c->mixed && (r = dalloc(c, c->allocs, &c->EB32, 6 * g.P))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_err, 1))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_counts, ncell))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_cursor, ncell))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_tile_sum, sort_tile_scratch(ncell)))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_counter, 1))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_wf, fdtd_blocks(g)))) return bail(r);
    if ((r = dalloc(c, c->allocs, &c->d_energy, 2))) return bail(r);
    if ((g.bc[0] | g.bc[1] | g.bc[2]) != 0 && g.absorb_cells > 0) {
        double* tab = nullptr;
        if ((r = dalloc(c, c->allocs, &tab, 2 * (g.n[0] + g.n[1] + g.n[2])))) return bail(r);
        if ((e = damp_table_launch(c->st, g, tab)) != cudaSuccess) {
            fail(c, PIC_ERR_CUDA, "init: %s", cudaGetErrorString(e));
            return bail(PIC_ERR_CUDA);
        }
        g.damp = tab;  // every later copy of g (kernel arguments) reads the table
    }
    if (c->adaptive) {
        if ((r = dalloc(c, c->allocs, &c->d_drift, DRIFT_ROWS))) return bail(r);
        cudaMemsetAsync(c->d_drift, 0, DRIFT_ROWS * sizeof(unsigned), c->st);
        if ((e = cudaEventCreateWithFlags(&c->ev_push, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&c->xst, cudaStreamNonBlocking)) != cudaSuccess) {
            fail(c, PIC_ERR_CUDA, "init: %s", cudaGetErrorString(e));
            return bail(PIC_ERR_CUDA);
        }
    }
    cudaMemsetAsync(c->EB, 0, 6 * g.P * sizeof(double), c->st);
    cudaMemsetAsync(c->J, 0, 3 * g.P * sizeof(double), c->st);
    cudaMemsetAsync(c->Jlast, 0, 3 * ncell * sizeof(double), c->st);
    if (c->EB32) cudaMemsetAsync(c->EB32, 0, 6 * g.P * sizeof(float), c->st);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    cudaMemsetAsync(c->d_counts, 0, ncell * sizeof(int), c->st);
    cudaMemsetAsync(c->d_energy, 0, 2 * sizeof(double), c->st);
    if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) {
        fail(c, PIC_ERR_CUDA, "init: %s", cudaGetErrorString(e));
        return bail(PIC_ERR_CUDA);
    }
    if ((r = encode_tmap(c, &c->tm64, c->EB, false))) return bail(r);
    if (c->mixed && (r = encode_tmap(c, &c->tm32, c->EB32, true))) return bail(r);
    int bps = 0;
    if ((r = c->mixed ? push_dispatch_setup<float>(c, g.S, &bps) : push_dispatch_setup<double>(c, g.S, &bps)))
        return bail(r);
    if (bps < 1) bps = 1;
    c->push_grid = c->nsm * bps;
    if ((r = c->mixed ? alloc_xqueue<float>(c) : alloc_xqueue<double>(c))) return bail(r);
    *out = c;
    return PIC_OK;
}

int pic_destroy(pic_ctx* c) {
    if (!c) return PIC_ERR_ARG;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->st);
    if (c->cst) cudaStreamSynchronize(c->cst);
    for (auto& s : c->sp) {
        free_species(s);
        if (s.d_up) cudaFree(s.d_up);
        if (s.up_done) cudaEventDestroy(s.up_done);
        if (s.up_free) cudaEventDestroy(s.up_free);
    }
    if (c->cst) cudaStreamDestroy(c->cst);
    if (c->xst) cudaStreamDestroy(c->xst);
    if (c->ev_push) cudaEventDestroy(c->ev_push);
    c->tape.release();
    for (void* p : c->allocs)
        if (p) cudaFree(p);
    for (auto& v : c->ev)
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    delete c;
    return PIC_OK;
}

const char* pic_last_error(const pic_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pic_add_species(pic_ctx* c, const pic_species_desc* s, int64_t n, const double* x, const double* y,
                    const double* z, const double* ux, const double* uy, const double* uz, const double* w,
                    int* species_id) {
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    return add_species_impl(c, s, n, src, false, species_id);
}

int pic_add_species_dev(pic_ctx* c, const pic_species_desc* s, int64_t n, const double* x, const double* y,
                        const double* z, const double* ux, const double* uy, const double* uz, const double* w,
                        int* species_id) {
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    return add_species_impl(c, s, n, src, true, species_id);
}

static int set_particles_impl(pic_ctx* c, int species, int64_t n, const double* const* src, bool device) {
    if (!c) return PIC_ERR_ARG;
    if (species < 0 || species >= (int)c->sp.size()) return fail(c, PIC_ERR_ARG, "bad species %d", species);
    CUDA_TRY(c, cudaSetDevice(c->dev));
    Species& s = c->sp[species];
    int r = load_particles(c, s, s.immobile ? 0 : n, src, device);
    if (r) return r;
    if (!device) CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_set_particles(pic_ctx* c, int species, int64_t n, const double* x, const double* y, const double* z,
                      const double* ux, const double* uy, const double* uz, const double* w) {
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    return set_particles_impl(c, species, n, src, false);
}

int pic_set_particles_dev(pic_ctx* c, int species, int64_t n, const double* x, const double* y, const double* z,
                          const double* ux, const double* uy, const double* uz, const double* w) {
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    return set_particles_impl(c, species, n, src, true);
}

int pic_upload_particles(pic_ctx* c, int species, int64_t n, const double* x, const double* y, const double* z,
                         const double* ux, const double* uy, const double* uz, const double* w) {
    if (!c) return PIC_ERR_ARG;
    if (species < 0 || species >= (int)c->sp.size()) return fail(c, PIC_ERR_ARG, "bad species %d", species);
    Species& s = c->sp[species];
    if (s.immobile) return fail(c, PIC_ERR_ARG, "species %d is immobile (it stores no particles)", species);
    if (n < 0 || n >= (1LL << 31) - 1) return fail(c, PIC_ERR_ARG, "particle count %lld out of range", (long long)n);
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    for (int k = 0; k < 7 && n > 0; ++k)
        if (!src[k]) return fail(c, PIC_ERR_ARG, "null particle array %d", k);
    CUDA_TRY(c, cudaSetDevice(c->dev));
    if (!c->cst) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cst, cudaStreamNonBlocking));
    if (!s.up_done) CUDA_TRY(c, cudaEventCreateWithFlags(&s.up_done, cudaEventDisableTiming));
    if (!s.up_free) CUDA_TRY(c, cudaEventCreateWithFlags(&s.up_free, cudaEventDisableTiming));
    if (n > s.up_cap) {
        // grow the area once nothing reads or fills it any more
        CUDA_TRY(c, cudaStreamSynchronize(c->cst));
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
        if (s.d_up) cudaFree(s.d_up);
        s.d_up = nullptr;
        s.up_cap = 0;
        s.up_n = -1;
        void* q = nullptr;
        if (cudaMalloc(&q, (size_t)7 * n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PIC_ERR_OOM, "upload area of %lld particles", (long long)n);
        }
        s.d_up = static_cast<double*>(q);
        s.up_cap = n;
    }
    // the load that consumed the previous upload must have read the area
    CUDA_TRY(c, cudaStreamWaitEvent(c->cst, s.up_free, 0));
    for (int k = 0; k < 7 && n > 0; ++k)
        CUDA_TRY(c, cudaMemcpyAsync(s.d_up + (size_t)k * s.up_cap, src[k], (size_t)n * sizeof(double),
                                    cudaMemcpyDefault, c->cst));
    CUDA_TRY(c, cudaEventRecord(s.up_done, c->cst));
    s.up_n = n;
    return PIC_OK;
}

int pic_set_particles_uploaded(pic_ctx* c, int species) {
    if (!c) return PIC_ERR_ARG;
    if (species < 0 || species >= (int)c->sp.size()) return fail(c, PIC_ERR_ARG, "bad species %d", species);
    Species& s = c->sp[species];
    if (s.up_n < 0) return fail(c, PIC_ERR_STATE, "no pending upload for species %d", species);
    CUDA_TRY(c, cudaSetDevice(c->dev));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st, s.up_done, 0));
    const double* src[7];
    for (int k = 0; k < 7; ++k) src[k] = s.d_up + (size_t)k * s.up_cap;
    const long long n = s.up_n;
    s.up_n = -1;
    const int r = load_particles(c, s, n, src, true);
    // recorded even on failure, so that the next upload never waits on a stale event
    cudaEventRecord(s.up_free, c->st);
    return r;
}

int pic_species_info(pic_ctx* c, int species, double* q, double* m, int32_t* immobile, int64_t* nid) {
    if (!c) return PIC_ERR_ARG;
    if (species < 0 || species >= (int)c->sp.size()) return fail(c, PIC_ERR_ARG, "bad species %d", species);
    const Species& s = c->sp[species];
    if (q) *q = s.q;
    if (m) *m = s.m;
    if (immobile) *immobile = s.immobile ? 1 : 0;
    if (nid) *nid = s.nid;
    return PIC_OK;
}

int pic_count_particles(pic_ctx* c, int species, int64_t* n) {
    if (!c) return PIC_ERR_ARG;
    if (!n || species < 0 || species >= (int)c->sp.size()) return fail(c, PIC_ERR_ARG, "bad species or null n");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    {
        const int rm = materialize(c);
        if (rm) return rm;
    }
    CUDA_TRY(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->st));
    Species& s = c->sp[species];
    cudaError_t e = c->mixed ? count_launch<float>(c->st, c->nsm, s.s32.a(), s.d_n, c->d_counter)
                             : count_launch<double>(c->st, c->nsm, s.s64.a(), s.d_n, c->d_counter);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "count: %s", cudaGetErrorString(e));
    int cnt = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&cnt, c->d_counter, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    *n = cnt;
    return PIC_OK;
}

static int get_particles_any(pic_ctx* c, int species, int64_t cap, int64_t* n, int64_t* id, double* x, double* y,
                             double* z, double* ux, double* uy, double* uz, double* w, bool device) {
    if (!c) return PIC_ERR_ARG;
    if (!n || !id || !x || !y || !z || !ux || !uy || !uz || !w) return fail(c, PIC_ERR_ARG, "null output array");
    if (species < 0 || species >= (int)c->sp.size()) return fail(c, PIC_ERR_ARG, "bad species %d", species);
    CUDA_TRY(c, cudaSetDevice(c->dev));
    double* dst[7] = {x, y, z, ux, uy, uz, w};
    return c->mixed ? get_particles_impl<float>(c, species, cap, n, id, dst, device)
                    : get_particles_impl<double>(c, species, cap, n, id, dst, device);
}

int pic_get_particles(pic_ctx* c, int species, int64_t cap, int64_t* n, int64_t* id, double* x, double* y,
                      double* z, double* ux, double* uy, double* uz, double* w) {
    return get_particles_any(c, species, cap, n, id, x, y, z, ux, uy, uz, w, false);
}

int pic_get_particles_dev(pic_ctx* c, int species, int64_t cap, int64_t* n, int64_t* id, double* x, double* y,
                          double* z, double* ux, double* uy, double* uz, double* w) {
    return get_particles_any(c, species, cap, n, id, x, y, z, ux, uy, uz, w, true);
}

int pic_set_fields(pic_ctx* c, const double* const E[3], const double* const B[3]) {
    return set_fields_impl(c, E, B, false);
}
int pic_set_fields_dev(pic_ctx* c, const double* const E[3], const double* const B[3]) {
    return set_fields_impl(c, E, B, true);
}
int pic_get_fields(pic_ctx* c, double* const E[3], double* const B[3]) { return get_fields_impl(c, E, B, false); }
int pic_get_fields_dev(pic_ctx* c, double* const E[3], double* const B[3]) { return get_fields_impl(c, E, B, true); }
int pic_get_current(pic_ctx* c, double* const J[3]) { return get_current_impl(c, J, false); }
int pic_get_current_dev(pic_ctx* c, double* const J[3]) { return get_current_impl(c, J, true); }

int pic_step(pic_ctx* c, int nsteps) {
    if (!c) return PIC_ERR_ARG;
    if (nsteps < 0) return fail(c, PIC_ERR_ARG, "nsteps < 0");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    const double h = 0.5 * c->g.dt;
    const int nwf = fdtd_blocks(c->g);
    for (int t = 0; t < nsteps; ++t) {
        cudaEvent_t e0 = nullptr;
        bool due = false;
        int rd = sort_due(c, &due);
        if (rd) return rd;
        if (due) {
            stage_begin(c, 2, &e0);
            // cloud-in-cell: the particle kernel below moves the particles
            const bool ranks = c->desc.form_factor != 2;
            int r = materialize(c);  // a permutation still pending (a load's) is applied first
            if (!r) r = ranks ? sort_all_ranks(c) : sort_all(c);
            if (r) return r;
            stage_end(c, 2, e0);
        }
        stage_begin(c, 0, &e0);
        for (auto& s : c->sp) {
            if (s.immobile) continue;
            int r = c->desc.form_factor == 2 ? push_species_tsc(c, s)
                                             : (c->mixed ? push_species<float>(c, s) : push_species<double>(c, s));
            if (r) return r;
        }
        if (c->adaptive) CUDA_TRY(c, cudaEventRecord(c->ev_push, c->st));
        stage_end(c, 0, e0);
        stage_begin(c, 1, &e0);
        CUDA_TRY(c, fdtd_b_launch(c->st, c->EB, c->g, h, 0, nullptr, nullptr));
        CUDA_TRY(c, fdtd_e_launch(c->st, c->EB, c->J, c->Jlast, c->g));
        CUDA_TRY(c, fdtd_b_launch(c->st, c->EB, c->g, h, 1, c->EB32, c->d_wf));
        c->launches += 3;
        stage_end(c, 1, e0);
        stage_begin(c, 3, &e0);
        int r = finalize_energy(c, nwf);
        if (r) return r;
        stage_end(c, 3, e0);
        c->energy_fresh = true;
        c->since_sort += 1;
        c->steps += 1;
    }
    return PIC_OK;
}

int pic_sync(pic_ctx* c) {
    if (!c) return PIC_ERR_ARG;
    CUDA_TRY(c, cudaSetDevice(c->dev));
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    return device_status(c);
}

int pic_energy(pic_ctx* c, double* wf, double* wk) {
    if (!c) return PIC_ERR_ARG;
    if (!wf || !wk) return fail(c, PIC_ERR_ARG, "null output");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    if (!c->energy_fresh) {
        const int rm = materialize(c);  // the kinetic energy reads the store
        if (rm) return rm;
        CUDA_TRY(c, field_energy_launch(c->st, c->EB, c->g, c->d_wf));
        c->launches += 1;
        for (auto& s : c->sp) {
            cudaError_t e = c->mixed ? kinetic_launch<float>(c->st, c->push_grid, s.s32.a(), s.d_n, s.m, s.d_ek)
                                     : kinetic_launch<double>(c->st, c->push_grid, s.s64.a(), s.d_n, s.m, s.d_ek);
            c->launches += 1;
            if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "kinetic: %s", cudaGetErrorString(e));
        }
        int r = finalize_energy(c, fdtd_blocks(c->g));
        if (r) return r;
        c->energy_fresh = true;
    }
    double out[2];
    CUDA_TRY(c, cudaMemcpyAsync(out, c->d_energy, sizeof out, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    *wf = out[0];
    *wk = out[1];
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) {
        int one = ERRBIT_NAN;
        cudaMemcpy(c->d_err, &one, sizeof(int), cudaMemcpyHostToDevice);
        return fail(c, PIC_ERR_NAN, "non-finite energy (wf=%g, wk=%g)", out[0], out[1]);
    }
    return device_status(c);
}

int pic_enable_timing(pic_ctx* c, int on) {
    if (!c) return PIC_ERR_ARG;
    c->timing = on != 0;
    return PIC_OK;
}

int pic_stage_times(pic_ctx* c, double out[4]) {
    if (!c) return PIC_ERR_ARG;
    if (!out) return fail(c, PIC_ERR_ARG, "null output");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    for (int s = 0; s < 4; ++s) {
        for (auto& pr : c->ev[s]) {
            float ms = 0;
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            c->stage_ms[s] += ms;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        c->ev[s].clear();
        out[s] = c->stage_ms[s];
    }
    return PIC_OK;
}

int pic_launch_count(pic_ctx* c, int64_t* n, int reset) {
    if (!c) return PIC_ERR_ARG;
    if (!n) return fail(c, PIC_ERR_ARG, "null output");
    *n = c->launches;
    if (reset) c->launches = 0;
    return PIC_OK;
}

int pic_get_state(pic_ctx* c, void* blob, int64_t* bytes) {
    if (!c) return PIC_ERR_ARG;
    if (!bytes) return fail(c, PIC_ERR_ARG, "null size");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    {
        const int rm = materialize(c);  // the blob holds the store in sorted order
        if (rm) return rm;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    std::vector<long long> n(c->sp.size());
    std::vector<int> nch(c->sp.size());
    size_t total = pad8(sizeof(StateHeader)) + grid_payload(c);
    for (size_t i = 0; i < c->sp.size(); ++i) {
        CUDA_TRY(c, cudaMemcpy(&n[i], c->sp[i].d_n, sizeof(long long), cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(&nch[i], c->sp[i].d_nchunks, sizeof(int), cudaMemcpyDeviceToHost));
        total += pad8(sizeof(SpeciesHeader)) + species_payload(c, n[i], nch[i]);
    }
    if (!blob) {
        *bytes = (int64_t)total;
        return PIC_OK;
    }
    if (*bytes < (int64_t)total) return fail(c, PIC_ERR_ARG, "state blob of %lld bytes, %zu needed", (long long)*bytes, total);
    Cursor cur{static_cast<unsigned char*>(blob), (size_t)*bytes};
    unsigned char* at;
    cur.take(sizeof(StateHeader), &at);
    StateHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, STATE_MAGIC, 8);
    h.precision = c->desc.precision;
    h.supercell = c->desc.supercell;
    h.sort_interval = c->desc.sort_interval;
    h.absorb_cells = c->desc.absorb_cells;
    for (int a = 0; a < 3; ++a) {
        h.n[a] = c->desc.n[a];
        h.bc[a] = c->desc.bc[a];
        h.d[a] = c->desc.d[a];
    }
    h.dt = c->desc.dt;
    h.absorb_sigma = c->desc.absorb_sigma;
    h.nspecies = (int32_t)c->sp.size();
    h.form_factor = c->desc.form_factor == 2 ? 2 : 1;
    h.chunk = CHUNK;
    h.steps = c->steps;
    h.since_sort = c->since_sort;
    {
        int r = drift_sum(c, h.drift);
        if (r) return r;
    }
    memcpy(at, &h, sizeof h);
    const long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
    cur.take(6 * c->g.P * sizeof(double), &at);
    CUDA_TRY(c, cudaMemcpyAsync(at, c->EB, 6 * c->g.P * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    cur.take(3 * c->g.P * sizeof(double), &at);
    CUDA_TRY(c, cudaMemcpyAsync(at, c->J, 3 * c->g.P * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    cur.take(3 * ncell * sizeof(double), &at);
    CUDA_TRY(c, cudaMemcpyAsync(at, c->Jlast, 3 * ncell * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    for (size_t i = 0; i < c->sp.size(); ++i) {
        Species& s = c->sp[i];
        SpeciesHeader sh{s.q, s.m, (int64_t)n[i], (int64_t)s.nid, s.immobile ? 1 : 0, nch[i]};
        cur.take(sizeof sh, &at);
        memcpy(at, &sh, sizeof sh);
        int r = c->mixed ? copy_store<float>(c, s, n[i], cur, true) : copy_store<double>(c, s, n[i], cur, true);
        if (r) return r;
        cur.take(((size_t)c->g.nbins + 1) * sizeof(int), &at);
        CUDA_TRY(c, cudaMemcpyAsync(at, s.d_bin_start, ((size_t)c->g.nbins + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                                    c->st));
        if (nch[i] > 0) {
            cur.take((size_t)nch[i] * sizeof(Chunk), &at);
            CUDA_TRY(c, cudaMemcpyAsync(at, s.d_chunks, (size_t)nch[i] * sizeof(Chunk), cudaMemcpyDeviceToHost, c->st));
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    *bytes = (int64_t)total;
    return PIC_OK;
}

int pic_set_state(pic_ctx* c, const void* blob, int64_t bytes) {
    if (!c) return PIC_ERR_ARG;
    if (!blob || bytes < (int64_t)sizeof(StateHeader)) return fail(c, PIC_ERR_ARG, "null or short state blob");
    CUDA_TRY(c, cudaSetDevice(c->dev));
    {
        // a refused blob leaves the context as it was, in sorted order
        const int rm = materialize(c);
        if (rm) return rm;
    }
    Cursor cur{const_cast<unsigned char*>(static_cast<const unsigned char*>(blob)), (size_t)bytes};
    unsigned char* at;
    cur.take(sizeof(StateHeader), &at);
    StateHeader h;
    memcpy(&h, at, sizeof h);
    if (memcmp(h.magic, STATE_MAGIC, 8) != 0) return fail(c, PIC_ERR_ARG, "not a state blob of this library");
    if (!same_desc(h, c->desc)) return fail(c, PIC_ERR_ARG, "state blob was written for another grid descriptor");
    if (h.nspecies < 0 || h.nspecies > MAX_SPECIES) return fail(c, PIC_ERR_ARG, "bad species count in state blob");
    // steps since the last sort: a larger value would delay the next sort past the
    // supercell slack the particle kernel's tile allows
    if (h.since_sort < 0 || h.since_sort > c->K || h.steps < 0)
        return fail(c, PIC_ERR_ARG, "bad step counters in state blob");
    // the displacement bound: zero right after a sort and outside the schedule that keeps it;
    // at or beyond the slack, particles may already have left their tile
    for (int a = 0; a < 3; ++a)
        if (!(h.drift[a] >= 0.0 && h.drift[a] < 1.0) || ((h.since_sort == 0 || !c->adaptive) && h.drift[a] != 0.0))
            return fail(c, PIC_ERR_ARG, "bad displacement bound in state blob");
    if (cur.left < grid_payload(c)) return fail(c, PIC_ERR_ARG, "state blob too small");
    // validate every species section before touching the context
    {
        Cursor probe = cur;
        const long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
        unsigned char* q;
        probe.take(6 * c->g.P * sizeof(double), &q);
        probe.take(3 * c->g.P * sizeof(double), &q);
        probe.take(3 * ncell * sizeof(double), &q);
        for (int i = 0; i < h.nspecies; ++i) {
            SpeciesHeader sh;
            if (!probe.take(sizeof sh, &q)) return fail(c, PIC_ERR_ARG, "state blob too small");
            memcpy(&sh, q, sizeof sh);
            const long long maxch = c->g.nbins + (sh.n > 0 ? sh.n : 1) / CHUNK + 1;
            if (sh.n < 0 || sh.n >= (1LL << 31) - 1 || sh.nchunks < 0 || sh.nchunks > maxch || !(sh.m > 0))
                return fail(c, PIC_ERR_ARG, "bad species record in state blob");
            const size_t need = species_payload(c, sh.n, sh.nchunks);
            if (probe.left < need) return fail(c, PIC_ERR_ARG, "state blob too small");
            if (!species_payload_valid(c, probe.p, sh.n, sh.nchunks))
                return fail(c, PIC_ERR_ARG, "state blob holds a cell or chunk outside the grid");
            probe.p += need;
            probe.left -= need;
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    for (auto& s : c->sp) free_species(s);
    c->sp.clear();
    c->tape.release();
    const long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
    cur.take(6 * c->g.P * sizeof(double), &at);
    CUDA_TRY(c, cudaMemcpyAsync(c->EB, at, 6 * c->g.P * sizeof(double), cudaMemcpyHostToDevice, c->st));
    cur.take(3 * c->g.P * sizeof(double), &at);
    CUDA_TRY(c, cudaMemcpyAsync(c->J, at, 3 * c->g.P * sizeof(double), cudaMemcpyHostToDevice, c->st));
    cur.take(3 * ncell * sizeof(double), &at);
    CUDA_TRY(c, cudaMemcpyAsync(c->Jlast, at, 3 * ncell * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CUDA_TRY(c, refresh_launch(c->st, c->EB, c->g, c->EB32));
    c->launches += 1;
    for (int i = 0; i < h.nspecies; ++i) {
        SpeciesHeader sh;
        cur.take(sizeof sh, &at);
        memcpy(&sh, at, sizeof sh);
        c->sp.emplace_back();
        Species& s = c->sp.back();
        s.q = sh.q;
        s.m = sh.m;
        s.immobile = sh.immobile != 0;
        s.nid = sh.nid;
        int r = alloc_species(c, s, sh.n);
        if (!r) r = c->mixed ? copy_store<float>(c, s, sh.n, cur, false) : copy_store<double>(c, s, sh.n, cur, false);
        if (r) return r;
        const long long nn[2] = {sh.n, sh.n};
        CUDA_TRY(c, cudaMemcpyAsync(s.d_n, nn, sizeof nn, cudaMemcpyHostToDevice, c->st));
        cur.take(((size_t)c->g.nbins + 1) * sizeof(int), &at);
        CUDA_TRY(c, cudaMemcpyAsync(s.d_bin_start, at, ((size_t)c->g.nbins + 1) * sizeof(int), cudaMemcpyHostToDevice,
                                    c->st));
        if (sh.nchunks > 0) {
            cur.take((size_t)sh.nchunks * sizeof(Chunk), &at);
            CUDA_TRY(c, cudaMemcpyAsync(s.d_chunks, at, (size_t)sh.nchunks * sizeof(Chunk), cudaMemcpyHostToDevice,
                                        c->st));
        }
        CUDA_TRY(c, cudaMemcpyAsync(s.d_nchunks, &sh.nchunks, sizeof(int), cudaMemcpyHostToDevice, c->st));
        if ((r = refresh_wmax(c, s))) return r;
        // the host values above are locals: finish the copies before they go out of scope
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
    int r = rebuild_ek(c);
    if (r) return r;
    c->steps = h.steps;
    c->since_sort = (int)h.since_sort;
    c->energy_fresh = false;
    if (c->adaptive) {
        // the restored bound as the speed sum before the run's first row; the rows empty
        c->vsum0 = 0.0;
        for (int a = 0; a < 3; ++a) c->vsum0 = std::max(c->vsum0, h.drift[a] / c->dtd[a]);
        CUDA_TRY(c, cudaMemsetAsync(c->d_drift, 0, DRIFT_ROWS * sizeof(unsigned), c->st));
        CUDA_TRY(c, cudaEventRecord(c->ev_push, c->st));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_selftest_wait_timeout(pic_ctx* c) {
    if (!c) return PIC_ERR_ARG;
    CUDA_TRY(c, cudaSetDevice(c->dev));
    if (device_status(c) != PIC_OK) return fail(c, PIC_ERR_STATE, "a device flag is already set");
    CUDA_TRY(c, wait_probe_launch(c->st, c->d_err, 10000000ull));
    c->launches += 1;
    const int r = device_status(c);
    CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return r;
}

int pic_index_status(int device) {
    if (cudaSetDevice(device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
#if PICGB_DEBUG
    const int idx = push_index_flags() | push32_index_flags() | tsc_index_flags() | tape_index_flags() |
                    sort_index_flags();
    return idx ? PIC_ERR_INDEX : PIC_OK;
#else
    return PIC_OK;
#endif
}

int pic_tape_forward(pic_ctx* c, int nsteps, int ckpt_every, double* wk) {
    if (!c) return PIC_ERR_ARG;
    CUDA_TRY(c, cudaSetDevice(c->dev));
    return tape_forward_impl(c, nsteps, ckpt_every, wk);
}

int pic_tape_backward(pic_ctx* c, double wk_weight, const double* const gE[3], const double* const gB[3],
                      double* const dE0[3], double* const dB0[3]) {
    if (!c) return PIC_ERR_ARG;
    CUDA_TRY(c, cudaSetDevice(c->dev));
    return tape_backward_impl(c, wk_weight, gE, gB, dE0, dB0);
}

int pic_tape_particle_grad(pic_ctx* c, int species, double* const dP[6]) {
    if (!c) return PIC_ERR_ARG;
    if (!dP) return fail(c, PIC_ERR_ARG, "null output");
    if (!c->tape.ready) return fail(c, PIC_ERR_STATE, "no tape recorded");
    if (species < 0 || species >= (int)c->tape.sp.size()) return fail(c, PIC_ERR_ARG, "bad species %d", species);
    CUDA_TRY(c, cudaSetDevice(c->dev));
    TapeSpecies& ts = c->tape.sp[species];
    if (ts.n == 0) return PIC_OK;
    double** d = nullptr;
    CUDA_TRY(c, cudaMalloc(&d, 6 * sizeof(double*)));
    double* h[6];
    for (int k = 0; k < 6; ++k) h[k] = dP[k];
    cudaError_t e = cudaMemcpyAsync(d, h, sizeof h, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = lam_to_phys_launch(c->st, ts.lam, ts.n, c->g, d);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(d);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, PIC_ERR_CUDA, "particle grad: %s", cudaGetErrorString(e));
    return PIC_OK;
}

}  // extern "C"

