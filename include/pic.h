/*
 * pic.h -- C ABI of the GB300 particle-in-cell hot path (libpicgb.so).
 *
 * The library advances the particle-in-cell cycle that arXiv:1608.01009
 * (Surmin et al., "Co-design of a particle-in-cell plasma simulation code for
 * Intel Xeon Phi: a first look at Knights Landing") sets out in Sec. 2 and
 * Sec. 3: Maxwell's equations integrated on a grid, the field interpolated to
 * each macro-particle with the cloud-in-cell form factor, the relativistic
 * equations of motion, and the Villasenor-Buneman charge-conserving current
 * deposition, in double precision.  The paper names neither pusher nor field
 * solver; this library uses the relativistic Boris pusher and the Yee FDTD
 * scheme (staggering below), with B split into two half steps so that E and B
 * are both known at integer time levels when the particles are pushed.
 *
 * Units are normalised to a reference frequency w_r: time 1/w_r, length
 * c/w_r, momentum u = gamma v / c, fields m_e c w_r / e, current e n_r c.
 * Maxwell: dE/dt = curl B - J, dB/dt = -curl E.  Motion: du/dt = (q/m)(E +
 * u x B / gamma), dx/dt = u / gamma.  Weight w = real particles per
 * macro-particle in these units (density x cell volume / particles per cell).
 *
 * Yee staggering (cell (i,j,k) has its corner node at (i dx, j dy, k dz)):
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)   (J the same)
 *   Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
 * Field arrays at this ABI are unpadded, nx*ny*nz doubles per component, x
 * fastest: element (i,j,k) at index i + nx*(j + ny*k).
 *
 * One step (state x^n, u^{n-1/2}, E^n, B^n):
 *   gather E^n, B^n at x^n; Boris u^{n-1/2} -> u^{n+1/2};
 *   x^{n+1} = x^n + dt u^{n+1/2} / gamma; deposit J^{n+1/2} from x^n -> x^{n+1};
 *   B^{n+1/2} = B^n - dt/2 curl E^n; E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2});
 *   B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}.
 *
 * Conventions of every call:
 *   - returns PIC_OK (0) or a negative pic_status; no exception crosses the
 *     ABI and no kernel traps; pic_last_error() gives a message;
 *   - "_dev" variants take device pointers (e.g. from torch tensors) and work
 *     asynchronously on the context's stream; the others take host pointers
 *     and return once the copy is complete (except pic_upload_particles, whose
 *     copy runs on the context's copy stream);
 *   - the caller owns every buffer it passes; the library owns its context
 *     and all device state, released by pic_destroy();
 *   - one context is used from one host thread at a time.
 */
#ifndef PICGB_PIC_H
#define PICGB_PIC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = -1,          /* invalid argument or descriptor */
    PIC_ERR_CFL = -2,          /* time step violates the Courant limit or the sort interval */
    PIC_ERR_OOM = -3,          /* device allocation failed */
    PIC_ERR_BIN_OVERFLOW = -4, /* a particle left its supercell's halo slack between sorts */
    PIC_ERR_NAN = -5,          /* a non-finite value reached the energy diagnostics */
    PIC_ERR_CUDA = -6,         /* a CUDA runtime call failed */
    PIC_ERR_STATE = -7,        /* call not valid in the current state */
    PIC_ERR_TIMEOUT = -8,      /* a bounded wait inside a kernel expired */
    PIC_ERR_INDEX = -9         /* debug build only: a kernel index fell outside its array */
} pic_status;

enum { PIC_BC_PERIODIC = 0, PIC_BC_ABSORBING = 1 };
enum { PIC_FP64 = 0, PIC_MIXED = 1 };

/* Grid and run descriptor.
 *   n[3]          cells per axis; each a multiple of `supercell`, 4..1024
 *   d[3]          cell sizes (c/w_r)
 *   dt            time step (1/w_r); needs dt * sqrt(sum 1/d^2) < 1 (Courant)
 *   bc[3]         PIC_BC_PERIODIC or PIC_BC_ABSORBING per axis.  Along an
 *                 absorbing axis the field is zero outside the domain, current
 *                 deposited outside it is dropped, particles leaving it are
 *                 deactivated, and after each field sub-update E and B inside a
 *                 layer of `absorb_cells` cells are multiplied by
 *                 1 - absorb_sigma ((L - dist)/L)^2 (dist = distance in cells of
 *                 the component's lattice point from the nearer boundary).
 *   precision     PIC_FP64: particles, interpolation, push and shared-memory
 *                 current sums in FP64.  PIC_MIXED: cell-relative FP32 particle
 *                 offsets, FP32 momenta, FP32 interpolation from an FP32 copy of
 *                 the fields and FP32 shared-memory current sums; global current,
 *                 fields and energy diagnostics stay FP64.
 *   supercell     S, cells per supercell edge: 4 or 8 (2 also for PIC_FP64)
 *   sort_interval K, steps between supercell re-sorts, K * max_a(dt / d_a) < 1
 *                 (a particle moves less than one cell per step along each
 *                 axis, and the supercell tiles carry one cell of slack).
 *                 0 = the library's schedule: PIC_FP64 with the cloud-in-cell
 *                 form factor sorts every step (its particle kernel is fastest
 *                 on freshly sorted particles); the second-order form factor
 *                 takes the largest allowed K; PIC_MIXED sorts when the
 *                 displacement bound requires it: the particle kernel records
 *                 each step's largest speed v_i, and a sort precedes the next
 *                 step once (sum_i v_i + 1) dt / d_a could reach one cell on
 *                 some axis (at most 64 steps between sorts)
 *   form_factor   0 or 1: cloud-in-cell with the Villasenor-Buneman current
 *                 (Sec. 3, the paper's scheme); 2: the second-order
 *                 (triangular-shaped cloud) form factor, quadratic B-spline
 *                 weights on the 3 x 3 x 3 nearest lattice points of each
 *                 staggered component, with Esirkepov's charge-conserving
 *                 current (PIC_FP64 only; the differentiable-run calls take
 *                 form factor 1 only)
 *   device        CUDA device ordinal
 *   stream        cudaStream_t the context works on (NULL = legacy default)
 */
typedef struct {
    int32_t n[3];
    double d[3];
    double dt;
    int32_t bc[3];
    int32_t absorb_cells;
    double absorb_sigma;
    int32_t precision;
    int32_t supercell;
    int32_t sort_interval;
    int32_t form_factor;
    int32_t device;
    void* stream;
} pic_grid_desc;

/* Species: charge q and mass m in units of e and m_e (electrons: -1, 1).
 * immobile != 0 declares a neutralising background of immobile ions (the
 * paper describes no ion model; this is the usual PIC convention): its
 * particles are neither stored nor pushed and carry no current; the species
 * keeps its id and reports 0 particles. */
typedef struct {
    double q;
    double m;
    int32_t immobile;
} pic_species_desc;

typedef struct pic_ctx pic_ctx;

/* Create a context (Sec. 2: the field and the current density are defined on
 * a discrete grid, on which Maxwell's equations are integrated): validates
 * `g` (PIC_ERR_ARG, PIC_ERR_CFL) before touching the GPU, then allocates the
 * ghost-padded FP64 E, B, J grids (and the FP32 field copy in mixed mode), all
 * zero.  *out receives the context. */
PIC_API int pic_create(const pic_grid_desc* g, pic_ctx** out);

/* Wait for the context's stream (and its copy stream) and release everything
 * it owns (a library facility; the paper has no counterpart). */
PIC_API int pic_destroy(pic_ctx* ctx);

/* Message of the last error of this context ("" if none); valid until the
 * next call on the context (a library facility). */
PIC_API const char* pic_last_error(const pic_ctx* ctx);

/* Add a species of n macro-particles (Sec. 2: the plasma is represented by
 * macro-particles).  x,y,z are physical positions inside the domain,
 * ux,uy,uz the momenta u^{-1/2}, w the weights; each array has n doubles.
 * Particles are given ids 0..n-1 in input order, binned by supercell and
 * stored in the library (FP64 or FP32 per `precision`).  *species_id receives
 * the species index.  Host variant: copies and returns when done; page-locked
 * host arrays (cudaHostAlloc, cudaHostRegister) are read in place by the load
 * kernel, pageable ones are staged through device memory. */
PIC_API int pic_add_species(pic_ctx* ctx, const pic_species_desc* s, int64_t n, const double* x, const double* y,
                    const double* z, const double* ux, const double* uy, const double* uz, const double* w,
                    int* species_id);
PIC_API int pic_add_species_dev(pic_ctx* ctx, const pic_species_desc* s, int64_t n, const double* x,
                        const double* y, const double* z, const double* ux, const double* uy,
                        const double* uz, const double* w, int* species_id);

/* Replace all particles of an existing species (Sec. 2: the macro-particle
 * ensemble; same layout as pic_add_species; ids restart at 0).  Used to load
 * a new state. */
PIC_API int pic_set_particles(pic_ctx* ctx, int species, int64_t n, const double* x, const double* y, const double* z,
                      const double* ux, const double* uy, const double* uz, const double* w);
PIC_API int pic_set_particles_dev(pic_ctx* ctx, int species, int64_t n, const double* x, const double* y,
                          const double* z, const double* ux, const double* uy, const double* uz,
                          const double* w);

/* Double-buffered replacement of a species' particles, for pipelines that
 * upload a new particle set every step (a library facility around the
 * macro-particle ensemble of Sec. 2).
 *
 * pic_upload_particles starts copying n particles (the seven arrays of
 * pic_add_species, host or device memory) into the species' upload area on the
 * context's copy stream and returns at once; the copy overlaps whatever the
 * context's stream is running.  The species' current particles are untouched.
 * Host arrays should be page-locked (pageable arrays are read before the call
 * returns, so their copy does not overlap).  The caller keeps every array
 * unchanged until the upload has been consumed by pic_set_particles_uploaded
 * and the context has been synchronised (pic_sync or any synchronising call).  A second upload
 * before consumption replaces the first.  The upload area is library-owned
 * (7 n doubles, grown on demand).  PIC_ERR_ARG: bad species, an immobile
 * species, n out of range or a null array.
 *
 * pic_set_particles_uploaded replaces the species' particles with the pending
 * upload, as pic_set_particles_dev would (ids restart at 0), ordered after the
 * copy on the context's stream; asynchronous.  The next upload's copy waits
 * for this load to have read the area.  PIC_ERR_STATE if no upload is
 * pending. */
PIC_API int pic_upload_particles(pic_ctx* ctx, int species, int64_t n, const double* x, const double* y,
                                 const double* z, const double* ux, const double* uy, const double* uz,
                                 const double* w);
PIC_API int pic_set_particles_uploaded(pic_ctx* ctx, int species);

/* Species properties (Sec. 2: each macro-particle species has its charge and
 * mass): q, m, the immobile flag, and nid, the number of ids given at the
 * species' last load (ids run 0..nid-1; particles that left
 * through an absorbing boundary keep their ids unused).  Any output pointer
 * may be NULL. */
PIC_API int pic_species_info(pic_ctx* ctx, int species, double* q, double* m, int32_t* immobile, int64_t* nid);

/* Number of active particles of a species (Sec. 2; particles that left
 * through an absorbing boundary are not counted).  Synchronises the stream. */
PIC_API int pic_count_particles(pic_ctx* ctx, int species, int64_t* n);

/* Copy out the active particles of a species (the macro-particle state of
 * Sec. 2 that the step advances): ids, physical positions
 * (wrapped into the domain on periodic axes), momenta and weights, FP64.
 * Order is the library's internal (binned) order; match by id.  `cap` is
 * the length of the caller's arrays; *n receives the count written
 * (PIC_ERR_ARG if cap is too small).  Synchronises the stream. */
PIC_API int pic_get_particles(pic_ctx* ctx, int species, int64_t cap, int64_t* n, int64_t* id, double* x, double* y,
                      double* z, double* ux, double* uy, double* uz, double* w);
PIC_API int pic_get_particles_dev(pic_ctx* ctx, int species, int64_t cap, int64_t* n, int64_t* id, double* x,
                          double* y, double* z, double* ux, double* uy, double* uz, double* w);

/* Set / get E and B, the grid fields of Sec. 2 (unpadded layout above; E[c],
 * B[c] one array per component).  Setting refreshes the periodic ghost layers
 * and the FP32 copy.  Getting returns E^n, B^n of the current state. */
PIC_API int pic_set_fields(pic_ctx* ctx, const double* const E[3], const double* const B[3]);
PIC_API int pic_set_fields_dev(pic_ctx* ctx, const double* const E[3], const double* const B[3]);
PIC_API int pic_get_fields(pic_ctx* ctx, double* const E[3], double* const B[3]);
PIC_API int pic_get_fields_dev(pic_ctx* ctx, double* const E[3], double* const B[3]);

/* The current density J^{n+1/2} deposited by the last step (Sec. 2: the
 * current computed from the particles feeds Maxwell's equations; Sec. 3: the
 * Villasenor-Buneman scheme), periodic images folded onto their owners, same
 * layout as E. */
PIC_API int pic_get_current(pic_ctx* ctx, double* const J[3]);
PIC_API int pic_get_current_dev(pic_ctx* ctx, double* const J[3]);

/* Advance nsteps whole steps (the stages of Sec. 2 in the order above: field
 * interpolation, equations of motion, current deposition, field update; with
 * the schemes of Sec. 3), asynchronously on the stream.  Particles are
 * processed by supercells (Sec. 4.3).  Every `sort_interval` steps the particles are re-binned by
 * supercell (an on-device counting sort).  Device-side faults are recorded in
 * a sticky flag that pic_sync() returns. */
PIC_API int pic_step(pic_ctx* ctx, int nsteps);

/* Wait for the stream; return the sticky device status (PIC_OK,
 * PIC_ERR_BIN_OVERFLOW, PIC_ERR_TIMEOUT, PIC_ERR_NAN) or PIC_ERR_CUDA (a
 * library facility). */
PIC_API int pic_sync(pic_ctx* ctx);

/* Energy of the current state (a diagnostic; the paper reports none, its
 * runs measure time only).  Synchronises.  Field energy
 * W_F = 1/2 dV sum (E^2 + B^2) and kinetic energy W_K = sum m w (gamma - 1)
 * over active particles, gamma from the stored u^{n-1/2}; FP64. */
PIC_API int pic_energy(pic_ctx* ctx, double* wf, double* wk);

/* Turn per-stage CUDA-event timing on (1) or off (0, the default), and read
 * the accumulated milliseconds (the stage split of the paper's Table 6: push,
 * deposit, other): out[0] particle push + current deposition
 * (one fused kernel per species), out[1] field solver, out[2] supercell sort,
 * out[3] diagnostics.  pic_stage_times synchronises. */
PIC_API int pic_enable_timing(pic_ctx* ctx, int on);
PIC_API int pic_stage_times(pic_ctx* ctx, double out[4]);

/* Kernels this context has launched since creation (or the last reset); a
 * library facility. */
PIC_API int pic_launch_count(pic_ctx* ctx, int64_t* n, int reset);

/* Differentiable runs: a hand-written discrete adjoint of the whole step
 * (push, deposit and FDTD) with checkpointed recomputation.
 *
 * pic_tape_forward advances nsteps whole steps from the current state on the
 * differentiable FP64 path -- the same step as pic_step (cloud-in-cell
 * gather, Boris push, Villasenor-Buneman deposit, Yee FDTD; Sec. 2-3), with
 * the particles kept in id order and no supercell sort, so that any segment
 * can be replayed exactly -- saving the FP64 state every `ckpt_every` steps in
 * library-owned device memory, and recording the last segment's steps (each
 * step's momenta, and the positions and active flags of every
 * ceil(sqrt(ckpt_every))-th step, from which the others are rebuilt exactly:
 * about 24 + 28 / sqrt(ckpt_every) bytes per particle and step, against 52 for
 * a whole state).  *wk receives the final kinetic energy
 * W_K = sum m w (gamma - 1).  The context continues from the final state.
 * PIC_ERR_OOM if the tape does not fit in device memory (nothing is kept).
 *
 * pic_tape_backward then computes the gradient of
 *     L = wk_weight * W_K(final) + <gE, E(final)> + <gB, B(final)>
 * with respect to the fields at the start of the tape: for each checkpoint
 * segment in reverse it restores the checkpoint, recomputes the segment while
 * recording its steps (the last segment was recorded by the forward), and runs
 * the adjoint kernels backwards through it.  gE, gB: unpadded device arrays or NULL (zero); dE0, dB0: unpadded
 * device arrays that receive dL/dE(start), dL/dB(start), or NULL.  Both calls
 * synchronise.  pic_tape_particle_grad then copies dL/d(x, y, z, ux, uy, uz)
 * of the starting particles of a species, in id order (device arrays of the
 * species' id count, NULL entries skipped; positions in physical units).
 * PIC_ERR_STATE if no tape has been recorded. */
PIC_API int pic_tape_forward(pic_ctx* ctx, int nsteps, int ckpt_every, double* wk);
PIC_API int pic_tape_backward(pic_ctx* ctx, double wk_weight, const double* const gE[3], const double* const gB[3],
                              double* const dE0[3], double* const dB0[3]);
PIC_API int pic_tape_particle_grad(pic_ctx* ctx, int species, double* const dP[6]);

/* Checkpoint and resume (the paper describes none; a library facility).
 * pic_get_state with blob == NULL stores in *bytes the size of the context's
 * state; with a host buffer of *bytes bytes it copies the whole state into
 * it and synchronises: a header (grid descriptor, step counters, species
 * count), the ghost-padded E, B, J grids, the last folded current, and every
 * species' q, m and binned particle store in its internal precision and
 * order, with its bin table.  PIC_ERR_ARG if *bytes is too small.
 * pic_set_state restores a blob written by pic_get_state into a context
 * created with the same descriptor (n, d, dt, bc, absorbing layer,
 * precision, supercell, sort_interval, form factor; PIC_ERR_ARG otherwise), replacing all
 * of its species and dropping a recorded tape; stepping on reproduces the
 * saved run up to the summation order of floating-point atomics.  The blob
 * is a plain byte image for this library build and machine (native byte
 * order); the caller owns it. */
PIC_API int pic_get_state(pic_ctx* ctx, void* blob, int64_t* bytes);
PIC_API int pic_set_state(pic_ctx* ctx, const void* blob, int64_t bytes);

/* Self test of the failure path of the kernels' bounded waits (a library
 * facility; the paper has no counterpart).  A one-thread kernel arms a
 * shared-memory barrier for a transfer that is never issued and waits on it
 * with the particle kernel's bounded wait, limited to 10 ms of device time;
 * the wait gives up and sets the sticky timeout flag.  Returns the status the
 * host then reads -- PIC_ERR_TIMEOUT when the path works -- after clearing
 * that flag, so the context stays usable; PIC_ERR_STATE if a device flag was
 * already set before the call.  Synchronises. */
PIC_API int pic_selftest_wait_timeout(pic_ctx* ctx);

/* Self test of the debug build's index checks (a library facility; the paper
 * has no counterpart).  The library built with PICGB_DEBUG=1
 * (libpicgb_debug.so) passes every index its particle, second-order
 * form-factor, differentiable-path and sort kernels use to address an array
 * through a check against that array's size; an index outside sets a flag and
 * the access is skipped, so a wrong index shows as PIC_ERR_INDEX from the next
 * status read (pic_sync, pic_step) instead of a memory fault.  The flags are
 * per device and process, not per context.  This call launches a one-thread
 * kernel on `device` that checks index 1 against an array of one element
 * (nothing is read or written but the flag), reads that flag and clears it.
 * Returns PIC_ERR_INDEX in the debug build (the check fired), PIC_OK in the
 * release build (the checks are compiled out), PIC_ERR_CUDA on a CUDA error.
 * Synchronises the device. */
PIC_API int pic_selftest_index_check(int device);

/* Index-check status of `device` (debug build): after synchronising the
 * device, PIC_ERR_INDEX if any checking kernel of any context saw an index
 * outside its array since the last pic_index_status (or context status read,
 * which also takes the flags), else PIC_OK; the flags are cleared.  The
 * release build returns PIC_OK (nothing is checked).  PIC_ERR_CUDA if the
 * device cannot be selected or synchronised. */
PIC_API int pic_index_status(int device);

/* Field energy W_F = 1/2 dx dy dz sum (E^2 + B^2) of caller-provided fields,
 * allocating nothing.  The paper has no counterpart: this is a library
 * facility for callers that cannot allocate device memory -- a host framework
 * that owns all device memory through its own pool, a process that has
 * already reserved the whole device, or a latency-critical loop that cannot
 * take cudaMalloc's implicit device-wide synchronisation.  It needs no
 * context.
 *   E[3], B[3]  device arrays in the unpadded layout above (nx*ny*nz doubles)
 *   n[3], d[3]  cells per axis and cell sizes (host arrays)
 *   wf          device pointer to one double; written when `stream` runs the work
 *   stream      cudaStream_t (NULL = legacy default stream)
 * Scratch: the per-block partial sums live in one fixed device array of
 * 65,536 doubles (512 KiB) that every GPU which loads the library holds until
 * the process exits, so grids are limited to 16,777,216 cells (256^3); larger
 * ones return PIC_ERR_ARG with a message on stderr.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU (unordered streams)
 * race.  Each call overwrites every partial it reads, so nothing is cleared
 * between calls.  Returns PIC_OK once the work is enqueued, PIC_ERR_ARG or
 * PIC_ERR_CUDA. */
PIC_API int pic_field_energy_noalloc(const double* const E[3], const double* const B[3], const int32_t n[3],
                                     const double d[3], double* wf, void* stream);

/* Measured FP64 fused multiply-add throughput of a device, the denominator
 * of the FP64 particle kernel's roofline (a library facility for
 * measurement; the paper has no counterpart).  It needs no context and
 * allocates nothing.  A kernel of independent FMA chains
 * (4 CTAs of 256 threads per SM, 8 chains per thread, `iters` FMAs per chain)
 * runs once untimed and three times timed on a private stream of `device`;
 * *tflops receives 2 x FMAs / the fastest timed launch in TFLOP/s and *ms
 * that launch's milliseconds.  iters in 1..2^30 (2048 takes a few ms on a
 * GB300).  Synchronises.  PIC_ERR_ARG for a null output or iters out of
 * range, PIC_ERR_CUDA if the device or a launch fails. */
PIC_API int pic_probe_fp64_fma(int device, int64_t iters, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* PICGB_PIC_H */
