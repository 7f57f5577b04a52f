/*
 * pic.h - C-ABI of the GB300 (sm_103a) hot-electron particle-in-cell step.
 *
 * The library advances the superparticle representation of the 1-D
 * spin-dependent hot-electron Boltzmann equation of Nenno, Rethfeld and
 * Schneider (arXiv:1807.04733), Eq. bte2 (Sec. II), with the PIC method of
 * Eq. PIC and the Strang splitting of Eq. strang (Sec. III.A):
 *
 *   Source(dt/2) -> Transport(dt/2) -> Scattering(dt) -> Transport(dt/2)
 *   -> Source(dt/2)
 *
 * Each superparticle carries depth z (nm), direction cosine mu, energy bin k
 * (E_k = k dE above E_F), spin sigma, layer index and generation.  All
 * device work runs in hand-written CUDA kernels on the stream given to
 * pic_init.  PyTorch (or any caller) provides only memory and streams.
 *
 * Conventions for every call:
 *   - Every call returns a pic_status; no call aborts or exits.
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *     device memory of the current device (e.g. torch.Tensor.data_ptr()).
 *   - The caller owns every buffer it passes; the library copies the tables
 *     at pic_init and owns the particle state, histograms and scratch.
 *   - Device-side faults (capacity overflow in strict mode, a bounded wait
 *     that ran out) set a status word on the device; it is returned by the
 *     next synchronising call (pic_moments, pic_records, pic_sync, pic_grad).
 *   - A context is not thread-safe; calls on one context must be serialised.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_MAX_LAYERS 16   /* layers per stack */
#define PIC_MAX_MAT 8       /* materials per table set */
#define PIC_MAX_NE 255      /* energy bins */
#define PIC_MAX_STACKS 256  /* stacks per context */
#define PIC_MAX_HITS 8      /* boundary hits handled per half flight */

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,       /* invalid argument; nothing was changed */
    PIC_ERR_ALLOC = 2,     /* device or host allocation failed */
    PIC_ERR_CAPACITY = 3,  /* strict capacity mode: a carrier did not fit */
    PIC_ERR_TIMEOUT = 4,   /* a bounded device wait ran out; results invalid */
    PIC_ERR_CUDA = 5,      /* a CUDA runtime call failed (see pic_last_error) */
    PIC_ERR_STATE = 6      /* call not valid in the current state */
} pic_status;

/* pic_params.flags */
#define PIC_F_DETERMINISTIC   1u  /* no fused multiply-add in the flight: the
                                     particle records are bit-identical to a
                                     scalar IEEE float32 evaluation */
#define PIC_F_NO_SECONDARIES  2u  /* Sec. V.A variant (3): inelastic events do
                                     not create a secondary carrier */
#define PIC_F_TRANSPARENT     4u  /* Sec. V.A variant (2): T = 1 everywhere */
#define PIC_F_LOWEST_BIN_ANY  8u  /* remove a lowest-bin carrier on any
                                     scattering event (default: inelastic only) */
#define PIC_F_STRICT_CAPACITY 16u /* overflow is PIC_ERR_CAPACITY instead of
                                     drop-and-count */
#define PIC_F_VELOCITY_MOMENTS 32u /* also sum the carriers' velocities along z
                                      per (time, spin, cell): pic_vel_moments */
#define PIC_F_WEIGHTS         64u /* superparticle weights w_i of Eq. PIC
                                     (Sec. III.A): every carrier carries a
                                     weight, set at birth by importance
                                     sampling of the source (pic_pulse
                                     cell_bias, e_bias) and inherited by its
                                     secondaries; pic_weighted_moments */

/* Global parameters of a context. */
typedef struct {
    int32_t n_e;            /* energy bins, 1..PIC_MAX_NE; E_k = k*dE, k=1..n_e */
    float dt;               /* time step, fs (> 0); Strang step of Eq. strang */
    float dz;               /* moment cell width, nm: a power of two (0.5, 1,
                               2 ...); layer thicknesses are whole cells */
    uint64_t seed;          /* Philox4x32-10 key */
    uint32_t flags;         /* PIC_F_* */
    int32_t compact_every;  /* stable removal of dead slots every N steps (>= 1) */
    int32_t moment_every;   /* density snapshot every N steps (>= 1); the flux
                               is taken over the same windows */
    int32_t n_steps_max;    /* steps this context may run; sizes the moment
                               buffers: n_out = ceil(n_steps_max/moment_every) */
    int32_t blocks_per_sm;  /* persistent blocks per SM for the step kernel;
                               0 = as many as fit */
    int32_t hist_mode;      /* density deposit: 0 = shared-memory atomics,
                               1 = warp-aggregated (match-any) atomics */
    int32_t ring_stages;    /* tiles in the step kernel's bulk-copy ring
                               (2..8); 0 = chosen from the occupancy */
    int32_t use_graph;      /* 1: pic_step replays whole periods (the least
                               common multiple of moment_every and
                               compact_every) from CUDA graphs captured once,
                               the kernels reading the step index from device
                               memory; 2: each whole period is one persistent
                               cooperative launch (every block resident, the
                               passes of every step separated by grid barriers
                               with bounded waits), captured in a CUDA graph;
                               0: one launch per kernel.  Results are
                               identical; kernel timing (pic_profile) always
                               uses single launches. */
    int32_t stack_base;     /* global index of the context's first stack
                               (0..65535 - n_stacks): stack s draws the random
                               streams of stack stack_base + s, so that stacks
                               split over several contexts (one per GPU or
                               process) give the results of one context that
                               holds them all */
    int32_t consumer_warps; /* warps of the streaming pass that work on the
                               carriers, 4 or 8 (each thread then takes 8 or 4
                               consecutive slots of a 1024-slot tile); 0 = 8.
                               Results do not depend on it. */
    int32_t event_pass;     /* 0: the ordinary steps of a single-stack context
                               with eight consumer warps run the general step
                               of the eventful carriers inside the streaming
                               pass (extra warps fed through a shared-memory
                               ring, while the carriers' sectors are in L2);
                               1: always a separate event pass after the
                               streaming pass.  Results do not depend on it. */
} pic_params;

/* Launch configuration a context chose (pic_launch_info). */
typedef struct {
    int32_t grid_step, grid_step_moments;   /* streaming pass */
    int32_t grid_slow, grid_slow_moments;   /* event pass */
    int32_t grid_compact, grid_inject;
    int32_t ring_step, ring_step_moments;   /* bulk-copy ring depth (tiles) */
    int64_t smem_step, smem_step_moments;   /* dynamic shared memory, bytes */
    int32_t warps_step, warps_step_moments; /* consumer warps per block */
    /* pic_grad's replay passes 1 and 2 (zero before the first pic_grad):
     * streaming pass with density weights, its ring depth and shared memory */
    int32_t grid_adj_step[2], ring_adj_step[2];
    int64_t smem_adj_step[2];
    /* the streaming pass with the general step inside (event_pass 0); grid
     * 0: ordinary steps use the separate event pass */
    int32_t grid_step_fused, ring_step_fused;
    int64_t smem_step_fused;
} pic_launch_info;

/* One laterally homogeneous layer stack (Sec. II: 1-D transport along z).
 * Layer l spans [sum_{j<l} cells_j, sum_{j<=l} cells_j) * dz; the outer
 * surfaces z = 0 and z = L are vacuum (full reflection, Sec. III). */
typedef struct {
    int32_t n_layers;                       /* 1..PIC_MAX_LAYERS */
    int32_t layer_cells[PIC_MAX_LAYERS];    /* thickness in cells (>= 1) */
    int32_t layer_mat[PIC_MAX_LAYERS];      /* index into the material tables */
    int64_t capacity;                       /* particle slots, < 2^30 */
} pic_stack_desc;

/* Physical tables of one stack (host pointers; copied by pic_init).
 * The shapes follow the paper's Fig. 1 quantities; index order is
 * [material][spin][k-1] with spin 0 = majority (up), 1 = minority (down). */
typedef struct {
    int32_t n_mat;          /* 1..PIC_MAX_MAT */
    const float *v;         /* [n_mat][2][n_e] group velocity, nm/fs (> 0) */
    const double *tau_in;   /* [n_mat][2][n_e] inelastic lifetime, fs; +inf = none */
    const double *tau_el;   /* [n_mat] elastic lifetime, fs; +inf = none */
    const double *T;        /* [n_layers-1][2 dir][2 spin][n_e] interface
                               transmittance in [0,1]; dir 0 = towards +z
                               (layer l -> l+1), dir 1 = towards -z */
    const double *p0;       /* [n_mat] equilibrium polarisation P0 of Eq. eq_pol,
                               in [-1,1]; spin of secondary carriers */
} pic_tables;

/* Excitation pulse of one stack (Sec. III, particle number; Sec. V.A). */
typedef struct {
    int64_t n0;             /* carriers created over the pulse (>= 0) */
    double fwhm;            /* Gaussian FWHM, fs (> 0 when n0 > 0) */
    double t0;              /* pulse centre, fs (> 0); the pulse is truncated
                               symmetrically to [0, 2 t0] */
    double abs_len;         /* absorption length, nm: profile exp(-z/abs_len);
                               0 = homogeneous in the excited layers */
    uint32_t excite_mask;   /* bit l set: layer l is excited */
    double up_frac;         /* probability that a created carrier is spin up */
    int32_t e_mode;         /* 0: k uniform on 1..n_e; 1: k = k_mono[spin] */
    int32_t k_mono[2];      /* bins for e_mode 1 */
    /* Importance sampling of the births (PIC_F_WEIGHTS only; host, copied,
     * may be NULL): relative sampling densities of the birth cell
     * (cell_bias[n_cells] of the stack, > 0 on excited cells) and of the
     * birth bin (e_bias[n_e], > 0, e_mode 0).  A carrier is drawn from
     * q proportional to p * bias instead of the physical profile p and
     * carries the weight p/q (Eq. PIC: "adjusted to improve the
     * representation of less likely events"); NULL = q = p, weight 1. */
    const double *cell_bias;
    const double *e_bias;
} pic_pulse;

/* Device-resident bookkeeping, per stack (exact integer counts). */
typedef struct {
    uint64_t injected, inject_dropped, spawned, spawn_dropped, absorbed;
    uint64_t q_injected;    /* energy quanta (bins) created by the source */
    uint64_t q_bath;        /* quanta handed to the thermal bath (removal,
                               or the secondary's share without secondaries) */
    uint64_t q_dropped;     /* quanta of secondaries dropped at capacity */
    uint64_t iface_hits, iface_transmit, truncated;
    uint64_t particle_steps;/* live carriers advanced, summed over steps */
    uint64_t changed;       /* advanced carriers whose direction, energy, spin,
                               layer or liveness changed (records rewritten) */
    uint64_t eventful;      /* advanced carriers that scattered or met a layer
                               boundary or surface during the step */
} pic_ledger;

/* Device time of the library's kernels, per kind: 0 = source, 1 = step
 * (streaming pass), 2 = step with density deposit (streaming pass),
 * 3 = compaction, 4 = step (event pass and placement of secondaries);
 * pic_grad's replays: 5 = streaming pass, 6 = event pass, 7 = the rest
 * (source, compaction, flux potential, flush, lineage totals);
 * 8 = the fluxes derived by pic_moments and pic_weighted_moments;
 * 9 = the weighted densities (PIC_F_WEIGHTS). */
#define PIC_KERNEL_KINDS 10
typedef struct {
    int64_t launches[PIC_KERNEL_KINDS];
    double ms[PIC_KERNEL_KINDS];
} pic_kernel_times;

/* One particle slot as returned by pic_records (16 bytes). */
typedef struct {
    float z;
    float mu;
    uint32_t id;            /* low 32 bits of the carrier id */
    uint32_t packed;        /* k:8 | spin:1 | layer:4 | gen:8 | id_hi:11;
                               k = 0 marks a removed carrier */
} pic_record;

typedef struct pic_ctx pic_ctx;

/* Create a context with n_stacks independent stacks, each with its own
 * tables (tables[n_stacks]).  Derives every probability threshold on the
 * host in double precision, allocates the particle state (double-buffered
 * structure of arrays), histograms and scratch on the current CUDA device,
 * and uploads the tables.  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream); all later device work of the context is ordered on it.
 * On error *out is NULL and nothing stays allocated. */
pic_status pic_init(pic_ctx **out, const pic_params *p, const pic_stack_desc *stacks,
                    int n_stacks, const pic_tables *tables, void *cuda_stream);

/* Set the excitation of one stack (Sec. III, "Number of Particles"): the
 * source creates floor(n0 F(t_{h+1})) - floor(n0 F(t_h)) carriers in half
 * step h, F the normalised pulse CDF; positions follow the absorption
 * profile over the excited layers' cells, directions are isotropic.
 * Host-side only (uploads a schedule); call before stepping through the
 * pulse.  stack = -1 applies the same pulse to every stack. */
pic_status pic_excite(pic_ctx *ctx, int stack, const pic_pulse *pulse);

/* Advance every stack by n_steps Strang steps (Eq. strang).  Asynchronous
 * on the context stream; returns PIC_ERR_ARG if the steps would exceed
 * n_steps_max. */
pic_status pic_step(pic_ctx *ctx, int n_steps);

/* Moments of one stack (Eq. firstmoment).  n_dev (device, may be NULL):
 * uint32 [n_out][2][n_e][n_cells] live carriers per (spin, bin, cell) at
 * the end of each moment window.  J_dev (device, may be NULL): int32
 * [n_out][2][n_cells+1] net number of carriers of each spin that crossed
 * each cell face towards +z during the window (the time-integrated spin
 * flux; face f sits at z = f*dz); the window still running holds the
 * crossings so far.  The library does not count crossings one by one: it
 * derives these integers, exactly, from the densities at the ends of the
 * windows and the cells where carriers were created and removed (a kernel
 * pass on the device per call; one over the current state when a window is
 * running).  ledger_host (host, may be NULL).  Synchronises the context
 * stream; returns any pending device status. */
pic_status pic_moments(pic_ctx *ctx, int stack, uint32_t *n_dev, int32_t *J_dev,
                       pic_ledger *ledger_host);

/* One moment window of one stack (Eq. firstmoment), into caller-owned
 * buffers in host memory (pageable or pinned) or device memory: n_out (may
 * be NULL) receives uint32 [2][n_e][n_cells] and J_out (may be NULL) int32
 * [2][n_cells+1] of window `window` (0 <= window < n_out), the layouts of
 * one window of pic_moments; ledger_host (host, may be NULL) as there.  The
 * copy moves one window only, not the whole run.  A window not reached yet
 * holds zeros (densities) and the crossings so far (fluxes).  Synchronises
 * the context stream; PIC_ERR_ARG for a bad stack or window; returns any
 * pending device status. */
pic_status pic_moment_window(pic_ctx *ctx, int stack, int window, uint32_t *n_out,
                             int32_t *J_out, pic_ledger *ledger_host);

/* Generation map of one stack (Figs. 5(b) and 7(b),(d), Sec. V): g_dev
 * (device, caller-owned, overwritten) receives uint64 [n_out][n_cells], the
 * generation labels (1 for a primary, the parent's + 1 for a secondary,
 * saturating at 255) of the live carriers in each cell summed at the same
 * instants as the densities of pic_moments; divided by the densities summed
 * over spin and bin it gives the mean generation of each space-time cell.
 * Asynchronous on the context stream; PIC_ERR_ARG for a bad stack or a NULL
 * g_dev. */
pic_status pic_gen_moments(pic_ctx *ctx, int stack, uint64_t *g_dev);

/* Velocity moment of one stack behind the spin current of Eq. spincurrent
 * (Sec. V), for a context made with PIC_F_VELOCITY_MOMENTS (else
 * PIC_ERR_ARG): v_dev (device, caller-owned, overwritten) receives int64
 * [n_out][2][n_cells], the velocities along z, v(material, spin, k) * mu,
 * of the live carriers of each spin in each cell, summed at the same instants
 * as the densities of pic_moments.  Each product is taken in float32 and
 * counted as an integer number of 2^-32 nm/fs (truncated toward zero), so
 * the sums are exact; (v[t][0][c] - v[t][1][c]) / (2^32 dz) is the
 * spin-current density of cell c in carriers nm/fs per nm.  Asynchronous on
 * the context stream; PIC_ERR_ARG for a bad stack or a NULL v_dev. */
pic_status pic_vel_moments(pic_ctx *ctx, int stack, int64_t *v_dev);

/* Weighted moments of one stack (PIC_F_WEIGHTS; Eq. PIC, Sec. III.A): the
 * densities and fluxes of pic_moments with every carrier counted with its
 * weight w_i, in units of 2^-20 (weights are kept as integers of that unit,
 * so the sums are exact).  nw_dev (device, may be NULL): uint64
 * [n_out][2][n_e][n_cells]; Jw_dev (device, may be NULL): int64
 * [n_out][2][n_cells+1]; w_injected_host (host, may be NULL): the summed
 * weight of the carriers the source has created, the denominator of the
 * normalisation C = rho_exc / sum w_i.  Synchronises; PIC_ERR_ARG for a
 * context made without PIC_F_WEIGHTS or a bad stack. */
pic_status pic_weighted_moments(pic_ctx *ctx, int stack, uint64_t *nw_dev, int64_t *Jw_dev,
                                uint64_t *w_injected_host);

/* The weights (2^-20 units) of one stack's slots, in slot order (PIC_F_WEIGHTS).
 * host_out NULL: only the count is written to *n.  Synchronises. */
pic_status pic_weights(pic_ctx *ctx, int stack, uint32_t *host_out, int64_t *n);

/* Replace the weights of one stack's slots (PIC_F_WEIGHTS), n = the slot
 * count, every weight > 0; pic_set_records gives loaded carriers weight 1
 * (2^20).  For the weighted fluxes of the running window the carriers count
 * as removed with their old weights and created with the new ones. */
pic_status pic_set_weights(pic_ctx *ctx, int stack, const uint32_t *host_in, int64_t n);

/* Score-function (likelihood-ratio) gradient of a linear functional of the
 * moments with respect to the lifetime and transmittance tables of every
 * stack.  grad_n_dev: float [n_stacks][n_out][2][n_e][n_cells_max] weights
 * of the densities; grad_J_dev: float [n_stacks][n_out][2][n_cells_max+1]
 * weights of the fluxes (either may be NULL = zero).  Outputs (device,
 * double, overwritten): grad_tau_dev [n_stacks][n_mat][2][n_e] (d/d tau_in),
 * grad_T_dev [n_stacks][PIC_MAX_LAYERS-1][2][2][n_e] (d/d T).  Replays the
 * forward trajectories from the Philox counters; the forward pass stores
 * nothing.  Requires a context that was stepped from an empty or loaded
 * initial state with no intervening pic_set_records. */
pic_status pic_grad(pic_ctx *ctx, const float *grad_n_dev, const float *grad_J_dev,
                    double *grad_tau_dev, double *grad_T_dev);

/* Copy the particle slots of one stack to host memory.  If host_out is NULL
 * only the slot count is written to *n.  Synchronises. */
pic_status pic_records(pic_ctx *ctx, int stack, pic_record *host_out, int64_t *n);

/* Replace the particle slots of one stack (test set-up and resume from a
 * saved state).  next_id is the id given to the next created carrier.
 * Every record must have k in 0..n_e, a layer of the stack, a finite
 * non-zero mu in [-1, 1] and z inside its layer (edges included); otherwise
 * PIC_ERR_ARG and nothing changes.  For the fluxes of the running window the
 * replaced carriers count as removed and the loaded ones as created where
 * they are (no crossing is counted for either). */
pic_status pic_set_records(pic_ctx *ctx, int stack, const pic_record *host_in,
                           int64_t n, uint64_t next_id);

/* Checkpoint of a context's evolving state into a caller-owned host buffer:
 * the step index, every stack's slots (records and, with PIC_F_WEIGHTS,
 * weights), counters and ledger, the moment windows (densities, births and
 * removals, generation and velocity sums, weighted sums) and the initial
 * records pic_grad replays from, behind a header with a fingerprint of the
 * parameters that define the run (launch-configuration fields excluded),
 * the stacks, their tables and their excitation.  Storage of the superparticle
 * state between runs is the paper's restart of the PIC dynamics; the format
 * is this library's own.  buf NULL: *bytes receives the size needed.
 * *bytes smaller than that: PIC_ERR_ARG (and *bytes = the size).
 * Synchronises; returns any pending device status first. */
pic_status pic_save(pic_ctx *ctx, void *buf, size_t *bytes);

/* Restore a checkpoint of pic_save into a context created with the same
 * parameters, stacks and tables and given the same excitation (pic_excite)
 * as the saved one; a different fingerprint, size or a corrupt header is
 * PIC_ERR_ARG and changes nothing.  Stepping on from the restored state
 * gives the results of the uninterrupted run bit for bit (the random
 * streams are keyed by step and slot). */
pic_status pic_load(pic_ctx *ctx, const void *buf, size_t bytes);

/* Wait for the context stream and return the pending device status. */
pic_status pic_sync(pic_ctx *ctx);

/* Host-only (no device work): the integer tables pic_init and pic_excite
 * derive for one stack.  P_thr, Q_thr: uint32 [n_mat][2][n_e]; T_thr:
 * uint32 [n_layers-1][2][2][n_e]; P0_thr: uint32 [n_mat]; up_thr: uint32;
 * inj_counts: int64 [2*n_steps_max] carriers created per half step.  Any
 * output pointer may be NULL. */
pic_status pic_derive_tables(const pic_params *p, const pic_stack_desc *stack,
                             const pic_tables *tables, const pic_pulse *pulse,
                             uint32_t *P_thr, uint32_t *Q_thr, uint32_t *T_thr,
                             uint32_t *P0_thr, uint32_t *up_thr, int64_t *inj_counts);

/* Sizes of one stack's outputs. */
pic_status pic_shape(const pic_ctx *ctx, int stack, int32_t *n_cells, int32_t *n_out,
                     int32_t *step);

/* Start (enable = 1) or stop (0) recording CUDA events around every kernel
 * launch on the context stream; starting clears earlier records. */
pic_status pic_profile(pic_ctx *ctx, int enable);

/* Sum the recorded kernel times (synchronises). */
pic_status pic_profile_read(pic_ctx *ctx, pic_kernel_times *out);

/* Stable removal of dead slots (k = 0) from particle arrays the caller owns,
 * without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as an
 * application whose device memory belongs entirely to its own allocator or
 * pool, or a latency-critical loop that must not allocate.  It runs the same
 * compaction kernel as pic_step, with that kernel's scratch (look-back words
 * for up to 4096 blocks, counters, control block: about 33 KB) held in a
 * static device array that every GPU which loads the library keeps until
 * the process exits.
 *   z, mu, id, packed (device, read): n slots in the pic_record field layout;
 *     16-byte aligned and readable up to round_up(n, 4) elements.
 *   z_out, mu_out, id_out, packed_out (device, written): the live slots in
 *     their original order; each must hold n elements and must not overlap
 *     the inputs.
 *   n_alive (host, written): number of live slots.
 *   cuda_stream: cudaStream_t the work is ordered on; the call synchronises it.
 * n must be below 2^30 (the look-back words carry 30-bit counts); larger n,
 * NULL pointers or a misaligned input array return PIC_ERR_ARG.  Every
 * call looks up the array's device address on the current device (so a
 * device reset between calls is harmless).  Calls share the array: each call
 * resets the part that must start from zero, and calls whose kernels overlap
 * on one GPU (different streams or host threads) race on it. */
pic_status pic_compact_static(const float *z, const float *mu, const uint32_t *id,
                              const uint32_t *packed, int64_t n, float *z_out, float *mu_out,
                              uint32_t *id_out, uint32_t *packed_out, int64_t *n_alive,
                              void *cuda_stream);

/* The launch configuration of a context's kernels. */
pic_status pic_launch_config(const pic_ctx *ctx, pic_launch_info *out);

/* One candidate launch configuration timed by pic_autotune. */
typedef struct {
    int32_t blocks_per_sm;  /* resident blocks per SM of the streaming pass */
    int32_t ring_stages;    /* its bulk-copy ring depth */
    int32_t hist_mode;      /* density deposit: 0 shared atomics, 1 warp-aggregated */
    int32_t chosen;         /* 1 for the configuration the context keeps */
    double ns_per_particle_step;  /* device time of the trial / carriers advanced */
    int32_t consumer_warps; /* warps of the streaming pass on the carriers (4 or 8),
                               i.e. 8 or 4 consecutive slots per thread */
    int32_t event_pass;     /* 0 the general step inside the streaming pass, 1 separate */
} pic_tune_entry;

/* Time candidate launch configurations of the step kernels on the running
 * simulation and keep the fastest.  Each candidate advances every stack by
 * trial_steps ordinary steps (results do not depend on the launch
 * configuration: the slot order and every random word are fixed by the
 * run), timed with CUDA events on the context stream and divided by the
 * carriers advanced.  Candidates: 8 or 4 consumer warps per block of the
 * streaming pass (4 or 8 slots per thread), 1 to 6 (8 with four warps)
 * resident blocks per SM, ring depth 2, 3, 4, 6 or 8 where it fits, both
 * deposit modes when the trial contains density steps, and (eight consumer
 * warps, a single stack) the general step inside the streaming pass or in a
 * separate pass.  entries (host, may be NULL): up to max_entries results in
 * the order tried; *n_entries (may be NULL): their number.  Needs steps left:
 * up to 200 * trial_steps.  Synchronises. */
pic_status pic_autotune(pic_ctx *ctx, int trial_steps, pic_tune_entry *entries,
                        int max_entries, int *n_entries);

/* Device kernels launched by the last pic_step call (for accounting). */
int64_t pic_launch_count(const pic_ctx *ctx);

/* Free every resource of the context (NULL is allowed). */
void pic_destroy(pic_ctx *ctx);

/* Text of the last error on this context (never NULL). */
const char *pic_last_error(const pic_ctx *ctx);

/* Name of a status code. */
const char *pic_status_string(pic_status s);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
