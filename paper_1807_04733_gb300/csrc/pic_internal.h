// Internal structures of the GB300 PIC library (not part of the C-ABI).
//
// Data layout in HBM
//   particles : structure of arrays, two buffers (ping-pong for compaction):
//               z[f32], mu[f32], id[u32], packed[u32], each of length
//               sum_s round_up(capacity_s, TILE); stack s owns slots
//               [base_s, base_s + capacity_s).  One thread moves four
//               consecutive slots with one 128-bit load/store per array.
//   staging   : float4 per slot (z_end, mu, packed bits, z_spawn): the
//               secondary of the carrier at that position, before its final
//               place is known, flagged by one bit per slot in spawn_bits.
//   tables    : per stack, per layer: {v, P_thr, Q_thr} (16 B) for
//               [layer][spin][k], the interface thresholds, P0 per layer;
//               the streaming pass's {v, P_thr, lo, hi} padded to 2^kb bins
//               per (layer, spin) so that the packed word indexes it directly.
//   moments   : uint32 densities and int32 fluxes per output window; the
//               births minus removals of carriers per window and cell, from
//               which the fluxes are derived (see k_flux in pic_kernels.cu).
#pragma once
#include <cstdint>

#include "pic.h"

namespace pic {

constexpr int TPB = 256;            // threads per block of the streaming kernels
constexpr int VEC = 4;              // particles per thread per tile (128-bit)
constexpr int TILE = TPB * VEC;     // particles per tile
constexpr int LEDGER_N = 14;        // fields of pic_ledger

// ledger field indices (order of pic_ledger)
enum {
    L_INJECTED, L_INJECT_DROPPED, L_SPAWNED, L_SPAWN_DROPPED, L_ABSORBED,
    L_Q_INJECTED, L_Q_BATH, L_Q_DROPPED, L_IFACE_HITS, L_IFACE_TRANSMIT,
    L_TRUNCATED, L_PARTICLE_STEPS, L_CHANGED, L_EVENTFUL
};

// Philox counter layout: ctr = {x, x_hi | global stack << 16, step, substream}
// with x the new carrier's id for the source draws and the drawing carrier's
// slot (within its stack) for every other word
enum : uint32_t {
    SUB_INJ = 0x300u,    // + j: source draws (id)
    SUB_TEST = 0x400u,   // scattering test: x = slot / 4, word slot % 4
    SUB_EVT = 0x500u,    // event words of a carrier that scatters (slot)
    SUB_SEC = 0x501u,    // its secondary's spin and direction (slot)
    SUB_IF = 0x600u,     // + 16*half + hit: boundary draws of a flight (slot)
    SUB_SIF = 0x700u,    // + hit: the secondary's flight (the parent's slot)
};

struct TabEnt {          // one (layer, spin, k) entry
    float v;             // nm/fs
    uint32_t P;          // scatter iff x0 < P   (P = floor(p 2^32))
    uint32_t Q;          // inelastic iff x1 < Q
    uint32_t pad;
};

struct FastEnt {         // the common path's (layer, spin, k) entry
    float v;             // nm/fs
    uint32_t P;          // scatter iff test word < P
    float lo, hi;        // edges of the layer, nm
};
// The streaming pass's table holds 2^kb entries per (layer, spin), kb the
// smallest power of two above n_e: entry ((layer * 2 + spin) << kb) + k, read
// with the index (pk & kmask) | ((pk >> (8 - kb)) & hmask) of the packed word
// pk = k:8 | spin:1 | layer:4 | ....  Entries k = 0 (a removed carrier) and
// k > n_e hold the inert entry {v = 0, P = 0, lo = -inf, hi = +inf}: such a
// slot never moves, scatters or meets a boundary.

struct AdjEnt {          // d log P / d tau_in of the outcomes of one (layer, spin, k) entry
    double noscat;       // no scattering in the step
    double scat_el;      // scattering, elastic channel
    double scat_inel;    // scattering, inelastic channel
    double pad;
};

struct DevStack {        // immutable per-stack description (device copy)
    int32_t n_layers, n_cells, tab_n, T_n;
    float edge[PIC_MAX_LAYERS + 1];
    uint32_t p0_thr[PIC_MAX_LAYERS];    // per layer
    int64_t base, cap;                  // slot range
    int64_t n_off, J_off;               // offsets in the moment arrays
    int64_t ent_off, T_off;             // offsets in the table arrays
    int64_t fent_off; int32_t ftab_n;   // padded streaming-pass table
    int64_t cdf_off; int32_t n_cdf;     // source profile
    uint32_t up_thr;
    int32_t e_mode, k_mono0, k_mono1;
    int32_t has_ebias;                  // weights: births drawn from the biased bin CDF
    int64_t inj_off;                    // source schedule, 2*n_steps_max
    int64_t id_off, n_ids;              // adjoint: range of the id-indexed arrays
};

struct DevCounters {     // mutable per stack
    unsigned long long n_slots, next_id, spawn_total, alive_total;
    unsigned long long led[LEDGER_N];
    unsigned long long live;   // live carriers (k > 0) among the slots
    unsigned long long w_injected;   // weights (2^-20 units) of the carriers created
};

struct DevCtl {
    unsigned int status;     // first error code (0 = ok)
    unsigned int epoch;      // tag of the look-back status words
    unsigned int done;       // blocks finished in the current launch
    unsigned int cur;        // current particle buffer (0/1)
    unsigned int timeout_where;
    unsigned int step;       // time step of graph-replayed steps
    unsigned int bar_count;  // grid barrier of the persistent kernel: arrivals,
    unsigned int bar_gen;    //   and its generation
};

struct Args {            // everything a kernel needs, passed by value
    const DevStack *stacks;
    int n_stacks;
    const TabEnt *ent;
    const FastEnt *fent;                     // padded: see FastEnt
    uint32_t kmask, hmask;                   // fast-table index of a packed word:
    int kshr, kb;                            //   (pk & kmask) | ((pk >> kshr) & hmask)
    const uint32_t *T_thr;
    const uint32_t *cdf_thr;
    const int32_t *cdf_cell;
    const int32_t *cdf_layer;
    const long long *inj;
    float *z[2];
    // mu and packed of slot i at mu[b][i * mp_stride] and pk[b][i * mp_stride]:
    // a context keeps them interleaved (stride 2, pk = mu + 1), so that an
    // event updates one 32-byte sector for both; the allocation-free
    // compaction takes separate arrays (stride 1)
    float *mu[2];
    uint32_t *id[2];
    uint32_t *pk[2];
    int mp_stride;
    float4 *stage;
    unsigned long long *status;      // one look-back word per block
    uint32_t *n_hist;
    // generation labels summed per [stack][n_out][n_cells], at n_off / (2 n_e)
    unsigned long long *g_hist;
    int32_t *J_hist;
    // births minus removals of carriers per [stack][n_out][2][n_cells+1]
    // (J layout, last entry unused): the fluxes are derived from these and
    // the densities
    int32_t *bd_hist;
    DevCounters *cnt;
    DevCtl *ctl;
    uint32_t seed_lo, seed_hi;
    int stack_base;                          // global index of stack 0 (Philox counters)
    uint32_t rk0[10], rk1[10];               // Philox round keys (key + r * Weyl)
    float half_dt, dz, inv_dz;
    int dz_pow2;
    uint32_t flags;
    int n_e;
    int moment_every;
    int compact_every;
    uint32_t step;                           // time step (plain launches)
    const unsigned int *step_dev;            // graph replay: the step is read here
    int bump_step;                           // this kernel's last block advances *step_dev
    int tab_max, T_max, nbin_max, jbin_max;  // shared-memory sizing
    int ftab_max;                            // entries of the padded fast table
    int gbin_max;                            // cells of the widest stack (generation sums)
    unsigned int spin_limit;                 // bound of every device-side wait
    int ring;                                // tiles in the streaming pass's copy ring
    int grid_fast;                           // the streaming pass's grid (read by k_event, k_place)
    uint32_t *spawn_bits;                    // one bit per position: secondary staged
    // superparticle weights (PIC_F_WEIGHTS; null otherwise): per slot in
    // 2^-20 units, both buffers; the source's importance ratios p/q per
    // birth-cell entry (cdf_off indexing) and per bin ([stack][n_e]), with
    // the biased bin thresholds; the weighted densities (n_hist layout),
    // births minus removals and fluxes (J layout)
    uint32_t *w[2];
    const double *wcell, *wbin;
    const uint32_t *kthr;
    unsigned long long *nhw;
    long long *bdw, *Jw;
    float4 *qrec;                            // eventful carriers: z, mu, packed, position
    uint32_t *qcnt;                          // queue length per fast block
    uint32_t *fspawn;                        // secondaries staged per fast block
    // adjoint replay (ADJ = 1, 2); unused by the forward step.  Rewards are
    // fixed-point integers in units of 2^-F (the weights quantised to int32):
    // sums are exact and independent of their order.
    long long *acc[2];                       // per slot: own reward so far (pass 1),
                                             // reward still to come (pass 2)
    long long *tot;                          // per id: own reward, then lineage total
    unsigned long long *parent;              // per id: index of the parent's entry
    uint8_t *gen;                            // per id: lineage depth (0 = no parent)
    unsigned int *gen_max;                   // largest depth created
    const AdjEnt *aent;                      // scores, ent indexing
    const double2 *aT;                       // scores (transmit, reflect), T_thr indexing
    double *g_ent;                           // gradient, ent indexing
    double *g_T;                             // gradient, T_thr indexing
    const int32_t *gn;                       // density weights [stack][n_out][2][n_e][ncm]
    const long long *gpot;                   // flux potential [stack][n_out][2][ncm]
    uint32_t *stage_l;                       // pass 2: start layer of a staged secondary
    int n_out, ncm;                          // moment windows, cells of the widest stack
    double inv_q;                            // 2^-F: reward units to weight units
    // velocity moment [stack][n_out][2][n_cells] at n_off / n_e, units of
    // 2^-32 nm/fs (PIC_F_VELOCITY_MOMENTS)
    long long *v_hist;
};

// reason of the last failure of a call without a context (pic_capi.cu);
// returned by pic_last_error(NULL)
void pic_set_static_error(const char *msg);

// host-side launchers (pic_kernels.cu)
struct LaunchCfg {
    int grid_fast, grid_fast_dep;          // streaming pass (without / with density deposit)
    int nw_fast, nw_fast_dep;              // its consumer warps per block (4 or 8)
    int grid_slow, grid_slow_dep;          // k_event
    int grid_place, grid_place_dep;        // k_place
    int grid_compact, grid_inject;
    int ring_fast, ring_fast_dep;
    size_t smem_fast, smem_fast_dep, smem_slow, smem_slow_dep, smem_place, smem_place_dep;
    // the fused streaming pass (plain steps of a single stack; grid 0: not used)
    int grid_fused, ring_fused;
    size_t smem_fused;
};
// blocks_per_sm, ring, nw: 0 = chosen from the occupancy
cudaError_t configure(const Args &a, int blocks_per_sm, int ring, int hist_mode, int nw,
                      LaunchCfg *cfg);
cudaError_t launch_inject(const Args &a, const LaunchCfg &c, int half, bool deposit,
                          cudaStream_t s);
cudaError_t launch_fast(const Args &a, const LaunchCfg &c, bool deterministic, bool deposit,
                        int hist_mode, cudaStream_t s);
cudaError_t launch_slow(const Args &a, const LaunchCfg &c, bool deterministic, bool deposit,
                        cudaStream_t s);
// a plain step in the fused form: the streaming pass with its event warps
// (Args a), then the placement (Args b, which may advance the step counter)
cudaError_t launch_fused(const Args &a, const LaunchCfg &c, bool deterministic, cudaStream_t s);
cudaError_t launch_place_fused(const Args &b, const LaunchCfg &c, bool deterministic,
                               cudaStream_t s);
cudaError_t launch_compact(const Args &a, const LaunchCfg &c, cudaStream_t s);
// live carriers of stacks [s0, s1) counted per (spin, cell) into out (int32,
// per stack at out + stack_off(s) ...): mode 0 = the windows' births-minus-
// removals histogram of window `win` (sign +1 or -1), mode 1 = a scratch
// [stack][2][ncm+1]
cudaError_t launch_state_hist(const Args &a, int s0, int s1, int mode, int win, int sign,
                              int32_t *scratch, int ncm, cudaStream_t st);
// the same, each carrier counted with its weight (births-minus-removals
// histogram bdw, or a scratch [stack][2][ncm+1] of int64)
cudaError_t launch_state_hist_w(const Args &a, int s0, int s1, int mode, int win, int sign,
                                long long *scratch, int ncm, cudaStream_t st);
// weighted densities of the density step just finished (PIC_F_WEIGHTS)
cudaError_t launch_wdep(const Args &a, const LaunchCfg &c, cudaStream_t st);
// fluxes of windows [w0, w1) of every stack from the densities and the
// births-minus-removals histograms; window w_now (unfinished) takes its end
// counts from `now` [stack][2][ncm+1] (the current state) instead
cudaError_t launch_flux(const Args &a, int w0, int w1, int w_now, const int32_t *now, int ncm,
                        cudaStream_t st);
// the weighted fluxes Jw from nhw, bdw (and `now` [stack][2][ncm+1] int64)
cudaError_t launch_flux_w(const Args &a, int w0, int w1, int w_now, const long long *now, int ncm,
                          cudaStream_t st);
// set the device step counter read by graph-replayed steps
cudaError_t launch_set_step(DevCtl *ctl, unsigned int step, cudaStream_t s);
// the persistent kernel: n_steps whole steps of every stack in one cooperative
// launch (the step read from and advanced in device memory)
struct PersistCfg {
    int grid = 0, ring = 0;
    size_t smem = 0;
    bool wsm = false;        // weighted densities privatised in shared memory
    bool ok = false;
};
cudaError_t configure_persistent(const Args &a, bool det, PersistCfg *pc);
cudaError_t launch_persistent(const Args &a, const PersistCfg &pc, bool det, int n_steps,
                              cudaStream_t s);

// adjoint replay (pic_adjoint.cu); pass = 1 or 2
cudaError_t configure_adjoint(const Args &a, int pass, LaunchCfg *cfg);
cudaError_t launch_inject_adj(const Args &a, const LaunchCfg &c, int pass, int half,
                              bool deposit, cudaStream_t s);
cudaError_t launch_fast_adj(const Args &a, const LaunchCfg &c, int pass, bool deterministic,
                            bool deposit, cudaStream_t s);
cudaError_t launch_slow_adj(const Args &a, const LaunchCfg &c, int pass, bool deterministic,
                            bool deposit, cudaStream_t s);
cudaError_t launch_compact_adj(const Args &a, const LaunchCfg &c, int pass, cudaStream_t s);
// largest |x| of n floats, as its bit pattern (non-negative floats order as
// their bits); NaN or infinity give 0x7F800000 or more
cudaError_t launch_absmax(const float *x, long long n, unsigned int *out, cudaStream_t s);
// density weights quantised: q[i] = rint(gn[i] * 2^F)
cudaError_t launch_quantize(const float *gn, long long n, int32_t *q, double scale, cudaStream_t s);
// flux potential from the flux weights gJ [stack][n_out][2][ncm+1], quantised
cudaError_t launch_flux_potential(const Args &a, const float *gJ, long long *gpot, int rows,
                                  double scale, cudaStream_t s);
// start of a pass: the double of every loaded carrier (0, or its lineage total)
cudaError_t launch_init_acc(const Args &a, const LaunchCfg &c, int pass, cudaStream_t s);
// pass 1 end: own reward of every carrier still in a slot
cudaError_t launch_flush_own(const Args &a, const LaunchCfg &c, cudaStream_t s);
// lineage totals of generation g added to their parents
cudaError_t launch_lineage(const Args &a, const LaunchCfg &c, long long n_ids, int g,
                           cudaStream_t s);

}  // namespace pic
