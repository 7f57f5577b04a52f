/*
 * CPU oracle for the spin-dependent particle-in-cell (PIC) hot-electron
 * step of Nenno, Rethfeld and Schneider, "Particle-in-cell simulation of
 * ultrafast hot-carrier transport in Fe/Au heterostructures" (arXiv:1807.04733).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, scalar implementation of
 * the method, written to be checked against the paper by eye.  It is used by
 * the test-suite, by the smoke check and by the timed CPU baseline of the
 * benchmark.  It shares no code, header, table or constant generator with the
 * CUDA library; the only thing both consume is the input generator module.
 *
 * Precision: particle state (z, mu) is float32, as the workload definition
 * fixes FP32 superparticles; every table (probabilities, thresholds,
 * injection counts) is derived here in double precision.  Build with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_LAYERS 16
#define OR_MAX_HITS 8          /* boundary hits per half flight */

/* flags (same bit values as the library's) */
#define OR_F_DETERMINISTIC   1u
#define OR_F_NO_SECONDARIES  2u
#define OR_F_TRANSPARENT     4u
#define OR_F_LOWEST_BIN_ANY  8u
#define OR_F_STRICT_CAPACITY 16u
#define OR_F_VELOCITY        32u  /* also sum the velocities v*mu per (time, spin, cell) */
#define OR_F_WEIGHTS         64u  /* superparticle weights w_i of Eq. PIC (Sec. III.A) */
/* Oracle-only: every random word of a carrier is keyed by its lineage (a
 * primary by its birth half step and index, a secondary by a hash of its
 * parent's key and its birth step) instead of by its slot, so that a
 * decision that flips in a perturbed run changes only that carrier's line:
 * common random numbers for central finite differences.  The trajectories
 * have the same law as with slot keys (every decision still draws a fresh
 * word); the library keys by slot. */
#define OR_F_LINEAGE_KEYS   128u

typedef struct {
    float z;          /* depth, nm */
    float mu;         /* cos(theta) */
    uint32_t id;      /* low 32 bits of the carrier id */
    uint32_t packed;  /* k:8 | spin:1 | layer:4 | gen:8 | id_hi:11 */
} or_rec;

typedef struct {
    int32_t n_e;
    float dt, dz;
    uint64_t seed;
    uint32_t stack_index;
    uint32_t flags;
    int64_t capacity;
    int32_t compact_every, moment_every, n_steps_max;
    int32_t n_layers;
    int32_t layer_cells[OR_MAX_LAYERS];
    int32_t layer_mat[OR_MAX_LAYERS];
    int32_t n_mat;
    const float *v;        /* [n_mat][2][n_e] */
    const double *tau_in;  /* [n_mat][2][n_e] */
    const double *tau_el;  /* [n_mat] */
    const double *T;       /* [n_layers-1][2][2][n_e] */
    const double *p0;      /* [n_mat] */
    int64_t n0;
    double fwhm, t0, abs_len;
    uint32_t excite_mask;
    double up_frac;
    int32_t e_mode;
    int32_t k_mono[2];
    /* importance sampling of the source (OR_F_WEIGHTS): relative sampling
     * densities of the birth cell ([n_cells] of the stack; only excited
     * cells matter) and of the birth bin ([n_e], e_mode 0); NULL = none */
    const double *cell_bias;
    const double *e_bias;
} or_config;

typedef struct {
    uint64_t injected, inject_dropped, spawned, spawn_dropped, absorbed;
    uint64_t q_injected, q_bath, q_dropped;
    uint64_t iface_hits, iface_transmit, truncated, particle_steps;
    uint64_t changed;     /* advanced carriers whose mu or packed word changed */
    uint64_t eventful;    /* advanced carriers that scattered or met a boundary */
} or_ledger;

typedef struct or_sim or_sim;

int  or_create(const or_config *cfg, or_sim **out);
void or_destroy(or_sim *s);
int  or_step(or_sim *s, int n_steps);             /* 0 ok, 3 capacity (strict) */
int64_t or_n_slots(const or_sim *s);
void or_records(const or_sim *s, or_rec *out);     /* n_slots records */
int  or_set_records(or_sim *s, const or_rec *in, int64_t n, uint64_t next_id);
void or_moments(const or_sim *s, uint32_t *n_out, int32_t *J_out, or_ledger *led);
/* generation label summed per [n_out][n_cells] (Figs. 5(b), 7(b),(d)) */
void or_gen_moments(const or_sim *s, uint64_t *g_out);
/* velocity moment per [n_out][2][n_cells] (OR_F_VELOCITY; Eq. spincurrent) */
void or_vel_moments(const or_sim *s, int64_t *v_out);
/* Superparticle weights (OR_F_WEIGHTS; Eq. PIC, Sec. III.A), in units of
 * 2^-20: the weighted densities [n_out][2][n_e][n_cells] and fluxes
 * [n_out][2][n_cells+1] (the counts with every carrier counted w times),
 * and the summed weight of the carriers the source created. */
void or_weighted_moments(const or_sim *s, uint64_t *nw_out, int64_t *Jw_out, uint64_t *w_injected);
void or_weights(const or_sim *s, uint32_t *w_out);                 /* n_slots weights */
int  or_set_weights(or_sim *s, const uint32_t *w, int64_t n);     /* after or_set_records */
int32_t or_n_cells(const or_sim *s);
int32_t or_n_out(const or_sim *s);
int32_t or_step_index(const or_sim *s);
void or_set_step(or_sim *s, int32_t step);          /* position in time (Philox counter) */
uint64_t or_next_id(const or_sim *s);
/* derived tables, for the test that the library derives the same ones */
void or_tables(const or_sim *s, uint32_t *P_thr, uint32_t *Q_thr, uint32_t *T_thr,
               uint32_t *P0_thr, uint32_t *up_thr, int64_t *inj_counts);
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* One carrier in slot `slot` advanced by one step (at the sim's step index,
 * or_set_step) on its own: *out receives its record; if it creates a
 * secondary and room != 0, *sec receives the secondary (its id fields are
 * not meaningful; the id counter is left untouched) and 1 is returned.  Densities are not deposited;
 * fluxes and the ledger of the sim are updated.  The sim's own records are
 * left as they were (needs capacity >= 1). */
int or_advance_one(or_sim *s, const or_rec *in, int64_t slot, int room, or_rec *out, or_rec *sec);

/* Score-function gradient of O = sum gn*n + sum gJ*J (gn: [n_out][2][n_e]
 * [n_cells], gJ: [n_out][2][n_cells+1], the moment layouts) over n_steps
 * steps from the initial records (ids below next_id), with respect to
 * tau_in ([n_mat][2][n_e]) and T ([n_layers-1][2][2][n_e]).  mag_*: the sums
 * of |score| (|total| + |earned|), a scale for rounding comparisons.
 * Returns 0, or non-zero on bad input. */
int or_grad(const or_config *cfg, const or_rec *init, int64_t n_init, uint64_t next_id,
            int n_steps, const float *gn, const float *gJ, double *g_tau, double *g_T,
            double *mag_tau, double *mag_T);

#ifdef __cplusplus
}
#endif
#endif
