/*
 * CPU oracle for the spin-dependent PIC hot-electron step (arXiv:1807.04733).
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, by the smoke check and by the
 * benchmark's CPU-baseline leg.  Never part of the product path.
 *
 * One time step follows the Strang splitting of Eq. strang (Sec. III.A):
 *
 *   Source(dt/2) -> Transport(dt/2) -> Scattering(dt) -> Transport(dt/2)
 *   -> Source(dt/2)
 *
 * with the superparticle rules of Sec. III:
 *   - particle number: carriers are created by a Gaussian pulse at the start
 *     and the end of every step (Sec. III, "Number of Particles");
 *   - transport: dz/dt = v_sigma(E) cos(theta); full reflection at the vacuum
 *     surfaces; stochastic transmission with probability T at an interface
 *     (Sec. III, transport part);
 *   - scattering: Monte-Carlo test against tau_eff of Eq. lifetimes within dt;
 *     elastic events redraw the direction and keep E and spin (Eq. split_w,
 *     Eq. elastic_scattering); inelastic events pick the final energy
 *     uniformly below the initial one (Eq. inelastic_collision) and lift a
 *     secondary whose spin follows the equilibrium polarisation P0
 *     (Eq. eq_pol); a lowest-bin carrier that scatters inelastically is
 *     removed (Sec. III, scattering part);
 *   - moments (Eq. firstmoment): spin- and energy-resolved densities per cell
 *     and the net spin-resolved particle flux through every cell face.
 *
 * Readings of points the paper leaves open are the ones listed in the design
 * notes (energy split k' ~ U{1..k-1} with the secondary taking k - k';
 * direction kept on transmission and mirrored on reflection; the flux as a
 * net crossing count; thresholds floor(p * 2^32) compared with Philox words).
 *
 * Processing order: particles in slot order; a secondary takes its second
 * half flight as soon as it is created and is appended after the slots that
 * existed at the start of the step, in parent order; dead slots stay until
 * the stable compaction every `compact_every` steps.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- Philox4x32-10 (Salmon et al., SC'11, "Parallel random numbers: as
 * easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies with the round
 * multipliers below; the key is bumped by the Weyl constants between rounds. */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PH_W0; k1 += PH_W1; }
        uint64_t p0 = (uint64_t)PH_M0 * c0;
        uint64_t p1 = (uint64_t)PH_M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* substreams: the fourth counter word.  The source draws are keyed by the
 * new carrier's id; every other word by the slot of the carrier that draws
 * it (one carrier per slot and step, so every decision gets a fresh word). */
#define SUB_INJ  0x300u   /* + j             : source draws (id) */
#define SUB_TEST 0x400u   /* scattering test: slot group of four, one word each */
#define SUB_EVT  0x500u   /* event words of a carrier that scatters (slot) */
#define SUB_SEC  0x501u   /* its secondary's spin and direction (slot) */
#define SUB_IF   0x600u   /* + 16*half + hit : boundary draws of a flight (slot) */
#define SUB_SIF  0x700u   /* + hit           : the secondary's flight (parent's slot) */

/* ---- packed word: k:8 | spin:1 | layer:4 | gen:8 | id_hi:11 ---- */
#define PK_K(w)     ((w) & 0xFFu)
#define PK_S(w)     (((w) >> 8) & 1u)
#define PK_L(w)     (((w) >> 9) & 0xFu)
#define PK_G(w)     (((w) >> 13) & 0xFFu)
#define PK_E(w)     ((w) >> 21)
static uint32_t pk(uint32_t k, uint32_t s, uint32_t l, uint32_t g, uint32_t e)
{
    return k | (s << 8) | (l << 9) | (g << 13) | (e << 21);
}

/* State of the adjoint replay (or_grad).  Pass 1 sums every carrier's own
 * reward (the weights of the densities it is counted in and of the faces it
 * crosses) and records its parent; pass 2 weights the score of every random
 * decision of a carrier by that carrier's reward-to-go. */
typedef struct {
    int pass;                     /* 1 or 2 */
    const float *gn;              /* [n_out][2][n_e][n_cells] */
    const float *gJ;              /* [n_out][2][n_cells+1] */
    uint64_t n_ids;               /* size of the id-indexed arrays */
    double *own;                  /* pass 1: own reward; then lineage total */
    double *acc;                  /* pass 2: rewards and child totals so far */
    uint64_t *parent;             /* UINT64_MAX: no parent */
    /* d log p / d theta of each outcome, per table entry */
    double *s_noscat, *s_scat, *s_el, *s_inel;   /* [n_mat][2][n_e], d/d tau_in */
    double *s_tr, *s_rf;                         /* [n_if][2][2][n_e], d/d T */
    double *g_tau, *g_T, *m_tau, *m_T;           /* sums of score x R and |score| x |R| */
    double R, Rmag;               /* reward-to-go of the carrier being advanced */
    int buffering, nbuf;          /* scores of a secondary wait for its id */
    int buf_T[OR_MAX_HITS + 1], buf_bin[OR_MAX_HITS + 1];
    double buf_s[OR_MAX_HITS + 1];
} or_adj;

struct or_sim {
    or_config cfg;
    or_adj *adj;                  /* NULL: plain forward run */
    /* owned copies of the physical tables */
    float *v; double *tau_in, *tau_el, *T, *p0;
    /* geometry */
    float edge[OR_MAX_LAYERS + 1];
    int32_t n_cells;
    /* derived thresholds */
    uint32_t *P_thr, *Q_thr, *T_thr, *P0_thr, up_thr;
    int32_t n_cdf; int32_t *cdf_cell, *cdf_layer; uint32_t *cdf_thr;
    int64_t *inj;                 /* per half step */
    /* particles */
    or_rec *recs; int64_t n_slots; uint64_t next_id; uint32_t step;
    /* superparticle weights (OR_F_WEIGHTS), units of 2^-20 per slot, and
     * the importance-sampling ratios p/q of the source: per entry of the
     * birth-cell table and per bin */
    uint32_t *wq; double *wcell, *wbin; uint32_t *kthr; int has_ebias;
    uint64_t *lkey;               /* OR_F_LINEAGE_KEYS: the random-stream key per slot */
    uint64_t *nhw; int64_t *Jhw; uint64_t w_injected;
    /* moments */
    int32_t n_out; uint32_t *nh; int32_t *Jh;
    uint64_t *gh;                 /* generation label summed per (output time, cell) */
    int64_t *vh;                  /* velocity v*mu summed per (output time, spin, cell) */
    or_ledger led;
    int err;
};

static uint32_t to_thr(double p)
{
    if (!(p > 0.0)) return 0u;
    if (p >= 1.0) return 0xFFFFFFFFu;
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)t;
}

/* direction cosine from a word: odd multiples of 2^-23 in (-1, 1), exact */
static float mu_from(uint32_t x)
{
    int32_t n = (int32_t)(2u * (x >> 9) + 1u) - 8388608;
    return (float)n * (1.0f / 8388608.0f);
}

/* uniform in (0,1): odd multiples of 2^-24, exact */
static float unit_from(uint32_t x)
{
    return (float)(2u * (x >> 9) + 1u) * (1.0f / 16777216.0f);
}

/* uniform integer in 0..n-1 from a word */
static uint32_t below(uint32_t x, uint32_t n)
{
    return (uint32_t)(((uint64_t)x * n) >> 32);
}

static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* normalised pulse CDF on [0, 2 t0] (a Gaussian of the given FWHM centred
 * at t0, truncated symmetrically so that exactly n0 carriers are created) */
static double pulse_F(const or_config *c, double t)
{
    if (t <= 0.0) return 0.0;
    if (t >= 2.0 * c->t0) return 1.0;
    double s = c->fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    double a = Phi(-c->t0 / s), b = Phi(c->t0 / s);
    return (Phi((t - c->t0) / s) - a) / (b - a);
}

/* Philox words of counter (x, stack, step, substream); x is a carrier id or
 * a slot */
static void draw(const or_sim *s, uint64_t x, uint32_t step, uint32_t sub, uint32_t r[4])
{
    uint32_t ctr[4] = { (uint32_t)x, (uint32_t)(x >> 32) | (s->cfg.stack_index << 16),
                        step, sub };
    uint32_t key[2] = { (uint32_t)s->cfg.seed, (uint32_t)(s->cfg.seed >> 32) };
    or_philox4x32_10(ctr, key, r);
}

/* Philox words of counter (key low, key high, step, substream): the draws
 * of a carrier with lineage key `key` (OR_F_LINEAGE_KEYS) */
static void draw_lineage(const or_sim *s, uint64_t key, uint32_t step, uint32_t sub, uint32_t r[4])
{
    uint32_t ctr[4] = { (uint32_t)key, (uint32_t)(key >> 32), step, sub };
    uint32_t k2[2] = { (uint32_t)s->cfg.seed, (uint32_t)(s->cfg.seed >> 32) };
    or_philox4x32_10(ctr, k2, r);
}

/* the draws of the carrier whose draw key is dk: its slot, or with
 * OR_F_LINEAGE_KEYS its lineage key */
static void draw_x(const or_sim *s, uint64_t dk, uint32_t step, uint32_t sub, uint32_t r[4])
{
    if (s->cfg.flags & OR_F_LINEAGE_KEYS) draw_lineage(s, dk, step, sub, r);
    else draw(s, dk, step, sub, r);
}

/* the lineage key of a secondary created at `step` by the carrier with
 * key `parent`: a Philox hash of both (the top two bits are the tags of
 * primaries and loaded carriers) */
static uint64_t child_key(uint64_t parent, uint32_t step)
{
    uint32_t ctr[4] = { (uint32_t)parent, (uint32_t)(parent >> 32), step, 0xC0DEu };
    uint32_t k2[2] = { 0x2545F491u, 0x4F6CDD1Du }, r[4];
    or_philox4x32_10(ctr, k2, r);
    return (((uint64_t)r[1] << 32) | r[0]) & ~(3ull << 62);
}

/* word of the scattering test of the carrier in slot i at this step: word
 * i mod 4 of the call for the slot group i / 4 */
static uint32_t test_word(const or_sim *s, int64_t slot)
{
    uint32_t ctr[4] = { (uint32_t)(slot >> 2), s->cfg.stack_index << 16, s->step, SUB_TEST };
    uint32_t key[2] = { (uint32_t)s->cfg.seed, (uint32_t)(s->cfg.seed >> 32) };
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    return r[slot & 3];
}

static int32_t cell_of(const or_sim *s, float z)
{
    float q = floorf(z / s->cfg.dz);
    int32_t c = (int32_t)q;
    if (q < 0.0f) c = 0;
    if (c > s->n_cells - 1) c = s->n_cells - 1;
    return c;
}

static int idx3(const or_sim *s, int m, int sg, int k) { return (m * 2 + sg) * s->cfg.n_e + (k - 1); }

/* net flux through the cell faces between the start cell a and end cell b
 * of a carrier of weight w (2^-20 units; the weighted flux counts it w times) */
static void flux(or_sim *s, int sg, int a, int b, uint32_t w)
{
    int64_t row = ((int64_t)(s->step / s->cfg.moment_every) * 2 + sg) * (s->n_cells + 1);
    int32_t *J = s->Jh + row;
    int64_t *Jw = s->Jhw + row;
    if (b > a) for (int f = a + 1; f <= b; ++f) { J[f] += 1; Jw[f] += w; }
    else       for (int f = b + 1; f <= a; ++f) { J[f] -= 1; Jw[f] -= w; }
}

/* ---- adjoint bookkeeping (used only when s->adj is set) ---- */

/* make room in the id-indexed arrays for ids below n */
static void adj_grow(or_sim *s, uint64_t n)
{
    or_adj *A = s->adj;
    if (n <= A->n_ids) return;
    uint64_t m = A->n_ids ? A->n_ids : 1024;
    while (m < n) m *= 2;
    A->own = (double *)realloc(A->own, sizeof(double) * m);
    A->acc = (double *)realloc(A->acc, sizeof(double) * m);
    A->parent = (uint64_t *)realloc(A->parent, sizeof(uint64_t) * m);
    for (uint64_t i = A->n_ids; i < m; ++i) {
        A->own[i] = 0.0; A->acc[i] = 0.0; A->parent[i] = UINT64_MAX;
    }
    A->n_ids = m;
}

/* weight of the flux a carrier of spin sg contributes when it moves from
 * cell a to cell b in this step: the signed sum over the faces it crosses */
static double flux_reward(const or_sim *s, int sg, int a, int b)
{
    const float *g = s->adj->gJ + ((int64_t)(s->step / s->cfg.moment_every) * 2 + sg) * (s->n_cells + 1);
    double r = 0.0;
    if (b > a) for (int f = a + 1; f <= b; ++f) r += g[f];
    else       for (int f = b + 1; f <= a; ++f) r -= g[f];
    return r;
}

/* a reward earned by carrier id: pass 1 sums it into the carrier's own
 * total, pass 2 into what the carrier has earned so far */
static void credit(or_sim *s, uint64_t id, double r)
{
    or_adj *A = s->adj;
    if (A->pass == 1) A->own[id] += r;
    else A->acc[id] += r;
}

/* the score of one decision (is_T: a transmittance entry, else a lifetime
 * entry), weighted by the reward-to-go of the carrier being advanced, or
 * held back while a secondary's flight has no id yet */
static void add_score(or_sim *s, int is_T, int bin, double sc)
{
    or_adj *A = s->adj;
    if (A->pass != 2) return;
    if (A->buffering) {
        A->buf_T[A->nbuf] = is_T; A->buf_bin[A->nbuf] = bin; A->buf_s[A->nbuf] = sc;
        A->nbuf++;
        return;
    }
    double *g = is_T ? A->g_T : A->g_tau, *m = is_T ? A->m_T : A->m_tau;
    g[bin] += sc * A->R;
    m[bin] += fabs(sc) * A->Rmag;
}

/* Transport for a time tau (Eq. Strang-transport): free flight inside the
 * current layer; at a vacuum surface the carrier is reflected; at an
 * interface a uniform draw against T decides transmission (layer changes,
 * direction kept) or reflection (direction mirrored); the remaining time is
 * then flown with the velocity of the layer the carrier is in. */
static int half_flight(or_sim *s, or_rec *p, float tau, uint64_t key, uint32_t sub0)
{
    int met = 0;      /* boundaries met (surfaces and interfaces) */
    const or_config *c = &s->cfg;
    uint32_t w0 = p->packed;
    int k = (int)PK_K(w0), sg = (int)PK_S(w0), layer = (int)PK_L(w0);
    for (int hit = 0;; ++hit) {
        int m = c->layer_mat[layer];
        float v = s->v[idx3(s, m, sg, k)];
        float w = v * p->mu;
        float d = w * tau;
        float z1 = p->z + d;
        float lo = s->edge[layer], hi = s->edge[layer + 1];
        float zb; int up;
        if (p->mu > 0.0f && z1 > hi) { zb = hi; up = 1; }
        else if (p->mu < 0.0f && z1 < lo) { zb = lo; up = 0; }
        else { p->z = z1; break; }
        ++met;
        if (hit == OR_MAX_HITS) { p->z = zb; s->led.truncated++; break; }
        float tb = (zb - p->z) / w;
        tau = tau - tb;
        if (!(tau > 0.0f)) tau = 0.0f;
        p->z = zb;
        int vacuum = up ? (layer == c->n_layers - 1) : (layer == 0);
        if (vacuum) {
            p->mu = -p->mu;
        } else {
            int iface = up ? layer : layer - 1, dir = up ? 0 : 1;
            int trans = 1;
            s->led.iface_hits++;
            if (!(c->flags & OR_F_TRANSPARENT)) {
                uint32_t r[4];
                draw_x(s, key, s->step, sub0 + (uint32_t)hit, r);
                int te = ((iface * 2 + dir) * 2 + sg) * c->n_e + (k - 1);
                trans = r[0] < s->T_thr[te];
                if (s->adj) add_score(s, 1, te, trans ? s->adj->s_tr[te] : s->adj->s_rf[te]);
            }
            if (trans) { layer += up ? 1 : -1; s->led.iface_transmit++; }
            else p->mu = -p->mu;
        }
    }
    p->packed = (w0 & ~(0xFu << 9)) | ((uint32_t)layer << 9);
    return met;
}

static int append(or_sim *s, or_rec r, uint32_t w, uint64_t lk)
{
    if (s->n_slots >= s->cfg.capacity) return 0;
    s->wq[s->n_slots] = w;
    s->lkey[s->n_slots] = lk;
    s->recs[s->n_slots++] = r;
    return 1;
}

/* Source(dt/2), Eq. Strang-source: carriers created in half step h = 2*step+half */
static void inject(or_sim *s, int half)
{
    const or_config *c = &s->cfg;
    int64_t h = 2 * (int64_t)s->step + half;
    int64_t n = s->inj[h];
    for (int64_t j = 0; j < n; ++j) {
        if (s->n_slots >= c->capacity) {
            s->led.inject_dropped += (uint64_t)(n - j);
            if (c->flags & OR_F_STRICT_CAPACITY) s->err = 3;
            return;
        }
        uint64_t id = s->next_id++;
        if (s->adj) adj_grow(s, s->next_id);
        uint32_t a[4], b[4];
        /* lineage key of a primary: its birth half step and index */
        const uint64_t lk = (1ull << 63) | ((uint64_t)h << 32) | (uint64_t)j;
        if (c->flags & OR_F_LINEAGE_KEYS) {
            draw_lineage(s, lk, s->step, SUB_INJ + 0, a);
            draw_lineage(s, lk, s->step, SUB_INJ + 1, b);
        } else {
            draw(s, id, s->step, SUB_INJ + 0, a);
            draw(s, id, s->step, SUB_INJ + 1, b);
        }
        int i = 0;
        while (i < s->n_cdf - 1 && !(a[0] < s->cdf_thr[i])) ++i;
        float z = ((float)s->cdf_cell[i] + unit_from(a[1])) * c->dz;
        uint32_t sg = a[2] < s->up_thr ? 0u : 1u;
        uint32_t k;
        if (c->e_mode == 1) {
            k = (uint32_t)c->k_mono[sg];
        } else if (s->has_ebias) {
            /* the bin from the biased sampling distribution q */
            k = 1u;
            while ((int)k < c->n_e && !(a[3] < s->kthr[k - 1])) ++k;
        } else {
            k = 1u + below(a[3], (uint32_t)c->n_e);
        }
        /* weight p/q of the carrier's birth cell and bin (Eq. PIC) */
        double wr = s->wcell[i] * s->wbin[k - 1] * 1048576.0;
        uint32_t w = wr < 1.0 ? 1u : wr > 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)nearbyint(wr);
        or_rec r;
        r.z = z;
        r.mu = mu_from(b[0]);
        r.id = (uint32_t)id;
        r.packed = pk(k, sg, (uint32_t)s->cdf_layer[i], 1u, (uint32_t)(id >> 32));
        append(s, r, w, lk);
        s->w_injected += w;
        s->led.injected++;
        s->led.q_injected += k;
    }
}

static void absorb(or_sim *s, or_rec *p)
{
    p->packed &= ~0xFFu;       /* k = 0 marks a removed carrier */
    s->led.absorbed++;
    s->led.q_bath += 1;
}

/* Transport(dt/2) -> Scattering(dt) -> Transport(dt/2) of the live carrier
 * p that sits in slot i; a secondary is appended to the slots. */
static void advance(or_sim *s, or_rec *p, int64_t i, uint32_t w, uint64_t dk)
{
    const or_config *c = &s->cfg;
    const float half = c->dt * 0.5f;
    {
        s->led.particle_steps++;
        uint64_t id = (uint64_t)p->id | ((uint64_t)PK_E(p->packed) << 32);
        const float mu_in = p->mu;
        const uint32_t pk_in = p->packed;
        int c_start = cell_of(s, p->z);
        int sg = (int)PK_S(p->packed);
        or_adj *A = s->adj;
        if (A && A->pass == 2) {
            /* every decision of this step is weighted by what the carrier
             * and its descendants still earn from the start of the step */
            A->R = A->own[id] - A->acc[id];
            A->Rmag = fabs(A->own[id]) + fabs(A->acc[id]);
        }

        const int met1 = half_flight(s, p, half, dk, SUB_IF + 0);

        /* Scattering(dt): one Monte-Carlo test against tau_eff (Eq. lifetimes);
         * the event words are drawn only for a carrier that scatters */
        uint32_t x[4] = { 0u, 0u, 0u, 0u };
        if (c->flags & OR_F_LINEAGE_KEYS) {
            uint32_t tw[4];
            draw_lineage(s, dk, s->step, SUB_TEST, tw);
            x[0] = tw[0];
        } else {
            x[0] = test_word(s, i);
        }
        if (x[0] < s->P_thr[idx3(s, c->layer_mat[PK_L(p->packed)], sg, (int)PK_K(p->packed))]) {
            uint32_t ev[4];
            draw_x(s, dk, s->step, SUB_EVT, ev);
            x[1] = ev[1]; x[2] = ev[2]; x[3] = ev[3];
        }
        int k = (int)PK_K(p->packed), layer = (int)PK_L(p->packed);
        int m = c->layer_mat[layer];
        int t = idx3(s, m, sg, k);
        if (met1 || x[0] < s->P_thr[t]) s->led.eventful++;
        if (A) {
            /* scores of the scattering test and, after a scattering, of the
             * choice between the elastic and the inelastic channel */
            double sc = A->s_noscat[t];
            if (x[0] < s->P_thr[t]) sc = A->s_scat[t] + (x[1] < s->Q_thr[t] ? A->s_inel[t] : A->s_el[t]);
            add_score(s, 0, t, sc);
        }
        if (x[0] < s->P_thr[t]) {
            int inel = x[1] < s->Q_thr[t];
            if (k == 1 && (inel || (c->flags & OR_F_LOWEST_BIN_ANY))) {
                absorb(s, p);
                flux(s, sg, c_start, cell_of(s, p->z), w);
                if (A) credit(s, id, flux_reward(s, sg, c_start, cell_of(s, p->z)));
                s->led.changed++;
                return;
            }
            p->mu = mu_from(x[2]);
            if (inel) {
                uint32_t kp = 1u + below(x[3], (uint32_t)(k - 1));
                uint32_t ks = (uint32_t)k - kp;
                p->packed = (p->packed & ~0xFFu) | kp;
                if (c->flags & OR_F_NO_SECONDARIES) {
                    s->led.q_bath += ks;
                } else {
                    /* secondary: same place, spin from P0 of this material,
                     * isotropic direction, one generation more */
                    uint32_t y[4];
                    draw_x(s, dk, s->step, SUB_SEC, y);
                    uint32_t g = PK_G(p->packed);
                    uint32_t sgs = y[0] < s->P0_thr[m] ? 0u : 1u;
                    or_rec q;
                    q.z = p->z;
                    q.mu = mu_from(y[1]);
                    q.id = 0;
                    q.packed = pk(ks, sgs, (uint32_t)layer, g < 255u ? g + 1u : 255u, 0u);
                    int cs = cell_of(s, q.z);
                    /* boundary events are counted for carriers that exist
                     * after the step: a dropped secondary's are taken back */
                    or_ledger keep = s->led;
                    if (A) { A->buffering = 1; A->nbuf = 0; }
                    half_flight(s, &q, half, dk, SUB_SIF);
                    if (A) A->buffering = 0;
                    if (s->n_slots < c->capacity) {
                        uint64_t nid = s->next_id++;
                        q.id = (uint32_t)nid;
                        q.packed |= (uint32_t)(nid >> 32) << 21;
                        /* the secondary carries its parent's weight */
                        append(s, q, w, child_key(dk, s->step));
                        s->led.spawned++;
                        flux(s, (int)sgs, cs, cell_of(s, q.z), w);
                        if (A) {
                            adj_grow(s, s->next_id);
                            if (A->pass == 1) {
                                A->parent[nid] = id;
                            } else {
                                /* the secondary's own decisions of this half
                                 * step, weighted by its whole lineage total;
                                 * the parent has now earned that total */
                                double Rp = A->R, Rm = A->Rmag;
                                A->R = A->own[nid];
                                A->Rmag = fabs(A->own[nid]);
                                for (int b = 0; b < A->nbuf; ++b)
                                    add_score(s, A->buf_T[b], A->buf_bin[b], A->buf_s[b]);
                                A->R = Rp; A->Rmag = Rm;
                                A->acc[id] += A->own[nid];
                            }
                            credit(s, nid, flux_reward(s, (int)sgs, cs, cell_of(s, q.z)));
                        }
                    } else {
                        s->led.iface_hits = keep.iface_hits;
                        s->led.iface_transmit = keep.iface_transmit;
                        s->led.truncated = keep.truncated;
                        s->led.spawn_dropped++;
                        s->led.q_dropped += ks;
                        if (c->flags & OR_F_STRICT_CAPACITY) s->err = 3;
                    }
                }
            }
        }

        const int met2 = half_flight(s, p, half, dk, SUB_IF + 16);
        if (met2 && !met1 && !(x[0] < s->P_thr[t])) s->led.eventful++;
        flux(s, sg, c_start, cell_of(s, p->z), w);
        if (A) credit(s, id, flux_reward(s, sg, c_start, cell_of(s, p->z)));
        if (p->mu != mu_in || p->packed != pk_in) s->led.changed++;
    }
}

static void step_once(or_sim *s)
{
    const or_config *c = &s->cfg;
    inject(s, 0);
    int64_t n_start = s->n_slots;
    for (int64_t i = 0; i < n_start; ++i) {
        or_rec *p = &s->recs[i];
        if (PK_K(p->packed) == 0) continue;
        advance(s, p, i, s->wq[i], (c->flags & OR_F_LINEAGE_KEYS) ? s->lkey[i] : (uint64_t)i);
    }
    inject(s, 1);

    if ((s->step + 1) % (uint32_t)c->moment_every == 0) {
        int64_t tout = (int64_t)(s->step + 1) / c->moment_every - 1;
        for (int64_t i = 0; i < s->n_slots; ++i) {
            const or_rec *p = &s->recs[i];
            uint32_t k = PK_K(p->packed);
            if (k == 0) continue;
            int64_t b = ((tout * 2 + PK_S(p->packed)) * c->n_e + (k - 1)) * s->n_cells
                        + cell_of(s, p->z);
            s->nh[b] += 1;
            s->nhw[b] += s->wq[i];
            s->gh[tout * s->n_cells + cell_of(s, p->z)] += PK_G(p->packed);
            if (c->flags & OR_F_VELOCITY) {
                /* the carrier's velocity along z, v(layer material, spin, k) * mu,
                 * in float32, kept as an integer number of 2^-32 nm/fs
                 * (truncated) so that sums do not depend on their order */
                const float w = s->v[idx3(s, c->layer_mat[PK_L(p->packed)], (int)PK_S(p->packed), (int)k)] *
                                p->mu;
                s->vh[(tout * 2 + PK_S(p->packed)) * s->n_cells + cell_of(s, p->z)] +=
                    (int64_t)(w * 4294967296.0f);
            }
            if (s->adj) credit(s, (uint64_t)p->id | ((uint64_t)PK_E(p->packed) << 32), s->adj->gn[b]);
        }
    }
    if ((s->step + 1) % (uint32_t)c->compact_every == 0) {
        int64_t j = 0;
        for (int64_t i = 0; i < s->n_slots; ++i)
            if (PK_K(s->recs[i].packed) != 0) {
                s->wq[j] = s->wq[i];
                s->lkey[j] = s->lkey[i];
                s->recs[j++] = s->recs[i];
            }
        s->n_slots = j;
    }
    s->step++;
}

int or_step(or_sim *s, int n_steps)
{
    for (int i = 0; i < n_steps; ++i) {
        if ((int64_t)s->step >= s->cfg.n_steps_max) return 2;
        step_once(s);
        if (s->err) return s->err;
    }
    return 0;
}

static void derive(or_sim *s)
{
    const or_config *c = &s->cfg;
    int ne = c->n_e;
    for (int m = 0; m < c->n_mat; ++m)
        for (int sg = 0; sg < 2; ++sg)
            for (int k = 1; k <= ne; ++k) {
                int t = idx3(s, m, sg, k);
                double ti = s->tau_in[t], te = s->tau_el[m];
                double r_in = isinf(ti) ? 0.0 : 1.0 / ti;
                double r_el = isinf(te) ? 0.0 : 1.0 / te;
                double r = r_el + r_in;
                double a = (double)c->dt * r;
                s->P_thr[t] = to_thr(-expm1(-a));
                s->Q_thr[t] = to_thr(r > 0.0 ? r_in / r : 0.0);
            }
    for (int i = 0; i < (c->n_layers - 1) * 2 * 2 * ne; ++i) s->T_thr[i] = to_thr(s->T[i]);
    for (int m = 0; m < c->n_mat; ++m) s->P0_thr[m] = to_thr((1.0 + s->p0[m]) / 2.0);
    s->up_thr = to_thr(c->up_frac);

    /* excitation profile: cell masses of exp(-z/abs_len) (or uniform) over
     * the excited layers, cumulated in cell order */
    int n = 0, cell = 0;
    double total = 0.0;
    double *mass = (double *)malloc(sizeof(double) * (size_t)(s->n_cells > 0 ? s->n_cells : 1));
    for (int l = 0; l < c->n_layers; ++l) {
        for (int j = 0; j < c->layer_cells[l]; ++j, ++cell) {
            if (!((c->excite_mask >> l) & 1u)) continue;
            double zc = (double)cell * c->dz, dz = c->dz, m;
            if (c->abs_len > 0.0) m = c->abs_len * (exp(-zc / c->abs_len) - exp(-(zc + dz) / c->abs_len));
            else m = dz;
            s->cdf_cell[n] = cell; s->cdf_layer[n] = l; mass[n] = m; total += m; ++n;
        }
    }
    s->n_cdf = n;
    double cum = 0.0;
    if (c->cell_bias && (c->flags & OR_F_WEIGHTS)) {
        /* importance sampling of the birth cell: q_i proportional to
         * mass_i * bias_i, weight p_i / q_i = (sum mass*bias / sum mass) / bias_i */
        double total_b = 0.0;
        for (int i = 0; i < n; ++i) total_b += mass[i] * c->cell_bias[s->cdf_cell[i]];
        for (int i = 0; i < n; ++i) {
            cum += mass[i] * c->cell_bias[s->cdf_cell[i]];
            s->cdf_thr[i] = (i == n - 1) ? 0xFFFFFFFFu : to_thr(cum / total_b);
            s->wcell[i] = (total_b / total) / c->cell_bias[s->cdf_cell[i]];
        }
    } else {
        for (int i = 0; i < n; ++i) {
            cum += mass[i];
            s->cdf_thr[i] = (i == n - 1) ? 0xFFFFFFFFu : to_thr(cum / total);
            s->wcell[i] = 1.0;
        }
    }
    free(mass);
    /* importance sampling of the birth bin (e_mode 0): q_k proportional to
     * bias_k, weight p_k / q_k = (sum bias / n_e) / bias_k */
    s->has_ebias = c->e_bias && (c->flags & OR_F_WEIGHTS) && c->e_mode == 0;
    if (s->has_ebias) {
        double tb = 0.0, cb = 0.0;
        for (int k = 0; k < ne; ++k) tb += c->e_bias[k];
        for (int k = 0; k < ne; ++k) {
            cb += c->e_bias[k];
            s->kthr[k] = (k == ne - 1) ? 0xFFFFFFFFu : to_thr(cb / tb);
            s->wbin[k] = (tb / (double)ne) / c->e_bias[k];
        }
    } else {
        for (int k = 0; k < ne; ++k) s->wbin[k] = 1.0;
    }

    /* injected carriers per half step: floor(N0 F(t_{h+1})) - floor(N0 F(t_h)) */
    int64_t nh = 2 * (int64_t)c->n_steps_max;
    double n0 = (double)c->n0;
    for (int64_t h = 0; h < nh; ++h) {
        double ta = (double)h * 0.5 * (double)c->dt, tb = (double)(h + 1) * 0.5 * (double)c->dt;
        if (c->n0 <= 0 || n == 0) { s->inj[h] = 0; continue; }
        s->inj[h] = (int64_t)floor(n0 * pulse_F(c, tb)) - (int64_t)floor(n0 * pulse_F(c, ta));
    }
}

int or_create(const or_config *cfg, or_sim **out)
{
    *out = NULL;
    if (cfg->n_e < 1 || cfg->n_e > 255 || cfg->n_layers < 1 || cfg->n_layers > OR_MAX_LAYERS ||
        cfg->capacity < 0 || cfg->moment_every < 1 || cfg->compact_every < 1 ||
        cfg->n_steps_max < 0 || cfg->n_mat < 1 || !(cfg->dt > 0.0f) || !(cfg->dz > 0.0f))
        return 1;
    if (cfg->n0 > 0 && !(cfg->fwhm > 0.0 && cfg->t0 > 0.0)) return 1;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->cfg = *cfg;
    int ne = cfg->n_e, nm = cfg->n_mat, nif = cfg->n_layers - 1;
    size_t tab = (size_t)nm * 2 * ne;
    s->v = (float *)malloc(sizeof(float) * tab); memcpy(s->v, cfg->v, sizeof(float) * tab);
    s->tau_in = (double *)malloc(sizeof(double) * tab); memcpy(s->tau_in, cfg->tau_in, sizeof(double) * tab);
    s->tau_el = (double *)malloc(sizeof(double) * nm); memcpy(s->tau_el, cfg->tau_el, sizeof(double) * nm);
    s->p0 = (double *)malloc(sizeof(double) * nm); memcpy(s->p0, cfg->p0, sizeof(double) * nm);
    s->T = (double *)malloc(sizeof(double) * (size_t)(nif * 4 * ne + 1));
    if (nif > 0) memcpy(s->T, cfg->T, sizeof(double) * (size_t)(nif * 4 * ne));
    s->cfg.v = s->v; s->cfg.tau_in = s->tau_in; s->cfg.tau_el = s->tau_el; s->cfg.T = s->T; s->cfg.p0 = s->p0;

    int32_t cells = 0;
    s->edge[0] = 0.0f;
    for (int l = 0; l < cfg->n_layers; ++l) {
        if (cfg->layer_cells[l] < 1 || cfg->layer_mat[l] < 0 || cfg->layer_mat[l] >= nm) { or_destroy(s); return 1; }
        cells += cfg->layer_cells[l];
        s->edge[l + 1] = (float)cells * cfg->dz;
    }
    s->n_cells = cells;
    s->P_thr = (uint32_t *)malloc(sizeof(uint32_t) * tab);
    s->Q_thr = (uint32_t *)malloc(sizeof(uint32_t) * tab);
    s->T_thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nif * 4 * ne + 1));
    s->P0_thr = (uint32_t *)malloc(sizeof(uint32_t) * nm);
    s->cdf_cell = (int32_t *)malloc(sizeof(int32_t) * cells);
    s->cdf_layer = (int32_t *)malloc(sizeof(int32_t) * cells);
    s->cdf_thr = (uint32_t *)malloc(sizeof(uint32_t) * cells);
    s->inj = (int64_t *)calloc((size_t)(2 * (int64_t)cfg->n_steps_max + 1), sizeof(int64_t));
    s->wcell = (double *)malloc(sizeof(double) * (size_t)(cells > 0 ? cells : 1));
    s->wbin = (double *)malloc(sizeof(double) * (size_t)ne);
    s->kthr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ne);
    derive(s);

    s->recs = (or_rec *)malloc(sizeof(or_rec) * (size_t)(cfg->capacity > 0 ? cfg->capacity : 1));
    s->wq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(cfg->capacity > 0 ? cfg->capacity : 1));
    s->lkey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cfg->capacity > 0 ? cfg->capacity : 1));
    s->n_out = (cfg->n_steps_max + cfg->moment_every - 1) / cfg->moment_every;
    s->nh = (uint32_t *)calloc((size_t)s->n_out * 2 * ne * cells + 1, sizeof(uint32_t));
    s->Jh = (int32_t *)calloc((size_t)s->n_out * 2 * (cells + 1) + 1, sizeof(int32_t));
    s->gh = (uint64_t *)calloc((size_t)s->n_out * cells + 1, sizeof(uint64_t));
    s->vh = (int64_t *)calloc((size_t)s->n_out * 2 * cells + 1, sizeof(int64_t));
    s->nhw = (uint64_t *)calloc((size_t)s->n_out * 2 * ne * cells + 1, sizeof(uint64_t));
    s->Jhw = (int64_t *)calloc((size_t)s->n_out * 2 * (cells + 1) + 1, sizeof(int64_t));
    if (!s->recs || !s->wq || !s->lkey || !s->nh || !s->Jh || !s->gh || !s->vh || !s->nhw || !s->Jhw) {
        or_destroy(s);
        return 4;
    }
    *out = s;
    return 0;
}

void or_destroy(or_sim *s)
{
    if (!s) return;
    free(s->v); free(s->tau_in); free(s->tau_el); free(s->T); free(s->p0);
    free(s->P_thr); free(s->Q_thr); free(s->T_thr); free(s->P0_thr);
    free(s->cdf_cell); free(s->cdf_layer); free(s->cdf_thr); free(s->inj);
    free(s->recs); free(s->nh); free(s->Jh); free(s->gh); free(s->vh);
    free(s->wq); free(s->lkey); free(s->wcell); free(s->wbin); free(s->kthr); free(s->nhw); free(s->Jhw);
    free(s);
}

int64_t or_n_slots(const or_sim *s) { return s->n_slots; }
int32_t or_n_cells(const or_sim *s) { return s->n_cells; }
int32_t or_n_out(const or_sim *s) { return s->n_out; }
int32_t or_step_index(const or_sim *s) { return (int32_t)s->step; }
void or_set_step(or_sim *s, int32_t step) { s->step = (uint32_t)step; }
uint64_t or_next_id(const or_sim *s) { return s->next_id; }

void or_records(const or_sim *s, or_rec *out)
{
    memcpy(out, s->recs, sizeof(or_rec) * (size_t)s->n_slots);
}

int or_set_records(or_sim *s, const or_rec *in, int64_t n, uint64_t next_id)
{
    if (n < 0 || n > s->cfg.capacity) return 1;
    memcpy(s->recs, in, sizeof(or_rec) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        s->wq[i] = 1u << 20;                               /* unit weight */
        s->lkey[i] = (1ull << 62) | (uint64_t)i;           /* lineage key of a loaded carrier */
    }
    s->n_slots = n;
    s->next_id = next_id;
    return 0;
}

void or_moments(const or_sim *s, uint32_t *n_out, int32_t *J_out, or_ledger *led)
{
    size_t nn = (size_t)s->n_out * 2 * s->cfg.n_e * s->n_cells;
    size_t nj = (size_t)s->n_out * 2 * (s->n_cells + 1);
    if (n_out) memcpy(n_out, s->nh, sizeof(uint32_t) * nn);
    if (J_out) memcpy(J_out, s->Jh, sizeof(int32_t) * nj);
    if (led) *led = s->led;
}

/* Mean-generation map of Figs. 5(b) and 7(b),(d) (Sec. V): the generation
 * label of every live carrier (1 for a primary, its parent's + 1 for a
 * secondary) summed per (output time, cell) at the same instants as the
 * densities; divided by the summed density it gives the mean label. */
void or_gen_moments(const or_sim *s, uint64_t *g_out)
{
    if (g_out) memcpy(g_out, s->gh, sizeof(uint64_t) * (size_t)s->n_out * s->n_cells);
}

/* Velocity moment behind the spin current of Eq. spincurrent (Sec. V):
 * with OR_F_VELOCITY, the velocities along z, v * mu, of the live carriers
 * of each spin summed per (output time, cell) at the density instants, in
 * units of 2^-32 nm/fs; (sum_up - sum_down) / dz is the spin-current
 * density of the cell in carriers nm/fs per nm. */
void or_vel_moments(const or_sim *s, int64_t *v_out)
{
    if (v_out) memcpy(v_out, s->vh, sizeof(int64_t) * (size_t)s->n_out * 2 * s->n_cells);
}

void or_weighted_moments(const or_sim *s, uint64_t *nw_out, int64_t *Jw_out, uint64_t *w_injected)
{
    if (nw_out) memcpy(nw_out, s->nhw, sizeof(uint64_t) * (size_t)s->n_out * 2 * s->cfg.n_e * s->n_cells);
    if (Jw_out) memcpy(Jw_out, s->Jhw, sizeof(int64_t) * (size_t)s->n_out * 2 * (s->n_cells + 1));
    if (w_injected) *w_injected = s->w_injected;
}

void or_weights(const or_sim *s, uint32_t *w_out)
{
    memcpy(w_out, s->wq, sizeof(uint32_t) * (size_t)s->n_slots);
}

int or_set_weights(or_sim *s, const uint32_t *w, int64_t n)
{
    if (n != s->n_slots) return 1;
    for (int64_t i = 0; i < n; ++i) if (w[i] == 0u) return 1;
    memcpy(s->wq, w, sizeof(uint32_t) * (size_t)n);
    return 0;
}

void or_tables(const or_sim *s, uint32_t *P_thr, uint32_t *Q_thr, uint32_t *T_thr,
               uint32_t *P0_thr, uint32_t *up_thr, int64_t *inj_counts)
{
    const or_config *c = &s->cfg;
    size_t tab = (size_t)c->n_mat * 2 * c->n_e;
    if (P_thr) memcpy(P_thr, s->P_thr, sizeof(uint32_t) * tab);
    if (Q_thr) memcpy(Q_thr, s->Q_thr, sizeof(uint32_t) * tab);
    if (T_thr) memcpy(T_thr, s->T_thr, sizeof(uint32_t) * (size_t)(c->n_layers - 1) * 4 * c->n_e);
    if (P0_thr) memcpy(P0_thr, s->P0_thr, sizeof(uint32_t) * c->n_mat);
    if (up_thr) *up_thr = s->up_thr;
    if (inj_counts) memcpy(inj_counts, s->inj, sizeof(int64_t) * 2 * (size_t)c->n_steps_max);
}

/* ---- adjoint: score-function gradient of a linear functional of the
 * moments, O = sum gn * n + sum gJ * J, with respect to tau_in and T.
 *
 * Every random decision of the step has an outcome probability that
 * depends on the tables: the scattering test (p = 1 - exp(-dt/tau_eff),
 * Eq. lifetimes), the channel (inelastic with q = tau_eff/tau_in) and each
 * interface draw (transmission with T).  The derivative of E[O] is the
 * expectation of sum over decisions of d log P(outcome)/d theta times the
 * reward that follows the decision.  The reward that may follow a decision
 * of carrier i in step s is what i earns from the start of step s on plus
 * the lineage totals of the secondaries it creates from then on (rewards
 * that cannot depend on the outcome add only zero-mean terms).
 *
 * Pass 1 replays the run and sums each carrier's own rewards and records
 * its parent; the lineage totals follow by adding every carrier's total to
 * its parent's, children first (a child's id is larger than its parent's).
 * Pass 2 replays the run again with the totals known. */
int or_grad(const or_config *cfg, const or_rec *init, int64_t n_init, uint64_t next_id,
            int n_steps, const float *gn, const float *gJ, double *g_tau, double *g_T,
            double *mag_tau, double *mag_T)
{
    for (int64_t i = 0; i < n_init; ++i) {
        uint64_t id = (uint64_t)init[i].id | ((uint64_t)PK_E(init[i].packed) << 32);
        if (id >= next_id) return 1;
    }
    const int ne = cfg->n_e, nm = cfg->n_mat;
    const size_t ntau = (size_t)nm * 2 * ne;
    const size_t nT = (size_t)(cfg->n_layers > 1 ? cfg->n_layers - 1 : 0) * 4 * ne;
    or_adj A;
    memset(&A, 0, sizeof(A));
    A.gn = gn; A.gJ = gJ;
    A.s_noscat = (double *)calloc(ntau + 1, sizeof(double));
    A.s_scat = (double *)calloc(ntau + 1, sizeof(double));
    A.s_el = (double *)calloc(ntau + 1, sizeof(double));
    A.s_inel = (double *)calloc(ntau + 1, sizeof(double));
    A.s_tr = (double *)calloc(nT + 1, sizeof(double));
    A.s_rf = (double *)calloc(nT + 1, sizeof(double));
    A.g_tau = (double *)calloc(ntau + 1, sizeof(double));
    A.m_tau = (double *)calloc(ntau + 1, sizeof(double));
    A.g_T = (double *)calloc(nT + 1, sizeof(double));
    A.m_T = (double *)calloc(nT + 1, sizeof(double));

    /* d log P / d tau_in with rates r_in = 1/tau_in, r_el = 1/tau_el,
     * r = r_in + r_el and d r_in / d tau_in = -r_in^2:
     *   no scattering  log(1-p) = -dt r          ->  dt r_in^2
     *   scattering     log p                     -> -dt r_in^2 e^{-dt r} / p
     *   inelastic      log(r_in/r)               -> -r_in r_el / r
     *   elastic        log(r_el/r)               ->  r_in^2 / r
     * d log P / d T: transmission 1/T, reflection -1/(1-T). */
    const double dt = (double)cfg->dt;
    for (int m = 0; m < nm; ++m)
        for (int sg = 0; sg < 2; ++sg)
            for (int k = 0; k < ne; ++k) {
                size_t t = ((size_t)m * 2 + sg) * ne + k;
                double ti = cfg->tau_in[t], te = cfg->tau_el[m];
                double r_in = isinf(ti) ? 0.0 : 1.0 / ti;
                double r_el = isinf(te) ? 0.0 : 1.0 / te;
                double r = r_in + r_el, a = dt * r, p = -expm1(-a);
                A.s_noscat[t] = dt * r_in * r_in;
                A.s_scat[t] = p > 0.0 ? -dt * r_in * r_in * exp(-a) / p : 0.0;
                A.s_inel[t] = r > 0.0 ? -r_in * r_el / r : 0.0;
                A.s_el[t] = (r > 0.0 && r_el > 0.0) ? r_in * r_in / r : 0.0;
            }
    for (size_t i = 0; i < nT; ++i) {
        double T = cfg->T[i];
        A.s_tr[i] = T > 0.0 ? 1.0 / T : 0.0;
        A.s_rf[i] = T < 1.0 ? -1.0 / (1.0 - T) : 0.0;
    }

    int rc = 0;
    for (int pass = 1; pass <= 2 && rc == 0; ++pass) {
        or_sim *s = NULL;
        rc = or_create(cfg, &s);
        if (rc) break;
        s->adj = &A;
        A.pass = pass;
        adj_grow(s, next_id);
        if (or_set_records(s, init, n_init, next_id)) rc = 1;
        if (!rc) rc = or_step(s, n_steps);
        s->adj = NULL;
        or_destroy(s);
        if (pass == 1 && !rc)
            for (uint64_t i = A.n_ids; i-- > 0;)
                if (A.parent[i] != UINT64_MAX) A.own[A.parent[i]] += A.own[i];
    }
    if (rc == 0) {
        if (g_tau) memcpy(g_tau, A.g_tau, sizeof(double) * ntau);
        if (mag_tau) memcpy(mag_tau, A.m_tau, sizeof(double) * ntau);
        if (g_T && nT) memcpy(g_T, A.g_T, sizeof(double) * nT);
        if (mag_T && nT) memcpy(mag_T, A.m_T, sizeof(double) * nT);
    }
    free(A.s_noscat); free(A.s_scat); free(A.s_el); free(A.s_inel); free(A.s_tr); free(A.s_rf);
    free(A.g_tau); free(A.m_tau); free(A.g_T); free(A.m_T);
    free(A.own); free(A.acc); free(A.parent);
    return rc;
}

int or_advance_one(or_sim *s, const or_rec *in, int64_t slot, int room, or_rec *out, or_rec *sec)
{
    or_rec p = *in;
    int64_t keep_n = s->n_slots, keep_cap = s->cfg.capacity;
    uint64_t keep_id = s->next_id;
    s->n_slots = 0;
    s->cfg.capacity = room ? 1 : 0;
    int made = 0;
    if (PK_K(p.packed) != 0) {
        advance(s, &p, slot, 1u << 20, (uint64_t)slot);
        made = s->n_slots == 1;
        if (made && sec) *sec = s->recs[0];
    }
    s->n_slots = keep_n;
    s->cfg.capacity = keep_cap;
    s->next_id = keep_id;
    if (out) *out = p;
    return made;
}
