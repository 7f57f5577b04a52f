// C-ABI of the GB300 hot-electron PIC library (declared in include/pic.h).
//
// Host responsibilities: argument checks, derivation of every probability
// threshold in double precision (no transcendental function runs on the
// device), allocation of the HBM state, and the per-step kernel sequence of
// the Strang splitting (Eq. strang, Sec. III.A).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct HostStack {
    pic_stack_desc d;
    int n_cells = 0, n_out = 0;
    int64_t base = 0, cap_round = 0;
    std::vector<float> v;           // [n_mat][2][n_e]
    std::vector<double> tau_in, tau_el, T, p0;
    int n_mat = 0;
    std::vector<uint32_t> P_thr, Q_thr, T_thr, P0_thr;   // material-indexed
    std::vector<long long> inj;     // per half step
    pic_pulse pulse{};
    bool excited = false;
    uint64_t bias_hash = 0;         // of the importance-sampling inputs of pic_excite
};

// Buffers of the adjoint replay, allocated by the first pic_grad: a second
// particle state (the forward state stays untouched), one double per slot,
// the id-indexed lineage arrays, score tables and gradient bins.
struct Replay {
    float *z[2] = {nullptr, nullptr}, *mu[2] = {nullptr, nullptr};
    uint32_t *id[2] = {nullptr, nullptr}, *pk[2] = {nullptr, nullptr};
    long long *acc[2] = {nullptr, nullptr};
    uint32_t *stage_l = nullptr;
    unsigned long long *status = nullptr;
    uint32_t *qcnt = nullptr, *fspawn = nullptr;
    DevCounters *cnt = nullptr;
    DevCtl *ctl = nullptr;
    DevStack *stacks = nullptr;
    AdjEnt *aent = nullptr;
    double2 *aT = nullptr;
    double *g_ent = nullptr, *g_T = nullptr;
    long long *gpot = nullptr;
    int32_t *qgn = nullptr;          // quantised density weights
    unsigned int *gen_max = nullptr, *absmax = nullptr;
    long long *tot = nullptr;
    unsigned long long *parent = nullptr;
    uint8_t *gen = nullptr;
    int64_t ids_cap = 0;        // entries of tot / parent / gen
    int n_status = 0;
    LaunchCfg lc[2]{};
    bool ready = false;
};

struct pic_ctx {
    pic_params p{};
    int n_stacks = 0;
    std::vector<HostStack> hs;
    std::vector<DevStack> ds;
    cudaStream_t stream = nullptr;
    // device memory
    DevStack *d_stacks = nullptr;
    TabEnt *d_ent = nullptr;
    FastEnt *d_fent = nullptr;
    uint32_t *d_T = nullptr, *d_cdf_thr = nullptr;
    int32_t *d_cdf_cell = nullptr, *d_cdf_layer = nullptr;
    long long *d_inj = nullptr;
    float *d_z[2] = {nullptr, nullptr}, *d_mu[2] = {nullptr, nullptr};
    uint32_t *d_id[2] = {nullptr, nullptr}, *d_pk[2] = {nullptr, nullptr};
    float4 *d_stage = nullptr, *d_qrec = nullptr;
    uint32_t *d_bits = nullptr, *d_qcnt = nullptr, *d_fspawn = nullptr;
    unsigned long long *d_status = nullptr;
    uint32_t *d_nh = nullptr;
    unsigned long long *d_gh = nullptr;          // generation sums [stack][n_out][n_cells]
    long long *d_vh = nullptr;                   // velocity sums [stack][n_out][2][n_cells]
    int32_t *d_J = nullptr;
    int32_t *d_bd = nullptr;                     // births minus removals, J layout
    // superparticle weights (PIC_F_WEIGHTS)
    uint32_t *d_w[2] = {nullptr, nullptr};       // per slot, 2^-20 units
    double *d_wcell = nullptr, *d_wbin = nullptr;
    uint32_t *d_kthr = nullptr;
    unsigned long long *d_nhw = nullptr;         // weighted densities, d_nh layout
    long long *d_bdw = nullptr, *d_Jw = nullptr; // weighted births-minus-removals, fluxes
    long long *d_hnow_w = nullptr;
    int flux_final_w = 0;
    int32_t *d_hnow = nullptr;                   // live carriers per [stack][2][ncm+1]
    int ncm = 1;                                 // cells of the widest stack
    int flux_final = 0;                          // windows whose fluxes are final
    DevCounters *d_cnt = nullptr;
    DevCtl *d_ctl = nullptr;
    int64_t total_slots = 0, nh_total = 0, J_total = 0;
    int n_status = 0;                // look-back words and queue counts allocated
    Args args{};
    LaunchCfg lc{};
    int step = 0;
    int64_t launches = 0;
    std::string err;
    // initial state the adjoint replays from: records loaded at step 0
    std::vector<std::vector<pic_record>> init_recs;
    std::vector<uint64_t> init_next_id;
    bool replayable = true;
    std::string replay_why;
    size_t n_ent = 0, n_T = 0;   // entries of the layer and interface tables
    int n_mat_max = 1;
    Replay rp;
    // CUDA graphs of one period of steps (use_graph): [0] with the source
    // kernels, [1] without (after the pulse); captured on a private stream
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t period_graph[2] = {nullptr, nullptr};
    int64_t period_launches[2] = {0, 0};
    int period = 0;
    bool dev_step_valid = false;     // d_ctl->step == step
    // the persistent kernel (use_graph 2): its configuration and the graph of
    // one launch covering a period
    PersistCfg pcfg;
    cudaGraphExec_t persist_graph = nullptr;
    bool persist_direct = false;     // the launch could not be captured: launched directly
    // kernel timing (pic_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_marks;   // (kind, index of start event)
    size_t ev_used = 0;
};

namespace {

thread_local std::string g_init_error;   // reason of the last failed pic_init

const char *kStatusNames[] = {"PIC_OK", "PIC_ERR_ARG", "PIC_ERR_ALLOC", "PIC_ERR_CAPACITY",
                              "PIC_ERR_TIMEOUT", "PIC_ERR_CUDA", "PIC_ERR_STATE"};

// 64-bit FNV-1a over bytes (the fingerprint of a checkpoint)
uint64_t fnv1a(const void *data, size_t n, uint64_t h = 0xcbf29ce484222325ull)
{
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 0x100000001b3ull; }
    return h;
}

// floor(p * 2^32) saturated to [0, 2^32-1]: "x < threshold" with a uniform
// 32-bit word x happens with probability threshold / 2^32.
uint32_t threshold_of(double p)
{
    if (!(p > 0.0)) return 0u;
    if (p >= 1.0) return 0xFFFFFFFFu;
    const double scaled = std::floor(p * 4294967296.0);
    return scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
}

pic_status fail(pic_ctx *c, pic_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

pic_status cuda_fail(pic_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool valid_params(const pic_params *p, std::string &why)
{
    if (!p) { why = "params is NULL"; return false; }
    if (p->n_e < 1 || p->n_e > PIC_MAX_NE) { why = "n_e out of range"; return false; }
    if (!(p->dt > 0.f) || !std::isfinite(p->dt)) { why = "dt must be > 0"; return false; }
    if (!(p->dz > 0.f) || !std::isfinite(p->dz)) { why = "dz must be > 0"; return false; }
    int dz_exp = 0;
    if (std::frexp(p->dz, &dz_exp) != 0.5f) { why = "dz must be a power of two"; return false; }
    if (p->compact_every < 1 || p->moment_every < 1) { why = "compact_every/moment_every < 1"; return false; }
    if (p->n_steps_max < 0) { why = "n_steps_max < 0"; return false; }
    if (p->hist_mode < 0 || p->hist_mode > 1) { why = "hist_mode must be 0 or 1"; return false; }
    if (p->blocks_per_sm < 0) { why = "blocks_per_sm < 0"; return false; }
    if (p->ring_stages != 0 && (p->ring_stages < 2 || p->ring_stages > 8)) {
        why = "ring_stages must be 0 or 2..8"; return false;
    }
    if (p->use_graph < 0 || p->use_graph > 2) { why = "use_graph must be 0, 1 or 2"; return false; }
    if (p->consumer_warps != 0 && p->consumer_warps != 4 && p->consumer_warps != 8) {
        why = "consumer_warps must be 0, 4 or 8"; return false;
    }
    if (p->event_pass != 0 && p->event_pass != 1) {
        why = "event_pass must be 0 or 1"; return false;
    }
    if (p->stack_base < 0 || p->stack_base > 65535) { why = "stack_base out of range"; return false; }
    return true;
}

bool valid_stack(const pic_params *p, const pic_stack_desc *s, const pic_tables *t, std::string &why)
{
    if (!s || !t) { why = "stack or tables is NULL"; return false; }
    if (s->n_layers < 1 || s->n_layers > PIC_MAX_LAYERS) { why = "n_layers out of range"; return false; }
    if (s->capacity < 0 || s->capacity >= (1ll << 30)) { why = "capacity must be in [0, 2^30)"; return false; }
    if (t->n_mat < 1 || t->n_mat > PIC_MAX_MAT) { why = "n_mat out of range"; return false; }
    if (!t->v || !t->tau_in || !t->tau_el || !t->p0 || (s->n_layers > 1 && !t->T)) {
        why = "a table pointer is NULL"; return false;
    }
    int64_t cells = 0;
    for (int l = 0; l < s->n_layers; ++l) {
        if (s->layer_cells[l] < 1) { why = "layer thickness must be >= 1 cell"; return false; }
        if (s->layer_mat[l] < 0 || s->layer_mat[l] >= t->n_mat) { why = "layer material out of range"; return false; }
        cells += s->layer_cells[l];
    }
    if (cells > (1 << 20)) { why = "too many cells"; return false; }
    const int ne = p->n_e;
    for (int i = 0; i < t->n_mat * 2 * ne; ++i) {
        if (!(t->v[i] > 0.f) || !std::isfinite(t->v[i])) { why = "v must be finite and > 0"; return false; }
        if (!(t->tau_in[i] > 0.0)) { why = "tau_in must be > 0"; return false; }
    }
    for (int m = 0; m < t->n_mat; ++m) {
        if (!(t->tau_el[m] > 0.0)) { why = "tau_el must be > 0"; return false; }
        if (!(t->p0[m] >= -1.0 && t->p0[m] <= 1.0)) { why = "p0 must be in [-1,1]"; return false; }
    }
    for (int i = 0; i < (s->n_layers - 1) * 4 * ne; ++i)
        if (!(t->T[i] >= 0.0 && t->T[i] <= 1.0)) { why = "T must be in [0,1]"; return false; }
    return true;
}

// Thresholds of one material table set: scatter within dt with probability
// p = 1 - exp(-dt (1/tau_el + 1/tau_in)) (Eq. lifetimes, Sec. III); the event
// is inelastic with probability (1/tau_in) / (1/tau_el + 1/tau_in) (competing
// rates, Eq. split_w); secondary spin up with probability (1 + P0)/2 (Eq. eq_pol).
void material_thresholds(const pic_params &p, const pic_stack_desc &s, const pic_tables &t,
                         std::vector<uint32_t> &P, std::vector<uint32_t> &Q,
                         std::vector<uint32_t> &T, std::vector<uint32_t> &P0)
{
    const int ne = p.n_e, nm = t.n_mat;
    P.assign((size_t)nm * 2 * ne, 0u);
    Q.assign((size_t)nm * 2 * ne, 0u);
    for (int m = 0; m < nm; ++m) {
        const double rate_el = std::isinf(t.tau_el[m]) ? 0.0 : 1.0 / t.tau_el[m];
        for (int sp = 0; sp < 2; ++sp)
            for (int k = 0; k < ne; ++k) {
                const size_t i = ((size_t)m * 2 + sp) * ne + k;
                const double rate_in = std::isinf(t.tau_in[i]) ? 0.0 : 1.0 / t.tau_in[i];
                const double rate = rate_el + rate_in;
                P[i] = threshold_of(-std::expm1(-((double)p.dt * rate)));
                Q[i] = threshold_of(rate > 0.0 ? rate_in / rate : 0.0);
            }
    }
    const size_t nT = (size_t)(s.n_layers - 1) * 4 * ne;
    T.resize(nT);
    for (size_t i = 0; i < nT; ++i) T[i] = threshold_of(t.T[i]);
    P0.resize(nm);
    for (int m = 0; m < nm; ++m) P0[m] = threshold_of((1.0 + t.p0[m]) / 2.0);
}

double std_normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Fraction of the pulse delivered by time t: a Gaussian of the given FWHM
// centred at t0, truncated to [0, 2 t0] and renormalised.
double pulse_fraction(const pic_pulse &u, double t)
{
    if (t <= 0.0) return 0.0;
    if (t >= 2.0 * u.t0) return 1.0;
    const double sd = u.fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const double lo = std_normal_cdf(-u.t0 / sd), hi = std_normal_cdf(u.t0 / sd);
    return (std_normal_cdf((t - u.t0) / sd) - lo) / (hi - lo);
}

// Source schedule and depth profile of one stack.  With PIC_F_WEIGHTS and a
// cell bias the birth cell is drawn from q proportional to mass * bias and
// wcell[i] = p_i / q_i = (sum mass*bias / sum mass) / bias_i; otherwise
// wcell = 1 (Eq. PIC weights).
void source_tables(const pic_params &p, const pic_stack_desc &s, const pic_pulse &u,
                   std::vector<uint32_t> &thr, std::vector<int32_t> &cell,
                   std::vector<int32_t> &layer, std::vector<long long> &inj,
                   std::vector<double> *wcell = nullptr)
{
    thr.clear(); cell.clear(); layer.clear();
    std::vector<double> mass;
    double total = 0.0;
    int c = 0;
    for (int l = 0; l < s.n_layers; ++l)
        for (int j = 0; j < s.layer_cells[l]; ++j, ++c) {
            if (!((u.excite_mask >> l) & 1u)) continue;
            const double z0 = (double)c * p.dz, w = p.dz;
            const double m = u.abs_len > 0.0
                                 ? u.abs_len * (std::exp(-z0 / u.abs_len) - std::exp(-(z0 + w) / u.abs_len))
                                 : w;
            mass.push_back(m); cell.push_back(c); layer.push_back(l);
            total += m;
        }
    double run = 0.0;
    const bool tilt = (p.flags & PIC_F_WEIGHTS) && u.cell_bias;
    if (wcell) wcell->assign(mass.size(), 1.0);
    if (tilt) {
        double total_b = 0.0;
        for (size_t i = 0; i < mass.size(); ++i) total_b += mass[i] * u.cell_bias[cell[i]];
        for (size_t i = 0; i < mass.size(); ++i) {
            run += mass[i] * u.cell_bias[cell[i]];
            thr.push_back(i + 1 == mass.size() ? 0xFFFFFFFFu : threshold_of(run / total_b));
            if (wcell) (*wcell)[i] = (total_b / total) / u.cell_bias[cell[i]];
        }
    } else {
        for (size_t i = 0; i < mass.size(); ++i) {
            run += mass[i];
            thr.push_back(i + 1 == mass.size() ? 0xFFFFFFFFu : threshold_of(run / total));
        }
    }
    const int64_t nh = 2 * (int64_t)p.n_steps_max;
    inj.assign((size_t)nh, 0);
    if (u.n0 <= 0 || mass.empty()) return;
    const double n0 = (double)u.n0;
    for (int64_t h = 0; h < nh; ++h) {
        const double ta = (double)h * 0.5 * (double)p.dt, tb = (double)(h + 1) * 0.5 * (double)p.dt;
        inj[h] = (long long)std::floor(n0 * pulse_fraction(u, tb)) -
                 (long long)std::floor(n0 * pulse_fraction(u, ta));
    }
}

bool valid_pulse(const pic_pulse *u, int n_layers, int n_e, std::string &why,
                 int n_cells = 0, uint32_t flags = 0)
{
    if (!u) { why = "pulse is NULL"; return false; }
    if (flags & PIC_F_WEIGHTS) {
        if (u->cell_bias)
            for (int i = 0; i < n_cells; ++i)
                if (!(u->cell_bias[i] > 0.0) || !std::isfinite(u->cell_bias[i])) {
                    why = "cell_bias must be finite and > 0"; return false;
                }
        if (u->e_bias)
            for (int k = 0; k < n_e; ++k)
                if (!(u->e_bias[k] > 0.0) || !std::isfinite(u->e_bias[k])) {
                    why = "e_bias must be finite and > 0"; return false;
                }
    }
    if (u->n0 < 0) { why = "n0 < 0"; return false; }
    if (u->n0 > 0 && !(u->fwhm > 0.0 && u->t0 > 0.0)) { why = "fwhm and t0 must be > 0"; return false; }
    if (!(u->abs_len >= 0.0)) { why = "abs_len < 0"; return false; }
    if (!(u->up_frac >= 0.0 && u->up_frac <= 1.0)) { why = "up_frac not in [0,1]"; return false; }
    if (u->e_mode != 0 && u->e_mode != 1) { why = "e_mode must be 0 or 1"; return false; }
    if (u->e_mode == 1 && (u->k_mono[0] < 1 || u->k_mono[0] > n_e || u->k_mono[1] < 1 || u->k_mono[1] > n_e)) {
        why = "k_mono out of range"; return false;
    }
    if (u->n0 > 0 && (u->excite_mask & ((1u << n_layers) - 1u)) == 0) { why = "no excited layer"; return false; }
    return true;
}

template <class T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

template <class T>
void release(T *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// Frees every device buffer of the context once; a failure here must not
// linger as the runtime's pending error for an unrelated later call.
void free_all(pic_ctx *c)
{
    for (cudaGraphExec_t &g : c->period_graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    if (c->persist_graph) cudaGraphExecDestroy(c->persist_graph);
    c->persist_graph = nullptr;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->cap_stream = nullptr;
    release(c->d_stacks); release(c->d_ent); release(c->d_fent); release(c->d_T);
    release(c->d_cdf_thr);
    release(c->d_cdf_cell); release(c->d_cdf_layer); release(c->d_inj);
    for (int b = 0; b < 2; ++b) {
        c->d_pk[b] = nullptr;                   // inside d_mu[b]
        release(c->d_z[b]); release(c->d_mu[b]); release(c->d_id[b]);
    }
    release(c->d_stage); release(c->d_bits); release(c->d_status); release(c->d_nh); release(c->d_gh); release(c->d_vh);
    release(c->d_qrec); release(c->d_qcnt); release(c->d_fspawn); release(c->d_J); release(c->d_cnt);
    release(c->d_bd); release(c->d_hnow);
    release(c->d_w[0]); release(c->d_w[1]); release(c->d_wcell); release(c->d_wbin);
    release(c->d_kthr); release(c->d_nhw); release(c->d_bdw); release(c->d_Jw); release(c->d_hnow_w);
    release(c->d_ctl);
    Replay &r = c->rp;
    for (int b = 0; b < 2; ++b) {
        r.pk[b] = nullptr;                      // inside r.mu[b]
        release(r.z[b]); release(r.mu[b]); release(r.id[b]); release(r.acc[b]);
    }
    release(r.stage_l); release(r.status); release(r.qcnt); release(r.fspawn); release(r.cnt); release(r.ctl); release(r.stacks);
    release(r.aent); release(r.aT); release(r.g_ent); release(r.g_T); release(r.gpot);
    release(r.gen_max); release(r.absmax); release(r.qgn); release(r.tot); release(r.parent);
    release(r.gen);
    r.ids_cap = 0;
    r.ready = false;
    cudaGetLastError();
}

// Launch one kernel through `fn`, bracketed by events when profiling.
template <class F>
cudaError_t timed(pic_ctx *c, int kind, F fn)
{
    if (!c->profiling) return fn();
    while (c->ev_used + 2 > c->ev_pool.size()) {
        cudaEvent_t ev;
        const cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        c->ev_pool.push_back(ev);
    }
    const size_t i = c->ev_used;
    cudaError_t e = cudaEventRecord(c->ev_pool[i], c->stream);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_pool[i + 1], c->stream);
    if (e == cudaSuccess) {
        c->ev_marks.push_back({kind, i});
        c->ev_used += 2;
    }
    return e;
}

pic_status device_status(pic_ctx *c)
{
    DevCtl h{};
    cudaError_t e = cudaMemcpyAsync(&h, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device status");
    if (h.status != 0) {
        const pic_status s = (pic_status)h.status;
        return fail(c, s, s == PIC_ERR_TIMEOUT    ? "a bounded device wait ran out"
                          : s == PIC_ERR_CAPACITY ? "capacity exceeded in strict mode"
                                                  : "the adjoint replay did not reproduce the forward run");
    }
    return PIC_OK;
}

}  // namespace

namespace pic {
void pic_set_static_error(const char *msg) { g_init_error = msg ? msg : ""; }
}

extern "C" {

const char *pic_status_string(pic_status s)
{
    return (s >= 0 && s <= PIC_ERR_STATE) ? kStatusNames[s] : "PIC_UNKNOWN";
}

const char *pic_last_error(const pic_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_init_error.empty() ? "no context" : g_init_error.c_str();
}

pic_status pic_derive_tables(const pic_params *p, const pic_stack_desc *stack,
                             const pic_tables *tables, const pic_pulse *pulse, uint32_t *P_thr,
                             uint32_t *Q_thr, uint32_t *T_thr, uint32_t *P0_thr, uint32_t *up_thr,
                             int64_t *inj_counts)
{
    std::string why;
    if (!valid_params(p, why) || !valid_stack(p, stack, tables, why)) return PIC_ERR_ARG;
    std::vector<uint32_t> P, Q, T, P0;
    material_thresholds(*p, *stack, *tables, P, Q, T, P0);
    if (P_thr) std::memcpy(P_thr, P.data(), P.size() * 4);
    if (Q_thr) std::memcpy(Q_thr, Q.data(), Q.size() * 4);
    if (T_thr && !T.empty()) std::memcpy(T_thr, T.data(), T.size() * 4);
    if (P0_thr) std::memcpy(P0_thr, P0.data(), P0.size() * 4);
    if (pulse) {
        if (!valid_pulse(pulse, stack->n_layers, p->n_e, why)) return PIC_ERR_ARG;
        if (up_thr) *up_thr = threshold_of(pulse->up_frac);
        std::vector<uint32_t> thr; std::vector<int32_t> cell, layer; std::vector<long long> inj;
        source_tables(*p, *stack, *pulse, thr, cell, layer, inj);
        if (inj_counts) for (size_t i = 0; i < inj.size(); ++i) inj_counts[i] = inj[i];
    }
    return PIC_OK;
}

pic_status pic_init(pic_ctx **out, const pic_params *p, const pic_stack_desc *stacks, int n_stacks,
                    const pic_tables *tables, void *cuda_stream)
{
    g_init_error.clear();
    if (!out) { g_init_error = "out is NULL"; return PIC_ERR_ARG; }
    *out = nullptr;
    std::string why;
    if (!valid_params(p, why)) { g_init_error = why; return PIC_ERR_ARG; }
    if (n_stacks < 1 || n_stacks > PIC_MAX_STACKS || !stacks || !tables) {
        g_init_error = "n_stacks out of range or NULL stacks/tables";
        return PIC_ERR_ARG;
    }
    if (p->stack_base + n_stacks > 65536) {
        g_init_error = "stack_base + n_stacks must not exceed 65536";
        return PIC_ERR_ARG;
    }
    for (int s = 0; s < n_stacks; ++s)
        if (!valid_stack(p, &stacks[s], &tables[s], why)) {
            g_init_error = "stack " + std::to_string(s) + ": " + why;
            return PIC_ERR_ARG;
        }

    pic_ctx *c = new pic_ctx();
    c->p = *p;
    c->n_stacks = n_stacks;
    c->stream = (cudaStream_t)cuda_stream;
    c->hs.resize(n_stacks);
    c->ds.resize(n_stacks);
    const int ne = p->n_e;
    // the streaming pass's table: 2^kb entries per (layer, spin), kb the
    // smallest power of two above n_e, so that the packed word indexes it
    int kb = 0;
    while ((1 << kb) < ne + 1) ++kb;
    const int KP = 1 << kb;
    const float inf = std::numeric_limits<float>::infinity();
    const FastEnt inert{0.f, 0u, -inf, inf};
    int tab_max = 1, T_max = 1, nbin_max = 1, jbin_max = 1, ftab_max = 1;
    std::vector<TabEnt> ent;
    std::vector<FastEnt> fent;
    std::vector<uint32_t> Tall;
    for (int s = 0; s < n_stacks; ++s) {
        HostStack &h = c->hs[s];
        const pic_tables &t = tables[s];
        h.d = stacks[s];
        h.n_mat = t.n_mat;
        const size_t nt = (size_t)t.n_mat * 2 * ne;
        h.v.assign(t.v, t.v + nt);
        h.tau_in.assign(t.tau_in, t.tau_in + nt);
        h.tau_el.assign(t.tau_el, t.tau_el + t.n_mat);
        h.p0.assign(t.p0, t.p0 + t.n_mat);
        h.T.assign(t.T ? t.T : nullptr, t.T ? t.T + (size_t)(h.d.n_layers - 1) * 4 * ne : nullptr);
        material_thresholds(*p, h.d, t, h.P_thr, h.Q_thr, h.T_thr, h.P0_thr);
        DevStack &d = c->ds[s];
        std::memset(&d, 0, sizeof(d));
        d.n_layers = h.d.n_layers;
        int cells = 0;
        d.edge[0] = 0.f;
        for (int l = 0; l < h.d.n_layers; ++l) {
            cells += h.d.layer_cells[l];
            d.edge[l + 1] = (float)cells * p->dz;
            d.p0_thr[l] = h.P0_thr[h.d.layer_mat[l]];
        }
        h.n_cells = d.n_cells = cells;
        h.n_out = (p->n_steps_max + p->moment_every - 1) / p->moment_every;
        // layer-indexed {v, P, Q} entries
        d.tab_n = h.d.n_layers * 2 * ne;
        d.ent_off = (int64_t)ent.size();
        d.ftab_n = h.d.n_layers * 2 * KP;
        d.fent_off = (int64_t)fent.size();
        for (int l = 0; l < h.d.n_layers; ++l)
            for (int sp = 0; sp < 2; ++sp) {
                fent.push_back(inert);                       // k = 0: a removed carrier
                for (int k = 0; k < ne; ++k) {
                    const size_t i = ((size_t)h.d.layer_mat[l] * 2 + sp) * ne + k;
                    ent.push_back(TabEnt{h.v[i], h.P_thr[i], h.Q_thr[i], 0u});
                    fent.push_back(FastEnt{h.v[i], h.P_thr[i], d.edge[l], d.edge[l + 1]});
                }
                for (int k = ne + 1; k < KP; ++k) fent.push_back(inert);
            }
        d.T_n = (h.d.n_layers - 1) * 4 * ne;
        d.T_off = (int64_t)Tall.size();
        Tall.insert(Tall.end(), h.T_thr.begin(), h.T_thr.end());
        d.cap = h.d.capacity;
        h.cap_round = (h.d.capacity + TILE - 1) / TILE * TILE;
        d.base = h.base = c->total_slots;
        c->total_slots += h.cap_round;
        d.n_off = c->nh_total;
        c->nh_total += (int64_t)h.n_out * 2 * ne * cells;
        d.J_off = c->J_total;
        c->J_total += (int64_t)h.n_out * 2 * (cells + 1);
        d.cdf_off = (int64_t)s * 0;      // set by pic_excite
        d.n_cdf = 0;
        d.inj_off = (int64_t)s * 2 * p->n_steps_max;
        tab_max = std::max(tab_max, d.tab_n);
        ftab_max = std::max(ftab_max, d.ftab_n);
        T_max = std::max(T_max, d.T_n);
        nbin_max = std::max(nbin_max, 2 * ne * cells);
        jbin_max = std::max(jbin_max, 2 * (cells + 1));
        h.inj.assign((size_t)2 * p->n_steps_max, 0);
    }
    c->n_ent = ent.size();
    c->n_T = Tall.size();
    for (int s = 0; s < n_stacks; ++s) c->n_mat_max = std::max(c->n_mat_max, c->hs[s].n_mat);
    c->init_recs.assign(n_stacks, {});
    c->init_next_id.assign(n_stacks, 0);
    if (c->total_slots >= (int64_t(1) << 32)) {
        g_init_error = "total capacity of a context must stay below 2^32 slots";
        delete c;
        return PIC_ERR_ARG;
    }
    int64_t total_cells = 0;
    for (int s = 0; s < n_stacks; ++s) {
        c->ds[s].cdf_off = total_cells;
        total_cells += c->hs[s].n_cells;
        c->ncm = std::max(c->ncm, c->hs[s].n_cells);
    }

    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n) do { if (e == cudaSuccess) e = dalloc(&ptr, n); } while (0)
    ALLOC(c->d_stacks, n_stacks);
    ALLOC(c->d_ent, ent.size());
    ALLOC(c->d_fent, fent.size());
    ALLOC(c->d_T, Tall.size());
    ALLOC(c->d_cdf_thr, total_cells);
    ALLOC(c->d_cdf_cell, total_cells);
    ALLOC(c->d_cdf_layer, total_cells);
    ALLOC(c->d_inj, (size_t)n_stacks * 2 * p->n_steps_max);
    for (int b = 0; b < 2; ++b) {
        ALLOC(c->d_z[b], c->total_slots);
        ALLOC(c->d_mu[b], 2 * c->total_slots);     // (mu, packed) pairs
        ALLOC(c->d_id[b], c->total_slots);
        if (e == cudaSuccess) c->d_pk[b] = reinterpret_cast<uint32_t *>(c->d_mu[b]) + 1;
    }
    ALLOC(c->d_stage, c->total_slots);
    ALLOC(c->d_bits, c->total_slots / 32 + 1);
    ALLOC(c->d_qrec, c->total_slots);
    ALLOC(c->d_nh, c->nh_total);
    ALLOC(c->d_gh, c->nh_total / (2 * p->n_e) + 1);
    ALLOC(c->d_vh, c->nh_total / p->n_e + 1);
    ALLOC(c->d_J, c->J_total);
    ALLOC(c->d_bd, c->J_total);
    if (p->flags & PIC_F_WEIGHTS) {
        ALLOC(c->d_w[0], c->total_slots);
        ALLOC(c->d_w[1], c->total_slots);
        ALLOC(c->d_wcell, total_cells);
        ALLOC(c->d_wbin, (size_t)n_stacks * ne);
        ALLOC(c->d_kthr, (size_t)n_stacks * ne);
        ALLOC(c->d_nhw, c->nh_total);
        ALLOC(c->d_bdw, c->J_total);
        ALLOC(c->d_Jw, c->J_total);
        ALLOC(c->d_hnow_w, (size_t)n_stacks * 2 * (c->ncm + 1));
    }
    ALLOC(c->d_hnow, (size_t)n_stacks * 2 * (c->ncm + 1));
    ALLOC(c->d_cnt, n_stacks);
    ALLOC(c->d_ctl, 1);
#undef ALLOC
    if (e != cudaSuccess) {
        g_init_error = std::string("device allocation: ") + cudaGetErrorString(e);
        free_all(c);
        delete c;
        cudaGetLastError();
        return PIC_ERR_ALLOC;
    }

    Args &a = c->args;
    a.stacks = c->d_stacks; a.n_stacks = n_stacks;
    a.ent = c->d_ent; a.fent = c->d_fent; a.T_thr = c->d_T;
    a.cdf_thr = c->d_cdf_thr; a.cdf_cell = c->d_cdf_cell; a.cdf_layer = c->d_cdf_layer;
    a.inj = c->d_inj;
    for (int b = 0; b < 2; ++b) {
        a.z[b] = c->d_z[b]; a.mu[b] = c->d_mu[b]; a.id[b] = c->d_id[b]; a.pk[b] = c->d_pk[b];
        a.mp_stride = 2;
    }
    a.stage = c->d_stage;
    a.spawn_bits = c->d_bits;
    a.qrec = c->d_qrec;
    a.n_hist = c->d_nh; a.J_hist = c->d_J; a.cnt = c->d_cnt; a.ctl = c->d_ctl;
    a.bd_hist = c->d_bd;
    a.w[0] = c->d_w[0]; a.w[1] = c->d_w[1];
    a.wcell = c->d_wcell; a.wbin = c->d_wbin; a.kthr = c->d_kthr;
    a.nhw = c->d_nhw; a.bdw = c->d_bdw; a.Jw = c->d_Jw;
    a.kb = kb;
    a.kshr = 8 - kb;
    a.kmask = (uint32_t)KP - 1u;
    a.hmask = 0x1Fu << kb;
    a.g_hist = c->d_gh;
    a.v_hist = c->d_vh;
    a.seed_lo = (uint32_t)p->seed; a.seed_hi = (uint32_t)(p->seed >> 32);
    a.stack_base = p->stack_base;
    for (int r = 0; r < 10; ++r) {      // Philox4x32-10 round keys (Weyl sequence)
        a.rk0[r] = a.seed_lo + (uint32_t)r * 0x9E3779B9u;
        a.rk1[r] = a.seed_hi + (uint32_t)r * 0xBB67AE85u;
    }
    a.half_dt = p->dt * 0.5f;
    a.dz = p->dz;
    a.dz_pow2 = 1;
    a.inv_dz = 1.0f / p->dz;      // exact: dz is a power of two
    a.flags = p->flags; a.n_e = ne; a.moment_every = p->moment_every;
    a.compact_every = p->compact_every;
    a.step = 0;
    a.tab_max = tab_max; a.T_max = T_max; a.nbin_max = nbin_max; a.jbin_max = jbin_max;
    a.ftab_max = ftab_max;
    a.gbin_max = nbin_max / (2 * ne);
    a.spin_limit = 1u << 24;

    e = configure(a, p->blocks_per_sm, p->ring_stages, p->hist_mode, p->consumer_warps, &c->lc);
    if (p->event_pass == 1) c->lc.grid_fused = 0;
    if (e != cudaSuccess) {
        g_init_error = std::string("kernel configuration (moment grid too large for shared "
                                   "memory, or no device): ") + cudaGetErrorString(e);
        free_all(c);
        delete c;
        cudaGetLastError();
        return PIC_ERR_ARG;   // moment grid too large for shared memory, or no device
    }
    // look-back words and per-block counts for the largest grid any launch
    // configuration (pic_autotune's included) can give
    int sms_now = 0, dev_now = 0;
    cudaGetDevice(&dev_now);
    cudaDeviceGetAttribute(&sms_now, cudaDevAttrMultiProcessorCount, dev_now);
    const int gmax = std::max({c->lc.grid_fast, c->lc.grid_fast_dep, c->lc.grid_slow,
                               c->lc.grid_slow_dep, c->lc.grid_place, c->lc.grid_place_dep,
                               c->lc.grid_compact, 16 * sms_now});
    c->n_status = gmax;
    if (dalloc(&c->d_status, (size_t)gmax) != cudaSuccess ||
        dalloc(&c->d_qcnt, (size_t)gmax) != cudaSuccess ||
        dalloc(&c->d_fspawn, (size_t)gmax) != cudaSuccess) {
        g_init_error = "device allocation of the look-back words";
        free_all(c);
        delete c;
        cudaGetLastError();
        return PIC_ERR_ALLOC;
    }
    a.status = c->d_status;
    a.qcnt = c->d_qcnt;
    a.fspawn = c->d_fspawn;

    cudaStream_t st = c->stream;
    DevCtl ctl{};
    ctl.epoch = 1u;
    std::vector<DevCounters> cnt(n_stacks);
    std::memset(cnt.data(), 0, sizeof(DevCounters) * n_stacks);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_stacks, c->ds.data(), sizeof(DevStack) * n_stacks, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !ent.empty()) e = cudaMemcpyAsync(c->d_ent, ent.data(), sizeof(TabEnt) * ent.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !fent.empty()) e = cudaMemcpyAsync(c->d_fent, fent.data(), sizeof(FastEnt) * fent.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !Tall.empty()) e = cudaMemcpyAsync(c->d_T, Tall.data(), 4 * Tall.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_inj, 0, sizeof(long long) * std::max<size_t>((size_t)n_stacks * 2 * p->n_steps_max, 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned long long) * gmax, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_fspawn, 0, sizeof(uint32_t) * gmax, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bits, 0, 4 * (size_t)(c->total_slots / 32 + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_nh, 0, 4 * (size_t)std::max<int64_t>(c->nh_total, 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gh, 0, 8 * (size_t)(c->nh_total / (2 * p->n_e) + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_vh, 0, 8 * (size_t)(c->nh_total / p->n_e + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_J, 0, 4 * (size_t)std::max<int64_t>(c->J_total, 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bd, 0, 4 * (size_t)std::max<int64_t>(c->J_total, 1), st);
    std::vector<double> ones((size_t)std::max<int64_t>(total_cells, (int64_t)n_stacks * ne), 1.0);
    if (p->flags & PIC_F_WEIGHTS) {
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_nhw, 0, 8 * (size_t)std::max<int64_t>(c->nh_total, 1), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bdw, 0, 8 * (size_t)std::max<int64_t>(c->J_total, 1), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_Jw, 0, 8 * (size_t)std::max<int64_t>(c->J_total, 1), st);
        if (e == cudaSuccess && total_cells) e = cudaMemcpyAsync(c->d_wcell, ones.data(), 8 * (size_t)total_cells, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_wbin, ones.data(), 8 * (size_t)n_stacks * ne, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cnt, cnt.data(), sizeof(DevCounters) * n_stacks, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_init_error = std::string("initial upload: ") + cudaGetErrorString(e);
        free_all(c);
        delete c;
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    *out = c;
    return PIC_OK;
}

pic_status pic_excite(pic_ctx *c, int stack, const pic_pulse *u)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < -1 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    const int s0 = stack < 0 ? 0 : stack, s1 = stack < 0 ? c->n_stacks : stack + 1;
    std::string why;
    for (int s = s0; s < s1; ++s)
        if (!valid_pulse(u, c->hs[s].d.n_layers, c->p.n_e, why, c->hs[s].n_cells, c->p.flags))
            return fail(c, PIC_ERR_ARG, why);
    if (c->step > 0) {
        c->replayable = false;
        c->replay_why = "pic_grad: the source changed after step 0";
    }
    for (int s = s0; s < s1; ++s) {
        HostStack &h = c->hs[s];
        DevStack &d = c->ds[s];
        std::vector<uint32_t> thr; std::vector<int32_t> cell, layer;
        std::vector<double> wcell;
        source_tables(c->p, h.d, *u, thr, cell, layer, h.inj, &wcell);
        h.pulse = *u;
        h.pulse.cell_bias = nullptr;      // not kept: the tables are
        h.pulse.e_bias = nullptr;
        h.bias_hash = fnv1a(u->cell_bias, u->cell_bias ? 8 * (size_t)h.n_cells : 0,
                            fnv1a(u->e_bias, u->e_bias ? 8 * (size_t)c->p.n_e : 0));
        h.excited = true;
        d.n_cdf = (int32_t)thr.size();
        d.up_thr = threshold_of(u->up_frac);
        d.e_mode = u->e_mode;
        d.k_mono0 = u->k_mono[0];
        d.k_mono1 = u->k_mono[1];
        cudaError_t e = cudaSuccess;
        if (!thr.empty()) {
            e = cudaMemcpyAsync(c->d_cdf_thr + d.cdf_off, thr.data(), 4 * thr.size(), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cdf_cell + d.cdf_off, cell.data(), 4 * cell.size(), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cdf_layer + d.cdf_off, layer.data(), 4 * layer.size(), cudaMemcpyHostToDevice, c->stream);
        }
        if (e == cudaSuccess && !h.inj.empty())
            e = cudaMemcpyAsync(c->d_inj + d.inj_off, h.inj.data(), sizeof(long long) * h.inj.size(), cudaMemcpyHostToDevice, c->stream);
        // importance sampling of the birth bin: q_k proportional to bias_k,
        // weight p_k / q_k = (sum bias / n_e) / bias_k (e_mode 0)
        const int ne = c->p.n_e;
        std::vector<uint32_t> kthr(ne, 0u);
        std::vector<double> wbin(ne, 1.0);
        d.has_ebias = ((c->p.flags & PIC_F_WEIGHTS) && u->e_bias && u->e_mode == 0) ? 1 : 0;
        if (d.has_ebias) {
            double tb = 0.0, cb = 0.0;
            for (int k = 0; k < ne; ++k) tb += u->e_bias[k];
            for (int k = 0; k < ne; ++k) {
                cb += u->e_bias[k];
                kthr[k] = k == ne - 1 ? 0xFFFFFFFFu : threshold_of(cb / tb);
                wbin[k] = (tb / (double)ne) / u->e_bias[k];
            }
        }
        if (e == cudaSuccess && (c->p.flags & PIC_F_WEIGHTS)) {
            if (!wcell.empty())
                e = cudaMemcpyAsync(c->d_wcell + d.cdf_off, wcell.data(), 8 * wcell.size(), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->d_wbin + (size_t)s * ne, wbin.data(), 8 * (size_t)ne, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->d_kthr + (size_t)s * ne, kthr.data(), 4 * (size_t)ne, cudaMemcpyHostToDevice, c->stream);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_stacks + s, &d, sizeof(DevStack), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "pic_excite upload");
    }
    return PIC_OK;
}

namespace {

// The kernels of time step s (Eq. strang): source half step, the streaming
// and event passes, the second source half step, compaction.  `graph`: the
// step is being captured; the source kernels run whatever the counts (they
// read them on the device) and the step's last kernel advances the device
// step counter.
cudaError_t enqueue_step(pic_ctx *c, const Args &a0, int s, bool inj0, bool inj1, bool graph,
                         cudaStream_t st, int64_t &launches)
{
    const bool det = (c->p.flags & PIC_F_DETERMINISTIC) != 0;
    const bool dep = ((s + 1) % c->p.moment_every) == 0;
    const LaunchCfg &lc = c->lc;
    Args a = a0;
    a.step = (uint32_t)s;
    a.bump_step = 0;
    cudaError_t e = cudaSuccess;
    if (inj0) {
        e = timed(c, 0, [&] { return launch_inject(a, lc, 0, false, st); });
        ++launches;
    }
    if (!dep && lc.grid_fused > 0) {
        // the fused form: the streaming pass runs the general step too
        if (e == cudaSuccess) {
            e = timed(c, 1, [&] { return launch_fused(a, lc, det, st); });
            ++launches;
        }
        if (e == cudaSuccess) {
            Args b = a;
            b.bump_step = graph && !inj1;
            e = timed(c, 4, [&] { return launch_place_fused(b, lc, det, st); });
            ++launches;
        }
    } else {
        if (e == cudaSuccess) {
            e = timed(c, dep ? 2 : 1, [&] { return launch_fast(a, lc, det, dep, c->p.hist_mode, st); });
            ++launches;
        }
        if (e == cudaSuccess) {
            Args b = a;
            b.bump_step = graph && !inj1;
            e = timed(c, 4, [&] { return launch_slow(b, lc, det, dep, st); });
            launches += 2;               // the event and placement passes
        }
    }
    if (e == cudaSuccess && inj1) {
        Args b = a;
        b.bump_step = graph;
        e = timed(c, 0, [&] { return launch_inject(b, lc, 1, dep, st); });
        ++launches;
    }
    if (e == cudaSuccess && dep && (c->p.flags & PIC_F_WEIGHTS)) {
        e = timed(c, 9, [&] { return launch_wdep(a, lc, st); });
        ++launches;
    }
    if (e == cudaSuccess && ((s + 1) % c->p.compact_every) == 0) {
        e = timed(c, 3, [&] { return launch_compact(a, lc, st); });
        ++launches;
    }
    return e;
}

bool any_source(const pic_ctx *c, int s0, int n)
{
    for (const HostStack &h : c->hs)
        for (int64_t i = 2 * (int64_t)s0; i < 2 * (int64_t)(s0 + n); ++i)
            if (h.inj[(size_t)i] > 0) return true;
    return false;
}

// Capture one period of steps (starting at a step that is a multiple of the
// period) into a graph; with_source: the source kernels of every half step.
cudaError_t capture_period(pic_ctx *c, int which)
{
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    Args a = c->args;
    a.step_dev = &c->d_ctl->step;
    const bool src = which == 0;
    cudaGraph_t g = nullptr;
    int64_t n = 0;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < c->period && e == cudaSuccess; ++i)
        e = enqueue_step(c, a, i, src, src, true, c->cap_stream, n);
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->period_graph[which], g, 0);
    if (g) cudaGraphDestroy(g);
    c->period_launches[which] = n;
    return e;
}

int gcd_int(int x, int y) { return y ? gcd_int(y, x % y) : x; }

// The fluxes of every window reached so far, from the densities and the
// births-minus-removals histograms (k_flux): windows that have ended are
// computed once; the running window (if any) is computed from a count of the
// current state each time it is asked for.
cudaError_t derive_fluxes(pic_ctx *c)
{
    const int me = c->p.moment_every, n_out = c->hs[0].n_out;
    const int ended = std::min(c->step / me, n_out);
    cudaError_t e = cudaSuccess;
    if (c->flux_final < ended) {
        e = timed(c, 8, [&] { return launch_flux(c->args, c->flux_final, ended, -1, nullptr, c->ncm, c->stream); });
        if (e != cudaSuccess) return e;
        c->flux_final = ended;
    }
    if (c->step % me != 0 && ended < n_out) {
        e = cudaMemsetAsync(c->d_hnow, 0, sizeof(int32_t) * (size_t)c->n_stacks * 2 * (c->ncm + 1), c->stream);
        if (e == cudaSuccess)
            e = timed(c, 8, [&] { return launch_state_hist(c->args, 0, c->n_stacks, 1, 0, 1, c->d_hnow, c->ncm, c->stream); });
        if (e == cudaSuccess)
            e = timed(c, 8, [&] { return launch_flux(c->args, ended, ended + 1, ended, c->d_hnow, c->ncm, c->stream); });
    }
    return e;
}

// The weighted fluxes, as derive_fluxes, from the weighted densities and
// the weighted births minus removals.
cudaError_t derive_fluxes_w(pic_ctx *c)
{
    const int me = c->p.moment_every, n_out = c->hs[0].n_out;
    const int ended = std::min(c->step / me, n_out);
    cudaError_t e = cudaSuccess;
    if (c->flux_final_w < ended) {
        e = timed(c, 8, [&] { return launch_flux_w(c->args, c->flux_final_w, ended, -1, nullptr, c->ncm, c->stream); });
        if (e != cudaSuccess) return e;
        c->flux_final_w = ended;
    }
    if (c->step % me != 0 && ended < n_out) {
        e = cudaMemsetAsync(c->d_hnow_w, 0, sizeof(long long) * (size_t)c->n_stacks * 2 * (c->ncm + 1), c->stream);
        if (e == cudaSuccess)
            e = timed(c, 8, [&] { return launch_state_hist_w(c->args, 0, c->n_stacks, 1, 0, 1, c->d_hnow_w, c->ncm, c->stream); });
        if (e == cudaSuccess)
            e = timed(c, 8, [&] { return launch_flux_w(c->args, ended, ended + 1, ended, c->d_hnow_w, c->ncm, c->stream); });
    }
    return e;
}

}  // namespace

pic_status pic_step(pic_ctx *c, int n_steps)
{
    if (!c) return PIC_ERR_ARG;
    if (n_steps < 0) return fail(c, PIC_ERR_ARG, "n_steps < 0");
    if ((int64_t)c->step + n_steps > c->p.n_steps_max)
        return fail(c, PIC_ERR_ARG, "steps would exceed n_steps_max");
    c->launches = 0;
    const bool persist = c->p.use_graph == 2 && !c->profiling;
    const bool graphs = (c->p.use_graph == 1 || persist) && !c->profiling;
    if (graphs && c->period == 0) {
        const int me = c->p.moment_every, ce = c->p.compact_every;
        const long long l = (long long)me / gcd_int(me, ce) * ce;
        c->period = l <= 100000 ? (int)l : -1;      // -1: no graphs for this context
    }
    int left = n_steps;
    while (left > 0) {
        const int s = c->step;
        cudaError_t e = cudaSuccess;
        if (persist && c->period > 0 && s % c->period == 0 && left >= c->period) {
            // one cooperative launch runs the whole period (captured in a
            // graph once; the kernel reads and advances the device step)
            if (!c->pcfg.ok) {
                e = configure_persistent(c->args, (c->p.flags & PIC_F_DETERMINISTIC) != 0, &c->pcfg);
                if (e != cudaSuccess) return cuda_fail(c, e, "pic_step persistent configuration");
                if (c->pcfg.grid > c->n_status)
                    return fail(c, PIC_ERR_CUDA, "pic_step: persistent grid larger than the look-back words");
            }
            Args a = c->args;
            a.step_dev = &c->d_ctl->step;
            const bool det = (c->p.flags & PIC_F_DETERMINISTIC) != 0;
            if (!c->persist_graph && !c->persist_direct) {
                if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
                cudaGraph_t g = nullptr;
                if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e1 = launch_persistent(a, c->pcfg, det, c->period, c->cap_stream);
                    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
                    if (e1 == cudaSuccess && e2 == cudaSuccess)
                        e1 = cudaGraphInstantiate(&c->persist_graph, g, 0);
                    if (g) cudaGraphDestroy(g);
                    if (e1 != cudaSuccess || e2 != cudaSuccess) {
                        cudaGetLastError();               // not capturable here: launch directly
                        c->persist_graph = nullptr;
                        c->persist_direct = true;
                    }
                }
                if (e != cudaSuccess) return cuda_fail(c, e, "pic_step persistent capture");
            }
            if (!c->dev_step_valid) {
                e = launch_set_step(c->d_ctl, (unsigned int)s, c->stream);
                c->launches += 1;
            }
            if (e == cudaSuccess)
                e = c->persist_graph ? cudaGraphLaunch(c->persist_graph, c->stream)
                                     : launch_persistent(a, c->pcfg, det, c->period, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "pic_step persistent launch");
            c->dev_step_valid = true;
            c->launches += 1;
            c->step = s + c->period;
            left -= c->period;
            continue;
        }
        if (graphs && !persist && c->period > 0 && s % c->period == 0 && left >= c->period) {
            const int which = any_source(c, s, c->period) ? 0 : 1;
            if (!c->period_graph[which]) {
                e = capture_period(c, which);
                if (e != cudaSuccess) return cuda_fail(c, e, "pic_step graph capture");
            }
            if (!c->dev_step_valid) {
                e = launch_set_step(c->d_ctl, (unsigned int)s, c->stream);
                c->launches += 1;
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(c->period_graph[which], c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "pic_step graph launch");
            c->dev_step_valid = true;
            c->launches += c->period_launches[which];
            c->step = s + c->period;
            left -= c->period;
            continue;
        }
        bool inj0 = false, inj1 = false;
        for (const HostStack &h : c->hs) {
            inj0 = inj0 || h.inj[2 * (size_t)s] > 0;
            inj1 = inj1 || h.inj[2 * (size_t)s + 1] > 0;
        }
        e = enqueue_step(c, c->args, s, inj0, inj1, false, c->stream, c->launches);
        if (e != cudaSuccess) return cuda_fail(c, e, "pic_step launch");
        c->dev_step_valid = false;
        c->step = s + 1;
        --left;
    }
    return PIC_OK;
}

namespace {

// What a checkpoint must match: the parameters that define the run (not the
// launch configuration), the stacks, their tables and their excitation.
uint64_t fingerprint(const pic_ctx *c)
{
    pic_params p = c->p;
    p.blocks_per_sm = 0; p.hist_mode = 0; p.ring_stages = 0; p.use_graph = 0; p.consumer_warps = 0;
    p.event_pass = 0;
    uint64_t h = fnv1a(&p, sizeof(p));
    h = fnv1a(&c->n_stacks, sizeof(c->n_stacks), h);
    for (const HostStack &s : c->hs) {
        h = fnv1a(&s.d, sizeof(s.d), h);
        h = fnv1a(s.v.data(), 4 * s.v.size(), h);
        h = fnv1a(s.tau_in.data(), 8 * s.tau_in.size(), h);
        h = fnv1a(s.tau_el.data(), 8 * s.tau_el.size(), h);
        h = fnv1a(s.T.data(), 8 * s.T.size(), h);
        h = fnv1a(s.p0.data(), 8 * s.p0.size(), h);
        h = fnv1a(s.inj.data(), 8 * s.inj.size(), h);
        pic_pulse u = s.pulse;
        u.cell_bias = nullptr; u.e_bias = nullptr;
        h = fnv1a(&u, sizeof(u), h);
        h = fnv1a(&s.bias_hash, 8, h);
    }
    return h;
}

constexpr uint64_t kSaveMagic = 0x3130455641534950ull;   // "PISAVE01"

struct SaveHeader {
    uint64_t magic, fingerprint, bytes;
    int32_t step, n_stacks, replayable, pad;
};

// The device arrays a checkpoint holds besides the particle slots, as
// (pointer, bytes) pairs, in a fixed order.
std::vector<std::pair<void *, size_t>> moment_arrays(pic_ctx *c)
{
    std::vector<std::pair<void *, size_t>> v;
    const size_t ng = (size_t)(c->nh_total / (2 * c->p.n_e) + 1);
    v.push_back({c->d_nh, 4 * (size_t)c->nh_total});
    v.push_back({c->d_bd, 4 * (size_t)c->J_total});
    v.push_back({c->d_gh, 8 * ng});
    if (c->p.flags & PIC_F_VELOCITY_MOMENTS) v.push_back({c->d_vh, 8 * (size_t)(c->nh_total / c->p.n_e + 1)});
    if (c->p.flags & PIC_F_WEIGHTS) {
        v.push_back({c->d_nhw, 8 * (size_t)c->nh_total});
        v.push_back({c->d_bdw, 8 * (size_t)c->J_total});
    }
    return v;
}

}  // namespace

pic_status pic_save(pic_ctx *c, void *buf, size_t *bytes)
{
    if (!c || !bytes) return PIC_ERR_ARG;
    const pic_status st0 = device_status(c);
    if (st0 != PIC_OK) return st0;
    const int S = c->n_stacks;
    const bool wts = (c->p.flags & PIC_F_WEIGHTS) != 0;
    std::vector<DevCounters> cnt(S);
    DevCtl ctl{};
    cudaError_t e = cudaMemcpyAsync(cnt.data(), c->d_cnt, sizeof(DevCounters) * S, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_save");
    const auto arrays = moment_arrays(c);
    size_t need = sizeof(SaveHeader) + sizeof(DevCounters) * S;
    for (int s = 0; s < S; ++s) {
        need += (size_t)cnt[s].n_slots * (sizeof(pic_record) + (wts ? 4 : 0));
        need += 16 + c->init_recs[s].size() * sizeof(pic_record);
    }
    for (const auto &x : arrays) need += x.second;
    if (!buf) { *bytes = need; return PIC_OK; }
    if (*bytes < need) { *bytes = need; return fail(c, PIC_ERR_ARG, "pic_save: buffer too small"); }
    unsigned char *o = static_cast<unsigned char *>(buf);
    SaveHeader hd{kSaveMagic, fingerprint(c), need, c->step, S, c->replayable ? 1 : 0, 0};
    std::memcpy(o, &hd, sizeof(hd)); o += sizeof(hd);
    std::memcpy(o, cnt.data(), sizeof(DevCounters) * S); o += sizeof(DevCounters) * S;
    for (int s = 0; s < S && e == cudaSuccess; ++s) {
        const int64_t n = (int64_t)cnt[s].n_slots, base = c->ds[s].base;
        std::vector<float> z(n);
        std::vector<uint32_t> id(n), mp(2 * n);
        if (n) {
            e = cudaMemcpyAsync(z.data(), c->d_z[ctl.cur] + base, 4 * n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(mp.data(), c->d_mu[ctl.cur] + 2 * base, 8 * n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(id.data(), c->d_id[ctl.cur] + base, 4 * n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess && wts)
                e = cudaMemcpyAsync(o + n * sizeof(pic_record), c->d_w[ctl.cur] + base, 4 * n, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        }
        for (int64_t i = 0; i < n; ++i) {
            pic_record r;
            r.z = z[i];
            std::memcpy(&r.mu, &mp[2 * i], 4);
            r.packed = mp[2 * i + 1];
            r.id = id[i];
            std::memcpy(o + i * sizeof(pic_record), &r, sizeof(r));
        }
        o += n * (sizeof(pic_record) + (wts ? 4 : 0));
        const uint64_t ni = c->init_recs[s].size(), nid = c->init_next_id[s];
        std::memcpy(o, &ni, 8); std::memcpy(o + 8, &nid, 8); o += 16;
        if (ni) std::memcpy(o, c->init_recs[s].data(), ni * sizeof(pic_record));
        o += ni * sizeof(pic_record);
    }
    for (const auto &x : arrays) {
        if (e == cudaSuccess && x.second) e = cudaMemcpyAsync(o, x.first, x.second, cudaMemcpyDeviceToHost, c->stream);
        o += x.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_save copy");
    *bytes = need;
    return PIC_OK;
}

pic_status pic_load(pic_ctx *c, const void *buf, size_t bytes)
{
    if (!c || !buf) return PIC_ERR_ARG;
    const int S = c->n_stacks;
    const bool wts = (c->p.flags & PIC_F_WEIGHTS) != 0;
    SaveHeader hd{};
    if (bytes < sizeof(hd)) return fail(c, PIC_ERR_ARG, "pic_load: not a checkpoint");
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kSaveMagic || hd.bytes != bytes || hd.n_stacks != S)
        return fail(c, PIC_ERR_ARG, "pic_load: not a checkpoint of this size");
    if (hd.fingerprint != fingerprint(c))
        return fail(c, PIC_ERR_ARG, "pic_load: the checkpoint belongs to other parameters, stacks, tables or excitation");
    if (hd.step < 0 || hd.step > c->p.n_steps_max) return fail(c, PIC_ERR_ARG, "pic_load: step out of range");
    const unsigned char *o = static_cast<const unsigned char *>(buf) + sizeof(hd);
    std::vector<DevCounters> cnt(S);
    std::memcpy(cnt.data(), o, sizeof(DevCounters) * S); o += sizeof(DevCounters) * S;
    const auto arrays = moment_arrays(c);
    size_t need = sizeof(SaveHeader) + sizeof(DevCounters) * S;
    {
        const unsigned char *q = o;
        for (int s = 0; s < S; ++s) {
            if (cnt[s].n_slots > (unsigned long long)c->hs[s].d.capacity)
                return fail(c, PIC_ERR_ARG, "pic_load: more slots than the capacity");
            const size_t rb = (size_t)cnt[s].n_slots * (sizeof(pic_record) + (wts ? 4 : 0));
            need += rb + 16;
            if (need > bytes) return fail(c, PIC_ERR_ARG, "pic_load: truncated checkpoint");
            q += rb;
            uint64_t ni = 0;
            std::memcpy(&ni, q, 8);
            if (ni > (uint64_t)c->hs[s].d.capacity) return fail(c, PIC_ERR_ARG, "pic_load: bad initial records");
            need += ni * sizeof(pic_record);
            q += 16 + ni * sizeof(pic_record);
        }
        for (const auto &x : arrays) need += x.second;
        if (need != bytes) return fail(c, PIC_ERR_ARG, "pic_load: checkpoint size does not match");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    DevCtl ctl{};
    ctl.epoch = 1u;                       // fresh look-back words, particle buffer 0
    for (int s = 0; s < S && e == cudaSuccess; ++s) {
        const int64_t n = (int64_t)cnt[s].n_slots, base = c->ds[s].base;
        std::vector<float> z(n);
        std::vector<uint32_t> id(n), mp(2 * n);
        for (int64_t i = 0; i < n; ++i) {
            pic_record r;
            std::memcpy(&r, o + i * sizeof(pic_record), sizeof(r));
            z[i] = r.z;
            std::memcpy(&mp[2 * i], &r.mu, 4);
            mp[2 * i + 1] = r.packed;
            id[i] = r.id;
        }
        if (n) {
            e = cudaMemcpyAsync(c->d_z[0] + base, z.data(), 4 * n, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mu[0] + 2 * base, mp.data(), 8 * n, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_id[0] + base, id.data(), 4 * n, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess && wts)
                e = cudaMemcpyAsync(c->d_w[0] + base, o + n * sizeof(pic_record), 4 * n, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);      // host vectors go out of scope
        }
        o += n * (sizeof(pic_record) + (wts ? 4 : 0));
        uint64_t ni = 0, nid = 0;
        std::memcpy(&ni, o, 8); std::memcpy(&nid, o + 8, 8); o += 16;
        c->init_recs[s].resize(ni);
        if (ni) std::memcpy(c->init_recs[s].data(), o, ni * sizeof(pic_record));
        c->init_next_id[s] = nid;
        o += ni * sizeof(pic_record);
    }
    for (const auto &x : arrays) {
        if (e == cudaSuccess && x.second) e = cudaMemcpyAsync(x.first, o, x.second, cudaMemcpyHostToDevice, c->stream);
        o += x.second;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cnt, cnt.data(), sizeof(DevCounters) * S, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned long long) * c->n_status, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_fspawn, 0, sizeof(uint32_t) * c->n_status, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_load copy");
    c->step = hd.step;
    c->flux_final = 0;                    // the fluxes are derived again from the counts
    c->flux_final_w = 0;
    c->dev_step_valid = false;
    c->replayable = hd.replayable != 0;
    c->replay_why = c->replayable ? "" : "pic_grad: the saved run could not be replayed";
    return PIC_OK;
}

pic_status pic_sync(pic_ctx *c)
{
    if (!c) return PIC_ERR_ARG;
    return device_status(c);
}

pic_status pic_moments(pic_ctx *c, int stack, uint32_t *n_dev, int32_t *J_dev, pic_ledger *led)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    const HostStack &h = c->hs[stack];
    const DevStack &d = c->ds[stack];
    cudaError_t e = J_dev ? derive_fluxes(c) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_moments fluxes");
    const size_t nn = (size_t)h.n_out * 2 * c->p.n_e * h.n_cells;
    const size_t nj = (size_t)h.n_out * 2 * (h.n_cells + 1);
    if (n_dev && nn) e = cudaMemcpyAsync(n_dev, c->d_nh + d.n_off, 4 * nn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && J_dev && nj) e = cudaMemcpyAsync(J_dev, c->d_J + d.J_off, 4 * nj, cudaMemcpyDeviceToDevice, c->stream);
    DevCounters hc{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, c->d_cnt + stack, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_moments copy");
    const pic_status st = device_status(c);
    if (led) {
        static_assert(sizeof(pic_ledger) == sizeof(unsigned long long) * LEDGER_N, "ledger layout");
        std::memcpy(led, hc.led, sizeof(pic_ledger));
    }
    return st;
}

pic_status pic_moment_window(pic_ctx *c, int stack, int window, uint32_t *n_out, int32_t *J_out,
                             pic_ledger *led)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    const HostStack &h = c->hs[stack];
    const DevStack &d = c->ds[stack];
    if (window < 0 || window >= h.n_out) return fail(c, PIC_ERR_ARG, "window index out of range");
    cudaError_t e = J_out ? derive_fluxes(c) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_moment_window fluxes");
    const size_t nn = (size_t)2 * c->p.n_e * h.n_cells;
    const size_t nj = (size_t)2 * (h.n_cells + 1);
    // the buffers may be host or device memory (unified addressing)
    if (n_out) e = cudaMemcpyAsync(n_out, c->d_nh + d.n_off + (size_t)window * nn, 4 * nn, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && J_out)
        e = cudaMemcpyAsync(J_out, c->d_J + d.J_off + (size_t)window * nj, 4 * nj, cudaMemcpyDefault, c->stream);
    DevCounters hc{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, c->d_cnt + stack, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_moment_window copy");
    const pic_status st = device_status(c);
    if (led) std::memcpy(led, hc.led, sizeof(pic_ledger));
    return st;
}

pic_status pic_weighted_moments(pic_ctx *c, int stack, uint64_t *nw_dev, int64_t *Jw_dev,
                                uint64_t *w_injected_host)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    if (!(c->p.flags & PIC_F_WEIGHTS))
        return fail(c, PIC_ERR_ARG, "the context was made without PIC_F_WEIGHTS");
    const HostStack &h = c->hs[stack];
    const DevStack &d = c->ds[stack];
    cudaError_t e = Jw_dev ? derive_fluxes_w(c) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_weighted_moments fluxes");
    const size_t nn = (size_t)h.n_out * 2 * c->p.n_e * h.n_cells;
    const size_t nj = (size_t)h.n_out * 2 * (h.n_cells + 1);
    if (nw_dev && nn) e = cudaMemcpyAsync(nw_dev, c->d_nhw + d.n_off, 8 * nn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && Jw_dev && nj) e = cudaMemcpyAsync(Jw_dev, c->d_Jw + d.J_off, 8 * nj, cudaMemcpyDeviceToDevice, c->stream);
    DevCounters hc{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, c->d_cnt + stack, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_weighted_moments copy");
    const pic_status st = device_status(c);
    if (w_injected_host) *w_injected_host = hc.w_injected;
    return st;
}

pic_status pic_weights(pic_ctx *c, int stack, uint32_t *out, int64_t *n)
{
    if (!c || !n) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    if (!(c->p.flags & PIC_F_WEIGHTS))
        return fail(c, PIC_ERR_ARG, "the context was made without PIC_F_WEIGHTS");
    DevCounters hc{};
    DevCtl ctl{};
    cudaError_t e = cudaMemcpyAsync(&hc, c->d_cnt + stack, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_weights");
    const int64_t cnt = (int64_t)hc.n_slots;
    if (!out) { *n = cnt; return PIC_OK; }
    if (*n < cnt) { *n = cnt; return fail(c, PIC_ERR_ARG, "output buffer too small"); }
    *n = cnt;
    if (cnt) e = cudaMemcpyAsync(out, c->d_w[ctl.cur] + c->ds[stack].base, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_weights copy");
    return PIC_OK;
}

pic_status pic_set_weights(pic_ctx *c, int stack, const uint32_t *in, int64_t n)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    if (!(c->p.flags & PIC_F_WEIGHTS))
        return fail(c, PIC_ERR_ARG, "the context was made without PIC_F_WEIGHTS");
    DevCounters hc{};
    DevCtl ctl{};
    cudaError_t e = cudaMemcpyAsync(&hc, c->d_cnt + stack, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_set_weights");
    if (n != (int64_t)hc.n_slots || (n > 0 && !in)) return fail(c, PIC_ERR_ARG, "one weight per slot");
    for (int64_t i = 0; i < n; ++i)
        if (in[i] == 0u) return fail(c, PIC_ERR_ARG, "weights must be > 0");
    // the carriers leave with their old weights and come back with the new
    const int win = c->step / c->p.moment_every;
    const bool in_run = win < c->hs[stack].n_out;
    if (in_run) e = launch_state_hist_w(c->args, stack, stack + 1, 0, win, -1, nullptr, c->ncm, c->stream);
    if (e == cudaSuccess && n)
        e = cudaMemcpyAsync(c->d_w[ctl.cur] + c->ds[stack].base, in, 4 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && in_run)
        e = launch_state_hist_w(c->args, stack, stack + 1, 0, win, 1, nullptr, c->ncm, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_set_weights copy");
    return PIC_OK;
}

pic_status pic_gen_moments(pic_ctx *c, int stack, uint64_t *g_dev)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    if (!g_dev) return fail(c, PIC_ERR_ARG, "g_dev is NULL");
    const HostStack &h = c->hs[stack];
    const DevStack &d = c->ds[stack];
    const size_t ng = (size_t)h.n_out * h.n_cells;
    cudaError_t e = cudaSuccess;
    if (ng)
        e = cudaMemcpyAsync(g_dev, c->d_gh + d.n_off / (2 * c->p.n_e), 8 * ng, cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_gen_moments copy");
    return PIC_OK;
}

pic_status pic_vel_moments(pic_ctx *c, int stack, int64_t *v_dev)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    if (!v_dev) return fail(c, PIC_ERR_ARG, "v_dev is NULL");
    if (!(c->p.flags & PIC_F_VELOCITY_MOMENTS))
        return fail(c, PIC_ERR_ARG, "the context was made without PIC_F_VELOCITY_MOMENTS");
    const HostStack &h = c->hs[stack];
    const DevStack &d = c->ds[stack];
    const size_t nv = (size_t)h.n_out * 2 * h.n_cells;
    cudaError_t e = cudaSuccess;
    if (nv)
        e = cudaMemcpyAsync(v_dev, c->d_vh + d.n_off / c->p.n_e, 8 * nv, cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_vel_moments copy");
    return PIC_OK;
}

pic_status pic_records(pic_ctx *c, int stack, pic_record *out, int64_t *n)
{
    if (!c || !n) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    DevCounters hc{};
    DevCtl ctl{};
    cudaError_t e = cudaMemcpyAsync(&hc, c->d_cnt + stack, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_records");
    const int64_t cnt = (int64_t)hc.n_slots;
    if (!out) { *n = cnt; return PIC_OK; }
    if (*n < cnt) { *n = cnt; return fail(c, PIC_ERR_ARG, "output buffer too small"); }
    *n = cnt;
    if (cnt == 0) return PIC_OK;
    const int b = (int)ctl.cur;
    const int64_t base = c->ds[stack].base;
    std::vector<float> z(cnt);
    std::vector<uint32_t> id(cnt), mp(2 * cnt);      // (mu, packed) pairs
    e = cudaMemcpyAsync(z.data(), c->d_z[b] + base, 4 * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mp.data(), c->d_mu[b] + 2 * base, 8 * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(id.data(), c->d_id[b] + base, 4 * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_records copy");
    for (int64_t i = 0; i < cnt; ++i) {
        float mu;
        std::memcpy(&mu, &mp[2 * i], 4);
        out[i] = pic_record{z[i], mu, id[i], mp[2 * i + 1]};
    }
    return PIC_OK;
}

pic_status pic_set_records(pic_ctx *c, int stack, const pic_record *in, int64_t n, uint64_t next_id)
{
    if (!c) return PIC_ERR_ARG;
    if (stack < 0 || stack >= c->n_stacks) return fail(c, PIC_ERR_ARG, "stack index out of range");
    if (n < 0 || n > c->hs[stack].d.capacity || (n > 0 && !in))
        return fail(c, PIC_ERR_ARG, "record count exceeds capacity");
    // every record must index valid tables: k in 0..n_e (0 = removed),
    // layer in the stack, z inside the stack, mu a finite non-zero cosine
    const HostStack &hs = c->hs[stack];
    const float L = c->ds[stack].edge[hs.d.n_layers];
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t w = in[i].packed;
        const uint32_t k = w & 0xFFu, layer = (w >> 9) & 0xFu;
        if (k > (uint32_t)c->p.n_e || (int)layer >= hs.d.n_layers || !(in[i].z >= 0.f) ||
            !(in[i].z <= L) || !(in[i].mu >= -1.f && in[i].mu <= 1.f) || in[i].mu == 0.f)
            return fail(c, PIC_ERR_ARG, "record " + std::to_string(i) + " is out of range");
        // a carrier sits inside the layer its state names (edges included)
        if (!(in[i].z >= c->ds[stack].edge[layer] && in[i].z <= c->ds[stack].edge[layer + 1]))
            return fail(c, PIC_ERR_ARG, "record " + std::to_string(i) + " lies outside its layer");
    }
    // the carriers the stack holds now leave it, in the current window, and
    // the loaded ones enter it (births and removals at their cells: the
    // fluxes count only crossings)
    const int win = c->step / c->p.moment_every;
    const bool in_run = win < hs.n_out;
    cudaError_t e = cudaSuccess;
    const bool wts = (c->p.flags & PIC_F_WEIGHTS) != 0;
    if (in_run) e = launch_state_hist(c->args, stack, stack + 1, 0, win, -1, nullptr, c->ncm, c->stream);
    if (e == cudaSuccess && in_run && wts)
        e = launch_state_hist_w(c->args, stack, stack + 1, 0, win, -1, nullptr, c->ncm, c->stream);
    DevCtl ctl{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_set_records");
    const int b = (int)ctl.cur;
    const int64_t base = c->ds[stack].base;
    std::vector<float> z(n);
    std::vector<uint32_t> id(n), mp(2 * n);          // (mu, packed) pairs
    for (int64_t i = 0; i < n; ++i) {
        z[i] = in[i].z;
        std::memcpy(&mp[2 * i], &in[i].mu, 4);
        mp[2 * i + 1] = in[i].packed;
        id[i] = in[i].id;
    }
    if (n) {
        e = cudaMemcpyAsync(c->d_z[b] + base, z.data(), 4 * n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mu[b] + 2 * base, mp.data(), 8 * n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_id[b] + base, id.data(), 4 * n, cudaMemcpyHostToDevice, c->stream);
    }
    const unsigned long long vals[2] = {(unsigned long long)n, (unsigned long long)next_id};
    unsigned long long live = 0;
    for (int64_t i = 0; i < n; ++i) live += (in[i].packed & 0xFFu) != 0u;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cnt + stack, vals, sizeof(vals), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&c->d_cnt[stack].live, &live, sizeof(live), cudaMemcpyHostToDevice, c->stream);
    std::vector<uint32_t> unit(wts ? (size_t)n : 0, 1u << 20);      // loaded carriers weigh 1
    if (e == cudaSuccess && wts && n)
        e = cudaMemcpyAsync(c->d_w[b] + base, unit.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && in_run)
        e = launch_state_hist(c->args, stack, stack + 1, 0, win, 1, nullptr, c->ncm, c->stream);
    if (e == cudaSuccess && in_run && wts)
        e = launch_state_hist_w(c->args, stack, stack + 1, 0, win, 1, nullptr, c->ncm, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_set_records copy");
    // the adjoint replays from records loaded before the first step, whose
    // ids all lie below next_id
    bool ids_ok = true;
    for (int64_t i = 0; i < n && ids_ok; ++i)
        ids_ok = ((uint64_t)in[i].id | ((uint64_t)(in[i].packed >> 21) << 32)) < next_id;
    if (c->step == 0 && ids_ok) {
        c->init_recs[stack].assign(in, in + n);
        c->init_next_id[stack] = next_id;
    } else {
        c->replayable = false;
        c->replay_why = c->step == 0 ? "pic_grad: a loaded record has an id >= next_id"
                                     : "pic_grad: records were replaced after step 0";
    }
    return PIC_OK;
}

pic_status pic_grad(pic_ctx *c, const float *grad_n, const float *grad_J, double *grad_tau,
                    double *grad_T)
{
    if (!c) return PIC_ERR_ARG;
    if (!grad_tau && !grad_T) return fail(c, PIC_ERR_ARG, "pic_grad: no output");
    if (!c->replayable) return fail(c, PIC_ERR_STATE, c->replay_why);
    const pic_status st0 = device_status(c);
    if (st0 != PIC_OK) return st0;
    const int S = c->n_stacks, ne = c->p.n_e;
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;

    // the forward run's counters: ids issued per stack and the ledger the
    // replay must reproduce
    std::vector<DevCounters> fwd(S);
    e = cudaMemcpyAsync(fwd.data(), c->d_cnt, sizeof(DevCounters) * S, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_grad: counters");
    std::vector<DevStack> ds = c->ds;
    int64_t n_ids = 0;
    for (int s = 0; s < S; ++s) {
        ds[s].id_off = n_ids;
        ds[s].n_ids = (int64_t)fwd[s].next_id;
        n_ids += ds[s].n_ids;
    }
    int ncm = 1;
    for (int s = 0; s < S; ++s) ncm = std::max(ncm, c->hs[s].n_cells);
    const int n_out = c->hs[0].n_out;

    Replay &r = c->rp;
    Args a = c->args;
#define RALLOC(ptr, n) do { if (e == cudaSuccess && !(ptr)) e = dalloc(&ptr, n); } while (0)
    if (!r.ready) {
        for (int b = 0; b < 2; ++b) {
            RALLOC(r.z[b], c->total_slots); RALLOC(r.mu[b], 2 * c->total_slots);
            RALLOC(r.id[b], c->total_slots);
            if (e == cudaSuccess) r.pk[b] = reinterpret_cast<uint32_t *>(r.mu[b]) + 1;
            RALLOC(r.acc[b], c->total_slots);
        }
        RALLOC(r.stage_l, c->total_slots);
        RALLOC(r.cnt, S); RALLOC(r.ctl, 1); RALLOC(r.stacks, S);
        RALLOC(r.aent, c->n_ent); RALLOC(r.aT, c->n_T);
        RALLOC(r.g_ent, c->n_ent); RALLOC(r.g_T, c->n_T);
        RALLOC(r.gpot, (size_t)S * n_out * 2 * ncm);
        RALLOC(r.qgn, (size_t)S * n_out * 2 * ne * ncm);
        RALLOC(r.gen_max, 1);
        RALLOC(r.absmax, 2);
        a.n_out = n_out; a.ncm = ncm;
        for (int pass = 1; pass <= 2 && e == cudaSuccess; ++pass)
            e = configure_adjoint(a, pass, &r.lc[pass - 1]);
        if (e == cudaSuccess) {
            r.n_status = 1;
            for (const LaunchCfg &l : r.lc)
                r.n_status = std::max({r.n_status, l.grid_fast, l.grid_fast_dep, l.grid_slow,
                                       l.grid_slow_dep, l.grid_place, l.grid_place_dep,
                                       l.grid_compact});
        }
        RALLOC(r.status, (size_t)r.n_status);
        RALLOC(r.qcnt, (size_t)r.n_status);
        RALLOC(r.fspawn, (size_t)r.n_status);
        if (e == cudaSuccess) e = cudaMemsetAsync(r.fspawn, 0, sizeof(uint32_t) * r.n_status, st);
        // d log P / d tau_in of each outcome per (layer, spin, k), with rates
        // r_in = 1/tau_in, r_el = 1/tau_el, r = r_in + r_el, p = 1 - e^{-dt r}
        // and d r_in / d tau_in = -r_in^2; d log P / d T per interface entry
        std::vector<AdjEnt> aent;
        std::vector<double2> aT;
        for (int s = 0; s < S && e == cudaSuccess; ++s) {
            const HostStack &h = c->hs[s];
            for (int l = 0; l < h.d.n_layers; ++l) {
                const int m = h.d.layer_mat[l];
                const double r_el = std::isinf(h.tau_el[m]) ? 0.0 : 1.0 / h.tau_el[m];
                for (int sp = 0; sp < 2; ++sp)
                    for (int k = 0; k < ne; ++k) {
                        const double ti = h.tau_in[((size_t)m * 2 + sp) * ne + k];
                        const double r_in = std::isinf(ti) ? 0.0 : 1.0 / ti;
                        const double rate = r_in + r_el, dtr = (double)c->p.dt * rate;
                        const double pr = -std::expm1(-dtr);
                        const double keep = (double)c->p.dt * r_in * r_in;
                        const double hit = pr > 0.0 ? -keep * std::exp(-dtr) / pr : 0.0;
                        const double inel = rate > 0.0 ? -r_in * r_el / rate : 0.0;
                        const double el = (rate > 0.0 && r_el > 0.0) ? r_in * r_in / rate : 0.0;
                        aent.push_back(AdjEnt{keep, hit + el, hit + inel, 0.0});
                    }
            }
            for (double T : h.T)
                aT.push_back(make_double2(T > 0.0 ? 1.0 / T : 0.0, T < 1.0 ? -1.0 / (1.0 - T) : 0.0));
        }
        if (e == cudaSuccess && !aent.empty())
            e = cudaMemcpyAsync(r.aent, aent.data(), sizeof(AdjEnt) * aent.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !aT.empty())
            e = cudaMemcpyAsync(r.aT, aT.data(), sizeof(double2) * aT.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PIC_ERR_ALLOC, std::string("pic_grad: replay buffers: ") + cudaGetErrorString(e));
        }
        r.ready = true;
    }
    if (n_ids > r.ids_cap) {
        release(r.tot); release(r.parent); release(r.gen);
        r.ids_cap = 0;
        RALLOC(r.tot, (size_t)n_ids); RALLOC(r.parent, (size_t)n_ids); RALLOC(r.gen, (size_t)n_ids);
        if (e != cudaSuccess) {
            cudaGetLastError();
            release(r.tot); release(r.parent); release(r.gen);
            return fail(c, PIC_ERR_ALLOC, "pic_grad: " + std::to_string(n_ids) +
                                              " carrier ids do not fit in device memory");
        }
        r.ids_cap = n_ids;
    }
#undef RALLOC

    for (int b = 0; b < 2; ++b) {
        a.z[b] = r.z[b]; a.mu[b] = r.mu[b]; a.id[b] = r.id[b]; a.pk[b] = r.pk[b];
        a.acc[b] = r.acc[b];
    }
    a.stacks = r.stacks; a.cnt = r.cnt; a.ctl = r.ctl; a.status = r.status; a.qcnt = r.qcnt;
    a.fspawn = r.fspawn;
    a.n_hist = nullptr; a.J_hist = nullptr; a.g_hist = nullptr; a.v_hist = nullptr;
    a.bd_hist = nullptr;
    a.w[0] = a.w[1] = nullptr;                // the replay carries no weights
    a.nhw = nullptr; a.bdw = nullptr; a.Jw = nullptr;
    a.tot = r.tot; a.parent = r.parent; a.gen = r.gen; a.gen_max = r.gen_max;
    a.aent = r.aent; a.aT = r.aT; a.g_ent = r.g_ent; a.g_T = r.g_T;
    a.gn = grad_n ? r.qgn : nullptr; a.gpot = r.gpot; a.stage_l = r.stage_l;
    a.n_out = n_out; a.ncm = ncm;

    // fixed-point scale 2^F: the largest weight maps to at most 2^30 (an
    // int32), and no lineage's reward can reach 2^62: a lineage holds at most
    // n_e carriers at a time, each earning at most (n_cells + 1) weights a step
    const int rows = S * n_out * 2;
    const long long n_gn = (long long)rows * ne * ncm, n_gJ = (long long)rows * (ncm + 1);
    unsigned int amax[2] = {0u, 0u};
    e = cudaMemsetAsync(r.absmax, 0, 2 * sizeof(unsigned int), st);
    if (e == cudaSuccess && grad_n) e = launch_absmax(grad_n, n_gn, r.absmax, st);
    if (e == cudaSuccess && grad_J) e = launch_absmax(grad_J, n_gJ, r.absmax + 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(amax, r.absmax, sizeof(amax), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_grad: weights");
    if (amax[0] >= 0x7F800000u || amax[1] >= 0x7F800000u)
        return fail(c, PIC_ERR_ARG, "pic_grad: the weights must be finite");
    float wmax_f;
    const unsigned int wbits = std::max(amax[0], amax[1]);
    std::memcpy(&wmax_f, &wbits, 4);
    int F = 0;
    if (wmax_f > 0.f) {
        int ex = 0;
        std::frexp((double)wmax_f, &ex);                  // wmax < 2^ex
        const double life = (double)ne * (double)std::max(c->step, 1) * (double)(ncm + 1);
        F = std::min(30 - ex, (int)std::floor(62.0 - std::log2(life)) - ex);
    }
    const double scale = std::ldexp(1.0, F);
    a.inv_q = std::ldexp(1.0, -F);

    e = cudaMemcpyAsync(r.stacks, ds.data(), sizeof(DevStack) * S, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && grad_n)
        e = timed(c, 7, [&] { return launch_quantize(grad_n, n_gn, r.qgn, scale, st); });
    if (e == cudaSuccess) {
        if (grad_J) e = timed(c, 7, [&] { return launch_flux_potential(a, grad_J, r.gpot, rows, scale, st); });
        else e = cudaMemsetAsync(r.gpot, 0, sizeof(long long) * (size_t)rows * ncm, st);
    }
    const bool det = (c->p.flags & PIC_F_DETERMINISTIC) != 0;
    for (int pass = 1; pass <= 2 && e == cudaSuccess; ++pass) {
        const LaunchCfg &lc = r.lc[pass - 1];
        // the initial state
        DevCtl ctl{};
        ctl.epoch = 1u;
        std::vector<DevCounters> cnt(S);
        std::memset(cnt.data(), 0, sizeof(DevCounters) * S);
        for (int s = 0; s < S && e == cudaSuccess; ++s) {
            const std::vector<pic_record> &ir = c->init_recs[s];
            cnt[s].n_slots = ir.size();
            cnt[s].next_id = c->init_next_id[s];
            for (const pic_record &q : ir) cnt[s].live += (q.packed & 0xFFu) != 0u;
            const int64_t n = (int64_t)ir.size();
            if (!n) continue;
            std::vector<float> z(n);
            std::vector<uint32_t> id(n), mp(2 * n);      // (mu, packed) pairs
            for (int64_t i = 0; i < n; ++i) {
                z[i] = ir[i].z;
                std::memcpy(&mp[2 * i], &ir[i].mu, 4);
                mp[2 * i + 1] = ir[i].packed;
                id[i] = ir[i].id;
            }
            const int64_t base = c->ds[s].base;
            e = cudaMemcpyAsync(r.z[0] + base, z.data(), 4 * n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r.mu[0] + 2 * base, mp.data(), 8 * n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r.id[0] + base, id.data(), 4 * n, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) break;
            e = cudaStreamSynchronize(st);          // host vectors go out of scope
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(r.cnt, cnt.data(), sizeof(DevCounters) * S, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r.ctl, &ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(r.status, 0, sizeof(unsigned long long) * r.n_status, st);
        // the own reward (pass 1) or reward-to-go (pass 2) of a loaded carrier
        // starts at 0 or at its lineage total
        if (e == cudaSuccess) e = timed(c, 7, [&] { return launch_init_acc(a, lc, pass, st); });
        if (e == cudaSuccess && pass == 1) {
            e = cudaMemsetAsync(r.gen, 0, (size_t)n_ids, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(r.tot, 0, sizeof(long long) * (size_t)n_ids, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(r.gen_max, 0, sizeof(unsigned int), st);
        }
        if (e == cudaSuccess && pass == 2) {
            e = cudaMemsetAsync(r.g_ent, 0, sizeof(double) * std::max<size_t>(c->n_ent, 1), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(r.g_T, 0, sizeof(double) * std::max<size_t>(c->n_T, 1), st);
        }
        // the steps of the forward run, in the same order
        for (int step = 0; step < c->step && e == cudaSuccess; ++step) {
            a.step = (uint32_t)step;
            bool inj0 = false, inj1 = false;
            for (const HostStack &h : c->hs) {
                inj0 = inj0 || h.inj[2 * (size_t)step] > 0;
                inj1 = inj1 || h.inj[2 * (size_t)step + 1] > 0;
            }
            const bool dep = ((step + 1) % c->p.moment_every) == 0;
            if (inj0) e = timed(c, 7, [&] { return launch_inject_adj(a, lc, pass, 0, false, st); });
            if (e == cudaSuccess)
                e = timed(c, 5, [&] { return launch_fast_adj(a, lc, pass, det, dep, st); });
            if (e == cudaSuccess)
                e = timed(c, 6, [&] { return launch_slow_adj(a, lc, pass, det, dep, st); });
            if (e == cudaSuccess && inj1)
                e = timed(c, 7, [&] { return launch_inject_adj(a, lc, pass, 1, dep, st); });
            if (e == cudaSuccess && ((step + 1) % c->p.compact_every) == 0)
                e = timed(c, 7, [&] { return launch_compact_adj(a, lc, pass, st); });
        }
        if (e == cudaSuccess && pass == 1) e = timed(c, 7, [&] { return launch_flush_own(a, lc, st); });
        if (e != cudaSuccess) break;

        // the replay must have reproduced the forward run exactly
        std::vector<DevCounters> rc(S);
        DevCtl rctl{};
        unsigned int gmax = 0;
        e = cudaMemcpyAsync(rc.data(), r.cnt, sizeof(DevCounters) * S, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&rctl, r.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&gmax, r.gen_max, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        if (rctl.status != 0)
            return fail(c, (pic_status)rctl.status,
                        rctl.status == PIC_ERR_TIMEOUT ? "pic_grad: a bounded device wait ran out"
                                                       : "pic_grad: the replay did not reproduce the forward run");
        for (int s = 0; s < S; ++s)
            if (rc[s].n_slots != fwd[s].n_slots || rc[s].next_id != fwd[s].next_id ||
                std::memcmp(rc[s].led, fwd[s].led, sizeof(fwd[s].led)) != 0)
                return fail(c, PIC_ERR_STATE, "pic_grad: the replay of stack " + std::to_string(s) +
                                                  " did not reproduce the forward run");
        // lineage totals, deepest generation first
        if (pass == 1)
            for (int g = (int)gmax; g >= 1 && e == cudaSuccess; --g)
                e = timed(c, 7, [&] { return launch_lineage(a, lc, n_ids, g, st); });
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_grad");

    // per-layer bins to the per-material and per-interface outputs
    std::vector<double> g_ent(c->n_ent), g_T(c->n_T);
    if (c->n_ent) e = cudaMemcpyAsync(g_ent.data(), r.g_ent, 8 * c->n_ent, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && c->n_T) e = cudaMemcpyAsync(g_T.data(), r.g_T, 8 * c->n_T, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_grad: gradient bins");
    const size_t per_tau = (size_t)c->n_mat_max * 2 * ne, per_T = (size_t)(PIC_MAX_LAYERS - 1) * 4 * ne;
    std::vector<double> out_tau((size_t)S * per_tau, 0.0), out_T((size_t)S * per_T, 0.0);
    for (int s = 0; s < S; ++s) {
        const HostStack &h = c->hs[s];
        const DevStack &d = c->ds[s];
        for (int l = 0; l < h.d.n_layers; ++l)
            for (int i = 0; i < 2 * ne; ++i)
                out_tau[s * per_tau + (size_t)h.d.layer_mat[l] * 2 * ne + i] +=
                    g_ent[d.ent_off + (size_t)l * 2 * ne + i];
        for (int i = 0; i < d.T_n; ++i) out_T[s * per_T + i] = g_T[d.T_off + i];
    }
    if (grad_tau) e = cudaMemcpyAsync(grad_tau, out_tau.data(), 8 * out_tau.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && grad_T) e = cudaMemcpyAsync(grad_T, out_T.data(), 8 * out_T.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_grad: outputs");
    return PIC_OK;
}

pic_status pic_shape(const pic_ctx *c, int stack, int32_t *n_cells, int32_t *n_out, int32_t *step)
{
    if (!c || stack < 0 || stack >= c->n_stacks) return PIC_ERR_ARG;
    if (n_cells) *n_cells = c->hs[stack].n_cells;
    if (n_out) *n_out = c->hs[stack].n_out;
    if (step) *step = c->step;
    return PIC_OK;
}

int64_t pic_launch_count(const pic_ctx *c) { return c ? c->launches : 0; }

pic_status pic_launch_config(const pic_ctx *c, pic_launch_info *out)
{
    if (!c || !out) return PIC_ERR_ARG;
    out->grid_step = c->lc.grid_fast;
    out->grid_step_moments = c->lc.grid_fast_dep;
    out->grid_slow = c->lc.grid_slow;
    out->grid_slow_moments = c->lc.grid_slow_dep;
    out->grid_compact = c->lc.grid_compact;
    out->grid_inject = c->lc.grid_inject;
    out->ring_step = c->lc.ring_fast;
    out->ring_step_moments = c->lc.ring_fast_dep;
    out->smem_step = (int64_t)c->lc.smem_fast;
    out->smem_step_moments = (int64_t)c->lc.smem_fast_dep;
    out->warps_step = c->lc.nw_fast;
    out->warps_step_moments = c->lc.nw_fast_dep;
    for (int i = 0; i < 2; ++i) {
        const bool r = c->rp.ready;
        out->grid_adj_step[i] = r ? c->rp.lc[i].grid_fast_dep : 0;
        out->ring_adj_step[i] = r ? c->rp.lc[i].ring_fast_dep : 0;
        out->smem_adj_step[i] = r ? (int64_t)c->rp.lc[i].smem_fast_dep : 0;
    }
    out->grid_step_fused = c->lc.grid_fused;
    out->ring_step_fused = c->lc.grid_fused ? c->lc.ring_fused : 0;
    out->smem_step_fused = c->lc.grid_fused ? (int64_t)c->lc.smem_fused : 0;
    return PIC_OK;
}

pic_status pic_autotune(pic_ctx *c, int trial_steps, pic_tune_entry *entries, int max_entries,
                        int *n_entries)
{
    if (!c) return PIC_ERR_ARG;
    if (trial_steps < 1) return fail(c, PIC_ERR_ARG, "pic_autotune: trial_steps < 1");
    if (c->profiling) return fail(c, PIC_ERR_STATE, "pic_autotune: profiling is on");
    struct Cand { int bps, ring, hm, nw, ev; };
    std::vector<Cand> cands;
    const bool dep_in_trial = trial_steps >= c->p.moment_every;
    // the fused form exists for one stack and eight consumer warps, with at
    // most PIC_EV_MIN_BLOCKS blocks per SM
    const bool fusable = c->n_stacks == 1;
    for (int hm = 0; hm <= (dep_in_trial ? 1 : 0); ++hm)
        for (int nw : {8, 4})
            for (int ev = (nw == 8 && fusable ? 0 : 1); ev <= 1; ++ev)
                for (int bps = 1; bps <= (ev == 0 ? 3 : nw == 4 ? 8 : 6); ++bps)
                    for (int ring : {2, 3, 4, 6, 8}) cands.push_back({bps, ring, hm, nw, ev});
    if ((int64_t)c->step + (int64_t)trial_steps * (int64_t)cands.size() > c->p.n_steps_max)
        return fail(c, PIC_ERR_ARG, "pic_autotune: not enough steps left for the trials");
    const int use_graph = c->p.use_graph;
    c->p.use_graph = 0;                       // trials use single launches
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    auto steps_done = [&](uint64_t &ps) {
        std::vector<DevCounters> h(c->n_stacks);
        cudaError_t r = cudaMemcpyAsync(h.data(), c->d_cnt, sizeof(DevCounters) * c->n_stacks,
                                        cudaMemcpyDeviceToHost, c->stream);
        if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
        ps = 0;
        for (const DevCounters &x : h) ps += x.led[L_PARTICLE_STEPS];
        return r;
    };
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const LaunchCfg keep = c->lc;
    const pic_params keep_p = c->p;
    double best = 0.0;
    LaunchCfg best_lc = keep;
    Cand best_c{keep_p.blocks_per_sm, keep_p.ring_stages, keep_p.hist_mode, keep_p.consumer_warps,
                keep_p.event_pass};
    std::vector<pic_tune_entry> res;
    for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) {
        const Cand &k = cands[i];
        LaunchCfg lc{};
        if (configure(c->args, k.bps, k.ring, k.hm, k.nw, &lc) != cudaSuccess) {
            cudaGetLastError();               // does not fit: not a candidate
            continue;
        }
        const int gmax = std::max({lc.grid_fast, lc.grid_fast_dep, lc.grid_slow,
                                   lc.grid_slow_dep, lc.grid_place, lc.grid_place_dep,
                                   lc.grid_compact});
        // a candidate whose ring leaves fewer resident blocks than asked for
        // is another candidate's duplicate
        if (k.ev == 1) lc.grid_fused = 0;
        if (gmax > c->n_status || lc.ring_fast != k.ring || lc.grid_fast != sms * k.bps ||
            lc.grid_fast_dep == 0)
            continue;
        if (k.ev == 0 && (lc.grid_fused != sms * k.bps || lc.ring_fused != k.ring)) continue;
        c->lc = lc;
        c->p.hist_mode = k.hm;
        uint64_t ps0 = 0, ps1 = 0;
        e = steps_done(ps0);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->stream);
        if (e != cudaSuccess) break;
        const pic_status st = pic_step(c, trial_steps);
        if (st != PIC_OK) { c->lc = keep; c->p = keep_p; c->p.use_graph = use_graph; return st; }
        e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess) e = steps_done(ps1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) break;
        const double ns = ps1 > ps0 ? 1e6 * (double)ms / (double)(ps1 - ps0) : 1e30;
        res.push_back(pic_tune_entry{k.bps, k.ring, k.hm, 0, ns, k.nw, k.ev});
        if (res.size() == 1 || ns < best) {
            best = ns;
            best_lc = lc;
            best_c = k;
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    c->p = keep_p;
    c->p.use_graph = use_graph;
    if (e != cudaSuccess) {
        c->lc = keep;
        return cuda_fail(c, e, "pic_autotune");
    }
    c->lc = best_lc;
    c->p.blocks_per_sm = best_c.bps;
    c->p.ring_stages = best_c.ring;
    c->p.hist_mode = best_c.hm;
    c->p.consumer_warps = best_c.nw;
    c->p.event_pass = best_c.ev;
    // graphs captured with the old configuration are stale
    for (cudaGraphExec_t &g : c->period_graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    if (c->persist_graph) cudaGraphExecDestroy(c->persist_graph);
    c->persist_graph = nullptr;
    for (pic_tune_entry &r : res)
        r.chosen = (r.blocks_per_sm == best_c.bps && r.ring_stages == best_c.ring &&
                    r.hist_mode == best_c.hm && r.consumer_warps == best_c.nw &&
                    r.event_pass == best_c.ev) ? 1 : 0;
    if (entries)
        for (int i = 0; i < (int)res.size() && i < max_entries; ++i) entries[i] = res[i];
    if (n_entries) *n_entries = (int)res.size();
    return PIC_OK;
}

pic_status pic_profile(pic_ctx *c, int enable)
{
    if (!c) return PIC_ERR_ARG;
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_profile");
    c->profiling = enable != 0;
    if (enable) {
        c->ev_marks.clear();
        c->ev_used = 0;
    }
    return PIC_OK;
}

pic_status pic_profile_read(pic_ctx *c, pic_kernel_times *out)
{
    if (!c || !out) return PIC_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pic_profile_read");
    for (const auto &m : c->ev_marks) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->ev_pool[m.second], c->ev_pool[m.second + 1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "pic_profile_read elapsed");
        out->launches[m.first] += 1;
        out->ms[m.first] += ms;
    }
    return PIC_OK;
}

void pic_destroy(pic_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
    free_all(c);
    delete c;
}

}  // extern "C"
