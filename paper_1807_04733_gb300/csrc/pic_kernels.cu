// CUDA kernels of the hot-electron PIC step (sm_103a).
//
// One Strang step (Eq. strang, Sec. III.A) is, per stack:
//   k_inject(half 0)   Source(dt/2): append new carriers
//   k_step             Transport(dt/2) -> Scattering(dt) -> Transport(dt/2)
//                      for every live slot, secondaries appended in parent
//                      slot order, densities and fluxes deposited
//   k_inject(half 1)   Source(dt/2), deposited at moment steps
//   k_compact          every compact_every steps: stable removal of dead slots
//
// The step kernel is a persistent streaming kernel: the tiles of all stacks
// are concatenated and cut into one contiguous chunk per block.  Each thread
// moves four consecutive slots with one 128-bit load and store per array.
// Secondary carriers are placed by a decoupled look-back over the blocks'
// chunks (the block's running count of secondaries, published as a tagged
// 64-bit word), so slot order and ids equal those of a scalar loop over the
// slots; every wait on another block is bounded and reports PIC_ERR_TIMEOUT.
// Densities and fluxes are privatised in shared memory and flushed to the
// global moment arrays once per block and stack segment.
#include <cuda_runtime.h>

#include "pic_internal.h"

namespace pic {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): two 32x32->64 products per round,
// round multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments
// 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// direction cosine from a word: odd multiples of 2^-23 in (-1, 1), exact
__device__ __forceinline__ float mu_of(uint32_t x)
{
    const int n = (int)(2u * (x >> 9) + 1u) - 8388608;
    return __fmul_rn(__int2float_rn(n), 1.1920928955078125e-07f);
}

// uniform in (0, 1): odd multiples of 2^-24, exact
__device__ __forceinline__ float unit_of(uint32_t x)
{
    return __fmul_rn(__uint2float_rn(2u * (x >> 9) + 1u), 5.9604644775390625e-08f);
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p)
{
    return *(volatile const unsigned long long *)p;
}

struct Tally {           // per-thread event counts, reduced per segment
    uint32_t steps, absorbed, bath, hits, trans, trunc, spawn_drop, q_drop, changed;
};

// Shared-memory view of the current stack.
struct Stk {
    const TabEnt *ent;
    const uint32_t *T;
    const float *edge;
    const uint32_t *p0;
    int n_layers, n_cells, n_e;
    uint32_t ctr_hi;     // stack << 16
};

__device__ __forceinline__ int cell_of(const Args &a, const Stk &s, float z)
{
    const float q = floorf(a.dz_pow2 ? __fmul_rn(z, a.inv_dz) : __fdiv_rn(z, a.dz));
    int c = (int)q;
    if (q < 0.f) c = 0;
    if (c > s.n_cells - 1) c = s.n_cells - 1;
    return c;
}

// Transport for a time tau (Eq. Strang-transport, Sec. III): free flight in
// the current layer, mirror reflection at the vacuum surfaces, a uniform
// draw against T at an interface (transmit: layer changes, mu kept;
// reflect: mu mirrored), the remaining time flown in the new layer.
template <bool DET>
__device__ __forceinline__ void flight(const Args &a, const Stk &s, float &z, float &mu,
                                       int &layer, int sg, int k, float tau, uint32_t id_lo,
                                       uint32_t ctr_y, uint32_t sub0, Tally &t)
{
    for (int hit = 0;; ++hit) {
        const float v = s.ent[(layer * 2 + sg) * s.n_e + (k - 1)].v;
        const float w = __fmul_rn(v, mu);
        const float z1 = DET ? __fadd_rn(z, __fmul_rn(w, tau)) : __fmaf_rn(w, tau, z);
        const float lo = s.edge[layer], hi = s.edge[layer + 1];
        float zb;
        bool up;
        if (mu > 0.f && z1 > hi) { zb = hi; up = true; }
        else if (mu < 0.f && z1 < lo) { zb = lo; up = false; }
        else { z = z1; return; }
        if (hit == PIC_MAX_HITS) { z = zb; ++t.trunc; return; }
        const float tb = __fdiv_rn(__fsub_rn(zb, z), w);
        tau = __fsub_rn(tau, tb);
        if (!(tau > 0.f)) tau = 0.f;
        z = zb;
        const bool vacuum = up ? (layer == s.n_layers - 1) : (layer == 0);
        if (vacuum) {
            mu = -mu;
        } else {
            const int iface = up ? layer : layer - 1, dir = up ? 0 : 1;
            bool trans = true;
            ++t.hits;
            if (!(a.flags & PIC_F_TRANSPARENT)) {
                const uint4 r = philox(make_uint4(id_lo, ctr_y, a.step, sub0 + (uint32_t)hit),
                                       a.seed_lo, a.seed_hi);
                trans = r.x < s.T[((iface * 2 + dir) * 2 + sg) * s.n_e + (k - 1)];
            }
            if (trans) { layer += up ? 1 : -1; ++t.trans; }
            else mu = -mu;
        }
    }
}

__device__ __forceinline__ void add_flux(int32_t *sJ, int nf, int sg, int c0, int c1)
{
    if (c1 > c0) for (int f = c0 + 1; f <= c1; ++f) atomicAdd(&sJ[sg * nf + f], 1);
    else         for (int f = c1 + 1; f <= c0; ++f) atomicAdd(&sJ[sg * nf + f], -1);
}

// Block-wide exclusive scan of small non-negative ints; returns the total.
__device__ __forceinline__ int block_scan(int v, int &excl, int *s_w)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < TPB / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < TPB / 32) s_w[lane] = w;        // inclusive warp totals
    }
    __syncthreads();
    excl = x - v + (wid ? s_w[wid - 1] : 0);
    const int total = s_w[TPB / 32 - 1];
    __syncthreads();
    return total;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long *s_r)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_r[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < TPB / 32; ++i) t += s_r[i];
    __syncthreads();
    return t;  // valid in thread 0
}

// Status word of the look-back: epoch:32 | flag:2 | value:30
constexpr unsigned long long FLAG_A = 1ull, FLAG_P = 2ull;
__device__ __forceinline__ void publish(unsigned long long *w, unsigned int ep,
                                        unsigned long long flag, long long value)
{
    __threadfence();
    atomicExch(w, ((unsigned long long)ep << 32) | (flag << 30) |
                      ((unsigned long long)value & 0x3FFFFFFFull));
}

// Exclusive prefix of the running count of the stack segment that starts
// this block's chunk at tile t0 (stack tiles start at ts): walk back over the
// blocks whose chunks end inside the same stack.  Bounded wait.
__device__ long long look_back(const Args &a, unsigned int ep, long long T, long long ts,
                               int b, int G)
{
    long long prefix = 0;
    for (int j = b - 1; j >= 0; --j) {
        const long long jt0 = T * j / G, jt1 = T * (j + 1) / G;
        if (jt1 <= ts) break;
        if (jt0 == jt1) continue;
        unsigned long long w = 0;
        unsigned int it = 0;
        for (;;) {
            w = ld_volatile_u64(&a.status[j]);
            if ((unsigned int)(w >> 32) == ep && ((w >> 30) & 3ull)) break;
            if (++it > a.spin_limit) {
                atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
                a.ctl->timeout_where = 1u;
                w = FLAG_P << 30;
                break;
            }
            if (it > 64) __nanosleep(128);
        }
        prefix += (long long)(w & 0x3FFFFFFFull);
        if (((w >> 30) & 3ull) == FLAG_P) break;
    }
    return prefix;
}

// Per-block plan shared by the streaming kernels: tiles of every stack
// concatenated; this block owns tiles [t0, t1).
struct Plan {
    long long T, t0, t1;
};

__device__ __forceinline__ void make_plan(const Args &a, long long *s_tpref,
                                          long long *s_nsl, Plan &p)
{
    for (int i = threadIdx.x; i < a.n_stacks; i += TPB)
        s_nsl[i] = (long long)a.cnt[i].n_slots;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < a.n_stacks; ++i) {
            s_tpref[i] = acc;
            acc += (s_nsl[i] + TILE - 1) / TILE;
        }
        s_tpref[a.n_stacks] = acc;
    }
    __syncthreads();
    p.T = s_tpref[a.n_stacks];
    p.t0 = p.T * blockIdx.x / gridDim.x;
    p.t1 = p.T * (blockIdx.x + 1) / gridDim.x;
}

__device__ __forceinline__ int stack_of(const long long *s_tpref, int n, long long t)
{
    int lo = 0, hi = n - 1;              // last s with s_tpref[s] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_tpref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Last-block-done: returns true in every thread of the block that finished last.
__device__ __forceinline__ bool last_block(const Args &a, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(&a.ctl->done, 1u);
        *s_flag = (t == gridDim.x - 1);
    }
    __syncthreads();
    const bool last = *s_flag != 0;
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ void load_stack(const Args &a, int s, Stk &k, DevStack *s_st,
                                           TabEnt *s_ent, uint32_t *s_T, float *s_edge,
                                           uint32_t *s_p0)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_st = a.stacks[s];
    __syncthreads();
    const DevStack &st = *s_st;
    for (int i = threadIdx.x; i < st.tab_n; i += TPB) s_ent[i] = a.ent[st.ent_off + i];
    for (int i = threadIdx.x; i < st.T_n; i += TPB) s_T[i] = a.T_thr[st.T_off + i];
    if (threadIdx.x <= st.n_layers) s_edge[threadIdx.x] = st.edge[threadIdx.x];
    if (threadIdx.x < st.n_layers) s_p0[threadIdx.x] = st.p0_thr[threadIdx.x];
    k.ent = s_ent; k.T = s_T; k.edge = s_edge; k.p0 = s_p0;
    k.n_layers = st.n_layers; k.n_cells = st.n_cells; k.n_e = a.n_e;
    k.ctr_hi = (uint32_t)s << 16;
}

// ---------------------------------------------------------------------------
// k_step: Transport(dt/2) -> Scattering(dt) -> Transport(dt/2) for all slots
// ---------------------------------------------------------------------------
template <bool DET, bool DEPN, bool WAGG>
__global__ void __launch_bounds__(TPB) k_step(const Args a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    TabEnt *s_ent = reinterpret_cast<TabEnt *>(smem);
    uint32_t *s_T = reinterpret_cast<uint32_t *>(s_ent + a.tab_max);
    int32_t *s_J = reinterpret_cast<int32_t *>(s_T + a.T_max);
    uint32_t *s_n = reinterpret_cast<uint32_t *>(s_J + a.jbin_max);
    __shared__ long long s_tpref[PIC_MAX_STACKS + 1];
    __shared__ long long s_nsl[PIC_MAX_STACKS];
    __shared__ float s_edge[PIC_MAX_LAYERS + 1];
    __shared__ uint32_t s_p0[PIC_MAX_LAYERS];
    __shared__ DevStack s_st;
    __shared__ int s_w[TPB / 32];
    __shared__ unsigned long long s_r[TPB / 32];
    __shared__ long long s_prefix;
    __shared__ int s_flag;

    const unsigned int ep = *(volatile unsigned int *)&a.ctl->epoch;
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    const int b = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
    Plan p;
    make_plan(a, s_tpref, s_nsl, p);
    const int tj = (int)(a.step / (uint32_t)a.moment_every);
    const int tout = (int)((a.step + 1) / (uint32_t)a.moment_every) - 1;
    const float half = a.half_dt;

    float *Z = a.z[cur], *MU = a.mu[cur];
    const uint32_t *ID = a.id[cur];
    uint32_t *PK = a.pk[cur];

    // the first segment (stack of tile t0) may start inside its stack; its
    // secondaries are staged until the look-back gives their prefix
    int seg_stack = -1;
    long long seg_first = 0, seg_count = 0, stage0 = p.t0 * TILE, stage_cur = p.t0 * TILE;
    bool staged_seg = false;          // current segment is the staged one
    int staged_stack = -1;
    long long staged_count = 0;
    Stk S{};
    Tally ty{};

    auto flush_segment = [&](int s, bool deposit_hist) {
        // moments and ledger of stack s
        __syncthreads();
        const DevStack &st = s_st;
        const int nf = st.n_cells + 1;
        int32_t *gJ = a.J_hist + st.J_off + (long long)tj * 2 * nf;
        for (int i = tid; i < 2 * nf; i += TPB) {
            const int v = s_J[i];
            if (v) atomicAdd(&gJ[i], v);
        }
        if (DEPN && deposit_hist) {
            const int nb = 2 * a.n_e * st.n_cells;
            uint32_t *gN = a.n_hist + st.n_off + (long long)tout * nb;
            for (int i = tid; i < nb; i += TPB) {
                const uint32_t v = s_n[i];
                if (v) atomicAdd(&gN[i], v);
            }
        }
        unsigned long long *L = a.cnt[s].led;
        const unsigned long long v0 = block_sum_u64(ty.steps, s_r);
        if (tid == 0 && v0) atomicAdd(&L[L_PARTICLE_STEPS], v0);
        const unsigned long long v1 = block_sum_u64(ty.absorbed, s_r);
        if (tid == 0 && v1) atomicAdd(&L[L_ABSORBED], v1);
        const unsigned long long v2 = block_sum_u64(ty.bath, s_r);
        if (tid == 0 && v2) atomicAdd(&L[L_Q_BATH], v2);
        const unsigned long long v3 = block_sum_u64(ty.hits, s_r);
        if (tid == 0 && v3) atomicAdd(&L[L_IFACE_HITS], v3);
        const unsigned long long v4 = block_sum_u64(ty.trans, s_r);
        if (tid == 0 && v4) atomicAdd(&L[L_IFACE_TRANSMIT], v4);
        const unsigned long long v5 = block_sum_u64(ty.trunc, s_r);
        if (tid == 0 && v5) atomicAdd(&L[L_TRUNCATED], v5);
        const unsigned long long v6 = block_sum_u64(ty.spawn_drop, s_r);
        if (tid == 0 && v6) atomicAdd(&L[L_SPAWN_DROPPED], v6);
        const unsigned long long v7 = block_sum_u64(ty.q_drop, s_r);
        if (tid == 0 && v7) atomicAdd(&L[L_Q_DROPPED], v7);
        const unsigned long long v8 = block_sum_u64(ty.changed, s_r);
        if (tid == 0 && v8) atomicAdd(&L[L_CHANGED], v8);
        ty = Tally{};
        __syncthreads();
    };

    // Place the staged secondaries [start, start+count) of stack s whose
    // exclusive prefix among the stack's secondaries of this step is `prefix`.
    // Deposits go to shared memory if `smem_hist`, else to global memory.
    auto place = [&](int s, long long start, long long count, long long prefix, bool smem_hist) {
        const DevStack &st = s_st;          // loaded stack == s when smem_hist
        const DevStack stg = a.stacks[s];
        const long long nsl = s_nsl[s];
        const long long room = stg.cap - nsl;
        const unsigned long long nid = a.cnt[s].next_id;
        const int nf = stg.n_cells + 1;
        uint32_t kept = 0;
        for (long long i = tid; i < count; i += TPB) {
            const float4 r = a.stage[start + i];
            const long long g = prefix + i;
            const uint32_t pk_staged = __float_as_uint(r.z);
            const uint32_t pk = pk_staged & 0x1FFFFFu;
            if (g < room) {
                ty.hits += (pk_staged >> 21) & 0xFu;
                ty.trans += (pk_staged >> 25) & 0xFu;
                ty.trunc += (pk_staged >> 29) & 0x1u;
                const unsigned long long id = nid + (unsigned long long)g;
                const long long d = stg.base + nsl + g;
                Z[d] = r.x;
                MU[d] = r.y;
                a.id[cur][d] = (uint32_t)id;
                PK[d] = pk | ((uint32_t)(id >> 32) << 21);
                ++kept;
                const int sg = (int)((pk >> 8) & 1u), k = (int)(pk & 0xFFu);
                Stk tmp; tmp.n_cells = stg.n_cells;
                const int c0 = cell_of(a, tmp, r.w), c1 = cell_of(a, tmp, r.x);
                if (smem_hist) {
                    if (c0 != c1) add_flux(s_J, nf, sg, c0, c1);
                    if (DEPN) atomicAdd(&s_n[(sg * a.n_e + (k - 1)) * stg.n_cells + c1], 1u);
                } else {
                    int32_t *gJ = a.J_hist + stg.J_off + (long long)tj * 2 * nf;
                    if (c0 != c1) add_flux(gJ, nf, sg, c0, c1);
                    if (DEPN)
                        atomicAdd(&a.n_hist[stg.n_off + (long long)tout * 2 * a.n_e * stg.n_cells +
                                            (sg * a.n_e + (k - 1)) * stg.n_cells + c1], 1u);
                }
            } else {
                ++ty.spawn_drop;
                ty.q_drop += pk & 0xFFu;
            }
        }
        (void)st;
        const unsigned long long kk = block_sum_u64(kept, s_r);
        if (tid == 0 && kk) atomicAdd(&a.cnt[s].led[L_SPAWNED], kk);
        if (tid == 0 && (a.flags & PIC_F_STRICT_CAPACITY) && prefix + count > room)
            atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_CAPACITY);
    };

    for (long long t = p.t0; t < p.t1; ++t) {
        const int s = stack_of(s_tpref, a.n_stacks, t);
        if (s != seg_stack) {
            if (seg_stack >= 0) {
                // close the previous segment: place its secondaries if their
                // prefix is known (segment started at its stack's first tile)
                if (!staged_seg) {
                    place(seg_stack, seg_first, seg_count, 0, true);
                    if (s_tpref[seg_stack + 1] == t && tid == 0)
                        a.cnt[seg_stack].spawn_total = (unsigned long long)seg_count;
                } else {
                    staged_count = seg_count;
                }
                flush_segment(seg_stack, true);
            }
            load_stack(a, s, S, &s_st, s_ent, s_T, s_edge, s_p0);
            const int nf = s_st.n_cells + 1;
            for (int i = tid; i < 2 * nf; i += TPB) s_J[i] = 0;
            if (DEPN)
                for (int i = tid; i < 2 * a.n_e * s_st.n_cells; i += TPB) s_n[i] = 0u;
            __syncthreads();
            staged_seg = (t > s_tpref[s]);
            if (staged_seg) staged_stack = s;
            seg_stack = s;
            seg_first = stage_cur;
            seg_count = 0;
        }
        const DevStack &st = s_st;
        const long long nsl = s_nsl[s];
        const bool room0 = (st.cap - nsl) <= 0;        // every secondary is dropped
        const long long slot0 = (t - s_tpref[s]) * TILE + (long long)tid * VEC;
        float4 sp[VEC];
        uint32_t spm = 0;
        if (slot0 < nsl) {
            const long long g = st.base + slot0;
            float4 z4 = *reinterpret_cast<const float4 *>(Z + g);
            float4 m4 = *reinterpret_cast<const float4 *>(MU + g);
            const uint4 i4 = *reinterpret_cast<const uint4 *>(ID + g);
            uint4 p4 = *reinterpret_cast<const uint4 *>(PK + g);
            const float4 m4_in = m4;
            const uint4 p4_in = p4;
            float *zz = &z4.x, *mm = &m4.x;
            const uint32_t *ii = &i4.x;
            uint32_t *pp = &p4.x;
            int bins[VEC];
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                bins[j] = -1;
                uint32_t pk = pp[j];
                int k = (int)(pk & 0xFFu);
                if (slot0 + j >= nsl || k == 0) continue;
                ++ty.steps;
                float z = zz[j], mu = mm[j];
                const int sg = (int)((pk >> 8) & 1u);
                int layer = (int)((pk >> 9) & 0xFu);
                const uint32_t id_lo = ii[j];
                const uint32_t ctr_y = (pk >> 21) | S.ctr_hi;
                const int c_start = cell_of(a, S, z);
                flight<DET>(a, S, z, mu, layer, sg, k, half, id_lo, ctr_y, SUB_IF, ty);
                // Scattering(dt): Monte-Carlo test against tau_eff (Eq. lifetimes)
                const uint4 x = philox(make_uint4(id_lo, ctr_y, a.step, SUB_SCAT),
                                       a.seed_lo, a.seed_hi);
                const TabEnt e = S.ent[(layer * 2 + sg) * S.n_e + (k - 1)];
                bool dead = false;
                if (x.x < e.P) {
                    const bool inel = x.y < e.Q;
                    if (k == 1 && (inel || (a.flags & PIC_F_LOWEST_BIN_ANY))) {
                        dead = true;
                        ++ty.absorbed;
                        ++ty.bath;
                    } else {
                        mu = mu_of(x.z);
                        if (inel) {
                            const int kp = 1 + (int)__umulhi(x.w, (uint32_t)(k - 1));
                            const int ks = k - kp;
                            k = kp;
                            if (a.flags & PIC_F_NO_SECONDARIES) {
                                ty.bath += (uint32_t)ks;
                            } else {
                                // secondary: same place, spin from P0, isotropic
                                const uint4 y = philox(make_uint4(id_lo, ctr_y, a.step, SUB_SEC),
                                                       a.seed_lo, a.seed_hi);
                                const uint32_t g0 = (pk >> 13) & 0xFFu;
                                const int sgs = y.x < S.p0[layer] ? 0 : 1;
                                const uint32_t gen = g0 < 255u ? g0 + 1u : 255u;
                                if (room0) {
                                    ++ty.spawn_drop;
                                    ty.q_drop += (uint32_t)ks;
                                    if (a.flags & PIC_F_STRICT_CAPACITY)
                                        atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_CAPACITY);
                                } else {
                                    float zs = z, mus = mu_of(y.y);
                                    int ls = layer;
                                    Tally ts{};
                                    flight<DET>(a, S, zs, mus, ls, sgs, ks, half, id_lo, ctr_y,
                                                SUB_SIF, ts);
                                    // the secondary's boundary events ride in the
                                    // (not yet used) id_hi bits until it is placed
                                    const uint32_t pks = (uint32_t)ks | ((uint32_t)sgs << 8) |
                                                         ((uint32_t)ls << 9) | (gen << 13) |
                                                         (ts.hits << 21) | (ts.trans << 25) |
                                                         (ts.trunc << 29);
                                    sp[j] = make_float4(zs, mus, __uint_as_float(pks), z);
                                    spm |= 1u << j;
                                }
                            }
                        }
                    }
                }
                if (dead) {
                    pk = (pk & ~0x1FFFu) | ((uint32_t)sg << 8) | ((uint32_t)layer << 9);
                    const int c_end = cell_of(a, S, z);
                    if (c_end != c_start) add_flux(s_J, S.n_cells + 1, sg, c_start, c_end);
                } else {
                    flight<DET>(a, S, z, mu, layer, sg, k, half, id_lo, ctr_y, SUB_IF + 16, ty);
                    const int c_end = cell_of(a, S, z);
                    if (c_end != c_start) add_flux(s_J, S.n_cells + 1, sg, c_start, c_end);
                    pk = (pk & ~0x1FFFu) | (uint32_t)k | ((uint32_t)sg << 8) |
                         ((uint32_t)layer << 9);
                    if (DEPN) bins[j] = (sg * S.n_e + (k - 1)) * S.n_cells + c_end;
                }
                ty.changed += (__float_as_uint(mu) != __float_as_uint(mm[j]) || pk != pp[j]) ? 1u : 0u;
                zz[j] = z; mm[j] = mu; pp[j] = pk;
            }
            if (slot0 + VEC <= nsl) {
                *reinterpret_cast<float4 *>(Z + g) = z4;
                if (__float_as_uint(m4.x) != __float_as_uint(m4_in.x) ||
                    __float_as_uint(m4.y) != __float_as_uint(m4_in.y) ||
                    __float_as_uint(m4.z) != __float_as_uint(m4_in.z) ||
                    __float_as_uint(m4.w) != __float_as_uint(m4_in.w))
                    *reinterpret_cast<float4 *>(MU + g) = m4;
                if (p4.x != p4_in.x || p4.y != p4_in.y || p4.z != p4_in.z || p4.w != p4_in.w)
                    *reinterpret_cast<uint4 *>(PK + g) = p4;
            } else {
                // ragged end of the stack: the slots past n_slots receive this
                // step's secondaries from other blocks, so only valid lanes
                // are written back
                const int nv = (int)(nsl - slot0);
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    if (j < nv) { Z[g + j] = zz[j]; MU[g + j] = mm[j]; PK[g + j] = pp[j]; }
            }
            if (DEPN && !WAGG) {
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    if (bins[j] >= 0) atomicAdd(&s_n[bins[j]], 1u);
            }
            if (DEPN && WAGG) {
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    const unsigned int act = __activemask();
                    const unsigned int m = __match_any_sync(act, bins[j]);
                    if (bins[j] >= 0 && (threadIdx.x & 31) == __ffs(m) - 1)
                        atomicAdd(&s_n[bins[j]], (uint32_t)__popc(m));
                }
            }
        }
        // append this tile's secondaries to the segment, in slot order
        int excl;
        const int tot = block_scan(__popc(spm), excl, s_w);
#pragma unroll
        for (int j = 0; j < VEC; ++j)
            if ((spm >> j) & 1u) a.stage[stage_cur + excl++] = sp[j];
        stage_cur += tot;
        seg_count += tot;
    }

    // close the last segment and publish its running count
    const bool have = seg_stack >= 0;
    long long lb_prefix = 0;
    if (have) {
        const bool ends_stack = s_tpref[seg_stack + 1] == p.t1;
        if (!staged_seg) {
            if (tid == 0) publish(&a.status[b], ep, FLAG_P, seg_count);
            place(seg_stack, seg_first, seg_count, 0, true);
            if (ends_stack && tid == 0) a.cnt[seg_stack].spawn_total = (unsigned long long)seg_count;
            flush_segment(seg_stack, true);
        } else {
            // single segment starting inside its stack
            if (tid == 0) {
                publish(&a.status[b], ep, FLAG_A, seg_count);
                s_prefix = look_back(a, ep, p.T, s_tpref[seg_stack], b, G);
                publish(&a.status[b], ep, FLAG_P, s_prefix + seg_count);
            }
            __syncthreads();
            lb_prefix = s_prefix;
            place(seg_stack, seg_first, seg_count, lb_prefix, true);
            if (ends_stack && tid == 0)
                a.cnt[seg_stack].spawn_total = (unsigned long long)(lb_prefix + seg_count);
            flush_segment(seg_stack, true);
            staged_stack = -1;
        }
        // an earlier staged segment (block spanning stacks): its prefix now
        if (staged_stack >= 0) {
            if (tid == 0) s_prefix = look_back(a, ep, p.T, s_tpref[staged_stack], b, G);
            __syncthreads();
            const long long pre = s_prefix;
            place(staged_stack, stage0, staged_count, pre, false);
            if (s_tpref[staged_stack + 1] <= p.t1 && tid == 0)
                a.cnt[staged_stack].spawn_total = (unsigned long long)(pre + staged_count);
            __syncthreads();
            // its counts belong to the staged stack
            unsigned long long *L = a.cnt[staged_stack].led;
            const unsigned long long v3 = block_sum_u64(ty.hits, s_r);
            if (tid == 0 && v3) atomicAdd(&L[L_IFACE_HITS], v3);
            const unsigned long long v4 = block_sum_u64(ty.trans, s_r);
            if (tid == 0 && v4) atomicAdd(&L[L_IFACE_TRANSMIT], v4);
            const unsigned long long v5 = block_sum_u64(ty.trunc, s_r);
            if (tid == 0 && v5) atomicAdd(&L[L_TRUNCATED], v5);
            const unsigned long long v6 = block_sum_u64(ty.spawn_drop, s_r);
            if (tid == 0 && v6) atomicAdd(&L[L_SPAWN_DROPPED], v6);
            const unsigned long long v7 = block_sum_u64(ty.q_drop, s_r);
            if (tid == 0 && v7) atomicAdd(&L[L_Q_DROPPED], v7);
            ty = Tally{};
        }
    }

    if (last_block(a, &s_flag)) {
        for (int s = tid; s < a.n_stacks; s += TPB) {
            if (s_tpref[s + 1] == s_tpref[s]) continue;
            DevCounters &c = a.cnt[s];
            const long long room = a.stacks[s].cap - (long long)c.n_slots;
            const long long tot = (long long)c.spawn_total;
            const long long kept = tot < room ? tot : (room > 0 ? room : 0);
            c.n_slots += (unsigned long long)kept;
            c.next_id += (unsigned long long)kept;
            c.spawn_total = 0;
        }
        if (tid == 0) {
            a.ctl->done = 0u;
            a.ctl->epoch = ep + 1u;
        }
    }
}

// ---------------------------------------------------------------------------
// k_inject: Source(dt/2) for half step h = 2*step + half (Eq. Strang-source)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_inject(const Args a, int half, int deposit)
{
    __shared__ long long s_pref[PIC_MAX_STACKS + 1];
    __shared__ long long s_n[PIC_MAX_STACKS];
    __shared__ unsigned long long s_q[PIC_MAX_STACKS];
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    const long long h = 2 * (long long)a.step + half;
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    for (int s = tid; s < a.n_stacks; s += TPB) {
        const DevStack &st = a.stacks[s];
        const long long n = a.inj[st.inj_off + h];
        const long long room = st.cap - (long long)a.cnt[s].n_slots;
        s_n[s] = n < room ? n : (room > 0 ? room : 0);
        s_q[s] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        long long acc = 0;
        for (int s = 0; s < a.n_stacks; ++s) { s_pref[s] = acc; acc += s_n[s]; }
        s_pref[a.n_stacks] = acc;
    }
    __syncthreads();
    const long long total = s_pref[a.n_stacks];
    const int tout = (int)((a.step + 1) / (uint32_t)a.moment_every) - 1;
    for (long long gidx = (long long)blockIdx.x * TPB + tid; gidx < total;
         gidx += (long long)gridDim.x * TPB) {
        const int s = stack_of(s_pref, a.n_stacks, gidx);
        const long long j = gidx - s_pref[s];
        const DevStack &st = a.stacks[s];
        const unsigned long long id = a.cnt[s].next_id + (unsigned long long)j;
        const uint32_t cy = (uint32_t)(id >> 32) | ((uint32_t)s << 16);
        const uint4 r0 = philox(make_uint4((uint32_t)id, cy, a.step, SUB_INJ + 0), a.seed_lo,
                                a.seed_hi);
        const uint4 r1 = philox(make_uint4((uint32_t)id, cy, a.step, SUB_INJ + 1), a.seed_lo,
                                a.seed_hi);
        int i = 0;
        const uint32_t *thr = a.cdf_thr + st.cdf_off;
        while (i < st.n_cdf - 1 && !(r0.x < thr[i])) ++i;
        const int cell = a.cdf_cell[st.cdf_off + i];
        const float z = __fmul_rn(__fadd_rn((float)cell, unit_of(r0.y)), a.dz);
        const uint32_t sg = r0.z < st.up_thr ? 0u : 1u;
        const uint32_t k = st.e_mode == 1 ? (uint32_t)(sg ? st.k_mono1 : st.k_mono0)
                                          : 1u + __umulhi(r0.w, (uint32_t)a.n_e);
        const uint32_t layer = (uint32_t)a.cdf_layer[st.cdf_off + i];
        const long long d = st.base + (long long)a.cnt[s].n_slots + j;
        a.z[cur][d] = z;
        a.mu[cur][d] = mu_of(r1.x);
        a.id[cur][d] = (uint32_t)id;
        a.pk[cur][d] = k | (sg << 8) | (layer << 9) | (1u << 13) | ((uint32_t)(id >> 32) << 21);
        atomicAdd(&s_q[s], (unsigned long long)k);
        if (deposit) {
            Stk tmp; tmp.n_cells = st.n_cells;
            const int c = cell_of(a, tmp, z);
            atomicAdd(&a.n_hist[st.n_off + (long long)tout * 2 * a.n_e * st.n_cells +
                                (sg * a.n_e + (k - 1)) * st.n_cells + c], 1u);
        }
    }
    __syncthreads();
    for (int s = tid; s < a.n_stacks; s += TPB)
        if (s_q[s]) atomicAdd(&a.cnt[s].led[L_Q_INJECTED], s_q[s]);
    if (last_block(a, &s_flag)) {
        for (int s = tid; s < a.n_stacks; s += TPB) {
            const DevStack &st = a.stacks[s];
            const long long n = a.inj[st.inj_off + h];
            DevCounters &c = a.cnt[s];
            const long long kept = s_n[s];
            c.n_slots += (unsigned long long)kept;
            c.next_id += (unsigned long long)kept;
            c.led[L_INJECTED] += (unsigned long long)kept;
            c.led[L_INJECT_DROPPED] += (unsigned long long)(n - kept);
            if (n > kept && (a.flags & PIC_F_STRICT_CAPACITY))
                atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_CAPACITY);
        }
        if (tid == 0) a.ctl->done = 0u;
    }
}

// ---------------------------------------------------------------------------
// k_compact: stable removal of dead slots (k = 0) into the other buffer
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_compact(const Args a)
{
    __shared__ long long s_tpref[PIC_MAX_STACKS + 1];
    __shared__ long long s_nsl[PIC_MAX_STACKS];
    __shared__ int s_w[TPB / 32];
    __shared__ long long s_prefix;
    __shared__ int s_flag;
    const unsigned int ep = *(volatile unsigned int *)&a.ctl->epoch;
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur, nxt = cur ^ 1;
    const int b = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
    Plan p;
    make_plan(a, s_tpref, s_nsl, p);

    auto alive4 = [&](int s, long long t, uint32_t &mask) {
        const DevStack &st = a.stacks[s];
        const long long nsl = s_nsl[s];
        const long long slot0 = (t - s_tpref[s]) * TILE + (long long)tid * VEC;
        mask = 0;
        if (slot0 < nsl) {
            const uint4 p4 = *reinterpret_cast<const uint4 *>(a.pk[cur] + st.base + slot0);
            const uint32_t *pp = &p4.x;
#pragma unroll
            for (int j = 0; j < VEC; ++j)
                if (slot0 + j < nsl && (pp[j] & 0xFFu)) mask |= 1u << j;
        }
    };

    if (p.t0 < p.t1) {
        const int s_first = stack_of(s_tpref, a.n_stacks, p.t0);
        const int s_last = stack_of(s_tpref, a.n_stacks, p.t1 - 1);
        const bool first_inside = p.t0 > s_tpref[s_first];
        // phase 1: count the first segment (if it needs the look-back) and the
        // last segment (its count is what later blocks need)
        long long c_first = 0, c_last = 0;
        for (long long t = p.t0; t < p.t1; ++t) {
            const int s = stack_of(s_tpref, a.n_stacks, t);
            const bool need = (s == s_first && first_inside) || s == s_last;
            if (!need) { t = s_tpref[s + 1] - 1; continue; }
            uint32_t m;
            alive4(s, t, m);
            int excl;
            const int tot = block_scan(__popc(m), excl, s_w);
            if (s == s_first) c_first += tot;
            if (s == s_last) c_last += tot;
        }
        long long pre_first = 0;
        if (tid == 0) {
            if (s_last == s_first && first_inside) {
                publish(&a.status[b], ep, FLAG_A, c_last);
                s_prefix = look_back(a, ep, p.T, s_tpref[s_first], b, G);
                publish(&a.status[b], ep, FLAG_P, s_prefix + c_last);
            } else {
                publish(&a.status[b], ep, FLAG_P, c_last);
                s_prefix = first_inside ? look_back(a, ep, p.T, s_tpref[s_first], b, G) : 0;
            }
        }
        __syncthreads();
        pre_first = s_prefix;
        (void)c_first;
        // phase 2: scatter live slots, stable, into the other buffer
        int seg = -1;
        long long run = 0;
        for (long long t = p.t0; t < p.t1; ++t) {
            const int s = stack_of(s_tpref, a.n_stacks, t);
            if (s != seg) {
                if (seg >= 0 && s_tpref[seg + 1] <= p.t1 && tid == 0)
                    a.cnt[seg].alive_total = (unsigned long long)run;
                seg = s;
                run = (s == s_first) ? pre_first : 0;
            }
            uint32_t m;
            alive4(s, t, m);
            int excl;
            const int tot = block_scan(__popc(m), excl, s_w);
            if (m) {
                const DevStack &st = a.stacks[s];
                const long long src = st.base + (t - s_tpref[s]) * TILE + (long long)tid * VEC;
                long long d = st.base + run + excl;
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    if (!((m >> j) & 1u)) continue;
                    a.z[nxt][d] = a.z[cur][src + j];
                    a.mu[nxt][d] = a.mu[cur][src + j];
                    a.id[nxt][d] = a.id[cur][src + j];
                    a.pk[nxt][d] = a.pk[cur][src + j];
                    ++d;
                }
            }
            run += tot;
        }
        if (seg >= 0 && s_tpref[seg + 1] <= p.t1 && tid == 0)
            a.cnt[seg].alive_total = (unsigned long long)run;
    }

    if (last_block(a, &s_flag)) {
        for (int s = tid; s < a.n_stacks; s += TPB) {
            DevCounters &c = a.cnt[s];
            c.n_slots = (s_tpref[s + 1] == s_tpref[s]) ? 0ull : c.alive_total;
            c.alive_total = 0;
        }
        if (tid == 0) {
            a.ctl->cur = (unsigned int)nxt;
            a.ctl->done = 0u;
            a.ctl->epoch = ep + 1u;
        }
    }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
template <bool DET, bool DEPN, bool WAGG>
static cudaError_t occupancy(size_t smem, int *blocks)
{
    // allow the largest dynamic shared memory the device offers, so that
    // contexts with different moment grids never lower each other's cap
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_step<DET, DEPN, WAGG>);
    if (e != cudaSuccess) return e;
    const int cap = optin - (int)fa.sharedSizeBytes;
    if ((int)smem > cap) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(k_step<DET, DEPN, WAGG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             cap);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_step<DET, DEPN, WAGG>, TPB,
                                                         smem);
}

cudaError_t configure(const Args &a, int blocks_per_sm, int hist_mode, LaunchCfg *cfg)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const size_t base = (size_t)a.tab_max * sizeof(TabEnt) + (size_t)a.T_max * 4 +
                        (size_t)a.jbin_max * 4;
    cfg->smem_step = (base + 15) & ~(size_t)15;
    cfg->smem_step_dep = (base + (size_t)a.nbin_max * 4 + 15) & ~(size_t)15;
    int occ[4] = {0, 0, 0, 0};
    // every template instance gets the attribute; the grids use the smallest
    // occupancy among the instances that share a shared-memory size
    const bool w = hist_mode == 1;
    if ((e = occupancy<false, false, false>(cfg->smem_step, &occ[0])) != cudaSuccess) return e;
    if ((e = occupancy<true, false, false>(cfg->smem_step, &occ[1])) != cudaSuccess) return e;
    if (w) {
        if ((e = occupancy<false, true, true>(cfg->smem_step_dep, &occ[2])) != cudaSuccess) return e;
        if ((e = occupancy<true, true, true>(cfg->smem_step_dep, &occ[3])) != cudaSuccess) return e;
    } else {
        if ((e = occupancy<false, true, false>(cfg->smem_step_dep, &occ[2])) != cudaSuccess) return e;
        if ((e = occupancy<true, true, false>(cfg->smem_step_dep, &occ[3])) != cudaSuccess) return e;
    }
    int o_plain = occ[0] < occ[1] ? occ[0] : occ[1];
    int o_dep = occ[2] < occ[3] ? occ[2] : occ[3];
    if (o_plain < 1 || o_dep < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm > 0) {
        o_plain = blocks_per_sm < o_plain ? blocks_per_sm : o_plain;
        o_dep = blocks_per_sm < o_dep ? blocks_per_sm : o_dep;
    }
    cfg->grid_step = sms * o_plain;
    cfg->grid_step_dep = sms * o_dep;
    int oc = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_compact, TPB, 0)) != cudaSuccess)
        return e;
    cfg->grid_compact = sms * (oc > 0 ? oc : 1);
    cfg->grid_inject = sms * 4;
    return cudaSuccess;
}

cudaError_t launch_step(const Args &a, const LaunchCfg &c, bool det, bool dep, int hist_mode,
                        cudaStream_t s)
{
    const int g = dep ? c.grid_step_dep : c.grid_step;
    const size_t sm = dep ? c.smem_step_dep : c.smem_step;
    const bool w = hist_mode == 1;
    if (det) {
        if (dep) {
            if (w) k_step<true, true, true><<<g, TPB, sm, s>>>(a);
            else k_step<true, true, false><<<g, TPB, sm, s>>>(a);
        } else {
            k_step<true, false, false><<<g, TPB, sm, s>>>(a);
        }
    } else {
        if (dep) {
            if (w) k_step<false, true, true><<<g, TPB, sm, s>>>(a);
            else k_step<false, true, false><<<g, TPB, sm, s>>>(a);
        } else {
            k_step<false, false, false><<<g, TPB, sm, s>>>(a);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_inject(const Args &a, const LaunchCfg &c, int half, bool deposit,
                          cudaStream_t s)
{
    k_inject<<<c.grid_inject, TPB, 0, s>>>(a, half, deposit ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_compact(const Args &a, const LaunchCfg &c, cudaStream_t s)
{
    k_compact<<<c.grid_compact, TPB, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
