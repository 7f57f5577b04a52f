// Device code of the PIC step (sm_103a): helpers and the kernel templates.
// Included by pic_kernels.cu (the forward step) and pic_adjoint.cu (the
// adjoint replay); each translation unit instantiates what it launches.
//
// One Strang step (Eq. strang, Sec. III.A) is, per stack:
//   k_inject(half 0)   Source(dt/2): append new carriers
//   k_stream           Transport(dt/2) -> Scattering(dt) -> Transport(dt/2)
//                      for every carrier that neither scatters nor meets a
//                      boundary in the step; the others are queued
//   k_event            the general step for the queued carriers; secondaries
//                      staged at their parents' positions
//   k_place            slots and ids of the secondaries, in parent slot order
//   k_inject(half 1)   Source(dt/2), deposited at moment steps
//   k_compact          every compact_every steps: stable removal of dead slots
//
// The tiles of all stacks are concatenated and cut into one contiguous chunk
// per block.  Secondary carriers are placed by a decoupled look-back over the
// blocks' chunks (a running count published as a tagged 64-bit word), so
// slot order and ids equal those of a scalar loop over the slots; every wait
// on another block is bounded and reports PIC_ERR_TIMEOUT.  Densities and
// fluxes are privatised in shared memory and flushed once per block and
// stack segment.
//
// ADJ (template parameter of the step kernels) selects the adjoint replay:
// 0 is the forward step; 1 and 2 are the two replay passes of the
// score-function gradient, which run the same trajectories (same slots, same
// Philox words) and carry one double per slot instead of depositing moments.

#pragma once
#include <cuda_runtime.h>

#include "pic_internal.h"

namespace pic {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// with the round multipliers 0xD2511F53 / 0xCD9E8D57; the key of round r is
// key + r * (0x9E3779B9, 0xBB67AE85).
// ---------------------------------------------------------------------------
// Philox4x32-10 with the ten round keys taken from the kernel arguments
// (precomputed on the host), so no key arithmetic runs per call
__device__ __forceinline__ uint4 philox_rk(uint4 c, const Args &a)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * c.x;
        const unsigned long long p1 = 0xCD9E8D57ull * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ a.rk0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ a.rk1[r], (uint32_t)p0);
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

// The time-step index: the kernel argument, or (steps replayed from a CUDA
// graph) the device counter that the last kernel of every step advances; it
// changes only between kernels, so a plain L2 load reads it.  (A volatile
// access here made the compiler copy the whole argument block to local
// memory.)
__device__ __forceinline__ uint32_t step_now(const Args &a)
{
    return a.step_dev ? __ldcg(a.step_dev) : a.step;
}

// advance the device step counter (last block of the step's last kernel)
__device__ __forceinline__ void bump_step(const Args &a)
{
    if (a.bump_step && a.step_dev) *const_cast<unsigned int *>(a.step_dev) += 1u;
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
    uint32_t ctr_hi;     // (stack_base + stack) << 16
    const double2 *aT;   // adjoint: interface scores of the stack (global memory)
};

// Cell of a depth z >= 0: floor(z / dz), clamped to the last cell.  dz is a
// power of two, so q = z * (1/dz) is exact; adding 2^23 with rounding toward
// -inf leaves floor(q) in the low mantissa bits (0 <= q < 2^23).
__device__ __forceinline__ int cell_of(const Args &a, const Stk &s, float z)
{
    const float q = __fmul_rn(z, a.inv_dz);
    const int c = __float_as_int(__fadd_rd(q, 8388608.0f)) - 0x4B000000;
    return c < s.n_cells - 1 ? c : s.n_cells - 1;
}

// Transport for a time tau (Eq. Strang-transport, Sec. III): free flight in
// the current layer, mirror reflection at the vacuum surfaces, a uniform
// draw against T at an interface (transmit: layer changes, mu kept;
// reflect: mu mirrored), the remaining time flown in the new layer.
// e, lo, hi: table entry and edges of the current layer (updated on transmission).
// SC (adjoint pass 2): each interface draw adds its score, d log P / d T of
// the outcome, times the carrier's reward-to-go R to the gradient bins gT
// (T_thr indexing of the stack).
template <bool DET, bool SC = false>
__device__ __forceinline__ void flight(const Args &a, const Stk &s, float &z, float &mu,
                                       int &layer, TabEnt &e, float &lo, float &hi, int sg,
                                       int k, float tau, uint32_t key_x, uint32_t key_y,
                                       uint32_t step, uint32_t sub0, Tally &t, double R = 0.0,
                                       double *gT = nullptr)
{
    for (int hit = 0;; ++hit) {
        const float w = __fmul_rn(e.v, mu);
        const float z1 = DET ? __fadd_rn(z, __fmul_rn(w, tau)) : __fmaf_rn(w, tau, z);
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
                const uint4 r = philox_rk(make_uint4(key_x, key_y, step, sub0 + (uint32_t)hit), a);
                const int ti = ((iface * 2 + dir) * 2 + sg) * s.n_e + (k - 1);
                trans = r.x < s.T[ti];
                if (SC && R != 0.0) {
                    const double2 sc = s.aT[ti];
                    atomicAdd(&gT[ti], (trans ? sc.x : sc.y) * R);
                }
            }
            if (trans) {
                layer += up ? 1 : -1;
                ++t.trans;
                e = s.ent[(layer * 2 + sg) * s.n_e + (k - 1)];
                lo = s.edge[layer];
                hi = s.edge[layer + 1];
            } else {
                mu = -mu;
            }
        }
    }
}

// Adjoint rewards (fixed point).  Flux: a carrier of spin sg moving from cell
// c0 to cell c1 in window tj earns the signed sum of the face weights it
// crosses, the difference of the potential gpot[c] = sum_{f=1..c} gJ[f].
// Density: the weight of the (spin, k, cell) bin it is counted in at the end
// of window tout.
__device__ __forceinline__ long long flux_w(const Args &a, int s, int tj, int sg, int c0, int c1)
{
    const long long *g = a.gpot + ((long long)(s * a.n_out + tj) * 2 + sg) * a.ncm;
    return g[c1] - g[c0];
}

__device__ __forceinline__ long long dep_w(const Args &a, int s, int tout, int sg, int k, int c)
{
    if (!a.gn) return 0;
    return a.gn[(((long long)(s * a.n_out + tout) * 2 + sg) * a.n_e + (k - 1)) * a.ncm + c];
}

__device__ __forceinline__ void add_flux(int32_t *sJ, int nf, int sg, int c0, int c1)
{
    if (c1 > c0) for (int f = c0 + 1; f <= c1; ++f) atomicAdd(&sJ[sg * nf + f], 1);
    else         for (int f = c1 + 1; f <= c0; ++f) atomicAdd(&sJ[sg * nf + f], -1);
}

// Barrier of the threads that run a 256-thread pass: the whole block in an
// ordinary launch; warps 0-7 in the persistent kernel, whose blocks have the
// streaming pass's 288 threads (its producer warp sits out the other passes).
// blockDim is uniform over a block, so the choice is too.
__device__ __forceinline__ void cta_sync()
{
    if (blockDim.x == TPB) __syncthreads();
    else asm volatile("bar.sync 2, %0;" ::"n"(TPB) : "memory");
}

__device__ __forceinline__ bool cta_sync_or(bool p)
{
    if (blockDim.x == TPB) return __syncthreads_or(p) != 0;
    uint32_t r;
    asm volatile("{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, 2, %2, q;\n"
                 " selp.u32 %0, 1, 0, o;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)p), "n"(TPB)
                 : "memory");
    return r != 0;
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
    cta_sync();
    if (wid == 0) {
        int w = lane < TPB / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < TPB / 32) s_w[lane] = w;        // inclusive warp totals
    }
    cta_sync();
    excl = x - v + (wid ? s_w[wid - 1] : 0);
    const int total = s_w[TPB / 32 - 1];
    cta_sync();
    return total;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long *s_r)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_r[threadIdx.x >> 5] = v;
    cta_sync();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < TPB / 32; ++i) t += s_r[i];
    cta_sync();
    return t;  // valid in thread 0
}

// Block sums of N per-thread counts in one reduction (one barrier instead
// of two per count): thread q < N receives the sum of count q.  s_w holds
// (TPB / 32) x N words.  A warp's sum of a count stays below 2^32 (a thread
// counts at most its share of a launch's items, times 59 quanta).
template <int N>
__device__ __forceinline__ unsigned long long block_sums(const uint32_t (&v)[N],
                                                         unsigned long long *s_w)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        uint32_t x = v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) s_w[warp * N + q] = x;
    }
    cta_sync();
    unsigned long long t = 0;
    if (threadIdx.x < N)
        for (int w = 0; w < TPB / 32; ++w) t += s_w[w * N + threadIdx.x];
    cta_sync();
    return t;
}

// 64-bit shared-memory sum as two native 32-bit atomic additions: the low
// word's old value gives the carry into the high word exactly, so the pair
// holds the sum modulo 2^64 (whatever the order of the additions).
__device__ __forceinline__ void add_u64_split(unsigned long long *p, unsigned long long v)
{
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    const uint32_t lo = (uint32_t)v;
    const uint32_t old = atomicAdd(&w[0], lo);
    const uint32_t hi = (uint32_t)(v >> 32) + (uint32_t)(old + lo < old);
    if (hi) atomicAdd(&w[1], hi);
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
// this block's chunk (the stack's tiles start at ts): walk back over the
// blocks whose chunks end inside the same stack, 32 of them at a time (one
// per lane of the calling warp, every lane of which must call), each with a
// bounded wait for its status word, down to the nearest block that has
// published an inclusive prefix.  `lo(j)` is the first tile of block j.
template <class Lo>
static __device__ long long look_back_warp(const Args &a, unsigned int ep, long long ts, int b,
                                           Lo lo)
{
    const int lane = threadIdx.x & 31;
    long long prefix = 0;
    for (int j0 = b - 1; j0 >= 0; j0 -= 32) {
        const int j = j0 - lane;
        // 2: the walk stops before this block; 1: an inclusive prefix; 0: an
        // aggregate, or a block without tiles
        int kind = 0;
        long long v = 0;
        if (j < 0) {
            kind = 2;
        } else {
            const long long jt0 = lo(j), jt1 = lo(j + 1);
            if (jt1 <= ts) {
                kind = 2;
            } else if (jt0 != jt1) {
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
                v = (long long)(w & 0x3FFFFFFFull);
                if (((w >> 30) & 3ull) == FLAG_P) kind = 1;
            }
        }
        // the nearest block that ends the walk, and the sum up to it
        const unsigned int term = __ballot_sync(0xffffffffu, kind != 0);
        const int tl = term ? __ffs(term) - 1 : 32;
        long long c = (lane < tl || (lane == tl && kind == 1)) ? v : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        prefix += c;
        if (term) break;
    }
    return prefix;
}

__device__ __forceinline__ long long look_back(const Args &a, unsigned int ep, long long T,
                                               long long ts, int b, int G)
{
    return look_back_warp(a, ep, ts, b, [&](int j) { return T * j / G; });
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
    cta_sync();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < a.n_stacks; ++i) {
            s_tpref[i] = acc;
            acc += (s_nsl[i] + TILE - 1) / TILE;
        }
        s_tpref[a.n_stacks] = acc;
    }
    cta_sync();
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
    cta_sync();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(&a.ctl->done, 1u);
        *s_flag = (t == gridDim.x - 1);
    }
    cta_sync();
    const bool last = *s_flag != 0;
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ void load_stack(const Args &a, int s, Stk &k, DevStack *s_st,
                                           TabEnt *s_ent, uint32_t *s_T, float *s_edge,
                                           uint32_t *s_p0)
{
    cta_sync();
    if (threadIdx.x == 0) *s_st = a.stacks[s];
    cta_sync();
    const DevStack &st = *s_st;
    for (int i = threadIdx.x; i < st.tab_n; i += TPB) s_ent[i] = a.ent[st.ent_off + i];
    for (int i = threadIdx.x; i < st.T_n; i += TPB) s_T[i] = a.T_thr[st.T_off + i];
    if (threadIdx.x <= st.n_layers) s_edge[threadIdx.x] = st.edge[threadIdx.x];
    if (threadIdx.x < st.n_layers) s_p0[threadIdx.x] = st.p0_thr[threadIdx.x];
    k.ent = s_ent; k.T = s_T; k.edge = s_edge; k.p0 = s_p0;
    k.n_layers = st.n_layers; k.n_cells = st.n_cells; k.n_e = a.n_e;
    k.ctr_hi = (uint32_t)(a.stack_base + s) << 16;
    k.aT = a.aT ? a.aT + st.T_off : nullptr;
}

// ---------------------------------------------------------------------------
// Tensor-memory-accelerator (bulk copy) helpers: 1-D cp.async.bulk of a tile
// of each particle array into a shared-memory ring, completion tracked by an
// mbarrier per ring stage.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One poll; a thread whose phase has not completed may be suspended, for at
// most `hint_ns` (the instruction's suspend-time hint), so that a wait
// bounded in polls is bounded in time too.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity,
                                              uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false if the phase did not complete within `limit` polls or
// within PIC_WAIT_NS of the global timer, whichever comes first.
#ifndef PIC_WAIT_NS
#define PIC_WAIT_NS 4000000000ull
#endif
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity,
                                          unsigned int limit)
{
    if (mbar_try_wait(bar, parity, 20000u)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned int it = 1; it < limit; ++it) {
        if (mbar_try_wait(bar, parity, 20000u)) return true;
        if (global_ns() - t0 > PIC_WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

constexpr int MAX_RING = 8;
constexpr uint32_t TILE_BYTES = TILE * 4u;      // one array of one tile

// Chunk of block j of a grid of G blocks over T tiles: [T*j/G, T*(j+1)/G).
__device__ __forceinline__ long long chunk_lo(long long T, int j, int G)
{
    return T * j / G;
}

// Tiles of placement block j: the union of the chunks of the streaming
// blocks [Gf*j/Gs, Gf*(j+1)/Gs), so that it covers whole streaming chunks.
__device__ __forceinline__ long long slow_lo(long long T, int j, int Gs, int Gf)
{
    return chunk_lo(T, (int)((long long)Gf * j / Gs), Gf);
}

// Exclusive prefix of the secondaries of the stack segment that starts slow
// block b's chunk (stack tiles start at ts); warp-wide, as look_back_warp.
__device__ __forceinline__ long long look_back_place(const Args &a, unsigned int ep, long long T,
                                                     long long ts, int b, int Gs, int Gf)
{
    return look_back_warp(a, ep, ts, b, [&](int j) { return slow_lo(T, j, Gs, Gf); });
}

// tile prefix over the stacks, in dynamic shared memory
__device__ __forceinline__ long long make_tiles(const Args &a, long long *s_tpref, long long *s_nsl)
{
    for (int i = threadIdx.x; i < a.n_stacks; i += TPB) s_nsl[i] = (long long)a.cnt[i].n_slots;
    cta_sync();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < a.n_stacks; ++i) {
            s_tpref[i] = acc;
            acc += (s_nsl[i] + TILE - 1) / TILE;
        }
        s_tpref[a.n_stacks] = acc;
    }
    cta_sync();
    return s_tpref[a.n_stacks];
}

// index of a carrier's entry in the padded streaming-pass table
__device__ __forceinline__ int fast_index(const Args &a, uint32_t pk)
{
    return (int)((pk & a.kmask) | ((pk >> a.kshr) & a.hmask));
}

// the velocity along z in fixed point: float32 product, 2^-32 nm/fs units,
// truncated toward zero (exact sums, independent of their order)
__device__ __forceinline__ long long vel_q(float w)
{
    return __float2ll_rz(__fmul_rn(w, 4294967296.0f));
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Shared memory and step constants of the general step (the event pass, and
// the event warps of the streaming pass in its fused form).
struct EvEnv {
    float *Z, *MU;                       // current buffer: depths, (mu, packed) pairs
    uint32_t step;
    float half;
    int cur, tj, tout;
    bool vmom;
    int32_t *s_J;                        // removals per (spin, cell)
    uint32_t *s_n, *s_gs;                // density steps: histograms
    unsigned long long *s_v;
    double *s_g, *s_gT;                  // adjoint pass 2: gradient bins
};

// The general step of one queued carrier (record rec: its depth, mu, packed
// word and position within its streaming block's tiles), of stack s whose
// tables S holds; f: its streaming block, whose first position is fpos0;
// tile0: the stack's first tile; room0: the stack's buffer was full before
// the step (secondaries are dropped).  TW: the slot's scattering-test word
// is given (xs_in, drawn by the streaming pass) instead of drawn again.
template <bool DET, bool DEPN, int ADJ, bool TW = false>
__device__ __forceinline__ void event_item(const Args &a, const DevStack &st, const Stk &S,
                                           const EvEnv &E, Tally &ty, int s, int f,
                                           long long fpos0, long long tile0, bool room0,
                                           const float4 rec, uint32_t xs_in = 0u)
{
    const int cur = E.cur, tj = E.tj, tout = E.tout;
    const uint32_t step = E.step;
    const float half = E.half;
    const bool vmom = E.vmom;
    float *Z = E.Z, *MU = E.MU;
    int32_t *s_J = E.s_J;
    uint32_t *s_n = E.s_n, *s_gs = E.s_gs;
    unsigned long long *s_v = E.s_v;
    double *s_g = E.s_g, *s_gT = E.s_gT;
    (void)cur; (void)tj; (void)tout; (void)vmom; (void)s_J; (void)s_n; (void)s_gs; (void)s_v;
    (void)s_g; (void)s_gT;
    const long long sbase = st.base - tile0 * TILE;          // position -> slot
    float z = rec.x, mu = rec.y;
    uint32_t pk = __float_as_uint(rec.z);
    const long long vpos = fpos0 + __float_as_uint(rec.w);
    const long long gslot = sbase + vpos;
    const long long slot = vpos - tile0 * TILE;       // slot within the stack
    int k = (int)(pk & 0xFFu);
    const float mu_in = mu;
    const uint32_t pk_in = pk;
    const int sg = (int)((pk >> 8) & 1u);
    int layer = (int)((pk >> 9) & 0xFu);
    const uint32_t key_x = (uint32_t)slot;              // draws keyed by the slot
    TabEnt e = S.ent[(layer * 2 + sg) * S.n_e + (k - 1)];
    float lo = S.edge[layer], hi = S.edge[layer + 1];
    const int c_start = ADJ ? cell_of(a, S, z) : 0;     // the replay's flux reward
    // adjoint: the slot's reward sum; in pass 2 the reward-to-go R
    // that weights every decision of this step
    const long long R = ADJ == 2 ? a.acc[cur][gslot] : 0;
    const double Rd = ADJ == 2 ? (double)R * a.inv_q : 0.0;
    flight<DET, ADJ == 2>(a, S, z, mu, layer, e, lo, hi, sg, k, half, key_x, S.ctr_hi,
                          step, SUB_IF, ty, Rd, s_gT);
    const int tb = (layer * 2 + sg) * S.n_e + (k - 1);     // entry of the test
    // Scattering(dt): Monte-Carlo test against tau_eff (Eq. lifetimes):
    // the slot group's test word, then the carrier's event words
    uint32_t xs = xs_in;
    if (!TW) {
        const uint4 xg = philox_rk(make_uint4((uint32_t)(slot >> 2), S.ctr_hi, step,
                                              SUB_TEST), a);
        xs = (slot & 3) == 0 ? xg.x : (slot & 3) == 1 ? xg.y : (slot & 3) == 2 ? xg.z : xg.w;
    }
    bool dead = false;
    if (ADJ == 2 && !(xs < e.P) && Rd != 0.0) atomicAdd(&s_g[tb], a.aent[st.ent_off + tb].noscat * Rd);
    if (xs < e.P) {
        const uint4 x = philox_rk(make_uint4(key_x, S.ctr_hi, step, SUB_EVT), a);
        const bool inel = x.y < e.Q;
        // scores of the test (scattered) and of the channel
        if (ADJ == 2 && Rd != 0.0) {
            const AdjEnt &ae = a.aent[st.ent_off + tb];
            atomicAdd(&s_g[tb], (inel ? ae.scat_inel : ae.scat_el) * Rd);
        }
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
                e = S.ent[(layer * 2 + sg) * S.n_e + (k - 1)];
                if (a.flags & PIC_F_NO_SECONDARIES) {
                    ty.bath += (uint32_t)ks;
                } else if (room0) {
                    ++ty.spawn_drop;
                    ty.q_drop += (uint32_t)ks;
                    if (a.flags & PIC_F_STRICT_CAPACITY)
                        atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_CAPACITY);
                } else {
                    // secondary: same place, spin from P0, isotropic
                    const uint4 y = philox_rk(make_uint4(key_x, S.ctr_hi, step, SUB_SEC), a);
                    const uint32_t g0 = (pk >> 13) & 0xFFu;
                    const int sgs = y.x < S.p0[layer] ? 0 : 1;
                    const uint32_t gen = g0 < 255u ? g0 + 1u : 255u;
                    float zs = z, mus = mu_of(y.y), los = lo, his = hi;
                    int ls = layer;
                    TabEnt es = S.ent[(ls * 2 + sgs) * S.n_e + (ks - 1)];
                    Tally ts{};
                    flight<DET>(a, S, zs, mus, ls, es, los, his, sgs, ks, half, key_x,
                                S.ctr_hi, step, SUB_SIF, ts);
                    // the secondary's boundary events ride in the (not yet
                    // used) id_hi bits until it is placed
                    const uint32_t pks = (uint32_t)ks | ((uint32_t)sgs << 8) |
                                         ((uint32_t)ls << 9) | (gen << 13) |
                                         (ts.hits << 21) | (ts.trans << 25) |
                                         (ts.trunc << 29);
                    a.stage[vpos] = make_float4(zs, mus, __uint_as_float(pks), z);
                    if (ADJ == 2) a.stage_l[vpos] = (uint32_t)layer;
                    atomicOr(&a.spawn_bits[vpos >> 5], 1u << (vpos & 31));
                    atomicAdd(&a.fspawn[f], 1u);
                }
            }
        }
    }
    long long rw = 0;        // adjoint: reward of the step
    if (dead) {
        pk = (pk & ~0x1FFFu) | ((uint32_t)sg << 8) | ((uint32_t)layer << 9);
        const int c_end = cell_of(a, S, z);
        // a removal, where the carrier stopped (with its weight)
        if (!ADJ) {
            atomicAdd(&s_J[sg * (S.n_cells + 1) + c_end], -1);
            if (a.w[0])
                atomicAdd(reinterpret_cast<unsigned long long *>(a.bdw) + st.J_off +
                              ((long long)tj * 2 + sg) * (S.n_cells + 1) + c_end,
                          0ull - (unsigned long long)a.w[cur][gslot]);
        }
        if (ADJ) rw = flux_w(a, s, tj, sg, c_start, c_end);
    } else {
        flight<DET, ADJ == 2>(a, S, z, mu, layer, e, lo, hi, sg, k, half, key_x, S.ctr_hi,
                              step, SUB_IF + 16, ty, Rd, s_gT);
        const int c_end = cell_of(a, S, z);
        pk = (pk & ~0x1FFFu) | (uint32_t)k | ((uint32_t)sg << 8) | ((uint32_t)layer << 9);
        if (DEPN && !ADJ) {
            atomicAdd(&s_n[(sg * S.n_e + (k - 1)) * S.n_cells + c_end], 1u);
            atomicAdd(&s_gs[c_end], (pk >> 13) & 0xFFu);
            if (vmom)
                add_u64_split(&s_v[sg * S.n_cells + c_end], (unsigned long long)vel_q(__fmul_rn(e.v, mu)));
        }
        if (ADJ) {
            rw = flux_w(a, s, tj, sg, c_start, c_end);
            if (DEPN) rw += dep_w(a, s, tout, sg, k, c_end);
        }
    }
    if (ADJ == 1 && rw != 0) a.acc[cur][gslot] += rw;
    if (ADJ == 2 && rw != 0) a.acc[cur][gslot] = R - rw;
    Z[gslot] = z;
    if (__float_as_uint(mu) != __float_as_uint(mu_in) || pk != pk_in) {
        ++ty.changed;
        *reinterpret_cast<uint2 *>(MU + 2 * gslot) = make_uint2(__float_as_uint(mu), pk);
    }
}

// ---------------------------------------------------------------------------
// k_stream: the streaming pass (Transport(dt/2) -> Scattering(dt) ->
// Transport(dt/2) for every carrier that neither scatters nor meets a
// boundary in the step; the others are queued for k_event).
//
// Warp-specialised: one producer warp issues the bulk copies of a
// tile's z and (mu, packed) pairs into a ring of shared-memory stages with
// full/empty mbarriers; NW consumer warps each take G = TILE / (32 NW)
// consecutive slots per thread (4 or 8: one Philox call per four slots).
// What a carrier costs on an ordinary step: one index of the padded table
// straight from its packed word, the two half flights, two compares against
// the layer edges and one against the scattering threshold, and its new
// depth written back with the others of the thread.  Nothing else is
// counted per carrier: the flux through the cell faces follows from the
// densities at the ends of the moment windows and the births and removals
// in between (k_flux), and the carriers advanced in the step are the live
// count kept by the kernels that create and remove carriers.  On a density
// step the carriers finished here are also deposited (density, generation
// label and, with PIC_F_VELOCITY_MOMENTS, velocity) into shared-memory
// histograms flushed once per block and stack segment.
//
// ADJ = 1, 2: the same pass in the two replays of the adjoint: a finished
// carrier earns the flux weights of the faces it crossed and, on a density
// step, the weight of its bin.  Pass 1 adds a nonzero reward to the slot's
// sum in memory (most carriers earn none in a step); pass 2 streams the
// slots' rewards-to-go as a further array of the ring, subtracts the
// rewards and adds each reward-to-go to the no-scattering sum of its table
// entry.
//
// EV (the fused form, plain steps of a single stack): PIC_EV_WARPS further
// warps run the general step of the block's own eventful carriers while the
// consumers stream on, so that the scattered updates of a carrier's depth and
// (mu, packed) pair land in sectors the pass has just read or written, still
// in L2, instead of in a separate pass after the whole buffer has gone
// through.  A consumer hands each eventful carrier's record to a
// shared-memory ring after the tile's depths are stored; every ring entry has
// a sequence word (2p: free for position p; 2p + 1: holds position p), so the
// consumers and the event warps wait only on the entries they write or read.
// ---------------------------------------------------------------------------
// resident blocks per SM the register budget must allow: four of 288
// threads (eight consumer warps, 56 registers) or five of 160 (four consumer
// warps with eight slots per thread, 80 registers)
#ifndef PIC_STREAM_MIN_BLOCKS_8
#define PIC_STREAM_MIN_BLOCKS_8 4
#endif
#ifndef PIC_STREAM_MIN_BLOCKS_4
#define PIC_STREAM_MIN_BLOCKS_4 5
#endif
// the second replay carries the slots' rewards-to-go as well: three blocks
// (72 registers); the first fits four
#ifndef PIC_EV_WARPS
#define PIC_EV_WARPS 2             // event warps of the fused streaming pass
#endif
#ifndef PIC_EV_MIN_BLOCKS
#define PIC_EV_MIN_BLOCKS 3        // its resident blocks per SM (56 registers)
#endif
constexpr int EV_CAP = 512;        // entries of its event ring (a power of two)

template <int NW, int ADJ>
constexpr int stream_min_blocks()
{
    return ADJ == 2 ? 3 : ADJ == 1 ? 4 : (NW == 8 ? PIC_STREAM_MIN_BLOCKS_8 : PIC_STREAM_MIN_BLOCKS_4);
}

template <int NW>
__device__ __forceinline__ void stream_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(32 * NW) : "memory");
}

template <int NW>
__device__ __forceinline__ unsigned long long stream_sum_u64(unsigned long long v,
                                                             unsigned long long *s_r)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_r[threadIdx.x >> 5] = v;
    stream_sync<NW>();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NW; ++i) t += s_r[i];
    stream_sync<NW>();
    return t;  // valid in thread 0
}

template <int NW>
constexpr int stream_threads() { return 32 * NW + 32; }

template <bool DET, bool DEPN, bool WAGG, int NW, int ADJ = 0, int GR = 1, bool EV = false>
__device__ __forceinline__ void phase_stream(const Args &a)
{
    static_assert(!EV || (!DEPN && ADJ == 0 && GR == 1), "fused form: plain steps only");
    // GR groups of NW consumer warps take the tiles of the ring in turn (two
    // groups where the density-step histograms leave room for one block per
    // SM); each group covers a whole tile
    constexpr int NT = 32 * NW;              // consumer threads of a group
    constexpr int NTT = NT * GR;             // consumer threads
    constexpr int G = TILE / NT;             // slots per consumer thread and tile
    constexpr int NC = G / 4;                // Philox calls (and float4s) per thread
    // ring arrays: z, (mu, packed) and, in pass 2, the reward-to-go (pass 1
    // only adds to the rewards: it does so in memory, for the carriers that
    // earn one)
    constexpr int STG = ADJ == 2 ? 5 : 3;
    static_assert(G % 4 == 0 && G <= 8, "4 or 8 slots per thread");
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring = reinterpret_cast<float *>(smem);                      // a.ring x STG x TILE
    FastEnt *s_ent = reinterpret_cast<FastEnt *>(ring + (size_t)a.ring * STG * TILE);
    // forward density steps: histograms; replay: the window's flux potential
    // [2][n_cells], density weights [2][n_e][n_cells] and (pass 2) the
    // no-scattering sums of the reward-to-go per entry (fixed point)
    unsigned long long *s_sr = reinterpret_cast<unsigned long long *>(s_ent + a.ftab_max);
    long long *s_gp = reinterpret_cast<long long *>(s_sr + (ADJ == 2 ? a.tab_max : 0));
    uint32_t *s_n = reinterpret_cast<uint32_t *>(s_gp + (ADJ ? a.jbin_max : 0));
    int32_t *s_gn = reinterpret_cast<int32_t *>(s_n);
    uint32_t *s_gs = s_n + (DEPN ? a.nbin_max : 0);                     // generation sums
    unsigned long long *s_v = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(s_gs + (DEPN && !ADJ ? a.gbin_max : 0)) + 7) & ~uintptr_t(7));
    long long *s_tpref = reinterpret_cast<long long *>(s_v + (DEPN && !ADJ ? 2 * a.gbin_max : 0));
    long long *s_nsl = s_tpref + a.n_stacks + 1;
    // fused form: the stack's tables of the general step, its removals per
    // (spin, cell) and the event ring (records and their sequence words)
    TabEnt *s_tab = reinterpret_cast<TabEnt *>(
        (reinterpret_cast<uintptr_t>(s_nsl + a.n_stacks) + 15) & ~uintptr_t(15));
    uint32_t *s_T = reinterpret_cast<uint32_t *>(s_tab + (EV ? a.tab_max : 0));
    int32_t *s_J = reinterpret_cast<int32_t *>(s_T + (EV ? a.T_max : 0));
    float4 *s_erec = reinterpret_cast<float4 *>(
        (reinterpret_cast<uintptr_t>(s_J + (EV ? a.jbin_max : 0)) + 15) & ~uintptr_t(15));
    uint32_t *s_eseq = reinterpret_cast<uint32_t *>(s_erec + (EV ? EV_CAP : 0));
    uint32_t *s_ews = s_eseq + (EV ? EV_CAP : 0);        // the records' test words
    __shared__ __align__(8) unsigned long long s_full[MAX_RING], s_empty[MAX_RING];
    __shared__ DevStack s_st;
    __shared__ unsigned long long s_r[NW * GR];
    __shared__ int s_qn, s_abort;
    // fused form: ring positions reserved and claimed, consumer warps done,
    // the final count once they are, the event warps' ledger sums
    __shared__ unsigned int s_etail, s_eclaim, s_cdone, s_efin_n;
    __shared__ int s_efin;
    __shared__ unsigned long long s_ev8[EV ? 8 : 1];
    __shared__ DevStack s_est;
    __shared__ float s_eedge[EV ? PIC_MAX_LAYERS + 1 : 1];
    __shared__ uint32_t s_ep0[EV ? PIC_MAX_LAYERS : 1];

    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    const int b = blockIdx.x, G_ = gridDim.x, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const unsigned int lt_mask = (1u << lane) - 1u;
    for (int i = tid; i < a.n_stacks; i += (int)blockDim.x) {
        s_nsl[i] = (long long)a.cnt[i].n_slots;
        // the carriers advanced in this step: every live one (the counts
        // change only in the source, event and placement kernels)
        if (b == 0) a.cnt[i].led[L_PARTICLE_STEPS] += a.cnt[i].live;
    }
    if (tid == 0) {
        for (int i = 0; i < a.ring; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&s_empty[i], NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_qn = 0;
        s_abort = 0;
        if (EV) {
            s_etail = s_eclaim = s_cdone = s_efin_n = 0u;
            s_efin = 0;
            for (int k = 0; k < 8; ++k) s_ev8[k] = 0ull;
        }
    }
    if (EV)
        for (int i = tid; i < EV_CAP; i += (int)blockDim.x) s_eseq[i] = 2u * (uint32_t)i;   // free for i
    __syncthreads();
    if (tid == 0) {
        long long acc = 0;
        for (int i = 0; i < a.n_stacks; ++i) {
            s_tpref[i] = acc;
            acc += (s_nsl[i] + TILE - 1) / TILE;
        }
        s_tpref[a.n_stacks] = acc;
    }
    __syncthreads();
    const long long T = s_tpref[a.n_stacks];
    const long long t0 = chunk_lo(T, b, G_), t1 = chunk_lo(T, b + 1, G_);
    const long long ntiles = t1 - t0;
    const int nring = a.ring;
    float *Z = a.z[cur];
    const float *MP = a.mu[cur];         // mu and packed, interleaved

    // ---------------- producer warp ----------------
    if (warp == NW * GR) {
        if (lane == 0) {
            // the bulk copies (async proxy) read global memory written with
            // ordinary stores by earlier passes: within one persistent launch
            // that order needs this fence (between launches it is implied)
            asm volatile("fence.proxy.async;" ::: "memory");
            long long issued = 0;
            int stg = 0;
            uint32_t phase = 0;          // completions of stage stg so far, mod 2
            for (long long i = 0; i < ntiles; ++i) {
                if (i >= nring &&
                    !mbar_wait(&s_empty[stg], phase ^ 1u, a.spin_limit)) {
                    atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
                    a.ctl->timeout_where = 4u;
                    s_abort = 1;
                }
                if (*(volatile int *)&s_abort) break;
                const long long t = t0 + i;
                const int s = stack_of(s_tpref, a.n_stacks, t);
                const long long off = a.stacks[s].base + (t - s_tpref[s]) * TILE;
                float *dst = ring + (size_t)stg * STG * TILE;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&s_full[stg], STG * TILE_BYTES);
                bulk_load(dst, Z + off, TILE_BYTES, &s_full[stg]);
                bulk_load(dst + TILE, MP + 2 * off, 2 * TILE_BYTES, &s_full[stg]);
                if (ADJ == 2) bulk_load(dst + 3 * TILE, a.acc[cur] + off, 2 * TILE_BYTES, &s_full[stg]);
                issued = i + 1;
                if (++stg == nring) { stg = 0; phase ^= 1u; }
            }
            if (*(volatile int *)&s_abort) {
                // wait (bounded) for the copies that may still be in flight,
                // so that none lands in shared memory after the block exits
                for (long long i = issued > nring ? issued - nring : 0; i < issued; ++i)
                    mbar_wait(&s_full[(int)(i % nring)], (uint32_t)((i / nring) & 1), a.spin_limit);
            }
        }
        return;
    }

    // ---------------- event warps (fused form) ----------------
    if constexpr (EV) {
        if (warp > NW) {
            constexpr int NET = 32 * PIC_EV_WARPS;
            const int etid = tid - 32 * (NW + 1);
            auto ev_sync = [] { asm volatile("bar.sync 3, %0;" ::"n"(NET) : "memory"); };
            if (etid == 0) s_est = a.stacks[0];
            ev_sync();
            const DevStack &st = s_est;
            for (int i = etid; i < st.tab_n; i += NET) s_tab[i] = a.ent[st.ent_off + i];
            for (int i = etid; i < st.T_n; i += NET) s_T[i] = a.T_thr[st.T_off + i];
            if (etid <= st.n_layers) s_eedge[etid] = st.edge[etid];
            if (etid < st.n_layers) s_ep0[etid] = st.p0_thr[etid];
            const int nf = st.n_cells + 1;
            for (int i = etid; i < 2 * nf; i += NET) s_J[i] = 0;
            Stk S{};
            S.ent = s_tab; S.T = s_T; S.edge = s_eedge; S.p0 = s_ep0;
            S.n_layers = st.n_layers; S.n_cells = st.n_cells; S.n_e = a.n_e;
            S.ctr_hi = (uint32_t)a.stack_base << 16;
            S.aT = nullptr;
            const uint32_t step = step_now(a);
            const int tj = (int)(step / (uint32_t)a.moment_every);
            const EvEnv env{Z, a.mu[cur], step, a.half_dt, cur, tj, 0, false, s_J,
                            nullptr, nullptr, nullptr, nullptr, nullptr};
            const bool room0 = (st.cap - s_nsl[0]) <= 0;
            const long long tile0 = s_tpref[0];
            Tally ty{};
            ev_sync();
#pragma unroll 1
            for (;;) {
                // 32 ring positions at a time; a lane waits for its record,
                // or for the end of the queue before its position
                unsigned int base = 0;
                if (lane == 0) {
                    // claim once 32 records are reserved past the claims (or
                    // the ring is closed), polling one word with back-off
                    unsigned int ns = 32, it = 0;
                    const unsigned long long tw0 = global_ns();
                    while (*(volatile unsigned int *)&s_etail - *(volatile unsigned int *)&s_eclaim < 32u &&
                           !*(volatile int *)&s_efin && !*(volatile int *)&s_abort) {
                        __nanosleep(ns);
                        if (ns < 512) ns *= 2;
                        if (++it > a.spin_limit || ((it & 255u) == 0 && global_ns() - tw0 > PIC_WAIT_NS)) {
                            atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
                            a.ctl->timeout_where = 5u;
                            s_abort = 1;
                        }
                    }
                    base = atomicAdd(&s_eclaim, 32u);
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                const uint32_t pos = base + (uint32_t)lane;
                volatile uint32_t *sq = s_eseq + (pos & (EV_CAP - 1));
                bool have = false;
                unsigned int it = 0;
                unsigned long long t_start = 0;
                for (;;) {
                    if (*sq == 2u * pos + 1u) { have = true; break; }
                    if (*(volatile int *)&s_efin && pos >= *(volatile unsigned int *)&s_efin_n) break;
                    if (*(volatile int *)&s_abort) break;
                    if (it == 0) t_start = global_ns();
                    if (++it > a.spin_limit || ((it & 255u) == 0 && global_ns() - t_start > PIC_WAIT_NS)) {
                        atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
                        a.ctl->timeout_where = 5u;
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(64);
                }
                float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t xs = 0u;
                if (have) {
                    __threadfence_block();
                    rec = s_erec[pos & (EV_CAP - 1)];
                    xs = s_ews[pos & (EV_CAP - 1)];
                    __threadfence_block();
                    *sq = 2u * (pos + (uint32_t)EV_CAP);         // free for pos + EV_CAP
                }
                const unsigned int any = __ballot_sync(0xffffffffu, have);
                if (have)
                    event_item<DET, false, 0, true>(a, st, S, env, ty, 0, b, t0 * TILE, tile0, room0,
                                                    rec, xs);
                if (!any) break;
            }
            // the event warps' ledger counts and removals
            const uint32_t vals[8] = {ty.absorbed, ty.bath, ty.hits, ty.trans, ty.trunc,
                                      ty.spawn_drop, ty.q_drop, ty.changed};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t v = __reduce_add_sync(0xffffffffu, vals[k]);
                if (lane == 0 && v) atomicAdd(&s_ev8[k], (unsigned long long)v);
            }
            ev_sync();
            {
                int32_t *gB = a.bd_hist + st.J_off + (long long)tj * 2 * nf;
                for (int i = etid; i < 2 * nf; i += NET) {
                    const int v = s_J[i];
                    if (v) atomicAdd(&gB[i], v);
                }
            }
            if (etid < 8) {
                const unsigned long long v = s_ev8[etid];
                const int idx[8] = {L_ABSORBED, L_Q_BATH, L_IFACE_HITS, L_IFACE_TRANSMIT,
                                    L_TRUNCATED, L_SPAWN_DROPPED, L_Q_DROPPED, L_CHANGED};
                if (v) {
                    atomicAdd(&a.cnt[0].led[idx[etid]], v);
                    if (etid == 0) atomicAdd(&a.cnt[0].live, 0ull - v);   // removed carriers
                }
            }
            return;
        }
    }

    // ---------------- consumer warps ----------------
    const uint32_t step = step_now(a);
    const int tj = (int)(step / (uint32_t)a.moment_every);
    const int tout = (int)((step + 1) / (uint32_t)a.moment_every) - 1;
    const float half = a.half_dt;
    const long long pos0 = t0 * TILE;                // queue region of this block
    const bool vmom = DEPN && !ADJ && (a.flags & PIC_F_VELOCITY_MOMENTS);
    const int grp = GR > 1 ? warp / NW : 0;          // the thread's group
    const int ltid = tid - grp * NT;                 // its index within the group
    const int i0 = G * ltid;                         // its first slot in a tile
    int seg_stack = -1, nc = 1, ne = a.n_e;
    long long seg_t0 = 0, seg_t1 = -1;               // tiles of the current stack
    int nsl = 0;
    float *gZs = Z;
    uint32_t ctr_hi = 0;
    uint32_t n_queued = 0;

    auto flush = [&](int s) {
        stream_sync<NW * GR>();
        const DevStack &st = s_st;
        if (ADJ == 2) {
            // the no-scattering score of an entry times the sum of the
            // reward-to-go of the carriers that passed the test with it
            for (int i = tid; i < st.tab_n; i += NTT) {
                const long long v = (long long)s_sr[i];
                if (v) atomicAdd(&a.g_ent[st.ent_off + i], (double)v * a.inv_q * a.aent[st.ent_off + i].noscat);
            }
        }
        if (DEPN && !ADJ) {
            const int nbins = 2 * a.n_e * st.n_cells;
            uint32_t *gN = a.n_hist + st.n_off + (long long)tout * nbins;
            for (int i = tid; i < nbins; i += NTT) {
                const uint32_t v = s_n[i];
                if (v) atomicAdd(&gN[i], v);
            }
            unsigned long long *gG = a.g_hist + st.n_off / (2 * a.n_e) + (long long)tout * st.n_cells;
            for (int i = tid; i < st.n_cells; i += NTT) {
                const uint32_t v = s_gs[i];
                if (v) atomicAdd(&gG[i], (unsigned long long)v);
            }
            if (vmom) {
                unsigned long long *gV = reinterpret_cast<unsigned long long *>(a.v_hist) +
                                         st.n_off / a.n_e + (long long)tout * 2 * st.n_cells;
                for (int i = tid; i < 2 * st.n_cells; i += NTT) {
                    const unsigned long long v = s_v[i];
                    if (v) atomicAdd(&gV[i], v);
                }
            }
        }
        const unsigned long long v1 = stream_sum_u64<NW * GR>(n_queued, s_r);
        if (tid == 0 && v1) atomicAdd(&a.cnt[s].led[L_EVENTFUL], v1);
        n_queued = 0;
        stream_sync<NW * GR>();
    };

    int stg = 0;
    uint32_t phase = 0;                  // completions of full[stg] consumed, mod 2
    for (long long i = 0; i < ntiles; ++i) {
        const long long t = t0 + i;
        if (t >= seg_t1) {
            // a new stack segment: its tables, histograms and constants
            const int s = stack_of(s_tpref, a.n_stacks, t);
            if (seg_stack >= 0) flush(seg_stack);
            stream_sync<NW * GR>();
            if (tid == 0) s_st = a.stacks[s];
            stream_sync<NW * GR>();
            const DevStack &st = s_st;
            for (int q = tid; q < st.ftab_n; q += NTT) s_ent[q] = a.fent[st.fent_off + q];
            if (DEPN && !ADJ) {
                for (int q = tid; q < 2 * a.n_e * st.n_cells; q += NTT) s_n[q] = 0u;
                for (int q = tid; q < st.n_cells; q += NTT) s_gs[q] = 0u;
                if (vmom)
                    for (int q = tid; q < 2 * st.n_cells; q += NTT) s_v[q] = 0ull;
            }
            if (ADJ == 2)
                for (int q = tid; q < st.tab_n; q += NTT) s_sr[q] = 0ull;
            if (ADJ) {
                const long long *gp = a.gpot + (long long)(s * a.n_out + tj) * 2 * a.ncm;
                for (int q = tid; q < 2 * st.n_cells; q += NTT)
                    s_gp[q] = gp[(q / st.n_cells) * a.ncm + q % st.n_cells];
                if (DEPN) {
                    const int rows = 2 * a.n_e;
                    for (int q = tid; q < rows * st.n_cells; q += NTT)
                        s_gn[q] = a.gn ? a.gn[((long long)(s * a.n_out + tout) * rows + q / st.n_cells) * a.ncm +
                                              q % st.n_cells]
                                       : 0;
                }
            }
            nc = st.n_cells;
            ctr_hi = (uint32_t)(a.stack_base + s) << 16;
            seg_stack = s;
            seg_t0 = s_tpref[s];
            seg_t1 = s_tpref[s + 1];
            nsl = (int)s_nsl[s];
            gZs = Z + st.base;
            stream_sync<NW * GR>();
        }
        const int slot0 = (int)(t - seg_t0) * TILE;  // first slot of the tile in its stack
        const int nvalid = nsl - slot0;              // valid slots of the tile (>= 1)
        if (GR > 1 && (int)(i % GR) != grp) {           // the other group's tile
            if (++stg == nring) { stg = 0; phase ^= 1u; }
            continue;
        }
        // after a failed wait every later wait is skipped: the warps run the
        // same control flow to the end (results are invalid, the status says so)
        if (!*(volatile int *)&s_abort && !mbar_wait(&s_full[stg], phase, a.spin_limit)) {
            atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
            a.ctl->timeout_where = 3u;
            s_abort = 1;
        }
        const float *rz = ring + (size_t)stg * STG * TILE;
        const uint4 *rmp = reinterpret_cast<const uint4 *>(rz + TILE);   // (mu, packed) pairs
        float zin[G], min_[G];
        uint32_t pin[G];
        long long av[ADJ == 2 ? G : 1];      // pass 2: the slots' rewards-to-go
        if (ADJ == 2) {
            const longlong2 *racc = reinterpret_cast<const longlong2 *>(rz + 3 * TILE);
#pragma unroll
            for (int c = 0; c < G / 2; ++c) {
                const longlong2 v = racc[(G / 2) * ltid + c];
                av[2 * c] = v.x;
                av[2 * c + 1] = v.y;
            }
        }
        bool achg = false;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float4 z4 = reinterpret_cast<const float4 *>(rz)[NC * ltid + c];
            const uint4 q01 = rmp[2 * (NC * ltid + c)], q23 = rmp[2 * (NC * ltid + c) + 1];
            zin[4 * c] = z4.x; zin[4 * c + 1] = z4.y; zin[4 * c + 2] = z4.z; zin[4 * c + 3] = z4.w;
            min_[4 * c] = __uint_as_float(q01.x); min_[4 * c + 1] = __uint_as_float(q01.z);
            min_[4 * c + 2] = __uint_as_float(q23.x); min_[4 * c + 3] = __uint_as_float(q23.z);
            pin[4 * c] = q01.y; pin[4 * c + 1] = q01.w; pin[4 * c + 2] = q23.y; pin[4 * c + 3] = q23.w;
        }
        // the stage is no longer needed by this warp
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[stg]);
        if (++stg == nring) { stg = 0; phase ^= 1u; }
        // slots past the stack's end read the inert entry
        if (nvalid < TILE) {
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (i0 + j >= nvalid) pin[j] = 0u;
        }
        // scattering-test words: word (slot mod 4) of the call for slot / 4
        uint32_t xw[G];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const uint4 x = philox_rk(make_uint4((uint32_t)(slot0 >> 2) + (uint32_t)(NC * ltid + c),
                                                 ctr_hi, step, SUB_TEST), a);
            xw[4 * c] = x.x; xw[4 * c + 1] = x.y; xw[4 * c + 2] = x.z; xw[4 * c + 3] = x.w;
        }
        float zo[G];
        uint32_t slowbits = 0;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const uint32_t pk = pin[j];
            const FastEnt e = s_ent[fast_index(a, pk)];
            const float w = __fmul_rn(e.v, min_[j]);
            const float z1 = DET ? __fadd_rn(zin[j], __fmul_rn(w, half)) : __fmaf_rn(w, half, zin[j]);
            const float z2 = DET ? __fadd_rn(z1, __fmul_rn(w, half)) : __fmaf_rn(w, half, z1);
            // the motion is monotone within the step and the carrier starts
            // inside its layer: the end point decides whether it meets a boundary
            const bool slow = (z2 > e.hi) | (z2 < e.lo) | (xw[j] < e.P);
            zo[j] = z2;          // an eventful carrier's final depth is written by k_event
            slowbits |= (uint32_t)slow << j;
            if (ADJ) {
                // the reward of a finished carrier: the faces it crossed,
                // then its density bin; pass 2 sums its reward-to-go into the
                // no-scattering sum of its entry
                const uint32_t k = pk & 0xFFu;
                if (!slow && k != 0u) {
                    const int sg = (int)((pk >> 8) & 1u), layer = (int)((pk >> 9) & 0xFu);
                    const int c0u = __float_as_int(__fmaf_rd(zin[j], a.inv_dz, 8388608.0f)) - 0x4B000000;
                    const int c1u = __float_as_int(__fmaf_rd(z2, a.inv_dz, 8388608.0f)) - 0x4B000000;
                    const int c0 = c0u < nc - 1 ? c0u : nc - 1, c1 = c1u < nc - 1 ? c1u : nc - 1;
                    long long r = s_gp[sg * nc + c1] - s_gp[sg * nc + c0];
                    if (DEPN) r += s_gn[(sg * ne + (int)k - 1) * nc + c1];
                    if (ADJ == 2 && av[j] != 0)
                        add_u64_split(&s_sr[(layer * 2 + sg) * ne + (int)k - 1], (unsigned long long)av[j]);
                    if (r != 0) {
                        if (ADJ == 1) {
                            // pass 1: added in memory (this thread owns the slot)
                            atomicAdd(reinterpret_cast<unsigned long long *>(a.acc[cur]) + (gZs - Z) +
                                          slot0 + i0 + j,
                                      (unsigned long long)r);
                        } else {
                            av[j] -= r;
                            achg = true;
                        }
                    }
                }
            }
            if (DEPN && !ADJ) {
                int bin = -1;
                const uint32_t k = pk & 0xFFu;
                if (!slow && k != 0u) {
                    const int sg = (int)((pk >> 8) & 1u);
                    const int cu = __float_as_int(__fmaf_rd(z2, a.inv_dz, 8388608.0f)) - 0x4B000000;
                    const int c1 = cu < nc - 1 ? cu : nc - 1;
                    bin = (sg * ne + (int)k - 1) * nc + c1;
                    atomicAdd(&s_gs[c1], (pk >> 13) & 0xFFu);
                    if (vmom) add_u64_split(&s_v[sg * nc + c1], (unsigned long long)vel_q(w));
                }
                if (!WAGG && bin >= 0) atomicAdd(&s_n[bin], 1u);
                if (WAGG) {
                    const unsigned int m = __match_any_sync(0xffffffffu, bin);
                    if (bin >= 0 && lane == __ffs(m) - 1) atomicAdd(&s_n[bin], (uint32_t)__popc(m));
                }
            }
        }
        // new depths (only slots below n_slots are written)
        float *gZ = gZs + slot0 + i0;
        if (i0 + G <= nvalid) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
                reinterpret_cast<float4 *>(gZ)[c] =
                    make_float4(zo[4 * c], zo[4 * c + 1], zo[4 * c + 2], zo[4 * c + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (i0 + j < nvalid) gZ[j] = zo[j];
        }
        if (ADJ == 2 && achg) {
            long long *gA = a.acc[cur] + (gZs - Z) + slot0 + i0;
            if (i0 + G <= nvalid) {
#pragma unroll
                for (int c = 0; c < G / 2; ++c)
                    reinterpret_cast<longlong2 *>(gA)[c] = make_longlong2(av[2 * c], av[2 * c + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < G; ++j)
                    if (i0 + j < nvalid) gA[j] = av[j];
            }
        }
        // queue the eventful carriers (record and position), in tile order:
        // the warp's exclusive prefix of the per-thread counts (0..G) from
        // ballots of their bits, one shared-counter reservation per warp
        {
            const uint32_t cnt = (uint32_t)__popc(slowbits);
            constexpr int NB = G == 4 ? 3 : 4;       // bits of a count 0..G
            unsigned int bal[NB];
            int tot = 0;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                bal[q] = __ballot_sync(0xffffffffu, (cnt >> q) & 1u);
                tot += __popc(bal[q]) << q;
            }
            if (tot && EV) {
                // fused form: into the event ring, after the depths above
                unsigned int base = 0;
                if (lane == 0) base = atomicAdd(&s_etail, (unsigned int)tot);
                base = __shfl_sync(0xffffffffu, base, 0);
                uint32_t p = base;
#pragma unroll
                for (int r = 0; r < NB; ++r) p += (uint32_t)__popc(bal[r] & lt_mask) << r;
                n_queued += cnt;
                const uint32_t rel = (uint32_t)((t - t0) * TILE) + (uint32_t)i0;
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    if (!((slowbits >> j) & 1u)) continue;
                    volatile uint32_t *sq = s_eseq + (p & (EV_CAP - 1));
                    unsigned int it = 0;
                    unsigned long long t_start = 0;
                    while (*sq != 2u * p && !*(volatile int *)&s_abort) {
                        if (it == 0) t_start = global_ns();
                        if (++it > a.spin_limit ||
                            ((it & 255u) == 0 && global_ns() - t_start > PIC_WAIT_NS)) {
                            atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
                            a.ctl->timeout_where = 6u;
                            s_abort = 1;
                        }
                        __nanosleep(32);
                    }
                    if (*(volatile int *)&s_abort) break;
                    s_erec[p & (EV_CAP - 1)] = make_float4(zin[j], min_[j], __uint_as_float(pin[j]),
                                                           __uint_as_float(rel + (uint32_t)j));
                    s_ews[p & (EV_CAP - 1)] = xw[j];
                    __threadfence_block();       // the record and this tile's depths first
                    *sq = 2u * p + 1u;
                    ++p;
                }
            } else if (tot) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_qn, tot);
                base = __shfl_sync(0xffffffffu, base, 0);
                long long q = pos0 + base;
#pragma unroll
                for (int r = 0; r < NB; ++r) q += (long long)(__popc(bal[r] & lt_mask) << r);
                n_queued += cnt;
                const uint32_t rel = (uint32_t)((t - t0) * TILE) + (uint32_t)i0;
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    if ((slowbits >> j) & 1u) {
                        a.qrec[q++] = make_float4(zin[j], min_[j], __uint_as_float(pin[j]),
                                                  __uint_as_float(rel + (uint32_t)j));
                    }
                }
            }
        }
    }
    if (EV) {
        // the last consumer warp to finish closes the ring: no position at or
        // after the final count will be written
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&s_cdone, 1u) == (unsigned int)(NW - 1)) {
                *(volatile unsigned int *)&s_efin_n = *(volatile unsigned int *)&s_etail;
                __threadfence_block();
                *(volatile int *)&s_efin = 1;
            }
        }
    }
    if (seg_stack >= 0) flush(seg_stack);
    stream_sync<NW * GR>();
    if (tid == 0) a.qcnt[b] = (uint32_t)s_qn;
}

template <int NW, int GR, bool EV>
constexpr int stream_threads_of() { return 32 * NW * GR + 32 + (EV ? 32 * PIC_EV_WARPS : 0); }

template <bool DET, bool DEPN, bool WAGG, int NW, int ADJ = 0, int GR = 1, bool EV = false>
__global__ void __launch_bounds__(stream_threads_of<NW, GR, EV>(),
                                  EV ? PIC_EV_MIN_BLOCKS : GR > 1 ? 1 : stream_min_blocks<NW, ADJ>())
    k_stream(const Args a)
{
    phase_stream<DET, DEPN, WAGG, NW, ADJ, GR, EV>(a);
}

// ---------------------------------------------------------------------------
// k_event: the general step for the queued (eventful) carriers.
//
// The queues of all streaming blocks, concatenated in tile order, are cut
// into equal contiguous item ranges, one per block; no block waits on
// another.  Within its range a block takes the items of one stack at a time,
// handed to warps 32 at a time from a shared counter (a warp that drew cheap
// items takes more): interface draws against T, mirror reflection, elastic
// and inelastic scattering, removal in the lowest bin and secondary
// generation (Sec. III).  A secondary is staged at its parent's position
// with one bit in a bitmap and counted for its parent's streaming block;
// k_place gives it its slot.
// ---------------------------------------------------------------------------
#ifndef PIC_SLOW_MIN_BLOCKS
#define PIC_SLOW_MIN_BLOCKS 2      // resident blocks per SM of the event pass
#endif
template <bool DET, bool DEPN, int ADJ = 0>
__device__ __forceinline__ void phase_event(const Args &a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    TabEnt *s_ent = reinterpret_cast<TabEnt *>(smem);
    uint32_t *s_T = reinterpret_cast<uint32_t *>(s_ent + a.tab_max);
    // pass 2: gradient bins of the lifetime and transmittance entries
    double *s_g = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(s_T + a.T_max) + 7) & ~uintptr_t(7));
    double *s_gT = s_g + (ADJ == 2 ? a.tab_max : 0);
    // removals per (spin, cell) of this step (the births-minus-removals
    // histogram the fluxes are derived from)
    int32_t *s_J = reinterpret_cast<int32_t *>(s_gT + (ADJ == 2 ? a.T_max : 0));
    uint32_t *s_n = reinterpret_cast<uint32_t *>(s_J + (ADJ ? 0 : a.jbin_max));
    uint32_t *s_gs = s_n + a.nbin_max;       // density steps: generation labels per cell
    // density steps: velocity sums per (spin, cell)
    unsigned long long *s_v = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(s_n + (DEPN && !ADJ ? a.nbin_max + a.gbin_max : 0)) + 7) & ~uintptr_t(7));
    long long *s_tpref = reinterpret_cast<long long *>(s_v + (DEPN && !ADJ ? 2 * a.gbin_max : 0)) + 1;
    long long *s_nsl = s_tpref + a.n_stacks + 1;
    long long *s_qpre = s_nsl + a.n_stacks;      // queue prefix over the streaming blocks
    __shared__ float s_edge[PIC_MAX_LAYERS + 1];
    __shared__ uint32_t s_p0[PIC_MAX_LAYERS];
    __shared__ DevStack s_st;
    __shared__ int s_w[TPB / 32];
    __shared__ unsigned long long s_r[TPB / 32];
    __shared__ unsigned long long s_r8[(TPB / 32) * 8];    // block sums of the ledger counts
    __shared__ unsigned long long s_next;
    __shared__ long long s_cut;

    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    const int b = blockIdx.x, G = gridDim.x, Gf = a.grid_fast, tid = threadIdx.x;
    const int lane = tid & 31;
    const bool vmom = DEPN && !ADJ && (a.flags & PIC_F_VELOCITY_MOMENTS);
    const long long T = make_tiles(a, s_tpref, s_nsl);
    const uint32_t step = step_now(a);
    const int tj = (int)(step / (uint32_t)a.moment_every);
    const int tout = (int)((step + 1) / (uint32_t)a.moment_every) - 1;
    const float half = a.half_dt;
    float *Z = a.z[cur], *MU = a.mu[cur];       // MU: (mu, packed) pairs

    // exclusive prefix of the queue lengths: item i of the concatenated queue
    // is entry i - s_qpre[f] of streaming block f
    long long run = 0;
    for (int c0 = 0; c0 < Gf; c0 += TPB) {
        const int f = c0 + tid;
        const int v = f < Gf ? (int)a.qcnt[f] : 0;
        int excl;
        const int tot = block_scan(v, excl, s_w);
        if (f < Gf) s_qpre[f] = run + excl;
        run += tot;
    }
    if (tid == 0) s_qpre[Gf] = run;
    cta_sync();
    const long long M = s_qpre[Gf];
    const long long i0 = M * b / G, i1 = M * (b + 1) / G;

    auto fast_block_of = [&](long long i) -> int {       // last f with s_qpre[f] <= i
        int lo = 0, hi = Gf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_qpre[mid] <= i) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    auto tile_of = [&](long long i) -> long long {
        const int f = fast_block_of(i);
        const long long ft0 = chunk_lo(T, f, Gf);
        return ft0 + (long long)(__float_as_uint(a.qrec[ft0 * TILE + (i - s_qpre[f])].w) / TILE);
    };
    auto first_at = [&](long long lo, long long hi, long long tb) -> long long {
        while (lo < hi) {                                 // items are in tile order
            const long long mid = (lo + hi) >> 1;
            if (tile_of(mid) < tb) lo = mid + 1; else hi = mid;
        }
        return lo;
    };

    Stk S{};
    Tally ty{};

    auto flush_segment = [&](int s) {
        cta_sync();
        const DevStack &st = s_st;
        const int nf = st.n_cells + 1;
        if (!ADJ) {
            int32_t *gB = a.bd_hist + st.J_off + (long long)tj * 2 * nf;
            for (int i = tid; i < 2 * nf; i += TPB) {
                const int v = s_J[i];
                if (v) atomicAdd(&gB[i], v);
            }
        }
        if (ADJ == 2) {
            for (int i = tid; i < st.tab_n; i += TPB)
                if (s_g[i] != 0.0) atomicAdd(&a.g_ent[st.ent_off + i], s_g[i]);
            for (int i = tid; i < st.T_n; i += TPB)
                if (s_gT[i] != 0.0) atomicAdd(&a.g_T[st.T_off + i], s_gT[i]);
        }
        if (DEPN && !ADJ) {
            const int nb = 2 * a.n_e * st.n_cells;
            uint32_t *gN = a.n_hist + st.n_off + (long long)tout * nb;
            for (int i = tid; i < nb; i += TPB) {
                const uint32_t v = s_n[i];
                if (v) atomicAdd(&gN[i], v);
            }
            unsigned long long *gG = a.g_hist + st.n_off / (2 * a.n_e) + (long long)tout * st.n_cells;
            for (int i = tid; i < st.n_cells; i += TPB) {
                const uint32_t v = s_gs[i];
                if (v) atomicAdd(&gG[i], (unsigned long long)v);
            }
            if (vmom) {
                unsigned long long *gV = reinterpret_cast<unsigned long long *>(a.v_hist) +
                                         st.n_off / a.n_e + (long long)tout * 2 * st.n_cells;
                for (int i = tid; i < 2 * st.n_cells; i += TPB) {
                    const unsigned long long v = s_v[i];
                    if (v) atomicAdd(&gV[i], v);
                }
            }
        }
        unsigned long long *L = a.cnt[s].led;
        const uint32_t vals[8] = {ty.absorbed, ty.bath, ty.hits, ty.trans, ty.trunc,
                                  ty.spawn_drop, ty.q_drop, ty.changed};
        const unsigned long long v = block_sums<8>(vals, s_r8);
        if (tid < 8 && v) {
            const int idx[8] = {L_ABSORBED, L_Q_BATH, L_IFACE_HITS, L_IFACE_TRANSMIT, L_TRUNCATED,
                                L_SPAWN_DROPPED, L_Q_DROPPED, L_CHANGED};
            atomicAdd(&L[idx[tid]], v);
            // removed carriers leave the live count
            if (tid == 0) atomicAdd(&a.cnt[s].live, 0ull - v);
        }
        ty = Tally{};
        cta_sync();
    };

    // the general step for item i of the concatenated queue, of stack s
    // (whose tables are loaded); f: its streaming block
    const EvEnv env{Z, MU, step, half, cur, tj, tout, vmom, s_J, s_n, s_gs, s_v, s_g, s_gT};
    auto item = [&](int s, long long i, int f, const float4 rec) {
        (void)i;
        event_item<DET, DEPN, ADJ>(a, s_st, S, env, ty, s, f, chunk_lo(T, f, Gf) * TILE, s_tpref[s],
                                   (s_st.cap - s_nsl[s]) <= 0, rec);
    };

    if (i0 < i1) {
        const int s_first = stack_of(s_tpref, a.n_stacks, tile_of(i0));
        const int s_last = stack_of(s_tpref, a.n_stacks, tile_of(i1 - 1));
        long long lo = i0;
        for (int s = s_first; s <= s_last; ++s) {
            if (s_tpref[s + 1] == s_tpref[s]) continue;       // a stack with no tiles
            if (tid == 0) s_cut = s == s_last ? i1 : first_at(lo, i1, s_tpref[s + 1]);
            load_stack(a, s, S, &s_st, s_ent, s_T, s_edge, s_p0);
            const long long hi = s_cut;
            if (!ADJ)
                for (int q = tid; q < 2 * (s_st.n_cells + 1); q += TPB) s_J[q] = 0;
            if (DEPN && !ADJ) {
                for (int q = tid; q < 2 * a.n_e * s_st.n_cells; q += TPB) s_n[q] = 0u;
                for (int q = tid; q < s_st.n_cells; q += TPB) s_gs[q] = 0u;
                if (vmom)
                    for (int q = tid; q < 2 * s_st.n_cells; q += TPB) s_v[q] = 0ull;
            }
            if (ADJ == 2) {
                for (int q = tid; q < s_st.tab_n; q += TPB) s_g[q] = 0.0;
                for (int q = tid; q < s_st.T_n; q += TPB) s_gT[q] = 0.0;
            }
            if (tid == 0) s_next = (unsigned long long)lo;
            cta_sync();
            // A warp takes 32 items at a time and loads the records of its
            // next batch while it runs the current one.
            auto grab = [&](long long &i, int &f, float4 &rec) -> bool {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&s_next, 32ull);
                base = __shfl_sync(0xffffffffu, base, 0);
                if ((long long)base >= hi) return false;
                // the batch's first streaming block, then at most a step or
                // two (a streaming block queues thousands of items)
                int ff = 0;
                if (lane == 0) ff = fast_block_of((long long)base);
                ff = __shfl_sync(0xffffffffu, ff, 0);
                i = (long long)base + lane;
                if (i < hi) {
                    while (s_qpre[ff + 1] <= i) ++ff;
                    rec = a.qrec[chunk_lo(T, ff, Gf) * TILE + (i - s_qpre[ff])];
                }
                f = ff;
                return true;
            };
            long long i_next = 0;
            int f_next = 0;
            float4 rec_next = make_float4(0.f, 0.f, 0.f, 0.f);
            bool more = grab(i_next, f_next, rec_next);
#pragma unroll 1
            while (more) {
                const long long i = i_next;
                const int f = f_next;
                const float4 rec = rec_next;
                more = grab(i_next, f_next, rec_next);
                if (i < hi) item(s, i, f, rec);
            }
            flush_segment(s);
            lo = hi;
        }
    }
}

template <bool DET, bool DEPN, int ADJ = 0>
__global__ void __launch_bounds__(TPB, PIC_SLOW_MIN_BLOCKS) k_event(const Args a)
{
    phase_event<DET, DEPN, ADJ>(a);
}

// ---------------------------------------------------------------------------
// k_place: slots and ids of the secondaries staged by k_event.
//
// Block j covers the tiles of streaming blocks [Gf j/Gp, Gf (j+1)/Gp).  The
// secondaries of a stack take the slots after the stack's live ones in the
// order of their parents' positions (the id order of a sequential loop over
// the slots): a block's rank offset in a stack is the number of the stack's
// secondaries in earlier blocks, found by a decoupled look-back with a
// bounded wait.  Every block publishes its own count before it waits.
// ---------------------------------------------------------------------------
template <bool DET, bool DEPN, int ADJ = 0>
__device__ __forceinline__ void phase_place(const Args &a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    // births per (spin, cell) of this step (the births-minus-removals
    // histogram the fluxes are derived from)
    int32_t *s_J = reinterpret_cast<int32_t *>(smem);
    uint32_t *s_n = reinterpret_cast<uint32_t *>(s_J + (ADJ ? 0 : a.jbin_max));
    uint32_t *s_gs = s_n + a.nbin_max;       // density steps: generation labels per cell
    // density steps: velocity sums per (spin, cell)
    unsigned long long *s_v = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(s_n + (DEPN && !ADJ ? a.nbin_max + a.gbin_max : 0)) + 7) & ~uintptr_t(7));
    long long *s_tpref = reinterpret_cast<long long *>(s_v + (DEPN && !ADJ ? 2 * a.gbin_max : 0)) + 1;
    long long *s_nsl = s_tpref + a.n_stacks + 1;
    __shared__ int s_w[TPB / 32];
    __shared__ unsigned long long s_r[TPB / 32];
    __shared__ unsigned long long s_r8[(TPB / 32) * 8];    // block sums of the ledger counts
    __shared__ long long s_pre[2], s_cl;
    __shared__ int s_flag;

    const unsigned int ep = *(volatile unsigned int *)&a.ctl->epoch;
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    const int b = blockIdx.x, Gs = gridDim.x, Gf = a.grid_fast, tid = threadIdx.x;
    const bool vmom = DEPN && !ADJ && (a.flags & PIC_F_VELOCITY_MOMENTS);
    const long long T = make_tiles(a, s_tpref, s_nsl);
    {
        // every stack's buffer was full before the step: the event pass
        // dropped every secondary, so nothing is staged, counted or placed;
        // one block ends the launch (the epoch of the look-back words, the
        // device step counter)
        bool full = true;
        for (int s = 0; s < a.n_stacks && full; ++s) full = a.stacks[s].cap - s_nsl[s] <= 0;
        if (full) {
            if (b == 0 && tid == 0) {
                a.ctl->epoch = ep + 1u;
                bump_step(a);
            }
            return;
        }
    }
    const int fb0 = (int)((long long)Gf * b / Gs), fb1 = (int)((long long)Gf * (b + 1) / Gs);
    const long long t0 = chunk_lo(T, fb0, Gf), t1 = chunk_lo(T, fb1, Gf);
    const uint32_t step = step_now(a);
    const int tj = (int)(step / (uint32_t)a.moment_every);
    const int tout = (int)((step + 1) / (uint32_t)a.moment_every) - 1;
    const float half = a.half_dt;
    float *Z = a.z[cur], *MU = a.mu[cur];       // MU: (mu, packed) pairs
    const uint32_t *PK = a.pk[cur];
    Tally ty{};

    // Adjoint bookkeeping of a secondary placed at slot d with id `id`, staged
    // at tile-space position pos (its parent's position).  Pass 1 records the
    // parent and starts the secondary's own reward with its birth step; pass
    // 2 flies the secondary's first half step again (the same words) to add
    // its interface scores weighted by its lineage total, which it still has
    // to earn and which its parent has now earned.
    auto place_adj = [&](int s, const DevStack &stg, long long pos, long long d,
                         unsigned long long id, uint32_t pk, int sg, int k, int c0, int c1,
                         const float4 &r) {
        const long long pslot = stg.base + pos - s_tpref[s] * TILE;
        const uint32_t ppk = PK[2 * pslot], pid_lo = a.id[cur][pslot];
        const unsigned long long pid = (unsigned long long)pid_lo | ((unsigned long long)(ppk >> 21) << 32);
        if (id >= (unsigned long long)stg.n_ids || pid >= (unsigned long long)stg.n_ids) {
            atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_STATE);
            return;
        }
        long long rw = flux_w(a, s, tj, sg, c0, c1);
        if (DEPN) rw += dep_w(a, s, tout, sg, k, c1);
        if (ADJ == 1) {
            const unsigned int depth = (unsigned int)a.gen[stg.id_off + pid] + 1u;
            a.parent[stg.id_off + id] = (unsigned long long)(stg.id_off + pid);
            a.gen[stg.id_off + id] = (uint8_t)depth;
            atomicMax(a.gen_max, depth);
            a.acc[cur][d] = rw;
        } else {
            const long long Rc = a.tot[stg.id_off + id];
            const uint32_t key_x = (uint32_t)(pos - s_tpref[s] * TILE);   // the parent's slot
            const uint32_t key_y = (uint32_t)(a.stack_base + s) << 16;
            const uint4 y = philox_rk(make_uint4(key_x, key_y, step, SUB_SEC), a);
            Stk gs;
            gs.ent = a.ent + stg.ent_off; gs.T = a.T_thr + stg.T_off;
            gs.edge = a.stacks[s].edge; gs.p0 = nullptr;
            gs.n_layers = stg.n_layers; gs.n_cells = stg.n_cells; gs.n_e = a.n_e;
            gs.ctr_hi = (uint32_t)(a.stack_base + s) << 16; gs.aT = a.aT + stg.T_off;
            int ls = (int)a.stage_l[pos];
            TabEnt es = gs.ent[(ls * 2 + sg) * a.n_e + (k - 1)];
            float los = gs.edge[ls], his = gs.edge[ls + 1];
            float zs = r.w, mus = mu_of(y.y);
            Tally tq{};
            flight<DET, true>(a, gs, zs, mus, ls, es, los, his, sg, k, half, key_x, key_y,
                              step, SUB_SIF, tq, (double)Rc * a.inv_q, a.g_T + stg.T_off);
            // the same words give the same flight: anything else means the
            // replay is not the forward run
            if (__float_as_uint(zs) != __float_as_uint(r.x))
                atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_STATE);
            a.acc[cur][d] = Rc - rw;
            a.acc[cur][pslot] -= Rc;
        }
    };

    // Place the staged secondaries of stack s in tiles [tl0, tl1) in slot
    // order, the first with rank `prefix` among the stack's secondaries of
    // this step; clears the bitmap words it reads; deposits into the shared
    // histograms.  Returns the number of the segment's secondaries.
    auto place = [&](int s, long long tl0, long long tl1, long long prefix) -> long long {
        const DevStack stg = a.stacks[s];
        const long long nsl = s_nsl[s];
        const long long room = stg.cap - nsl;
        const unsigned long long nid = a.cnt[s].next_id;
        const int nf = stg.n_cells + 1;
        uint32_t kept = 0;
        Stk tmp;
        tmp.n_cells = stg.n_cells;
        long long run = prefix;
        // q consecutive bitmap words per thread: PW where the words left fill
        // the block that way, fewer (down to one) near the end of the range,
        // so that a short range still spreads over all the threads
        constexpr int PW = 8;
        const long long w0 = tl0 * (TILE / 32), w1 = tl1 * (TILE / 32);
        for (long long wb = w0; wb < w1;) {
            const long long left = w1 - wb;
            const int q = left >= (long long)PW * TPB ? PW : (int)((left + TPB - 1) / TPB);
            const long long span = left < (long long)q * TPB ? left : (long long)q * TPB;
            const long long wt = wb + (long long)q * tid, we = wb + span;
            uint32_t wd[PW];
#pragma unroll
            for (int u = 0; u < PW; ++u) wd[u] = (u < q && wt + u < we) ? a.spawn_bits[wt + u] : 0u;
            int cnt = 0;
#pragma unroll
            for (int u = 0; u < PW; ++u) cnt += __popc(wd[u]);
            if (!cta_sync_or(cnt != 0)) {               // no secondary here
                wb += span;
                continue;
            }
            int excl;
            const int tot = block_scan(cnt, excl, s_w);
            if (cnt) {
#pragma unroll
                for (int u = 0; u < PW; ++u)
                    if (wd[u]) a.spawn_bits[wt + u] = 0u;
            }
            long long g = run + excl;
#pragma unroll 1
            for (int u = 0; u < q; ++u) {
                uint32_t bits = wd[0];                  // word u, by selects (no local array)
#pragma unroll
                for (int v = 1; v < PW; ++v)
                    if (u == v) bits = wd[v];
                const long long w = wt + u;
                while (bits) {
                    const int j = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const float4 r = a.stage[w * 32 + j];
                    const uint32_t pk_staged = __float_as_uint(r.z);
                    const uint32_t pk = pk_staged & 0x1FFFFFu;
                    if (g < room) {
                        ty.hits += (pk_staged >> 21) & 0xFu;
                        ty.trans += (pk_staged >> 25) & 0xFu;
                        ty.trunc += (pk_staged >> 29) & 0x1u;
                        const unsigned long long id = nid + (unsigned long long)g;
                        const long long d = stg.base + nsl + g;
                        Z[d] = r.x;
                        *reinterpret_cast<uint2 *>(MU + 2 * d) =
                            make_uint2(__float_as_uint(r.y), pk | ((uint32_t)(id >> 32) << 21));
                        a.id[cur][d] = (uint32_t)id;
                        ++kept;
                        const int sg = (int)((pk >> 8) & 1u), k = (int)(pk & 0xFFu);
                        const int c0 = cell_of(a, tmp, r.w), c1 = cell_of(a, tmp, r.x);
                        if (ADJ) {
                            place_adj(s, stg, w * 32 + j, d, id, pk, sg, k, c0, c1, r);
                        } else {
                            // a birth, where the parent created it; the
                            // secondary carries its parent's weight
                            atomicAdd(&s_J[sg * nf + c0], 1);
                            if (a.w[0]) {
                                const long long pos = w * 32 + j;
                                const uint32_t wp = a.w[cur][stg.base + pos - s_tpref[s] * TILE];
                                a.w[cur][d] = wp;
                                atomicAdd(reinterpret_cast<unsigned long long *>(a.bdw) + stg.J_off +
                                              ((long long)tj * 2 + sg) * nf + c0,
                                          (unsigned long long)wp);
                            }
                            if (DEPN) {
                                atomicAdd(&s_n[(sg * a.n_e + (k - 1)) * stg.n_cells + c1], 1u);
                                atomicAdd(&s_gs[c1], (pk >> 13) & 0xFFu);
                                if (vmom) {
                                    const int ls = (int)((pk >> 9) & 0xFu);
                                    const float v = a.ent[stg.ent_off + (ls * 2 + sg) * a.n_e + (k - 1)].v;
                                    add_u64_split(&s_v[sg * stg.n_cells + c1],
                                                  (unsigned long long)vel_q(__fmul_rn(v, r.y)));
                                }
                            }
                        }
                    } else {
                        ++ty.spawn_drop;
                        ty.q_drop += pk & 0xFFu;
                    }
                    ++g;
                }
            }
            run += tot;
            wb += span;
        }
        const unsigned long long kk = block_sum_u64(kept, s_r);
        if (tid == 0 && kk) atomicAdd(&a.cnt[s].led[L_SPAWNED], kk);
        if (tid == 0 && (a.flags & PIC_F_STRICT_CAPACITY) && run > room)
            atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_CAPACITY);
        return run - prefix;
    };

    // deposits and boundary tallies of the placed secondaries of stack s
    auto flush = [&](int s) {
        cta_sync();
        const DevStack &st = a.stacks[s];
        const int nf = st.n_cells + 1;
        if (!ADJ) {
            int32_t *gB = a.bd_hist + st.J_off + (long long)tj * 2 * nf;
            for (int i = tid; i < 2 * nf; i += TPB) {
                const int v = s_J[i];
                if (v) atomicAdd(&gB[i], v);
            }
        }
        if (DEPN && !ADJ) {
            const int nb = 2 * a.n_e * st.n_cells;
            uint32_t *gN = a.n_hist + st.n_off + (long long)tout * nb;
            for (int i = tid; i < nb; i += TPB) {
                const uint32_t v = s_n[i];
                if (v) atomicAdd(&gN[i], v);
            }
            unsigned long long *gG = a.g_hist + st.n_off / (2 * a.n_e) + (long long)tout * st.n_cells;
            for (int i = tid; i < st.n_cells; i += TPB) {
                const uint32_t v = s_gs[i];
                if (v) atomicAdd(&gG[i], (unsigned long long)v);
            }
            if (vmom) {
                unsigned long long *gV = reinterpret_cast<unsigned long long *>(a.v_hist) +
                                         st.n_off / a.n_e + (long long)tout * 2 * st.n_cells;
                for (int i = tid; i < 2 * st.n_cells; i += TPB) {
                    const unsigned long long v = s_v[i];
                    if (v) atomicAdd(&gV[i], v);
                }
            }
        }
        unsigned long long *L = a.cnt[s].led;
        const uint32_t vals[5] = {ty.hits, ty.trans, ty.trunc, ty.spawn_drop, ty.q_drop};
        const unsigned long long v = block_sums<5>(vals, s_r8);
        if (tid < 5 && v) {
            const int idx[5] = {L_IFACE_HITS, L_IFACE_TRANSMIT, L_TRUNCATED, L_SPAWN_DROPPED,
                                L_Q_DROPPED};
            atomicAdd(&L[idx[tid]], v);
        }
        ty = Tally{};
        cta_sync();
    };

    // staged secondaries in tiles [tl0, tl1): the block's count (thread 0)
    auto count_bits = [&](long long tl0, long long tl1) -> long long {
        unsigned long long c = 0;
        for (long long w = tl0 * (TILE / 32) + tid; w < tl1 * (TILE / 32); w += TPB)
            c += (unsigned long long)__popc(a.spawn_bits[w]);
        return (long long)block_sum_u64(c, s_r);
    };

    if (t0 < t1) {
        const int s_first = stack_of(s_tpref, a.n_stacks, t0);
        const int s_last = stack_of(s_tpref, a.n_stacks, t1 - 1);
        const bool inside_first = t0 > s_tpref[s_first];     // first segment starts inside its stack
        const bool inside_last = s_first == s_last && inside_first;
        long long c_first = 0, c_last = 0;
        if (s_first == s_last) {
            // one stack: the streaming blocks' counts
            unsigned long long c = 0;
            for (int f = fb0 + tid; f < fb1; f += TPB) c += a.fspawn[f];
            c_last = (long long)block_sum_u64(c, s_r);
        } else {
            if (inside_first) c_first = count_bits(t0, s_tpref[s_first + 1]);
            c_last = count_bits(s_tpref[s_last] > t0 ? s_tpref[s_last] : t0, t1);
        }
        for (int f = fb0 + tid; f < fb1; f += TPB) a.fspawn[f] = 0u;   // consumed
        if (tid < 32) {
            // the count of the last segment goes out before any wait; the
            // look-back takes the whole warp
            if (!inside_last) {
                if (tid == 0) {
                    publish(&a.status[b], ep, FLAG_P, c_last);
                    s_pre[1] = 0;
                }
            } else {
                if (tid == 0) publish(&a.status[b], ep, FLAG_A, c_last);
                const long long pre = look_back_place(a, ep, T, s_tpref[s_last], b, Gs, Gf);
                if (tid == 0) {
                    s_pre[1] = pre;
                    publish(&a.status[b], ep, FLAG_P, pre + c_last);
                }
            }
            const long long pre0 = (s_first < s_last && inside_first)
                                       ? look_back_place(a, ep, T, s_tpref[s_first], b, Gs, Gf) : 0;
            if (tid == 0) {
                s_pre[0] = pre0;
                s_cl = c_last;
            }
        }
        cta_sync();
        (void)c_first;
        for (int s = s_first; s <= s_last; ++s) {
            const long long sg0 = s_tpref[s] > t0 ? s_tpref[s] : t0;
            const long long sg1 = s_tpref[s + 1] < t1 ? s_tpref[s + 1] : t1;
            if (sg0 >= sg1) continue;                   // a stack with no tiles
            const long long prefix = s == s_last ? s_pre[1] : (s == s_first ? s_pre[0] : 0);
            if (s == s_last && s_cl == 0) {
                // no secondary staged in the segment: nothing to place or deposit
                if (sg1 == s_tpref[s + 1] && tid == 0) a.cnt[s].spawn_total = (unsigned long long)prefix;
                continue;
            }
            const int nc = a.stacks[s].n_cells;
            if (!ADJ)
                for (int q = tid; q < 2 * (nc + 1); q += TPB) s_J[q] = 0;
            if (DEPN && !ADJ) {
                for (int q = tid; q < 2 * a.n_e * nc; q += TPB) s_n[q] = 0u;
                for (int q = tid; q < nc; q += TPB) s_gs[q] = 0u;
                if (vmom)
                    for (int q = tid; q < 2 * nc; q += TPB) s_v[q] = 0ull;
            }
            cta_sync();
            const long long n = place(s, sg0, sg1, prefix);
            if (sg1 == s_tpref[s + 1] && tid == 0)
                a.cnt[s].spawn_total = (unsigned long long)(prefix + n);
            flush(s);
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
            c.live += (unsigned long long)kept;
            c.spawn_total = 0;
        }
        if (tid == 0) {
            a.ctl->done = 0u;
            a.ctl->epoch = ep + 1u;
            bump_step(a);
        }
    }
}

template <bool DET, bool DEPN, int ADJ = 0>
__global__ void __launch_bounds__(TPB) k_place(const Args a)
{
    phase_place<DET, DEPN, ADJ>(a);
}

// ---------------------------------------------------------------------------
// k_inject: Source(dt/2) for half step h = 2*step + half (Eq. Strang-source)
// ---------------------------------------------------------------------------
template <int ADJ = 0>
__device__ __forceinline__ void phase_inject(const Args &a, int half, int deposit)
{
    __shared__ long long s_pref[PIC_MAX_STACKS + 1];
    __shared__ long long s_n[PIC_MAX_STACKS];
    __shared__ unsigned long long s_q[PIC_MAX_STACKS];
    __shared__ unsigned long long s_wsum[PIC_MAX_STACKS];   // weights created
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    const uint32_t step = step_now(a);
    const long long h = 2 * (long long)step + half;
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    for (int s = tid; s < a.n_stacks; s += TPB) {
        const DevStack &st = a.stacks[s];
        const long long n = a.inj[st.inj_off + h];
        const long long room = st.cap - (long long)a.cnt[s].n_slots;
        s_n[s] = n < room ? n : (room > 0 ? room : 0);
        s_q[s] = 0;
        s_wsum[s] = 0;
    }
    cta_sync();
    if (tid == 0) {
        long long acc = 0;
        for (int s = 0; s < a.n_stacks; ++s) { s_pref[s] = acc; acc += s_n[s]; }
        s_pref[a.n_stacks] = acc;
    }
    cta_sync();
    const long long total = s_pref[a.n_stacks];
    const int tj = (int)(step / (uint32_t)a.moment_every);
    const int tout = (int)((step + 1) / (uint32_t)a.moment_every) - 1;
    const bool vmom = !ADJ && deposit && (a.flags & PIC_F_VELOCITY_MOMENTS);
    for (long long gidx = (long long)blockIdx.x * TPB + tid; gidx < total;
         gidx += (long long)gridDim.x * TPB) {
        const int s = stack_of(s_pref, a.n_stacks, gidx);
        const long long j = gidx - s_pref[s];
        const DevStack &st = a.stacks[s];
        const unsigned long long id = a.cnt[s].next_id + (unsigned long long)j;
        const uint32_t cy = (uint32_t)(id >> 32) | ((uint32_t)(a.stack_base + s) << 16);
        const uint4 r0 = philox_rk(make_uint4((uint32_t)id, cy, step, SUB_INJ + 0), a);
        const uint4 r1 = philox_rk(make_uint4((uint32_t)id, cy, step, SUB_INJ + 1), a);
        int i = 0;
        const uint32_t *thr = a.cdf_thr + st.cdf_off;
        while (i < st.n_cdf - 1 && !(r0.x < thr[i])) ++i;
        const int cell = a.cdf_cell[st.cdf_off + i];
        const float z = __fmul_rn(__fadd_rn((float)cell, unit_of(r0.y)), a.dz);
        const uint32_t sg = r0.z < st.up_thr ? 0u : 1u;
        uint32_t k;
        if (st.e_mode == 1) {
            k = (uint32_t)(sg ? st.k_mono1 : st.k_mono0);
        } else if (st.has_ebias) {
            // the bin from the biased sampling distribution (weights)
            const uint32_t *kt = a.kthr + (long long)s * a.n_e;
            k = 1u;
            while ((int)k < a.n_e && !(r0.w < kt[k - 1])) ++k;
        } else {
            k = 1u + __umulhi(r0.w, (uint32_t)a.n_e);
        }
        const uint32_t layer = (uint32_t)a.cdf_layer[st.cdf_off + i];
        const long long d = st.base + (long long)a.cnt[s].n_slots + j;
        a.z[cur][d] = z;
        *reinterpret_cast<uint2 *>(a.mu[cur] + 2 * d) = make_uint2(
            __float_as_uint(mu_of(r1.x)),
            k | (sg << 8) | (layer << 9) | (1u << 13) | ((uint32_t)(id >> 32) << 21));
        a.id[cur][d] = (uint32_t)id;
        atomicAdd(&s_q[s], (unsigned long long)k);
        uint32_t wq = 1u << 20;
        if (!ADJ && a.w[0]) {
            // weight p/q of the birth cell and bin (Eq. PIC), 2^-20 units
            const double wr = __dmul_rn(__dmul_rn(a.wcell[st.cdf_off + i],
                                                  a.wbin[(long long)s * a.n_e + k - 1]), 1048576.0);
            wq = wr < 1.0 ? 1u : (wr > 4294967295.0 ? 0xFFFFFFFFu : __double2uint_rn(wr));
            a.w[cur][d] = wq;
            atomicAdd(&s_wsum[s], (unsigned long long)wq);
        }
        if (!ADJ) {
            Stk tmp; tmp.n_cells = st.n_cells;
            const int c = cell_of(a, tmp, z);
            // a birth (the births-minus-removals histogram of the window);
            // the warp's carriers born in the same bin are added at once
            const long long bi = st.J_off + ((long long)tj * 2 + sg) * (st.n_cells + 1) + c;
            const unsigned int grp = __match_any_sync(__activemask(), (unsigned long long)bi);
            if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&a.bd_hist[bi], __popc(grp));
            if (a.w[0]) atomicAdd(reinterpret_cast<unsigned long long *>(a.bdw) + bi, (unsigned long long)wq);
            if (deposit) {
                atomicAdd(&a.n_hist[st.n_off + (long long)tout * 2 * a.n_e * st.n_cells +
                                    (sg * a.n_e + (k - 1)) * st.n_cells + c], 1u);
                atomicAdd(&a.g_hist[st.n_off / (2 * a.n_e) + (long long)tout * st.n_cells + c], 1ull);
                if (vmom) {
                    const float v = a.ent[st.ent_off + (layer * 2 + sg) * a.n_e + (k - 1)].v;
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.v_hist) + st.n_off / a.n_e +
                                  ((long long)tout * 2 + sg) * st.n_cells + c,
                              (unsigned long long)vel_q(__fmul_rn(v, mu_of(r1.x))));
                }
            }
        }
        if (ADJ) {
            // a new carrier: no parent (lineage depth 0, set when the replay
            // starts); its reward so far is its density weight if deposited
            long long rw = 0;
            if (deposit) {
                Stk tmp; tmp.n_cells = st.n_cells;
                rw = dep_w(a, s, tout, (int)sg, (int)k, cell_of(a, tmp, z));
            }
            if (id >= (unsigned long long)st.n_ids) {
                atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_STATE);
            } else {
                a.acc[cur][d] = ADJ == 1 ? rw : a.tot[st.id_off + (long long)id] - rw;
            }
        }
    }
    cta_sync();
    for (int s = tid; s < a.n_stacks; s += TPB) {
        if (s_q[s]) atomicAdd(&a.cnt[s].led[L_Q_INJECTED], s_q[s]);
        if (s_wsum[s]) atomicAdd(&a.cnt[s].w_injected, s_wsum[s]);
    }
    if (last_block(a, &s_flag)) {
        for (int s = tid; s < a.n_stacks; s += TPB) {
            const DevStack &st = a.stacks[s];
            const long long n = a.inj[st.inj_off + h];
            DevCounters &c = a.cnt[s];
            const long long kept = s_n[s];
            c.n_slots += (unsigned long long)kept;
            c.next_id += (unsigned long long)kept;
            c.live += (unsigned long long)kept;
            c.led[L_INJECTED] += (unsigned long long)kept;
            c.led[L_INJECT_DROPPED] += (unsigned long long)(n - kept);
            if (n > kept && (a.flags & PIC_F_STRICT_CAPACITY))
                atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_CAPACITY);
        }
        if (tid == 0) {
            a.ctl->done = 0u;
            bump_step(a);
        }
    }
}

template <int ADJ = 0>
__global__ void __launch_bounds__(TPB) k_inject(const Args a, int half, int deposit)
{
    phase_inject<ADJ>(a, half, deposit);
}

// ---------------------------------------------------------------------------
// k_compact: stable removal of dead slots (k = 0) into the other buffer
// ---------------------------------------------------------------------------
template <int ADJ = 0>
__device__ __forceinline__ void phase_compact(const Args &a)
{
    __shared__ long long s_tpref[PIC_MAX_STACKS + 1];
    __shared__ long long s_nsl[PIC_MAX_STACKS];
    __shared__ int s_w[TPB / 32];
    __shared__ long long s_prefix;
    __shared__ int s_flag;
    const unsigned int ep = *(volatile unsigned int *)&a.ctl->epoch;
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur, nxt = cur ^ 1;
    const int b = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
    const long long S = a.mp_stride;
    Plan p;
    make_plan(a, s_tpref, s_nsl, p);

    // Slots are taken in groups of TPB * CV (one tile): warp w takes the
    // 32 * CV slots [w * 32 CV, (w + 1) * 32 CV) of a group as CV rows of 32, lane l
    // the slot l of each row, so that loads and the stores of the live slots
    // are coalesced; a slot's rank is the live slots of the earlier warps
    // (one block scan of the warps' counts), of the earlier rows and of the
    // lower lanes of its row (ballots).  A group lies in one stack; lim = the
    // first slot not in it, or the stack's slot count; nothing at or past lim
    // is read.
    constexpr int CV = 4;
    constexpr long long GT = (long long)TPB * CV / TILE;      // tiles per group
    const int warp = tid >> 5, lane = tid & 31;
    const unsigned int lt = (1u << lane) - 1u;
    uint32_t pkv[CV], bal[CV];
    auto alive_rows = [&](const DevStack &st, long long g0, long long lim) -> int {
        int n = 0;
        const long long sl0 = g0 + warp * (32 * CV) + lane;
        const uint32_t *P = a.pk[cur] + (st.base + sl0) * S;
        const int left = lim - sl0 > 32 * CV ? 32 * CV : (int)(lim - sl0);   // rows i with i*32 < left
#pragma unroll
        for (int i = 0; i < CV; ++i) {
            pkv[i] = i * 32 < left ? P[i * 32 * S] : 0u;
            bal[i] = __ballot_sync(0xffffffffu, (pkv[i] & 0xFFu) != 0u);
            n += __popc(bal[i]);
        }
        return n;                     // the warp's live slots
    };
    // exclusive prefix of the warps' counts and the group's total
    auto warp_scan = [&](int n, int &excl) -> int {
        if (lane == 0) s_w[warp] = n;
        cta_sync();
        int pre = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < TPB / 32; ++w) {
            const int v = s_w[w];
            pre += w < warp ? v : 0;
            tot += v;
        }
        cta_sync();
        excl = pre;
        return tot;
    };
    // the groups of stack s inside this block's chunk: [ta, tb) tiles
    auto seg_tiles = [&](int s, long long &ta, long long &tb) {
        ta = p.t0 > s_tpref[s] ? p.t0 : s_tpref[s];
        tb = p.t1 < s_tpref[s + 1] ? p.t1 : s_tpref[s + 1];
    };

    if (p.t0 < p.t1) {
        const int s_first = stack_of(s_tpref, a.n_stacks, p.t0);
        const int s_last = stack_of(s_tpref, a.n_stacks, p.t1 - 1);
        const bool first_inside = p.t0 > s_tpref[s_first];
        // phase 1: count the first segment (if it needs the look-back) and the
        // last segment (its count is what later blocks need)
        long long c_first = 0, c_last = 0;
        for (int s = s_first; s <= s_last; ++s) {
            const bool need = (s == s_first && first_inside) || s == s_last;
            if (!need) continue;
            const DevStack &st = a.stacks[s];
            long long ta, tb;
            seg_tiles(s, ta, tb);
            for (long long t = ta; t < tb; t += GT) {
                const long long g0 = (t - s_tpref[s]) * TILE;
                const long long ge = ((t + GT < tb ? t + GT : tb) - s_tpref[s]) * TILE;
                int excl;
                const int tot = warp_scan(alive_rows(st, g0, ge < s_nsl[s] ? ge : s_nsl[s]), excl);
                if (s == s_first) c_first += tot;
                if (s == s_last) c_last += tot;
            }
        }
        long long pre_first = 0;
        if (tid < 32) {
            // the look-back takes the whole warp
            if (s_last == s_first && first_inside) {
                if (tid == 0) publish(&a.status[b], ep, FLAG_A, c_last);
                const long long pre = look_back(a, ep, p.T, s_tpref[s_first], b, G);
                if (tid == 0) {
                    s_prefix = pre;
                    publish(&a.status[b], ep, FLAG_P, pre + c_last);
                }
            } else {
                if (tid == 0) publish(&a.status[b], ep, FLAG_P, c_last);
                const long long pre = first_inside ? look_back(a, ep, p.T, s_tpref[s_first], b, G) : 0;
                if (tid == 0) s_prefix = pre;
            }
        }
        cta_sync();
        pre_first = s_prefix;
        (void)c_first;
        // phase 2: scatter live slots, stable, into the other buffer
        for (int s = s_first; s <= s_last; ++s) {
            const DevStack &st = a.stacks[s];
            long long ta, tb;
            seg_tiles(s, ta, tb);
            if (ta >= tb) continue;
            long long run = (s == s_first) ? pre_first : 0;
            for (long long t = ta; t < tb; t += GT) {
                const long long g0 = (t - s_tpref[s]) * TILE;
                const long long ge = ((t + GT < tb ? t + GT : tb) - s_tpref[s]) * TILE;
                const long long lim = ge < s_nsl[s] ? ge : s_nsl[s];
                const long long sl0 = g0 + warp * (32 * CV) + lane;  // this lane's first slot
                const int left = lim - sl0 > 32 * CV ? 32 * CV : (int)(lim - sl0);
                const float *Zc = a.z[cur] + st.base + sl0;
                const float *Mc = a.mu[cur] + (st.base + sl0) * S;
                const uint32_t *Ic = a.id[cur] + st.base + sl0;
                float zv[CV], muv[CV];
                uint32_t idv[CV];
#pragma unroll
                for (int i = 0; i < CV; ++i) {
                    const bool in = i * 32 < left;
                    zv[i] = in ? Zc[i * 32] : 0.f;
                    muv[i] = in ? Mc[i * 32 * S] : 0.f;
                    idv[i] = in ? Ic[i * 32] : 0u;
                }
                int excl;
                const int tot = warp_scan(alive_rows(st, g0, lim), excl);
                long long d = st.base + run + excl;
#pragma unroll
                for (int i = 0; i < CV; ++i) {
                    const long long src = st.base + sl0 + i * 32;
                    if ((bal[i] >> lane) & 1u) {
                        const long long o = d + __popc(bal[i] & lt);
                        a.z[nxt][o] = zv[i];
                        if (S == 2) {
                            *reinterpret_cast<uint2 *>(a.mu[nxt] + 2 * o) =
                                make_uint2(__float_as_uint(muv[i]), pkv[i]);
                        } else {
                            a.mu[nxt][o] = muv[i];
                            a.pk[nxt][o] = pkv[i];
                        }
                        a.id[nxt][o] = idv[i];
                        if (!ADJ && a.w[0]) a.w[nxt][o] = a.w[cur][src];
                        if (ADJ) a.acc[nxt][o] = a.acc[cur][src];
                    } else if (ADJ == 1 && i * 32 < left) {
                        // pass 1: a removed carrier's own reward is final
                        const unsigned long long id = (unsigned long long)idv[i] |
                                                      ((unsigned long long)(pkv[i] >> 21) << 32);
                        if (id < (unsigned long long)st.n_ids) a.tot[st.id_off + (long long)id] = a.acc[cur][src];
                        else atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_STATE);
                    }
                    d += __popc(bal[i]);
                }
                run += tot;
            }
            if (s_tpref[s + 1] <= p.t1 && tid == 0)
                a.cnt[s].alive_total = (unsigned long long)run;
        }
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

template <int ADJ = 0>
__global__ void __launch_bounds__(TPB) k_compact(const Args a)
{
    phase_compact<ADJ>(a);
}

// ---------------------------------------------------------------------------
// host-side launch-configuration helpers shared by the forward and adjoint
// translation units
// ---------------------------------------------------------------------------
// Occupancy of a kernel with `smem` bytes of dynamic shared memory; the
// largest dynamic shared memory the device offers is allowed, so that
// contexts with different moment grids never lower each other's cap.
template <class K>
static cudaError_t occupancy(K kernel, size_t smem, int *blocks, int threads = TPB)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int cap = optin - (int)fa.sharedSizeBytes;
    *blocks = 0;
    if ((int)smem > cap) return cudaSuccess;       // does not fit: zero blocks
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kernel, threads, smem);
}

// Ring depth and resident blocks of k_stream for one variant, both builds
// (with and without fused multiply-add) fitting: the most resident blocks per
// SM such that at least three tiles per SM are in flight, then the deepest
// ring (blocks_per_sm, ring_req: 0 = free).
template <bool DEPN, bool WAGG, int NW, int ADJ = 0, int GR = 1, bool EV = false>
static cudaError_t pick_stream_ring(size_t fixed, int blocks_per_sm, int ring_req, int *ring,
                                    int *blocks, size_t *smem)
{
    int best = -1;
    for (int r = 2; r <= MAX_RING; ++r) {
        if (ring_req > 0 && r != ring_req) continue;
        const size_t sm = fixed + (size_t)r * (ADJ == 2 ? 5 : 3) * TILE_BYTES;
        int o1 = 0, o2 = 0;
        constexpr int nthr = stream_threads_of<NW, GR, EV>();
        cudaError_t e = occupancy(k_stream<false, DEPN, WAGG, NW, ADJ, GR, EV>, sm, &o1, nthr);
        if (e == cudaSuccess) e = occupancy(k_stream<true, DEPN, WAGG, NW, ADJ, GR, EV>, sm, &o2, nthr);
        if (e != cudaSuccess) return e;
        int o = o1 < o2 ? o1 : o2;
        if (blocks_per_sm > 0 && o > blocks_per_sm) o = blocks_per_sm;
        if (o < 1) continue;
        const int enough = o * (r - 1) >= 3 ? 1 : 0;
        const int score = enough * 10000 + o * 100 + r;
        if (score > best) { best = score; *ring = r; *blocks = o; *smem = sm; }
    }
    return best < 0 ? cudaErrorInvalidConfiguration : cudaSuccess;
}
// Waves of resident blocks in the event pass's grid (its blocks take equal
// shares of the queue and never wait on one another).  One wave: a block's
// fixed work (queue prefix, tables, histograms) is paid once per SM slot,
// which matters when the queue is short (densities every step).
#ifndef PIC_EVENT_WAVES
#define PIC_EVENT_WAVES 1
#endif
template <bool DEPN, int ADJ = 0>
static cudaError_t event_cfg(size_t sm, int *grid, int sms)
{
    int o1 = 0, o2 = 0;
    cudaError_t e = occupancy(k_event<false, DEPN, ADJ>, sm, &o1);
    if (e == cudaSuccess) e = occupancy(k_event<true, DEPN, ADJ>, sm, &o2);
    if (e != cudaSuccess) return e;
    const int o = o1 < o2 ? o1 : o2;
    if (o < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * o * PIC_EVENT_WAVES;
    return cudaSuccess;
}

#ifndef PIC_PLACE_DEP_BLOCKS
#define PIC_PLACE_DEP_BLOCKS 2     // resident placement blocks per SM on density steps
#endif
template <bool DEPN, int ADJ = 0>
static cudaError_t place_cfg(size_t sm, int *grid, int sms)
{
    int o1 = 0, o2 = 0;
    cudaError_t e = occupancy(k_place<false, DEPN, ADJ>, sm, &o1);
    if (e == cudaSuccess) e = occupancy(k_place<true, DEPN, ADJ>, sm, &o2);
    if (e != cudaSuccess) return e;
    int o = o1 < o2 ? o1 : o2;
    if (o < 1) return cudaErrorInvalidConfiguration;
    // density steps: every block that places a secondary zeroes and flushes
    // the whole histogram, so fewer blocks than fit
    if (DEPN && o > PIC_PLACE_DEP_BLOCKS) o = PIC_PLACE_DEP_BLOCKS;
    *grid = sms * o;            // look-back: every block resident
    return cudaSuccess;
}

// Shared memory of the event and placement passes (ADJ: replay pass).
inline size_t event_smem(const Args &a, bool dep, int adj, int gf_max)
{
    const size_t tiles = (size_t)(2 * a.n_stacks + 1) * 8 + 16;
    return (size_t)a.tab_max * sizeof(TabEnt) + (size_t)a.T_max * 4 + 8 +
           (adj == 2 ? (size_t)(a.tab_max + a.T_max) * 8 : 0) +
           (adj ? 0 : (size_t)a.jbin_max * 4) + (dep && !adj ? (size_t)(a.nbin_max + a.gbin_max) * 4 : 0) +
           (dep && !adj ? (size_t)a.gbin_max * 16 : 0) + 16 + tiles + (size_t)(gf_max + 1) * 8;
}

inline size_t place_smem(const Args &a, bool dep, int adj)
{
    const size_t tiles = (size_t)(2 * a.n_stacks + 1) * 8 + 16;
    return (adj ? 0 : (size_t)a.jbin_max * 4) +
           (dep && !adj ? (size_t)(a.nbin_max + a.gbin_max) * 4 + (size_t)a.gbin_max * 16 : 0) + 16 +
           tiles;
}

}  // namespace pic
