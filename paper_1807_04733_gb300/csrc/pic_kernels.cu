// Forward step of the hot-electron PIC method: launch configuration and
// launchers of the kernels in pic_step.cuh, and the two small kernels that
// turn the densities and the births and removals of carriers into the
// fluxes through the cell faces.
#include <cuda_runtime.h>

#include <algorithm>

#include "pic_step.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// Fluxes from counts.  The spin flux of a moment window through face f (the
// net number of carriers of one spin that crossed it towards +z, reading of
// Eq. spincurrent) is, carrier by carrier, [cell at the end >= f] - [cell at
// the start >= f], the ends being the window's ends or the carrier's birth
// and removal.  Summed over carriers:
//
//   J_w[f] = sum_{c >= f} ( N_w[c] - N_{w-1}[c] - B_w[c] )
//
// with N_w the live carriers per cell at the end of window w (the densities
// summed over energy; N_{-1} = 0), and B_w the births minus removals per cell
// in window w (source, secondaries, removals, replaced records).  The result
// is the same integer as counting every crossing step by step.
// ---------------------------------------------------------------------------

// One block per (stack, window, spin) row: J of window w from the densities
// of windows w and w - 1 (or `now` for an unfinished window w == w_now).
__global__ void __launch_bounds__(TPB) k_flux(const Args a, int w0, int w1, int w_now,
                                              const int32_t *now, int ncm)
{
    __shared__ int s_w[TPB / 32];
    const int nw = w1 - w0;
    const int row = blockIdx.x;
    const int s = row / (2 * nw), rem = row % (2 * nw), w = w0 + rem / 2, sg = rem % 2;
    const DevStack &st = a.stacks[s];
    const int nc = st.n_cells, nf = nc + 1, ne = a.n_e;
    const long long nbins = 2LL * ne * nc;
    const uint32_t *Ne = a.n_hist + st.n_off + (long long)w * nbins + (long long)sg * ne * nc;
    const uint32_t *Ns = w > 0 ? Ne - nbins : nullptr;
    const int32_t *B = a.bd_hist + st.J_off + ((long long)w * 2 + sg) * nf;
    const int32_t *Nn = (w == w_now && now) ? now + ((long long)s * 2 + sg) * (ncm + 1) : nullptr;
    int32_t *J = a.J_hist + st.J_off + ((long long)w * 2 + sg) * nf;
    // suffix sums over cells, in chunks of TPB cells from the top
    int carry = 0;
    for (int c1 = nc; c1 > 0; c1 -= TPB) {
        const int c = c1 - 1 - threadIdx.x;          // descending cell of this thread
        int d = 0;
        if (c >= 0) {
            long long ne_c = 0, ns_c = 0;
            if (Nn) {
                ne_c = Nn[c];
            } else {
                for (int k = 0; k < ne; ++k) ne_c += Ne[(long long)k * nc + c];
            }
            if (Ns)
                for (int k = 0; k < ne; ++k) ns_c += Ns[(long long)k * nc + c];
            d = (int)(ne_c - ns_c) - B[c];
        }
        int excl;
        const int tot = block_scan(d, excl, s_w);
        if (c >= 0) J[c] = carry + excl + d;
        carry += tot;
    }
    if (threadIdx.x == 0) J[nc] = 0;
}

// Live carriers of stacks [s0, s1) per (spin, cell): mode 0 adds `sign` per
// carrier to the births-minus-removals histogram of window `win`; mode 1
// counts into out[stack][2][ncm + 1] (zeroed by the caller).
__global__ void __launch_bounds__(TPB) k_state_hist(const Args a, int s0, int s1, int mode,
                                                    int win, int sign, int32_t *out, int ncm)
{
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    for (int s = s0; s < s1; ++s) {
        const DevStack &st = a.stacks[s];
        const long long n = (long long)a.cnt[s].n_slots;
        Stk tmp;
        tmp.n_cells = st.n_cells;
        int32_t *h = mode == 0 ? a.bd_hist + st.J_off + (long long)win * 2 * (st.n_cells + 1)
                               : out + (long long)s * 2 * (ncm + 1);
        const int nf = mode == 0 ? st.n_cells + 1 : ncm + 1;
        for (long long i = (long long)blockIdx.x * TPB + threadIdx.x; i < n;
             i += (long long)gridDim.x * TPB) {
            const long long g = st.base + i;
            const uint32_t pk = a.pk[cur][g * a.mp_stride];
            if ((pk & 0xFFu) == 0u) continue;
            const int sg = (int)((pk >> 8) & 1u);
            atomicAdd(&h[sg * nf + cell_of(a, tmp, a.z[cur][g])], sign);
        }
    }
}

// The weighted fluxes (PIC_F_WEIGHTS): the same sums over the weighted
// densities (2^-20 units) and the weighted births minus removals.
__global__ void __launch_bounds__(TPB) k_flux_w(const Args a, int w0, int w1, int w_now,
                                                const long long *now, int ncm)
{
    __shared__ long long s_w[TPB / 32];
    __shared__ long long s_tot;
    const int nw = w1 - w0;
    const int row = blockIdx.x;
    const int s = row / (2 * nw), rem = row % (2 * nw), w = w0 + rem / 2, sg = rem % 2;
    const DevStack &st = a.stacks[s];
    const int nc = st.n_cells, nf = nc + 1, ne = a.n_e;
    const long long nbins = 2LL * ne * nc;
    const unsigned long long *Ne = a.nhw + st.n_off + (long long)w * nbins + (long long)sg * ne * nc;
    const unsigned long long *Ns = w > 0 ? Ne - nbins : nullptr;
    const long long *B = a.bdw + st.J_off + ((long long)w * 2 + sg) * nf;
    const long long *Nn = (w == w_now && now) ? now + ((long long)s * 2 + sg) * (ncm + 1) : nullptr;
    long long *J = a.Jw + st.J_off + ((long long)w * 2 + sg) * nf;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long carry = 0;
    for (int c1 = nc; c1 > 0; c1 -= TPB) {
        const int c = c1 - 1 - threadIdx.x;          // descending cell of this thread
        long long d = 0;
        if (c >= 0) {
            long long ne_c = 0, ns_c = 0;
            if (Nn) {
                ne_c = Nn[c];
            } else {
                for (int k = 0; k < ne; ++k) ne_c += (long long)Ne[(long long)k * nc + c];
            }
            if (Ns)
                for (int k = 0; k < ne; ++k) ns_c += (long long)Ns[(long long)k * nc + c];
            d = ne_c - ns_c - B[c];
        }
        // block-wide inclusive scan of d in thread order (descending cells)
        long long x = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        long long before = 0;
        for (int q = 0; q < wid; ++q) before += s_w[q];
        if (threadIdx.x == TPB - 1) s_tot = before + x;
        if (c >= 0) J[c] = carry + before + x;
        __syncthreads();
        carry += s_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) J[nc] = 0;
}

// Weighted live carriers of stacks [s0, s1) per (spin, cell), as
// k_state_hist: mode 0 adds sign * w to the weighted births-minus-removals
// histogram of window `win`; mode 1 sums into out[stack][2][ncm + 1].
__global__ void __launch_bounds__(TPB) k_state_hist_w(const Args a, int s0, int s1, int mode,
                                                      int win, int sign, long long *out, int ncm)
{
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    for (int s = s0; s < s1; ++s) {
        const DevStack &st = a.stacks[s];
        const long long n = (long long)a.cnt[s].n_slots;
        Stk tmp;
        tmp.n_cells = st.n_cells;
        long long *h = mode == 0 ? a.bdw + st.J_off + (long long)win * 2 * (st.n_cells + 1)
                                 : out + (long long)s * 2 * (ncm + 1);
        const int nf = mode == 0 ? st.n_cells + 1 : ncm + 1;
        for (long long i = (long long)blockIdx.x * TPB + threadIdx.x; i < n;
             i += (long long)gridDim.x * TPB) {
            const long long g = st.base + i;
            const uint32_t pk = a.pk[cur][g * a.mp_stride];
            if ((pk & 0xFFu) == 0u) continue;
            const int sg = (int)((pk >> 8) & 1u);
            const long long v = (long long)a.w[cur][g] * sign;
            atomicAdd(reinterpret_cast<unsigned long long *>(&h[sg * nf + cell_of(a, tmp, a.z[cur][g])]),
                      (unsigned long long)v);
        }
    }
}

// Weighted densities at the end of density step `step`: every live carrier
// adds its weight to its (spin, bin, cell) entry.  One block owns a
// contiguous chunk of tiles; with SM the stack's histogram is privatised in
// shared memory and flushed once per stack segment, otherwise added in
// global memory.
template <bool SM>
__device__ __forceinline__ void phase_wdep(const Args &a, uint32_t step)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_h = reinterpret_cast<unsigned long long *>(smem);
    __shared__ long long s_tpref[PIC_MAX_STACKS + 1];
    __shared__ long long s_nsl[PIC_MAX_STACKS];
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    const int tid = threadIdx.x;
    const int tout = (int)((step + 1) / (uint32_t)a.moment_every) - 1;
    Plan p;
    make_plan(a, s_tpref, s_nsl, p);
    const uint2 *MP = reinterpret_cast<const uint2 *>(a.mu[cur]);   // (mu, packed) pairs
    auto hist = [&](int s) {
        const DevStack &st = a.stacks[s];
        return a.nhw + st.n_off + (long long)tout * 2 * a.n_e * st.n_cells;
    };
    auto flush = [&](int s) {
        cta_sync();
        const int nb = 2 * a.n_e * a.stacks[s].n_cells;
        unsigned long long *gh = hist(s);
        for (int i = tid; i < nb; i += TPB)
            if (s_h[i]) atomicAdd(&gh[i], s_h[i]);
        cta_sync();
    };
    int seg = -1;
    unsigned long long *gh = nullptr;
    for (long long t = p.t0; t < p.t1; ++t) {
        const int s = stack_of(s_tpref, a.n_stacks, t);
        if (s != seg) {
            if (SM) {
                if (seg >= 0) flush(seg);
                for (int i = tid; i < 2 * a.n_e * a.stacks[s].n_cells; i += TPB) s_h[i] = 0ull;
                cta_sync();
            }
            gh = hist(s);
            seg = s;
        }
        const DevStack &st = a.stacks[s];
        Stk tmp;
        tmp.n_cells = st.n_cells;
        const long long slot0 = (t - s_tpref[s]) * TILE + (long long)tid * VEC;
        const long long nsl = s_nsl[s];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            const long long slot = slot0 + j;
            if (slot >= nsl) break;
            const long long g = st.base + slot;
            const uint32_t pk = MP[g].y;
            const int k = (int)(pk & 0xFFu);
            if (k == 0) continue;
            const int sg = (int)((pk >> 8) & 1u);
            const int b = (sg * a.n_e + (k - 1)) * st.n_cells + cell_of(a, tmp, a.z[cur][g]);
            const unsigned long long w = a.w[cur][g];
            if (SM) add_u64_split(&s_h[b], w);
            else atomicAdd(&gh[b], w);
        }
    }
    if (SM && seg >= 0) flush(seg);
}

// Launched after the step's last kernel: in a graph replay that kernel has
// already advanced the device step counter.
template <bool SM>
__global__ void __launch_bounds__(TPB) k_wdep(const Args a)
{
    phase_wdep<SM>(a, a.step_dev ? __ldcg(a.step_dev) - 1u : a.step);
}

cudaError_t launch_flux_w(const Args &a, int w0, int w1, int w_now, const long long *now, int ncm,
                          cudaStream_t st)
{
    if (w1 <= w0) return cudaSuccess;
    k_flux_w<<<a.n_stacks * 2 * (w1 - w0), TPB, 0, st>>>(a, w0, w1, w_now, now, ncm);
    return cudaGetLastError();
}

cudaError_t launch_state_hist_w(const Args &a, int s0, int s1, int mode, int win, int sign,
                                long long *scratch, int ncm, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    k_state_hist_w<<<sms * 4, TPB, 0, st>>>(a, s0, s1, mode, win, sign, scratch, ncm);
    return cudaGetLastError();
}

cudaError_t launch_wdep(const Args &a, const LaunchCfg &c, cudaStream_t st)
{
    // privatised in shared memory when the widest stack's histogram fits
    const size_t sm = (size_t)a.nbin_max * sizeof(unsigned long long);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t static_sm = (size_t)(2 * PIC_MAX_STACKS + 1) * 8;
    if (sm + static_sm <= (size_t)optin) {
        e = cudaFuncSetAttribute(k_wdep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_wdep<true><<<c.grid_compact, TPB, sm, st>>>(a);
    } else {
        k_wdep<false><<<c.grid_compact, TPB, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_flux(const Args &a, int w0, int w1, int w_now, const int32_t *now, int ncm,
                        cudaStream_t st)
{
    if (w1 <= w0) return cudaSuccess;
    k_flux<<<a.n_stacks * 2 * (w1 - w0), TPB, 0, st>>>(a, w0, w1, w_now, now, ncm);
    return cudaGetLastError();
}

cudaError_t launch_state_hist(const Args &a, int s0, int s1, int mode, int win, int sign,
                              int32_t *scratch, int ncm, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    k_state_hist<<<sms * 4, TPB, 0, st>>>(a, s0, s1, mode, win, sign, scratch, ncm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
// plain steps of a single stack in the fused form (0: separate event pass)
#ifndef PIC_FUSED_STEP
#define PIC_FUSED_STEP 1
#endif

namespace {

// k_stream's configuration for one deposit variant and consumer-warp count
template <bool DEPN, bool WAGG>
cudaError_t stream_cfg(size_t fixed, int blocks_per_sm, int ring_req, int nw, int *ring,
                       int *blocks, size_t *smem)
{
    // 16: two groups of eight warps (the density-step pass only)
    if (nw == 16) {
        if constexpr (DEPN)
            return pick_stream_ring<DEPN, WAGG, 8, 0, 2>(fixed, blocks_per_sm, ring_req, ring, blocks, smem);
        return cudaErrorInvalidValue;
    }
    return nw == 4 ? pick_stream_ring<DEPN, WAGG, 4>(fixed, blocks_per_sm, ring_req, ring, blocks, smem)
                   : pick_stream_ring<DEPN, WAGG, 8>(fixed, blocks_per_sm, ring_req, ring, blocks, smem);
}

}  // namespace

cudaError_t configure(const Args &a, int blocks_per_sm, int ring_req, int hist_mode, int nw,
                      LaunchCfg *cfg)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if (nw != 0 && nw != 4 && nw != 8) return cudaErrorInvalidValue;
    const size_t tiles = (size_t)(2 * a.n_stacks + 1) * 8 + 16;      // tile prefix, counts
    const size_t fixed = (size_t)a.ftab_max * sizeof(FastEnt) + tiles;
    const size_t fixed_dep = fixed + (size_t)(a.nbin_max + a.gbin_max) * 4 + (size_t)a.gbin_max * 16 + 8;
    // consumer warps: eight unless four were asked for (the density-step
    // variant, which holds large histograms, always takes eight)
    const int nw_plain = nw == 4 ? 4 : 8;
    int o_plain = 0, o_dep = 0;
    if ((e = stream_cfg<false, false>(fixed, blocks_per_sm, ring_req, nw_plain, &cfg->ring_fast,
                                      &o_plain, &cfg->smem_fast)) != cudaSuccess)
        return e;
    if (hist_mode == 1)
        e = stream_cfg<true, true>(fixed_dep, blocks_per_sm, 0, 8, &cfg->ring_fast_dep, &o_dep,
                                   &cfg->smem_fast_dep);
    else
        e = stream_cfg<true, false>(fixed_dep, blocks_per_sm, 0, 8, &cfg->ring_fast_dep, &o_dep,
                                    &cfg->smem_fast_dep);
    if (e != cudaSuccess) return e;
    int nw_dep = 8;
    if (o_dep == 1) {
        // room for one block per SM only (large histograms): a second group
        // of eight consumer warps in the same block shares them
        int ring2 = 0, o2 = 0;
        size_t sm2 = 0;
        e = hist_mode == 1
                ? stream_cfg<true, true>(fixed_dep, blocks_per_sm, 0, 16, &ring2, &o2, &sm2)
                : stream_cfg<true, false>(fixed_dep, blocks_per_sm, 0, 16, &ring2, &o2, &sm2);
        if (e == cudaSuccess && o2 >= 1) {
            nw_dep = 16;
            cfg->ring_fast_dep = ring2;
            cfg->smem_fast_dep = sm2;
        }
        e = cudaSuccess;
        cudaGetLastError();
    }
    cfg->nw_fast = nw_plain;
    cfg->nw_fast_dep = nw_dep;
    // the fused form, for the plain steps of a single stack with eight
    // consumer warps: the general step's tables, the removals histogram and
    // the event ring besides the streaming pass's own shared memory
    cfg->grid_fused = 0;
    cfg->ring_fused = 0;
    cfg->smem_fused = 0;
#if PIC_FUSED_STEP
    if (a.n_stacks == 1 && nw_plain == 8) {
        const size_t fixed_ev = fixed + 16 + (size_t)a.tab_max * sizeof(TabEnt) + (size_t)a.T_max * 4 +
                                (size_t)a.jbin_max * 4 + 16 + (size_t)EV_CAP * (16 + 4 + 4);
        int rf = 0, of = 0;
        size_t sf = 0;
        e = pick_stream_ring<false, false, 8, 0, 1, true>(fixed_ev, blocks_per_sm, ring_req, &rf, &of, &sf);
        if (e == cudaSuccess && of >= 1) {
            cfg->grid_fused = sms * of;
            cfg->ring_fused = rf;
            cfg->smem_fused = sf;
        }
        e = cudaSuccess;
        cudaGetLastError();
    }
#endif
    cfg->grid_fast = sms * o_plain;
    cfg->grid_fast_dep = sms * o_dep;
    const int gf_max = cfg->grid_fast > cfg->grid_fast_dep ? cfg->grid_fast : cfg->grid_fast_dep;
    cfg->smem_slow = event_smem(a, false, 0, gf_max);
    cfg->smem_slow_dep = event_smem(a, true, 0, gf_max);
    if ((e = event_cfg<false>(cfg->smem_slow, &cfg->grid_slow, sms)) != cudaSuccess) return e;
    if ((e = event_cfg<true>(cfg->smem_slow_dep, &cfg->grid_slow_dep, sms)) != cudaSuccess) return e;
    cfg->smem_place = place_smem(a, false, 0);
    cfg->smem_place_dep = place_smem(a, true, 0);
    if ((e = place_cfg<false>(cfg->smem_place, &cfg->grid_place, sms)) != cudaSuccess) return e;
    if ((e = place_cfg<true>(cfg->smem_place_dep, &cfg->grid_place_dep, sms)) != cudaSuccess) return e;
    int oc = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_compact<0>, TPB, 0)) != cudaSuccess)
        return e;
    cfg->grid_compact = sms * (oc > 0 ? oc : 1);
    cfg->grid_inject = sms * 4;
    return cudaSuccess;
}

namespace {

template <bool DET, bool DEPN, bool WAGG>
void stream_launch(const Args &a, int g, int nw, size_t sm, cudaStream_t s)
{
    if constexpr (DEPN) {
        if (nw == 16) {
            k_stream<DET, DEPN, WAGG, 8, 0, 2><<<g, stream_threads<16>(), sm, s>>>(a);
            return;
        }
    }
    if (nw == 4) k_stream<DET, DEPN, WAGG, 4><<<g, stream_threads<4>(), sm, s>>>(a);
    else k_stream<DET, DEPN, WAGG, 8><<<g, stream_threads<8>(), sm, s>>>(a);
}

}  // namespace

cudaError_t launch_fast(const Args &a0, const LaunchCfg &c, bool det, bool dep, int hist_mode,
                        cudaStream_t s)
{
    Args a = a0;
    a.ring = dep ? c.ring_fast_dep : c.ring_fast;
    const int g = dep ? c.grid_fast_dep : c.grid_fast;
    const int nw = dep ? c.nw_fast_dep : c.nw_fast;
    const size_t sm = dep ? c.smem_fast_dep : c.smem_fast;
    const bool w = hist_mode == 1;
    if (det) {
        if (dep) {
            if (w) stream_launch<true, true, true>(a, g, nw, sm, s);
            else stream_launch<true, true, false>(a, g, nw, sm, s);
        } else {
            stream_launch<true, false, false>(a, g, nw, sm, s);
        }
    } else {
        if (dep) {
            if (w) stream_launch<false, true, true>(a, g, nw, sm, s);
            else stream_launch<false, true, false>(a, g, nw, sm, s);
        } else {
            stream_launch<false, false, false>(a, g, nw, sm, s);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_slow(const Args &a0, const LaunchCfg &c, bool det, bool dep, cudaStream_t s)
{
    Args a = a0;
    a.grid_fast = dep ? c.grid_fast_dep : c.grid_fast;
    const int g = dep ? c.grid_slow_dep : c.grid_slow;
    const size_t sm = dep ? c.smem_slow_dep : c.smem_slow;
    const int gp = dep ? c.grid_place_dep : c.grid_place;
    const size_t smp = dep ? c.smem_place_dep : c.smem_place;
    Args ae = a;
    ae.bump_step = 0;                    // the placement pass ends the step
    if (det) {
        if (dep) { k_event<true, true><<<g, TPB, sm, s>>>(ae); k_place<true, true><<<gp, TPB, smp, s>>>(a); }
        else { k_event<true, false><<<g, TPB, sm, s>>>(ae); k_place<true, false><<<gp, TPB, smp, s>>>(a); }
    } else {
        if (dep) { k_event<false, true><<<g, TPB, sm, s>>>(ae); k_place<false, true><<<gp, TPB, smp, s>>>(a); }
        else { k_event<false, false><<<g, TPB, sm, s>>>(ae); k_place<false, false><<<gp, TPB, smp, s>>>(a); }
    }
    return cudaGetLastError();
}

cudaError_t launch_fused(const Args &a0, const LaunchCfg &c, bool det, cudaStream_t s)
{
    Args a = a0;
    a.ring = c.ring_fused;
    a.bump_step = 0;                     // the placement pass ends the step
    constexpr int nthr = stream_threads_of<8, 1, true>();
    if (det) k_stream<true, false, false, 8, 0, 1, true><<<c.grid_fused, nthr, c.smem_fused, s>>>(a);
    else k_stream<false, false, false, 8, 0, 1, true><<<c.grid_fused, nthr, c.smem_fused, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_place_fused(const Args &b0, const LaunchCfg &c, bool det, cudaStream_t s)
{
    Args b = b0;
    b.grid_fast = c.grid_fused;          // the streaming blocks whose secondaries it places
    if (det) k_place<true, false><<<c.grid_place, TPB, c.smem_place, s>>>(b);
    else k_place<false, false><<<c.grid_place, TPB, c.smem_place, s>>>(b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The persistent kernel: whole steps of every stack in one cooperative launch
// (batched stacks, use_graph = 2).  Blocks of 288 threads run the streaming
// pass with all nine warps (eight consumers and the producer) and every other
// pass on warps 0-7 (the passes' 256-thread barriers become a named barrier
// of those warps); a grid barrier separates the passes.  The step is read
// from and advanced in device memory, so the launch replays from a graph.
// ---------------------------------------------------------------------------

// Grid barrier: every block resident (a cooperative launch).  Sense by
// generation; the wait is bounded in polls, after which the status says
// PIC_ERR_TIMEOUT and every later barrier of the launch passes at once.
__device__ __forceinline__ void grid_sync(const Args &a)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &a.ctl->bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&a.ctl->bar_count, 1u) == gridDim.x - 1) {
            a.ctl->bar_count = 0u;           // the next arrivals follow the new generation
            __threadfence();
            atomicAdd(&a.ctl->bar_gen, 1u);
        } else {
            unsigned int it = 0;
            while (*gen == g) {
                if (*(volatile unsigned int *)&a.ctl->status != 0u) break;
                if (++it > a.spin_limit) {
                    atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_TIMEOUT);
                    a.ctl->timeout_where = 5u;
                    break;
                }
                if (it > 64) __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// a source half step with carriers in some stack (uniform: device data)
__device__ __forceinline__ bool any_source(const Args &a, long long h)
{
    for (int s = 0; s < a.n_stacks; ++s)
        if (a.inj[a.stacks[s].inj_off + h] > 0) return true;
    return false;
}

template <bool DET, bool WSM>
__global__ void __launch_bounds__(stream_threads<8>(), 2) k_period(const Args a, int n_steps)
{
    __shared__ int s_stop;
    const bool low = threadIdx.x < TPB;      // the warps of the 256-thread passes
    for (int i = 0; i < n_steps; ++i) {
        // stop after a failure (a decision of the whole block)
        if (threadIdx.x == 0) s_stop = *(volatile unsigned int *)&a.ctl->status != 0u;
        __syncthreads();
        if (s_stop) break;
        const uint32_t s = __ldcg(a.step_dev);
        const bool dep = ((s + 1) % (uint32_t)a.moment_every) == 0;
        if (any_source(a, 2 * (long long)s)) {
            if (low) phase_inject<0>(a, 0, 0);
            grid_sync(a);
        }
        if (dep) phase_stream<DET, true, false, 8>(a);
        else phase_stream<DET, false, false, 8>(a);
        grid_sync(a);
        if (low) {
            if (dep) phase_event<DET, true>(a);
            else phase_event<DET, false>(a);
        }
        grid_sync(a);
        if (low) {
            if (dep) phase_place<DET, true>(a);
            else phase_place<DET, false>(a);
        }
        grid_sync(a);
        if (any_source(a, 2 * (long long)s + 1)) {
            if (low) phase_inject<0>(a, 1, dep ? 1 : 0);
            grid_sync(a);
        }
        if (dep && a.w[0]) {
            if (low) phase_wdep<WSM>(a, s);
            grid_sync(a);
        }
        if (((s + 1) % (uint32_t)a.compact_every) == 0) {
            if (low) phase_compact<0>(a);
            grid_sync(a);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *const_cast<unsigned int *>(a.step_dev) = s + 1u;
            __threadfence();
        }
        grid_sync(a);
    }
}

cudaError_t configure_persistent(const Args &a, bool det, PersistCfg *pc)
{
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // dynamic shared memory: the largest pass
    const size_t tiles = (size_t)(2 * a.n_stacks + 1) * 8 + 16;
    const size_t fixed_dep = (size_t)a.ftab_max * sizeof(FastEnt) + tiles +
                             (size_t)(a.nbin_max + a.gbin_max) * 4 + (size_t)a.gbin_max * 16 + 8;
    const int gmax = 16 * sms;
    const size_t other = std::max({event_smem(a, true, 0, gmax), place_smem(a, true, 0)});
    const size_t wsm = (size_t)a.nbin_max * 8;
    const bool wsm_ok = a.w[0] && wsm + (size_t)(2 * PIC_MAX_STACKS + 1) * 8 + 4096 <= (size_t)optin;
    PersistCfg best;
    for (int ring = 8; ring >= 2; --ring) {
        size_t sm = std::max(fixed_dep + (size_t)ring * 3 * TILE_BYTES, other);
        if (wsm_ok) sm = std::max(sm, wsm);
        int o = 0;
        auto k = det ? (wsm_ok ? k_period<true, true> : k_period<true, false>)
                     : (wsm_ok ? k_period<false, true> : k_period<false, false>);
        e = occupancy(k, sm, &o, stream_threads<8>());
        if (e != cudaSuccess) return e;
        if (o < 1) continue;
        // the most resident blocks, then the deepest ring
        if (!best.ok || o > best.grid / sms) {
            best.grid = sms * o;
            best.ring = ring;
            best.smem = sm;
            best.wsm = wsm_ok;
            best.ok = true;
        }
    }
    *pc = best;
    return best.ok ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t launch_persistent(const Args &a0, const PersistCfg &pc, bool det, int n_steps,
                              cudaStream_t s)
{
    Args a = a0;
    a.ring = pc.ring;
    a.grid_fast = pc.grid;
    a.bump_step = 0;
    const bool wsm_ok = pc.wsm;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)pc.grid);
    cfg.blockDim = dim3((unsigned)stream_threads<8>());
    cfg.dynamicSmemBytes = pc.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (det) {
        if (wsm_ok) return cudaLaunchKernelEx(&cfg, k_period<true, true>, a, n_steps);
        return cudaLaunchKernelEx(&cfg, k_period<true, false>, a, n_steps);
    }
    if (wsm_ok) return cudaLaunchKernelEx(&cfg, k_period<false, true>, a, n_steps);
    return cudaLaunchKernelEx(&cfg, k_period<false, false>, a, n_steps);
}

cudaError_t launch_inject(const Args &a, const LaunchCfg &c, int half, bool deposit,
                          cudaStream_t s)
{
    k_inject<0><<<c.grid_inject, TPB, 0, s>>>(a, half, deposit ? 1 : 0);
    return cudaGetLastError();
}

__global__ void k_set_step(DevCtl *ctl, unsigned int step) { ctl->step = step; }

cudaError_t launch_set_step(DevCtl *ctl, unsigned int step, cudaStream_t s)
{
    k_set_step<<<1, 1, 0, s>>>(ctl, step);
    return cudaGetLastError();
}

cudaError_t launch_compact(const Args &a, const LaunchCfg &c, cudaStream_t s)
{
    k_compact<0><<<c.grid_compact, TPB, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
