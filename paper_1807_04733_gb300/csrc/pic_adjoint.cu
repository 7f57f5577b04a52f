// Adjoint replay of the PIC step: launch configuration and launchers of the
// replay variants of the step kernels (pic_step.cuh, ADJ = 1, 2) and the
// small kernels of the score-function gradient (flux potential, end-of-pass
// flush, lineage totals).
//
// The gradient of E[O], O = sum gn * n + sum gJ * J, with respect to the
// lifetime and transmittance tables is the expectation of the sum, over the
// random decisions of the run (scattering test, channel, interface draws),
// of d log P(outcome)/d theta times the reward that can follow the decision.
// The forward run stores nothing: both passes recompute the trajectories from
// the initial state and the Philox counters.
//   pass 1   every carrier's own reward (its density weights and the signed
//            weights of the faces it crosses), into an id-indexed array when it
//            is removed or the pass ends; each secondary's parent and depth
//   lineage  totals: every carrier's total added to its parent's, deepest
//            generation first
//   pass 2   reward-to-go R per slot (total minus what the carrier and its
//            secondaries have earned); every decision of a step adds its
//            score times R to per-block gradient bins
// Rewards are fixed-point integers: the weights are quantised to int32 in
// units of 2^-F (F chosen on the host from the largest weight and a bound on
// any lineage's reward), so that every reward sum, lineage total and
// reward-to-go is exact and independent of the summation order, and the
// streaming pass runs integer adds instead of double-precision arithmetic.
#include <cuda_runtime.h>

#include "pic_step.cuh"

namespace pic {

namespace {

// flux potential of one (stack, window, spin) row, in fixed point:
// gpot[c] = sum_{f=1..c} rint(gJ[f] 2^F)
__global__ void k_flux_potential(const Args a, const float *gJ, long long *gpot, int rows,
                                 double scale)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int s = r / (2 * a.n_out);
    const int nc = a.stacks[s].n_cells;
    const float *g = gJ + (long long)r * (a.ncm + 1);
    long long *p = gpot + (long long)r * a.ncm;
    long long acc = 0;
    p[0] = 0;
    for (int c = 1; c < nc; ++c) {
        acc += (long long)rint((double)g[c] * scale);
        p[c] = acc;
    }
}

__global__ void k_absmax(const float *x, long long n, unsigned int *out)
{
    unsigned int m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned int b = __float_as_uint(x[i]) & 0x7FFFFFFFu;
        m = b > m ? b : m;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned int y = __shfl_down_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void k_quantize(const float *x, long long n, int32_t *q, double scale)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        q[i] = (int32_t)rint((double)x[i] * scale);
}

// start of a pass: the loaded carriers' own reward so far (0, pass 1) or
// reward-to-go (their lineage total, pass 2)
__global__ void k_init_acc(const Args a, int pass)
{
    for (int s = 0; s < a.n_stacks; ++s) {
        const DevStack &st = a.stacks[s];
        const long long n = (long long)a.cnt[s].n_slots;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const long long slot = st.base + i;
            const unsigned long long id = (unsigned long long)a.id[0][slot] |
                                          ((unsigned long long)(a.pk[0][slot * a.mp_stride] >> 21) << 32);
            long long v = 0;
            if (pass == 2) {
                if (id < (unsigned long long)st.n_ids) v = a.tot[st.id_off + (long long)id];
                else atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_STATE);
            }
            a.acc[0][slot] = v;
        }
    }
}

// end of pass 1: the own reward of every carrier still in a slot
__global__ void k_flush_own(const Args a)
{
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    for (int s = 0; s < a.n_stacks; ++s) {
        const DevStack &st = a.stacks[s];
        const long long n = (long long)a.cnt[s].n_slots;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const long long slot = st.base + i;
            const unsigned long long id = (unsigned long long)a.id[cur][slot] |
                                          ((unsigned long long)(a.pk[cur][slot * a.mp_stride] >> 21) << 32);
            if (id < (unsigned long long)st.n_ids) a.tot[st.id_off + (long long)id] = a.acc[cur][slot];
            else atomicCAS(&a.ctl->status, 0u, (unsigned int)PIC_ERR_STATE);
        }
    }
}

// lineage: the totals of the carriers at depth g are complete (all their
// descendants are deeper); add them to their parents'
__global__ void k_lineage(const Args a, long long n_ids, int g)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ids;
         i += (long long)gridDim.x * blockDim.x)
        if (a.gen[i] == (uint8_t)g)
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.tot[a.parent[i]]),
                      (unsigned long long)a.tot[i]);
}

template <int ADJ>
cudaError_t configure_pass(const Args &a, LaunchCfg *cfg)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const size_t tiles = (size_t)(2 * a.n_stacks + 1) * 8 + 16;
    // tables, pass 2's sums of R, the flux potential slice and (with the
    // density deposit) the density-weight slice
    const size_t fixed = (size_t)a.ftab_max * sizeof(FastEnt) +
                         (ADJ == 2 ? (size_t)a.tab_max * 8 : 0) + (size_t)a.jbin_max * 8 + 8 +
                         tiles;
    const size_t fixed_dep = fixed + (size_t)a.nbin_max * 4;
    int o_plain = 0, o_dep = 0;
    if ((e = pick_stream_ring<false, false, 8, ADJ>(fixed, 0, 0, &cfg->ring_fast, &o_plain,
                                                    &cfg->smem_fast)) != cudaSuccess)
        return e;
    if ((e = pick_stream_ring<true, false, 8, ADJ>(fixed_dep, 0, 0, &cfg->ring_fast_dep, &o_dep,
                                                   &cfg->smem_fast_dep)) != cudaSuccess)
        return e;
    cfg->nw_fast = cfg->nw_fast_dep = 8;
    cfg->grid_fast = sms * o_plain;
    cfg->grid_fast_dep = sms * o_dep;
    const int gf_max = cfg->grid_fast > cfg->grid_fast_dep ? cfg->grid_fast : cfg->grid_fast_dep;
    cfg->smem_slow = event_smem(a, false, ADJ, gf_max);
    cfg->smem_slow_dep = event_smem(a, true, ADJ, gf_max);
    if ((e = event_cfg<false, ADJ>(cfg->smem_slow, &cfg->grid_slow, sms)) != cudaSuccess) return e;
    if ((e = event_cfg<true, ADJ>(cfg->smem_slow_dep, &cfg->grid_slow_dep, sms)) != cudaSuccess) return e;
    cfg->smem_place = place_smem(a, false, ADJ);
    cfg->smem_place_dep = place_smem(a, true, ADJ);
    if ((e = place_cfg<false, ADJ>(cfg->smem_place, &cfg->grid_place, sms)) != cudaSuccess) return e;
    if ((e = place_cfg<true, ADJ>(cfg->smem_place_dep, &cfg->grid_place_dep, sms)) != cudaSuccess) return e;
    int oc = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_compact<ADJ>, TPB, 0)) != cudaSuccess)
        return e;
    cfg->grid_compact = sms * (oc > 0 ? oc : 1);
    cfg->grid_inject = sms * 4;
    return cudaSuccess;
}

template <int ADJ>
void fast_pass(const Args &a, const LaunchCfg &c, bool det, bool dep, cudaStream_t s)
{
    const int g = dep ? c.grid_fast_dep : c.grid_fast;
    const size_t sm = dep ? c.smem_fast_dep : c.smem_fast;
    constexpr int T = stream_threads<8>();
    if (det) {
        if (dep) k_stream<true, true, false, 8, ADJ><<<g, T, sm, s>>>(a);
        else k_stream<true, false, false, 8, ADJ><<<g, T, sm, s>>>(a);
    } else {
        if (dep) k_stream<false, true, false, 8, ADJ><<<g, T, sm, s>>>(a);
        else k_stream<false, false, false, 8, ADJ><<<g, T, sm, s>>>(a);
    }
}

template <int ADJ>
void slow_pass(const Args &a, const LaunchCfg &c, bool det, bool dep, cudaStream_t s)
{
    const int g = dep ? c.grid_slow_dep : c.grid_slow;
    const size_t sm = dep ? c.smem_slow_dep : c.smem_slow;
    const int gp = dep ? c.grid_place_dep : c.grid_place;
    const size_t smp = dep ? c.smem_place_dep : c.smem_place;
    if (det) {
        if (dep) { k_event<true, true, ADJ><<<g, TPB, sm, s>>>(a); k_place<true, true, ADJ><<<gp, TPB, smp, s>>>(a); }
        else { k_event<true, false, ADJ><<<g, TPB, sm, s>>>(a); k_place<true, false, ADJ><<<gp, TPB, smp, s>>>(a); }
    } else {
        if (dep) { k_event<false, true, ADJ><<<g, TPB, sm, s>>>(a); k_place<false, true, ADJ><<<gp, TPB, smp, s>>>(a); }
        else { k_event<false, false, ADJ><<<g, TPB, sm, s>>>(a); k_place<false, false, ADJ><<<gp, TPB, smp, s>>>(a); }
    }
}

}  // namespace

cudaError_t configure_adjoint(const Args &a, int pass, LaunchCfg *cfg)
{
    return pass == 1 ? configure_pass<1>(a, cfg) : configure_pass<2>(a, cfg);
}

cudaError_t launch_fast_adj(const Args &a0, const LaunchCfg &c, int pass, bool det, bool dep,
                            cudaStream_t s)
{
    Args a = a0;
    a.ring = dep ? c.ring_fast_dep : c.ring_fast;
    if (pass == 1) fast_pass<1>(a, c, det, dep, s);
    else fast_pass<2>(a, c, det, dep, s);
    return cudaGetLastError();
}

cudaError_t launch_slow_adj(const Args &a0, const LaunchCfg &c, int pass, bool det, bool dep,
                            cudaStream_t s)
{
    Args a = a0;
    a.grid_fast = dep ? c.grid_fast_dep : c.grid_fast;
    if (pass == 1) slow_pass<1>(a, c, det, dep, s);
    else slow_pass<2>(a, c, det, dep, s);
    return cudaGetLastError();
}

cudaError_t launch_inject_adj(const Args &a, const LaunchCfg &c, int pass, int half, bool deposit,
                              cudaStream_t s)
{
    if (pass == 1) k_inject<1><<<c.grid_inject, TPB, 0, s>>>(a, half, deposit ? 1 : 0);
    else k_inject<2><<<c.grid_inject, TPB, 0, s>>>(a, half, deposit ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_compact_adj(const Args &a, const LaunchCfg &c, int pass, cudaStream_t s)
{
    if (pass == 1) k_compact<1><<<c.grid_compact, TPB, 0, s>>>(a);
    else k_compact<2><<<c.grid_compact, TPB, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flux_potential(const Args &a, const float *gJ, long long *gpot, int rows,
                                  double scale, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_flux_potential<<<(rows + TPB - 1) / TPB, TPB, 0, s>>>(a, gJ, gpot, rows, scale);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const float *x, long long n, unsigned int *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + TPB - 1) / TPB;
    if (blocks > 4096) blocks = 4096;
    k_absmax<<<(int)blocks, TPB, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float *gn, long long n, int32_t *q, double scale, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + TPB - 1) / TPB;
    if (blocks > 4096) blocks = 4096;
    k_quantize<<<(int)blocks, TPB, 0, s>>>(gn, n, q, scale);
    return cudaGetLastError();
}

cudaError_t launch_init_acc(const Args &a, const LaunchCfg &c, int pass, cudaStream_t s)
{
    k_init_acc<<<c.grid_compact, TPB, 0, s>>>(a, pass);
    return cudaGetLastError();
}

cudaError_t launch_flush_own(const Args &a, const LaunchCfg &c, cudaStream_t s)
{
    k_flush_own<<<c.grid_compact, TPB, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lineage(const Args &a, const LaunchCfg &c, long long n_ids, int g,
                           cudaStream_t s)
{
    if (n_ids <= 0) return cudaSuccess;
    long long blocks = (n_ids + TPB - 1) / TPB;
    if (blocks > c.grid_compact) blocks = c.grid_compact;
    k_lineage<<<(int)blocks, TPB, 0, s>>>(a, n_ids, g);
    return cudaGetLastError();
}

}  // namespace pic
