// Forward step of the hot-electron PIC method: launch configuration and
// launchers of the kernels in pic_step.cuh.
#include <cuda_runtime.h>

#include "pic_step.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
cudaError_t configure(const Args &a, int blocks_per_sm, int ring_req, int hist_mode, LaunchCfg *cfg)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const size_t tiles = (size_t)(2 * a.n_stacks + 1) * 8 + 16;      // tile prefix, counts
    const size_t fixed = (size_t)a.tab_max * sizeof(FastEnt) + (size_t)a.jbin_max * 4 + 4 + tiles;
    const size_t fixed_dep = fixed + (size_t)(a.nbin_max + a.gbin_max) * 4;
    int o_plain = 0, o_dep = 0;
    if ((e = pick_ring<false, false>(fixed, blocks_per_sm, ring_req, &cfg->ring_fast, &o_plain,
                                     &cfg->smem_fast)) != cudaSuccess)
        return e;
    if (hist_mode == 1)
        e = pick_ring<true, true>(fixed_dep, blocks_per_sm, 0, &cfg->ring_fast_dep, &o_dep,
                                  &cfg->smem_fast_dep);
    else
        e = pick_ring<true, false>(fixed_dep, blocks_per_sm, 0, &cfg->ring_fast_dep, &o_dep,
                                   &cfg->smem_fast_dep);
    if (e != cudaSuccess) return e;
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

cudaError_t launch_fast(const Args &a0, const LaunchCfg &c, bool det, bool dep, int hist_mode,
                        cudaStream_t s)
{
    Args a = a0;
    a.ring = dep ? c.ring_fast_dep : c.ring_fast;
    const int g = dep ? c.grid_fast_dep : c.grid_fast;
    const size_t sm = dep ? c.smem_fast_dep : c.smem_fast;
    const bool w = hist_mode == 1;
    if (det) {
        if (dep) {
            if (w) k_fast<true, true, true><<<g, FAST_THREADS, sm, s>>>(a);
            else k_fast<true, true, false><<<g, FAST_THREADS, sm, s>>>(a);
        } else {
            k_fast<true, false, false><<<g, FAST_THREADS, sm, s>>>(a);
        }
    } else {
        if (dep) {
            if (w) k_fast<false, true, true><<<g, FAST_THREADS, sm, s>>>(a);
            else k_fast<false, true, false><<<g, FAST_THREADS, sm, s>>>(a);
        } else {
            k_fast<false, false, false><<<g, FAST_THREADS, sm, s>>>(a);
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
