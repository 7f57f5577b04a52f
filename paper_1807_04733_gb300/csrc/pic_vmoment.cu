// Velocity moment behind the spin current (Eq. spincurrent, Sec. V).
//
// At the end of a density step (the same instants as the densities of
// Eq. firstmoment), the velocity along z of every live carrier, v(material
// of its layer, spin, k) * mu, is summed per (spin, cell).  The product is
// taken in float32 and kept as an integer number of 2^-32 nm/fs (truncated
// toward zero), so the sums are exact and do not depend on the order of the
// atomic additions.  (sum_up - sum_down) / dz is the spin-current density of
// the cell.  Opt-in (PIC_F_VELOCITY_MOMENTS): one extra read of the state
// per density step.
//
// One block owns a contiguous chunk of tiles, as the other streaming
// kernels; four consecutive slots per thread; per-stack sums in shared
// memory, flushed once per stack segment.
#include <cuda_runtime.h>

#include "pic_step.cuh"

namespace pic {

__global__ void __launch_bounds__(TPB) k_vmoment(const Args a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_v = reinterpret_cast<unsigned long long *>(smem);   // [2][n_cells]
    __shared__ long long s_tpref[PIC_MAX_STACKS + 1];
    __shared__ long long s_nsl[PIC_MAX_STACKS];
    const int cur = (int)*(volatile unsigned int *)&a.ctl->cur;
    const int tid = threadIdx.x;
    // launched after the step's last kernel: in a graph replay that kernel
    // has already advanced the device step counter
    const uint32_t step = a.step_dev ? __ldcg(a.step_dev) - 1u : a.step;
    const int tout = (int)((step + 1) / (uint32_t)a.moment_every) - 1;
    Plan p;
    make_plan(a, s_tpref, s_nsl, p);
    const uint2 *MP = reinterpret_cast<const uint2 *>(a.mu[cur]);   // (mu, packed) pairs
    const float *Z = a.z[cur];

    auto flush = [&](int s) {
        __syncthreads();
        const DevStack &st = a.stacks[s];
        unsigned long long *gV = reinterpret_cast<unsigned long long *>(a.v_hist) + st.n_off / a.n_e +
                                 (long long)tout * 2 * st.n_cells;
        for (int i = tid; i < 2 * st.n_cells; i += TPB) {
            const unsigned long long v = s_v[i];
            if (v) atomicAdd(&gV[i], v);
        }
        __syncthreads();
    };

    int seg = -1;
    for (long long t = p.t0; t < p.t1; ++t) {
        const int s = stack_of(s_tpref, a.n_stacks, t);
        if (s != seg) {
            if (seg >= 0) flush(seg);
            for (int i = tid; i < 2 * a.stacks[s].n_cells; i += TPB) s_v[i] = 0ull;
            __syncthreads();
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
            const uint2 mp = MP[g];
            const uint32_t pk = mp.y;
            const int k = (int)(pk & 0xFFu);
            if (k == 0) continue;
            const int sg = (int)((pk >> 8) & 1u), layer = (int)((pk >> 9) & 0xFu);
            const float v = a.fent[st.ent_off + (layer * 2 + sg) * a.n_e + (k - 1)].v;
            const float w = __fmul_rn(v, __uint_as_float(mp.x));
            const long long q = __float2ll_rz(__fmul_rn(w, 4294967296.0f));
            const int c = cell_of(a, tmp, Z[g]);
            atomicAdd(&s_v[sg * st.n_cells + c], (unsigned long long)q);
        }
    }
    if (seg >= 0) flush(seg);
}

cudaError_t launch_vmoment(const Args &a, const LaunchCfg &c, cudaStream_t s)
{
    const size_t sm = (size_t)2 * (a.gbin_max > 0 ? a.gbin_max : 1) * sizeof(unsigned long long);
    k_vmoment<<<c.grid_compact, TPB, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
