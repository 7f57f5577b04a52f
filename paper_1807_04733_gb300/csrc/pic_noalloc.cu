// Allocation-free compaction entry point (declared in include/pic.h).
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// owned entirely by its own allocator or memory pool (and which must not have
// a library allocate or free behind its back), or a latency-critical loop
// that must not allocate at all.  pic_compact_static lets them run the
// stable removal of dead slots on particle arrays they own.  The kernel is
// the library's compaction kernel; its scratch (per-block look-back words,
// the control block and the counters) lives in the file-scope device array
// below instead of in a context's allocation.
//
// The array is static device memory: every GPU that loads the library holds
// it (about 33 KB) until the process exits.  All calls on a device share it
// and it keeps the last call's contents, so every call re-initialises the
// part that must start from a known value; two calls whose kernels overlap
// on the GPU (different streams, or host threads) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "pic_internal.h"

using namespace pic;

namespace {

constexpr int kMaxBlocks = 4096;       // look-back words: one per block
constexpr int kMaxDevices = 64;

struct Scratch {
    DevCtl ctl;
    DevCounters cnt;
    DevStack stack;
    unsigned long long status[kMaxBlocks];
};

static __device__ __align__(256) unsigned char g_compact_scratch[sizeof(Scratch)];

struct DeviceSetup {
    bool ready = false;
    Scratch *addr = nullptr;     // device address of g_compact_scratch
    int grid = 0;
    unsigned int epoch = 0;      // tag of this device's look-back words
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

pic_status cuda_error(cudaError_t e, const char *where)
{
    pic_set_static_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
    return PIC_ERR_CUDA;
}

}  // namespace

extern "C" pic_status pic_compact_static(const float *z, const float *mu, const uint32_t *id,
                                         const uint32_t *packed, int64_t n, float *z_out,
                                         float *mu_out, uint32_t *id_out, uint32_t *packed_out,
                                         int64_t *n_alive, void *cuda_stream)
{
    if (!n_alive || n < 0) return PIC_ERR_ARG;
    // the look-back words carry counts in 30 bits
    if (n >= (int64_t(1) << 30)) return PIC_ERR_ARG;
    if (n > 0 && (!z || !mu || !id || !packed || !z_out || !mu_out || !id_out || !packed_out))
        return PIC_ERR_ARG;
    // the kernel reads the inputs in 16-byte vectors
    if (n > 0 && ((reinterpret_cast<uintptr_t>(packed) | reinterpret_cast<uintptr_t>(z) |
                   reinterpret_cast<uintptr_t>(mu) | reinterpret_cast<uintptr_t>(id)) & 15u))
        return PIC_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "pic_compact_static: current device");
    if (dev < 0 || dev >= kMaxDevices) return PIC_ERR_ARG;

    Scratch *scr = nullptr;
    int grid = 0;
    unsigned int epoch = 0;
    {
        // set-up, with the device current: the device address of the static
        // array (its host-side name is only a stand-in).  It is looked up on
        // every call, not cached: after a cudaDeviceReset the module is loaded
        // again and the array may sit at another address.
        std::lock_guard<std::mutex> lock(g_mu);
        DeviceSetup &d = g_dev[dev];
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_compact_scratch);
        if (e != cudaSuccess) return cuda_error(e, "pic_compact_static: scratch address");
        d.addr = static_cast<Scratch *>(p);
        if (!d.ready) {
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_error(e, "pic_compact_static: SM count");
            d.grid = sms * (2048 / TPB);
            if (d.grid > kMaxBlocks) d.grid = kMaxBlocks;
            d.ready = true;
        }
        scr = d.addr;
        grid = d.grid;
        epoch = ++d.epoch;           // words of earlier calls carry older tags
        if (epoch == 0) epoch = ++d.epoch;
    }
    if (n == 0) { *n_alive = 0; return PIC_OK; }

    // control block, counters and the one-"stack" description start fresh
    struct Header { DevCtl ctl; DevCounters cnt; DevStack stack; } h;
    std::memset(&h, 0, sizeof(h));
    h.ctl.epoch = epoch;
    h.cnt.n_slots = (unsigned long long)n;
    h.stack.n_layers = 1;
    h.stack.base = 0;
    h.stack.cap = n;
    static_assert(offsetof(Scratch, ctl) == offsetof(Header, ctl), "layout");
    static_assert(offsetof(Scratch, cnt) == offsetof(Header, cnt), "layout");
    static_assert(offsetof(Scratch, stack) == offsetof(Header, stack), "layout");
    e = cudaMemcpyAsync(scr, &h, sizeof(h), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_error(e, "pic_compact_static: scratch reset");

    Args a{};
    a.stacks = &scr->stack;
    a.n_stacks = 1;
    a.z[0] = const_cast<float *>(z);  a.z[1] = z_out;
    a.mu[0] = const_cast<float *>(mu); a.mu[1] = mu_out;
    a.id[0] = const_cast<uint32_t *>(id); a.id[1] = id_out;
    a.pk[0] = const_cast<uint32_t *>(packed); a.pk[1] = packed_out;
    a.mp_stride = 1;                      // separate mu and packed arrays
    a.status = scr->status;
    a.cnt = &scr->cnt;
    a.ctl = &scr->ctl;
    a.spin_limit = 1u << 24;
    LaunchCfg c{};
    c.grid_compact = grid;
    e = launch_compact(a, c, stream);
    if (e != cudaSuccess) return cuda_error(e, "pic_compact_static: launch");

    unsigned long long alive = 0;
    unsigned int status = 0;
    e = cudaMemcpyAsync(&alive, &scr->cnt.n_slots, sizeof(alive), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, &scr->ctl.status, sizeof(status), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_error(e, "pic_compact_static: result");
    if (status != 0) return (pic_status)status;
    *n_alive = (int64_t)alive;
    return PIC_OK;
}
