// chem_static.cu -- chem_advance_host_static: the host-buffer chemistry step
// without any device allocation.
//
// Who needs it: a caller that must not allocate device memory once it is
// running -- a host-side flow solver embedded in a framework that reserves
// the whole device through its own memory pool, or a real-time loop that
// forbids cudaMalloc/cudaFree after start-up (allocation latency, device-wide
// synchronisation, fragmentation).  chem_advance_host grows a staging buffer
// with cudaMalloc; this variant stages the cell state, the per-cell outputs
// and the kernel's work counter in one fixed, file-scope device array
// instead, so a call allocates nothing.
//
// The array is kStaticScratchBytes (16 MiB) and lives on every GPU that loads
// the library, until the process exits.  Every call shares it and it keeps
// the last call's contents; the work counter is zeroed in-stream before each
// launch, and the state area is overwritten by the call's own host-to-device
// copies before the kernel reads it.  Calls from one process are serialised
// by a per-device mutex; two calls that overlapped on the GPU (for example
// from two copies of the library in one process) would race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/chem.h"
#include "chem_handle.h"

namespace chem {

constexpr size_t kStaticScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

// Device-side scratch.  Host code must not pass this name to a kernel: on the
// host it is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticSlot {
    std::mutex mu;
    bool ready = false;
    unsigned char *addr = nullptr;   // device address of g_static_scratch on this device
};
static StaticSlot g_slots[kMaxDevices];

}  // namespace chem

using namespace chem;

extern "C" int chem_static_scratch_bytes(int64_t *bytes) {
    if (!bytes) return fail(CHEM_E_INVALID_ARG, "bytes pointer is NULL");
    *bytes = (int64_t)kStaticScratchBytes;
    return CHEM_OK;
}

extern "C" int chem_advance_host_static(chem_handle_t hh, int64_t n_cells, int64_t ld, double *rho_s,
                                        double *e, double dt, double *T_out, int32_t *status) {
    Handle *h = hh;
    if (!h || !rho_s || !e) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n_cells < 0 || (ld != 0 && ld < n_cells)) return fail(CHEM_E_INVALID_ARG, "sizes");
    if (!(dt >= 0) || dt != dt || dt > 1e300) return fail(CHEM_E_INVALID_ARG, "dt %g", dt);
    if (n_cells == 0) return CHEM_OK;
    if (ld == 0) ld = n_cells;
    const int ns = h->ns;
    // layout: [counter: 256 B][rho_s: ns*n][e: n][T_out: n][status: n]
    const size_t per_cell = (size_t)ns * 8 + 8 + 8 + 4;
    const size_t head = 256;
    const size_t need = head + (size_t)n_cells * per_cell;
    if (need > kStaticScratchBytes) {
        const long long max_cells = (long long)((kStaticScratchBytes - head) / per_cell);
        return fail(CHEM_E_UNSUPPORTED,
                    "chem_advance_host_static: %lld cells need %zu bytes of static scratch; the "
                    "array holds %zu bytes, i.e. at most %lld cells of this %d-species mechanism "
                    "per call -- split the call",
                    (long long)n_cells, need, kStaticScratchBytes, max_cells, ns);
    }
    int dev = -1;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if (dev != h->device)
        return fail(CHEM_E_INVALID_ARG, "the current device (%d) is not the handle's (%d)", dev, h->device);
    if (dev < 0 || dev >= kMaxDevices) return fail(CHEM_E_UNSUPPORTED, "device index %d", dev);
    StaticSlot &slot = g_slots[dev];
    std::lock_guard<std::mutex> lk(slot.mu);
    if (!slot.ready) {
        // once per device, with that device current
        void *p = nullptr;
        ce = cudaGetSymbolAddress(&p, g_static_scratch);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetSymbolAddress of the static scratch");
        slot.addr = static_cast<unsigned char *>(p);
        slot.ready = true;
    }
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(slot.addr);
    double *d_rho = reinterpret_cast<double *>(slot.addr + head);
    double *d_e = d_rho + (size_t)n_cells * ns;
    double *d_T = d_e + n_cells;
    int32_t *d_st = reinterpret_cast<int32_t *>(d_T + n_cells);
    cudaStream_t st = h->stream;
    ce = cudaMemcpy2DAsync(d_rho, (size_t)n_cells * 8, rho_s, (size_t)ld * 8, (size_t)n_cells * 8, ns,
                           cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_e, e, (size_t)n_cells * 8, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "host-to-device copy");
    chem_advance_args a;
    memset(&a, 0, sizeof a);
    a.n_cells = n_cells;
    a.ld = n_cells;
    a.rho_s = d_rho;
    a.e = d_e;
    a.dt = dt;
    a.T_out = T_out ? d_T : nullptr;
    a.status = status ? d_st : nullptr;
    a.stream = st;
    const int prec = h->opts.precision;
    // zeroes the counter in-stream, then launches the step kernel
    int rc = launch_step(h, &a, prec, h->lanes[prec], counter);
    if (rc) return rc;
    ce = cudaMemcpy2DAsync(rho_s, (size_t)ld * 8, d_rho, (size_t)n_cells * 8, (size_t)n_cells * 8, ns,
                           cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(e, d_e, (size_t)n_cells * 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && T_out) ce = cudaMemcpyAsync(T_out, d_T, (size_t)n_cells * 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && status)
        ce = cudaMemcpyAsync(status, d_st, (size_t)n_cells * 4, cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "device-to-host copy");
    ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "synchronising the step");
    return CHEM_OK;
}
