// chem_handle.h -- the object behind chem_handle_t.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/chem.h"
#include "chem_internal.h"

namespace chem {

struct LaunchCfg {
    const void *fn = nullptr;
    int block = 0;       // threads per block
    int grid = 0;        // persistent grid: blocks per SM x SMs
    size_t smem = 0;     // dynamic shared memory per block
    int G = 0;           // lanes per cell
};

// Work counters: one per launch, taken round-robin, zeroed in-stream before
// the launch that uses it.  A counter is reused after kCounterRing further
// launches of the handle, so at most that many of its launches may be in
// flight at once (on whatever streams); chem.h states the limit.
constexpr unsigned kCounterRing = 4096;

struct ServingState;

}  // namespace chem

struct chem_handle_s {
    chem_options opts{};
    int ns = 0, nr = 0;
    int device = 0;
    int num_sms = 0;
    long long max_smem_optin = 0;
    chem::DeviceMech mech{};
    void *dev_tables = nullptr;
    size_t dev_tables_bytes = 0;
    unsigned long long *counters = nullptr;
    std::atomic<unsigned> counter_idx{0};
    std::atomic<long long> launches{0};
    cudaStream_t stream = nullptr;      // the handle's own stream (host calls, serving)
    int lanes[2] = {0, 0};              // lanes per cell by precision
    int wpb[2] = {0, 0};                // warps per block by precision (0 = most resident warps)
    bool tuned[2] = {false, false};     // autotuned already
    std::mutex mu;
    std::map<int, chem::LaunchCfg> cfgs;
    // chem_advance_host staging
    std::mutex host_mu;
    void *host_rho = nullptr;
    size_t host_bytes = 0;
    chem::ServingState *serving = nullptr;
    std::vector<double> ef_host;        // formation energies per unit mass
};

namespace chem {
using Handle = ::chem_handle_s;

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
int get_cfg(Handle *h, int prec, int G, LaunchCfg **out, bool queue = false);
int configure(Handle *h, int prec, int G, int wpb, LaunchCfg &cfg, bool queue = false);
const void *be_kernel_queue(int prec, int G);
int launch_step(Handle *h, const chem_advance_args *a, int prec, int G, unsigned long long *counter);
int launch_cfg(Handle *h, const chem_advance_args *a, int prec, const LaunchCfg *cfg,
               unsigned long long *counter);
unsigned long long *next_counter(Handle *h);
StepOptions step_options(const Handle *h, int prec);
void fill_log_table(std::vector<double> &tab);
void destroy_serving(Handle *h);
}  // namespace chem
