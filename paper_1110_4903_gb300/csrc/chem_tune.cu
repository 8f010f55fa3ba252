// chem_tune.cu -- launch-shape autotuner and captured CUDA graphs of the step.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/chem.h"
#include "chem_handle.h"

namespace chem {

// A sample is grown until one step of it takes this long in the default shape.
constexpr float kTuneTargetMs = 100.f;

// Gathers a strided sample of cells into contiguous buffers.
__global__ void gather_cells_kernel(int ns, long long m, long long stride, long long ld, const double *rho,
                                    const double *e, const double *T, double *rho_o, double *e_o,
                                    double *T_o) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long src = i * stride;
    for (int s = 0; s < ns; ++s) rho_o[(size_t)s * m + i] = rho[(size_t)s * ld + src];
    e_o[i] = e[src];
    T_o[i] = T ? T[src] : 1500.0;
}

}  // namespace chem

using namespace chem;

struct chem_graph_s {
    Handle *h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long *counter = nullptr;
};

extern "C" int chem_autotune(chem_handle_t hh, int32_t prec, int64_t n_cells, int64_t ld, const double *rho_s,
                             const double *e, double dt, const double *T_in, void *stream, int32_t *lanes_out,
                             int32_t *wpb_out) {
    Handle *h = hh;
    if (!h || !rho_s || !e || n_cells < 1) return fail(CHEM_E_INVALID_ARG, "bad argument");
    if (prec != CHEM_FP64 && prec != CHEM_MIXED) return fail(CHEM_E_INVALID_ARG, "precision %d", prec);
    if (ld == 0) ld = n_cells;
    if (ld < n_cells || !(dt >= 0)) return fail(CHEM_E_INVALID_ARG, "sizes or dt");
    const int ns = h->ns;
    const int Gs_small[] = {2, 4, 8, 16};
    const int Gs_large[] = {8, 16, 32};
    const bool small = ns + 1 <= 16;
    const int *Gs = small ? Gs_small : Gs_large;
    const int nG = small ? 4 : 3;
    // the sample fills the GPU with at least eight waves of the candidate that
    // holds the most cells at once (a sample smaller than a wave times the
    // slowest cell, not the throughput)
    long long wave = 0;
    for (int gi = 0; gi < nG; ++gi) {
        LaunchCfg cfg;
        if (configure(h, prec, Gs[gi], 0, cfg) != CHEM_OK) continue;
        const long long cells = (long long)cfg.grid * (cfg.block / 32) * (32 / Gs[gi]);
        if (cells > wave) wave = cells;
    }
    long long m = 8 * wave > 16384 ? 8 * wave : 16384;
    if (m > n_cells) m = n_cells;
    cudaStream_t st = (cudaStream_t)stream;
    // pristine sample, work copy, temperature guesses
    double *buf = nullptr, *s_rho = nullptr, *s_e = nullptr, *w_rho = nullptr, *w_e = nullptr, *s_T = nullptr;
    size_t per = 0;
    auto take_sample = [&](long long mm) -> int {
        if (buf) cudaFree(buf);
        buf = nullptr;
        per = (size_t)mm * (ns + 1);
        const cudaError_t ce = cudaMalloc(&buf, sizeof(double) * (2 * per + mm));
        if (ce != cudaSuccess) return fail(CHEM_E_OOM, "autotune sample buffers");
        s_rho = buf;
        s_e = buf + (size_t)mm * ns;
        w_rho = buf + per;
        w_e = w_rho + (size_t)mm * ns;
        s_T = buf + 2 * per;
        gather_cells_kernel<<<(unsigned)((mm + 127) / 128), 128, 0, st>>>(ns, mm, n_cells / mm, ld, rho_s, e, T_in,
                                                                         s_rho, s_e, s_T);
        h->launches.fetch_add(1);
        return CHEM_OK;
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one step of the sample in shape cfg; the second of two runs is timed
    auto time_cfg = [&](LaunchCfg &cfg, float &ms) -> int {
        for (int rep = 0; rep < 2; ++rep) {
            cudaMemcpyAsync(w_rho, s_rho, sizeof(double) * per, cudaMemcpyDeviceToDevice, st);
            chem_advance_args a;
            memset(&a, 0, sizeof a);
            a.n_cells = m;
            a.ld = m;
            a.rho_s = w_rho;
            a.e = w_e;
            a.dt = dt;
            a.T_in = s_T;
            a.stream = st;
            cudaEventRecord(e0, st);
            const int r = launch_cfg(h, &a, prec, &cfg, next_counter(h));
            cudaEventRecord(e1, st);
            if (r) return r;
            const cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) return cuda_fail(ce, "autotune run");
            cudaEventElapsedTime(&ms, e0, e1);
        }
        return CHEM_OK;
    };
    int rc = take_sample(m);
    // Work per cell can vary by orders of magnitude across a field (a flame
    // front among cold gas): a sample that runs for less time than its
    // hardest cells times their latency, not the throughput.  Grow it until
    // the library's default shape needs kTuneTargetMs on it.
    {
        LaunchCfg cfg;
        for (int grow = 0; rc == CHEM_OK && grow < 4 && m < n_cells; ++grow) {
            float ms = 0.f;
            if (configure(h, prec, h->lanes[prec], 0, cfg) != CHEM_OK) break;
            rc = time_cfg(cfg, ms);
            if (rc || ms >= kTuneTargetMs) break;
            const double f = ms > 0.f ? kTuneTargetMs / ms : 64.0;
            long long mm = (long long)(m * (f < 2.0 ? 2.0 : f > 64.0 ? 64.0 : f));
            m = mm < n_cells ? mm : n_cells;
            rc = take_sample(m);
        }
    }
    int best_G = 0, best_w = 0;
    float best_ms = 1e30f;
    for (int gi = 0; gi < nG && rc == CHEM_OK; ++gi) {
        for (int wpb = 1; wpb <= kMaxBlockThreads / 32; ++wpb) {
            LaunchCfg cfg;
            if (configure(h, prec, Gs[gi], wpb, cfg) != CHEM_OK) continue;   // does not fit
            float ms = 0.f;
            rc = time_cfg(cfg, ms);
            if (rc) break;
            if (ms < best_ms) {
                best_ms = ms;
                best_G = Gs[gi];
                best_w = wpb;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) return rc;
    if (!best_G) return fail(CHEM_E_UNSUPPORTED, "no launch shape fits");
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->lanes[prec] = best_G;
        h->wpb[prec] = best_w;
        h->tuned[prec] = true;
    }
    if (lanes_out) *lanes_out = best_G;
    if (wpb_out) *wpb_out = best_w;
    return CHEM_OK;
}

extern "C" int chem_graph_create(chem_handle_t hh, const chem_advance_args *a, chem_graph_t *out) {
    Handle *h = hh;
    if (!h || !a || !out) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (a->n_cells < 1 || !a->rho_s || !a->e || (a->ld != 0 && a->ld < a->n_cells) || !(a->dt >= 0))
        return fail(CHEM_E_INVALID_ARG, "bad step arguments");
    const int prec = a->precision < 0 ? h->opts.precision : a->precision;
    if (prec != CHEM_FP64 && prec != CHEM_MIXED) return fail(CHEM_E_INVALID_ARG, "precision %d", prec);
    const int G = a->lanes_per_cell ? a->lanes_per_cell : h->lanes[prec];
    LaunchCfg *cfg = nullptr;
    int rc = get_cfg(h, prec, G, &cfg);   // resolve attributes before capturing
    if (rc) return rc;
    chem_graph_s *g = new chem_graph_s();
    g->h = h;
    cudaError_t ce = cudaMalloc(&g->counter, sizeof(unsigned long long));
    if (ce != cudaSuccess) { delete g; return fail(CHEM_E_OOM, "graph work counter"); }
    cudaStream_t cs;
    ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) { cudaFree(g->counter); delete g; return cuda_fail(ce, "capture stream"); }
    chem_advance_args b = *a;
    b.stream = cs;
    ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        rc = launch_step(h, &b, prec, G, g->counter);
        const cudaError_t ce2 = cudaStreamEndCapture(cs, &g->graph);
        if (rc == CHEM_OK && ce2 != cudaSuccess) rc = cuda_fail(ce2, "ending the capture");
    } else {
        rc = cuda_fail(ce, "beginning the capture");
    }
    if (rc == CHEM_OK) {
        ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (ce != cudaSuccess) rc = cuda_fail(ce, "instantiating the graph");
    }
    cudaStreamDestroy(cs);
    // the captured launch was counted by launch_step; it has not run
    h->launches.fetch_sub(1);
    if (rc) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        cudaFree(g->counter);
        delete g;
        return rc;
    }
    *out = g;
    return CHEM_OK;
}

extern "C" int chem_graph_launch(chem_graph_t g, void *stream) {
    if (!g) return fail(CHEM_E_INVALID_ARG, "graph is NULL");
    const cudaError_t ce = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "launching the graph");
    g->h->launches.fetch_add(1);
    return CHEM_OK;
}

extern "C" int chem_graph_destroy(chem_graph_t g) {
    if (!g) return fail(CHEM_E_INVALID_ARG, "graph is NULL");
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->counter) cudaFree(g->counter);
    delete g;
    return CHEM_OK;
}
