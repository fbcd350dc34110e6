// Launch-shape autotuner and CUDA-graph batches of heterogeneous problems.
//
// ftwa_autotune times every feasible stepper shape (variant x cluster size)
// of one plan on a short probe integration and pins the fastest.
// ftwa_batch_create captures the evolves of many plans (lattices of uneven
// size, several U) into one CUDA graph: each problem's persistent stepper is
// a kernel node on its own branch, so the graph is one launch and kernels of
// different problems overlap at their tails.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ftwa_internal.h"

using namespace ftwa;

extern "C" {

int ftwa_autotune(ftwa_plan_t *plan, int64_t M, int32_t probe_steps, void *stream)
{
    Plan *p = plan;
    if (!p || M < 1 || probe_steps < 1) return FTWA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int saved_variant = p->variant_override, saved_cluster = p->cluster_override;
    const int64_t Mp = std::min<int64_t>(M, 8192);
    const size_t elem = p->precision == FTWA_FP64 ? 16 : 8;
    void *rho = nullptr;
    cudaError_t e = cudaMalloc(&rho, elem * 2 * (size_t)p->N * p->N * (size_t)Mp);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 0.0f;
    int best_v = 0, best_c = 0;
    int rc = FTWA_OK;
    for (int v = 1; v <= 3 && rc == FTWA_OK; ++v) {
        for (int c = 1; c <= kMaxCluster && rc == FTWA_OK; c *= 2) {
            p->variant_override = v;
            p->cluster_override = c;
            StepperShape ss;
            BandShape bs;
            const bool ok = v == 1 ? choose_band_shape(p, Mp, &bs) == FTWA_OK
                                   : v == 2 ? choose_stepper_shape(p, Mp, &ss) == FTWA_OK
                                            : tile_supported(p);
            if (!ok) continue;
            rc = launch_sample(p, 12345, 0, Mp, rho, s);
            if (rc != FTWA_OK) break;
            int r1 = launch_evolve(p, rho, Mp, 2, nullptr, s);   // warm-up (also uploads tables)
            if (r1 == FTWA_ERR_UNSUPPORTED) continue;             // e.g. no co-resident cluster of this size
            if (r1 != FTWA_OK) {
                rc = r1;
                break;
            }
            cudaEventRecord(e0, s);
            rc = launch_evolve(p, rho, Mp, probe_steps, nullptr, s);
            cudaEventRecord(e1, s);
            if (rc != FTWA_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = FTWA_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_v == 0 || ms < best_ms) {
                best_ms = ms;
                best_v = v;
                best_c = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(rho);
    if (rc != FTWA_OK || best_v == 0) {
        p->variant_override = saved_variant;
        p->cluster_override = saved_cluster;
        return rc != FTWA_OK ? rc : FTWA_ERR_UNSUPPORTED;
    }
    p->variant_override = best_v;
    p->cluster_override = best_c;
    // record the chosen shape in the plan
    p->dry_run = true;
    rc = launch_evolve(p, nullptr, M, 0, nullptr, s);
    p->dry_run = false;
    return rc;
}

int ftwa_batch_create(ftwa_plan_t *const *plans, int32_t n, void *const *rho_dev, const int64_t *M, int64_t n_steps,
                      void *const *snap_dev, ftwa_batch_t **out)
{
    if (!out || !plans || !rho_dev || !M || n < 1 || n_steps < 0) return FTWA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!plans[i] || M[i] < 0 || (M[i] > 0 && !rho_dev[i])) return FTWA_ERR_INVALID_ARGUMENT;
    // a time-dependent drive fills its pulse table per call, and graphs carry
    // only the plain steppers: driven and long-range plans are not captured
    for (int i = 0; i < n; ++i)
        if (plans[i]->drive || plans[i]->longrange || plans[i]->hop_drive) return FTWA_ERR_UNSUPPORTED;
    cudaStream_t prep = nullptr, cap = nullptr;
    if (cudaStreamCreateWithFlags(&prep, cudaStreamNonBlocking) != cudaSuccess) return FTWA_ERR_CUDA;
    // prepare: choose every shape and upload every table outside the capture
    int rc = FTWA_OK;
    for (int i = 0; i < n && rc == FTWA_OK; ++i) {
        Plan *p = plans[i];
        p->dry_run = true;
        rc = launch_evolve(p, rho_dev[i], M[i], n_steps, snap_dev ? snap_dev[i] : nullptr, prep);
        p->dry_run = false;
    }
    if (rc == FTWA_OK && cudaStreamSynchronize(prep) != cudaSuccess) rc = FTWA_ERR_CUDA;
    cudaStreamDestroy(prep);
    if (rc != FTWA_OK) return rc;

    ftwa_batch *b = new (std::nothrow) ftwa_batch();
    if (!b) return FTWA_ERR_OUT_OF_MEMORY;
    b->n = n;
    std::vector<cudaStream_t> st(n, nullptr);
    std::vector<cudaEvent_t> ev(n, nullptr);
    cudaEvent_t fork = nullptr;
    bool capturing = false;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    capturing = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
    for (int i = 0; i < n && e == cudaSuccess && rc == FTWA_OK; ++i) {
        e = cudaStreamWaitEvent(st[i], fork, 0);
        if (e != cudaSuccess) break;
        rc = launch_evolve(plans[i], rho_dev[i], M[i], n_steps,
                           snap_dev ? snap_dev[i] : nullptr, st[i]);
        if (rc != FTWA_OK) break;
        e = cudaEventRecord(ev[i], st[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[i], 0);
    }
    if (capturing) {
        const cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && rc == FTWA_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    for (int i = 0; i < n; ++i) {
        if (st[i]) cudaStreamDestroy(st[i]);
        if (ev[i]) cudaEventDestroy(ev[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (rc == FTWA_OK && e != cudaSuccess) rc = set_cuda_error(e);
    if (rc != FTWA_OK) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return rc;
    }
    *out = b;
    return FTWA_OK;
}

int ftwa_batch_launch(ftwa_batch_t *b, void *stream)
{
    if (!b || !b->exec) return FTWA_ERR_INVALID_ARGUMENT;
    return set_cuda_error(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
}

void ftwa_batch_destroy(ftwa_batch_t *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_owned) cudaFree(b->d_owned);
    delete b;
}

}  // extern "C"
