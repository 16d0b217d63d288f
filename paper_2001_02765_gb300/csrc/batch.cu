// Batches of independent solves replayed as one CUDA graph.
//
// sg_batch_create binds n solves (plan + caller buffers each) and captures them
// once: the capture forks one stream per member from a root stream, enqueues
// the member's solve on its own workspace there, and joins all members back,
// so the graph holds n independent branches that the GPU runs concurrently.
// sg_batch_launch replays the whole batch with a single graph launch, which
// removes the per-kernel launch overhead of uneven small solves.
#include "common.cuh"

#include <new>
#include <vector>

struct sg_batch {
    int n = 0;
    std::vector<sg_workspace> ws;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

namespace {

void batch_free(sg_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (sg_workspace &w : b->ws) sg_workspace_free(&w, 0, false);
    delete b;
}

}  // namespace

extern "C" {

sg_status sg_batch_create(int n, sg_plan *const *plans, const void *const *sigma, const void *const *deltax,
                          const void *const *deltay, void *const *fx, void *const *fy, sg_batch **out)
{
    if (n < 1 || !plans || !sigma || !fx || !fy || !out) return SG_EINVAL;
    int dev = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !sigma[i] || !fx[i] || !fy[i] || plans[i]->device != dev) return SG_EINVAL;
        if (plans[i]->geom.slope_mode == SG_SLOPES_CALLER && (!deltax || !deltay || !deltax[i] || !deltay[i]))
            return SG_EINVAL;
    }
    sg_batch *b = new (std::nothrow) sg_batch();
    if (!b) return SG_ENOMEM;
    b->n = n;
    b->device = dev;
    b->ws.resize(n);
    for (int i = 0; i < n; ++i) {
        sg_status a = sg_workspace_alloc(plans[i], &b->ws[i], 0, false);
        if (a != SG_OK) {
            b->ws.resize(i);
            batch_free(b);
            return a;
        }
        // the members already run side by side: keep each member's work on its own branch
        sg_workspace &w = b->ws[i];
        if (w.aux) {
            cudaStreamDestroy(w.aux);
            cudaEventDestroy(w.ev_fork);
            cudaEventDestroy(w.ev_join);
            w.aux = nullptr;
            w.ev_fork = w.ev_join = nullptr;
        }
    }
    // capture: root stream -> one branch per member -> join
    std::vector<cudaStream_t> streams(n + 1, nullptr);
    std::vector<cudaEvent_t> events(n + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i <= n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&events[i], cudaEventDisableTiming);
    }
    sg_status st = e == cudaSuccess ? SG_OK : SG_ECUDA;
    bool capturing = false;
    if (st == SG_OK) {
        e = cudaStreamBeginCapture(streams[n], cudaStreamCaptureModeRelaxed);
        capturing = e == cudaSuccess;
        if (e == cudaSuccess) e = cudaEventRecord(events[n], streams[n]);
        if (e != cudaSuccess) st = SG_ECUDA;
    }
    for (int i = 0; i < n && st == SG_OK; ++i) {
        if (cudaStreamWaitEvent(streams[i], events[n], 0) != cudaSuccess) {
            st = SG_ECUDA;
            break;
        }
        st = sg_force_ws(plans[i], &b->ws[i], sigma[i], deltax ? deltax[i] : nullptr, deltay ? deltay[i] : nullptr,
                         fx[i], fy[i], streams[i]);
        if (st == SG_OK && (cudaEventRecord(events[i], streams[i]) != cudaSuccess ||
                            cudaStreamWaitEvent(streams[n], events[i], 0) != cudaSuccess))
            st = SG_ECUDA;
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(streams[n], &g);
        if (st == SG_OK && e == cudaSuccess) {
            b->graph = g;
            e = cudaGraphInstantiate(&b->exec, g, 0);
            if (e != cudaSuccess) st = SG_ECUDA;
        } else {
            if (g) cudaGraphDestroy(g);
            if (st == SG_OK) st = SG_ECUDA;
        }
    }
    if (st != SG_OK && e != cudaSuccess) sg_set_last_cuda_error(e, "sg_batch_create");
    cudaGetLastError();
    for (int i = 0; i <= n; ++i) {
        if (streams[i]) cudaStreamDestroy(streams[i]);
        if (events[i]) cudaEventDestroy(events[i]);
    }
    if (st != SG_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return SG_OK;
}

sg_status sg_batch_launch(sg_batch *b, void *stream)
{
    if (!b) return SG_EINVAL;
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->device) return SG_EINVAL;
    SG_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return SG_OK;
}

sg_status sg_batch_destroy(sg_batch *b)
{
    batch_free(b);
    return SG_OK;
}

}  // extern "C"
