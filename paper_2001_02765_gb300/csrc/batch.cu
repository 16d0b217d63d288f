// Batches of independent solves replayed as one CUDA graph.
//
// sg_batch_create binds n solves (plan + caller buffers each) and captures them
// once into a CUDA graph, so that sg_batch_launch replays the whole batch with
// a single graph launch. Members that are single in-plane patches with padded
// lengths up to 2048 run together in ONE persistent kernel per precision
// (batch_run.cuh): every pass of every such member is a work item of that
// launch, whatever their lengths and slope handling, ordered per member by
// completion counters, so uneven small solves fill the GPU together and the
// batch pays one kernel launch. Other members (hierarchies, off-plane plans,
// 4096-point transforms) keep a graph branch of their own, running beside it.
// Results are the members' sg_force results bit for bit.
#include "common.cuh"
#include "batch_run.cuh"

#include <algorithm>
#include <new>
#include <vector>

struct sg_batch {
    int n = 0;
    std::vector<sg_workspace> ws;
    std::vector<void *> dev_args;  // item lists, member arguments and counters of the persistent launches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    int launches = 0;  // kernels per replay
};

namespace {

void batch_free(sg_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (sg_workspace &w : b->ws) sg_workspace_free(&w, 0, false);
    for (void *a : b->dev_args) cudaFree(a);
    delete b;
}

// a member of the persistent launch: one unmasked in-plane patch, lengths <= 2048
bool persistent_member(const sg_plan *p)
{
    return p->npatches == 1 && !p->composite && !p->lv && p->geom.z == 0.0 &&
           sgk::batch_run_smem(p->prec == SG_FP64, p->pp[0].d.px, p->pp[0].d.py) > 0;
}

// The persistent launch of the members `mem` (one precision): item list,
// member arguments and counters uploaded (owned by the batch), before capture.
template <typename T>
struct persistent_run {
    const sgk::batch_item *items = nullptr;
    const sgk::batch_member<T> *members = nullptr;
    int *ctl = nullptr;
    int nitems = 0, nmem = 0, smem = 0, tries = 0;
    int *err = nullptr;
};

template <typename T>
sg_status persistent_upload(sg_batch *b, const std::vector<int> &mem, sg_plan *const *plans,
                            const void *const *sigma, const void *const *deltax, const void *const *deltay,
                            void *const *fx, void *const *fy, persistent_run<T> &run)
{
    using namespace sgk;
    const int m = (int)mem.size();
    std::vector<batch_member<T>> ms(m);
    std::vector<batch_item> fwd, col, inv;
    run.smem = 0;
    run.tries = SG_MBAR_MAX_TRIES;
    for (int k = 0; k < m; ++k) {
        const int i = mem[k];
        sg_plan *p = plans[i];
        const bool caller = p->geom.slope_mode == SG_SLOPES_CALLER;
        const uniform_passes<T> u = uniform_setup<T>(p, &b->ws[i], 0, sigma[i], caller ? deltax[i] : nullptr,
                                                      caller ? deltay[i] : nullptr, fx[i], fy[i], nullptr);
        batch_member<T> &bm = ms[k];
        bm.rf = u.rf;
        bm.ed = u.ed;
        bm.col = u.col;
        bm.ri = u.ri;
        bm.twx = u.twx;
        bm.twy = u.twy;
        bm.px = u.px;
        bm.py = u.py;
        bm.qx = u.qx;
        bm.nf_cols = u.nf_cols;
        bm.central = u.central ? 1 : 0;
        const int ny = p->pp[0].d.ny;
        const int groups = (ny + 2 * batch_nb(u.px) - 1) / (2 * batch_nb(u.px));
        for (int f = 0; f < u.nf_rows; ++f)
            for (int bx = 0; bx < groups; ++bx) fwd.push_back({BI_ROWF, k, bx, f});
        if (u.central) fwd.push_back({BI_EDGE, k, 0, 0});
        bm.need_fwd = u.nf_rows * groups + (u.central ? 1 : 0);
        const int cgroups = (u.qx + batch_cb(u.py) - 1) / batch_cb(u.py);
        for (int bx = 0; bx < cgroups; ++bx) col.push_back({BI_COL, k, bx, 0});
        bm.need_col = cgroups;
        for (int o = 0; o < 2; ++o)
            for (int bx = 0; bx < groups; ++bx) inv.push_back({BI_ROWI, k, bx, o});
        run.smem = std::max(run.smem, batch_run_smem(p->prec == SG_FP64, u.px, u.py));
        run.tries = std::min(run.tries, p->wait_tries);
    }
    std::vector<batch_item> items;
    items.reserve(fwd.size() + col.size() + inv.size());
    items.insert(items.end(), fwd.begin(), fwd.end());
    items.insert(items.end(), col.begin(), col.end());
    items.insert(items.end(), inv.begin(), inv.end());
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t si = items.size() * sizeof(batch_item), sm = ms.size() * sizeof(batch_member<T>);
    const size_t sc = (1 + 2 * (size_t)m) * sizeof(int);
    char *d = nullptr;
    SG_CUDA_TRY(cudaMalloc(&d, up(si) + up(sm) + up(sc)));
    b->dev_args.push_back(d);
    SG_CUDA_TRY(cudaMemcpy(d, items.data(), si, cudaMemcpyHostToDevice));
    SG_CUDA_TRY(cudaMemcpy(d + up(si), ms.data(), sm, cudaMemcpyHostToDevice));
    run.items = (const batch_item *)d;
    run.members = (const batch_member<T> *)(d + up(si));
    run.ctl = (int *)(d + up(si) + up(sm));
    run.nitems = (int)items.size();
    run.nmem = m;
    run.err = b->ws[mem[0]].err;
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_batch_create(int n, sg_plan *const *plans, const void *const *sigma, const void *const *deltax,
                          const void *const *deltay, void *const *fx, void *const *fy, sg_batch **out)
{
    if (n < 1 || !plans || !sigma || !fx || !fy || !out) return SG_EINVAL;
    int dev = 0, nsm = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    SG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
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
    }
    // members of the persistent launches (per precision) and the rest
    std::vector<int> mem32, mem64, rest;
    for (int i = 0; i < n; ++i) {
        if (!persistent_member(plans[i])) rest.push_back(i);
        else if (plans[i]->prec == SG_FP64) mem64.push_back(i);
        else mem32.push_back(i);
    }
    sg_status st = SG_OK;
    persistent_run<float> r32;
    persistent_run<double> r64;
    if (!mem32.empty()) st = persistent_upload<float>(b, mem32, plans, sigma, deltax, deltay, fx, fy, r32);
    if (st == SG_OK && !mem64.empty()) st = persistent_upload<double>(b, mem64, plans, sigma, deltax, deltay, fx, fy, r64);
    // capture: root stream -> one branch per persistent launch and per other member -> join
    const int nb = (int)rest.size() + 2;
    std::vector<cudaStream_t> streams(nb + 1, nullptr);
    std::vector<cudaEvent_t> events(nb + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i <= nb && e == cudaSuccess && st == SG_OK; ++i) {
        e = cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&events[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) st = SG_ECUDA;
    bool capturing = false;
    if (st == SG_OK) {
        e = cudaStreamBeginCapture(streams[nb], cudaStreamCaptureModeRelaxed);
        capturing = e == cudaSuccess;
        if (e == cudaSuccess) e = cudaEventRecord(events[nb], streams[nb]);
        if (e != cudaSuccess) st = SG_ECUDA;
    }
    int branch = 0;
    auto fork = [&](cudaStream_t bs) { return cudaStreamWaitEvent(bs, events[nb], 0) == cudaSuccess ? SG_OK : SG_ECUDA; };
    auto join = [&](cudaStream_t bs) {
        return cudaEventRecord(events[branch], bs) == cudaSuccess &&
                       cudaStreamWaitEvent(streams[nb], events[branch], 0) == cudaSuccess
                   ? SG_OK
                   : SG_ECUDA;
    };
    if (st == SG_OK && !mem32.empty()) {
        cudaStream_t bs = streams[branch];
        st = fork(bs);
        if (st == SG_OK)
            st = sgk::batch_run_launch<float>(r32.items, r32.nitems, r32.members, r32.nmem, r32.ctl, r32.err,
                                              r32.tries, r32.smem, nsm, bs);
        if (st == SG_OK) st = join(bs);
        b->launches += 1;
        ++branch;
    }
    if (st == SG_OK && !mem64.empty()) {
        cudaStream_t bs = streams[branch];
        st = fork(bs);
        if (st == SG_OK)
            st = sgk::batch_run_launch<double>(r64.items, r64.nitems, r64.members, r64.nmem, r64.ctl, r64.err,
                                               r64.tries, r64.smem, nsm, bs);
        if (st == SG_OK) st = join(bs);
        b->launches += 1;
        ++branch;
    }
    for (size_t k = 0; k < rest.size() && st == SG_OK; ++k) {
        const int i = rest[k];
        cudaStream_t bs = streams[branch];
        st = fork(bs);
        const bool caller = plans[i]->geom.slope_mode == SG_SLOPES_CALLER;
        if (st == SG_OK)
            st = sg_force_ws(plans[i], &b->ws[i], sigma[i], caller ? deltax[i] : nullptr,
                             caller ? deltay[i] : nullptr, fx[i], fy[i], bs);
        if (st == SG_OK) st = join(bs);
        b->launches += plans[i]->launches;
        ++branch;
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(streams[nb], &g);
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
    for (int i = 0; i <= nb; ++i) {
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

sg_status sg_batch_check_error(sg_batch *b)
{
    if (!b) return SG_EINVAL;
    SG_CUDA_TRY(cudaDeviceSynchronize());
    sg_status r = SG_OK;
    for (sg_workspace &w : b->ws) {
        int e = 0;
        if (!w.err) continue;
        SG_CUDA_TRY(cudaMemcpy(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            SG_CUDA_TRY(cudaMemset(w.err, 0, sizeof(int)));
            sg_set_last_error_message("a bounded wait for a bulk copy ran out in a kernel of the batch");
            r = SG_ETIMEOUT;
        }
    }
    return r;
}

sg_status sg_batch_launches(const sg_batch *b, int *out)
{
    if (!b || !out) return SG_EINVAL;
    *out = b->launches;
    return SG_OK;
}

}  // extern "C"
