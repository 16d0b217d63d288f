// Batches of independent solves replayed as one CUDA graph.
//
// sg_batch_create binds n solves (plan + caller buffers each) and captures them
// once: the capture forks one stream per member from a root stream, enqueues
// the member's solve on its own workspace there, and joins all members back,
// so the graph holds n independent branches that the GPU runs concurrently.
// sg_batch_launch replays the whole batch with a single graph launch, which
// removes the per-kernel launch overhead of uneven small solves.
//
// Members that are single in-plane patches with the same padded lengths,
// precision and slope handling form a group: each pass of the group is one
// launch over all its members (blockIdx.z = member, arguments from a device
// array), so that small solves fill the GPU together instead of as many
// concurrent small kernels. Other members keep their own branch.
#include "common.cuh"
#include "fftconv.cuh"

#include <map>
#include <new>
#include <tuple>
#include <vector>

struct sg_batch {
    int n = 0;
    std::vector<sg_workspace> ws;
    std::vector<void *> dev_args;  // per-group argument arrays
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

bool groupable(const sg_plan *p)
{
    return p->npatches == 1 && !p->composite && !p->lv && p->geom.z == 0.0;
}

// A group's passes: the members' arguments in one device array per pass.
template <typename T>
struct group_passes {
    sgk::uniform_passes<T> u;  // lengths, shapes and twiddles are common to the group
    const sgk::row_fwd_args<T> *rf = nullptr;
    const sgk::edge_args<T> *ed = nullptr;
    const sgk::col_args<T> *col = nullptr;
    const sgk::row_inv_args<T> *ri = nullptr;
    sgk::batch_shape bs = {0, 0};
    int *err = nullptr;
};

// Upload the argument arrays of a group (owned by the batch); before capture.
template <typename T>
sg_status group_upload(sg_batch *b, const std::vector<sgk::uniform_passes<T>> &us, int *err, group_passes<T> &g)
{
    const int m = (int)us.size();
    std::vector<sgk::row_fwd_args<T>> rf(m);
    std::vector<sgk::edge_args<T>> ed(m);
    std::vector<sgk::col_args<T>> col(m);
    std::vector<sgk::row_inv_args<T>> ri(m);
    int maxny = 0;
    for (int i = 0; i < m; ++i) {
        rf[i] = us[i].rf;
        ed[i] = us[i].ed;
        col[i] = us[i].col;
        ri[i] = us[i].ri;
        if (us[i].rf.src.ny > maxny) maxny = us[i].rf.src.ny;
    }
    const size_t s0 = m * sizeof(rf[0]), s1 = m * sizeof(ed[0]), s2 = m * sizeof(col[0]), s3 = m * sizeof(ri[0]);
    auto up = [](size_t n) { return (n + 255) & ~(size_t)255; };
    char *d = nullptr;
    SG_CUDA_TRY(cudaMalloc(&d, up(s0) + up(s1) + up(s2) + up(s3)));
    b->dev_args.push_back(d);
    SG_CUDA_TRY(cudaMemcpy(d, rf.data(), s0, cudaMemcpyHostToDevice));
    SG_CUDA_TRY(cudaMemcpy(d + up(s0), ed.data(), s1, cudaMemcpyHostToDevice));
    SG_CUDA_TRY(cudaMemcpy(d + up(s0) + up(s1), col.data(), s2, cudaMemcpyHostToDevice));
    SG_CUDA_TRY(cudaMemcpy(d + up(s0) + up(s1) + up(s2), ri.data(), s3, cudaMemcpyHostToDevice));
    g.u = us[0];
    g.rf = (const sgk::row_fwd_args<T> *)d;
    g.ed = (const sgk::edge_args<T> *)(d + up(s0));
    g.col = (const sgk::col_args<T> *)(d + up(s0) + up(s1));
    g.ri = (const sgk::row_inv_args<T> *)(d + up(s0) + up(s1) + up(s2));
    g.bs = {m, maxny};
    g.err = err;
    return SG_OK;
}

// One launch per pass for all the group's members.
template <typename T>
sg_status group_enqueue(const group_passes<T> &g, cudaStream_t st)
{
    const sgk::uniform_passes<T> &u = g.u;
    SG_TRY(sgk::rows_fwd<T>(u.px, u.shx[0], u.rf, u.nf_rows, u.twx, st, g.rf, g.bs));
    if (u.central) SG_TRY(sgk::edge_cols<T>(u.py, u.ed, u.twy, st, g.ed, g.bs));
    if (u.central) SG_TRY(sgk::cols_central<T>(u.py, u.shy[3], u.col, u.qx, u.twy, g.err, st, g.col, g.bs));
    else SG_TRY(sgk::cols<T>(u.py, u.shy[2], u.nout, u.col, u.qx, u.nf_cols, u.twy, g.err, st, g.col, g.bs));
    SG_TRY(sgk::rows_inv<T>(u.px, u.shx[1], u.ri, u.nout, u.twx, st, g.ri, g.bs));
    return SG_OK;
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
    // groups of single in-plane patches: (precision, Px, Py, central slopes, fields) -> members
    std::map<std::tuple<int, int, int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
        const sg_plan *p = plans[i];
        if (!groupable(p)) continue;
        const bool caller = p->geom.slope_mode == SG_SLOPES_CALLER;
        const bool central = p->geom.slope_mode == SG_SLOPES_CENTRAL && p->pp[0].phase;
        groups[std::make_tuple((int)p->prec, p->pp[0].d.px, p->pp[0].d.py, central ? 1 : 0,
                               caller ? 3 : (p->geom.slope_mode == SG_SLOPES_NONE ? 1 : 3))]
            .push_back(i);
    }
    std::vector<char> grouped(n, 0);
    std::vector<group_passes<float>> g32;
    std::vector<group_passes<double>> g64;
    auto dxp = [&](int i) { return deltax ? deltax[i] : nullptr; };
    auto dyp = [&](int i) { return deltay ? deltay[i] : nullptr; };
    for (auto &g : groups) {
        const std::vector<int> &mem = g.second;
        if (mem.size() < 2 || st != SG_OK) continue;
        const int i0 = mem[0];
        if (plans[i0]->prec == SG_FP64) {
            std::vector<sgk::uniform_passes<double>> us;
            for (int i : mem)
                us.push_back(sgk::uniform_setup<double>(plans[i], &b->ws[i], 0, sigma[i], dxp(i), dyp(i), fx[i], fy[i],
                                                        nullptr));
            g64.emplace_back();
            st = group_upload<double>(b, us, b->ws[i0].err, g64.back());
        } else {
            std::vector<sgk::uniform_passes<float>> us;
            for (int i : mem)
                us.push_back(sgk::uniform_setup<float>(plans[i], &b->ws[i], 0, sigma[i], dxp(i), dyp(i), fx[i], fy[i],
                                                       nullptr));
            g32.emplace_back();
            st = group_upload<float>(b, us, b->ws[i0].err, g32.back());
        }
        for (int i : mem) grouped[i] = 1;
    }
    bool capturing = false;
    if (st == SG_OK) {
        e = cudaStreamBeginCapture(streams[n], cudaStreamCaptureModeRelaxed);
        capturing = e == cudaSuccess;
        if (e == cudaSuccess) e = cudaEventRecord(events[n], streams[n]);
        if (e != cudaSuccess) st = SG_ECUDA;
    }
    int branch = 0;  // streams[0 .. n) serve groups and single members alike
    auto fork = [&](cudaStream_t bs) { return cudaStreamWaitEvent(bs, events[n], 0) == cudaSuccess ? SG_OK : SG_ECUDA; };
    auto join = [&](cudaStream_t bs) {
        return cudaEventRecord(events[branch], bs) == cudaSuccess &&
                       cudaStreamWaitEvent(streams[n], events[branch], 0) == cudaSuccess
                   ? SG_OK
                   : SG_ECUDA;
    };
    for (size_t k = 0; k < g32.size() && st == SG_OK; ++k, ++branch) {
        st = fork(streams[branch]);
        if (st == SG_OK) st = group_enqueue<float>(g32[k], streams[branch]);
        if (st == SG_OK) st = join(streams[branch]);
        b->launches += g32[k].u.central ? 4 : 3;
    }
    for (size_t k = 0; k < g64.size() && st == SG_OK; ++k, ++branch) {
        st = fork(streams[branch]);
        if (st == SG_OK) st = group_enqueue<double>(g64[k], streams[branch]);
        if (st == SG_OK) st = join(streams[branch]);
        b->launches += g64[k].u.central ? 4 : 3;
    }
    for (int i = 0; i < n && st == SG_OK; ++i) {
        if (grouped[i]) continue;
        cudaStream_t bs = streams[branch];
        st = fork(bs);
        if (st == SG_OK)
            st = sg_force_ws(plans[i], &b->ws[i], sigma[i], dxp(i), dyp(i), fx[i], fy[i], bs);
        if (st == SG_OK) st = join(bs);
        b->launches += plans[i]->launches;
        ++branch;
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
