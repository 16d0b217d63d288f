// Batches of independent solves replayed as one CUDA graph.
//
// sg_batch_create binds n solves (plan + caller buffers each) and captures them
// once into a CUDA graph, so that sg_batch_launch replays the whole batch with
// a single graph launch. Members that are single in-plane patches run in one of
// two layouts:
//  * persistent: the members with padded lengths up to 2048 run together in
//    ONE persistent kernel per precision (batch_run.cuh): every pass of every
//    such member is a work item of that launch, whatever their lengths and
//    slope handling, ordered per member by completion counters, so uneven small
//    solves fill the GPU together and the batch pays one kernel launch;
//  * grouped: members of the same precision, padded lengths and slope handling
//    form a group, and each pass of a group is one launch of that pass's own
//    kernel (with its tuned launch shape) over all the group's members; the
//    groups run as concurrent graph branches.
// SG_BATCH_AUTO captures both and keeps the one that replays faster. Other
// members (hierarchies, off-plane plans, 4096-point transforms, a group of
// one) keep a graph branch of their own. Results are the members' sg_force
// results bit for bit in either layout.
#include "common.cuh"
#include "batch_run.cuh"
#include "group.cuh"

#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

// A captured layout: its graph, the device argument arrays it reads, the
// kernels one replay launches.
struct batch_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> dev_args;
    int launches = 0;
};

struct sg_batch {
    int n = 0;
    std::vector<sg_workspace> ws;
    batch_graph g;
    int mode = 0;  // SG_BATCH_PERSISTENT or SG_BATCH_GROUPED
    double ms[2] = {0.0, 0.0};  // replay times measured by SG_BATCH_AUTO (persistent, grouped)
    int device = 0;
};

namespace {

void graph_free(batch_graph &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    for (void *a : g.dev_args) cudaFree(a);
    g = batch_graph();
}

void batch_free(sg_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    graph_free(b->g);
    for (sg_workspace &w : b->ws) sg_workspace_free(&w, 0, false);
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
sg_status persistent_upload(sg_batch *b, batch_graph &g, const std::vector<int> &mem, sg_plan *const *plans,
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
        // items of up to BATCH_TILES consecutive groups
        auto add = [](std::vector<batch_item> &v, int kind, int k, int ngroups, int f) {
            int n = 0;
            for (int bx = 0; bx < ngroups; bx += BATCH_TILES, ++n)
                v.push_back({(short)kind, (short)std::min(BATCH_TILES, ngroups - bx), k, bx, f});
            return n;
        };
        bm.need_fwd = 0;
        for (int f = 0; f < u.nf_rows; ++f) bm.need_fwd += add(fwd, BI_ROWF, k, groups, f);
        if (u.central) {
            fwd.push_back({(short)BI_EDGE, 1, k, 0, 0});
            ++bm.need_fwd;
        }
        const int cgroups = (u.qx + batch_cb(u.py) - 1) / batch_cb(u.py);
        bm.need_col = add(col, BI_COL, k, cgroups, 0);
        for (int o = 0; o < 2; ++o) add(inv, BI_ROWI, k, groups, o);
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
    g.dev_args.push_back(d);
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

// Upload the argument arrays of a group (owned by the layout); before capture.
template <typename T>
sg_status group_upload(batch_graph &bg, const std::vector<sgk::uniform_passes<T>> &us, int *err,
                       sgk::group_passes<T> &g)
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
        maxny = std::max(maxny, us[i].rf.src.ny);
    }
    const size_t s0 = m * sizeof(rf[0]), s1 = m * sizeof(ed[0]), s2 = m * sizeof(col[0]), s3 = m * sizeof(ri[0]);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *d = nullptr;
    SG_CUDA_TRY(cudaMalloc(&d, up(s0) + up(s1) + up(s2) + up(s3)));
    bg.dev_args.push_back(d);
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

// The inputs of one batch creation.
struct batch_inputs {
    int n;
    sg_plan *const *plans;
    const void *const *sigma, *const *deltax, *const *deltay;
    void *const *fx, *const *fy;
    const void *dx(int i) const { return deltax && plans[i]->geom.slope_mode == SG_SLOPES_CALLER ? deltax[i] : nullptr; }
    const void *dy(int i) const { return deltay && plans[i]->geom.slope_mode == SG_SLOPES_CALLER ? deltay[i] : nullptr; }
};

}  // namespace

namespace {

// Capture one layout of the batch into bg (persistent: true for the persistent
// kernel, false for grouped launches). Members outside it get a branch each.
sg_status capture_layout(sg_batch *b, const batch_inputs &in, bool persistent, int nsm, batch_graph &bg)
{
    const int n = in.n;
    // members of the layout and the rest
    std::vector<int> mem32, mem64, rest;
    std::map<std::tuple<int, int, int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
        const sg_plan *p = in.plans[i];
        if (persistent) {
            if (!persistent_member(p)) rest.push_back(i);
            else if (p->prec == SG_FP64) mem64.push_back(i);
            else mem32.push_back(i);
        } else if (sgk::groupable(p)) {
            groups[sgk::group_key(p)].push_back(i);
        } else {
            rest.push_back(i);
        }
    }
    sg_status st = SG_OK;
    persistent_run<float> r32;
    persistent_run<double> r64;
    std::vector<sgk::group_passes<float>> g32;
    std::vector<sgk::group_passes<double>> g64;
    if (persistent) {
        if (!mem32.empty())
            st = persistent_upload<float>(b, bg, mem32, in.plans, in.sigma, in.deltax, in.deltay, in.fx, in.fy, r32);
        if (st == SG_OK && !mem64.empty())
            st = persistent_upload<double>(b, bg, mem64, in.plans, in.sigma, in.deltax, in.deltay, in.fx, in.fy, r64);
    } else {
        for (auto &gr : groups) {
            const std::vector<int> &mem = gr.second;
            if (st != SG_OK) break;
            if (mem.size() < 2) {  // a group of one is an ordinary member
                rest.push_back(mem[0]);
                continue;
            }
            const int i0 = mem[0];
            if (in.plans[i0]->prec == SG_FP64) {
                std::vector<sgk::uniform_passes<double>> us;
                for (int i : mem)
                    us.push_back(sgk::uniform_setup<double>(in.plans[i], &b->ws[i], 0, in.sigma[i], in.dx(i), in.dy(i),
                                                            in.fx[i], in.fy[i], nullptr));
                g64.emplace_back();
                st = group_upload<double>(bg, us, b->ws[i0].err, g64.back());
            } else {
                std::vector<sgk::uniform_passes<float>> us;
                for (int i : mem)
                    us.push_back(sgk::uniform_setup<float>(in.plans[i], &b->ws[i], 0, in.sigma[i], in.dx(i), in.dy(i),
                                                           in.fx[i], in.fy[i], nullptr));
                g32.emplace_back();
                st = group_upload<float>(bg, us, b->ws[i0].err, g32.back());
            }
        }
        std::sort(rest.begin(), rest.end());
    }
    if (st != SG_OK) return st;
    // capture: root stream -> one branch per persistent launch, group and other member -> join
    const int nb = (int)(rest.size() + g32.size() + g64.size()) + 2;
    std::vector<cudaStream_t> streams(nb + 1, nullptr);
    std::vector<cudaEvent_t> events(nb + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i <= nb && e == cudaSuccess; ++i) {
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
    // each branch: fork, enqueue, join
    auto run_branch = [&](auto enqueue, int kernels) {
        if (st != SG_OK) return;
        cudaStream_t bs = streams[branch];
        st = fork(bs);
        if (st == SG_OK) st = enqueue(bs);
        if (st == SG_OK) st = join(bs);
        bg.launches += kernels;
        ++branch;
    };
    if (!mem32.empty())
        run_branch([&](cudaStream_t bs) {
            return sgk::batch_run_launch<float>(r32.items, r32.nitems, r32.members, r32.nmem, r32.ctl, r32.err,
                                                r32.tries, r32.smem, nsm, bs);
        }, 1);
    if (!mem64.empty())
        run_branch([&](cudaStream_t bs) {
            return sgk::batch_run_launch<double>(r64.items, r64.nitems, r64.members, r64.nmem, r64.ctl, r64.err,
                                                 r64.tries, r64.smem, nsm, bs);
        }, 1);
    for (const sgk::group_passes<float> &g : g32)
        run_branch([&](cudaStream_t bs) { return sgk::group_enqueue<float>(g, bs); }, g.u.central ? 4 : 3);
    for (const sgk::group_passes<double> &g : g64)
        run_branch([&](cudaStream_t bs) { return sgk::group_enqueue<double>(g, bs); }, g.u.central ? 4 : 3);
    for (int i : rest)
        run_branch([&](cudaStream_t bs) {
            return sg_force_ws(in.plans[i], &b->ws[i], in.sigma[i], in.dx(i), in.dy(i), in.fx[i], in.fy[i], bs);
        }, in.plans[i]->launches);
    if (capturing) {
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(streams[nb], &g);
        if (st == SG_OK && e == cudaSuccess) {
            bg.graph = g;
            e = cudaGraphInstantiate(&bg.exec, g, 0);
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
    return st;
}

// Median replay time of a layout (one warm-up replay, then `reps`).
sg_status time_layout(const batch_graph &bg, int reps, double *ms)
{
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sg_status st = SG_OK;
    std::vector<float> t;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        st = SG_ECUDA;
    for (int r = 0; r <= reps && st == SG_OK; ++r) {
        float x = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(bg.exec, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&x, e0, e1) != cudaSuccess)
            st = SG_ECUDA;
        if (r > 0) t.push_back(x);
    }
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != SG_OK) {
        sg_set_last_cuda_error(cudaGetLastError(), "sg_batch_create (timing a layout)");
        return st;
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_batch_create_mode(int n, sg_plan *const *plans, const void *const *sigma, const void *const *deltax,
                               const void *const *deltay, void *const *fx, void *const *fy, int mode, sg_batch **out)
{
    if (n < 1 || !plans || !sigma || !fx || !fy || !out) return SG_EINVAL;
    if (mode != SG_BATCH_AUTO && mode != SG_BATCH_PERSISTENT && mode != SG_BATCH_GROUPED) return SG_EINVAL;
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
    const batch_inputs in{n, plans, sigma, deltax, deltay, fx, fy};
    sg_status st = SG_OK;
    if (mode != SG_BATCH_AUTO) {
        st = capture_layout(b, in, mode == SG_BATCH_PERSISTENT, nsm, b->g);
        b->mode = mode;
    } else {
        // both layouts, each replayed a few times on the bound buffers; the faster stays
        batch_graph gp, gg;
        st = capture_layout(b, in, true, nsm, gp);
        if (st == SG_OK) st = capture_layout(b, in, false, nsm, gg);
        if (st == SG_OK) st = time_layout(gp, 3, &b->ms[0]);
        if (st == SG_OK) st = time_layout(gg, 3, &b->ms[1]);
        if (st == SG_OK) {
            const bool p = b->ms[0] <= b->ms[1];
            b->g = p ? gp : gg;
            graph_free(p ? gg : gp);
            b->mode = p ? SG_BATCH_PERSISTENT : SG_BATCH_GROUPED;
            // the timing replays' error words are not the caller's
            for (sg_workspace &w : b->ws)
                if (w.err && st == SG_OK && cudaMemset(w.err, 0, sizeof(int)) != cudaSuccess) st = SG_ECUDA;
        } else {
            cudaDeviceSynchronize();
            graph_free(gp);
            graph_free(gg);
        }
    }
    if (st != SG_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return SG_OK;
}

sg_status sg_batch_create(int n, sg_plan *const *plans, const void *const *sigma, const void *const *deltax,
                          const void *const *deltay, void *const *fx, void *const *fy, sg_batch **out)
{
    return sg_batch_create_mode(n, plans, sigma, deltax, deltay, fx, fy, SG_BATCH_AUTO, out);
}

sg_status sg_batch_launch(sg_batch *b, void *stream)
{
    if (!b) return SG_EINVAL;
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->device) return SG_EINVAL;
    SG_CUDA_TRY(cudaGraphLaunch(b->g.exec, (cudaStream_t)stream));
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
    *out = b->g.launches;
    return SG_OK;
}

sg_status sg_batch_layout(const sg_batch *b, int *mode, double *ms_persistent, double *ms_grouped)
{
    if (!b || !mode) return SG_EINVAL;
    *mode = b->mode;
    if (ms_persistent) *ms_persistent = b->ms[0];
    if (ms_grouped) *ms_grouped = b->ms[1];
    return SG_OK;
}

}  // extern "C"
