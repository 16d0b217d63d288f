// Launch-shape tuning of the uniform-patch passes and of a plan's cross-patch
// direct sum (not in the paper).
//
// For every padded length and precision a process-wide table holds the launch
// shape of each pass: row sequences per CTA of the forward and inverse row
// passes and columns per CTA of the column passes, each one of three compiled
// candidates (half, the measured default, twice the default, where shared
// memory and CTA size allow; fftconv.cuh). The shape changes only how
// sequences are grouped into CTAs, never the arithmetic of a sequence, so
// results are bit-identical under every shape. sg_autotune times the
// candidates on a square patch of each length and keeps the fastest.
#include "common.cuh"
#include "fftconv.cuh"

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace {

constexpr int NPAD = 7;  // 64 .. 4096
std::atomic<int> g_shape[2][NPAD][SG_TUNE_KNOBS];  // 0 = default
std::mutex g_tune_mutex;                            // one sg_autotune at a time

int pad_index(int pad)
{
    for (int i = 0; i < NPAD; ++i)
        if (pad == (SG_MIN_PAD << i)) return i;
    return -1;
}

int knob_default(int knob, int pad)
{
    if (knob == 0) return sgk::row_nb_default(pad);
    if (knob == 1) return sgk::row_nb_inv_default(pad);
    return sgk::col_cb_default(pad);
}

// shared memory of a column pass with CB columns, NPL spectrum planes (runtime form of col_smem_bytes)
int64_t col_smem(int pad, int cb, int npl, bool fp64)
{
    const int64_t cs = fp64 ? 16 : 8, rs = fp64 ? 8 : 4;
    const int64_t n = (int64_t)cb * pad;
    const int64_t padded = fp64 ? (n - 1) + ((n - 1) >> 3) + 1 : (n - 1) + ((n - 1) >> 4) + 1;
    const int64_t nbuf = fp64 && pad >= 4096 ? 1 : 2;  // col_nbuf
    return nbuf * ((padded * cs + 15) & ~15LL) + (int64_t)cb * npl * (((pad / 2 + 1) + 3) & ~3) * rs;
}

bool knob_feasible(int knob, int pad, int v, bool fp64)
{
    const int d = knob_default(knob, pad);
    if (v != d && v != d / 2 && v != 2 * d) return false;
    if (v < 1) return false;
    if (knob <= 1) {
        const int64_t n = (int64_t)v * pad;
        const int64_t padded = fp64 ? (n - 1) + ((n - 1) >> 3) + 1 : (n - 1) + ((n - 1) >> 4) + 1;
        return v <= 64 && padded * (fp64 ? 16 : 8) <= 200 * 1024;
    }
    const int threads = v * pad / 8;
    if (threads < 32 || threads > 512) return false;
    // the generic column pass is compiled with 3, 6 and 9 planes, the central one with 6
    return col_smem(pad, v, knob == 2 ? 9 : 6, fp64) <= 200 * 1024 && col_smem(pad, v, 3, fp64) <= 200 * 1024;
}

std::vector<int> knob_candidates(int knob, int pad, bool fp64)
{
    std::vector<int> c;
    const int d = knob_default(knob, pad);
    for (int v : {d / 2, d, 2 * d})
        if (knob_feasible(knob, pad, v, fp64)) c.push_back(v);
    return c;
}

}  // namespace

void sg_tune_shape(sg_precision prec, int pad, int *shape)
{
    const int i = pad_index(pad);
    for (int k = 0; k < SG_TUNE_KNOBS; ++k) {
        const int v = i >= 0 ? g_shape[prec == SG_FP64 ? 1 : 0][i][k].load(std::memory_order_relaxed) : 0;
        shape[k] = v ? v : knob_default(k, pad);
    }
}

extern "C" {

sg_status sg_tune_get(int precision, int pad, int *shape)
{
    if ((precision != SG_FP64 && precision != SG_FP32) || pad_index(pad) < 0 || !shape) {
        sg_set_last_error_message("sg_tune_get: precision, padded length (64..4096, power of two) or shape invalid");
        return SG_EINVAL;
    }
    sg_tune_shape((sg_precision)precision, pad, shape);
    return SG_OK;
}

sg_status sg_tune_set(int precision, int pad, const int *shape)
{
    const int i = pad_index(pad);
    if ((precision != SG_FP64 && precision != SG_FP32) || i < 0 || !shape) {
        sg_set_last_error_message("sg_tune_set: precision, padded length (64..4096, power of two) or shape invalid");
        return SG_EINVAL;
    }
    for (int k = 0; k < SG_TUNE_KNOBS; ++k) {
        if (shape[k] != 0 && !knob_feasible(k, pad, shape[k], precision == SG_FP64)) {
            char msg[128];
            snprintf(msg, sizeof(msg), "sg_tune_set: shape %d = %d is not a compiled candidate for length %d", k,
                     shape[k], pad);
            sg_set_last_error_message(msg);
            return SG_EINVAL;
        }
    }
    for (int k = 0; k < SG_TUNE_KNOBS; ++k)
        g_shape[precision == SG_FP64 ? 1 : 0][i][k].store(shape[k], std::memory_order_relaxed);
    return SG_OK;
}

sg_status sg_autotune(int precision, int min_pad, int max_pad, int reps, double *best_ms)
{
    if ((precision != SG_FP64 && precision != SG_FP32) || pad_index(min_pad) < 0 || pad_index(max_pad) < 0 ||
        min_pad > max_pad || reps < 1) {
        sg_set_last_error_message("sg_autotune: invalid precision, lengths or repetitions");
        return SG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const bool fp64 = precision == SG_FP64;
    const int pi = fp64 ? 1 : 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SG_CUDA_TRY(cudaEventCreate(&e0));
    SG_CUDA_TRY(cudaEventCreate(&e1));
    sg_status st = SG_OK;
    for (int pad = min_pad, slot = 0; pad <= max_pad && st == SG_OK; pad <<= 1, ++slot) {
        const int n = pad / 2;  // the largest patch that pads to this length
        // a caller-slope plan (three fields) for the row and generic column passes,
        // a central-slope plan for the central column pass
        sg_plan *plans[2] = {nullptr, nullptr};
        void *buf = nullptr;
        for (int m = 0; m < 2 && st == SG_OK; ++m) {
            sg_patch p = {0, n, n, 0.0, 0.0, 1.0 / n};
            sg_geom g;
            memset(&g, 0, sizeof(g));
            g.npatches = 1;
            g.patches = &p;
            g.G = 1.0;
            g.slope_mode = m == 0 ? SG_SLOPES_CALLER : SG_SLOPES_CENTRAL;
            st = sg_plan_create(&g, (sg_precision)precision, 0, &plans[m]);
        }
        const int64_t cells = (int64_t)n * n, es = fp64 ? 8 : 4;
        if (st == SG_OK && cudaMalloc(&buf, (size_t)(5 * cells * es)) != cudaSuccess) {
            cudaGetLastError();
            st = SG_ENOMEM;
        }
        if (st == SG_OK && cudaMemset(buf, 0, (size_t)(5 * cells * es)) != cudaSuccess) st = SG_ECUDA;  // timing only
        char *b = (char *)buf;
        auto time_plan = [&](int m, double &ms) -> sg_status {
            sg_plan *plan = plans[m];
            const void *dx = m == 0 ? b + cells * es : nullptr, *dy = m == 0 ? b + 2 * cells * es : nullptr;
            SG_TRY(sg_force(plan, b, dx, dy, b + 3 * cells * es, b + 4 * cells * es, nullptr));  // warm-up
            std::vector<float> t;
            for (int r = 0; r < reps; ++r) {
                SG_CUDA_TRY(cudaEventRecord(e0, nullptr));
                SG_TRY(sg_force(plan, b, dx, dy, b + 3 * cells * es, b + 4 * cells * es, nullptr));
                SG_CUDA_TRY(cudaEventRecord(e1, nullptr));
                SG_CUDA_TRY(cudaEventSynchronize(e1));
                float x = 0;
                SG_CUDA_TRY(cudaEventElapsedTime(&x, e0, e1));
                t.push_back(x);
            }
            std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
            ms = t[t.size() / 2];
            return SG_OK;
        };
        double best = 0.0;
        for (int k = 0; k < SG_TUNE_KNOBS && st == SG_OK; ++k) {
            const int m = k == 3 ? 1 : 0;
            int choice = g_shape[pi][pad_index(pad)][k].load();
            double best_k = 1e300;
            for (int v : knob_candidates(k, pad, fp64)) {
                g_shape[pi][pad_index(pad)][k].store(v);
                double ms = 0;
                st = time_plan(m, ms);
                if (st != SG_OK) break;
                if (ms < best_k) {
                    best_k = ms;
                    choice = v;
                }
            }
            g_shape[pi][pad_index(pad)][k].store(choice);
            if (m == 0) best = best_k;
        }
        if (best_ms && st == SG_OK) best_ms[slot] = best;
        cudaFree(buf);
        for (sg_plan *p : plans) sg_plan_destroy(p);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// The cross-patch direct sum of one plan: source-tile ranges per target block
// (the plan's value, a half and a quarter of it: the partial-sum buffers were
// sized for the plan's value) and, for FP32 plans, the CTAs of the persistent
// far-field launch (1, 2, 3, 4, 6 or 8 per SM), timed on the plan's own
// workspace with zero fields, the fastest kept.
sg_status sg_plan_autotune(sg_plan *plan, int reps, double *best_ms)
{
    if (!plan || reps < 1) {
        sg_set_last_error_message("sg_plan_autotune: null plan or repetitions below 1");
        return SG_EINVAL;
    }
    if (plan->ntiles == 0 || plan->ntargets == 0) {  // no direct sum to tune
        if (best_ms) *best_ms = 0.0;
        return SG_OK;
    }
    int dev = 0, nsm = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device) return SG_EINVAL;
    SG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t es = plan->prec == SG_FP64 ? 8 : 4, n = plan->ncells;
    char *buf = nullptr;
    SG_CUDA_TRY(cudaMalloc(&buf, (size_t)(6 * n * es)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sg_status st = cudaMemset(buf, 0, (size_t)(6 * n * es)) == cudaSuccess ? SG_OK : SG_ECUDA;
    if (st == SG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = SG_ECUDA;
    auto solve = [&]() -> sg_status {
        if (plan->geom.z != 0.0) return sg_force3(plan, buf, buf + n * es, buf + 2 * n * es, buf + 3 * n * es,
                                                  buf + 4 * n * es, buf + 5 * n * es, nullptr);
        return sg_force(plan, buf, buf + n * es, buf + 2 * n * es, buf + 3 * n * es, buf + 4 * n * es, nullptr);
    };
    auto time_it = [&](double &ms) -> sg_status {
        SG_TRY(solve());  // warm-up
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            SG_CUDA_TRY(cudaEventRecord(e0, nullptr));
            SG_TRY(solve());
            SG_CUDA_TRY(cudaEventRecord(e1, nullptr));
            SG_CUDA_TRY(cudaEventSynchronize(e1));
            float x = 0;
            SG_CUDA_TRY(cudaEventElapsedTime(&x, e0, e1));
            t.push_back(x);
        }
        std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
        ms = t[t.size() / 2];
        return SG_OK;
    };
    const bool fp32 = plan->prec == SG_FP32;
    const int built = plan->nsplit;
    int per_sm = fp32 ? std::max(1, (plan->far_grid + nsm - 1) / nsm) : 0;
    auto set_shape = [&](int ns, int psm) {
        plan->nsplit = ns;
        if (fp32) {
            const int64_t items = (int64_t)plan->nblocks * ns;
            plan->far_grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)nsm * psm));
        }
    };
    double best = 1e300;
    int best_ns = built, best_psm = per_sm;
    for (int ns : {built, built / 2, built / 4}) {
        if (st != SG_OK || ns < 1 || (ns != built && ns == best_ns)) continue;
        set_shape(ns, per_sm);
        double ms = 0;
        st = time_it(ms);
        if (st == SG_OK && ms < best) {
            best = ms;
            best_ns = ns;
        }
    }
    if (fp32)
        for (int psm : {1, 2, 3, 4, 6, 8}) {
            if (st != SG_OK || psm == per_sm) continue;
            set_shape(best_ns, psm);
            double ms = 0;
            st = time_it(ms);
            if (st == SG_OK && ms < best) {
                best = ms;
                best_psm = psm;
            }
        }
    set_shape(best_ns, best_psm);
    if (st == SG_OK && best_ms) *best_ms = best;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaDeviceSynchronize();
    cudaFree(buf);
    return st;
}

sg_status sg_plan_direct_shape(const sg_plan *plan, int *nsplit, int *far_grid)
{
    if (!plan || !nsplit || !far_grid) return SG_EINVAL;
    *nsplit = plan->nsplit;
    *far_grid = plan->far_grid;
    return SG_OK;
}

}  // extern "C"
