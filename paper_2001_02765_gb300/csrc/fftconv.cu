// Uniform-patch force as a zero-padded 2-D FFT convolution: the solve of one
// patch (row pass, column pass, inverse row pass; the kernels and the
// algorithm are described in fftconv.cuh), with the launch shapes of the tuning
// table (tune.cu), and the mid-plane potential through the same passes.
#include "fftconv.cuh"

namespace {

// pot_spec != NULL: the potential (one output, three spectrum planes) with the
// forward scratch wf_pot, slopes formed in the row pass.
template <typename T>
sg_status uniform_solve_t(sg_plan *plan, const sg_workspace *ws, int p, const void *sigma, const void *dx,
                          const void *dy, void *fx, void *fy, void *fz, cudaStream_t st, const T *pot_spec = nullptr,
                          void *wf_pot = nullptr)
{
    using C = cplx_t<T>;
    const sg_patch_plan &pp = plan->pp[p];
    const sg_patch_dev &d = pp.d;
    const int64_t off = d.cell_off;
    sgk::field_src<T> src;
    src.sigma = (const T *)sigma + off;
    src.dx = dx ? (const T *)dx + off : nullptr;
    src.dy = dy ? (const T *)dy + off : nullptr;
    src.nx = d.nx;
    src.ny = d.ny;
    src.inv2h = (T)(0.5 / d.h);
    src.mode = plan->geom.slope_mode;
    if (plan->composite) {
        // AMR or masks: the composite source fields (three planes, zero where no cell exists)
        const T *S = (const T *)ws->sfield;
        src.sigma = S + off;
        src.dx = S + plan->ncells + off;
        src.dy = S + 2 * plan->ncells + off;
        src.mode = SG_SLOPES_CALLER;
    }
    const int nf = src.mode == SG_SLOPES_NONE ? 1 : 3;
    const int qx = d.px / 2 + 1;
    C *wf = pot_spec ? (C *)wf_pot : (C *)ws->work_fwd;
    C *wi = (C *)ws->work_inv;
    const int64_t *twoff = sizeof(T) == 8 ? plan->tw64_off : plan->tw32_off;
    const C *twx = (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(d.px)]);
    const C *twy = (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(d.py)]);
    T *ox = (T *)fx + off, *oy = (T *)fy + off;
    T *oz = fz ? (T *)fz + off : nullptr;  // off-plane plans only
    const bool central = src.mode == SG_SLOPES_CENTRAL && pp.phase && !pot_spec;
    int shx[SG_TUNE_KNOBS], shy[SG_TUNE_KNOBS];  // launch shapes of the x and y lengths (tuning table)
    sg_tune_shape(plan->prec, d.px, shx);
    sg_tune_shape(plan->prec, d.py, shy);
    sg_timing_begin(ws, SG_STAGE_ROW_FWD, st);
    if (central) {
        // the edge-column transform is independent of the row pass: run it beside it
        C *edge = wf + (int64_t)qx * d.ny;  // after sigma's row transforms
        cudaStream_t es = st;
        if (ws->aux) {
            SG_CUDA_TRY(cudaEventRecord(ws->ev_fork, st));
            SG_CUDA_TRY(cudaStreamWaitEvent(ws->aux, ws->ev_fork, 0));
            es = ws->aux;
        }
        SG_TRY(sgk::edge_cols<T>(d.py, src.sigma, d.nx, d.ny, edge, twy, es));
        if (ws->aux) SG_CUDA_TRY(cudaEventRecord(ws->ev_join, ws->aux));
    }
    SG_TRY(sgk::rows_fwd<T>(d.px, shx[0], src, wf, central ? 1 : nf, twx, st));
    if (central && ws->aux) SG_CUDA_TRY(cudaStreamWaitEvent(st, ws->ev_join, 0));
    sg_timing_end(ws, SG_STAGE_ROW_FWD, st);
    sg_timing_begin(ws, SG_STAGE_COL_CONV, st);
    if (central) {
        const C *edge = wf + (int64_t)qx * d.ny;
        SG_TRY(sgk::cols_central<T>(d.py, shy[3], wf, wi, (const T *)pp.spectra, edge, (const T *)pp.phase, d.ny, qx,
                                    twy, ws->err, st));
    } else {
        const int nout = pot_spec ? 1 : (oz ? 3 : 2);
        SG_TRY(sgk::cols<T>(d.py, shy[2], nout, wf, wi, pot_spec ? pot_spec : (const T *)pp.spectra, d.ny, qx, nf, twy,
                            ws->err, st));
    }
    sg_timing_end(ws, SG_STAGE_COL_CONV, st);
    sg_timing_begin(ws, SG_STAGE_ROW_INV, st);
    SG_TRY(sgk::rows_inv<T>(d.px, shx[1], wi, ox, pot_spec ? nullptr : oy, oz, d.nx, d.ny, twx, st));
    sg_timing_end(ws, SG_STAGE_ROW_INV, st);
    return SG_OK;
}

}  // namespace

sg_status sg_uniform_solve(sg_plan *plan, const sg_workspace *ws, int patch, const void *sigma, const void *dx,
                           const void *dy, void *fx, void *fy, void *fz, cudaStream_t st)
{
    if (plan->prec == SG_FP64) return uniform_solve_t<double>(plan, ws, patch, sigma, dx, dy, fx, fy, fz, st);
    return uniform_solve_t<float>(plan, ws, patch, sigma, dx, dy, fx, fy, fz, st);
}

sg_status sg_uniform_potential(sg_plan *plan, const sg_workspace *ws, void *wf, const void *sigma, const void *dx,
                               const void *dy, void *phi, cudaStream_t st)
{
    const sg_patch_plan &pp = plan->pp[0];
    if (plan->prec == SG_FP64)
        return uniform_solve_t<double>(plan, ws, 0, sigma, dx, dy, phi, nullptr, nullptr, st,
                                       (const double *)pp.pspectra, wf);
    return uniform_solve_t<float>(plan, ws, 0, sigma, dx, dy, phi, nullptr, nullptr, st, (const float *)pp.pspectra,
                                  wf);
}
