// Uniform-patch force as a zero-padded 2-D FFT convolution: the solve of one
// patch (row pass, column pass, inverse row pass; the kernels and the
// algorithm are described in fftconv.cuh), with the launch shapes of the tuning
// table (tune.cu), and the mid-plane potential through the same passes.
#include "fftconv.cuh"

namespace {

template <typename T>
sg_status uniform_solve_t(sg_plan *plan, const sg_workspace *ws, int p, const void *sigma, const void *dx,
                          const void *dy, void *fx, void *fy, void *fz, cudaStream_t st, const T *pot_spec = nullptr,
                          void *wf_pot = nullptr)
{
    const sgk::uniform_passes<T> u = sgk::uniform_setup<T>(plan, ws, p, sigma, dx, dy, fx, fy, fz, pot_spec, wf_pot);
    // the passes' scratch must hold what they write (checked before any launch)
    const int64_t q = (int64_t)u.qx * plan->pp[p].d.ny * (int64_t)sizeof(cplx_t<T>);
    const int64_t need_f = u.nf_rows * q + (u.central ? (2LL * u.py + 1) * (int64_t)sizeof(cplx_t<T>) : 0);
    const int64_t have_f = pot_spec && wf_pot != ws->work_fwd ? plan->pot_fwd_bytes : plan->ws_fwd_bytes;
    if (need_f > have_f || u.nout * q > plan->ws_inv_bytes) {
        sg_set_last_error_message("internal: a transform pass needs more scratch than the plan sized");
        return SG_EINVAL;
    }
    sg_timing_begin(ws, SG_STAGE_ROW_FWD, st);
    // central slopes: the one-CTA edge-column transform first, the row pass
    // beside it as a dependent launch that waits for it at its end (k_edge_cols)
    if (u.central) SG_TRY(sgk::edge_cols<T>(u.py, u.ed, u.twy, st));
    SG_TRY(sgk::rows_fwd<T>(u.px, u.shx[0], u.rf, u.nf_rows, u.twx, st, nullptr, {0, 0}, u.central));
    sg_timing_end(ws, SG_STAGE_ROW_FWD, st);
    sg_timing_begin(ws, SG_STAGE_COL_CONV, st);
    if (u.central) SG_TRY(sgk::cols_central<T>(u.py, u.shy[3], u.col, u.qx, u.twy, ws->err, st));
    else SG_TRY(sgk::cols<T>(u.py, u.shy[2], u.nout, u.col, u.qx, u.nf_cols, u.twy, ws->err, st));
    sg_timing_end(ws, SG_STAGE_COL_CONV, st);
    sg_timing_begin(ws, SG_STAGE_ROW_INV, st);
    SG_TRY(sgk::rows_inv<T>(u.px, u.shx[1], u.ri, u.nout, u.twx, st));
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

sg_status sg_uniform_potential(sg_plan *plan, const sg_workspace *ws, int patch, void *wf, const void *sigma,
                               const void *dx, const void *dy, void *phi, cudaStream_t st)
{
    const sg_patch_plan &pp = plan->pp[patch];
    if (plan->prec == SG_FP64)
        return uniform_solve_t<double>(plan, ws, patch, sigma, dx, dy, phi, nullptr, nullptr, st,
                                       (const double *)pp.pspectra, wf);
    return uniform_solve_t<float>(plan, ws, patch, sigma, dx, dy, phi, nullptr, nullptr, st,
                                  (const float *)pp.pspectra, wf);
}
