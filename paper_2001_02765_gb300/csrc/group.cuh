// Grouped launches of single in-plane patches of equal padded lengths,
// precision and slope handling: each pass of the uniform-patch convolution is
// one launch over all the group's members (blockIdx.z = member; the members'
// pass arguments in device arrays), with the same arithmetic per member as a
// solve of its own, so results are bit-identical. Used by batches (batch.cu)
// and by the request server (server.cu).
#pragma once
#include "fftconv.cuh"

#include <tuple>

namespace sgk {

// A member of a group: one in-plane patch (any length), no composite source.
inline bool groupable(const sg_plan *p)
{
    return p->npatches == 1 && !p->composite && !p->lv && p->geom.z == 0.0;
}

// A group's passes: the members' arguments in one device array per pass.
template <typename T>
struct group_passes {
    uniform_passes<T> u;  // lengths, shapes and twiddles are common to the group
    const row_fwd_args<T> *rf = nullptr;
    const edge_args<T> *ed = nullptr;
    const col_args<T> *col = nullptr;
    const row_inv_args<T> *ri = nullptr;
    batch_shape bs = {0, 0};
    int *err = nullptr;
};

// The key members of one group share: precision, padded lengths, central
// slopes formed in the spectrum, fields of the row pass.
inline std::tuple<int, int, int, int, int> group_key(const sg_plan *p)
{
    const bool central = p->geom.slope_mode == SG_SLOPES_CENTRAL && p->pp[0].phase;
    return std::make_tuple((int)p->prec, p->pp[0].d.px, p->pp[0].d.py, central ? 1 : 0,
                           p->geom.slope_mode == SG_SLOPES_NONE ? 1 : 3);
}

// One launch per pass for all the group's members.
template <typename T>
inline sg_status group_enqueue(const group_passes<T> &g, cudaStream_t st)
{
    const uniform_passes<T> &u = g.u;
    if (u.central) SG_TRY(edge_cols<T>(u.py, u.ed, u.twy, st, g.ed, g.bs));
    SG_TRY(rows_fwd<T>(u.px, u.shx[0], u.rf, u.nf_rows, u.twx, st, g.rf, g.bs, u.central));
    if (u.central) SG_TRY(cols_central<T>(u.py, u.shy[3], u.col, u.qx, u.twy, g.err, st, g.col, g.bs));
    else SG_TRY(cols<T>(u.py, u.shy[2], u.nout, u.col, u.qx, u.nf_cols, u.twy, g.err, st, g.col, g.bs));
    SG_TRY(rows_inv<T>(u.px, u.shx[1], u.ri, u.nout, u.twx, st, g.ri, g.bs));
    return SG_OK;
}

}  // namespace sgk
