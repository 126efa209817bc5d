// Pass kernels instantiated for float (see hg_kernels.cuh).
#include "hg_kernels.cuh"

namespace hgk {
// the host's tile limits (hg_internal.h) are the kernels' own
static_assert(MAX_REAL_ROWS == MAX_REAL_ROWS_HOST, "host row tiles and device offset table disagree");
cudaError_t launch_row_fwd_f32(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                const RowFwdArgs& a, cudaStream_t s) {
    return launch_row_fwd_t<float>(g, pl, tw, c, a, s);
}
cudaError_t launch_row_inv_f32(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                const RowInvArgs& a, cudaStream_t s) {
    return launch_row_inv_t<float>(g, pl, tw, c, a, s);
}
cudaError_t launch_strided_f32(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& c,
                                const StrArgs& a, cudaStream_t s) {
    return launch_strided_t<float>(g, pl, tw, c, a, s);
}
cudaError_t launch_row_fwd_batch_f32(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                    const RowFwdArgs* items, int P, int L, cudaStream_t s) {
    return launch_row_fwd_batch_t<float>(g, pl, tw, c, items, P, L, s);
}
cudaError_t launch_row_inv_batch_f32(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                    const RowInvArgs* items, int P, int L, cudaStream_t s) {
    return launch_row_inv_batch_t<float>(g, pl, tw, c, items, P, L, s);
}
cudaError_t launch_strided_batch_f32(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& c,
                                    const StrArgs* items, int P, int L, int n, long long inner,
                                    long long outer, cudaStream_t s) {
    return launch_strided_batch_t<float>(g, pl, tw, c, items, P, L, n, inner, outer, s);
}
cudaError_t configure_f32(int max_smem, const double* ctw) { return configure_t<float>(max_smem, ctw); }
}  // namespace hgk
