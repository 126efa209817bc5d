// Pass kernels instantiated for double (see hg_kernels.cuh).
#include "hg_kernels.cuh"

namespace hgk {
cudaError_t launch_row_fwd_f64(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                const RowFwdArgs& a, cudaStream_t s) {
    return launch_row_fwd_t<double>(g, pl, tw, c, a, s);
}
cudaError_t launch_row_inv_f64(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                const RowInvArgs& a, cudaStream_t s) {
    return launch_row_inv_t<double>(g, pl, tw, c, a, s);
}
cudaError_t launch_strided_f64(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& c,
                                const StrArgs& a, cudaStream_t s) {
    return launch_strided_t<double>(g, pl, tw, c, a, s);
}
cudaError_t launch_row_fwd_batch_f64(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                    const RowFwdArgs* items, int P, int L, cudaStream_t s) {
    return launch_row_fwd_batch_t<double>(g, pl, tw, c, items, P, L, s);
}
cudaError_t launch_row_inv_batch_f64(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& c,
                                    const RowInvArgs* items, int P, int L, cudaStream_t s) {
    return launch_row_inv_batch_t<double>(g, pl, tw, c, items, P, L, s);
}
cudaError_t launch_strided_batch_f64(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& c,
                                    const StrArgs* items, int P, int L, int n, long long inner,
                                    long long outer, cudaStream_t s) {
    return launch_strided_batch_t<double>(g, pl, tw, c, items, P, L, n, inner, outer, s);
}
cudaError_t configure_f64(int max_smem, const double* ctw) { return configure_t<double>(max_smem, ctw); }
}  // namespace hgk
