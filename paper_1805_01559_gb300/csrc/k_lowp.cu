// Dispatch of the stored-kernel solver by storage format.
#include "ot_internal.h"

namespace ota {

ot_status lowp_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, double absorb_log2, SolveSummary* sum_host);
ot_status lowp_solve_bf16(ot_assoc_ctx* ctx, const SolveArgs& a, double absorb_log2, SolveSummary* sum_host);
ot_status lowp_solve_f16(ot_assoc_ctx* ctx, const SolveArgs& a, double absorb_log2, SolveSummary* sum_host);

ot_status launch_solve_lowp(ot_assoc_ctx* ctx, const SolveArgs& a, int format, double absorb_log2,
                            SolveSummary* sum_host) {
    switch (format) {
        case OT_KERNEL_F32: return lowp_solve_f32(ctx, a, absorb_log2, sum_host);
        case OT_KERNEL_BF16: return lowp_solve_bf16(ctx, a, absorb_log2, sum_host);
        case OT_KERNEL_F16: return lowp_solve_f16(ctx, a, absorb_log2, sum_host);
        default: return set_error(ctx, OT_EINVAL, "unknown kernel format %d", format);
    }
}

}  // namespace ota
